"""Kuhn-split cube mesh, its boundary and integer-scaled P1 finite-element assembly.

Paper: "standard linear tetrahedral finite elements are used for space
discretization" (abstract, Sec. 2.1 "finite element discretization"); the energy
gradient is a sparse matrix-vector product (Table 2).  The paper gives no mesh
for the cube workloads; the reading used here:

  * node (i, j, k), 0 <= i, j, k <= n, has id i + (n+1)(j + (n+1)k);
  * cell (i, j, k) (id i + n(j + nk)) is split into the six Kuhn tetrahedra
    {v0, v0+e_a, v0+e_a+e_b, v0+e_a+e_b+e_c} for the permutations (a, b, c) of
    the axes in lexicographic order; for odd permutations the last two vertices
    are swapped so that every tetrahedron has positive volume.  All six share the
    cell's 000-111 diagonal, so neighbouring cells conform;
  * tetrahedra are listed cell-major, then by permutation.

Everything below is exact integer arithmetic on lattice coordinates (unit = the
cell edge h).  With phi_a the hat functions and c_a the cofactor vectors of a
tetrahedron of signed volume det/6 (grad phi_a = c_a / det, in units 1/h):
  K_ij  = sum_e vol_e grad phi_i . grad phi_j      = (h/6)    * Kint_ij
  G_ij  = sum_e (vol_e/4) grad phi_i |_e  (e ∋ i,j) = (h^2/24) * Gint_ij   (3-vector)
  V_i   = sum_e vol_e / 4                          = (h^3/24) * Vint_i
with Kint_ij = sum_e c_i.c_j / det, Gint_ij = sum_e c_i, Vint_i = sum_e det.
b_i = sum_j G_ij . m_j equals int m . grad phi_i exactly for P1 m, and the
lumped projection of -grad u is  -(1/V_i) sum_j G_ji u_j.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


def node_id(i, j, k, n):
    return i + (n + 1) * (j + (n + 1) * k)


def kuhn_cube(n: int):
    """Integer node coordinates (N, 3) and tetrahedra (6 n^3, 4), positive volume."""
    n1 = n + 1
    k, j, i = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    nodes = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int64)
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v0 = node_id(ci.ravel(), cj.ravel(), ck.ravel(), n).astype(np.int64)
    step = np.array([1, n1, n1 * n1], dtype=np.int64)
    tets = np.empty((v0.size, 6, 4), dtype=np.int64)
    for p, perm in enumerate(itertools.permutations(range(3))):
        a, b, c = perm
        p0 = v0
        p1 = p0 + step[a]
        p2 = p1 + step[b]
        p3 = p2 + step[c]
        # parity of the permutation = sign of det[e_a, e_b, e_c]
        inv = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y])
        if inv % 2 == 0:
            tets[:, p] = np.stack([p0, p1, p2, p3], axis=1)
        else:
            tets[:, p] = np.stack([p0, p1, p3, p2], axis=1)
    return nodes, tets.reshape(-1, 4)


def cofactors(nodes: np.ndarray, tets: np.ndarray):
    """Cofactor vectors c_a (T, 4, 3) and det = 6 vol (T,) of each tetrahedron."""
    P = nodes[tets]                      # (T, 4, 3)
    e1, e2, e3 = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]
    c1 = np.cross(e2, e3)
    c2 = np.cross(e3, e1)
    c3 = np.cross(e1, e2)
    c0 = -(c1 + c2 + c3)
    det = np.einsum("ij,ij->i", e1, c1)
    return np.stack([c0, c1, c2, c3], axis=1), det


@dataclass
class IntOperators:
    """Integer FEM tables on the common CSR pattern (rows sorted, columns ascending)."""
    indptr: np.ndarray     # (N+1,) int64
    indices: np.ndarray    # (nnz,) int64
    K: np.ndarray          # (nnz,) int64   Kint_ij
    G: np.ndarray          # (nnz, 3) int64 Gint_ij
    Gt: np.ndarray         # (nnz, 3) int64 Gint_ji (transpose at the same position)
    V: np.ndarray          # (N,) int64     Vint_i


def assemble_int(nodes: np.ndarray, tets: np.ndarray) -> IntOperators:
    """Exact integer assembly of Kint, Gint, Vint (requires det = 1, as for Kuhn tets)."""
    N = nodes.shape[0]
    c, det = cofactors(nodes, tets)
    if not np.all(det == 1):
        raise ValueError("integer assembly needs unit-determinant tetrahedra")
    rows = np.repeat(tets, 4, axis=1).ravel()          # a-major
    cols = np.tile(tets, (1, 4)).ravel()
    kloc = np.einsum("tad,tbd->tab", c, c).ravel()     # c_a . c_b / det (det = 1)
    gloc = np.repeat(c, 4, axis=1).reshape(-1, 3)      # c_a for every b
    Km = sp.coo_matrix((kloc, (rows, cols)), shape=(N, N)).tocsr()
    Km.sum_duplicates()
    Km.sort_indices()
    pattern = sp.coo_matrix((np.ones_like(rows), (rows, cols)), shape=(N, N)).tocsr()
    pattern.sum_duplicates()
    pattern.sort_indices()
    if not (np.array_equal(Km.indptr, pattern.indptr)
            and np.array_equal(Km.indices, pattern.indices)):
        raise AssertionError("stiffness pattern differs from element-adjacency pattern")
    G = np.empty((Km.nnz, 3), dtype=np.int64)
    Gt = np.empty((Km.nnz, 3), dtype=np.int64)
    for d in range(3):
        Gd = sp.coo_matrix((gloc[:, d], (rows, cols)), shape=(N, N)).tocsr()
        Gd.sum_duplicates()
        Gd.sort_indices()
        assert np.array_equal(Gd.indices, Km.indices)
        G[:, d] = Gd.data
        GdT = Gd.T.tocsr()
        GdT.sum_duplicates()
        GdT.sort_indices()
        assert np.array_equal(GdT.indices, Km.indices)
        Gt[:, d] = GdT.data
    V = np.bincount(tets.ravel(), weights=np.repeat(det, 4), minlength=N).astype(np.int64)
    return IntOperators(Km.indptr.astype(np.int64), Km.indices.astype(np.int64),
                        Km.data.astype(np.int64), G, Gt, V)


def boundary_nodes(nodes: np.ndarray, n: int) -> np.ndarray:
    """Ids (ascending) of nodes on the cube surface."""
    on = np.any((nodes == 0) | (nodes == n), axis=1)
    return np.nonzero(on)[0].astype(np.int64)


def boundary_triangles(nodes: np.ndarray, tets: np.ndarray, n: int) -> np.ndarray:
    """Outward-oriented surface triangles (F, 3) of the tetrahedral mesh.

    A face lies on the surface iff its three vertices share one coordinate equal
    to 0 or n (the surface of a box is its six planes).  Orientation: the normal
    (b-a) x (c-a) points away from the tetrahedron's fourth vertex.  Canonical
    form: the smallest id first, cyclic order kept; rows sorted."""
    tris = []
    for opp in range(4):
        face = [v for v in range(4) if v != opp]
        F = tets[:, face]
        X = nodes[F]                                     # (T, 3, 3)
        on = np.zeros(F.shape[0], dtype=bool)
        for d in range(3):
            for val in (0, n):
                on |= np.all(X[:, :, d] == val, axis=1)
        F, X = F[on], X[on]
        Xo = nodes[tets[on, opp]]
        nrm = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
        flip = np.einsum("ij,ij->i", nrm, Xo - X[:, 0]) > 0
        F = F.copy()
        F[flip] = F[flip][:, [0, 2, 1]]
        tris.append(F)
    T = np.concatenate(tris, axis=0)
    r = np.argmin(T, axis=1)
    T = np.stack([T[np.arange(len(T)), (r + s) % 3] for s in range(3)], axis=1)
    order = np.lexsort((T[:, 2], T[:, 1], T[:, 0]))
    return T[order]


def closed_form_counts(n: int):
    """Node, boundary-node, tetrahedron, surface-triangle and nonzero counts."""
    N = (n + 1) ** 3
    nb = N - (n - 1) ** 3 if n >= 1 else N
    E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    return dict(N=N, nb=nb, T=6 * n ** 3, F=12 * n * n, nnz=N + 2 * E)


@dataclass
class CubeMesh:
    n: int
    cell: float                 # edge h in metres
    nodes: np.ndarray           # (N, 3) int lattice coordinates
    tets: np.ndarray            # (T, 4)
    ops: IntOperators
    bnd: np.ndarray             # (nb,) boundary node ids, ascending
    tris: np.ndarray            # (F, 3) outward surface triangles (node ids)

    @property
    def N(self) -> int:
        return self.nodes.shape[0]

    def xyz(self) -> np.ndarray:
        return self.nodes.astype(np.float64) * self.cell

    def stiffness(self) -> sp.csr_matrix:
        """K (metres): int grad phi_i . grad phi_j."""
        N = self.N
        return sp.csr_matrix((self.ops.K * (self.cell / 6.0), self.ops.indices, self.ops.indptr),
                             shape=(N, N))

    def coupling(self):
        """G_d (m^2), d = x, y, z:  (G_d)_ij = sum_e (vol_e/4) d_d phi_i |_e."""
        N = self.N
        s = self.cell ** 2 / 24.0
        return [sp.csr_matrix((self.ops.G[:, d] * s, self.ops.indices, self.ops.indptr),
                              shape=(N, N)) for d in range(3)]

    def volumes(self) -> np.ndarray:
        """Lumped nodal volumes V_i (m^3)."""
        return self.ops.V * (self.cell ** 3 / 24.0)


def cube_mesh(n: int, cell: float = 2e-9) -> CubeMesh:
    nodes, tets = kuhn_cube(n)
    ops = assemble_int(nodes, tets)
    return CubeMesh(n=n, cell=cell, nodes=nodes, tets=tets, ops=ops,
                    bnd=boundary_nodes(nodes, n), tris=boundary_triangles(nodes, tets, n))


# ---- general tetrahedral meshes (FP64 assembly) -----------------------------------------
#
# The same P1 operators on an arbitrary conforming tetrahedral mesh, assembled
# in FP64 from the definitions above: with the cofactors c_a of a tetrahedron
# and det = 6 x its signed volume, grad phi_a = c_a / det and vol = |det|/6, so
#   K_ab (element)        = vol grad phi_a . grad phi_b = c_a . c_b / (6 |det|)
#   (vol/4) grad phi_a    = sgn(det) c_a / 24
#   V_a (element share)   = |det| / 24.
# The surface is the set of faces that belong to one tetrahedron only.

@dataclass
class FloatOperators:
    """FP64 FEM operators (SI units) on the element-adjacency CSR pattern."""
    indptr: np.ndarray     # (N+1,) int64
    indices: np.ndarray    # (nnz,) int64
    K: np.ndarray          # (nnz,)   K_ij (m)
    G: np.ndarray          # (nnz, 3) G_ij (m^2)
    Gt: np.ndarray         # (nnz, 3) G_ji at the position of (i, j)
    V: np.ndarray          # (N,)     V_i (m^3)


def assemble_fp64(xyz: np.ndarray, tets: np.ndarray) -> FloatOperators:
    """K, G, V of the P1 space on any conforming tetrahedral mesh (FP64)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    N = xyz.shape[0]
    c, det = cofactors(xyz, tets)
    if np.any(det == 0.0):
        raise ValueError("degenerate tetrahedron")
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    kloc = (np.einsum("tad,tbd->tab", c, c) / (6.0 * np.abs(det))[:, None, None]).ravel()
    gloc = np.repeat(c * (np.sign(det) / 24.0)[:, None, None], 4, axis=1).reshape(-1, 3)
    Km = sp.coo_matrix((kloc, (rows, cols)), shape=(N, N)).tocsr()
    Km.sum_duplicates()
    Km.sort_indices()
    G = np.empty((Km.nnz, 3))
    Gt = np.empty((Km.nnz, 3))
    for d in range(3):
        Gd = sp.coo_matrix((gloc[:, d], (rows, cols)), shape=(N, N)).tocsr()
        Gd.sum_duplicates()
        Gd.sort_indices()
        assert np.array_equal(Gd.indices, Km.indices)
        G[:, d] = Gd.data
        GdT = Gd.T.tocsr()
        GdT.sum_duplicates()
        GdT.sort_indices()
        assert np.array_equal(GdT.indices, Km.indices)
        Gt[:, d] = GdT.data
    V = np.bincount(tets.ravel(), weights=np.repeat(np.abs(det) / 24.0, 4), minlength=N)
    return FloatOperators(Km.indptr.astype(np.int64), Km.indices.astype(np.int64), Km.data.copy(), G, Gt, V)


def surface_faces(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Outward-oriented surface triangles (F, 3): the faces of exactly one
    tetrahedron; normal (b-a) x (c-a) away from that tetrahedron's fourth
    vertex.  Canonical form as in boundary_triangles (smallest id first, cyclic
    order kept, rows sorted).  Raises on faces shared by more than two."""
    tets = np.asarray(tets, dtype=np.int64)
    faces, opp = [], []
    for o in range(4):
        faces.append(tets[:, [v for v in range(4) if v != o]])
        opp.append(tets[:, o])
    faces = np.concatenate(faces)
    opp = np.concatenate(opp)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    if np.any(cnt > 2):
        raise ValueError("non-manifold mesh: a face belongs to more than two tetrahedra")
    on = cnt[inv.ravel()] == 1
    F, O = faces[on].copy(), opp[on]
    X = xyz[F]
    nrm = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    flip = np.einsum("ij,ij->i", nrm, xyz[O] - X[:, 0]) > 0
    F[flip] = F[flip][:, [0, 2, 1]]
    r = np.argmin(F, axis=1)
    F = np.stack([F[np.arange(len(F)), (r + s) % 3] for s in range(3)], axis=1)
    order = np.lexsort((F[:, 2], F[:, 1], F[:, 0]))
    return F[order]


def length_unit(xyz: np.ndarray, tets: np.ndarray) -> float:
    """The mesh's length unit L = (mean |det|)^(1/3) = (6 x mean volume)^(1/3):
    the cell edge for a 6-tetrahedra cube split.  Reduced quantities use it
    the way the cube meshes use their cell edge."""
    _, det = cofactors(np.asarray(xyz, dtype=np.float64), np.asarray(tets, dtype=np.int64))
    return float(np.cbrt(np.mean(np.abs(det))))


@dataclass
class TetMesh:
    """A general mesh with the interface of CubeMesh (n = 0; cell = L)."""
    xyz_m: np.ndarray           # (N, 3) metres
    tets: np.ndarray            # (T, 4)
    ops: FloatOperators
    bnd: np.ndarray             # (nb,) surface node ids, ascending
    tris: np.ndarray            # (F, 3) outward surface triangles
    cell: float                 # length unit L (m)
    n: int = 0

    @property
    def N(self) -> int:
        return self.xyz_m.shape[0]

    @property
    def nodes(self) -> np.ndarray:
        """Coordinates in units of L (the BEM operator is scale free)."""
        return self.xyz_m / self.cell

    def xyz(self) -> np.ndarray:
        return self.xyz_m

    def stiffness(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.ops.K, self.ops.indices, self.ops.indptr), shape=(self.N, self.N))

    def coupling(self):
        return [sp.csr_matrix((self.ops.G[:, d], self.ops.indices, self.ops.indptr), shape=(self.N, self.N))
                for d in range(3)]

    def volumes(self) -> np.ndarray:
        return self.ops.V


def tet_mesh(xyz: np.ndarray, tets: np.ndarray) -> TetMesh:
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    tris = surface_faces(xyz, tets)
    return TetMesh(xyz_m=xyz, tets=tets, ops=assemble_fp64(xyz, tets), bnd=np.unique(tris),
                   tris=tris, cell=length_unit(xyz, tets))
