"""Open boundary by space transformation: a cube magnet, an air box and a shell
mapped onto the rest of space.

Oracle -- test infrastructure only: the GPU library neither imports nor links it.

Paper, Sec. 3.1: the paper's steepest-descent solver treats the open boundary of
the magnetostatic problem by a space transformation (Brunotte, Meunier and
Imhoff, 1992) rather than the accelerated boundary element method, because it
ports more easily to the GPU.  The paper gives no construction; the reading
used here (a parallelepipedic shell):

Domain.  Lattice units h; the magnet is the cube [0, n]^3 with centre
c = (n/2)(1, 1, 1).  With rho(x) = max_k |x_k - c_k| (the max-norm about c),
air fills rho <= R1 = n/2 + a outside the magnet and the shell is
R1 <= rho <= R2 = R1 + s.  One Kuhn grid of spacing h covers the whole box
[-(a+s), n+a+s]^3 (node and tetrahedron order as oracle.mesh.kuhn_cube, shifted
by a+s); its cells inside [0, n]^3 are the magnet's cells, split the same way.

Transformation.  The shell is mapped onto the exterior rho' >= R1 by
    x' - c = sig(rho) (x - c),   sig = g/rho,   g(rho) = R1 (R2 - R1)/(R2 - rho),
which fixes the inner face (g(R1) = R1) and sends the outer face rho = R2 to
infinity.  In the sector where coordinate k attains the max,
grad rho = sign(x_k - c_k) e_k and
    J = dx'/dx = sig I + sig'(rho) (x - c) grad rho^T,   det J = sig^2 g'(rho),
(since sig + sig' rho = g').  By the chain rule and the change of variables, the
Laplace form over the exterior is a form over the shell with the tensor
    M = |det J| J^-1 J^-T:    int grad' u . grad' v dx' = int grad u . M grad v dx;
M = I in the magnet and the air.

Discrete problem.  P1 on the whole grid, each tetrahedron's M taken at its
centroid (one-point rule): K_ij = sum_e vol_e grad phi_i . M_e grad phi_j;
u = 0 on the outer face (the image of infinity); b = G m over the magnet's
tetrahedra; K u = b on all other nodes.  u is the total reduced potential
(U = Ms u, u in metres): no splitting and no boundary matrix.  K is symmetric,
so the stray field at the magnet's nodes,
    mu0 h_d,i = -(Js/V_i) sum_j G_ji u_j,
is exactly the gradient field of
    E_d = -(Js/(2 mu0)) sum_i V_i m_i . mu0 h_d,i = (Js^2/(2 mu0)) b^T K^-1 b.
Exchange, anisotropy and Zeeman terms are those of oracle.micromag on the
magnet.  The linear system is solved directly (sparse LU).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import cofactors, kuhn_cube
from .micromag import MU0, CubeProblem, Evaluation


def shell_map(x: np.ndarray, c: np.ndarray, R1: float, R2: float) -> np.ndarray:
    """x' for points x of the shell (identity where rho <= R1)."""
    d = np.asarray(x, dtype=np.float64) - c
    rho = np.max(np.abs(d), axis=-1)
    out = np.array(d)
    sh = rho > R1
    with np.errstate(divide="ignore", invalid="ignore"):
        g = R1 * (R2 - R1) / (R2 - rho[sh])             # inf on the outer face
        out[sh] = d[sh] * (g / rho[sh])[:, None]
    return out + c


def shell_jacobian(x: np.ndarray, c: np.ndarray, R1: float, R2: float):
    """J (P, 3, 3) and det J (P,) of the map at points x with R1 < rho < R2;
    the sector is the first coordinate that attains the max."""
    d = np.asarray(x, dtype=np.float64) - c
    P = d.shape[0]
    k = np.argmax(np.abs(d), axis=1)
    rho = np.abs(d[np.arange(P), k])
    grad_rho = np.zeros((P, 3))
    grad_rho[np.arange(P), k] = np.sign(d[np.arange(P), k])
    g = R1 * (R2 - R1) / (R2 - rho)
    dg = R1 * (R2 - R1) / (R2 - rho) ** 2
    sig = g / rho
    dsig = (dg * rho - g) / rho ** 2
    J = sig[:, None, None] * np.eye(3)[None] + dsig[:, None, None] * d[:, :, None] * grad_rho[:, None, :]
    return J, sig * sig * dg


def shell_tensor(x: np.ndarray, c: np.ndarray, R1: float, R2: float) -> np.ndarray:
    """M = |det J| J^-1 J^-T (P, 3, 3) at points x of the shell."""
    J, detJ = shell_jacobian(x, c, R1, R2)
    Ji = np.linalg.inv(J)
    return np.abs(detJ)[:, None, None] * np.einsum("pij,pkj->pik", Ji, Ji)


class ShellProblem(CubeProblem):
    """One material on the Kuhn cube [0, n]^3 with the stray field from the
    space-transformation open boundary (air a cells deep, shell s cells deep)."""

    def __init__(self, n: int, Js: float, A: float, K1: float, axis, a: int, s: int,
                 cell: float = 2e-9):
        super().__init__(n, Js, A, K1, axis, cell=cell, demag=False)
        self.demag = True
        self.a, self.s = a, s
        nt = n + 2 * (a + s)
        lat, tets = kuhn_cube(nt)
        off = a + s
        self.grid_nodes = lat - off                                     # lattice, magnet at [0, n]^3
        self.grid_tets = tets
        self.c = np.full(3, n / 2.0)
        self.R1, self.R2 = n / 2.0 + a, n / 2.0 + a + s
        xyz = self.grid_nodes.astype(np.float64) * cell
        cof, det = cofactors(xyz, tets)
        cen = self.grid_nodes[tets].mean(axis=1)                        # lattice units
        rho_c = np.max(np.abs(cen - self.c), axis=1)
        M = np.broadcast_to(np.eye(3), (tets.shape[0], 3, 3)).copy()
        sh = rho_c > self.R1
        M[sh] = shell_tensor(cen[sh], self.c, self.R1, self.R2)
        self.shell_tets = sh
        self.tensor = M
        N = xyz.shape[0]
        kloc = np.einsum("tad,tde,tbe->tab", cof, M, cof) / (6.0 * np.abs(det))[:, None, None]
        rows = np.repeat(tets, 4, axis=1).ravel()
        cols = np.tile(tets, (1, 4)).ravel()
        Kg = sp.coo_matrix((kloc.ravel(), (rows, cols)), shape=(N, N)).tocsr()
        Kg.sum_duplicates()
        Kg.sort_indices()
        self.Kgrid = Kg
        rho_n = np.max(np.abs(self.grid_nodes - self.c), axis=1)
        self.outer = np.nonzero(rho_n == self.R2)[0]
        self.free = np.nonzero(rho_n < self.R2)[0]
        self._lu = None                                                 # factorised on first use
        # magnet node (i, j, k) -> grid node (i + off, j + off, k + off)
        mn = self.mesh.nodes.astype(np.int64) + off
        self.magnet_in_grid = mn[:, 0] + (nt + 1) * (mn[:, 1] + (nt + 1) * mn[:, 2])

    @property
    def lu_grid(self):
        """Sparse LU of K restricted to the nodes off the outer face."""
        if self._lu is None:
            self._lu = spla.splu(self.Kgrid[self.free][:, self.free].tocsc())
        return self._lu

    def grid_potential(self, m: np.ndarray) -> np.ndarray:
        """u on the whole grid (0 on the outer face) for the magnetisation m."""
        rhs = np.zeros(self.Kgrid.shape[0])
        rhs[self.magnet_in_grid] = self.rhs(m)
        u = np.zeros_like(rhs)
        u[self.free] = self.lu_grid.solve(rhs[self.free])
        return u

    def evaluate(self, m: np.ndarray, h_ext) -> Evaluation:
        m = np.asarray(m, dtype=np.float64)
        h_ext = np.asarray(h_ext, dtype=np.float64)
        Js, V = self.Js, self.V
        Km = self.Kcsr @ m
        h_ex = -(2.0 * self.A * MU0 / Js) * Km / V[:, None]
        ma = m @ self.axis
        h_an = (2.0 * self.K1 * MU0 / Js) * ma[:, None] * self.axis[None, :]
        ug = self.grid_potential(m)
        u = ug[self.magnet_in_grid]
        h_d = -Js * np.stack([self.Gt[d] @ u for d in range(3)], axis=1) / V[:, None]
        e_ex = self.A * float(np.sum(m * Km))
        e_an = self.K1 * float(np.dot(V, 1.0 - ma * ma))
        e_z = -(Js / MU0) * float(np.dot(V, m @ h_ext))
        e_d = -(Js / (2.0 * MU0)) * float(np.dot(V, np.sum(m * h_d, axis=1)))
        h = h_ex + h_an + h_ext[None, :] + h_d
        grad = -(Js / MU0) * V[:, None] * h / self.E0
        torque = float(np.max(np.linalg.norm(np.cross(m, h), axis=1))) / Js
        terms = dict(ex=e_ex, an=e_an, z=e_z, d=e_d)
        zero = np.zeros(m.shape[0])
        return Evaluation(E=e_ex + e_an + e_z + e_d, terms=terms, h=h, grad=grad, torque=torque,
                          u1=u, u2=zero, uT=u)

