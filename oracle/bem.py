"""Double-layer boundary matrix of the hybrid FEM/BEM (Fredkin-Koehler) open boundary.

Paper, Sec. 3.1: the magnetostatic field comes from a magnetic scalar potential;
the open boundary is deferred to cited schemes (hybrid finite element / boundary
element method for the LLG solver).  Reading used here (the dense hybrid
FEM/BEM): split U = U1 + U2 with
  * U1: Delta U1 = div M inside, dU1/dn = M.n on the surface, U1 = 0 outside;
  * U2: harmonic inside and outside, jump U2_in - U2_out = -U1 across the surface,
    hence the double-layer potential of density U1:
        U2(x) = 1/(4 pi) int_S U1(y) (x-y).n_y / |x-y|^3 dS_y,
    and on the surface (limit from inside, interior solid angle Omega(x)):
        U2(x_i) = sum_j B_ij U1(x_j),
        B_ij = 1/(4 pi) sum_{t ∋ j} I_t,j(x_i) + (Omega_i/(4 pi) - 1) delta_ij,
    where I_t,j(x) = int_t phi_j(y) (x-y).n / |x-y|^3 dS_y for the linear hat
    phi_j on the flat surface triangle t.  The constant density 1 gives U2 = -1
    on the surface, i.e. B 1 = -1.

Closed form of I (derived here; equivalent to Lindholm's 1984 formulas).  Let h =
(y_1 - x).n, p = x + h n the foot point, eta_k = |y_k - x|, s_k the length of
edge k (y_k -> y_k+1), nu_k its outward in-plane normal, P_k = ln((eta_k +
eta_k+1 + s_k)/(eta_k + eta_k+1 - s_k)) = int_edge dl/|y - x|, and Omega_t the
signed solid angle int_t (y-x).n/|y-x|^3 dS (Van Oosterom-Strackee).  Writing
phi_k(y) = phi_k(p) + grad phi_k.(y - p) and using int_t grad_y(1/r) = oint 1/r nu:
        I_k = -phi_k(p) Omega_t + h grad phi_k . sum_e nu_e P_e.
Coplanar pairs (h = 0, including the triangles that contain x) give 0.

All coordinates are lattice units; the operator is scale free.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def hat_double_layer(x: np.ndarray, tri: np.ndarray, exclude: np.ndarray | None = None,
                     log1p_edges: bool = False) -> np.ndarray:
    """I[p, t, k] = int_t phi_k(y) (x_p - y).n_t / |x_p - y|^3 dS_y.

    x: (P, 3) targets; tri: (T, 3, 3) vertices ordered counter-clockwise seen
    from the outside (normal (y2-y1) x (y3-y1) outward).  exclude: optional
    (P, T) mask of pairs known to be coplanar (x_p a vertex of t), which give
    0 whatever rounding does to h.  log1p_edges: evaluate P_e = ln((a+s)/(a-s)),
    a = eta_k + eta_k+1, as log1p(2s/(a-s)) -- the same value; far from the
    triangle the ratio is 1 + O(s/r) and its plain logarithm loses a factor r/s
    of relative accuracy."""
    x = np.asarray(x, dtype=np.float64)[:, None, :]          # (P, 1, 3)
    y = np.asarray(tri, dtype=np.float64)[None, :, :, :]      # (1, T, 3, 3)
    y1, y2, y3 = y[..., 0, :], y[..., 1, :], y[..., 2, :]
    cr = np.cross(y2 - y1, y3 - y1)                           # (1, T, 3)
    a2 = np.linalg.norm(cr, axis=-1, keepdims=True)           # 2 * area
    nrm = cr / a2
    r = [y1 - x, y2 - x, y3 - x]                              # (P, T, 3) each
    eta = [np.linalg.norm(rk, axis=-1) for rk in r]
    h = np.einsum("ptd,ptd->pt", r[0], np.broadcast_to(nrm, r[0].shape))
    # signed solid angle of the triangle seen from x
    num = np.einsum("ptd,ptd->pt", r[0], np.cross(r[1], r[2]))
    den = (eta[0] * eta[1] * eta[2]
           + eta[0] * np.einsum("ptd,ptd->pt", r[1], r[2])
           + eta[1] * np.einsum("ptd,ptd->pt", r[2], r[0])
           + eta[2] * np.einsum("ptd,ptd->pt", r[0], r[1]))
    omega = 2.0 * np.arctan2(num, den)
    ys = [y1, y2, y3]
    foot = x + h[..., None] * nrm                             # (P, T, 3)
    coplanar = h == 0.0
    if exclude is not None:
        coplanar = coplanar | exclude
    hs = np.where(coplanar, 1.0, h)                           # avoid 0/0 in unused logs
    edge_sum = np.zeros_like(foot)
    for k in range(3):
        a, b = ys[k], ys[(k + 1) % 3]
        e = b - a
        s = np.linalg.norm(e, axis=-1)                        # (1, T)
        nu = np.cross(e, nrm) / s[..., None]
        ea, eb = eta[k], eta[(k + 1) % 3]
        with np.errstate(divide="ignore", invalid="ignore"):
            if log1p_edges:
                P = np.log1p(2.0 * s / (ea + eb - s))
            else:
                P = np.log((ea + eb + s) / (ea + eb - s))
        P = np.where(coplanar, 0.0, P)
        edge_sum = edge_sum + nu * P[..., None]
    out = np.empty(h.shape + (3,))
    for k in range(3):
        a, b = ys[(k + 1) % 3], ys[(k + 2) % 3]               # the edge opposite vertex k
        phi_p = np.einsum("ptd,ptd->pt", np.cross(np.broadcast_to(b - a, foot.shape), foot - a),
                          np.broadcast_to(nrm, foot.shape)) / a2[..., 0]
        grad = np.cross(nrm, b - a) / a2                      # (1, T, 3)
        val = -phi_p * omega + hs * np.einsum("ptd,ptd->pt",
                                              np.broadcast_to(grad, edge_sum.shape), edge_sum)
        out[..., k] = np.where(coplanar, 0.0, val)
    return out


def box_interior_solid_angle(nodes: np.ndarray, n: int) -> np.ndarray:
    """Interior solid angle of the cube at surface lattice points: 2 pi on a face,
    pi on an edge, pi/2 at a corner (number of coordinates at 0 or n)."""
    c = np.sum((nodes == 0) | (nodes == n), axis=1)
    table = np.array([4.0 * math.pi, 2.0 * math.pi, math.pi, 0.5 * math.pi])
    return table[c]


def incidence(tris: np.ndarray, bnd: np.ndarray, N: int) -> sp.csr_matrix:
    """S (3F, nb): S[3t+k, col(tris[t,k])] = 1, mapping triangle-vertex slots to
    boundary columns."""
    pos = -np.ones(N, dtype=np.int64)
    pos[bnd] = np.arange(bnd.size)
    cols = pos[tris.ravel()]
    assert np.all(cols >= 0)
    return sp.csr_matrix((np.ones(cols.size), (np.arange(cols.size), cols)),
                         shape=(cols.size, bnd.size))


def bem_matrix(nodes: np.ndarray, n: int, bnd: np.ndarray, tris: np.ndarray,
               rows=None, chunk: int = 128) -> np.ndarray:
    """Dense B (len(rows) x nb), rows given as boundary positions (default: all)."""
    nb = bnd.size
    if rows is None:
        rows = np.arange(nb)
    rows = np.asarray(rows)
    S = incidence(tris, bnd, nodes.shape[0])
    txyz = nodes[tris].astype(np.float64)                    # (F, 3, 3)
    omega = box_interior_solid_angle(nodes[bnd[rows]], n)
    out = np.empty((rows.size, nb))
    for s in range(0, rows.size, chunk):
        r = rows[s:s + chunk]
        I = hat_double_layer(nodes[bnd[r]].astype(np.float64), txyz)   # (p, F, 3)
        out[s:s + chunk] = (S.T @ I.reshape(r.size, -1).T).T / (4.0 * math.pi)
    out[np.arange(rows.size), rows] += omega / (4.0 * math.pi) - 1.0
    return out


def interior_solid_angle(xyz: np.ndarray, bnd: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Interior solid angle of a closed triangulated surface at its vertices, by
    Girard's theorem: the cone of the incident triangles cuts a spherical
    polygon out of the unit sphere around x_i, whose area is the sum of its
    angles minus (m - 2) pi.  Its angle at fan edge u_b is the interior
    dihedral angle between the two incident triangles that share the edge,
    atan2(u_b . (w_a x w_c), w_a . w_c) in [0, 2 pi), where w_a, w_c are the
    neighbouring fan edges projected orthogonally to u_b and (x_i, a, b),
    (x_i, b, c) are consecutive triangles in outward counter-clockwise order.
    2 pi on a flat face, pi on a straight edge, pi/2 at a box corner."""
    xyz = np.asarray(xyz, dtype=np.float64)
    out = np.empty(bnd.size)
    nxt = {}
    for t in np.asarray(tris):
        for k in range(3):
            nxt.setdefault(int(t[k]), {})[int(t[(k + 1) % 3])] = int(t[(k + 2) % 3])
    for q, i in enumerate(np.asarray(bnd)):
        fan = nxt[int(i)]                        # a -> b for every triangle (i, a, b)
        m = len(fan)
        x = xyz[i]
        total = 0.0
        for a, b in fan.items():
            c = fan[b]                           # the next triangle (i, b, c)
            u = xyz[b] - x
            u = u / np.linalg.norm(u)
            wa = xyz[a] - x
            wa = wa - np.dot(wa, u) * u
            wc = xyz[c] - x
            wc = wc - np.dot(wc, u) * u
            th = math.atan2(float(np.dot(u, np.cross(wa, wc))), float(np.dot(wa, wc)))
            total += th % (2.0 * math.pi)
        out[q] = total - (m - 2) * math.pi
    return out


def bem_matrix_general(nodes: np.ndarray, bnd: np.ndarray, tris: np.ndarray, rows=None,
                       chunk: int = 128) -> np.ndarray:
    """Dense B (len(rows) x nb) on any closed triangulated surface: as
    bem_matrix, with the interior solid angles from interior_solid_angle and
    the triangles incident to the collocation node excluded explicitly."""
    nb = bnd.size
    if rows is None:
        rows = np.arange(nb)
    rows = np.asarray(rows)
    nodes = np.asarray(nodes, dtype=np.float64)
    S = incidence(tris, bnd, nodes.shape[0])
    txyz = nodes[tris]
    omega = interior_solid_angle(nodes, bnd[rows], tris)
    out = np.empty((rows.size, nb))
    for s in range(0, rows.size, chunk):
        r = rows[s:s + chunk]
        ids = bnd[r]
        excl = np.any(tris[None, :, :] == ids[:, None, None], axis=2)
        I = hat_double_layer(nodes[ids], txyz, exclude=excl)
        out[s:s + chunk] = (S.T @ I.reshape(r.size, -1).T).T / (4.0 * math.pi)
    out[np.arange(rows.size), rows] += omega / (4.0 * math.pi) - 1.0
    return out


def bem_block(nodes: np.ndarray, bnd: np.ndarray, tris: np.ndarray, rows, cols) -> np.ndarray:
    """B[rows][:, cols] (boundary positions) without assembling the rest of B:
    the same entries as bem_matrix_general, from the triangles around the column
    nodes only, with the solid-angle term where a row meets its own column."""
    nodes = np.asarray(nodes, dtype=np.float64)
    rows, cols = np.asarray(rows), np.asarray(cols)
    pos = -np.ones(nodes.shape[0], dtype=np.int64)
    pos[bnd] = np.arange(bnd.size)
    local = -np.ones(bnd.size, dtype=np.int64)
    local[cols] = np.arange(cols.size)
    slot = local[pos[tris]]                                  # (F, 3): block column of each vertex, or -1
    sel = np.nonzero((slot >= 0).any(axis=1))[0]
    ids = bnd[rows]
    out = np.zeros((rows.size, cols.size))
    if sel.size:
        excl = np.any(tris[sel][None, :, :] == ids[:, None, None], axis=2)
        I = hat_double_layer(nodes[ids], nodes[tris[sel]], exclude=excl)   # (P, S, 3)
        for k in range(3):
            c = slot[sel, k]
            ok = c >= 0
            np.add.at(out.T, c[ok], I[:, ok, k].T)
        out /= 4.0 * math.pi
    a, b = np.nonzero(rows[:, None] == cols[None, :])
    if a.size:
        omega = interior_solid_angle(nodes, bnd[rows[a]], tris)
        out[a, b] += omega / (4.0 * math.pi) - 1.0
    return out
