"""Hierarchical-matrix (H-matrix) form of the double-layer boundary matrix B.

Oracle -- test infrastructure only: the GPU library neither imports nor links it.

Paper, Sec. 3.1: the LLG solver of the comparison speeds up its boundary element
method with hierarchical matrices; the paper gives no construction.  This module
restates the textbook one (Hackbusch; Grasedyck & Hackbusch; Bebendorf) on the
boundary nodes of the hybrid FEM/BEM of oracle.bem, in three plain steps:

1. Cluster tree.  A cluster is a set of boundary positions (indices into bnd,
   kept in ascending order).  It is split in two when it holds more than n_min
   positions: its nodes are ordered by their coordinate along the longest side
   of their bounding box (ties by position) and the first floor(m/2) form the
   first child, the rest the second.
2. Block tree.  A block (tau, sigma) pairs a row cluster (collocation points
   x_i, box Q_r(tau)) with a column cluster (supports of the hat functions
   phi_j, i.e. the union of the surface triangles around node j, box
   Q_c(sigma)).  It is admissible when
        dist(Q_r(tau), Q_c(sigma)) > 0  and
        min(diam Q_r(tau), diam Q_c(sigma)) <= eta dist(Q_r(tau), Q_c(sigma)),
   with diam the length of a box's diagonal and dist the Euclidean distance
   between two boxes (both sqrt(x^2 + y^2 + z^2), summed in that order, so
   that every decision is reproducible to the bit).  Starting from (root, root): an admissible block is a
   low-rank leaf; otherwise, if tau or sigma is a leaf cluster, a dense leaf;
   otherwise its four children blocks (tau_a, sigma_b), a, b in (0, 1), in that
   order.
3. Low-rank leaves.  The block A (entries of B) is replaced by U V with the
   smallest rank k for which ||A - U V||_F <= eps ||A||_F, either from the
   truncated singular value decomposition (Eckart-Young: the optimal rank-k
   approximation in the Frobenius norm) or by cross approximation with full
   pivoting: repeatedly take the entry of largest modulus of the residual R
   (first in row-major order on ties), i*, j*, append u = R[:, j*],
   v = R[i*, :] / R[i*, j*] and subtract u v from R, until
   ||R||_F <= eps ||A||_F.  Each step zeroes row i* and column j* of R.
   A leaf whose factors would hold at least as many values as the block
   itself (k (m + n) >= m n) keeps the block's exact entries instead.

Since the admissible blocks are disjoint, ||B - B_H||_F <= eps ||B||_F for
either compression: every bound below follows from that.  Dense leaves hold
the exact entries of B.  Matrix-vector products are plain sums over the
leaves in block-tree order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    idx: np.ndarray                     # boundary positions, ascending
    lo_r: np.ndarray                    # bounding box of the collocation points
    hi_r: np.ndarray
    lo_c: np.ndarray                    # bounding box of the hat supports
    hi_c: np.ndarray
    children: list = field(default_factory=list)

    @property
    def leaf(self) -> bool:
        return not self.children


def support_boxes(xyz: np.ndarray, bnd: np.ndarray, tris: np.ndarray):
    """Per boundary position j, the bounding box (lo, hi) of the surface
    triangles that contain node bnd[j] (the support of the hat phi_j)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    pos = -np.ones(xyz.shape[0], dtype=np.int64)
    pos[bnd] = np.arange(bnd.size)
    lo = np.full((bnd.size, 3), np.inf)
    hi = np.full((bnd.size, 3), -np.inf)
    for t in np.asarray(tris):
        tlo, thi = xyz[t].min(axis=0), xyz[t].max(axis=0)
        for v in t:
            j = pos[v]
            lo[j] = np.minimum(lo[j], tlo)
            hi[j] = np.maximum(hi[j], thi)
    return lo, hi


def _cluster(idx, pts, slo, shi) -> Cluster:
    return Cluster(idx, pts[idx].min(axis=0), pts[idx].max(axis=0), slo[idx].min(axis=0), shi[idx].max(axis=0))


def cluster_tree(pts: np.ndarray, slo: np.ndarray, shi: np.ndarray, n_min: int = 32) -> Cluster:
    """Step 1: the cluster tree over all boundary positions."""
    root = _cluster(np.arange(pts.shape[0]), pts, slo, shi)
    stack = [root]
    while stack:
        c = stack.pop()
        m = c.idx.size
        if m <= n_min:
            continue
        axis = int(np.argmax(c.hi_r - c.lo_r))
        order = np.lexsort((c.idx, pts[c.idx, axis]))          # by coordinate, then position
        half = m // 2
        a, b = np.sort(c.idx[order[:half]]), np.sort(c.idx[order[half:]])
        c.children = [_cluster(a, pts, slo, shi), _cluster(b, pts, slo, shi)]
        stack.extend(c.children)
    return root


def _length(v) -> float:
    """sqrt(v0^2 + v1^2 + v2^2), summed in that order (IEEE double)."""
    x, y, z = float(v[0]), float(v[1]), float(v[2])
    return math.sqrt(x * x + y * y + z * z)


def box_diam(lo, hi) -> float:
    return _length(hi - lo)


def box_dist(lo1, hi1, lo2, hi2) -> float:
    gap = np.maximum(0.0, np.maximum(lo1 - hi2, lo2 - hi1))
    return _length(gap)


def admissible(tau: Cluster, sigma: Cluster, eta: float) -> bool:
    d = box_dist(tau.lo_r, tau.hi_r, sigma.lo_c, sigma.hi_c)
    return d > 0.0 and min(box_diam(tau.lo_r, tau.hi_r), box_diam(sigma.lo_c, sigma.hi_c)) <= eta * d


def block_tree(root: Cluster, eta: float = 1.0):
    """Step 2: the leaves of the block tree, in depth-first order, as
    (tau, sigma, is_low_rank)."""
    out = []

    def visit(tau, sigma):
        if admissible(tau, sigma, eta):
            out.append((tau, sigma, True))
        elif tau.leaf or sigma.leaf:
            out.append((tau, sigma, False))
        else:
            for t in tau.children:
                for s in sigma.children:
                    visit(t, s)

    visit(root, root)
    return out


def truncated_svd(A: np.ndarray, eps: float):
    """Step 3, optimal form: the smallest k with ||A - U V||_F <= eps ||A||_F."""
    m, n = A.shape
    norm = float(np.linalg.norm(A))
    if norm == 0.0:
        return np.zeros((m, 0)), np.zeros((0, n))
    W, s, Vt = np.linalg.svd(A, full_matrices=False)
    tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])              # tail[k] = ||A - A_k||_F
    tail = np.append(tail, 0.0)
    k = int(np.nonzero(tail <= eps * norm)[0][0])
    return W[:, :k] * s[:k], Vt[:k]


def cross_approximation(A: np.ndarray, eps: float):
    """Step 3, cross approximation with full pivoting."""
    R = np.array(A, dtype=np.float64)
    norm = float(np.linalg.norm(R))
    us, vs = [], []
    while np.linalg.norm(R) > eps * norm:
        i, j = np.unravel_index(int(np.argmax(np.abs(R))), R.shape)
        u = R[:, j].copy()
        v = R[i, :] / R[i, j]
        R -= np.outer(u, v)
        us.append(u)
        vs.append(v)
    m, n = R.shape
    U = np.stack(us, axis=1) if us else np.zeros((m, 0))
    V = np.stack(vs, axis=0) if vs else np.zeros((0, n))
    return U, V


@dataclass
class Leaf:
    rows: np.ndarray
    cols: np.ndarray
    low_rank: bool
    D: np.ndarray | None = None         # dense leaf: the entries
    U: np.ndarray | None = None         # low-rank leaf: A ~ U V
    V: np.ndarray | None = None

    @property
    def rank(self) -> int:
        return self.U.shape[1] if self.low_rank else min(self.rows.size, self.cols.size)

    @property
    def stored(self) -> int:
        if self.low_rank:
            return self.U.shape[1] * (self.rows.size + self.cols.size)
        return self.rows.size * self.cols.size


class HMatrix:
    """B_H: the leaves of the block tree, dense or low rank.  Supports B_H @ x
    and B_H.T @ x for x of shape (nb,) or (nb, k)."""

    def __init__(self, nb: int, leaves: list):
        self.nb = nb
        self.leaves = leaves
        self.shape = (nb, nb)

    def __matmul__(self, x):
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros((self.nb,) + x.shape[1:])
        for L in self.leaves:
            xs = x[L.cols]
            y[L.rows] += L.U @ (L.V @ xs) if L.low_rank else L.D @ xs
        return y

    def rmatvec(self, x):
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros((self.nb,) + x.shape[1:])
        for L in self.leaves:
            xs = x[L.rows]
            y[L.cols] += L.V.T @ (L.U.T @ xs) if L.low_rank else L.D.T @ xs
        return y

    @property
    def T(self):
        return _Transposed(self)

    def to_dense(self) -> np.ndarray:
        out = np.zeros(self.shape)
        for L in self.leaves:
            out[np.ix_(L.rows, L.cols)] += L.U @ L.V if L.low_rank else L.D
        return out

    def stored(self) -> int:
        """Number of stored values (dense entries plus k (m + n) per low-rank leaf)."""
        return sum(L.stored for L in self.leaves)


class _Transposed:
    def __init__(self, H: HMatrix):
        self.H = H

    def __matmul__(self, x):
        return self.H.rmatvec(x)


def build_hmatrix(block, xyz: np.ndarray, bnd: np.ndarray, tris: np.ndarray, eps: float = 1e-6,
                  eta: float = 1.0, n_min: int = 32, method: str = "svd") -> HMatrix:
    """B_H for the boundary matrix whose sub-blocks block(rows, cols) returns
    (rows, cols: arrays of boundary positions)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    pts = xyz[bnd]
    slo, shi = support_boxes(xyz, bnd, tris)
    root = cluster_tree(pts, slo, shi, n_min)
    compress = {"svd": truncated_svd, "aca": cross_approximation}[method]
    leaves = []
    for tau, sigma, low in block_tree(root, eta):
        A = np.asarray(block(tau.idx, sigma.idx), dtype=np.float64)
        if low:
            U, V = compress(A, eps)
            if U.shape[1] * (A.shape[0] + A.shape[1]) < A.size:
                leaves.append(Leaf(tau.idx, sigma.idx, True, U=U, V=V))
                continue
        leaves.append(Leaf(tau.idx, sigma.idx, False, D=A))
    return HMatrix(bnd.size, leaves)


def dense_blocks(B: np.ndarray):
    """Sub-blocks of an assembled boundary matrix, for build_hmatrix."""
    B = np.asarray(B)
    return lambda rows, cols: B[np.ix_(rows, cols)]


def storage_fraction(H: HMatrix) -> float:
    return H.stored() / float(H.nb * H.nb)

