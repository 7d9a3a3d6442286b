"""Pins of the oracle's hierarchical-matrix (H-matrix) boundary operator
(oracle/hmatrix.py; the paper's Sec. 3.1 names hierarchical matrices for the
boundary element method): the cluster and block trees are partitions with the
stated admissibility, checked from the raw coordinates; the two compressions
give the minimal rank on matrices of known singular values and recover exact
low rank; and the assembled B_H obeys ||B - B_H||_F <= eps ||B||_F against the
dense double-layer matrix (itself pinned by B 1 = -1 and the closed-form
integrals), with the consequences for row sums and demagnetising energies."""
import math

import numpy as np
import pytest

from oracle import hmatrix as hm
from oracle.bem import bem_block, bem_matrix, bem_matrix_general
from oracle.mesh import cube_mesh, tet_mesh
from oracle.micromag import CubeProblem
from synth import ball_mesh


@pytest.fixture(scope="module")
def cube12():
    c = cube_mesh(12, 1.0)
    return c, bem_matrix(c.nodes, 12, c.bnd, c.tris)


@pytest.fixture(scope="module")
def ball():
    xyz, tets = ball_mesh(10, 1.0)
    t = tet_mesh(xyz, tets)
    return t, bem_matrix_general(t.nodes, t.bnd, t.tris)


def _surfaces(cube12, ball):
    (c, Bc), (t, Bb) = cube12, ball
    return [(c.nodes.astype(np.float64), c.bnd, c.tris, Bc), (t.nodes, t.bnd, t.tris, Bb)]


def test_block_extraction_matches_the_dense_matrix(cube12, ball):
    """bem_block gives B's entries from the column triangles alone, diagonal
    (solid-angle) terms included, on the cube and on a curved surface."""
    rng = np.random.default_rng(3)
    for xyz, bnd, tris, B in _surfaces(cube12, ball):
        nb = bnd.size
        for _ in range(3):
            rows = np.sort(rng.choice(nb, 40, replace=False))
            cols = np.unique(np.concatenate([rows[:12], rng.choice(nb, 50, replace=False)]))
            blk = bem_block(xyz, bnd, tris, rows, cols)
            assert np.abs(blk - B[np.ix_(rows, cols)]).max() <= 1e-14 * np.abs(B).max()


@pytest.mark.parametrize("n_min", [8, 32])
def test_cluster_tree_is_a_balanced_geometric_bisection(cube12, ball, n_min):
    for xyz, bnd, tris, _ in _surfaces(cube12, ball):
        pts = xyz[bnd]
        slo, shi = hm.support_boxes(xyz, bnd, tris)
        root = hm.cluster_tree(pts, slo, shi, n_min)
        assert np.array_equal(root.idx, np.arange(bnd.size))
        leaves, stack = [], [root]
        while stack:
            c = stack.pop()
            assert np.all(np.diff(c.idx) > 0)
            assert np.allclose(c.lo_r, pts[c.idx].min(0)) and np.allclose(c.hi_r, pts[c.idx].max(0))
            assert np.all(c.lo_c <= pts[c.idx].min(0)) and np.all(c.hi_c >= pts[c.idx].max(0))
            if c.leaf:
                assert c.idx.size <= n_min
                leaves.append(c.idx)
                continue
            a, b = c.children
            assert c.idx.size > n_min
            assert (a.idx.size, b.idx.size) == (c.idx.size // 2, c.idx.size - c.idx.size // 2)
            assert np.array_equal(np.sort(np.concatenate([a.idx, b.idx])), c.idx)
            axis = int(np.argmax(pts[c.idx].max(0) - pts[c.idx].min(0)))
            assert pts[a.idx, axis].max() <= pts[b.idx, axis].min()
            stack.extend(c.children)
        assert np.array_equal(np.sort(np.concatenate(leaves)), np.arange(bnd.size))


def _support_box_direct(xyz, bnd, tris, j):
    """Bounding box of the triangles that contain node bnd[j], from scratch."""
    mine = tris[np.any(tris == bnd[j], axis=1)]
    v = xyz[mine.ravel()]
    return v.min(0), v.max(0)


@pytest.mark.parametrize("eta", [1.0, 2.0])
def test_block_tree_covers_every_entry_once_and_admits_only_separated_pairs(cube12, ball, eta):
    for xyz, bnd, tris, _ in _surfaces(cube12, ball):
        pts = xyz[bnd]
        slo, shi = hm.support_boxes(xyz, bnd, tris)
        for j in range(0, bnd.size, 97):
            lo, hi = _support_box_direct(xyz, bnd, tris, j)
            assert np.array_equal(lo, slo[j]) and np.array_equal(hi, shi[j])
        root = hm.cluster_tree(pts, slo, shi, 16)
        count = np.zeros((bnd.size, bnd.size), dtype=np.int64)
        n_low = 0
        for tau, sigma, low in hm.block_tree(root, eta):
            count[np.ix_(tau.idx, sigma.idx)] += 1
            # admissibility recomputed from the points and supports themselves
            rlo, rhi = pts[tau.idx].min(0), pts[tau.idx].max(0)
            clo, chi = slo[sigma.idx].min(0), shi[sigma.idx].max(0)
            gap = np.maximum(0.0, np.maximum(rlo - chi, clo - rhi))
            dist = math.sqrt(float(gap @ gap))
            diam = min(float(np.linalg.norm(rhi - rlo)), float(np.linalg.norm(chi - clo)))
            if low:
                n_low += 1
                assert dist > 0.0 and diam <= eta * dist
                assert not np.intersect1d(tau.idx, sigma.idx).size
            else:
                assert tau.leaf or sigma.leaf
                assert not (dist > 0.0 and diam <= eta * dist)
        assert np.all(count == 1)
        assert n_low > 0


def _known_spectrum(m, n, s, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.normal(size=(m, s.size)))
    Q2, _ = np.linalg.qr(rng.normal(size=(n, s.size)))
    return (Q1 * s) @ Q2.T


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-7])
def test_truncated_svd_takes_the_smallest_sufficient_rank(eps):
    """With singular values 2^-k, the smallest k with sqrt(sum_{i>=k} s_i^2) <=
    eps ||A||_F is known in closed form; the error at that rank is the tail."""
    s = 2.0 ** -np.arange(30)
    A = _known_spectrum(60, 45, s, seed=7)
    U, V = hm.truncated_svd(A, eps)
    norm = math.sqrt(float(np.sum(s * s)))
    tails = [math.sqrt(float(np.sum(s[k:] ** 2))) for k in range(s.size + 1)]
    k = next(k for k in range(s.size + 1) if tails[k] <= eps * norm)
    assert U.shape == (60, k) and V.shape == (k, 45)
    assert np.linalg.norm(A - U @ V) == pytest.approx(tails[k], rel=1e-6, abs=1e-15)
    U0, V0 = hm.truncated_svd(np.zeros((5, 4)), eps)
    assert U0.shape == (5, 0) and V0.shape == (0, 4)


@pytest.mark.parametrize("r", [1, 2, 5, 9])
def test_cross_approximation_recovers_exact_low_rank(r):
    """A rank-r matrix is reproduced in exactly r pivots (each pivot removes
    one rank from the residual), to rounding."""
    rng = np.random.default_rng(r)
    A = rng.normal(size=(50, r)) @ rng.normal(size=(r, 37))
    U, V = hm.cross_approximation(A, 1e-12)
    assert U.shape[1] == r
    assert np.linalg.norm(A - U @ V) <= 1e-12 * np.linalg.norm(A)


def test_cross_approximation_meets_the_tolerance_on_a_smooth_kernel():
    """1/|x - y| between two separated point clouds: the residual bound holds
    and the rank stays close to the optimal (SVD) rank."""
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, size=(120, 3))
    y = rng.uniform(0, 1, size=(90, 3)) + np.array([3.0, 0.0, 0.0])
    A = 1.0 / np.linalg.norm(x[:, None] - y[None], axis=-1)
    for eps in (1e-3, 1e-6, 1e-10):
        U, V = hm.cross_approximation(A, eps)
        Us, _ = hm.truncated_svd(A, eps)
        assert np.linalg.norm(A - U @ V) <= eps * np.linalg.norm(A)
        assert Us.shape[1] <= U.shape[1] <= 2 * Us.shape[1] + 2


@pytest.mark.parametrize("method", ["svd", "aca"])
@pytest.mark.parametrize("eps", [1e-4, 1e-8])
def test_hmatrix_obeys_the_frobenius_bound(cube12, ball, method, eps):
    rng = np.random.default_rng(5)
    for xyz, bnd, tris, B in _surfaces(cube12, ball):
        H = hm.build_hmatrix(hm.dense_blocks(B), xyz, bnd, tris, eps=eps, eta=2.0, n_min=16, method=method)
        D = H.to_dense()
        nB = np.linalg.norm(B)
        assert np.linalg.norm(D - B) <= eps * nB
        assert any(L.low_rank for L in H.leaves)
        for L in H.leaves:
            if not L.low_rank:
                assert np.array_equal(L.D, B[np.ix_(L.rows, L.cols)])
            else:
                A = B[np.ix_(L.rows, L.cols)]
                assert np.linalg.norm(A - L.U @ L.V) <= eps * np.linalg.norm(A) * (1 + 1e-9)
                assert L.U.shape[1] * (L.rows.size + L.cols.size) < L.rows.size * L.cols.size
        X = rng.normal(size=(bnd.size, 3))
        assert np.abs(H @ X - D @ X).max() <= 1e-12 * np.abs(D @ X).max()
        assert np.abs(H.T @ X - D.T @ X).max() <= 1e-12 * np.abs(D.T @ X).max()
        # B 1 = -1 holds for the dense matrix; B_H moves it by at most ||B - B_H||_2 sqrt(nb)
        one = np.ones(bnd.size)
        assert np.linalg.norm(H @ one + 1.0) <= eps * nB * math.sqrt(bnd.size) + 1e-12 * bnd.size


def test_on_demand_blocks_build_the_same_operator(cube12):
    """Built from entries computed block by block (no dense B), the operator
    has the same leaves and the same bound."""
    c, B = cube12
    xyz = c.nodes.astype(np.float64)
    Hd = hm.build_hmatrix(hm.dense_blocks(B), xyz, c.bnd, c.tris, eps=1e-6, eta=2.0, n_min=16)
    Ho = hm.build_hmatrix(lambda r, k: bem_block(xyz, c.bnd, c.tris, r, k), xyz, c.bnd, c.tris,
                          eps=1e-6, eta=2.0, n_min=16)
    assert len(Hd.leaves) == len(Ho.leaves)
    for a, b in zip(Hd.leaves, Ho.leaves):
        assert np.array_equal(a.rows, b.rows) and np.array_equal(a.cols, b.cols) and a.low_rank == b.low_rank
    assert np.linalg.norm(Ho.to_dense() - B) <= 1e-6 * np.linalg.norm(B)


def test_storage_falls_with_the_mesh_size():
    """The stored fraction of the nb^2 entries shrinks as the surface grows
    (n = 8, 12, 16 cells per side, eps 1e-4)."""
    fr = []
    for n in (8, 12, 16):
        c = cube_mesh(n, 1.0)
        xyz = c.nodes.astype(np.float64)
        H = hm.build_hmatrix(lambda r, k: bem_block(xyz, c.bnd, c.tris, r, k), xyz, c.bnd, c.tris,
                             eps=1e-4, eta=2.0, n_min=16)
        fr.append(hm.storage_fraction(H))
    assert fr[0] > fr[1] > fr[2]
    assert fr[2] < 0.5


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_demag_energy_and_field_with_the_hmatrix(eps):
    """The full energy and field with B_H in place of B: the demagnetising
    energy moves by less than eps Kd V and the field by less than eps of its
    largest value, on a random state of a 10^3-cell cube."""
    n = 10
    p = CubeProblem(n, 1.61, 7.7e-12, 4.3e6, [0, 0, 1])
    c = p.mesh
    H = hm.build_hmatrix(hm.dense_blocks(p.B), c.nodes.astype(np.float64), c.bnd, c.tris, eps=eps,
                         eta=2.0, n_min=16)
    assert any(L.low_rank for L in H.leaves)
    ph = CubeProblem(n, 1.61, 7.7e-12, 4.3e6, [0, 0, 1], B=H)
    rng = np.random.default_rng(2)
    m = rng.normal(size=(c.N, 3))
    m /= np.linalg.norm(m, axis=1)[:, None]
    e, eh = p.evaluate(m, [0, 0, -1.0]), ph.evaluate(m, [0, 0, -1.0])
    assert abs(eh.terms["d"] - e.terms["d"]) <= eps * p.Kd * p.V.sum()
    assert np.abs(eh.h - e.h).max() <= eps * np.abs(e.h).max()
    for k in ("ex", "an", "z"):
        assert eh.terms[k] == e.terms[k]


def test_minimiser_with_the_hmatrix_follows_the_dense_one():
    """The full minimisation with B_H (eps 1e-6) in place of the dense B takes the
    same steps and ends at the same energy and torque, to far below the solver's
    1e-6 (two instances of the batched workload's distribution on a 10^3 cube)."""
    import copy
    from oracle.minimise import minimise
    from synth.inputs import A_JM, JS_T, K1_JM3, batched_case
    insts = batched_case(10, 2, seed=4)
    dense = CubeProblem(10, JS_T, A_JM, K1_JM3, insts[0].axis)
    c = dense.mesh
    H = hm.build_hmatrix(hm.dense_blocks(dense.B), c.nodes.astype(np.float64), c.bnd, c.tris, eps=1e-6,
                         eta=2.0, n_min=16)
    assert any(L.low_rank for L in H.leaves)
    compressed = copy.copy(dense)
    compressed.B = H
    scale = dense.Kd * dense.V.sum()
    for inst in insts:
        for p in (dense, compressed):
            p.axis = inst.axis / np.linalg.norm(inst.axis)
        a = minimise(dense, inst.m0, inst.h_ext, tol=1e-6, max_iter=5000)
        b = minimise(compressed, inst.m0, inst.h_ext, tol=1e-6, max_iter=5000)
        assert a.status == b.status == 0 and a.evaluations == b.evaluations
        assert abs(a.E - b.E) <= 1e-9 * scale
        assert abs(dense.evaluate(b.m, inst.h_ext).torque - b.torque) <= 1e-8
