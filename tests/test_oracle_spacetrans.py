"""Pins of the oracle's space-transformation open boundary (oracle/spacetrans.py;
the paper's Sec. 3.1: its steepest-descent solver maps a shell onto the
exterior instead of using a boundary element method).  The map and its
Jacobian are checked against finite differences and their closed-form
determinants; the stiffness against its kernel, symmetry and the patch test;
the discrete potential of a uniformly magnetised cube against the exact
closed-form potential of a box (inside the magnet and, through the map, out to
many box sizes), converging under refinement; the demagnetising factors against
1/3 and against the independent FEM/BEM discretisation; the stray field against
finite differences of the energy (exact, since the operator is symmetric); and
the minimiser runs on it."""
import math
import warnings

import numpy as np
import pytest

from oracle.micromag import CubeProblem
from oracle.minimise import minimise
import oracle.spacetrans as st
from oracle.spacetrans import ShellProblem
from test_oracle_pins import _box_potential

JS, A, K1 = 1.61, 7.7e-12, 4.3e6
LEVELS = ((4, 2, 4), (6, 3, 6), (8, 4, 8))          # (n, air cells, shell cells): one geometry, h halving


@pytest.fixture(scope="module")
def shells():
    return {lv: ShellProblem(lv[0], JS, A, K1, [0, 0, 1], lv[1], lv[2], cell=1.0) for lv in LEVELS}


def _sector_points(rng, c, R1, R2, count):
    """Random shell points, away from the sector boundaries and both faces."""
    pts = []
    while len(pts) < count:
        d = rng.uniform(-R2, R2, size=3)
        a = np.sort(np.abs(d))
        if R1 + 0.05 < a[2] < R2 - 0.05 and a[2] - a[1] > 0.05:
            pts.append(c + d)
    return np.array(pts)


def test_map_fixes_the_inner_face_and_sends_the_outer_face_to_infinity():
    c, R1, R2 = np.full(3, 2.0), 4.0, 8.0
    rng = np.random.default_rng(1)
    inner = c + np.array([[R1, 0.3, -1.2], [-0.7, -R1, 2.5], [1.1, 3.9, R1], [R1, R1, -R1]])
    assert np.allclose(st.shell_map(inner, c, R1, R2), inner, rtol=0, atol=1e-14)
    inside = c + rng.uniform(-R1, R1, size=(50, 3))
    assert np.array_equal(st.shell_map(inside, c, R1, R2), inside)
    # along any ray the max-norm radius grows monotonically and without bound towards R2
    d = rng.normal(size=3)
    d /= np.abs(d).max()
    rhos = np.linspace(R1, R2 - 1e-9, 400)
    rp = np.abs(st.shell_map(c + rhos[:, None] * d, c, R1, R2) - c).max(axis=1)
    assert np.all(np.diff(rp) > 0) and rp[-1] > 1e8
    # directions are kept: x' - c is a positive multiple of x - c
    pts = _sector_points(rng, c, R1, R2, 40)
    xp = st.shell_map(pts, c, R1, R2)
    cr = np.cross(xp - c, pts - c)
    assert np.abs(cr).max() <= 1e-12 * np.abs(xp - c).max() * np.abs(pts - c).max()
    assert np.all(np.sum((xp - c) * (pts - c), axis=1) > 0)


def test_jacobian_is_the_derivative_of_the_map():
    c, R1, R2 = np.array([1.0, 2.0, 1.5]), 3.0, 7.0
    rng = np.random.default_rng(2)
    pts = _sector_points(rng, c, R1, R2, 60)
    J, detJ = st.shell_jacobian(pts, c, R1, R2)
    h = 1e-6
    for p, x in enumerate(pts):
        fd = np.stack([(st.shell_map(x[None] + h * e, c, R1, R2)
                        - st.shell_map(x[None] - h * e, c, R1, R2))[0] / (2 * h) for e in np.eye(3)], axis=1)
        assert np.abs(fd - J[p]).max() <= 1e-6 * np.abs(J[p]).max()
    assert np.allclose(detJ, np.linalg.det(J), rtol=1e-12)
    assert np.all(detJ > 0)


def test_tensor_is_spd_with_determinant_det_J_and_identity_outside(shells):
    c, R1, R2 = np.zeros(3), 2.0, 5.0
    pts = _sector_points(np.random.default_rng(3), c, R1, R2, 50)
    M = st.shell_tensor(pts, c, R1, R2)
    _, detJ = st.shell_jacobian(pts, c, R1, R2)
    assert np.abs(M - np.transpose(M, (0, 2, 1))).max() <= 1e-14 * np.abs(M).max()
    assert np.all(np.linalg.eigvalsh(M) > 0)
    # det(|det J| J^-1 J^-T) = |det J|^3 / det J^2 = |det J|
    assert np.allclose(np.linalg.det(M), np.abs(detJ), rtol=1e-12)
    p = shells[LEVELS[1]]
    assert p.shell_tets.any() and not p.shell_tets.all()
    assert np.array_equal(p.tensor[~p.shell_tets], np.broadcast_to(np.eye(3), p.tensor[~p.shell_tets].shape))


def test_grid_stiffness_symmetry_kernel_and_patch_test(shells):
    p = shells[LEVELS[1]]
    K = p.Kgrid
    scale = np.abs(K.data).max()
    assert abs(K - K.T).max() <= 1e-14 * scale
    assert np.abs(K @ np.ones(K.shape[0])).max() <= 1e-12 * scale
    assert np.all(K.diagonal() > 0)
    # rows whose tetrahedra all carry M = I reproduce linear functions
    plain = np.ones(K.shape[0], dtype=bool)
    plain[np.unique(p.grid_tets[p.shell_tets])] = False
    x = p.grid_nodes.astype(np.float64)
    rho = np.max(np.abs(x - p.c), axis=1)
    rows = plain & (rho < p.R1)
    assert rows.sum() > 0
    for lin in (x[:, 0], x[:, 1] - 2.0 * x[:, 2], 3.0 * x[:, 2] + 0.5):
        assert np.abs((K @ lin)[rows]).max() <= 1e-12 * scale * np.abs(lin).max()


def _potential_errors(p):
    """Discrete potential of the uniformly z-magnetised magnet against the exact
    box potential, at every node not on the outer face, taken at its image x'."""
    x = p.grid_nodes.astype(np.float64)
    rho = np.max(np.abs(x - p.c), axis=1)
    ok = rho < p.R2
    m = np.zeros((p.mesh.N, 3))
    m[:, 2] = 1.0
    u = p.grid_potential(m)[ok]
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        ue = _box_potential(st.shell_map(x[ok], p.c, p.R1, p.R2), float(p.n))
    fin = np.isfinite(ue)                       # points on an edge line of the box: the formula's 0 * log 0
    e, sc = u[fin] - ue[fin], np.abs(ue[fin]).max()
    outside = rho[ok][fin] > p.n / 2.0
    far = np.abs(st.shell_map(x[ok], p.c, p.R1, p.R2) - p.c).max(axis=1)[fin] >= 4.0 * p.n
    return np.abs(e).max() / sc, math.sqrt(float(np.mean(e[outside] ** 2))) / sc, int(far.sum())


def test_potential_converges_to_the_box_solution_inside_and_outside(shells):
    errs = [_potential_errors(shells[lv]) for lv in LEVELS]
    mx = [e[0] for e in errs]
    rms = [e[1] for e in errs]
    assert mx[0] > mx[1] > mx[2] and mx[2] < 0.05
    assert rms[0] > rms[1] > rms[2] and rms[2] < 0.006
    assert all(e[2] > 0 for e in errs)                 # the comparison reaches 4 box sizes and beyond


def test_demag_factors_converge_to_one_third_and_to_the_fem_bem_values(shells):
    Ns, gaps = [], []
    for lv in LEVELS:
        p = shells[lv]
        N = []
        for d in range(3):
            m = np.zeros((p.mesh.N, 3))
            m[:, d] = 1.0
            N.append(p.evaluate(m, [0.0, 0.0, 0.0]).terms["d"] / (p.Kd * p.V.sum()))
        assert max(N) - min(N) < 2e-4                   # cubic symmetry up to the Kuhn split
        assert all(0 < v < 1 / 3 for v in N)
        q = CubeProblem(lv[0], JS, A, K1, [0, 0, 1], cell=1.0)
        m = np.zeros((q.mesh.N, 3))
        m[:, 2] = 1.0
        gaps.append(abs(N[2] - q.evaluate(m, [0.0, 0.0, 0.0]).terms["d"] / (q.Kd * q.V.sum())))
        Ns.append(N[2])
    err = [1 / 3 - v for v in Ns]
    assert err[0] > err[1] > err[2] and err[2] < 0.02
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 0.01


def test_stray_field_is_the_exact_energy_gradient():
    """The operator is symmetric, so -(Js/mu0) V_i h_i is dE/dm_i with no adjoint
    (central differences of the total energy on a small problem)."""
    p = ShellProblem(2, JS, A, K1, [0.2, 0.1, 1.0], 1, 2, cell=2e-9)
    rng = np.random.default_rng(4)
    m = rng.normal(size=(p.mesh.N, 3))
    m /= np.linalg.norm(m, axis=1)[:, None]
    h_ext = np.array([0.3, -0.2, 0.5])
    ev = p.evaluate(m, h_ext)
    dE = -(JS / (4e-7 * math.pi)) * p.V[:, None] * ev.h
    eps = 1e-6
    for i in (0, 5, 13, p.mesh.N - 1):
        for d in range(3):
            mp, mm = m.copy(), m.copy()
            mp[i, d] += eps
            mm[i, d] -= eps
            fd = (p.evaluate(mp, h_ext).E - p.evaluate(mm, h_ext).E) / (2 * eps)
            assert abs(fd - dE[i, d]) <= 1e-6 * np.abs(dE).max()


def test_minimiser_reaches_a_minimum_with_the_shell_boundary():
    p = ShellProblem(4, JS, A, K1, [0, 0, 1], 2, 4)
    m0 = np.zeros((p.mesh.N, 3))
    m0[:, 2] = 1.0
    m0[:, 0] = 0.3
    m0 /= np.linalg.norm(m0, axis=1)[:, None]
    res = minimise(p, m0, np.array([0.0, 0.0, -1.0]), tol=1e-6, max_iter=3000)
    assert res.status == 0 and res.iterations > 5 and res.torque < 1e-6
    assert np.allclose(np.linalg.norm(res.m, axis=1), 1.0, atol=1e-12)
    assert res.E < p.evaluate(m0, np.array([0.0, 0.0, -1.0])).E
