"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: integer and index tables bit-exact; FP64 fields/energies to 1e-10
relative (potential solves are iterative to a 1e-13 residual on the device, a
direct LU in the oracle); FP64 trajectories m to 1e-10 over the first 50
iterations; final energies to 1e-6 relative; mixed precision to the stated
tolerances.
"""
import math

import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from oracle.bem import bem_matrix
from oracle.mesh import closed_form_counts, cube_mesh
from oracle.micromag import CubeProblem
from oracle.minimise import minimise as oracle_minimise
from synth.inputs import (A_JM, JS_T, K1_JM3, m_perturbed, m_random_sphere, single_fp64_case,
                          tilted_axis)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def _canon_tris(t):
    t = np.asarray(t, dtype=np.int64)
    r = np.argmin(t, axis=1)
    t = np.stack([t[np.arange(len(t)), (r + s) % 3] for s in range(3)], axis=1)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


@pytest.mark.parametrize("n", [1, 2, 5, 10, 30])
def test_mesh_tables_bit_exact(ctx, n):
    h = ctx.mesh_cube(2e-9, n)
    g = ctx.mesh_export(h)
    o = cube_mesh(n)
    c = closed_form_counts(n)
    info = ctx.mesh_info(h)
    assert info["N"] == c["N"] and info["nb"] == c["nb"] and info["nnz"] == c["nnz"]
    assert np.array_equal(g["tets"], o.tets)
    assert np.array_equal(g["rowptr"], o.ops.indptr)
    assert np.array_equal(g["col"], o.ops.indices)
    assert np.array_equal(g["kval"], o.ops.K)
    assert np.array_equal(g["gval"], o.ops.G)
    assert np.array_equal(g["gtval"], o.ops.Gt)
    assert np.array_equal(g["vol"], o.ops.V)
    assert np.array_equal(g["bnd"], o.bnd)
    assert np.array_equal(_canon_tris(g["tris"]), o.tris)
    ctx.mesh_destroy(h)


@pytest.mark.parametrize("n", [1, 2, 6, 10])
def test_bem_matrix_full(ctx, n):
    h = ctx.mesh_cube(2e-9, n)
    nb = ctx.mesh_info(h)["nb"]
    Bg = ctx.bem_rows(h, 0, nb)
    o = cube_mesh(n)
    Bo = bem_matrix(o.nodes, n, o.bnd, o.tris)
    assert np.abs(Bg - Bo).max() < 1e-12
    assert np.abs(Bg.sum(axis=1) + 1).max() < 1e-12
    ctx.mesh_destroy(h)


@pytest.mark.parametrize("n", [30, 80])
def test_bem_matrix_sampled_rows(ctx, n):
    """Full-size meshes: sampled rows (first, last, random) against the oracle."""
    h = ctx.mesh_cube(2e-9, n)
    nb = ctx.mesh_info(h)["nb"]
    rows = np.unique(np.r_[0, nb - 1, np.random.default_rng(7).integers(0, nb, 6)])
    o = cube_mesh(n)
    Bo = bem_matrix(o.nodes, n, o.bnd, o.tris, rows=rows, chunk=2)
    for k, r in enumerate(rows):
        Bg = ctx.bem_rows(h, int(r), 1)[0]
        assert np.abs(Bg - Bo[k]).max() < 1e-11
        assert abs(Bg.sum() + 1) < 1e-10
    ctx.mesh_destroy(h)


def _setup(ctx, n, B, prec, axes, fields, m0):
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    inst.set_m(m0)
    return mesh, inst


@pytest.mark.parametrize("prec,rtol", [(lbm.LBM_FP64, 1e-10), (lbm.LBM_MIXED, 2e-5)])
@pytest.mark.parametrize("n", [1, 3, 7])
def test_field_and_energy(ctx, n, prec, rtol):
    N = (n + 1) ** 3
    m0 = m_random_sphere(N, 11 + n)
    axis = tilted_axis(20.0, 0.3)
    h_ext = np.array([0.3, -0.7, 1.9])
    mesh, inst = _setup(ctx, n, 1, prec, axis, h_ext, m0)
    res, h, u = inst.evaluate(lbm.default_opts(prec))
    p = CubeProblem(n, JS_T, A_JM, K1_JM3, axis)
    ev = p.evaluate(m0, h_ext)
    hs = np.abs(ev.h).max()
    assert np.abs(h[0] - ev.h).max() <= rtol * hs
    us = np.abs(ev.u1 + ev.u2).max()
    assert np.abs((u[0, 0] + u[0, 1]) - (ev.u1 + ev.u2)).max() <= rtol * us * 10
    Eunit = p.Kd * p.cell ** 3 * N
    for k, key in enumerate(("ex", "an", "z", "d")):
        assert abs(res[0]["energy"][k] - ev.terms[key]) <= rtol * Eunit, key
    assert abs(res[0]["energy"][4] - ev.E) <= rtol * Eunit
    assert abs(res[0]["torque"] - ev.torque) <= rtol * hs
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_trajectory_fp64_first_50_iterations(ctx):
    """Sec. 2.2-2.3 iteration: m after k = 1, 5, 20, 50 accepted steps agrees
    with the oracle to 1e-10 (configuration: 20 nm cube, -6 T at 1 degree)."""
    case = single_fp64_case()
    p = CubeProblem(case.n, case.Js, case.A, case.K1, case.axis)
    checkpoints = (1, 5, 20, 50)
    ref = oracle_minimise(p, case.m0, case.h_ext, tol=1e-6, max_iter=50, record=checkpoints)
    traj = dict(ref.trajectory)
    mesh, inst = _setup(ctx, case.n, 1, lbm.LBM_FP64, case.axis, case.h_ext, case.m0)
    for k in checkpoints:
        inst.set_m(case.m0)
        r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=k))
        assert r[0]["iterations"] == k
        mg = inst.get_m()[0]
        assert np.abs(mg - traj[k]).max() < 1e-10, (k, np.abs(mg - traj[k]).max())
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_full_minimisation_fp64_config(ctx):
    """20 nm cube to max|m x h|/Js < 1e-6: final energy within 1e-6 relative,
    unit length preserved, stop test met."""
    case = single_fp64_case()
    p = CubeProblem(case.n, case.Js, case.A, case.K1, case.axis)
    ref = oracle_minimise(p, case.m0, case.h_ext, tol=1e-6, max_iter=20000)
    mesh, inst = _setup(ctx, case.n, 1, lbm.LBM_FP64, case.axis, case.h_ext, case.m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_FP64))[0]
    assert r["status"] == lbm.LBM_OK and r["torque"] < 1e-6
    ref_scale = max(abs(ref.E), p.Kd * (case.n * p.cell) ** 3)
    assert abs(r["energy"][4] - ref.E) / ref_scale < 1e-6
    m = inst.get_m()[0]
    assert np.abs(np.linalg.norm(m, axis=1) - 1).max() < 1e-12
    assert abs(r["iterations"] - ref.iterations) <= max(5, ref.iterations // 10)
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_full_minimisation_mixed_config(ctx):
    """Mixed precision (FP32 vectors, FP64 reductions): final energy within
    1e-6 relative of the FP64 oracle."""
    case = single_fp64_case()
    p = CubeProblem(case.n, case.Js, case.A, case.K1, case.axis)
    ref = oracle_minimise(p, case.m0, case.h_ext, tol=1e-6, max_iter=20000)
    mesh, inst = _setup(ctx, case.n, 1, lbm.LBM_MIXED, case.axis, case.h_ext, case.m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_MIXED))[0]
    ref_scale = max(abs(ref.E), p.Kd * (case.n * p.cell) ** 3)
    assert r["status"] == lbm.LBM_OK
    assert abs(r["energy"][4] - ref.E) / ref_scale < 1e-6
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_batch_equals_single(ctx):
    """A batch of 5 instances (different fields and axes) gives, per instance,
    the result of solving it alone (FP64)."""
    n, B = 4, 5
    N = (n + 1) ** 3
    rng = np.random.default_rng(3)
    axes = np.array([tilted_axis(5.0 * rng.random(), 6.28 * rng.random()) for _ in range(B)])
    fields = np.array([[0.0, 0.0, -8.0 * rng.random()] for _ in range(B)])
    m0 = np.stack([m_perturbed(N, 100 + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, B, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    inst.set_m(m0)
    rb = inst.minimise(lbm.default_opts(lbm.LBM_FP64))
    mb = inst.get_m()
    single = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    for b in range(B):
        single.set_material(JS_T, A_JM, K1_JM3, axes[b])
        single.set_field(fields[b])
        single.set_m(m0[b])
        rs = single.minimise(lbm.default_opts(lbm.LBM_FP64))[0]
        assert rs["status"] == rb[b]["status"] == lbm.LBM_OK
        assert abs(rs["energy"][4] - rb[b]["energy"][4]) <= 1e-9 * abs(rs["energy"][4])
        assert np.abs(single.get_m()[0] - mb[b]).max() < 1e-6
    single.destroy()
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_single_domain_switching_on_gpu(ctx):
    """Stoner-Wohlfarth check of the paper (Sec. 3.1): a 2 nm cube, field at 45
    degrees, demag off, reverses at the first step past H_K/2."""
    from oracle.micromag import MU0
    psi = math.radians(45.0)
    HK = 2 * K1_JM3 * MU0 / JS_T
    step = 0.02
    fields = -np.arange(round(HK / 2 * 0.97 / step) * step, HK / 2 * 1.03, step)
    mesh = ctx.mesh_cube(1e-9, 2)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, [0, 0, 1])
    inst.set_m(np.tile([0, 0, 1.0], (27, 1)))
    o = lbm.default_opts(lbm.LBM_FP64, tol=1e-8, demag=0)
    d = np.array([math.sin(psi), 0, math.cos(psi)])
    mpar, energy, res = inst.hysteresis(d, fields, o)
    mz = np.array([r["mean_m"][2] for r in res])
    k = np.nonzero(mz < 0)[0][0]
    assert abs(abs(fields[k]) - HK / 2) <= step + 1e-9
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_hysteresis_matches_oracle_small(ctx):
    """A short warm-started sweep on a 6^3-cell cube with demag: per-point
    energies within 1e-6 relative and the same switching point."""
    from oracle.minimise import hysteresis as oracle_hyst
    n = 6
    N = (n + 1) ** 3
    axis = tilted_axis(1.0, 0.7)
    fields = np.arange(4.0, -8.01, -1.0)
    p = CubeProblem(n, JS_T, A_JM, K1_JM3, axis)
    mpar_o, e_o, _ = oracle_hyst(p, np.tile([0, 0, 1.0], (N, 1)), [0, 0, 1], fields, tol=1e-6)
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, axis)
    inst.set_m(np.tile([0, 0, 1.0], (N, 1)))
    mpar, energy, res = inst.hysteresis([0, 0, 1], fields, lbm.default_opts(lbm.LBM_FP64))
    scale = p.Kd * (n * p.cell) ** 3
    assert np.abs(energy[:, 0] - e_o).max() / scale < 1e-6
    assert np.array_equal(np.sign(mpar[:, 0]), np.sign(mpar_o))
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_uniform_state_zero_exchange_on_gpu(ctx):
    n = 4
    N = (n + 1) ** 3
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, [0, 0, 1])
    inst.set_m(np.tile([0.6, 0.0, 0.8], (N, 1)))
    res, h, u = inst.evaluate(lbm.default_opts(lbm.LBM_FP64))
    assert res[0]["energy"][0] == 0.0
    inst.destroy()
    ctx.mesh_destroy(mesh)


def _golden(name):
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", name)))


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_sweep_config2_vs_oracle(ctx, prec):
    """40 nm cube, axis tilted 1 degree, +8 -> -8 T in 0.1 T steps (161 warm-started
    points): per-point energies within 1e-6 relative of the oracle's sweep and the
    same switching field (within one field step)."""
    from oracle.micromag import MU0
    from synth.inputs import sweep_case
    g = _golden("sweep_n20.json")
    c = sweep_case(20, seed=2)
    assert np.allclose(c["axis"], g["axis"], atol=0) and np.allclose(c["fields"], g["fields"], atol=0)
    mesh = ctx.mesh_cube(2e-9, 20)
    inst = ctx.instance_create(mesh, 1, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, c["axis"])
    inst.set_m(c["m0"])
    mpar, energy, res = inst.hysteresis(c["direction"], c["fields"], lbm.default_opts(prec))
    inst.destroy()
    ctx.mesh_destroy(mesh)
    assert all(r["status"] == lbm.LBM_OK for r in res)
    Kd = JS_T ** 2 / (2 * MU0)
    scale = np.maximum(np.abs(g["energy"]), Kd * (20 * 2e-9) ** 3)
    assert np.max(np.abs(energy[:, 0] - g["energy"]) / scale) < 1e-6
    f = np.array(c["fields"])
    def switch(mp):
        return [f[k] for k in range(1, len(f)) if np.sign(mp[k]) != np.sign(mp[k - 1])]
    sw_gpu, sw_ora = switch(mpar[:, 0]), switch(np.array(g["m_par"]))
    assert len(sw_gpu) == len(sw_ora) == 1
    assert abs(sw_gpu[0] - sw_ora[0]) <= 0.1 + 1e-9


@pytest.mark.parametrize("prec", [lbm.LBM_MIXED, lbm.LBM_MIXED_TC])
def test_batched_config4_vs_oracle(ctx, prec):
    """The benchmark's workload in its launch configuration (64 instances on the
    30^3-cell cube, mixed precision with SIMT or tensor-core BEM products): every
    instance converges and its energy is within 1e-6 relative of the oracle's
    (golden, written by the oracle)."""
    from oracle.micromag import MU0
    from synth.inputs import batched_case
    g = _golden("batched_n30.json")["results"]
    insts = batched_case(30, 64, seed=4)
    mesh = ctx.mesh_cube(2e-9, 30)
    inst = ctx.instance_create(mesh, 64, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, np.stack([i.axis for i in insts]))
    inst.set_field(np.stack([i.h_ext for i in insts]))
    inst.set_m(np.stack([i.m0 for i in insts]))
    res = inst.minimise(lbm.default_opts(prec))
    inst.destroy()
    ctx.mesh_destroy(mesh)
    Kd = JS_T ** 2 / (2 * MU0)
    for b, (r, o) in enumerate(zip(res, g)):
        assert r["status"] == lbm.LBM_OK and r["torque"] < 1e-6, b
        scale = max(abs(o["E"]), Kd * (30 * 2e-9) ** 3)
        assert abs(r["energy"][4] - o["E"]) / scale < 1e-6, (b, r["energy"][4], o["E"])


@pytest.mark.parametrize("n,B", [(3, 1), (7, 1), (6, 8)])
def test_fp64_solves_with_fp32_iterations_match_plain(ctx, n, B):
    """FP64 potential solves iterated in FP32 with the FP64 residual recomputed
    at every restart end on the same FP64 residual test (1e-13), so fields,
    potentials and energies equal those of plain FP64 PCG to 1e-10 and the
    oracle's to 1e-10."""
    N = (n + 1) ** 3
    axes = np.array([tilted_axis(20.0 + b, 0.3 * b) for b in range(B)])
    fields = np.array([[0.3, -0.7, 1.9 - 0.5 * b] for b in range(B)])
    m0 = np.stack([m_random_sphere(N, 70 + n + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    out = []
    for mixed_iter in (0, 1):
        inst = ctx.instance_create(mesh, B, lbm.LBM_FP64)
        inst.set_material(JS_T, A_JM, K1_JM3, axes)
        inst.set_field(fields)
        inst.set_m(m0)
        out.append(inst.evaluate(lbm.default_opts(lbm.LBM_FP64, cg_mixed_iter=mixed_iter)))
        inst.destroy()
    (r0, h0, u0), (r1, h1, u1) = out
    assert np.abs(h1 - h0).max() <= 1e-10 * np.abs(h0).max()
    assert np.abs(u1 - u0).max() <= 1e-9 * np.abs(u0).max()
    p = CubeProblem(n, JS_T, A_JM, K1_JM3, axes[0])
    ev = p.evaluate(m0[0], fields[0])
    assert np.abs(h1[0] - ev.h).max() <= 1e-10 * np.abs(ev.h).max()
    Eunit = p.Kd * p.cell ** 3 * N
    for a, b in zip(r0, r1):
        assert np.abs(np.array(a["energy"]) - np.array(b["energy"])).max() <= 1e-10 * Eunit
    ctx.mesh_destroy(mesh)


def test_mixed_polish_with_fp32_iterations_reaches_same_minima(ctx):
    """Mixed-precision minimisation: the FP64 phase with FP32-iteration solves
    and with plain FP64 PCG end at the same minima (energies within 1e-8)."""
    n, B = 8, 8
    N = (n + 1) ** 3
    rng = np.random.default_rng(9)
    axes = np.array([tilted_axis(5 * rng.random(), 6.3 * rng.random()) for _ in range(B)])
    fields = np.array([[0.0, 0.0, -8 * rng.random()] for _ in range(B)])
    m0 = np.stack([m_perturbed(N, 900 + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    res = []
    for mixed_iter in (0, 1):
        inst = ctx.instance_create(mesh, B, lbm.LBM_MIXED)
        inst.set_material(JS_T, A_JM, K1_JM3, axes)
        inst.set_field(fields)
        inst.set_m(m0)
        res.append(inst.minimise(lbm.default_opts(lbm.LBM_MIXED, cg_mixed_iter=mixed_iter)))
        inst.destroy()
    ctx.mesh_destroy(mesh)
    Kd = JS_T ** 2 / (2 * 4e-7 * math.pi)
    scale = Kd * (n * 2e-9) ** 3
    for a, b in zip(*res):
        assert a["status"] == b["status"] == lbm.LBM_OK
        assert abs(a["energy"][4] - b["energy"][4]) <= 1e-8 * max(abs(a["energy"][4]), scale)


def test_repeated_solve_is_bitwise_identical(ctx):
    """set_m restarts the potentials from zero: solving the same inputs twice
    gives the same bits (deterministic reductions, no carried-over state)."""
    n, B = 6, 4
    N = (n + 1) ** 3
    axes = np.array([tilted_axis(3.0 * b, 0.4 * b) for b in range(B)])
    fields = np.array([[0.0, 0.0, -2.5 * b] for b in range(B)])
    m0 = np.stack([m_perturbed(N, 1200 + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, B, lbm.LBM_MIXED)
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    out = []
    for _ in range(2):
        inst.set_m(m0)
        r = inst.minimise(lbm.default_opts(lbm.LBM_MIXED))
        out.append((r, inst.get_m()))
    assert np.array_equal(out[0][1], out[1][1])
    for a, b in zip(out[0][0], out[1][0]):
        assert a["energy"] == b["energy"] and a["iterations"] == b["iterations"]
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_stalled_fp32_phase_hands_over_to_fp64(ctx):
    """A switch tolerance the FP32 phase cannot reach: the phase gives up after
    stall_iters steps without a new smallest torque and the FP64 phase finishes
    at the FP64 answer."""
    n, B = 8, 4
    N = (n + 1) ** 3
    axes = np.array([tilted_axis(2.0 * b, 0.3 * b) for b in range(B)])
    fields = np.array([[0.0, 0.0, -1.5 * b] for b in range(B)])
    m0 = np.stack([m_perturbed(N, 1300 + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    res = {}
    for prec, kw in ((lbm.LBM_FP64, {}), (lbm.LBM_MIXED, dict(switch_tol=1e-12, stall_iters=40))):
        inst = ctx.instance_create(mesh, B, prec)
        inst.set_material(JS_T, A_JM, K1_JM3, axes)
        inst.set_field(fields)
        inst.set_m(m0)
        res[prec] = inst.minimise(lbm.default_opts(prec, **kw))
        inst.destroy()
    ctx.mesh_destroy(mesh)
    scale = JS_T ** 2 / (2 * 4e-7 * math.pi) * (n * 2e-9) ** 3
    for a, b in zip(res[lbm.LBM_FP64], res[lbm.LBM_MIXED]):
        assert b["status"] == lbm.LBM_OK and b["torque"] < 1e-6
        assert abs(a["energy"][4] - b["energy"][4]) <= 1e-6 * max(abs(a["energy"][4]), scale)
