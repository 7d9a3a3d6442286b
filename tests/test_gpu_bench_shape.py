"""Element-wise parity at the benchmark's launch shape, and the paper's stop test.

The benchmark runs 64 instances on the 30^3-cell cube: potential solves of
128 systems at once (forward and adjoint chains), the BEM products as batched
products (FP64 SIMT, FP32 SIMT or tensor cores), the field kernel over 64
instances.  Here one field evaluation in that shape is compared with the FP64
oracle, field and potential element by element and every energy term, for
instances 0, 31 and 63 (random magnetisation directions, the benchmark's
fields and easy axes): 2e-5 of the largest value in mixed precision, 1e-10 in
FP64.  Also the paper's stop test sum|g|^2 < tol_g (Sec. 3.1) on the GPU
against the oracle's trajectory.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from oracle.micromag import CubeProblem
from oracle.minimise import minimise as oracle_minimise
from synth.inputs import A_JM, JS_T, K1_JM3, batched_case, m_random_sphere, single_fp64_case

pytestmark = pytest.mark.gpu

N_CELLS, BATCH = 30, 64
CHECKED = (0, 31, 63)


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def oracle_fields():
    """The oracle's evaluation of the checked instances (one problem set-up,
    the easy axis switched per instance)."""
    insts = batched_case(N_CELLS, BATCH, seed=4)
    N = (N_CELLS + 1) ** 3
    m0 = np.stack([m_random_sphere(N, 500 + b) for b in range(BATCH)])
    p = CubeProblem(N_CELLS, JS_T, A_JM, K1_JM3, insts[0].axis)
    out = {}
    for b in CHECKED:
        p.axis = np.asarray(insts[b].axis, float) / np.linalg.norm(insts[b].axis)
        out[b] = p.evaluate(m0[b], insts[b].h_ext)
    return insts, m0, out, p


@pytest.mark.parametrize("prec,rtol", [(lbm.LBM_MIXED, 2e-5), (lbm.LBM_MIXED_TC, 2e-5), (lbm.LBM_FP64, 1e-10)])
def test_bench_shape_field_parity(ctx, oracle_fields, prec, rtol):
    insts, m0, ref, p = oracle_fields
    N = (N_CELLS + 1) ** 3
    mesh = ctx.mesh_cube(2e-9, N_CELLS)
    inst = ctx.instance_create(mesh, BATCH, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, np.stack([i.axis for i in insts]))
    inst.set_field(np.stack([i.h_ext for i in insts]))
    inst.set_m(m0)
    res, h, u = inst.evaluate(lbm.default_opts(prec))
    inst.destroy()
    ctx.mesh_destroy(mesh)
    Eunit = p.Kd * p.cell ** 3 * N
    for b in CHECKED:
        ev = ref[b]
        hs = np.abs(ev.h).max()
        assert np.abs(h[b] - ev.h).max() <= rtol * hs, (b, np.abs(h[b] - ev.h).max() / hs)
        uo = ev.u1 + ev.u2
        us = np.abs(uo).max()
        assert np.abs((u[b, 0] + u[b, 1]) - uo).max() <= rtol * us * 10, b
        for k, key in enumerate(("ex", "an", "z", "d")):
            assert abs(res[b]["energy"][k] - ev.terms[key]) <= rtol * Eunit, (b, key)
        assert abs(res[b]["energy"][4] - ev.E) <= rtol * Eunit, b
        assert abs(res[b]["torque"] - ev.torque) <= rtol * hs, b


def _gg(p, m, h):
    ev = p.evaluate(m, h)
    g = ev.grad - np.sum(m * ev.grad, axis=1, keepdims=True) * m
    return float(np.sum(g * g))


def test_grad_tol_stop_on_gpu(ctx):
    """The paper's stop test sum|g|^2 < tol_g (Sec. 3.1) in FP64: the GPU stops
    at the oracle's iterate (chosen within the first 50 steps, where the
    trajectories agree to 1e-10) with the oracle's m to 1e-10."""
    case = single_fp64_case()
    p = CubeProblem(case.n, case.Js, case.A, case.K1, case.axis)
    K = 50
    full = oracle_minimise(p, case.m0, case.h_ext, tol=0.0, max_iter=K, record=range(K + 1))
    gg = [_gg(p, m, case.h_ext) for _, m in full.trajectory]
    # the last new minimum of sum|g|^2 (by a margin) within the first K steps
    k = max(j for j in range(1, len(gg)) if gg[j] < 0.9 * min(gg[:j]))
    G = 0.5 * (gg[k] + min(gg[:k]))
    ref = oracle_minimise(p, case.m0, case.h_ext, tol=1e-30, grad_tol=G)
    assert ref.status == 0 and ref.iterations == k
    mesh = ctx.mesh_cube(2e-9, case.n)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, case.axis)
    inst.set_field(case.h_ext)
    inst.set_m(case.m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, tol=1e-30, grad_tol=G))[0]
    mg = inst.get_m()[0]
    inst.destroy()
    ctx.mesh_destroy(mesh)
    assert r["status"] == lbm.LBM_OK and r["iterations"] == k and r["gg"] < G
    assert np.abs(mg - ref.m).max() < 1e-10
