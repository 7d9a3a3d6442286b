"""Step-rule variants and LaBonte's method on the GPU against the oracle.

BB1-only, BB2-only and BB1/BB2 alternation (Sec. 2.3): FP64 trajectories to
1e-10 over the first 50 iterations and final energies to 1e-6 relative.
LaBonte's rotate-to-field iteration with relaxation (Sec. 1.2), all nodes at
once: FP64 trajectory to 1e-10 and, on a single-domain particle, the same
equilibrium as the oracle.
"""
import math

import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from oracle.micromag import MU0, CubeProblem
from oracle.minimise import StepRule, labonte
from oracle.minimise import minimise as oracle_minimise
from synth.inputs import A_JM, JS_T, K1_JM3, single_fp64_case

pytestmark = pytest.mark.gpu

RULES = {1: "bb1", 2: "bb2", 3: "alternate"}


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def _inst(ctx, mesh, axis, h, m0):
    i = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    i.set_material(JS_T, A_JM, K1_JM3, axis)
    i.set_field(h)
    i.set_m(m0)
    return i


@pytest.mark.parametrize("rule", [1, 2, 3])
def test_bb_rule_trajectory_and_minimum(ctx, rule):
    case = single_fp64_case(n=6)
    p = CubeProblem(case.n, case.Js, case.A, case.K1, case.axis)
    checkpoints = (1, 5, 20, 50)
    sr = StepRule(bb=RULES[rule])
    ref = oracle_minimise(p, case.m0, case.h_ext, tol=1e-6, max_iter=50, record=checkpoints, rule=sr)
    traj = dict(ref.trajectory)
    full = oracle_minimise(p, case.m0, case.h_ext, tol=1e-6, rule=sr)
    mesh = ctx.mesh_cube(2e-9, case.n)
    inst = _inst(ctx, mesh, case.axis, case.h_ext, case.m0)
    for k in checkpoints:
        inst.set_m(case.m0)
        r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=k, bb_rule=rule))
        assert r[0]["iterations"] == k
        assert np.abs(inst.get_m()[0] - traj[k]).max() < 1e-10, (rule, k)
    inst.set_m(case.m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, bb_rule=rule))[0]
    assert r["status"] == lbm.LBM_OK
    scale = max(abs(full.E), p.Kd * (case.n * p.cell) ** 3)
    assert abs(r["energy"][4] - full.E) / scale < 1e-6
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_labonte_trajectory(ctx):
    case = single_fp64_case(n=5)
    p = CubeProblem(case.n, case.Js, case.A, case.K1, case.axis)
    checkpoints = (1, 4, 12, 30)
    ref = labonte(p, case.m0, case.h_ext, omega=0.1, max_iter=30, record=checkpoints)
    traj = dict(ref.trajectory)
    mesh = ctx.mesh_cube(2e-9, case.n)
    inst = _inst(ctx, mesh, case.axis, case.h_ext, case.m0)
    for k in checkpoints:
        inst.set_m(case.m0)
        r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=k, method=1, omega=0.1))
        assert r[0]["iterations"] == k and r[0]["line_searches"] == 0
        assert np.abs(inst.get_m()[0] - traj[k]).max() < 1e-10, k
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_labonte_single_domain_equilibrium(ctx):
    p = CubeProblem(2, JS_T, A_JM, K1_JM3, np.array([0.0, 0.0, 1.0]), cell=1e-9, demag=False)
    HK = 2 * K1_JM3 * MU0 / JS_T
    psi = math.radians(150.0)
    h = 0.8 * HK * np.array([math.sin(psi), 0.0, math.cos(psi)])
    m0 = np.tile([0.0, 0.0, 1.0], (p.mesh.N, 1))
    ref = labonte(p, m0, h, omega=0.1, tol=1e-9, max_iter=20000)
    mesh = ctx.mesh_cube(1e-9, 2)
    inst = _inst(ctx, mesh, [0.0, 0.0, 1.0], h, m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, method=1, omega=0.1, tol=1e-9, demag=0))[0]
    assert r["status"] == lbm.LBM_OK
    assert abs(r["iterations"] - ref.iterations) <= 2
    mm = np.array(r["mean_m"])
    assert abs(math.atan2(mm[0], mm[2]) - math.atan2(*(p.mean_m(ref.m)[[0, 2]]))) < 1e-8
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_invalid_method_options_rejected(ctx):
    mesh = ctx.mesh_cube(2e-9, 2)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    for kw in (dict(bb_rule=4), dict(method=2), dict(method=1, omega=0.0), dict(method=1, omega=2.5)):
        with pytest.raises(lbm.LBMError):
            inst.minimise(lbm.default_opts(lbm.LBM_FP64, **kw))
    inst.destroy()
    ctx.mesh_destroy(mesh)
