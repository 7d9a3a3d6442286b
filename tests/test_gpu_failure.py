"""Failure paths on the GPU, in forms that fault, trap or hang nothing.

* A device wait that runs out: a test hook makes every grid barrier of the
  cooperative potential solve wait for one arrival more than the grid makes,
  with a 50 ms limit; the kernel gives up, sets the context's error word and
  returns, the call returns LBM_E_TIMEOUT, and the same context then solves
  correctly (field equal to the oracle's).
* The iteration limit: max_iter = 1 ends with LBM_E_NOT_CONVERGED after one step.
* A non-finite magnetisation injected on the host: the result is LBM_E_NAN
  (FP64 and mixed precision), and the context stays usable.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from oracle.micromag import CubeProblem
from synth.inputs import A_JM, JS_T, K1_JM3, m_random_sphere, single_fp64_case, tilted_axis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def test_device_wait_timeout_is_reported_and_context_survives(ctx):
    n = 10                       # FP64, one instance: the cooperative (grid-barrier) solve
    N = (n + 1) ** 3
    m0 = m_random_sphere(N, 41)
    axis = tilted_axis(10.0, 0.2)
    h_ext = np.array([0.1, 0.2, -1.0])
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, axis)
    inst.set_field(h_ext)
    inst.set_m(m0)
    ctx.set_wait_limit(0.05, unreachable=True)
    try:
        with pytest.raises(lbm.LBMError) as ei:
            inst.evaluate(lbm.default_opts(lbm.LBM_FP64))
        assert ei.value.code == lbm.LBM_E_TIMEOUT
    finally:
        ctx.set_wait_limit(0.0, unreachable=False)
    inst.set_m(m0)
    res, h, _ = inst.evaluate(lbm.default_opts(lbm.LBM_FP64))
    ev = CubeProblem(n, JS_T, A_JM, K1_JM3, axis).evaluate(m0, h_ext)
    assert res[0]["status"] == lbm.LBM_OK
    assert np.abs(h[0] - ev.h).max() <= 1e-10 * np.abs(ev.h).max()
    inst.destroy()
    ctx.mesh_destroy(mesh)


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_iteration_limit(ctx, prec):
    case = single_fp64_case()
    mesh = ctx.mesh_cube(2e-9, case.n)
    inst = ctx.instance_create(mesh, 1, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, case.axis)
    inst.set_field(case.h_ext)
    inst.set_m(case.m0)
    r = inst.minimise(lbm.default_opts(prec, max_iter=1))[0]
    assert r["status"] == lbm.LBM_E_NOT_CONVERGED
    assert 1 <= r["iterations"] <= 2
    inst.destroy()
    ctx.mesh_destroy(mesh)


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_nonfinite_magnetisation(ctx, prec):
    n, B = 4, 2
    N = (n + 1) ** 3
    m0 = np.stack([m_random_sphere(N, 60 + b) for b in range(B)])
    m0[1, 7] = [np.nan, 0.0, 1.0]
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, [0.0, 0.0, 1.0])
    inst.set_field(np.array([[0.0, 0.0, -1.0]] * B))
    inst.set_m(m0)
    r = inst.minimise(lbm.default_opts(prec, cg_max_iter=200))
    assert r[1]["status"] == lbm.LBM_E_NAN
    assert r[0]["status"] == lbm.LBM_OK          # the other instance of the batch is unaffected
    m0[1, 7] = [0.0, 0.0, 1.0]
    inst.set_m(m0)
    r = inst.minimise(lbm.default_opts(prec))
    assert all(x["status"] == lbm.LBM_OK for x in r)
    inst.destroy()
    ctx.mesh_destroy(mesh)
