"""Tensor-core (tcgen05, 3xTF32) BEM products against the SIMT FP32 path.

The 3xTF32 split (head/tail products, FP32 accumulation) keeps about FP32
accuracy, so fields and energies agree with the SIMT FP32 products to the
mixed-precision tolerance, and a batched mixed-precision minimisation reaches
the same minima (energies within 1e-6 relative)."""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, m_perturbed, m_random_sphere, tilted_axis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def _inst(ctx, mesh, B, prec, axes, fields, m0):
    i = ctx.instance_create(mesh, B, prec)
    i.set_material(JS_T, A_JM, K1_JM3, axes)
    i.set_field(fields)
    i.set_m(m0)
    return i


@pytest.mark.parametrize("n,B", [(6, 8), (10, 64), (13, 5)])
def test_tc_field_matches_simt(ctx, n, B):
    N = (n + 1) ** 3
    rng = np.random.default_rng(n)
    axes = np.array([tilted_axis(5 * rng.random(), 6.3 * rng.random()) for _ in range(B)])
    fields = np.array([[0.1, -0.2, -8 * rng.random()] for _ in range(B)])
    m0 = np.stack([m_random_sphere(N, 300 + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    a = _inst(ctx, mesh, B, lbm.LBM_MIXED, axes, fields, m0)
    t = _inst(ctx, mesh, B, lbm.LBM_MIXED_TC, axes, fields, m0)
    o = lbm.default_opts(lbm.LBM_MIXED)
    ra, ha, ua = a.evaluate(o)
    rt, ht, ut = t.evaluate(o)
    a.destroy()
    t.destroy()
    ctx.mesh_destroy(mesh)
    hs = np.abs(ha).max()
    assert np.abs(ht - ha).max() <= 2e-5 * hs
    for x, y in zip(ra, rt):
        assert abs(x["energy"][4] - y["energy"][4]) <= 2e-5 * (abs(x["energy"][4]) + 1e-20)


def test_tc_batched_minimisation(ctx):
    n, B = 8, 16
    N = (n + 1) ** 3
    rng = np.random.default_rng(5)
    axes = np.array([tilted_axis(5 * rng.random(), 6.3 * rng.random()) for _ in range(B)])
    fields = np.array([[0.0, 0.0, -8 * rng.random()] for _ in range(B)])
    m0 = np.stack([m_perturbed(N, 500 + b) for b in range(B)])
    mesh = ctx.mesh_cube(2e-9, n)
    a = _inst(ctx, mesh, B, lbm.LBM_FP64, axes, fields, m0)
    t = _inst(ctx, mesh, B, lbm.LBM_MIXED_TC, axes, fields, m0)
    ra = a.minimise(lbm.default_opts(lbm.LBM_FP64))
    rt = t.minimise(lbm.default_opts(lbm.LBM_MIXED_TC))
    a.destroy()
    t.destroy()
    ctx.mesh_destroy(mesh)
    for x, y in zip(ra, rt):
        assert x["status"] == y["status"] == lbm.LBM_OK
        assert abs(x["energy"][4] - y["energy"][4]) <= 1e-6 * abs(x["energy"][4])
