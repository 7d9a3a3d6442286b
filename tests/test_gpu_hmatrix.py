"""The hierarchical (H-matrix) boundary operator on the device (Sec. 3.1).

lbm_mesh_hmatrix builds B_H on the host, uploads it with its transpose, and the
BEM products of the mesh then run in the two passes of the packed layout.
Checked here through the C ABI:
  * the products y = B_H x and y = B_H^T x (lbm_bem_apply) against the oracle's
    dense B within (eps + the vector precision) |B|_F |x|, column by column, and
    against the oracle's own H-matrix of the same tolerance within twice that;
    the dense operator again after eps = 0;
  * an FP64 field evaluation with B_H (eps 1e-10) equals the dense one;
  * the benchmark's workload (64 instances, 30^3 cells, mixed precision)
    minimised with B_H at eps 1e-8: every instance converges and its energy is
    within 1e-6 relative of the oracle's (golden, dense B).
"""
import json
import os

import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
import oracle.hmatrix as hm
from oracle.bem import bem_matrix
from oracle.mesh import cube_mesh
from synth.inputs import A_JM, JS_T, K1_JM3, batched_case, m_random_sphere, tilted_axis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cube12():
    n = 12
    o = cube_mesh(n)
    B = bem_matrix(o.nodes, n, o.bnd, o.tris)
    return n, o, B


@pytest.mark.parametrize("prec,fp", [(lbm.LBM_FP64, 1e-13), (lbm.LBM_MIXED, 1e-6)])
@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_hmatrix_products(ctx, cube12, eps, prec, fp):
    n, o, B = cube12
    nb = B.shape[0]
    x = np.random.default_rng(5).normal(size=(nb, 3))
    mesh = ctx.mesh_cube(2e-9, n)
    info = ctx.mesh_hmatrix(mesh, eps, eta=2.0, n_min=16)
    assert info["dense"] == nb * nb and 0 < info["stored"] < nb * nb
    y, yt = ctx.bem_apply(mesh, x, prec)
    nB = np.linalg.norm(B)
    for k in range(x.shape[1]):
        bound = (eps + fp) * nB * np.linalg.norm(x[:, k])
        assert np.linalg.norm(y[:, k] - B @ x[:, k]) <= bound, (k, np.linalg.norm(y[:, k] - B @ x[:, k]) / bound)
        assert np.linalg.norm(yt[:, k] - B.T @ x[:, k]) <= bound
    # the oracle's H-matrix of the same tolerance (another construction of B_H)
    Ho = hm.build_hmatrix(hm.dense_blocks(B), o.nodes, o.bnd, o.tris, eps=eps, eta=2.0, n_min=16)
    yo, yto = Ho @ x, Ho.T @ x
    for k in range(x.shape[1]):
        bound = 2 * (eps + fp) * nB * np.linalg.norm(x[:, k])
        assert np.linalg.norm(y[:, k] - yo[:, k]) <= bound
        assert np.linalg.norm(yt[:, k] - yto[:, k]) <= bound
    # back to the dense matrix
    ctx.mesh_hmatrix(mesh, 0.0)
    y0, yt0 = ctx.bem_apply(mesh, x, lbm.LBM_FP64)
    assert np.abs(y0 - B @ x).max() <= 1e-12 * np.abs(B @ x).max()
    assert np.abs(yt0 - B.T @ x).max() <= 1e-12 * np.abs(B.T @ x).max()
    ctx.mesh_destroy(mesh)


def test_hmatrix_evaluation_equals_dense(ctx):
    """An FP64 evaluation (field, energies) with B_H at eps 1e-10 is the dense
    one to 1e-8 of the largest field value."""
    n = 10
    N = (n + 1) ** 3
    m0 = m_random_sphere(N, 77)
    axis = tilted_axis(15.0, 0.5)
    h_ext = np.array([0.2, -0.1, -1.0])
    mesh = ctx.mesh_cube(2e-9, n)
    out = []
    for eps in (0.0, 1e-10):
        ctx.mesh_hmatrix(mesh, eps)
        inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
        inst.set_material(JS_T, A_JM, K1_JM3, axis)
        inst.set_field(h_ext)
        inst.set_m(m0)
        out.append(inst.evaluate(lbm.default_opts(lbm.LBM_FP64)))
        inst.destroy()
    (r0, h0, _), (r1, h1, _) = out
    assert np.abs(h1 - h0).max() <= 1e-8 * np.abs(h0).max()
    scale = JS_T ** 2 / (2 * 4e-7 * np.pi) * (n * 2e-9) ** 3
    assert abs(r1[0]["energy"][4] - r0[0]["energy"][4]) <= 1e-8 * scale
    ctx.mesh_destroy(mesh)


def test_hmatrix_batched_minimisation(ctx):
    """The benchmark's workload with B_H (eps 1e-8, 39 % of the dense entries):
    every instance converges and matches the oracle's energy (dense B) to 1e-6."""
    from oracle.micromag import MU0
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "batched_n30.json")))["results"]
    insts = batched_case(30, 64, seed=4)
    mesh = ctx.mesh_cube(2e-9, 30)
    info = ctx.mesh_hmatrix(mesh, 1e-8)
    assert info["fraction"] < 0.5
    inst = ctx.instance_create(mesh, 64, lbm.LBM_MIXED)
    inst.set_material(JS_T, A_JM, K1_JM3, np.stack([i.axis for i in insts]))
    inst.set_field(np.stack([i.h_ext for i in insts]))
    inst.set_m(np.stack([i.m0 for i in insts]))
    res = inst.minimise(lbm.default_opts(lbm.LBM_MIXED))
    inst.destroy()
    ctx.mesh_destroy(mesh)
    Kd = JS_T ** 2 / (2 * MU0)
    for b, (r, o) in enumerate(zip(res, g)):
        assert r["status"] == lbm.LBM_OK and r["torque"] < 1e-6, b
        scale = max(abs(o["E"]), Kd * (30 * 2e-9) ** 3)
        assert abs(r["energy"][4] - o["E"]) / scale < 1e-6, (b, r["energy"][4], o["E"])
