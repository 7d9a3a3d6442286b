"""Captured CUDA graphs of the iteration chunks.

With use_graphs = 1 every chunk of check_every iterations after the first is
captured once as a CUDA graph and replayed; the same kernels run in the same
order, so a minimisation gives the same bits with and without graphs.  Checked
for a plain FP64 solve (one instance), a mixed-precision batch of 16 (cluster
potential solves; FP32 phase then FP64 phase) and a mixed batch of 64 with
tensor-core BEM products; and the graphs were really used (replays counted,
no capture refused)."""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, batched_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec,n,B", [(lbm.LBM_FP64, 8, 1), (lbm.LBM_MIXED, 10, 16), (lbm.LBM_MIXED_TC, 12, 64)])
def test_graphs_give_the_same_bits(ctx, prec, n, B):
    insts = batched_case(n, B, seed=9)
    mesh = ctx.mesh_cube(2e-9, n)
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, np.stack([i.axis for i in insts]))
    inst.set_field(np.stack([i.h_ext for i in insts]))
    out = []
    for graphs in (0, 1):
        inst.set_m(np.stack([i.m0 for i in insts]))
        g0 = ctx.graph_stats()
        r = inst.minimise(lbm.default_opts(prec, use_graphs=graphs))
        g1 = ctx.graph_stats()
        out.append((r, inst.get_m(), {k: g1[k] - g0[k] for k in g1}))
    inst.destroy()
    ctx.mesh_destroy(mesh)
    (ra, ma, ga), (rb, mb, gb) = out
    assert ga["replays"] == 0 and ga["captures"] == 0
    assert gb["replays"] > 0 and gb["refused"] == 0
    assert np.array_equal(ma, mb)
    for a, b in zip(ra, rb):
        assert a["status"] == b["status"] == lbm.LBM_OK
        assert a["energy"] == b["energy"] and a["iterations"] == b["iterations"]
        assert a["evaluations"] == b["evaluations"]
