"""The batched workload's mixed-precision minima meet the stop test of the exact
FP64 problem, not only that of the mixed path's own arithmetic.

64 instances on the 30^3-cell cube are minimised in LBM_MIXED_TC (FP32 phase,
then an FP64 phase whose potential solves stop at a 1e-10 relative residual),
and the final states are re-evaluated with plain FP64 solves (1e-13) and the
FP64 boundary matrix.  The FP64 phase stops at 0.9 of the requested torque
(1e-6), on its own field; the re-evaluated torque differs from it by the field
error of those solves (measured ~1e-10 on this workload), so every final state
keeps a 10 % margin against the requested 1e-6 in the exact problem: the bar
here is 0.9e-6 + 1e-9.  This file is collected last, so that a run that stops
at the first failure has already run every other test.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, batched_case

pytestmark = pytest.mark.gpu


def test_mixed_final_states_converged_in_the_fp64_problem():
    from paper_1309_5796_gb300 import build
    build.build()
    ctx = lbm.Context(0)
    try:
        insts = batched_case(30, 64, seed=4)
        axes = np.stack([i.axis for i in insts])
        fields = np.stack([i.h_ext for i in insts])
        mesh = ctx.mesh_cube(2e-9, 30)
        inst = ctx.instance_create(mesh, 64, lbm.LBM_MIXED_TC)
        inst.set_material(JS_T, A_JM, K1_JM3, axes)
        inst.set_field(fields)
        inst.set_m(np.stack([i.m0 for i in insts]))
        res = inst.minimise(lbm.default_opts(lbm.LBM_MIXED_TC))
        m = inst.get_m()
        inst.destroy()
        chk = ctx.instance_create(mesh, 64, lbm.LBM_FP64)
        chk.set_material(JS_T, A_JM, K1_JM3, axes)
        chk.set_field(fields)
        chk.set_m(m)
        r64, _, _ = chk.evaluate(lbm.default_opts(lbm.LBM_FP64), want_h=False, want_u=False)
        chk.destroy()
        ctx.mesh_destroy(mesh)
    finally:
        ctx.close()
    for a, b in zip(res, r64):
        assert a["status"] == lbm.LBM_OK and a["torque"] < 0.9e-6
        assert b["torque"] < 0.9e-6 + 1e-9
