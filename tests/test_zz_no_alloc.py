"""The allocation-free evaluation entry point against the regular one.

lbm_evaluate_noalloc serves callers that must not allocate device memory while
they run -- a host application that reserves all of its GPU memory at start-up,
or a time-critical loop in which the CUDA allocator may not be touched.  It
keeps its intermediate vectors in one fixed device array inside the library.
Here it must give what lbm_evaluate gives (FP64 field, potentials and energy
terms, to the 1e-10 tolerance of the other FP64 parity tests) on two calls in a
row with different inputs, and reject meshes larger than its fixed array.
This file is collected near the end so that a run stopping at the first
failure has already run the other tests.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, m_random_sphere, tilted_axis

pytestmark = pytest.mark.gpu


def test_noalloc_evaluation_matches_lbm_evaluate():
    torch = pytest.importorskip("torch")
    from paper_1309_5796_gb300 import build
    build.build()
    stream = torch.cuda.current_stream()
    ctx = lbm.Context(0, stream=stream.cuda_stream)
    try:
        n = 7
        N = (n + 1) ** 3
        mesh = ctx.mesh_cube(2e-9, n)
        axis = tilted_axis(10.0, 0.4)
        opts = lbm.default_opts(lbm.LBM_FP64)
        for seed, h_ext in ((21, np.array([0.2, 0.0, -3.0])), (22, np.array([-1.0, 0.5, 2.0]))):
            m0 = m_random_sphere(N, seed)
            inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
            inst.set_material(JS_T, A_JM, K1_JM3, axis)
            inst.set_field(h_ext)
            inst.set_m(m0)
            res, h_ref, u_ref = inst.evaluate(opts)
            inst.destroy()
            d_m = torch.from_numpy(np.ascontiguousarray(m0)).to("cuda:0")
            d_h = torch.empty(3 * N, dtype=torch.float64, device="cuda:0")
            d_u = torch.empty(2 * N, dtype=torch.float64, device="cuda:0")
            d_e = torch.empty(5, dtype=torch.float64, device="cuda:0")
            ctx.evaluate_noalloc(mesh, JS_T, A_JM, K1_JM3, axis, h_ext, d_m.data_ptr(), d_h.data_ptr(),
                                 d_u.data_ptr(), d_e.data_ptr(), opts)
            torch.cuda.synchronize()
            h = d_h.cpu().numpy().reshape(N, 3)
            u = d_u.cpu().numpy().reshape(2, N)
            e = d_e.cpu().numpy()
            hs = np.abs(h_ref[0]).max()
            assert np.abs(h - h_ref[0]).max() <= 1e-10 * hs
            us = np.abs(u_ref[0]).max()
            assert np.abs(u - u_ref[0]).max() <= 1e-9 * us
            scale = np.abs(np.array(res[0]["energy"])).max()
            assert np.abs(e - np.array(res[0]["energy"])).max() <= 1e-10 * scale
        big = ctx.mesh_cube(2e-9, 25)
        with pytest.raises(lbm.LBMError):
            ctx.evaluate_noalloc(big, JS_T, A_JM, K1_JM3, axis, np.zeros(3), d_m.data_ptr())
        ctx.mesh_destroy(big)
        ctx.mesh_destroy(mesh)
    finally:
        ctx.close()
