"""The allocation-free evaluation entry point against the regular one.

lbm_evaluate_noalloc serves callers that must not allocate device memory while
they run -- a host application that reserves all of its GPU memory at start-up,
or a time-critical loop in which the CUDA allocator may not be touched.  It
keeps its intermediate vectors in one fixed device array inside the library.
Here it must give what lbm_evaluate gives (FP64 field, potentials and energy
terms, to the 1e-10 tolerance of the other FP64 parity tests) on two calls
queued back to back on one stream with different inputs (no host
synchronisation between them, so the second reuses the shared array in stream
order), with the field and potential outputs omitted on a third call, and
reject meshes larger than its fixed array.  A device wait that runs out (made
to, by the context's test hook) shows up as NaN energies and a NaN first field
value, and the next call is correct again.  This file is collected near the
end so that a run stopping at the first failure has already run the other
tests.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, m_random_sphere, tilted_axis

pytestmark = pytest.mark.gpu


def _reference(ctx, mesh, axis, h_ext, m0, opts):
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, axis)
    inst.set_field(h_ext)
    inst.set_m(m0)
    res, h, u = inst.evaluate(opts)
    inst.destroy()
    return np.array(res[0]["energy"]), h[0], u[0]


def _close(e, h, u, ref):
    e_ref, h_ref, u_ref = ref
    assert np.abs(h - h_ref).max() <= 1e-10 * np.abs(h_ref).max()
    assert np.abs(u - u_ref).max() <= 1e-10 * np.abs(u_ref).max()
    assert np.abs(e - e_ref).max() <= 1e-10 * np.abs(e_ref).max()


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
        cases = [(21, np.array([0.2, 0.0, -3.0])), (22, np.array([-1.0, 0.5, 2.0]))]
        refs, outs = [], []
        for seed, h_ext in cases:
            m0 = m_random_sphere(N, seed)
            refs.append(_reference(ctx, mesh, axis, h_ext, m0, opts))
        torch.cuda.synchronize()
        for seed, h_ext in cases:                  # both calls queued, one synchronisation
            d_m = torch.from_numpy(np.ascontiguousarray(m_random_sphere(N, seed))).to("cuda:0")
            d_h = torch.empty(3 * N, dtype=torch.float64, device="cuda:0")
            d_u = torch.empty(2 * N, dtype=torch.float64, device="cuda:0")
            d_e = torch.empty(5, dtype=torch.float64, device="cuda:0")
            ctx.evaluate_noalloc(mesh, JS_T, A_JM, K1_JM3, axis, h_ext, d_m.data_ptr(), d_h.data_ptr(),
                                 d_u.data_ptr(), d_e.data_ptr(), opts)
            outs.append((d_m, d_h, d_u, d_e))
        torch.cuda.synchronize()
        for (d_m, d_h, d_u, d_e), ref in zip(outs, refs):
            _close(d_e.cpu().numpy(), d_h.cpu().numpy().reshape(N, 3), d_u.cpu().numpy().reshape(2, N), ref)
        # energies only (no field or potential output)
        d_e = torch.full((5,), -1.0, dtype=torch.float64, device="cuda:0")
        ctx.evaluate_noalloc(mesh, JS_T, A_JM, K1_JM3, axis, cases[0][1], outs[0][0].data_ptr(), 0, 0,
                             d_e.data_ptr(), opts)
        torch.cuda.synchronize()
        e = d_e.cpu().numpy()
        assert np.abs(e - refs[0][0]).max() <= 1e-10 * np.abs(refs[0][0]).max()
        big = ctx.mesh_cube(2e-9, 25)
        with pytest.raises(lbm.LBMError):
            ctx.evaluate_noalloc(big, JS_T, A_JM, K1_JM3, axis, np.zeros(3), outs[0][0].data_ptr())
        ctx.mesh_destroy(big)
        ctx.mesh_destroy(mesh)
    finally:
        ctx.close()


def test_noalloc_failed_wait_is_visible():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.current_stream()
    ctx = lbm.Context(0, stream=stream.cuda_stream)
    try:
        n = 10                                     # large enough for the grid-barrier solve
        N = (n + 1) ** 3
        mesh = ctx.mesh_cube(2e-9, n)
        axis = tilted_axis(4.0, 1.1)
        h_ext = np.array([0.0, 0.3, -2.0])
        m0 = m_random_sphere(N, 31)
        opts = lbm.default_opts(lbm.LBM_FP64)
        ref = _reference(ctx, mesh, axis, h_ext, m0, opts)
        d_m = torch.from_numpy(np.ascontiguousarray(m0)).to("cuda:0")
        d_h = torch.empty(3 * N, dtype=torch.float64, device="cuda:0")
        d_u = torch.empty(2 * N, dtype=torch.float64, device="cuda:0")
        d_e = torch.empty(5, dtype=torch.float64, device="cuda:0")
        ctx.set_wait_limit(0.05, unreachable=True)
        try:
            ctx.evaluate_noalloc(mesh, JS_T, A_JM, K1_JM3, axis, h_ext, d_m.data_ptr(), d_h.data_ptr(),
                                 d_u.data_ptr(), d_e.data_ptr(), opts)
            torch.cuda.synchronize()
        finally:
            ctx.set_wait_limit(0.0, unreachable=False)
        assert np.all(np.isnan(d_e.cpu().numpy())) and np.isnan(d_h[0].item())
        ctx.evaluate_noalloc(mesh, JS_T, A_JM, K1_JM3, axis, h_ext, d_m.data_ptr(), d_h.data_ptr(),
                             d_u.data_ptr(), d_e.data_ptr(), opts)
        torch.cuda.synchronize()
        _close(d_e.cpu().numpy(), d_h.cpu().numpy().reshape(N, 3), d_u.cpu().numpy().reshape(2, N), ref)
        ctx.mesh_destroy(mesh)
    finally:
        ctx.close()
