"""Continuous-batching server (config 5 workload pattern) on the GPU.

A request gives the same result alone and in a mix of concurrent requests of
other cube sizes (each instance's arithmetic and reduction order is independent
of what else is in its batch), and the same result as the batch API.
"""

import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, m_perturbed, tilted_axis

pytestmark = pytest.mark.gpu


def _req(n, seed, hz, tilt):
    N = (n + 1) ** 3
    return dict(n=n, cell_m=2e-9, Js=JS_T, A=A_JM, K1=K1_JM3, axis=tilted_axis(tilt, 0.3 * seed),
                h=np.array([0.0, 0.0, hz]), m0=m_perturbed(N, seed))


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def test_alone_and_in_the_mix(ctx):
    target = _req(8, 11, -5.0, 3.0)
    others = [_req(n, 20 + k, -8.0 + 1.3 * k, 1.0 + k) for k, n in enumerate((4, 6, 8, 8, 10, 5, 7))]
    N = (target["n"] + 1) ** 3
    ctx.serve_start(slots=4, chunk=4)
    try:
        t0 = ctx.submit(**target)
        alone, m_alone = ctx.wait(t0, N, timeout_s=300)
        tickets = [ctx.submit(**r) for r in others[:3]]
        t1 = ctx.submit(**target)
        tickets += [ctx.submit(**r) for r in others[3:]]
        mix, m_mix = ctx.wait(t1, N, timeout_s=300)
        rest = [ctx.wait(t, None, timeout_s=300)[0] for t in tickets]
        stats = ctx.serve_stats()
    finally:
        ctx.serve_stop()
    assert alone["status"] == lbm.LBM_OK and alone["torque"] < 1e-6
    assert all(r["status"] == lbm.LBM_OK and r["torque"] < 1e-6 for r in rest)
    # same arithmetic alone and in the mix
    assert mix["energy"][4] == alone["energy"][4]
    assert np.array_equal(m_mix, m_alone)
    assert stats["completed"] == 2 + len(others) and stats["pending"] == 0
    assert stats["groups"] >= 4
    # the batch API on the same problem (one instance): same minimum
    mesh = ctx.mesh_cube(2e-9, target["n"])
    inst = ctx.instance_create(mesh, 1, lbm.LBM_MIXED)
    inst.set_material(JS_T, A_JM, K1_JM3, target["axis"])
    inst.set_field(target["h"])
    inst.set_m(target["m0"])
    r = inst.minimise(lbm.default_opts(lbm.LBM_MIXED))[0]
    inst.destroy()
    ctx.mesh_destroy(mesh)
    assert r["status"] == lbm.LBM_OK
    scale = max(abs(r["energy"][4]), 1.0e-20)
    assert abs(r["energy"][4] - alone["energy"][4]) / scale < 1e-6


def test_fp64_requests_and_latency(ctx):
    reqs = [_req(n, 40 + n, -6.0, 2.0) for n in (3, 5, 6)]
    ctx.serve_start(slots=2, chunk=8)
    try:
        ts = [ctx.submit(**r, precision=lbm.LBM_FP64) for r in reqs]
        res = [ctx.wait(t, None, timeout_s=300)[0] for t in ts]
        pending = ctx.poll(ctx.submit(**reqs[0]))
    finally:
        ctx.serve_stop()
    assert all(r["status"] == lbm.LBM_OK and r["torque"] < 1e-6 for r in res)
    assert all(r["wall_ms"] > 0 for r in res)
    assert pending is None or pending[0]["status"] == lbm.LBM_OK


def test_size_groups_overlap_on_the_device(ctx):
    """Requests of three cube sizes served together: the serving loop's device
    trace (CUDA events on each size group's stream) has chunks of different
    groups whose intervals intersect, i.e. their kernels ran concurrently."""
    from synth.inputs import m_perturbed, tilted_axis
    ctx.serve_start(slots=16, chunk=8)
    try:
        tickets = []
        for k, n in enumerate((10, 14, 18) * 3):
            N = (n + 1) ** 3
            tickets.append(ctx.submit(n, 2e-9, JS_T, A_JM, K1_JM3, tilted_axis(2.0 + k, 0.3 * k),
                                      np.array([0.0, 0.0, -1.0 - 0.4 * k]), m_perturbed(N, 4000 + k)))
        res = [ctx.wait(t, None, timeout_s=600)[0] for t in tickets]
        tr = ctx.serve_trace()
    finally:
        ctx.serve_stop()
    assert all(r["status"] == lbm.LBM_OK for r in res)
    sizes = sorted(set(tr[:, 0].astype(int)))
    assert len(sizes) == 3
    overlaps = 0
    for i in range(len(tr)):
        for j in range(i + 1, len(tr)):
            if tr[i, 0] != tr[j, 0] and max(tr[i, 1], tr[j, 1]) < min(tr[i, 2], tr[j, 2]):
                overlaps += 1
    assert overlaps > 0
