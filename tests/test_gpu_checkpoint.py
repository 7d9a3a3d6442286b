"""Checkpoint and resume of an instance batch (lbm_get_state / lbm_set_state and
lbm_solve_opts.resume).

A minimisation stopped by the iteration limit, saved, restored into a fresh
instance and resumed gives the same bits as one uninterrupted run: the same
magnetisation, energies, iteration and evaluation counts.  Converged
instances stay done; states of another batch size are refused; mixed
precision refuses resume.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from synth.inputs import A_JM, JS_T, K1_JM3, m_perturbed, single_fp64_case, tilted_axis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def _batch(ctx, mesh, B, n, prec=lbm.LBM_FP64):
    N = (n + 1) ** 3
    inst = ctx.instance_create(mesh, B, prec)
    axes = np.array([tilted_axis(1.0 + 2.0 * b, 0.5 * b) for b in range(B)])
    fields = np.array([[0.1 * b, 0.0, -5.0 - 0.4 * b] for b in range(B)])
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    m0 = np.stack([m_perturbed(N, 70 + b) for b in range(B)])
    inst.set_m(m0)
    return inst


@pytest.mark.parametrize("B,k", [(1, 25), (4, 20), (16, 37)])
def test_resume_gives_the_uninterrupted_bits(ctx, B, k):
    n = 8
    mesh = ctx.mesh_cube(2e-9, n)
    full = _batch(ctx, mesh, B, n)
    r_full = full.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=3000))
    m_full = full.get_m()
    full.destroy()

    part = _batch(ctx, mesh, B, n)
    r_part = part.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=k))
    assert all(r["iterations"] <= k for r in r_part)
    state = part.get_state()
    part.destroy()

    fresh = ctx.instance_create(mesh, B, lbm.LBM_FP64)   # constants, materials and m from the state
    fresh.set_state(state)
    r_res = fresh.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=3000, resume=1))
    m_res = fresh.get_m()
    assert fresh.get_state() != state
    fresh.destroy()
    ctx.mesh_destroy(mesh)
    assert np.array_equal(m_res, m_full)
    for a, b in zip(r_full, r_res):
        assert a["status"] == b["status"] == lbm.LBM_OK
        assert a["energy"] == b["energy"]
        assert (a["iterations"], a["evaluations"], a["line_searches"]) == \
               (b["iterations"], b["evaluations"], b["line_searches"])
        assert (a["cg_iters1"], a["cg_iters2"]) == (b["cg_iters1"], b["cg_iters2"])


def test_converged_instances_stay_done(ctx):
    """Resuming a converged batch changes nothing."""
    case = single_fp64_case()
    mesh = ctx.mesh_cube(2e-9, case.n)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, case.axis)
    inst.set_field(case.h_ext)
    inst.set_m(case.m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_FP64))[0]
    assert r["status"] == lbm.LBM_OK
    m = inst.get_m()
    r2 = inst.minimise(lbm.default_opts(lbm.LBM_FP64, resume=1))[0]
    assert np.array_equal(inst.get_m(), m)
    assert r2["iterations"] == r["iterations"] and r2["energy"] == r["energy"]
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_state_refusals(ctx):
    mesh = ctx.mesh_cube(2e-9, 3)
    a = _batch(ctx, mesh, 2, 3)
    state = a.get_state()
    b = ctx.instance_create(mesh, 3, lbm.LBM_FP64)          # another batch size
    with pytest.raises(lbm.LBMError):
        b.set_state(state)
    c = ctx.instance_create(mesh, 2, lbm.LBM_MIXED)          # another precision
    with pytest.raises(lbm.LBMError):
        c.set_state(state)
    bad = bytearray(state)
    bad[0] ^= 0xff                                           # not a state
    with pytest.raises(lbm.LBMError):
        a.set_state(bytes(bad))
    with pytest.raises(lbm.LBMError):
        a.set_state(state[:-8])                              # truncated
    with pytest.raises(lbm.LBMError):                        # resume is for FP64 batches
        c.minimise(lbm.default_opts(lbm.LBM_MIXED, resume=1))
    a.set_state(state)                                       # its own state is accepted
    for i in (a, b, c):
        i.destroy()
    ctx.mesh_destroy(mesh)
