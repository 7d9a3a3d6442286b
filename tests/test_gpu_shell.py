"""The open boundary by space transformation on the device (Sec. 3.1: the
paper's own solver maps a shell onto the exterior) against the oracle's
ShellProblem (oracle/spacetrans.py: the same grid, tensor-weighted stiffness
and Dirichlet face, solved by a sparse LU).

Bars: FP64 fields, potentials and energies to 1e-10 relative (the device solve
is Jacobi-PCG to a 1e-13 relative residual); the mixed precision's FP32 phase
to 2e-5; a full FP64 minimisation to the oracle's final energy within 1e-6
relative; batches give each instance its own result.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from oracle.minimise import minimise as oracle_minimise
from oracle.spacetrans import ShellProblem
from synth.inputs import A_JM, JS_T, K1_JM3, m_random_sphere, single_fp64_case, tilted_axis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


def _shell_mesh(ctx, n, a, s):
    mesh = ctx.mesh_cube(2e-9, n)
    info = ctx.mesh_shell(mesh, a, s)
    nt = n + 2 * (a + s)
    assert info["grid_nodes"] == (nt + 1) ** 3
    return mesh, info


@pytest.mark.parametrize("prec,rtol", [(lbm.LBM_FP64, 1e-10), (lbm.LBM_MIXED, 2e-5)])
@pytest.mark.parametrize("n,a,s,B", [(1, 1, 1, 3), (3, 2, 3, 5), (6, 2, 4, 2)])
def test_shell_field_and_energy(ctx, n, a, s, B, prec, rtol):
    """A batch of B random states: per instance the field at every node, the
    potential, the four energy terms and the torque of the oracle."""
    N = (n + 1) ** 3
    rng = np.random.default_rng(5 + n)
    axes = np.array([tilted_axis(30.0 * rng.random(), 6.28 * rng.random()) for _ in range(B)])
    fields = rng.normal(size=(B, 3))
    m0 = np.stack([m_random_sphere(N, 40 + 7 * n + b) for b in range(B)])
    mesh, info = _shell_mesh(ctx, n, a, s)
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    inst.set_m(m0)
    res, h, u = inst.evaluate(lbm.default_opts(prec))
    for b in range(B):
        p = ShellProblem(n, JS_T, A_JM, K1_JM3, axes[b], a, s)
        if b == 0:
            assert info["nnz"] == p.Kgrid.nnz and info["shell_tets"] == int(p.shell_tets.sum())
        ev = p.evaluate(m0[b], fields[b])
        hs = np.abs(ev.h).max()
        assert np.abs(h[b] - ev.h).max() <= rtol * hs, b
        us = np.abs(ev.u1).max()
        assert np.abs(u[b, 0] - ev.u1).max() <= 10 * rtol * us
        assert np.abs(u[b, 1]).max() == 0.0
        Eunit = p.Kd * p.cell ** 3 * N
        for k, key in enumerate(("ex", "an", "z", "d")):
            assert abs(res[b]["energy"][k] - ev.terms[key]) <= rtol * Eunit, (b, key)
        assert abs(res[b]["energy"][4] - ev.E) <= rtol * Eunit
        assert abs(res[b]["torque"] - ev.torque) <= rtol * hs
        assert res[b]["cg_iters1"] > 0 and res[b]["cg_iters2"] == 0
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_shell_uniform_state_energy_bounds(ctx):
    """A uniformly magnetised cube (along x and along z): the stray-field energy
    equals the oracle's to 1e-10 and lies below the closed-form continuum value
    of the cube (demagnetising factor 1/3): the discrete potential energy
    b^T K^-1 b / 2 of a conforming P1 space is a lower bound of it."""
    n = 4
    N = (n + 1) ** 3
    Kd = JS_T ** 2 / (2 * 4e-7 * np.pi)
    E_cube = Kd / 3.0 * (n * 2e-9) ** 3
    for a in (1, 3):
        mesh, _ = _shell_mesh(ctx, n, a, 4)
        inst = ctx.instance_create(mesh, 2, lbm.LBM_FP64)
        inst.set_material(JS_T, A_JM, K1_JM3, [0, 0, 1])
        inst.set_field([0.0, 0.0, 0.0])
        m = np.zeros((2, N, 3))
        m[0, :, 0] = 1.0
        m[1, :, 2] = 1.0
        inst.set_m(m)
        res, _, _ = inst.evaluate(lbm.default_opts(lbm.LBM_FP64), want_h=False, want_u=False)
        p = ShellProblem(n, JS_T, A_JM, K1_JM3, [0, 0, 1], a, 4)
        for b in range(2):
            e = res[b]["energy"][3]
            assert 0.5 * E_cube < e < E_cube
            assert abs(e - p.evaluate(m[b], np.zeros(3)).terms["d"]) <= 1e-10 * E_cube
        inst.destroy()
        ctx.mesh_destroy(mesh)


def test_shell_minimisation_fp64(ctx):
    """20 nm cube, -6 T at 1 degree, with the transformed open boundary (air 3
    cells, shell 5 cells): the device minimiser reaches the oracle's final energy
    within 1e-6 relative, with the stop test met."""
    case = single_fp64_case()
    a, s = 3, 5
    p = ShellProblem(case.n, JS_T, A_JM, K1_JM3, case.axis, a, s)
    ref = oracle_minimise(p, case.m0, case.h_ext, tol=1e-6, max_iter=20000)
    mesh, _ = _shell_mesh(ctx, case.n, a, s)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    inst.set_material(JS_T, A_JM, K1_JM3, case.axis)
    inst.set_field(case.h_ext)
    inst.set_m(case.m0)
    r = inst.minimise(lbm.default_opts(lbm.LBM_FP64))[0]
    assert r["status"] == lbm.LBM_OK and r["torque"] < 1e-6
    scale = max(abs(ref.E), p.Kd * (case.n * p.cell) ** 3)
    assert abs(r["energy"][4] - ref.E) / scale < 1e-6
    assert abs(r["iterations"] - ref.iterations) <= max(5, ref.iterations // 10)
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_shell_minimisation_mixed_batch(ctx):
    """Mixed precision, a batch of 4 (different tilts): every instance reaches
    its own FP64 oracle energy within 1e-6 relative."""
    n, a, s, B = 5, 2, 4, 4
    N = (n + 1) ** 3
    rng = np.random.default_rng(21)
    axes = np.array([tilted_axis(2.0 + 3.0 * rng.random(), 6.28 * rng.random()) for _ in range(B)])
    fields = np.array([[0.0, 0.0, -4.0 - 2.0 * rng.random()] for _ in range(B)])
    m0 = np.tile([0.0, 0.0, 1.0], (B, N, 1))
    mesh, _ = _shell_mesh(ctx, n, a, s)
    inst = ctx.instance_create(mesh, B, lbm.LBM_MIXED)
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    inst.set_m(m0)
    res = inst.minimise(lbm.default_opts(lbm.LBM_MIXED))
    for b in range(B):
        p = ShellProblem(n, JS_T, A_JM, K1_JM3, axes[b], a, s)
        ref = oracle_minimise(p, m0[b], fields[b], tol=1e-6, max_iter=20000)
        scale = max(abs(ref.E), p.Kd * (n * p.cell) ** 3)
        assert res[b]["status"] == lbm.LBM_OK, b
        assert abs(res[b]["energy"][4] - ref.E) / scale < 1e-6, b
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_shell_attach_rules(ctx):
    """Refusals: a general mesh, a mesh with instances, a or s below 1, a grid
    beyond 200 cells a side; the no-allocation entry refuses a mesh with the
    shell; detach (a = s = 0) returns the mesh to the FEM/BEM coupling."""
    torch = pytest.importorskip("torch")
    from oracle.mesh import cube_mesh
    o = cube_mesh(2)
    gen = ctx.mesh_upload(o.nodes * 2e-9, o.tets)
    with pytest.raises(lbm.LBMError):
        ctx.mesh_shell(gen, 2, 2)
    ctx.mesh_destroy(gen)
    mesh = ctx.mesh_cube(2e-9, 2)
    for a, s in ((0, 2), (2, 0), (-1, 3)):
        with pytest.raises(lbm.LBMError):
            ctx.mesh_shell(mesh, a, s)
    with pytest.raises(lbm.LBMError):
        ctx.mesh_shell(mesh, 60, 60)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    with pytest.raises(lbm.LBMError):
        ctx.mesh_shell(mesh, 2, 2)
    inst.destroy()
    ctx.mesh_shell(mesh, 2, 2)
    d_m = torch.zeros(27 * 3, dtype=torch.float64, device="cuda")
    d_m[2::3] = 1.0
    with pytest.raises(lbm.LBMError):
        ctx.evaluate_noalloc(mesh, JS_T, A_JM, K1_JM3, [0, 0, 1], np.zeros(3), d_m.data_ptr())
    ctx.mesh_shell(mesh, 0, 0)
    inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
    res, _, _ = inst.evaluate(lbm.default_opts(lbm.LBM_FP64), want_h=False, want_u=False)
    assert res[0]["cg_iters2"] > 0          # the two Poisson solves are back
    inst.destroy()
    ctx.mesh_destroy(mesh)


class _ShellProblemCG(ShellProblem):
    """The oracle's problem with the grid system solved by Jacobi-preconditioned
    CG (scipy) to a 1e-14 relative residual instead of the sparse LU: the same
    definition, usable at the bench's grid size (166 375 grid nodes)."""

    def grid_potential(self, m):
        import scipy.sparse.linalg as spla
        rhs = np.zeros(self.Kgrid.shape[0])
        rhs[self.magnet_in_grid] = self.rhs(m)
        Kf = self.Kgrid[self.free][:, self.free].tocsr()
        d = 1.0 / Kf.diagonal()
        M = spla.LinearOperator(Kf.shape, matvec=lambda v: d * v)
        kw = {"rtol": 1e-14} if "rtol" in spla.cg.__code__.co_varnames else {"tol": 1e-14}
        uf, info = spla.cg(Kf, rhs[self.free], M=M, maxiter=20000, atol=0.0, **kw)
        assert info == 0
        u = np.zeros_like(rhs)
        u[self.free] = uf
        return u


_BENCH = dict(n=30, a=4, s=8, B=64, sample=(0, 17, 42, 63))


@pytest.fixture(scope="module")
def bench_ref():
    """Inputs of the bench-shape case and the oracle's evaluations of the
    sampled instances (shared by both precisions)."""
    n, a, s, B = (_BENCH[k] for k in ("n", "a", "s", "B"))
    N = (n + 1) ** 3
    rng = np.random.default_rng(77)
    axis = tilted_axis(1.0, 0.4)
    fields = rng.normal(size=(B, 3))
    m0 = np.stack([m_random_sphere(N, 900 + b) for b in range(B)])
    p = _ShellProblemCG(n, JS_T, A_JM, K1_JM3, axis, a, s)
    evs = {b: p.evaluate(m0[b], fields[b]) for b in _BENCH["sample"]}
    return p, axis, fields, m0, evs


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_shell_bench_shape_sampled(ctx, bench_ref, prec):
    """The bench's shape: 64 instances on the 30^3-cell cube, air 4 and shell 8
    cells (a 54^3-cell grid, every SM a block, four instances per thread in the
    FP32 kernel).  Four sampled instances: fields at every magnet node and the
    energy terms against the oracle's definition (grid system by CG to 1e-14).
    FP64 solves to a 1e-14 relative residual: 1e-10 of the largest field value;
    the mixed precision's FP32 phase (FP32 CG to 1e-6): 1e-6 (measured 1.1e-7)."""
    p, axis, fields, m0, evs = bench_ref
    n, a, s, B = (_BENCH[k] for k in ("n", "a", "s", "B"))
    N = (n + 1) ** 3
    mesh, info = _shell_mesh(ctx, n, a, s)
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, axis)
    inst.set_field(fields)
    inst.set_m(m0)
    opts = lbm.default_opts(prec)
    rtol = 1e-6
    if prec == lbm.LBM_FP64:
        opts.cg_tol = 1e-14
        rtol = 1e-10
    res, h, _ = inst.evaluate(opts, want_u=False)
    inst.destroy()
    ctx.mesh_destroy(mesh)
    Eunit = p.Kd * p.cell ** 3 * N
    errs = []
    for b, ev in evs.items():
        hs = np.abs(ev.h).max()
        errs.append(np.abs(h[b] - ev.h).max() / hs)
        assert errs[-1] <= rtol, (b, errs)
        for k, key in enumerate(("ex", "an", "z", "d")):
            assert abs(res[b]["energy"][k] - ev.terms[key]) <= rtol * Eunit, (b, key)
    print("max relative field error", max(errs))


def test_shell_serving(ctx):
    """The server with the space-transformation boundary on every group's cube
    (serve option shell_a/shell_s): requests of two cube sizes, mixed and FP64
    precision, each reaching its own oracle minimum within 1e-6 relative; a
    request gives the same bits alone and after other requests reused its slot
    (the slot's grid potential starts from zero)."""
    from synth.inputs import m_perturbed
    a, s = 2, 3
    reqs = []
    for k, (n, hz, prec) in enumerate(((3, -5.0, lbm.LBM_MIXED), (4, -6.0, lbm.LBM_MIXED),
                                       (3, -4.5, lbm.LBM_FP64), (4, -5.5, lbm.LBM_MIXED))):
        N = (n + 1) ** 3
        reqs.append(dict(n=n, cell_m=2e-9, Js=JS_T, A=A_JM, K1=K1_JM3, axis=tilted_axis(2.0 + k, 0.7 * k),
                         h=np.array([0.0, 0.0, hz]), m0=m_perturbed(N, 60 + k), precision=prec))
    ctx.serve_start(slots=2, chunk=4, shell_a=a, shell_s=s)
    try:
        first = ctx.wait(ctx.submit(**reqs[0]), (reqs[0]["n"] + 1) ** 3, timeout_s=300)
        tickets = [ctx.submit(**r) for r in reqs]
        out = [ctx.wait(t, (r["n"] + 1) ** 3, timeout_s=300) for t, r in zip(tickets, reqs)]
    finally:
        ctx.serve_stop()
    assert out[0][0]["energy"][4] == first[0]["energy"][4]
    assert np.array_equal(out[0][1], first[1])
    for (res, _), r in zip(out, reqs):
        p = ShellProblem(r["n"], JS_T, A_JM, K1_JM3, r["axis"], a, s)
        ref = oracle_minimise(p, r["m0"], r["h"], tol=1e-6, max_iter=20000)
        scale = max(abs(ref.E), p.Kd * (r["n"] * p.cell) ** 3)
        assert res["status"] == lbm.LBM_OK, r
        assert abs(res["energy"][4] - ref.E) / scale < 1e-6, (r["n"], res["energy"][4], ref.E)
