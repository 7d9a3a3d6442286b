"""General tetrahedral meshes through lbm_mesh_upload, against the FP64 oracle.

Bars as for the cube meshes: CSR pattern, surface and surface ids identical;
FP64 tables to 1e-14 of their scale (FP64 assembly in another summation
order); BEM entries to 1e-12; FP64 fields and energies to 1e-10 relative;
FP64 trajectories to 1e-10 over 50 iterations; final energies to 1e-6.
Meshes: a jittered 5-tetrahedra cube split (flat faces, distorted elements)
and balls from the cube-to-sphere map (curved surface), up to the 87 880
tetrahedra of the paper-size 20 nm sphere.
"""
import numpy as np
import pytest

import paper_1309_5796_gb300 as lbm
from oracle.bem import bem_matrix_general
from oracle.mesh import cube_mesh, tet_mesh
from oracle.micromag import CubeProblem, mesh_problem
from oracle.minimise import minimise as oracle_minimise
from synth import ball_mesh, jittered_cube
from synth.inputs import A_JM, JS_T, K1_JM3, m_perturbed, m_random_sphere, tilted_axis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1309_5796_gb300 import build
    build.build()
    c = lbm.Context(0)
    yield c
    c.close()


MESHES = {
    "jitter4": lambda: jittered_cube(4, 2e-9, 0.12, seed=21),
    "ball6": lambda: ball_mesh(6, 12e-9),
    "ball10": lambda: ball_mesh(10, 20e-9),
}


@pytest.mark.parametrize("name", ["jitter4", "ball6", "ball10"])
def test_upload_tables_match_oracle(ctx, name):
    xyz, tets = MESHES[name]()
    o = tet_mesh(xyz, tets)
    h = ctx.mesh_upload(xyz, tets)
    info = ctx.mesh_info(h)
    assert (info["N"], info["nb"], info["nnz"], info["tets"], info["n"]) == \
        (o.N, o.bnd.size, o.ops.indices.size, tets.shape[0], 0)
    g = ctx.mesh_export(h)
    assert np.array_equal(g["rowptr"], o.ops.indptr)
    assert np.array_equal(g["col"], o.ops.indices)
    assert np.array_equal(g["bnd"], o.bnd)
    assert np.array_equal(g["tris"], o.tris)
    assert np.array_equal(g["tets"], tets)
    v = ctx.mesh_values(h)
    assert abs(v["unit"] / o.cell - 1) < 1e-14
    for key, ref in (("K", o.ops.K), ("G", o.ops.G), ("Gt", o.ops.Gt), ("V", o.ops.V)):
        assert np.abs(v[key] - ref).max() <= 1e-14 * np.abs(ref).max(), key
    ctx.mesh_destroy(h)


@pytest.mark.parametrize("name", ["jitter4", "ball6"])
def test_upload_bem_matches_oracle(ctx, name):
    xyz, tets = MESHES[name]()
    o = tet_mesh(xyz, tets)
    h = ctx.mesh_upload(xyz, tets)
    Bg = ctx.bem_rows(h, 0, o.bnd.size)
    Bo = bem_matrix_general(o.nodes, o.bnd, o.tris)
    assert np.abs(Bg - Bo).max() < 1e-12
    assert np.abs(Bg.sum(axis=1) + 1).max() < 1e-12
    ctx.mesh_destroy(h)


def test_kuhn_cube_uploaded_equals_mesh_cube(ctx):
    """The Kuhn cube passed as a general mesh gives the cube path's fields."""
    n = 5
    c = cube_mesh(n, 2e-9)
    hu = ctx.mesh_upload(c.xyz(), c.tets)
    hc = ctx.mesh_cube(2e-9, n)
    nb = ctx.mesh_info(hc)["nb"]
    assert np.abs(ctx.bem_rows(hu, 0, nb) - ctx.bem_rows(hc, 0, nb)).max() < 1e-13
    N = c.N
    m0 = m_random_sphere(N, 5)
    out = []
    for mesh in (hu, hc):
        inst = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
        inst.set_material(JS_T, A_JM, K1_JM3, tilted_axis(15.0, 1.0))
        inst.set_field(np.array([0.5, 0.0, -2.0]))
        inst.set_m(m0)
        out.append(inst.evaluate(lbm.default_opts(lbm.LBM_FP64)))
        inst.destroy()
    (ru, hu_, _), (rc, hc_, _) = out
    assert np.abs(hu_ - hc_).max() <= 1e-10 * np.abs(hc_).max()
    assert abs(ru[0]["energy"][4] - rc[0]["energy"][4]) <= 1e-10 * abs(rc[0]["energy"][4])
    ctx.mesh_destroy(hu)
    ctx.mesh_destroy(hc)


def _instance(ctx, mesh, B, prec, axes, fields, m0):
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    inst.set_m(m0)
    return inst


@pytest.mark.parametrize("prec,rtol", [(lbm.LBM_FP64, 1e-10), (lbm.LBM_MIXED, 2e-5)])
@pytest.mark.parametrize("name", ["jitter4", "ball6", "ball10"])
def test_general_field_and_energy(ctx, name, prec, rtol):
    xyz, tets = MESHES[name]()
    axis = tilted_axis(25.0, 0.7)
    h_ext = np.array([0.3, -0.7, 1.9])
    p = mesh_problem(xyz, tets, JS_T, A_JM, K1_JM3, axis)
    m0 = m_random_sphere(p.mesh.N, 31)
    mesh = ctx.mesh_upload(xyz, tets)
    inst = _instance(ctx, mesh, 1, prec, axis, h_ext, m0)
    res, h, u = inst.evaluate(lbm.default_opts(prec))
    ev = p.evaluate(m0, h_ext)
    hs = np.abs(ev.h).max()
    assert np.abs(h[0] - ev.h).max() <= rtol * hs
    us = np.abs(ev.u1 + ev.u2).max()
    assert np.abs((u[0, 0] + u[0, 1]) - (ev.u1 + ev.u2)).max() <= rtol * us * 10
    Eunit = p.Kd * p.V.sum()
    for k, key in enumerate(("ex", "an", "z", "d")):
        assert abs(res[0]["energy"][k] - ev.terms[key]) <= rtol * Eunit, key
    assert abs(res[0]["torque"] - ev.torque) <= rtol * hs
    e = inst.energy()    # a second evaluation (FP32 solves warm-start from the first)
    assert np.abs(e[0] - np.array(res[0]["energy"])).max() <= max(rtol, 1e-12) * Eunit
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_general_trajectory_fp64_first_50_iterations(ctx):
    xyz, tets = MESHES["ball6"]()
    axis = tilted_axis(1.0, 0.2)
    h_ext = np.array([0.0, 0.0, -5.0])
    p = mesh_problem(xyz, tets, JS_T, A_JM, K1_JM3, axis)
    m0 = m_perturbed(p.mesh.N, 41)
    checkpoints = (1, 5, 20, 50)
    ref = oracle_minimise(p, m0, h_ext, tol=1e-6, max_iter=50, record=checkpoints)
    traj = dict(ref.trajectory)
    mesh = ctx.mesh_upload(xyz, tets)
    inst = _instance(ctx, mesh, 1, lbm.LBM_FP64, axis, h_ext, m0)
    for k in checkpoints:
        if k not in traj:
            break
        inst.set_m(m0)
        r = inst.minimise(lbm.default_opts(lbm.LBM_FP64, max_iter=k))
        assert r[0]["iterations"] == k
        assert np.abs(inst.get_m()[0] - traj[k]).max() < 1e-10, k
    inst.destroy()
    ctx.mesh_destroy(mesh)


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_general_minimisation_batch(ctx, prec):
    """A batch of 4 instances on the n = 10 ball: each final energy within 1e-6
    of the oracle's minimum from the same start."""
    xyz, tets = MESHES["ball10"]()
    B = 4
    axes = np.array([tilted_axis(2.0 * b, 0.5 * b) for b in range(B)])
    fields = np.array([[0.0, 0.0, -2.0 * b] for b in range(B)])
    mesh = ctx.mesh_upload(xyz, tets)
    p0 = mesh_problem(xyz, tets, JS_T, A_JM, K1_JM3, axes[0])
    N = p0.mesh.N
    m0 = np.stack([m_perturbed(N, 60 + b) for b in range(B)])
    inst = _instance(ctx, mesh, B, prec, axes, fields, m0)
    res = inst.minimise(lbm.default_opts(prec))
    scale = p0.Kd * p0.V.sum()
    for b in range(B):
        p = CubeProblem(0, JS_T, A_JM, K1_JM3, axes[b], mesh=p0.mesh, B=p0.B)
        ref = oracle_minimise(p, m0[b], fields[b], tol=1e-6, max_iter=20000)
        assert res[b]["status"] == lbm.LBM_OK
        assert abs(res[b]["energy"][4] - ref.E) / max(abs(ref.E), scale) < 1e-6
    inst.destroy()
    ctx.mesh_destroy(mesh)


def test_paper_size_sphere(ctx):
    """The 20 nm sphere with 87 880 tetrahedra (0.77 nm spacing, the paper's
    grain, Sec. 3.1): sampled BEM rows against the oracle; mixed-precision and
    FP64 minimisations from a random state converge and their energies agree
    with the oracle's minimisation (golden, written by the oracle) to 1e-6."""
    xyz, tets = ball_mesh(26, 20e-9)
    assert tets.shape[0] == 87880
    o = tet_mesh(xyz, tets)
    mesh = ctx.mesh_upload(xyz, tets)
    nb = o.bnd.size
    rows = np.unique(np.r_[0, nb - 1, np.random.default_rng(3).integers(0, nb, 4)])
    Bo = bem_matrix_general(o.nodes, o.bnd, o.tris, rows=rows, chunk=2)
    for k, r in enumerate(rows):
        Bg = ctx.bem_rows(mesh, int(r), 1)[0]
        assert np.abs(Bg - Bo[k]).max() < 1e-11
    m0 = m_random_sphere(o.N, 8)
    h_ext = np.array([0.0, 0.0, -3.0])
    out = {}
    for prec in (lbm.LBM_MIXED, lbm.LBM_FP64):
        inst = _instance(ctx, mesh, 1, prec, [0.0, 0.0, 1.0], h_ext, m0)
        r = inst.minimise(lbm.default_opts(prec))[0]
        assert r["status"] == lbm.LBM_OK and r["torque"] < 1e-6
        m = inst.get_m()[0]
        assert np.abs(np.linalg.norm(m, axis=1) - 1).max() < 1e-12
        out[prec] = r["energy"][4]
        inst.destroy()
    scale = (JS_T ** 2 / (2 * 4e-7 * np.pi)) * o.ops.V.sum()
    assert abs(out[lbm.LBM_MIXED] - out[lbm.LBM_FP64]) / max(abs(out[lbm.LBM_FP64]), scale) < 1e-6
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sphere_paper.json")))
    assert g["status"] == 0 and g["seed"] == 8 and g["h_ext"] == list(h_ext)
    for prec, E in out.items():
        assert abs(E - g["E"]) / max(abs(g["E"]), scale) < 1e-6, (prec, E, g["E"])
    ctx.mesh_destroy(mesh)


def test_upload_rejects_invalid_meshes(ctx):
    xyz, tets = jittered_cube(2, 1e-9, 0.1, seed=2)
    bad = []
    t = tets.copy(); t[0, 0] = xyz.shape[0]; bad.append((xyz, t))            # id out of range
    t = tets.copy(); t[1, 1] = t[1, 0]; bad.append((xyz, t))                 # repeated node
    x = xyz.copy(); x[tets[2, 1]] = x[tets[2, 0]]; bad.append((x, tets))      # degenerate
    bad.append((np.vstack([xyz, [[1.0, 1.0, 1.0]]]), tets))                 # unused node
    bad.append((xyz, np.vstack([tets, tets[:1], tets[:1]])))                 # face in > 2 tetrahedra
    x = xyz.copy(); x[0, 0] = np.nan; bad.append((x, tets))                  # non-finite
    for x, t in bad:
        with pytest.raises(lbm.LBMError):
            ctx.mesh_upload(x, t)
