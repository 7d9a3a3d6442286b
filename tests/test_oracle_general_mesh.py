"""Pins of the oracle's general-tetrahedral-mesh path (FP64 assembly, general
surface, solid angles by Girard's theorem, BEM with explicit coplanar pairs).

Fixed against: the exact integer assembly of the Kuhn cube (itself pinned by
closed forms), P1 reproduction identities on distorted meshes, the Gauss
solid-angle identity, the double-layer identity B 1 = -1, the demagnetising
factor 1/3 of a sphere, and finite differences of the energy.
"""
import math

import numpy as np
import pytest

from oracle.bem import bem_matrix_general, box_interior_solid_angle, hat_double_layer, interior_solid_angle
from oracle.mesh import cube_mesh, length_unit, surface_faces, tet_mesh
from oracle.micromag import MU0, mesh_problem
from oracle.minimise import OK, minimise
from synth import ball_mesh, jittered_cube
from synth.inputs import A_JM, JS_T, K1_JM3

RNG = np.random.default_rng(777)


def _rand_unit(n):
    v = RNG.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_fp64_assembly_reproduces_integer_kuhn_tables(n):
    """On the Kuhn cube the FP64 assembly equals the exact integer tables
    scaled by h/6, h^2/24, h^3/24; the surface is the same; L = h."""
    m = cube_mesh(n, 2e-9)
    g = tet_mesh(m.xyz(), m.tets)
    h = m.cell
    assert np.array_equal(g.ops.indptr, m.ops.indptr) and np.array_equal(g.ops.indices, m.ops.indices)
    # each entry sums at most 24 element terms of size ~h (resp. h^2, h^3)
    assert np.abs(g.ops.K - m.ops.K * h / 6).max() <= 1e-14 * h
    assert np.abs(g.ops.G - m.ops.G * h * h / 24).max() <= 1e-14 * h * h
    assert np.abs(g.ops.Gt - m.ops.Gt * h * h / 24).max() <= 1e-14 * h * h
    assert np.abs(g.ops.V - m.ops.V * h ** 3 / 24).max() <= 1e-14 * h ** 3
    assert np.array_equal(g.tris, m.tris) and np.array_equal(g.bnd, m.bnd)
    assert abs(g.cell / h - 1.0) < 1e-14


@pytest.mark.parametrize("mesh", ["jitter", "ball"])
def test_p1_reproduction_on_distorted_meshes(mesh):
    """For any conforming P1 mesh: K 1 = 0; K x_lin = 0 on interior rows (patch
    test); the lumped gradient -(1/V_i) sum_j G_ji u_j of a linear u = a.x is
    exactly -a; sum_i (G m)_i (a.x_i) = (m.a) Vol for constant m; sum V =
    sum of element volumes (for the jittered cube: the cube's volume)."""
    xyz, tets = jittered_cube(4, 2e-9, 0.12, seed=9) if mesh == "jitter" else ball_mesh(6, 20e-9)
    g = tet_mesh(xyz, tets)
    K = g.stiffness()
    G = g.coupling()
    V = g.volumes()
    kscale = np.abs(g.ops.K).max()
    assert np.abs(K @ np.ones(g.N)).max() < 1e-14 * kscale * 16
    inner = np.setdiff1d(np.arange(g.N), g.bnd)
    a = np.array([0.3, -1.2, 0.7])
    ulin = xyz @ a
    assert np.abs((K @ ulin)[inner]).max() < 1e-13 * kscale * np.abs(ulin).max() * 16
    Gt = [Gd.T.tocsr() for Gd in G]
    grad = -np.stack([Gt[d] @ ulin for d in range(3)], axis=1) / V[:, None]
    assert np.abs(grad + a).max() < 1e-12 * np.abs(a).max()
    mc = np.array([0.6, 0.0, -0.8])
    b = G[0] @ np.full(g.N, mc[0]) + G[1] @ np.full(g.N, mc[1]) + G[2] @ np.full(g.N, mc[2])
    P = xyz[tets]
    vol = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))).sum() / 6
    assert abs(np.dot(b, ulin) - np.dot(mc, a) * vol) < 1e-13 * vol * np.abs(a).sum()
    assert abs(V.sum() / vol - 1.0) < 1e-14
    if mesh == "jitter":
        assert abs(vol / (8e-9) ** 3 - 1.0) < 1e-13


def test_surface_of_a_jittered_cube():
    """The surface of the 5-tetrahedra cube split: 2 triangles per face square
    (F = 12 n^2), nb = N - (n-1)^3, all outward (the signed volume of the
    surface, sum x . n dA / 3, equals the mesh volume)."""
    n = 5
    xyz, tets = jittered_cube(n, 1.0, 0.15, seed=3)
    tris = surface_faces(xyz, tets)
    assert tris.shape[0] == 12 * n * n
    assert np.unique(tris).size == (n + 1) ** 3 - (n - 1) ** 3
    X = xyz[tris]
    flux = np.einsum("ij,ij->i", X[:, 0], np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])).sum() / 6
    assert abs(flux - n ** 3) < 1e-10


def test_solid_angles_girard_vs_box_and_gauss():
    """Girard's theorem gives the box's exact solid angles on the cube surface
    and agrees with the Gauss identity (the closed surface seen from one of its
    points subtends the interior angle there) on the ball."""
    m = cube_mesh(3)
    om = interior_solid_angle(m.nodes, m.bnd, m.tris)
    assert np.abs(om - box_interior_solid_angle(m.nodes[m.bnd], 3)).max() < 1e-14
    g = tet_mesh(*ball_mesh(6))
    om = interior_solid_angle(g.nodes, g.bnd, g.tris)
    excl = np.any(g.tris[None] == g.bnd[:, None, None], axis=2)
    gauss = -hat_double_layer(g.nodes[g.bnd], g.nodes[g.tris], exclude=excl).sum(axis=(1, 2))
    assert np.abs(om - gauss).max() < 1e-12
    assert np.all((om > math.pi) & (om < 4 * math.pi))        # a convex-ish closed surface


@pytest.mark.parametrize("mesh", ["jitter", "ball"])
def test_general_bem_row_sums(mesh):
    """B 1 = -1 (a constant double layer jumps by its density) on any closed surface."""
    xyz, tets = jittered_cube(3, 2e-9, 0.1, seed=4) if mesh == "jitter" else ball_mesh(6)
    p = mesh_problem(xyz, tets, JS_T, A_JM, K1_JM3, [0, 0, 1])
    assert np.abs(p.B.sum(axis=1) + 1.0).max() < 1e-12


def test_ball_demag_factor_tends_to_one_third():
    """A uniformly magnetised sphere has N = 1/3 along every axis; the
    discrete factors of the ball meshes are isotropic and converge to it."""
    errs = []
    for n in (4, 6, 8):
        p = mesh_problem(*ball_mesh(n), JS_T, A_JM, 0.0, [0, 0, 1])
        Nd = []
        for d in range(3):
            m = np.zeros((p.mesh.N, 3))
            m[:, d] = 1.0
            Nd.append(p.evaluate(m, np.zeros(3)).terms["d"] / (p.Kd * p.V.sum()))
        assert max(Nd) - min(Nd) < 1e-12
        errs.append(abs(Nd[0] - 1.0 / 3.0))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 4e-3


def test_general_field_is_energy_gradient():
    """On a jittered mesh, -(Js/mu0) V_i h_i is the finite-difference gradient
    of E, demag included (the adjoint chain)."""
    xyz, tets = jittered_cube(2, 2e-9, 0.12, seed=11)
    p = mesh_problem(xyz, tets, JS_T, A_JM, K1_JM3, (0.2, -0.3, 0.9))
    m = _rand_unit(p.mesh.N)
    h_ext = np.array([0.4, -1.1, 0.7])
    ev = p.evaluate(m, h_ext)
    dE = -(JS_T / MU0) * p.V[:, None] * ev.h
    eps = 1e-6
    fd = np.zeros_like(m)
    for i in range(p.mesh.N):
        for d in range(3):
            mp, mm = m.copy(), m.copy()
            mp[i, d] += eps
            mm[i, d] -= eps
            fd[i, d] = (p.evaluate(mp, h_ext).E - p.evaluate(mm, h_ext).E) / (2 * eps)
    assert np.abs(fd - dE).max() < 1e-7 * np.abs(dE).max()


def test_length_unit_is_scale_covariant():
    xyz, tets = ball_mesh(4, 1.0)
    assert abs(length_unit(xyz * 3e-9, tets) / (3e-9 * length_unit(xyz, tets)) - 1) < 1e-14


def test_minimiser_on_ball_reaches_a_minimum():
    """The minimiser on a small ball: converges, the energy decreases, and the
    final state is (near) uniform along the field, as for a single-domain
    sphere well above its switching field."""
    p = mesh_problem(*ball_mesh(4, 10e-9), JS_T, A_JM, K1_JM3, (0, 0, 1))
    m0 = _rand_unit(p.mesh.N)
    res = minimise(p, m0, np.array([0.0, 0.0, 8.0]), tol=1e-6)
    assert res.status == OK
    E0 = p.evaluate(m0, np.array([0.0, 0.0, 8.0])).E
    assert res.E < E0
    mz = (p.V * res.m[:, 2]).sum() / p.V.sum()
    assert mz > 0.999


def test_non_convex_surface_solid_angles_and_bem():
    """An L-shaped prism (a reflex edge along z): Girard's theorem gives 3 pi on
    the reflex edge (interior dihedral 3 pi / 2 on a straight edge), pi on the
    convex edges and 2 pi on the faces, and it agrees with the Gauss sum at
    every surface node; B 1 = -1 still holds."""
    from synth import l_shape
    n, h = 4, 1.0
    xyz, tets = l_shape(n, h)
    g = tet_mesh(xyz, tets)
    om = interior_solid_angle(g.nodes, g.bnd, g.tris)
    excl = np.any(g.tris[None] == g.bnd[:, None, None], axis=2)
    gauss = -hat_double_layer(g.nodes[g.bnd], g.nodes[g.tris], exclude=excl).sum(axis=(1, 2))
    assert np.abs(om - gauss).max() < 1e-12
    P = g.xyz_m[g.bnd]
    on_reflex = (np.abs(P[:, 0] - n / 2 * h) < 1e-12) & (np.abs(P[:, 1] - n / 2 * h) < 1e-12) & \
        (P[:, 2] > 0.5 * h) & (P[:, 2] < (n - 0.5) * h)
    assert on_reflex.sum() == n - 1
    assert np.abs(om[on_reflex] - 3 * math.pi).max() < 1e-12
    on_face = (np.abs(P[:, 2]) < 1e-12) & (P[:, 0] > 0.5 * h) & (P[:, 0] < 1.5 * h) & \
        (P[:, 1] > 0.5 * h) & (P[:, 1] < 1.5 * h)
    assert on_face.sum() >= 1 and np.abs(om[on_face] - 2 * math.pi).max() < 1e-12
    B = bem_matrix_general(g.nodes, g.bnd, g.tris)
    assert np.abs(B.sum(axis=1) + 1.0).max() < 1e-12


def test_assembly_is_independent_of_tetrahedron_orientation():
    """lbm_mesh_upload accepts any vertex order: reversing the orientation of
    every other tetrahedron leaves K, G, G^T, V and the outward surface unchanged."""
    xyz, tets = jittered_cube(3, 2e-9, 0.1, seed=13)
    flipped = tets.copy()
    flipped[::2] = flipped[::2][:, [0, 1, 3, 2]]
    a = tet_mesh(xyz, tets)
    b = tet_mesh(xyz, flipped)
    for key in ("K", "G", "Gt", "V"):
        ref = getattr(a.ops, key)
        assert np.abs(getattr(b.ops, key) - ref).max() <= 1e-15 * np.abs(ref).max(), key
    assert np.array_equal(a.tris, b.tris) and np.array_equal(a.bnd, b.bnd)
