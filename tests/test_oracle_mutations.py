"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle (on the CPU, for the duration of the
test) and checks that a pin written against the paper or the mathematics
fails with it: a wrong sign in the Eq. (8) update, the adjoint chain dropped
from the stray field, the BEM term dropped from the potential, a wrong interior
solid angle, BB1 and BB2 swapped, a wrong cofactor, reflex dihedral angles
folded into [0, pi]; and in the hierarchical-matrix boundary operator a cluster
that loses a node, admissibility by the larger diameter or without the hat
supports, a truncation one rank short, a wrong residual sign in the cross
approximation, and low-rank products added into the wrong rows; in the step
control the kappa factors of the adaptive BB rule swapped, the largest instead
of the smallest remembered tau^2, and the Armijo test with a flipped sign or
without c1; and in the
space-transformation boundary a shell tensor built from J instead of its
inverse, one without the |det J| factor, and a shell left untransformed.
"""
import importlib.util
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location(f"_mut_{name}", os.path.join(HERE, f"{name}.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


pins = _load("test_oracle_pins")
gpins = _load("test_oracle_general_mesh")


def _caught(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_pins_pass_unmutated():
    pins.test_cayley_solves_implicit_equation()
    pins.test_bb_steps_on_quadratic()
    pins.test_bem_row_sums(3)
    pins.test_stiffness_kernel_and_patch(2)


def test_flipped_update_sign(monkeypatch):
    good = pins.cayley
    monkeypatch.setattr(pins, "cayley", lambda m, H, tau: good(m, H, -tau))
    _caught(pins.test_cayley_solves_implicit_equation)
    _caught(pins.test_cayley_first_order_is_steepest_descent)


def test_dropped_adjoint_chain(monkeypatch):
    from oracle.micromag import CubeProblem
    monkeypatch.setattr(CubeProblem, "adjoint_potential", lambda self, m: np.zeros(self.mesh.N))
    _caught(pins.test_demag_field_is_energy_gradient)


def test_dropped_bem_term(monkeypatch):
    from oracle.micromag import CubeProblem
    orig = CubeProblem.potential

    def without_bem(self, m):
        u1, u2 = orig(self, m)
        return u1, np.zeros_like(u2)

    monkeypatch.setattr(CubeProblem, "potential", without_bem)
    _caught(pins.test_potential_converges_to_box_solution)


def test_wrong_solid_angle(monkeypatch):
    import oracle.bem as bem
    monkeypatch.setattr(bem, "box_interior_solid_angle", lambda nodes, n: np.full(len(nodes), 2.0 * math.pi))
    _caught(pins.test_bem_row_sums, 3)


def test_swapped_bb_steps(monkeypatch):
    good = pins.bb_steps

    def swapped(s, y):
        r = good(s, y)
        return None if r is None else (r[1], r[0])

    monkeypatch.setattr(pins, "bb_steps", swapped)
    _caught(pins.test_bb_steps_on_quadratic)


def test_wrong_cofactor(monkeypatch):
    import oracle.mesh as mesh
    good = mesh.cofactors

    def bad(nodes, tets):
        c, det = good(nodes, tets)
        c = c.copy()
        c[:, 0] = -c[:, 0]
        return c, det

    monkeypatch.setattr(mesh, "cofactors", bad)
    _caught(pins.test_stiffness_kernel_and_patch, 2)


def test_reflex_angles_folded(monkeypatch):
    """Dihedral angles taken by arccos of unit vectors (in [0, pi]) instead of
    the oriented atan2: wrong at reflex edges of a non-convex surface."""
    import oracle.bem as bem

    def folded(xyz, bnd, tris):
        xyz = np.asarray(xyz, dtype=np.float64)
        nxt = {}
        for t in np.asarray(tris):
            for k in range(3):
                nxt.setdefault(int(t[k]), {})[int(t[(k + 1) % 3])] = int(t[(k + 2) % 3])
        out = np.empty(len(bnd))
        for q, i in enumerate(np.asarray(bnd)):
            fan, total = nxt[int(i)], 0.0
            for a, b in fan.items():
                c = fan[b]
                u = xyz[b] - xyz[i]
                u /= np.linalg.norm(u)
                wa = xyz[a] - xyz[i]
                wa -= np.dot(wa, u) * u
                wc = xyz[c] - xyz[i]
                wc -= np.dot(wc, u) * u
                cosv = np.dot(wa, wc) / (np.linalg.norm(wa) * np.linalg.norm(wc))
                total += math.acos(max(-1.0, min(1.0, cosv)))
            out[q] = total - (len(fan) - 2) * math.pi
        return out

    monkeypatch.setattr(gpins, "interior_solid_angle", folded)
    _caught(gpins.test_non_convex_surface_solid_angles_and_bem)


# -- hierarchical-matrix boundary operator ------------------------------------

hpins = _load("test_oracle_hmatrix")


@pytest.fixture(scope="module")
def hm_inputs():
    from oracle.bem import bem_matrix, bem_matrix_general
    from oracle.mesh import cube_mesh, tet_mesh
    from synth import ball_mesh
    c = cube_mesh(12, 1.0)
    xyz, tets = ball_mesh(10, 1.0)
    t = tet_mesh(xyz, tets)
    return (c, bem_matrix(c.nodes, 12, c.bnd, c.tris)), (t, bem_matrix_general(t.nodes, t.bnd, t.tris))


def test_hmatrix_pins_pass_unmutated(hm_inputs):
    hpins.test_cluster_tree_is_a_balanced_geometric_bisection(*hm_inputs, 16)
    hpins.test_block_tree_covers_every_entry_once_and_admits_only_separated_pairs(*hm_inputs, 2.0)
    hpins.test_hmatrix_obeys_the_frobenius_bound(*hm_inputs, "svd", 1e-4)
    hpins.test_truncated_svd_takes_the_smallest_sufficient_rank(1e-4)
    hpins.test_cross_approximation_recovers_exact_low_rank(5)


def test_cluster_loses_a_node(monkeypatch, hm_inputs):
    from oracle import hmatrix as hm
    good = hm._cluster
    monkeypatch.setattr(hm, "_cluster", lambda idx, pts, slo, shi: good(
        idx if idx.size == pts.shape[0] else idx[:-1], pts, slo, shi))
    _caught(hpins.test_cluster_tree_is_a_balanced_geometric_bisection, *hm_inputs, 16)
    _caught(hpins.test_block_tree_covers_every_entry_once_and_admits_only_separated_pairs, *hm_inputs, 2.0)


def test_admissibility_with_the_larger_diameter(monkeypatch, hm_inputs):
    from oracle import hmatrix as hm

    def max_rule(tau, sigma, eta):
        d = hm.box_dist(tau.lo_r, tau.hi_r, sigma.lo_c, sigma.hi_c)
        return d > 0.0 and max(hm.box_diam(tau.lo_r, tau.hi_r), hm.box_diam(sigma.lo_c, sigma.hi_c)) <= eta * d

    monkeypatch.setattr(hm, "admissible", max_rule)
    _caught(hpins.test_block_tree_covers_every_entry_once_and_admits_only_separated_pairs, *hm_inputs, 2.0)


def test_admissibility_without_the_hat_supports(monkeypatch, hm_inputs):
    from oracle import hmatrix as hm

    def points_only(tau, sigma, eta):
        d = hm.box_dist(tau.lo_r, tau.hi_r, sigma.lo_r, sigma.hi_r)
        return d > 0.0 and min(hm.box_diam(tau.lo_r, tau.hi_r), hm.box_diam(sigma.lo_r, sigma.hi_r)) <= eta * d

    monkeypatch.setattr(hm, "admissible", points_only)
    _caught(hpins.test_block_tree_covers_every_entry_once_and_admits_only_separated_pairs, *hm_inputs, 2.0)


def test_truncation_one_rank_short(monkeypatch, hm_inputs):
    from oracle import hmatrix as hm
    good = hm.truncated_svd

    def short(A, eps):
        U, V = good(A, eps)
        k = max(U.shape[1] - 1, 0)
        return U[:, :k], V[:k]

    monkeypatch.setattr(hm, "truncated_svd", short)
    _caught(hpins.test_truncated_svd_takes_the_smallest_sufficient_rank, 1e-4)
    _caught(hpins.test_hmatrix_obeys_the_frobenius_bound, *hm_inputs, "svd", 1e-4)


def test_cross_approximation_residual_sign(monkeypatch):
    from oracle import hmatrix as hm

    def wrong_sign(A, eps):
        R = np.array(A, dtype=np.float64)
        norm = float(np.linalg.norm(R))
        us, vs = [], []
        while np.linalg.norm(R) > eps * norm and len(us) < min(R.shape):
            i, j = np.unravel_index(int(np.argmax(np.abs(R))), R.shape)
            u, v = R[:, j].copy(), R[i, :] / R[i, j]
            R += np.outer(u, v)
            us.append(u)
            vs.append(v)
        return np.stack(us, axis=1), np.stack(vs, axis=0)

    monkeypatch.setattr(hm, "cross_approximation", wrong_sign)
    _caught(hpins.test_cross_approximation_recovers_exact_low_rank, 5)


def test_low_rank_product_into_the_wrong_rows(monkeypatch, hm_inputs):
    from oracle import hmatrix as hm

    def matmul(self, x):
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros((self.nb,) + x.shape[1:])
        for L in self.leaves:
            if L.low_rank:
                y[L.rows[::-1]] += L.U @ (L.V @ x[L.cols])
            else:
                y[L.rows] += L.D @ x[L.cols]
        return y

    monkeypatch.setattr(hm.HMatrix, "__matmul__", matmul)
    _caught(hpins.test_hmatrix_obeys_the_frobenius_bound, *hm_inputs, "svd", 1e-4)
    _caught(hpins.test_demag_energy_and_field_with_the_hmatrix, 1e-4)


# -- space-transformation open boundary ----------------------------------------

spins = _load("test_oracle_spacetrans")


def _shells(levels):
    from oracle.spacetrans import ShellProblem
    return {lv: ShellProblem(lv[0], spins.JS, spins.A, spins.K1, [0, 0, 1], lv[1], lv[2], cell=1.0)
            for lv in levels}


def test_shell_pins_pass_unmutated():
    spins.test_tensor_is_spd_with_determinant_det_J_and_identity_outside(_shells(spins.LEVELS[1:2]))


def test_shell_tensor_from_J_instead_of_its_inverse(monkeypatch):
    from oracle import spacetrans as st

    def forward(x, c, R1, R2):
        J, detJ = st.shell_jacobian(x, c, R1, R2)
        return np.abs(detJ)[:, None, None] * np.einsum("pij,pkj->pik", J, J)

    monkeypatch.setattr(st, "shell_tensor", forward)
    _caught(spins.test_tensor_is_spd_with_determinant_det_J_and_identity_outside, _shells(spins.LEVELS[1:2]))


def test_shell_tensor_without_the_volume_factor(monkeypatch):
    from oracle import spacetrans as st

    def no_det(x, c, R1, R2):
        J, _ = st.shell_jacobian(x, c, R1, R2)
        Ji = np.linalg.inv(J)
        return np.einsum("pij,pkj->pik", Ji, Ji)

    monkeypatch.setattr(st, "shell_tensor", no_det)
    _caught(spins.test_tensor_is_spd_with_determinant_det_J_and_identity_outside, _shells(spins.LEVELS[1:2]))


def test_shell_left_untransformed(monkeypatch):
    from oracle import spacetrans as st
    monkeypatch.setattr(st, "shell_tensor", lambda x, c, R1, R2: np.broadcast_to(np.eye(3), (len(x), 3, 3)).copy())
    _caught(spins.test_potential_converges_to_the_box_solution_inside_and_outside, _shells(spins.LEVELS))


# --- step control (Sec. 2.3) --------------------------------------------------

def test_kappa_factors_swapped(monkeypatch):
    import oracle.minimise as om
    monkeypatch.setattr(om, "KAPPA_SHRINK", 1.1)
    monkeypatch.setattr(om, "KAPPA_GROW", 0.9)
    _caught(pins.test_adaptive_bb_rule_hand_sequence)


def test_tau2_memory_max_for_min(monkeypatch):
    import oracle.minimise as om
    monkeypatch.setattr(om, "TAU2_PICK", max)
    _caught(pins.test_adaptive_bb_rule_hand_sequence)


def test_armijo_sign_flipped(monkeypatch):
    import oracle.minimise as om
    monkeypatch.setattr(om, "armijo_accepts", lambda phit, E_ref, c1, tau, gg: phit <= E_ref + c1 * tau * gg)
    _caught(pins.test_first_step_armijo_boundary)


def test_armijo_without_c1(monkeypatch):
    import oracle.minimise as om
    monkeypatch.setattr(om, "armijo_accepts", lambda phit, E_ref, c1, tau, gg: phit <= E_ref - tau * gg)
    _caught(pins.test_first_step_armijo_boundary)
