"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle (on the CPU, for the duration of the
test) and checks that a pin written against the paper or the mathematics
fails with it: a wrong sign in the Eq. (8) update, the adjoint chain dropped
from the stray field, the BEM term dropped from the potential, a wrong interior
solid angle, BB1 and BB2 swapped, a wrong cofactor, and reflex dihedral angles
folded into [0, pi].
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
