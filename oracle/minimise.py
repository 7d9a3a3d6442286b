"""Curvilinear steepest descent with Barzilai-Borwein steps (FP64 reference).

Paper, Sec. 2.1-2.3:
  * H(m) := -m x grad phi_t(m)                         (Sec. 2.1)
  * m^{n+1} = m^n - tau (m^n + m^{n+1})/2 x H(m^n)     (Eq. 8, curvilinear search)
    keeps |m^{n+1}| = |m^n| and has an explicit solution (cited to Goldfarb et
    al.; the explicit form below is derived here, see `cayley`);
  * g^n := m^n x (-m^n x grad phi_t(m^n)) = m^n x H(m^n), s^{n-1} = m^n - m^{n-1},
    y^{n-1} = g^n - g^{n-1}; tau^1 = s.s/s.y, tau^2 = s.y/y.y            (Sec. 2.3)
  * the first step by inexact line search; then BB steps chosen by the adaptive
    rule from gradient-projection methods; a line search whenever the new energy
    exceeds the previous 20 energies (nonmonotone globalisation)           (Sec. 2.3)
  * hysteresis: the applied field is stepped and each point starts from the
    previous minimum                                                      (Sec. 1.1, 3.1)

Readings where the paper prints no detail:
  * explicit update: with w = tau H/2 the implicit equation is x + x x w = m - m x w,
    solved by x = [(1 - |w|^2) m - 2 m x w + 2 (m.w) w] / (1 + |w|^2);
  * first trial step tau = 1 / max_i |H_i|;  Armijo test
    E(tau) <= E_ref - c1 tau sum_i |g_i|^2 with c1 = 1e-4 (dE/dtau at 0 is
    -sum |g|^2 because dY/dtau(0) = -m x H = -g), step halving, at most 30
    halvings (then status LINESEARCH);
  * nonmonotone test: a BB trial is rejected iff its energy is strictly larger
    than the maximum of the last min(k, 20) accepted energies (the initial one
    included); the line search then uses E_ref = that maximum;
  * adaptive BB rule: if s.y <= 0 (no positive curvature along the step) restart
    with the first-step trial tau = 1/max_i |H_i| at the new point; else push
    tau^2 into a memory of the last 3 values; if tau^2/tau^1 <= kappa take tau = min of that
    memory and kappa *= 0.9, else tau = tau^1 and kappa *= 1.1; kappa_0 = 0.5;
    tau clamped to [1e-10, 1e10];
  * stop when max_i |m_i x h_i| / Js < tol (or, optionally, sum |g|^2 < tol_g,
    the paper's grad h^T grad h < 1e-12 of Sec. 3.1);
  * sweep: at every field point the step memory, the energy history and the
    first-step line search start afresh.

Step-rule variants (StepRule.bb): "adaptive" (above, the default), "bb1" (tau^1
always), "bb2" (tau^2 always) and "alternate" (tau^1 and tau^2 on alternate
steps, the plain alternation that the adaptive rule refines, Sec. 2.3); all
restart from tau = 1/max|H| when s.y <= 0 and share the clamp.

LaBonte's method (Sec. 1.2 history): every node's magnetisation is replaced
by its normalised effective field; over- and under-relaxation rotate it part
of the way or beyond.  Data-parallel reading used here (all nodes at once,
relaxation factor omega):  m_i <- normalize((1 - omega) m_i + omega h_i/|h_i|),
omega = 1 the plain replacement; no line search; stop test as above.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .micromag import CubeProblem

OK, MAX_ITER, LINESEARCH = 0, 1, 2


@dataclass
class StepRule:
    c1: float = 1e-4
    max_backtracks: int = 30
    memory: int = 20
    kappa0: float = 0.5
    m_alpha: int = 3
    tau_min: float = 1e-10
    tau_max: float = 1e10
    bb: str = "adaptive"          # "adaptive" | "bb1" | "bb2" | "alternate"


def cayley(m: np.ndarray, H: np.ndarray, tau: float) -> np.ndarray:
    """Explicit solution x of x = m - tau (m + x)/2 x H, row-wise."""
    w = 0.5 * tau * H
    ww = np.sum(w * w, axis=1, keepdims=True)
    mw = np.sum(m * w, axis=1, keepdims=True)
    return ((1.0 - ww) * m - 2.0 * np.cross(m, w) + 2.0 * mw * w) / (1.0 + ww)


def bb_steps(s: np.ndarray, y: np.ndarray):
    """(tau^1, tau^2) of the secant equation tau^-1 s = y, or None if s.y <= 0."""
    sy = float(np.sum(s * y))
    if sy <= 0.0:
        return None
    return float(np.sum(s * s)) / sy, sy / float(np.sum(y * y))


@dataclass
class BBState:
    kappa: float
    tau2: list = field(default_factory=list)
    k: int = 0                    # BB steps taken (parity for "alternate")


# Adaptive rule constants (Sec. 2.3 names the rule, not its constants; see the
# module docstring): kappa shrinks by KAPPA_SHRINK when the short step tau^2 is
# chosen, grows by KAPPA_GROW otherwise; the short step is the smallest of the
# last m_alpha values of tau^2 (TAU2_PICK).
KAPPA_SHRINK = 0.9
KAPPA_GROW = 1.1
TAU2_PICK = min


def armijo_accepts(phit: float, E_ref: float, c1: float, tau: float, gg: float) -> bool:
    """Sufficient decrease along the curve Y(tau) of Eq. (8): dE/dtau at 0 is
    -sum |g|^2, so the Armijo test is E(tau) <= E_ref - c1 tau sum |g|^2."""
    return phit <= E_ref - c1 * tau * gg


def nonmonotone_rejects(phit: float, hist: list, memory: int) -> bool:
    """Sec. 2.3: a BB trial is rejected iff its energy is strictly larger than
    every one of the last `memory` accepted energies (their maximum)."""
    return phit > max(hist[-memory:])


def next_bb_tau(s, y, tau_restart: float, st: BBState, rule: StepRule) -> float:
    steps = bb_steps(s, y)
    k = st.k
    st.k += 1
    if steps is None:
        tau = tau_restart
    elif rule.bb == "bb1":
        tau = steps[0]
    elif rule.bb == "bb2":
        tau = steps[1]
    elif rule.bb == "alternate":
        tau = steps[0] if k % 2 == 0 else steps[1]
    else:
        t1, t2 = steps
        st.tau2.append(t2)
        del st.tau2[:-rule.m_alpha]
        if t2 / t1 <= st.kappa:
            tau = TAU2_PICK(st.tau2)
            st.kappa *= KAPPA_SHRINK
        else:
            tau = t1
            st.kappa *= KAPPA_GROW
    return float(min(max(tau, rule.tau_min), rule.tau_max))


@dataclass
class Result:
    m: np.ndarray
    E: float
    terms: dict
    torque: float
    status: int
    iterations: int
    evaluations: int
    line_searches: int
    trajectory: list = field(default_factory=list)
    history: list = field(default_factory=list)      # accepted energies / E0


def minimise(prob: CubeProblem, m0: np.ndarray, h_ext, tol: float = 1e-6, max_iter: int = 100000,
             rule: StepRule | None = None, record=(), grad_tol: float | None = None) -> Result:
    """Minimise phi_t from m0 at applied field h_ext (tesla).  `record` lists
    iteration counts after which a copy of m is kept in `trajectory`."""
    rule = rule or StepRule()
    record = set(record)
    m = np.array(m0, dtype=np.float64)
    ev = prob.evaluate(m, h_ext)
    evals = 1
    H = -np.cross(m, ev.grad)
    g = np.cross(m, H)
    E0 = prob.E0                             # energies compared in the unit of grad phi
    hist = [ev.E / E0]
    traj = []
    if 0 in record:
        traj.append((0, m.copy()))

    def converged(e, gg):
        if grad_tol is not None:
            return gg < grad_tol
        return e.torque < tol

    gg = float(np.sum(g * g))
    if converged(ev, gg):
        return Result(m, ev.E, ev.terms, ev.torque, OK, 0, evals, 0, traj, hist)
    hmax = float(np.max(np.linalg.norm(H, axis=1)))
    tau = 1.0 / hmax
    searching, E_ref = True, ev.E / E0       # first step: inexact line search
    backtracks, line_searches = 0, 1
    bb = BBState(kappa=rule.kappa0)
    it = 0
    status = MAX_ITER
    while it < max_iter:
        mt = cayley(m, H, tau)
        et = prob.evaluate(mt, h_ext)
        evals += 1
        phit = et.E / E0
        if searching:
            accept = armijo_accepts(phit, E_ref, rule.c1, tau, gg)
        else:
            accept = not nonmonotone_rejects(phit, hist, rule.memory)
            if not accept:
                searching, E_ref = True, max(hist[-rule.memory:])
                line_searches += 1
                backtracks = 0
        if not accept:
            backtracks += 1
            if backtracks > rule.max_backtracks:
                status = LINESEARCH
                break
            tau *= 0.5
            continue
        Ht = -np.cross(mt, et.grad)
        gt = np.cross(mt, Ht)
        s, y = mt - m, gt - g
        m, H, g, ev = mt, Ht, gt, et
        gg = float(np.sum(g * g))
        hist.append(phit)
        it += 1
        if it in record:
            traj.append((it, m.copy()))
        if converged(ev, gg):
            status = OK
            break
        tau = next_bb_tau(s, y, 1.0 / float(np.max(np.linalg.norm(H, axis=1))), bb, rule)
        searching, backtracks = False, 0
    return Result(m, ev.E, ev.terms, ev.torque, status, it, evals, line_searches, traj, hist)


def labonte(prob: CubeProblem, m0: np.ndarray, h_ext, omega: float = 1.0, tol: float = 1e-6,
            max_iter: int = 100000, record=()) -> Result:
    """LaBonte's rotate-to-field iteration with relaxation factor omega, all
    nodes at once: m_i <- normalize((1 - omega) m_i + omega h_i/|h_i|)."""
    record = set(record)
    m = np.array(m0, dtype=np.float64)
    ev = prob.evaluate(m, h_ext)
    evals, it, traj = 1, 0, []
    hist = [ev.E / prob.E0]
    status = MAX_ITER
    while True:
        if ev.torque < tol:
            status = OK
            break
        if it >= max_iter:
            break
        hn = np.linalg.norm(ev.h, axis=1, keepdims=True)
        hhat = np.where(hn > 0.0, ev.h / np.where(hn > 0.0, hn, 1.0), m)
        x = (1.0 - omega) * m + omega * hhat
        m = x / np.linalg.norm(x, axis=1, keepdims=True)
        ev = prob.evaluate(m, h_ext)
        evals += 1
        it += 1
        hist.append(ev.E / prob.E0)
        if it in record:
            traj.append((it, m.copy()))
    return Result(m, ev.E, ev.terms, ev.torque, status, it, evals, 0, traj, hist)


def hysteresis(prob: CubeProblem, m0: np.ndarray, direction, fields, tol: float = 1e-6,
               max_iter: int = 100000, rule: StepRule | None = None):
    """Field continuation: minimise at each field value (tesla along `direction`),
    warm-started from the previous minimum.  Returns per-point V-weighted
    m.direction, energy, and the list of results."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    m = np.array(m0, dtype=np.float64)
    mpar, energy, results = [], [], []
    for hv in fields:
        r = minimise(prob, m, hv * d, tol=tol, max_iter=max_iter, rule=rule)
        m = r.m
        mpar.append(float(prob.mean_m(m) @ d))
        energy.append(r.E)
        results.append(r)
    return np.array(mpar), np.array(energy), results


def switching_field(fields, mpar) -> float | None:
    """First field value at which the mean projection changes sign."""
    for k in range(1, len(fields)):
        if np.sign(mpar[k]) != np.sign(mpar[k - 1]) and mpar[k - 1] != 0.0:
            return float(fields[k])
    return None
