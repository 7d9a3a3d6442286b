"""Discrete micromagnetic energy, effective field and magnetostatic potential (FP64).

Paper, Eq. (1): the total Gibbs free energy phi_t is the sum of stray-field,
exchange, anisotropy and external (Zeeman) energy; Sec. 2.1: phi_t is a spatial
(finite element) approximation, h_eff = -delta phi_t / delta m; Table 2: the
gradient is a sparse matrix-vector product and the scalar potential a linear
solve (the CPU code solved it directly, by LU, Table 1 caption).

Discrete forms (SI units, P1 magnetisation m with |m_i| = 1 at the nodes):
  E_ex = A  sum_c m_c^T K m_c                       (exact for P1)
  E_an = K1 sum_i V_i (1 - (m_i . a)^2)             (lumped; >= 0)
  E_z  = -(Js/mu0) sum_i V_i m_i . (mu0 H_ext)        (exact for P1: int phi_i = V_i)
  E_d  = -(Js/(2 mu0)) sum_i V_i m_i . (mu0 h_d,i)
and the effective field as mu0*H in tesla, mu0 h_i = -(mu0/(Js V_i)) dE/dm_i
(so that -(Js/mu0) V_i h_i is exactly the gradient of the discrete energy):
  mu0 h_ex,i = -(2 A mu0/(Js V_i)) (K m)_i
  mu0 h_an,i = (2 K1 mu0/Js) (m_i . a) a
  mu0 h_d,i  = -(Js/V_i) sum_j G_ji (u_j + uT_j)/2
with the potential (U = Ms u, u in metres) from the hybrid FEM/BEM:
  b = G m;  K u1 = b  (Neumann; gauge: the V-weighted mean of u1 is removed),
  u2|S = B u1|S,   K_II u2,I = -K_IS u2,S,   u = u1 + u2 =: X b,
and the adjoint potential uT = X^T b:
  K_II w_I = b_I (w_S = 0),  t_S = b_S - K_SI w_I,  c_S = B^T t_S,
  K uT = b + c (scattered to the surface; Neumann, defined up to a constant).
Reading: Sec. 2.1-2.3 define the step from grad phi_t, the gradient of the
discrete energy.  E_d is the quadratic form (Js^2/(2 mu0)) b^T X b / 2 (b = G m), so
its gradient involves (X + X^T)/2; the collocation BEM makes X non-symmetric,
and the plain forward field (X b alone) is then not the gradient of E_d --
with it the energy-based line search of Sec. 2.3 fails near the minimum.
The potential solves here are direct sparse LU factorisations (the exact
solution of the linear systems), not the iterative solver of the GPU path.

Minimiser units (reading of "grad phi_t", Sec. 2.1-2.3): the Euclidean gradient
of the discrete energy in the fixed unit E0 = Kd h^3, Kd = Js^2/(2 mu0):
grad_i phi = (dE/dm_i) / E0 = -(Js/mu0) V_i (mu0 h_i) / E0.
General tetrahedral meshes (mesh_problem) use the same formulas with the FP64
operators of oracle.mesh.tet_mesh, the general BEM, and h replaced by the
mesh's length unit L.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from .bem import bem_matrix, bem_matrix_general
from .mesh import CubeMesh, cube_mesh, tet_mesh

MU0 = 4e-7 * math.pi


@dataclass
class Evaluation:
    E: float                 # total energy (J)
    terms: dict              # 'ex', 'an', 'z', 'd' (J)
    h: np.ndarray            # (N, 3) mu0 h_eff in tesla
    grad: np.ndarray         # (N, 3) grad phi in units of E0
    torque: float            # max_i |m_i x h_i| / Js
    u1: np.ndarray
    u2: np.ndarray
    uT: np.ndarray


class CubeProblem:
    """One material on one Kuhn cube; evaluates energy, field and gradient."""

    def __init__(self, n: int, Js: float, A: float, K1: float, axis, cell: float = 2e-9,
                 demag: bool = True, mesh: CubeMesh | None = None, B: np.ndarray | None = None):
        self.mesh = mesh if mesh is not None else cube_mesh(n, cell)
        if mesh is not None:
            cell = mesh.cell            # a general mesh carries its own length unit
        self.n, self.cell = n, cell
        self.Js, self.A, self.K1 = Js, A, K1
        self.axis = np.asarray(axis, dtype=np.float64)
        self.axis = self.axis / np.linalg.norm(self.axis)
        self.demag = demag
        self.Kd = Js * Js / (2.0 * MU0)
        self.E0 = self.Kd * cell ** 3
        self.K = self.mesh.stiffness().tocsc()
        self.Kcsr = self.mesh.stiffness()
        self.G = self.mesh.coupling()
        self.Gt = [g.T.tocsr() for g in self.G]
        self.V = self.mesh.volumes()
        N = self.mesh.N
        self.bnd = self.mesh.bnd
        isb = np.zeros(N, dtype=bool)
        isb[self.bnd] = True
        self.interior = np.nonzero(~isb)[0]
        if demag:
            if B is not None:
                self.B = B
            elif self.mesh.n == 0:
                self.B = bem_matrix_general(self.mesh.nodes, self.bnd, self.mesh.tris)
            else:
                self.B = bem_matrix(self.mesh.nodes, n, self.bnd, self.mesh.tris)
            # Neumann problem: fix node 0, solve the reduced SPD system exactly
            self.lu_neu = spla.splu(self.K[1:, 1:].tocsc())
            Kd_ = self.Kcsr
            self.K_II = Kd_[self.interior][:, self.interior].tocsc()
            self.K_IS = Kd_[self.interior][:, self.bnd].tocsr()
            self.K_SI = Kd_[self.bnd][:, self.interior].tocsr()
            self.lu_dir = spla.splu(self.K_II) if self.interior.size else None

    # -- magnetostatics -----------------------------------------------------
    def rhs(self, m: np.ndarray) -> np.ndarray:
        """b_i = sum_j G_ij . m_j = int m . grad phi_i (m^2)."""
        return self.G[0] @ m[:, 0] + self.G[1] @ m[:, 1] + self.G[2] @ m[:, 2]

    def _neumann(self, rhs: np.ndarray) -> np.ndarray:
        """Solution of K u = rhs (rhs made consistent by removing its mean), node 0
        pinned, then the V-weighted mean removed."""
        rhs = rhs - rhs.mean()
        u = np.zeros(rhs.shape[0])
        u[1:] = self.lu_neu.solve(rhs[1:])
        return u - np.dot(self.V, u) / self.V.sum()

    def potential(self, m: np.ndarray):
        b = self.rhs(m)
        u1 = self._neumann(b)
        u2 = np.zeros_like(u1)
        u2[self.bnd] = self.B @ u1[self.bnd]
        if self.interior.size:
            u2[self.interior] = self.lu_dir.solve(-(self.K_IS @ u2[self.bnd]))
        return u1, u2

    def adjoint_potential(self, m: np.ndarray) -> np.ndarray:
        """uT = X^T b, the transposed FEM/BEM chain applied to b = G m."""
        b = self.rhs(m)
        t = b[self.bnd].copy()
        if self.interior.size:
            w = self.lu_dir.solve(b[self.interior])
            t -= self.K_SI @ w
        rhs = b.copy()
        rhs[self.bnd] += self.B.T @ t
        return self._neumann(rhs)

    # -- fields and energies -------------------------------------------------
    def evaluate(self, m: np.ndarray, h_ext) -> Evaluation:
        m = np.asarray(m, dtype=np.float64)
        h_ext = np.asarray(h_ext, dtype=np.float64)
        Js, V = self.Js, self.V
        Km = self.Kcsr @ m                                         # (N, 3)
        h_ex = -(2.0 * self.A * MU0 / Js) * Km / V[:, None]
        ma = m @ self.axis
        h_an = (2.0 * self.K1 * MU0 / Js) * ma[:, None] * self.axis[None, :]
        h_z = np.broadcast_to(h_ext, m.shape)
        if self.demag:
            u1, u2 = self.potential(m)
            uT = self.adjoint_potential(m)
            u = 0.5 * (u1 + u2 + uT)
            h_d = -Js * np.stack([self.Gt[d] @ u for d in range(3)], axis=1) / V[:, None]
        else:
            u1 = u2 = uT = np.zeros(m.shape[0])
            h_d = np.zeros_like(m)
        e_ex = self.A * float(np.sum(m * Km))
        e_an = self.K1 * float(np.dot(V, 1.0 - ma * ma))
        e_z = -(Js / MU0) * float(np.dot(V, m @ h_ext))
        e_d = -(Js / (2.0 * MU0)) * float(np.dot(V, np.sum(m * h_d, axis=1)))
        h = h_ex + h_an + h_z + h_d
        grad = -(Js / MU0) * V[:, None] * h / self.E0
        torque = float(np.max(np.linalg.norm(np.cross(m, h), axis=1))) / Js
        terms = dict(ex=e_ex, an=e_an, z=e_z, d=e_d)
        return Evaluation(E=e_ex + e_an + e_z + e_d, terms=terms, h=h, grad=grad,
                          torque=torque, u1=u1, u2=u2, uT=uT)

    def energy_only(self, m: np.ndarray, h_ext) -> float:
        return self.evaluate(m, h_ext).E

    def mean_m(self, m: np.ndarray) -> np.ndarray:
        return (self.V[:, None] * m).sum(axis=0) / self.V.sum()


def mesh_problem(xyz, tets, Js: float, A: float, K1: float, axis, demag: bool = True) -> CubeProblem:
    """The same problem on a general tetrahedral mesh (coordinates in metres)."""
    mesh = tet_mesh(xyz, tets)
    return CubeProblem(0, Js, A, K1, axis, mesh=mesh, demag=demag)
