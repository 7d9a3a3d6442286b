"""Counter-based seeded input generators (SplitMix64 -> uniforms -> Box-Muller).

SplitMix64 (Steele, Lea, Flood 2014): the k-th output of stream `seed` is
mix(seed + (k+1) * 0x9E3779B97F4A7C15) with the published 64-bit finaliser.
Uniform doubles take the top 53 bits.  Normals come from Box-Muller on
consecutive pairs of uniforms.  Everything is plain numpy uint64 arithmetic,
so the same bytes come out on x86_64 and aarch64 and across numpy versions.

Workloads (all lengths in metres, fields as mu0*H in tesla):
  * material: Nd2Fe14B, Js = 1.61 T, A = 7.7 pJ/m, K1 = 4.3 MJ/m^3
  * cubes of n^3 cells with edge 2 nm, 6 Kuhn tetrahedra per cell
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Nd2Fe14B, the grain material of the paper's Sec. 3.1 experiment.
JS_T = 1.61
A_JM = 7.7e-12
K1_JM3 = 4.3e6
CELL_M = 2.0e-9


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream `seed`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GAMMA * k
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller over consecutive uniform pairs."""
    npair = (count + 1) // 2
    u = uniforms(seed, 2 * npair, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    t = 2.0 * math.pi * u2
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


def _normalise_rows(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cube_nodes(n: int) -> int:
    return (n + 1) ** 3


def m_perturbed(n_nodes: int, seed: int, sigma: float = 0.01,
                base=(0.0, 0.0, 1.0)) -> np.ndarray:
    """m0 = base + N(0, sigma^2) per component, renormalised; shape (N, 3)."""
    g = normals(seed, 3 * n_nodes).reshape(n_nodes, 3)
    return _normalise_rows(np.asarray(base, dtype=np.float64)[None, :] + sigma * g)


def m_random_sphere(n_nodes: int, seed: int) -> np.ndarray:
    """Per-node directions uniform on S^2 (normalised Gaussian triples)."""
    g = normals(seed, 3 * n_nodes).reshape(n_nodes, 3)
    return _normalise_rows(g)


def tilted_axis(polar_deg: float, azimuth: float) -> np.ndarray:
    p = math.radians(polar_deg)
    return np.array([math.sin(p) * math.cos(azimuth), math.sin(p) * math.sin(azimuth),
                     math.cos(p)])


@dataclass
class Instance:
    """One minimisation problem on an n^3-cell cube."""
    n: int
    m0: np.ndarray            # (N, 3) unit vectors
    h_ext: np.ndarray         # (3,) mu0*H_ext in tesla
    axis: np.ndarray          # (3,) unit easy axis
    Js: float = JS_T
    A: float = A_JM
    K1: float = K1_JM3
    cell: float = CELL_M


def single_fp64_case(n: int = 10, seed: int = 1) -> Instance:
    """20 nm cube (10^3 cells), field -6 T at 1 degree from -z, m0 = +z perturbed."""
    N = cube_nodes(n)
    d = math.radians(1.0)
    h = 6.0 * np.array([math.sin(d), 0.0, -math.cos(d)])
    return Instance(n=n, m0=m_perturbed(N, seed), h_ext=h, axis=np.array([0.0, 0.0, 1.0]))


def sweep_case(n: int = 20, seed: int = 2):
    """40 nm cube, easy axis tilted 1 degree (azimuth by seed), field +8 -> -8 T
    along z in 0.1 T steps (161 points), m0 = +z."""
    N = cube_nodes(n)
    az = 2.0 * math.pi * float(uniforms(seed, 1)[0])
    axis = tilted_axis(1.0, az)
    fields = np.round(np.linspace(8.0, -8.0, 161), 12)
    return dict(n=n, m0=np.tile([0.0, 0.0, 1.0], (N, 1)), axis=axis,
                direction=np.array([0.0, 0.0, 1.0]), fields=fields)


def large_case(n: int = 80, seed: int = 3) -> Instance:
    """160 nm cube (80^3 cells), random-angle start, -3 T along z."""
    N = cube_nodes(n)
    return Instance(n=n, m0=m_random_sphere(N, seed), h_ext=np.array([0.0, 0.0, -3.0]),
                    axis=np.array([0.0, 0.0, 1.0]))


def batched_case(n: int = 30, batch: int = 64, seed: int = 4):
    """64 instances on one 60 nm cube: fields U[-8,0] T along z, easy-axis tilt
    U[0,5] degrees with uniform azimuth, m0 = +z perturbed (one stream each)."""
    N = cube_nodes(n)
    u = uniforms(seed, 3 * batch).reshape(batch, 3)
    insts = []
    for b in range(batch):
        hz = -8.0 * u[b, 0]
        axis = tilted_axis(5.0 * u[b, 1], 2.0 * math.pi * u[b, 2])
        m0 = m_perturbed(N, seed * 1000003 + b)
        insts.append(Instance(n=n, m0=m0, h_ext=np.array([0.0, 0.0, hz]), axis=axis))
    return insts


@dataclass
class Request:
    rid: int
    arrival_s: float
    inst: Instance = field(repr=False)


def served_stream(count: int = 512, rate_per_s: float = 20.0, seed: int = 5,
                  n_min: int = 10, n_max: int = 50):
    """Poisson arrivals of minimisation requests: n ~ U{n_min..n_max}, field
    U[-8,8] T along z, axis tilt U[0,10] deg, m0 = +z perturbed."""
    u = uniforms(seed, 5 * count).reshape(count, 5)
    t = 0.0
    reqs = []
    for r in range(count):
        t += -math.log1p(-u[r, 0]) / rate_per_s
        n = n_min + min(int(u[r, 1] * (n_max - n_min + 1)), n_max - n_min)
        hz = -8.0 + 16.0 * u[r, 2]
        axis = tilted_axis(10.0 * u[r, 3], 2.0 * math.pi * u[r, 4])
        m0 = m_perturbed(cube_nodes(n), seed * 7919 + r)
        reqs.append(Request(rid=r, arrival_s=t,
                            inst=Instance(n=n, m0=m0, h_ext=np.array([0.0, 0.0, hz]),
                                          axis=axis)))
    return reqs
