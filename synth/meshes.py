"""Seeded unstructured tetrahedral meshes (input geometry for the general-mesh path).

Two families, both built from a 5-tetrahedra split of n^3 cubes (a central
tetrahedron on four alternate corners plus four corner tetrahedra; the choice
of corners alternates with the parity of the cell so that neighbouring cells
share face diagonals).  This topology differs from the 6-tetrahedra split the
library uses for its own cube meshes, so the general path sees other element
shapes and another sparsity pattern.

  * jittered_cube: the interior nodes of the cube moved by up to `amp` cells
    per coordinate (seeded); surface nodes stay on the six faces.
  * ball_mesh: the cube [-1, 1]^3 mapped onto the unit ball by the elliptical
    cube-to-sphere map x' = x sqrt(1 - y^2/2 - z^2/2 + y^2 z^2/3) (cyclic),
    then scaled to the requested diameter.  The surface nodes land on the
    sphere.  With n = 24 this is an 82 944-tetrahedra ball, the size of the
    20 nm Nd2Fe14B grain mesh of the paper's experiment (Sec. 3.1).

Both return (xyz (N, 3) float64 metres, tets (T, 4) int32) with every
tetrahedron positively oriented.  No arithmetic of the minimisation method
lives here.
"""
from __future__ import annotations

import numpy as np

from .inputs import uniforms


def _five_tet_split(n: int):
    """Lattice nodes (N, 3) int and tetrahedra (5 n^3, 4) of the alternating
    5-tetrahedra split of the n^3 cube lattice, node id i + (n+1)(j + (n+1)k)."""
    n1 = n + 1
    g = np.arange(n1)
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def nid(x, y, z):
        return x + n1 * (y + n1 * z)

    even = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    odd = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]

    def tets_of(a, b):
        # central tetrahedron on corners `a`; each corner of `b` with its three
        # neighbours in `a` (the corners at lattice distance 1)
        out = [a]
        for c in b:
            nb = [p for p in a if sum(abs(p[d] - c[d]) for d in range(3)) == 1]
            out.append([c] + nb)
        return out

    pattern = {0: tets_of(even, odd), 1: tets_of(odd, even)}
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    par = (cx + cy + cz) % 2
    tets = np.empty((n ** 3, 5, 4), dtype=np.int64)
    for p in (0, 1):
        sel = par == p
        for t, corners in enumerate(pattern[p]):
            for v, (dx, dy, dz) in enumerate(corners):
                tets[sel, t, v] = nid(cx[sel] + dx, cy[sel] + dy, cz[sel] + dz)
    return nodes, tets.reshape(-1, 4)


def _orient(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    P = xyz[tets]
    det = np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))
    if np.any(det == 0.0):
        raise ValueError("degenerate tetrahedron")
    tets = tets.copy()
    neg = det < 0
    tets[neg] = tets[neg][:, [0, 1, 3, 2]]
    return tets.astype(np.int32)


def jittered_cube(n: int, cell: float = 2e-9, amp: float = 0.1, seed: int = 6):
    """n^3 cells of edge `cell`; interior nodes moved by U[-amp, amp] cells per
    coordinate (SplitMix64 stream `seed`)."""
    nodes, tets = _five_tet_split(n)
    xyz = nodes.astype(np.float64)
    inner = np.all((nodes > 0) & (nodes < n), axis=1)
    u = uniforms(seed, 3 * nodes.shape[0]).reshape(-1, 3)
    xyz[inner] += amp * (2.0 * u[inner] - 1.0)
    xyz *= cell
    return xyz, _orient(xyz, tets)


def l_shape(n: int, cell: float = 2e-9):
    """The n^3 cube lattice without the cells with i >= n/2 and j >= n/2: an
    L-shaped prism (a non-convex body with a reflex edge along z), 5-tetrahedra
    split, unused nodes removed and the rest renumbered in order."""
    if n < 2 or n % 2:
        raise ValueError("l_shape needs an even n >= 2")
    nodes, tets = _five_tet_split(n)
    h = n // 2
    cells = np.arange(n ** 3)
    cx, cy = cells % n, (cells // n) % n
    keep_cell = ~((cx >= h) & (cy >= h))
    tets = tets.reshape(n ** 3, 5, 4)[keep_cell].reshape(-1, 4)
    used = np.unique(tets)
    new_id = -np.ones(nodes.shape[0], dtype=np.int64)
    new_id[used] = np.arange(used.size)
    xyz = nodes[used].astype(np.float64) * cell
    return xyz, _orient(xyz, new_id[tets])


def ball_mesh(n: int, diameter: float = 20e-9):
    """The n^3 lattice of [-1, 1]^3 mapped onto a ball of the given diameter."""
    if n < 2 or n % 2:
        raise ValueError("ball_mesh needs an even n >= 2")
    nodes, tets = _five_tet_split(n)
    p = nodes.astype(np.float64) * (2.0 / n) - 1.0
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    q = np.stack([x * np.sqrt(1.0 - y * y / 2 - z * z / 2 + y * y * z * z / 3),
                  y * np.sqrt(1.0 - z * z / 2 - x * x / 2 + z * z * x * x / 3),
                  z * np.sqrt(1.0 - x * x / 2 - y * y / 2 + x * x * y * y / 3)], axis=1)
    xyz = q * (0.5 * diameter)
    return xyz, _orient(xyz, tets)
