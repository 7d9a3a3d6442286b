"""Writes the oracle's reference results used by the GPU parity tests.

Calls only the FP64 oracle (oracle/) and the seeded input generators (synth/);
nothing here touches the CUDA path.  Outputs JSON files beside this script:

  batched_n30.json   per-instance minimisation results of the batched workload
                     (64 instances on the 30^3-cell cube, seed 4)
  sweep_n20.json     the hysteresis sweep of the 20^3-cell cube (seed 2),
                     +8 -> -8 T in 0.1 T steps, warm-started
  sphere_paper.json  the minimisation on the paper-size 20 nm sphere (87 880
                     tetrahedra) from a random state (seed 8) at -3 T along z

Usage: python tests/golden/make_golden.py [batched|sweep|sphere] [--procs P]
"""
from __future__ import annotations

import copy
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle.micromag import CubeProblem  # noqa: E402
from oracle.minimise import hysteresis, minimise  # noqa: E402
from synth.inputs import batched_case, sweep_case, A_JM, JS_T, K1_JM3  # noqa: E402

_BASE = None
_INSTS = None


def _solve(b):
    inst = _INSTS[b]
    p = copy.copy(_BASE)
    p.axis = inst.axis / np.linalg.norm(inst.axis)
    t0 = time.time()
    r = minimise(p, inst.m0, inst.h_ext, tol=1e-6, max_iter=20000)
    return dict(b=b, status=r.status, iterations=r.iterations, evaluations=r.evaluations,
                line_searches=r.line_searches, E=r.E, terms=r.terms, torque=r.torque,
                mean_m=p.mean_m(r.m).tolist(), h_ext=inst.h_ext.tolist(), axis=inst.axis.tolist(),
                seconds=time.time() - t0)


def batched(procs: int):
    global _BASE, _INSTS
    _INSTS = batched_case(30, 64, seed=4)
    _BASE = CubeProblem(30, JS_T, A_JM, K1_JM3, _INSTS[0].axis)
    with mp.get_context("fork").Pool(procs) as pool:
        out = pool.map(_solve, range(len(_INSTS)), chunksize=1)
    json.dump(dict(n=30, batch=64, seed=4, tol=1e-6, results=out),
              open(os.path.join(HERE, "batched_n30.json"), "w"), indent=1)


def sweep():
    c = sweep_case(20, seed=2)
    p = CubeProblem(20, JS_T, A_JM, K1_JM3, c["axis"])
    mpar, energy, res = hysteresis(p, c["m0"], c["direction"], c["fields"], tol=1e-6, max_iter=20000)
    json.dump(dict(n=20, seed=2, axis=c["axis"].tolist(), fields=c["fields"].tolist(),
                   m_par=mpar.tolist(), energy=energy.tolist(),
                   status=[r.status for r in res], iterations=[r.iterations for r in res]),
              open(os.path.join(HERE, "sweep_n20.json"), "w"), indent=1)


def sphere():
    from oracle.micromag import mesh_problem
    from synth.inputs import m_random_sphere
    from synth.meshes import ball_mesh
    xyz, tets = ball_mesh(26, 20e-9)
    p = mesh_problem(xyz, tets, JS_T, A_JM, K1_JM3, [0.0, 0.0, 1.0])
    m0 = m_random_sphere(p.mesh.N, 8)
    h = np.array([0.0, 0.0, -3.0])
    t0 = time.time()
    r = minimise(p, m0, h, tol=1e-6, max_iter=20000)
    json.dump(dict(mesh="ball_mesh(26, 20e-9)", seed=8, h_ext=h.tolist(), tol=1e-6, status=r.status,
                   iterations=r.iterations, evaluations=r.evaluations, E=r.E, terms=r.terms,
                   torque=r.torque, mean_m=p.mean_m(r.m).tolist(), seconds=time.time() - t0),
              open(os.path.join(HERE, "sphere_paper.json"), "w"), indent=1)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "batched"
    procs = int(sys.argv[sys.argv.index("--procs") + 1]) if "--procs" in sys.argv else os.cpu_count()
    if what == "batched":
        batched(procs)
    elif what == "sweep":
        sweep()
    elif what == "sphere":
        sphere()
