"""The library's native host topology of a general tetrahedral mesh (the part of
lbm_mesh_upload that runs on the CPU: validation, CSR pattern, outward surface,
surface ids, length unit), run through a small C++ driver and compared with the
CPU oracle's tet_mesh -- bit-identical index structures, L to rounding."""
import os
import re
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.mesh import cube_mesh, tet_mesh
from paper_1309_5796_gb300 import build as lbm_build
from synth import ball_mesh, jittered_cube, l_shape

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib_dir = os.path.dirname(lbm_build.build())
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "topology_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", *lbm_build.ARCH,
                        "-I", os.path.join(ROOT, "include"), "-I", lbm_build.CSRC,
                        os.path.join(ROOT, "tests", "native", "topology_check.cpp"), "-L", lib_dir, "-llbm",
                        "-Xlinker", "-rpath", "-Xlinker", lib_dir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(tmp, ignore_errors=True)


def _run(exe, xyz, tets):
    with tempfile.TemporaryDirectory() as tmp:
        fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
        with open(fin, "wb") as f:
            f.write(struct.pack("ii", xyz.shape[0], tets.shape[0]))
            f.write(np.ascontiguousarray(xyz, np.float64).tobytes())
            f.write(np.ascontiguousarray(tets, np.int32).tobytes())
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stderr
        raw = open(fout, "rb").read()
    if raw[:6] == b"error ":
        return raw[6:].decode().strip()
    assert raw[:2] == b"ok"
    counts = np.frombuffer(raw[2:18], np.int32)
    o = 18
    parts = []
    for c in counts:
        parts.append(np.frombuffer(raw[o:o + 4 * int(c)], np.int32))
        o += 4 * int(c)
    L = struct.unpack("d", raw[o:o + 8])[0]
    return dict(rowptr=parts[0], col=parts[1], tris=parts[2].reshape(-1, 3), bidx=parts[3], L=L)


@pytest.mark.parametrize("mesh", ["ball", "jitter", "lshape", "kuhn"])
def test_topology_matches_oracle(driver, mesh):
    if mesh == "ball":
        xyz, tets = ball_mesh(6, 12e-9)
    elif mesh == "jitter":
        xyz, tets = jittered_cube(4, 2e-9, 0.12, seed=5)
    elif mesh == "lshape":
        xyz, tets = l_shape(4, 2e-9)
    else:
        c = cube_mesh(4, 2e-9)
        xyz, tets = c.xyz(), c.tets
    got = _run(driver, xyz, tets)
    ref = tet_mesh(xyz, tets)
    assert np.array_equal(got["rowptr"], ref.ops.indptr)
    assert np.array_equal(got["col"], ref.ops.indices)
    assert np.array_equal(got["tris"], ref.tris)
    assert np.array_equal(got["bidx"], ref.bnd)
    assert abs(got["L"] / ref.cell - 1.0) < 1e-14


def test_topology_rejects_invalid_meshes(driver):
    xyz, tets = jittered_cube(2, 1e-9, 0.1, seed=2)
    t = tets.copy()
    t[0, 0] = xyz.shape[0]
    assert "outside" in _run(driver, xyz, t)
    t = tets.copy()
    t[1, 1] = t[1, 0]
    assert "repeats node" in _run(driver, xyz, t)
    x = xyz.copy()
    x[tets[2, 1]] = x[tets[2, 0]]
    assert "degenerate" in _run(driver, x, tets)
    assert "belongs to no tetrahedron" in _run(driver, np.vstack([xyz, [[1.0, 1.0, 1.0]]]), tets)
    msg = _run(driver, xyz, np.vstack([tets, tets[:1]]))    # every face of tet 0 now in 2 or 3 cells
    assert re.search(r"belongs to [3-9] tetrahedra", msg), msg
