"""The library's packing of the hierarchical boundary matrix for a device
product (csrc/hpack.cu: leaf table sorted by kind and size, FP32 values with V
before U, a first pass t = V x and row owners that sum their entries in
block-tree order), applied to B vectors by a plain reference product in a C++
driver, against the oracle's dense matrix on the CPU: the leaves tile the matrix,
are sorted as stated, and |y - B x|_F <= (eps + FP32 rounding) |B|_F |x|_F."""
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.bem import bem_matrix, bem_matrix_general
from oracle.mesh import cube_mesh, tet_mesh
from paper_1309_5796_gb300 import build as lbm_build
from synth import ball_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib_dir = os.path.dirname(lbm_build.build())
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "hpack_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", *lbm_build.ARCH,
                        "-I", os.path.join(ROOT, "include"), "-I", lbm_build.CSRC,
                        os.path.join(ROOT, "tests", "native", "hpack_check.cpp"), "-L", lib_dir, "-llbm",
                        "-Xlinker", "-rpath", "-Xlinker", lib_dir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(tmp, ignore_errors=True)


def _run(exe, xyz, bnd, tris, x, eps, eta=2.0, n_min=16, threads=4):
    nb, B = x.shape
    with tempfile.TemporaryDirectory() as tmp:
        fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
        with open(fin, "wb") as f:
            f.write(struct.pack("<iiiiii", xyz.shape[0], nb, tris.shape[0], n_min, threads, B))
            f.write(struct.pack("<dd", eta, eps))
            f.write(np.ascontiguousarray(xyz, np.float64).tobytes())
            f.write(np.ascontiguousarray(bnd, np.int32).tobytes())
            f.write(np.ascontiguousarray(tris, np.int32).tobytes())
            f.write(np.ascontiguousarray(x, np.float64).tobytes())
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        raw = open(fout, "rb").read()
    assert raw[:2] == b"ok", raw[:80]
    (nl,) = struct.unpack_from("<i", raw, 2)
    table = np.frombuffer(raw, np.int32, 6 * nl, 6).reshape(nl, 6)
    o = 6 + 24 * nl
    (ni,) = struct.unpack_from("<i", raw, o)
    idx = np.frombuffer(raw, np.int32, ni, o + 4)
    o += 4 + 4 * ni
    y = np.frombuffer(raw, np.float64, nb * B, o).reshape(nb, B)
    assert o + 8 * nb * B == len(raw)
    return table, idx, y


def _surfaces():
    c = cube_mesh(12, 1.0)
    yield "kuhn12", c.nodes.astype(np.float64), c.bnd, c.tris, bem_matrix(c.nodes, 12, c.bnd, c.tris)
    xyz, tets = ball_mesh(10, 1.0)
    t = tet_mesh(xyz, tets)
    yield "ball10", np.asarray(xyz, np.float64), t.bnd, t.tris, bem_matrix_general(t.nodes, t.bnd, t.tris)


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_packed_product_matches_the_dense_matrix(driver, eps):
    rng = np.random.default_rng(9)
    for name, xyz, bnd, tris, B in _surfaces():
        x = rng.normal(size=(bnd.size, 5))
        table, idx, y = _run(driver, xyz, bnd, tris, x, eps)
        # the leaves tile the matrix exactly once and are sorted by (kind, rows, columns)
        cover = np.zeros((bnd.size, bnd.size), dtype=np.int64)
        for rb, m, cb, n, kind, k in table:
            cover[np.ix_(idx[rb:rb + m], idx[cb:cb + n])] += 1
        assert np.all(cover == 1), name
        keys = [tuple(r) for r in table[:, [4, 1, 3]]]
        assert keys == sorted(keys), name
        assert table[:, 4].any() and not table[:, 4].all(), name
        ref = B @ x
        bound = (eps + 1e-6) * np.linalg.norm(B) * np.linalg.norm(x)
        assert np.linalg.norm(y - ref) <= bound, (name, np.linalg.norm(y - ref) / bound)
