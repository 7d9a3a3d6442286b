"""The library's host set-up of the hierarchical boundary matrix (support
boxes, cluster tree, block-tree leaves with their admissibility: index and
comparison work) is identical, bit for bit, to the oracle's
(oracle/hmatrix.py), run through a small C++ driver on the CPU."""
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import hmatrix as hm
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
    exe = os.path.join(tmp, "hpartition_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", *lbm_build.ARCH,
                        "-I", os.path.join(ROOT, "include"), "-I", lbm_build.CSRC,
                        os.path.join(ROOT, "tests", "native", "hpartition_check.cpp"), "-L", lib_dir, "-llbm",
                        "-Xlinker", "-rpath", "-Xlinker", lib_dir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(tmp, ignore_errors=True)


def _run(exe, xyz, bnd, tris, eta, n_min):
    with tempfile.TemporaryDirectory() as tmp:
        fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
        with open(fin, "wb") as f:
            f.write(struct.pack("iiii", xyz.shape[0], bnd.size, tris.shape[0], n_min))
            f.write(struct.pack("d", eta))
            f.write(np.ascontiguousarray(xyz, np.float64).tobytes())
            f.write(np.ascontiguousarray(bnd, np.int32).tobytes())
            f.write(np.ascontiguousarray(tris, np.int32).tobytes())
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        raw = open(fout, "rb").read()
    if raw[:6] == b"error ":
        return raw[6:].decode().strip()
    assert raw[:2] == b"ok"
    nb = bnd.size
    o = 2
    lo = np.frombuffer(raw[o:o + 24 * nb], np.float64).reshape(nb, 3)
    o += 24 * nb
    hi = np.frombuffer(raw[o:o + 24 * nb], np.float64).reshape(nb, 3)
    o += 24 * nb
    (nc,) = struct.unpack_from("i", raw, o)
    o += 4
    clusters = []
    for _ in range(nc):
        (sz,) = struct.unpack_from("i", raw, o)
        o += 4
        clusters.append(np.frombuffer(raw[o:o + 4 * sz], np.int32))
        o += 4 * sz
    (nl,) = struct.unpack_from("i", raw, o)
    o += 4
    leaves = np.frombuffer(raw[o:o + 12 * nl], np.int32).reshape(nl, 3)
    return lo, hi, clusters, leaves


def _oracle_bfs(root):
    order, q = [], [root]
    while q:
        c = q.pop(0)
        order.append(c)
        q.extend(c.children)
    return order


def _surfaces():
    c = cube_mesh(12, 2e-9)
    yield "kuhn12", c.xyz(), c.bnd, c.tris
    for name, (xyz, tets) in (("ball10", ball_mesh(10, 10e-9)), ("jitter8", jittered_cube(8, 2e-9, 0.15, seed=4)),
                              ("lshape6", l_shape(6, 2e-9))):
        t = tet_mesh(xyz, tets)
        yield name, np.asarray(xyz, np.float64), t.bnd, t.tris


@pytest.mark.parametrize("eta,n_min", [(2.0, 16), (1.0, 32), (0.5, 7)])
def test_partition_is_identical_to_the_oracle(driver, eta, n_min):
    n_low = 0
    for name, xyz, bnd, tris in _surfaces():
        lo, hi, clusters, leaves = _run(driver, xyz, bnd, tris, eta, n_min)
        slo, shi = hm.support_boxes(xyz, bnd, tris)
        assert np.array_equal(lo, slo) and np.array_equal(hi, shi), name
        root = hm.cluster_tree(xyz[bnd], slo, shi, n_min)
        bfs = _oracle_bfs(root)
        assert len(bfs) == len(clusters), name
        for a, b in zip(bfs, clusters):
            assert np.array_equal(a.idx, b), name
        ident = {id(c): k for k, c in enumerate(bfs)}
        ref = np.array([(ident[id(t)], ident[id(s)], int(low)) for t, s, low in hm.block_tree(root, eta)])
        assert np.array_equal(leaves, ref), name
        n_low += int(leaves[:, 2].sum())
    assert n_low > 0


def test_partition_rejects_bad_input(driver):
    c = cube_mesh(4, 1.0)
    xyz, bnd, tris = c.xyz(), c.bnd, c.tris
    assert "eta" in _run(driver, xyz, bnd, tris, 0.0, 16)
    assert "eta" in _run(driver, xyz, bnd, tris, float("nan"), 16)
    assert "n_min" in _run(driver, xyz, bnd, tris, 2.0, 0)
    assert "no boundary" in _run(driver, xyz, bnd[:0], tris[:0], 2.0, 16)
    x = xyz.copy()
    x[bnd[3], 0] = np.inf
    assert "outside its support box" in _run(driver, x, bnd, tris, 2.0, 16)
