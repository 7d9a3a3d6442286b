"""The library's host construction of the hierarchical boundary matrix
(csrc/hbuild.cu: exact dense leaves, adaptive cross approximation with partial
pivoting on the admissible leaves, a sampled residual check with an exact
fallback, recompression of the factors) against the oracle's dense double-layer
matrix, run through a C++ driver on the CPU: the partition is the oracle's,
dense leaves equal the dense matrix's entries, every low-rank leaf is within a
small multiple of its tolerance (the sampled check is statistical), the whole
operator ||B - B_H||_F <= eps ||B||_F, and the storage is
within 15 % of the optimal ranks (the oracle's truncated SVD of every leaf)."""
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import hmatrix as hm
from oracle.bem import bem_matrix, bem_matrix_general
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
    exe = os.path.join(tmp, "hbuild_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", *lbm_build.ARCH,
                        "-I", os.path.join(ROOT, "include"), "-I", lbm_build.CSRC,
                        os.path.join(ROOT, "tests", "native", "hbuild_check.cpp"), "-L", lib_dir, "-llbm",
                        "-Xlinker", "-rpath", "-Xlinker", lib_dir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(tmp, ignore_errors=True)


def _run(exe, xyz, bnd, tris, eta, n_min, eps, threads=4):
    with tempfile.TemporaryDirectory() as tmp:
        fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
        with open(fin, "wb") as f:
            f.write(struct.pack("iiiii", xyz.shape[0], bnd.size, tris.shape[0], n_min, threads))
            f.write(struct.pack("dd", eta, eps))
            f.write(np.ascontiguousarray(xyz, np.float64).tobytes())
            f.write(np.ascontiguousarray(bnd, np.int32).tobytes())
            f.write(np.ascontiguousarray(tris, np.int32).tobytes())
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        raw = open(fout, "rb").read()
    if raw[:6] == b"error ":
        return raw[6:].decode().strip()
    assert raw[:2] == b"ok"
    nl, fallbacks = struct.unpack_from("ii", raw, 2)
    o = 10
    leaves = []
    for _ in range(nl):
        m, n, kind, k = struct.unpack_from("iiii", raw, o)
        o += 16
        rows = np.frombuffer(raw, np.int32, m, o)
        o += 4 * m
        cols = np.frombuffer(raw, np.int32, n, o)
        o += 4 * n
        cnt = k * (m + n) if kind else m * n
        vals = np.frombuffer(raw, np.float64, cnt, o)
        o += 8 * cnt
        if kind:
            leaves.append((rows, cols, True, vals[:m * k].reshape(m, k), vals[m * k:].reshape(k, n)))
        else:
            leaves.append((rows, cols, False, vals.reshape(m, n), None))
    assert o == len(raw)
    return leaves, fallbacks


def _surfaces():
    c = cube_mesh(12, 1.0)
    lat = c.nodes.astype(np.float64)
    yield "kuhn12", lat, c.bnd, c.tris, bem_matrix(c.nodes, 12, c.bnd, c.tris)
    for name, (xyz, tets) in (("jitter8", jittered_cube(8, 1.0, 0.15, seed=4)), ("ball10", ball_mesh(10, 1.0)),
                              ("lshape8", l_shape(8, 1.0))):
        t = tet_mesh(xyz, tets)
        yield name, np.asarray(xyz, np.float64), t.bnd, t.tris, bem_matrix_general(t.nodes, t.bnd, t.tris)


@pytest.mark.parametrize("eps", [1e-4, 1e-8])
def test_native_hmatrix_meets_the_bound_on_the_dense_matrix(driver, eps):
    eta, n_min = 2.0, 16
    n_low = 0
    for name, xyz, bnd, tris, B in _surfaces():
        leaves, fallbacks = _run(driver, xyz, bnd, tris, eta, n_min, eps)
        slo, shi = hm.support_boxes(xyz, bnd, tris)
        ref = hm.block_tree(hm.cluster_tree(xyz[bnd], slo, shi, n_min), eta)
        assert len(leaves) == len(ref), name
        D = np.zeros_like(B)
        scale = np.abs(B).max()
        for (rows, cols, low, X, Y), (tau, sigma, adm) in zip(leaves, ref):
            assert np.array_equal(rows, tau.idx) and np.array_equal(cols, sigma.idx), name
            A = B[np.ix_(rows, cols)]
            if low:
                assert adm, name
                n_low += 1
                approx = X @ Y
                # the sampled check bounds a leaf's error statistically (32 entries), not
                # strictly: a leaf may exceed eps a little; the operator bound below is strict
                assert np.linalg.norm(A - approx) <= 3.0 * eps * np.linalg.norm(A) + 1e-15 * scale, name
                assert X.shape[1] * (rows.size + cols.size) < rows.size * cols.size
            else:
                approx = X
                assert np.abs(A - approx).max() <= 1e-13 * scale, name
            D[np.ix_(rows, cols)] += approx
        assert np.linalg.norm(D - B) <= eps * np.linalg.norm(B), (name, np.linalg.norm(D - B) / np.linalg.norm(B))
        # after recompression the storage is close to the optimal ranks (truncated SVD of every leaf)
        stored = sum(X.size + (Y.size if Y is not None else 0) for (_, _, _, X, Y) in leaves)
        best = hm.build_hmatrix(hm.dense_blocks(B), xyz, bnd, tris, eps=eps, eta=eta, n_min=n_min).stored()
        assert stored <= 1.15 * best, (name, stored / best)
    assert n_low > 0


def test_native_hmatrix_is_independent_of_the_thread_count(driver):
    c = cube_mesh(10, 1.0)
    lat = c.nodes.astype(np.float64)
    one, fb1 = _run(driver, lat, c.bnd, c.tris, 2.0, 16, 1e-6, threads=1)
    many, fb7 = _run(driver, lat, c.bnd, c.tris, 2.0, 16, 1e-6, threads=7)
    assert fb1 == fb7 and len(one) == len(many)
    for a, b in zip(one, many):
        assert a[2] == b[2] and np.array_equal(a[3], b[3])
        assert (a[4] is None and b[4] is None) or np.array_equal(a[4], b[4])


def test_native_hmatrix_rejects_bad_input(driver):
    c = cube_mesh(4, 1.0)
    lat = c.nodes.astype(np.float64)
    assert "eps" in _run(driver, lat, c.bnd, c.tris, 2.0, 16, 0.0)
    assert "eps" in _run(driver, lat, c.bnd, c.tris, 2.0, 16, 1.5)
    bad = c.tris.copy()
    bad[0] = bad[0, [0, 2, 1]]                                # one triangle turned inside out: its fans break
    assert "fan" in _run(driver, lat, c.bnd, bad, 2.0, 16, 1e-6)
