"""The library's host set-up of the space-transformation open boundary
(csrc/shell.cu: grid, shell tensors from the closed-form inverse Jacobian,
tensor-weighted stiffness, Dirichlet rows, magnet map) against the oracle's
ShellProblem (oracle/spacetrans.py, which inverts the Jacobian numerically), run
through a C++ driver on the CPU: identical CSR pattern, outer face, magnet map
and shell count; stiffness values to rounding."""
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.spacetrans import ShellProblem
from paper_1309_5796_gb300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib_dir = os.path.dirname(lbm_build.build())
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "shell_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", *lbm_build.ARCH,
                        "-I", os.path.join(ROOT, "include"), "-I", lbm_build.CSRC,
                        os.path.join(ROOT, "tests", "native", "shell_check.cpp"), "-L", lib_dir, "-llbm",
                        "-Xlinker", "-rpath", "-Xlinker", lib_dir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(tmp, ignore_errors=True)


def _run(exe, n, a, s, cell):
    with tempfile.TemporaryDirectory() as tmp:
        fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
        with open(fin, "wb") as f:
            f.write(struct.pack("<iiid", n, a, s, cell))
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        raw = open(fout, "rb").read()
    if raw[:6] == b"error ":
        return raw[6:].decode().strip()
    assert raw[:2] == b"ok"
    N, nnz, no, nm, nsh = struct.unpack_from("iiiii", raw, 2)
    o = 22
    out = {}
    for key, cnt in (("rowptr", N + 1), ("col", nnz), ("outer", no), ("magnet", nm)):
        out[key] = np.frombuffer(raw, np.int32, cnt, o)
        o += 4 * cnt
    out["K"] = np.frombuffer(raw, np.float64, nnz, o)
    out["shell_tets"] = nsh
    assert o + 8 * nnz == len(raw)
    return out


@pytest.mark.parametrize("n,a,s,cell", [(4, 2, 4, 1.0), (5, 2, 3, 2e-9), (3, 1, 2, 1.0)])
def test_shell_setup_matches_the_oracle(driver, n, a, s, cell):
    got = _run(driver, n, a, s, cell)
    p = ShellProblem(n, 1.61, 7.7e-12, 4.3e6, [0, 0, 1], a, s, cell=cell)
    K = p.Kgrid
    assert np.array_equal(got["rowptr"], K.indptr)
    assert np.array_equal(got["col"], K.indices)
    assert np.abs(got["K"] - K.data).max() <= 1e-13 * np.abs(K.data).max()
    assert np.array_equal(got["outer"], p.outer)
    assert np.array_equal(got["magnet"], p.magnet_in_grid)
    assert got["shell_tets"] == int(p.shell_tets.sum())


def test_shell_setup_rejects_bad_input(driver):
    assert "at least 1" in _run(driver, 4, 0, 4, 1.0)
    assert "positive" in _run(driver, 4, 2, 4, 0.0)
    assert "too large" in _run(driver, 100, 100, 101, 1.0)
