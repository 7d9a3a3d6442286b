"""CPU-side checks of the C ABI: the library builds, loads, and exports every
symbol include/lbm.h declares, with a binding for each (no GPU calls)."""
import os
import re

import pytest

import paper_1309_5796_gb300 as lbm
from paper_1309_5796_gb300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def library():
    lbm_build.build()
    return lbm.lib()


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for s in ("lbm_create", "lbm_mesh_cube", "lbm_instance_create", "lbm_set_field", "lbm_minimise",
              "lbm_hysteresis", "lbm_get_m", "lbm_evaluate"):
        assert s in syms


def test_library_exports_every_declared_symbol(library):
    for s in _declared_symbols():
        assert hasattr(library, s), s


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in lbm.SIGNATURES}
    assert set(_declared_symbols()) == bound


def test_struct_sizes_match_header(library):
    import ctypes as C
    assert C.sizeof(lbm.Material) == 6 * 8
    assert C.sizeof(lbm.Result) == 4 * 4 + 2 * 8 + 5 * 8 + 2 * 8 + 3 * 8 + 8
    o = lbm.default_opts(lbm.LBM_FP64)
    assert o.memory == 20 and o.tol == 1e-6 and o.max_backtracks == 30 and o.m_alpha == 3
    assert lbm.default_opts(lbm.LBM_MIXED).cg_tol > o.cg_tol


def test_create_without_gpu_fails_cleanly(library):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm.LBMError):
        lbm.Context(0)


def test_header_is_plain_c():
    """include/lbm.h is a C interface: it compiles as C99 and as C++17."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    hdr = os.path.join(ROOT, "include", "lbm.h")
    for args in (["-std=c99", "-x", "c"], ["-std=c++17", "-x", "c++"]):
        r = subprocess.run([gcc, "-fsyntax-only", "-Wall", "-Wextra", "-Werror", *args, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_c_client_builds_and_runs():
    """tests/c_client/minimise.c, a plain C99 program using only include/lbm.h,
    compiles and links against liblbm.so; run, it either minimises (a GPU is
    present: exit 0) or reports the failed context creation cleanly (no GPU:
    exit 1 with the library's message), never crashes."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib_dir = os.path.dirname(lbm_build.build())
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "minimise")
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "c_client", "minimise.c"), "-L", lib_dir, "-llbm", "-lm",
                            "-Wl,-rpath," + lib_dir, "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        if run.returncode == 0:
            assert run.stdout.count("status 0") == 2
        else:
            assert run.returncode == 1 and "lbm_create" in run.stderr, (run.returncode, run.stderr)


def test_ctypes_structs_match_the_header():
    """Every ctypes structure of the binding has the C struct's field names in the
    same order, the same offsets and the same size (checked by compiling a C
    program that prints offsetof/sizeof from include/lbm.h)."""
    import json
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    pairs = [("lbm_material", lbm.Material), ("lbm_solve_opts", lbm.SolveOpts), ("lbm_result", lbm.Result),
             ("lbm_profile_stats", lbm.ProfileStats), ("lbm_request", lbm.Request),
             ("lbm_serve_opts", lbm.ServeOpts)]
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "lbm.h"', "int main(void) {", 'printf("{");']
    for k, (cname, py) in enumerate(pairs):
        sep = "," if k else ""
        src.append(f'printf("{sep}\\"{cname}\\": {{\\"size\\": %zu, \\"fields\\": [", sizeof({cname}));')
        for j, (fname, _) in enumerate(py._fields_):
            fsep = "," if j else ""
            src.append(f'printf("{fsep}[\\"{fname}\\", %zu]", offsetof({cname}, {fname}));')
        src.append('printf("]}");')
    src += ['printf("}\\n");', "return 0; }"]
    with tempfile.TemporaryDirectory() as tmp:
        c_file, exe = os.path.join(tmp, "layout.c"), os.path.join(tmp, "layout")
        open(c_file, "w").write("\n".join(src))
        r = subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), c_file, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr     # a field missing from the C struct fails here
        layout = json.loads(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)
    for cname, py in pairs:
        c = layout[cname]
        assert c["size"] == ctypes_sizeof(py), (cname, c["size"], ctypes_sizeof(py))
        for (fname, off) in c["fields"]:
            assert getattr(py, fname).offset == off, (cname, fname, off, getattr(py, fname).offset)


def ctypes_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)


def test_binding_argument_counts_match_the_header():
    """Each prototype in include/lbm.h has as many parameters as the binding's
    argtypes for that symbol (a wrong count would misread arguments silently)."""
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(?:int|void|const char\*)\s+(lbm_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = m.group(2).strip()
        protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    assert len(protos) == len(lbm.SIGNATURES)
    for name, _, args in lbm.SIGNATURES:
        assert protos[name] == len(args), (name, protos[name], len(args))


def test_default_options_are_the_documented_ones(library):
    """lbm_default_opts and lbm_default_serve_opts fill in what include/lbm.h
    documents (no GPU needed)."""
    import ctypes as C
    common = dict(tol=1e-6, grad_tol=0.0, memory=20, c1=1e-4, max_backtracks=30, kappa0=0.5, m_alpha=3,
                  switch_tol=1e-4, cg_tol_polish=1e-10, bb_rule=0, method=0, omega=1.0, demag=1, resume=0)
    per = {lbm.LBM_FP64: dict(cg_tol=1e-13, cg_mixed_iter=0, stall_iters=0, cg_tol_fp32=0.0),
           lbm.LBM_MIXED: dict(cg_tol=1e-6, cg_mixed_iter=1, stall_iters=200, cg_tol_fp32=3e-5),
           lbm.LBM_MIXED_TC: dict(cg_tol=1e-6, cg_mixed_iter=1, stall_iters=200, cg_tol_fp32=3e-5)}
    for prec, extra in per.items():
        o = lbm.default_opts(prec)
        for k, v in {**common, **extra}.items():
            assert getattr(o, k) == v, (prec, k, getattr(o, k))
    assert lbm.LBM_MIXED_TF32 == lbm.LBM_MIXED_TC
    s = lbm.ServeOpts()
    library.lbm_default_serve_opts(C.byref(s))
    assert (s.slots, s.chunk, s.max_pcg_blocks, s.mem_reserve) == (16, 8, 0, 0.05)
    assert s.opt.cg_mixed_iter == 1 and s.opt.stall_iters == 200


def test_failed_call_leaves_its_message(library):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm.LBMError) as e:
        lbm.Context(0)
    msg = library.lbm_last_error().decode()
    assert msg and msg in str(e.value)
