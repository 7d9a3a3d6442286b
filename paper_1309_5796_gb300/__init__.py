"""Python binding of liblbm, the GB300 curvilinear steepest-descent micromagnetic
minimiser (Exl et al., "LaBonte's method revisited", arXiv:1309.5796).

Thin ctypes marshalling over the C ABI of include/lbm.h: every call here maps
one-to-one onto an `lbm_*` entry point, and all computation happens in the
library's CUDA kernels.  There is no CPU fallback: importing `lib()` fails
loudly when liblbm.so has not been built (run `python -m
paper_1309_5796_gb300.build`).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblbm.so")

LBM_OK, LBM_E_INVALID, LBM_E_OOM, LBM_E_NOT_CONVERGED = 0, 1, 2, 3
LBM_E_NAN, LBM_E_TIMEOUT, LBM_E_LINESEARCH, LBM_E_CUDA, LBM_E_PENDING = 4, 5, 6, 7, 8
LBM_FP64, LBM_MIXED, LBM_MIXED_TC = 0, 1, 2
LBM_MIXED_TF32 = LBM_MIXED_TC
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "NOT_CONVERGED", 4: "NAN", 5: "TIMEOUT",
                6: "LINESEARCH", 7: "CUDA", 8: "PENDING"}


class Material(C.Structure):
    _fields_ = [("Js", C.c_double), ("A", C.c_double), ("K1", C.c_double), ("axis", C.c_double * 3)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("grad_tol", C.c_double), ("max_iter", C.c_int32),
                ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32), ("c1", C.c_double),
                ("max_backtracks", C.c_int32), ("memory", C.c_int32), ("kappa0", C.c_double),
                ("m_alpha", C.c_int32), ("tau_min", C.c_double), ("tau_max", C.c_double),
                ("demag", C.c_int32), ("check_every", C.c_int32), ("switch_tol", C.c_double),
                ("cg_tol_polish", C.c_double), ("cg_mixed_iter", C.c_int32), ("bb_rule", C.c_int32),
                ("method", C.c_int32), ("omega", C.c_double), ("stall_iters", C.c_int32),
                ("pcg_kernel", C.c_int32), ("use_graphs", C.c_int32), ("cg_tol_fp32", C.c_double),
                ("resume", C.c_int32)]


class ProfileStats(C.Structure):
    _fields_ = [("launches", C.c_int64 * 8), ("ms", C.c_double * 8), ("cg_iters", C.c_int64 * 2),
                ("cg_sweeps", C.c_int64 * 4)]


PROFILE_KINDS = ("trial_update", "pcg1_fp32", "bem_product", "pcg2_fp32", "field", "decide",
                 "pcg1_fp64", "pcg2_fp64")


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("evaluations", C.c_int32),
                ("line_searches", C.c_int32), ("cg_iters1", C.c_int64), ("cg_iters2", C.c_int64),
                ("energy", C.c_double * 5), ("torque", C.c_double), ("gg", C.c_double),
                ("mean_m", C.c_double * 3), ("wall_ms", C.c_double)]

    def as_dict(self):
        return dict(status=self.status, iterations=self.iterations, evaluations=self.evaluations,
                    line_searches=self.line_searches, cg_iters1=self.cg_iters1,
                    cg_iters2=self.cg_iters2, energy=list(self.energy), torque=self.torque,
                    gg=self.gg, mean_m=list(self.mean_m), wall_ms=self.wall_ms)


class Request(C.Structure):
    _fields_ = [("n", C.c_int32), ("cell_m", C.c_double), ("mat", Material), ("h", C.c_double * 3),
                ("m0", C.POINTER(C.c_double)), ("precision", C.c_int32)]


class ServeOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("chunk", C.c_int32), ("max_pcg_blocks", C.c_int32),
                ("mem_reserve", C.c_double), ("opt", SolveOpts), ("shell_a", C.c_int32),
                ("shell_s", C.c_int32)]


_P = C.c_void_p
_I64 = C.c_int64
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)

# (name, restype, argtypes) of every exported symbol of include/lbm.h
SIGNATURES = [
    ("lbm_default_opts", None, [C.POINTER(SolveOpts), C.c_int32]),
    ("lbm_create", C.c_int, [C.POINTER(_P), C.c_int32, _P]),
    ("lbm_destroy", C.c_int, [_P]),
    ("lbm_last_error", C.c_char_p, []),
    ("lbm_mesh_cube", C.c_int, [_P, C.c_double, C.c_int32, C.POINTER(_I64)]),
    ("lbm_mesh_upload", C.c_int, [_P, _DP, _I64, _IP, _I64, C.POINTER(_I64)]),
    ("lbm_mesh_values", C.c_int, [_P, _I64, _DP, _DP, _DP, _DP, _DP]),
    ("lbm_energy", C.c_int, [_P, _I64, _DP]),
    ("lbm_mesh_destroy", C.c_int, [_P, _I64]),
    ("lbm_mesh_info", C.c_int, [_P, _I64, C.POINTER(_I64)]),
    ("lbm_mesh_export", C.c_int, [_P, _I64] + [_IP] * 9),
    ("lbm_bem_rows", C.c_int, [_P, _I64, _I64, _I64, _DP]),
    ("lbm_hmatrix_plan", C.c_int, [_DP, _I64, _IP, _I64, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                   C.POINTER(_I64)]),
    ("lbm_instance_create", C.c_int, [_P, _I64, C.c_int32, C.c_int32, C.POINTER(_I64)]),
    ("lbm_instance_destroy", C.c_int, [_P, _I64]),
    ("lbm_set_material", C.c_int, [_P, _I64, C.POINTER(Material)]),
    ("lbm_set_field", C.c_int, [_P, _I64, _DP]),
    ("lbm_set_m", C.c_int, [_P, _I64, _DP]),
    ("lbm_get_m", C.c_int, [_P, _I64, _DP]),
    ("lbm_evaluate", C.c_int, [_P, _I64, C.POINTER(SolveOpts), _DP, _DP, C.POINTER(Result)]),
    ("lbm_minimise", C.c_int, [_P, _I64, C.POINTER(SolveOpts), C.POINTER(Result)]),
    ("lbm_hysteresis", C.c_int, [_P, _I64, _DP, _DP, C.c_int32, C.POINTER(SolveOpts), _DP, _DP,
                                 C.POINTER(Result)]),
    ("lbm_launch_count", C.c_int, [_P, C.POINTER(_I64)]),
    ("lbm_set_m_device", C.c_int, [_P, _I64, C.c_void_p]),
    ("lbm_profile_enable", C.c_int, [_P, C.c_int32]),
    ("lbm_profile_read", C.c_int, [_P, C.POINTER(ProfileStats), C.c_int32]),
    ("lbm_evaluate_noalloc", C.c_int, [_P, _I64, C.POINTER(Material), _DP, C.POINTER(SolveOpts),
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_set_wait_limit", C.c_int, [_P, C.c_double, C.c_int32]),
    ("lbm_graph_stats", C.c_int, [_P, C.POINTER(_I64)]),
    ("lbm_serve_trace", C.c_int, [_P, _DP, _I64, C.POINTER(_I64)]),
    ("lbm_mesh_hmatrix", C.c_int, [_P, _I64, C.c_double, C.c_double, C.c_int32, C.c_int32, C.POINTER(_I64)]),
    ("lbm_mesh_shell", C.c_int, [_P, _I64, C.c_int32, C.c_int32, C.POINTER(_I64)]),
    ("lbm_get_state", C.c_int, [_P, _I64, C.c_void_p, C.POINTER(_I64)]),
    ("lbm_set_state", C.c_int, [_P, _I64, C.c_void_p, _I64]),
    ("lbm_bem_apply", C.c_int, [_P, _I64, C.c_int32, C.c_int32, _DP, _DP, _DP]),
    ("lbm_default_serve_opts", None, [C.POINTER(ServeOpts)]),
    ("lbm_serve_start", C.c_int, [_P, C.POINTER(ServeOpts)]),
    ("lbm_submit", C.c_int, [_P, C.POINTER(Request), C.POINTER(_I64)]),
    ("lbm_poll", C.c_int, [_P, _I64, C.POINTER(Result), _DP]),
    ("lbm_wait", C.c_int, [_P, _I64, C.c_double, C.POINTER(Result), _DP]),
    ("lbm_serve_stats", C.c_int, [_P, C.POINTER(_I64)]),
    ("lbm_serve_stop", C.c_int, [_P]),
]

_lib = None


def lib():
    """The loaded liblbm.so with typed signatures (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblbm.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_1309_5796_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, lib().lbm_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(_IP) if a is not None else None


def default_opts(precision=LBM_FP64, **kw) -> SolveOpts:
    o = SolveOpts()
    lib().lbm_default_opts(C.byref(o), precision)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def hmatrix_plan(xyz, tets, eps: float = 1e-6, eta: float = 2.0, n_min: int = 16, threads: int | None = None) -> dict:
    """Storage of the hierarchical form of the mesh's boundary matrix (lbm_hmatrix_plan;
    host only, no GPU): stored values, the dense matrix's nb^2, leaves, low-rank leaves."""
    x = np.ascontiguousarray(np.asarray(xyz, np.float64))
    t = np.ascontiguousarray(np.asarray(tets, np.int32))
    out = (C.c_int64 * 4)()
    th = threads if threads is not None else max(1, os.cpu_count() or 1)
    _check(lib().lbm_hmatrix_plan(_dptr(x), x.shape[0], _iptr(t), t.shape[0], eps, eta, n_min, th, out))
    return dict(stored=out[0], dense=out[1], leaves=out[2], low_rank=out[3], fraction=out[0] / out[1])


class Context:
    """A liblbm context on one CUDA device (lbm_create / lbm_destroy)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._h = _P()
        _check(lib().lbm_create(C.byref(self._h), device, stream))

    def close(self):
        if self._h:
            lib().lbm_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- meshes --------------------------------------------------------------
    def mesh_cube(self, cell_m: float, n: int) -> int:
        h = _I64()
        _check(lib().lbm_mesh_cube(self._h, cell_m, n, C.byref(h)))
        return h.value

    def mesh_upload(self, xyz, tets) -> int:
        """A general tetrahedral mesh: xyz (N, 3) metres, tets (T, 4) node ids."""
        x = np.ascontiguousarray(np.asarray(xyz, np.float64))
        t = np.ascontiguousarray(np.asarray(tets, np.int32))
        if x.ndim != 2 or x.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 4:
            raise ValueError("xyz must be (N, 3) and tets (T, 4)")
        h = _I64()
        _check(lib().lbm_mesh_upload(self._h, _dptr(x), x.shape[0], _iptr(t), t.shape[0], C.byref(h)))
        return h.value

    def mesh_values(self, mesh: int) -> dict:
        """FP64 operators in SI units: K (nnz,), G, Gt (nnz, 3), V (N,), unit (m)."""
        i = self.mesh_info(mesh)
        out = dict(K=np.empty(i["nnz"]), G=np.empty((i["nnz"], 3)), Gt=np.empty((i["nnz"], 3)),
                   V=np.empty(i["N"]))
        unit = C.c_double()
        _check(lib().lbm_mesh_values(self._h, mesh, _dptr(out["K"]), _dptr(out["G"]), _dptr(out["Gt"]),
                                     _dptr(out["V"]), C.byref(unit)))
        out["unit"] = unit.value
        return out

    def mesh_destroy(self, mesh: int):
        _check(lib().lbm_mesh_destroy(self._h, mesh))

    def mesh_info(self, mesh: int) -> dict:
        info = (_I64 * 8)()
        _check(lib().lbm_mesh_info(self._h, mesh, info))
        keys = ("N", "nb", "nnz", "tets", "tris", "bytes", "n")
        return {k: int(info[i]) for i, k in enumerate(keys)}

    def mesh_export(self, mesh: int) -> dict:
        """Topology and (cube meshes) the integer tables; an uploaded mesh has no
        integer tables, so kval/gval/gtval/vol are left out for it."""
        i = self.mesh_info(mesh)
        N, nb, nnz, T, F = i["N"], i["nb"], i["nnz"], i["tets"], i["tris"]
        out = dict(tets=np.empty((T, 4), np.int32), rowptr=np.empty(N + 1, np.int32),
                   col=np.empty(nnz, np.int32), kval=np.empty(nnz, np.int32),
                   gval=np.empty((nnz, 3), np.int32), gtval=np.empty((nnz, 3), np.int32),
                   vol=np.empty(N, np.int32), bnd=np.empty(nb, np.int32),
                   tris=np.empty((F, 3), np.int32))
        keys = ("tets", "rowptr", "col", "kval", "gval", "gtval", "vol", "bnd", "tris")
        if i["n"] == 0:
            for k in ("kval", "gval", "gtval", "vol"):
                del out[k]
        _check(lib().lbm_mesh_export(self._h, mesh, *[_iptr(out[k]) if k in out else None for k in keys]))
        return out

    def bem_rows(self, mesh: int, row0: int, nrows: int) -> np.ndarray:
        nb = self.mesh_info(mesh)["nb"]
        out = np.empty((nrows, nb))
        _check(lib().lbm_bem_rows(self._h, mesh, row0, nrows, _dptr(out)))
        return out

    # -- instances -----------------------------------------------------------
    def instance_create(self, mesh: int, batch: int = 1, precision: int = LBM_FP64) -> "Instance":
        h = _I64()
        _check(lib().lbm_instance_create(self._h, mesh, batch, precision, C.byref(h)))
        return Instance(self, h.value, mesh, batch, precision)

    def evaluate_noalloc(self, mesh: int, Js, A, K1, axis, h_ext, d_m: int, d_h: int = 0, d_u: int = 0,
                         d_energy: int = 0, opts: SolveOpts | None = None):
        """lbm_evaluate_noalloc with device pointers (e.g. torch tensors' data_ptr());
        queued on the context's stream."""
        mat = Material()
        mat.Js, mat.A, mat.K1 = Js, A, K1
        for d in range(3):
            mat.axis[d] = axis[d]
        h = np.ascontiguousarray(np.asarray(h_ext, np.float64))
        _check(lib().lbm_evaluate_noalloc(self._h, mesh, C.byref(mat), _dptr(h),
                                          C.byref(opts) if opts else None, C.c_void_p(d_m),
                                          C.c_void_p(d_h or None), C.c_void_p(d_u or None),
                                          C.c_void_p(d_energy or None)))

    def mesh_hmatrix(self, mesh: int, eps: float, eta: float = 2.0, n_min: int = 16, threads: int | None = None) -> dict:
        """lbm_mesh_hmatrix: build and use the hierarchical form of the mesh's
        boundary matrix (eps <= 0: back to the dense matrix)."""
        out = (C.c_int64 * 4)()
        th = threads if threads is not None else max(1, os.cpu_count() or 1)
        _check(lib().lbm_mesh_hmatrix(self._h, mesh, float(eps), float(eta), int(n_min), int(th), out))
        return dict(stored=out[0], dense=out[1], leaves=out[2], low_rank=out[3],
                    fraction=(out[0] / out[1]) if out[1] else 0.0)

    def mesh_shell(self, mesh: int, a: int, s: int) -> dict:
        """lbm_mesh_shell: attach the space-transformation open boundary (air a
        cells deep, shell s cells deep; a = s = 0 detaches it)."""
        out = (C.c_int64 * 3)()
        _check(lib().lbm_mesh_shell(self._h, mesh, int(a), int(s), out))
        return dict(grid_nodes=out[0], nnz=out[1], shell_tets=out[2])

    def bem_apply(self, mesh: int, x, precision=LBM_FP64):
        """lbm_bem_apply: (B x, B^T x) for x of shape [nb] or [nb, batch]."""
        xa = np.ascontiguousarray(np.asarray(x, np.float64))
        one = xa.ndim == 1
        if one:
            xa = xa[:, None].copy()
        nb, batch = xa.shape
        y, yt = np.empty_like(xa), np.empty_like(xa)
        _check(lib().lbm_bem_apply(self._h, mesh, precision, batch, _dptr(xa), _dptr(y), _dptr(yt)))
        return (y[:, 0], yt[:, 0]) if one else (y, yt)

    def graph_stats(self) -> dict:
        """lbm_graph_stats: CUDA-graph replays, captures and refused captures."""
        out = (C.c_int64 * 3)()
        _check(lib().lbm_graph_stats(self._h, out))
        return dict(replays=out[0], captures=out[1], refused=out[2])

    def serve_trace(self, max_entries: int = 100000) -> np.ndarray:
        """lbm_serve_trace: [k, 3] rows (cube size, start ms, end ms) of the serving
        loop's chunks on the device."""
        out = np.empty((max_entries, 3))
        n = C.c_int64()
        _check(lib().lbm_serve_trace(self._h, _dptr(out), max_entries, C.byref(n)))
        return out[:n.value].copy()

    def set_wait_limit(self, seconds: float, unreachable: bool = False):
        """lbm_set_wait_limit: the device-wait limit of this context's kernels
        (0: the default 2 s); `unreachable` makes every grid barrier's wait run
        out (a test of the timeout path)."""
        _check(lib().lbm_set_wait_limit(self._h, float(seconds), 1 if unreachable else 0))

    # -- serving (continuous batching) ---------------------------------------
    def serve_start(self, **kw):
        o = ServeOpts()
        lib().lbm_default_serve_opts(C.byref(o))
        for k, v in kw.items():
            if k == "opt":
                o.opt = v
            else:
                setattr(o, k, v)
        _check(lib().lbm_serve_start(self._h, C.byref(o)))

    def submit(self, n, cell_m, Js, A, K1, axis, h, m0, precision=LBM_MIXED) -> int:
        m0 = np.ascontiguousarray(np.asarray(m0, np.float64))
        r = Request()
        r.n, r.cell_m, r.precision = n, cell_m, precision
        r.mat.Js, r.mat.A, r.mat.K1 = Js, A, K1
        for d in range(3):
            r.mat.axis[d] = axis[d]
            r.h[d] = h[d]
        r.m0 = _dptr(m0)
        t = _I64()
        _check(lib().lbm_submit(self._h, C.byref(r), C.byref(t)))
        return t.value

    def poll(self, ticket: int, N: int | None = None):
        """(result dict, m) when finished, None while pending."""
        res = Result()
        m = np.empty((N, 3)) if N else None
        rc = lib().lbm_poll(self._h, ticket, C.byref(res), _dptr(m))
        if rc == LBM_E_PENDING:
            return None
        _check(rc)
        return res.as_dict(), m

    def wait(self, ticket: int, N: int | None = None, timeout_s: float = 600.0):
        res = Result()
        m = np.empty((N, 3)) if N else None
        _check(lib().lbm_wait(self._h, ticket, timeout_s, C.byref(res), _dptr(m)))
        return res.as_dict(), m

    def serve_stats(self) -> dict:
        st = (_I64 * 8)()
        _check(lib().lbm_serve_stats(self._h, st))
        keys = ("submitted", "admitted", "completed", "pending", "active_slots", "groups", "stalls",
                "evicted")
        return {k: int(st[i]) for i, k in enumerate(keys)}

    def serve_stop(self):
        _check(lib().lbm_serve_stop(self._h))

    def launch_count(self) -> int:
        c = _I64()
        _check(lib().lbm_launch_count(self._h, C.byref(c)))
        return c.value

    def profile_enable(self, on: bool = True):
        _check(lib().lbm_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset: bool = True) -> dict:
        s = ProfileStats()
        _check(lib().lbm_profile_read(self._h, C.byref(s), 1 if reset else 0))
        out = {k: dict(launches=int(s.launches[i]), ms=float(s.ms[i]))
               for i, k in enumerate(PROFILE_KINDS)}
        out["cg_iters"] = [int(s.cg_iters[0]), int(s.cg_iters[1])]
        out["cg_sweeps"] = [int(s.cg_sweeps[k]) for k in range(4)]
        return out


class Instance:
    """A batch of problems on one mesh (lbm_instance_* calls)."""

    def __init__(self, ctx: Context, handle: int, mesh: int, batch: int, precision: int):
        self.ctx, self.h, self.mesh, self.B, self.precision = ctx, handle, mesh, batch, precision
        self.N = ctx.mesh_info(mesh)["N"]

    def destroy(self):
        _check(lib().lbm_instance_destroy(self.ctx._h, self.h))

    def set_material(self, Js, A, K1, axes):
        axes = np.broadcast_to(np.asarray(axes, dtype=np.float64), (self.B, 3))
        mats = (Material * self.B)()
        for b in range(self.B):
            mats[b].Js, mats[b].A, mats[b].K1 = Js, A, K1
            for d in range(3):
                mats[b].axis[d] = axes[b, d]
        _check(lib().lbm_set_material(self.ctx._h, self.h, mats))

    def set_field(self, h):
        h = np.ascontiguousarray(np.broadcast_to(np.asarray(h, np.float64), (self.B, 3)))
        _check(lib().lbm_set_field(self.ctx._h, self.h, _dptr(h)))

    def set_m(self, m):
        m = np.ascontiguousarray(np.broadcast_to(np.asarray(m, np.float64), (self.B, self.N, 3)))
        _check(lib().lbm_set_m(self.ctx._h, self.h, _dptr(m)))

    def get_state(self) -> bytes:
        """lbm_get_state: the batch's full state (checkpoint)."""
        n = _I64()
        _check(lib().lbm_get_state(self.ctx._h, self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib().lbm_get_state(self.ctx._h, self.h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def set_state(self, state: bytes):
        """lbm_set_state: restore a state written by get_state (then minimise
        with resume=1 continues it)."""
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(lib().lbm_set_state(self.ctx._h, self.h, buf, len(state)))

    def set_m_device(self, ptr: int):
        """m from a device buffer (batch*N*3 doubles), e.g. a torch tensor's data_ptr()."""
        _check(lib().lbm_set_m_device(self.ctx._h, self.h, C.c_void_p(ptr)))

    def get_m(self, out: np.ndarray | None = None) -> np.ndarray:
        """m of every instance, [B, N, 3]; written into `out` when given (a C-contiguous
        float64 array of that shape, e.g. a view of page-locked memory)."""
        if out is None:
            out = np.empty((self.B, self.N, 3))
        elif out.shape != (self.B, self.N, 3) or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of shape (B, N, 3)")
        _check(lib().lbm_get_m(self.ctx._h, self.h, _dptr(out)))
        return out

    def evaluate(self, opts: SolveOpts | None = None, want_h=True, want_u=True):
        res = (Result * self.B)()
        h = np.empty((self.B, self.N, 3)) if want_h else None
        u = np.empty((self.B, 2, self.N)) if want_u else None
        _check(lib().lbm_evaluate(self.ctx._h, self.h, C.byref(opts) if opts else None,
                                  _dptr(h), _dptr(u), res))
        return [r.as_dict() for r in res], h, u

    def energy(self) -> np.ndarray:
        """(B, 5) exchange, anisotropy, Zeeman, stray-field and total energy (J)."""
        out = np.empty((self.B, 5))
        _check(lib().lbm_energy(self.ctx._h, self.h, _dptr(out)))
        return out

    def minimise(self, opts: SolveOpts | None = None):
        res = (Result * self.B)()
        _check(lib().lbm_minimise(self.ctx._h, self.h, C.byref(opts) if opts else None, res))
        return [r.as_dict() for r in res]

    def hysteresis(self, direction, fields, opts: SolveOpts | None = None):
        d = np.ascontiguousarray(np.asarray(direction, np.float64))
        f = np.ascontiguousarray(np.asarray(fields, np.float64))
        npts = f.size
        mpar = np.empty((npts, self.B))
        energy = np.empty((npts, self.B))
        res = (Result * (npts * self.B))()
        _check(lib().lbm_hysteresis(self.ctx._h, self.h, _dptr(d), _dptr(f), npts,
                                    C.byref(opts) if opts else None, _dptr(mpar), _dptr(energy),
                                    res))
        return mpar, energy, [r.as_dict() for r in res]
