"""GB300 (sm_103a) density-matrix RT-TDDFT step: Python binding of librtdm.so.

The binding only marshals arguments: every step of the method runs in the CUDA
kernels of librtdm.so behind the C ABI declared in include/rt.h.  PyTorch
supplies device memory (the caching allocator, through the allocator hook of
rt_create) and the CUDA stream.  There is no CPU fallback: if the library is
missing or no GPU is present the calls raise.

Functions with the names of the C ABI (rt_create, rt_inverse, rt_step, ...)
are exported as thin wrappers; the class RT bundles them for one context.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

# ----------------------------------------------------------------------------
# constants (mirror include/rt.h)
# ----------------------------------------------------------------------------
RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOTCONV, RT_ENUMERIC, RT_ETIMEOUT, RT_EINTERNAL, RT_ESTATE = range(9)
RT_FAULT_HOTELLING_MAXITER1, RT_FAULT_NAN_IN_H, RT_FAULT_WAIT_TIMEOUT_0 = 1, 2, 4
STATUS_NAMES = {0: "RT_OK", 1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ENOTCONV", 5: "RT_ENUMERIC",
                6: "RT_ETIMEOUT", 7: "RT_EINTERNAL", 8: "RT_ESTATE"}
RT_PROP_EM, RT_PROP_CN, RT_PROP_ETRS, RT_PROP_M4 = 0, 1, 2, 3
RT_FP64, RT_FP32 = 0, 1
RT_FIELD_NONE, RT_FIELD_GAUSSIAN, RT_FIELD_CONSTANT = 0, 1, 2
RT_MAT_S, RT_MAT_H0, RT_MAT_DX, RT_MAT_DY, RT_MAT_DZ, RT_MAT_SINV, RT_MAT_T, RT_MAT_U, RT_MAT_K, RT_MAT_X = range(10)
RT_PAT_S, RT_PAT_H, RT_PAT_SINV, RT_PAT_T, RT_PAT_U, RT_PAT_K, RT_PAT_M, RT_PAT_A, RT_PAT_W = range(9)
RT_NOBS = 12
RT_NOALLOC_MAX_CTAS = 1024
OBS_FIELDS = ["t", "trks_re", "trks_im", "trkdx_re", "trkdx_im", "trkdy_re", "trkdy_im", "trkdz_re", "trkdz_im",
              "herm", "hot_iters", "hot_resid"]

EXPORTED = ["rt_default_params", "rt_create", "rt_set_field", "rt_inverse", "rt_set_density", "rt_ground_state",
            "rt_kick", "rt_propagator", "rt_step", "rt_observables", "rt_pattern_size", "rt_get_pattern",
            "rt_matrix_size", "rt_get_matrix", "rt_unitarity", "rt_step_work", "rt_step_kernels", "rt_profile", "rt_profile_read",
            "rt_get_state", "rt_set_state", "rt_synchronize", "rt_last_error", "rt_destroy", "rt_traces_noalloc",
            "rt_debug_inject", "rt_check_triples", "rt_debug_check", "rt_autotune", "rt_set_launch_shape",
            "rt_get_launch_shape"]


class rt_system(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("pos", ctypes.c_void_p), ("cell", ctypes.c_void_p),
                ("bsize", ctypes.c_void_p), ("r_S", ctypes.c_double), ("r_H", ctypes.c_double),
                ("s_rowptr", ctypes.c_void_p), ("s_col", ctypes.c_void_p), ("s_val", ctypes.c_void_p),
                ("h_rowptr", ctypes.c_void_p), ("h_col", ctypes.c_void_p), ("h_val", ctypes.c_void_p),
                ("d_val", ctypes.c_void_p * 3)]


class rt_params(ctypes.Structure):
    _fields_ = [("r_Sinv", ctypes.c_double), ("r_T", ctypes.c_double), ("r_U", ctypes.c_double),
                ("r_K", ctypes.c_double), ("r_M", ctypes.c_double), ("dt", ctypes.c_double),
                ("prop", ctypes.c_int32), ("taylor_terms", ctypes.c_int32), ("hot_tol", ctypes.c_double),
                ("hot_maxit", ctypes.c_int32), ("hot_step_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("full_step", ctypes.c_int32), ("n_kick", ctypes.c_int32), ("kick_terms", ctypes.c_int32),
                ("obs_capacity", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("incremental", ctypes.c_int32),
                ("field_poly", ctypes.c_int32), ("hot_fp64_iters", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32),
                ("packed_fma", ctypes.c_int32)]


class rt_field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dir", ctypes.c_int32), ("E0", ctypes.c_double),
                ("t0", ctypes.c_double), ("sigma", ctypes.c_double), ("omega", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Loads librtdm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1404_5776_gb300._build.build() "
                           "(the CUDA path has no fallback)")
    L = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "rt_default_params": [P],
        "rt_create": [P, P, I32, P, P, ALLOC_FN, FREE_FN, P],
        "rt_set_field": [P, P],
        "rt_inverse": [P, I32, P, P],
        "rt_set_density": [P, I32, I32, P],
        "rt_ground_state": [P, I32, I32, D, D, D, D],
        "rt_kick": [P, I32, I32, I32, D],
        "rt_propagator": [P, D],
        "rt_step": [P, I32],
        "rt_observables": [P, I32, I32, P, I32, P],
        "rt_pattern_size": [P, I32, I32, P],
        "rt_get_pattern": [P, I32, I32, P, P],
        "rt_matrix_size": [P, I32, I32, P],
        "rt_get_matrix": [P, I32, I32, I32, P, I64],
        "rt_unitarity": [P, I32, I32, P, P],
        "rt_step_work": [P, P, P],
        "rt_step_kernels": [P, P],
        "rt_profile": [P, I32],
        "rt_profile_read": [P, I32, P, P, P, P, P, P],
        "rt_get_state": [P, P, P],
        "rt_set_state": [P, P, ctypes.c_size_t],
        "rt_synchronize": [P],
        "rt_debug_inject": [P, ctypes.c_uint32],
        "rt_check_triples": [I32, P, P, I32, P, P, I32, P, P, I32, I64, P, P, P, I64, P],
        "rt_debug_check": [P, P],
        "rt_traces_noalloc": [P, I64, P, P, P, I32, P, P, P, P, P, P, I32, P, P],
        "rt_autotune": [P, I32, I32, P, P, P],
        "rt_set_launch_shape": [P, I32, I32, I32],
        "rt_get_launch_shape": [P, I32, P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.rt_last_error.argtypes = [P]
    L.rt_last_error.restype = ctypes.c_char_p
    L.rt_destroy.argtypes = [P]
    L.rt_destroy.restype = None
    _lib = L
    return L


class RTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ----------------------------------------------------------------------------
# thin wrappers with the C ABI names
# ----------------------------------------------------------------------------

def rt_default_params() -> rt_params:
    p = rt_params()
    _check(None, load().rt_default_params(ctypes.byref(p)))
    return p


def rt_check_triples(n_atoms, a_rowptr, a_col, a_dag, b_rowptr, b_col, b_dag, c_rowptr, c_col, upper_only,
                     item_blk, ptr, ab):
    """Structural check of a triple list against its patterns (host arrays,
    no GPU; the conditions are those of rt_check_triples in rt.h).  ab is an
    (n_triples, 2) array of (A block, B block).  Returns (status, bad_item)."""
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    a_rowptr, a_col, b_rowptr, b_col, c_rowptr, c_col, item_blk = map(
        i32, (a_rowptr, a_col, b_rowptr, b_col, c_rowptr, c_col, item_blk))
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    ab = np.ascontiguousarray(ab, dtype=np.int32).reshape(-1, 2)
    bad = ctypes.c_int64(-1)
    st = load().rt_check_triples(int(n_atoms), _p(a_rowptr), _p(a_col), int(a_dag), _p(b_rowptr), _p(b_col),
                                 int(b_dag), _p(c_rowptr), _p(c_col), int(upper_only), int(item_blk.size),
                                 _p(item_blk), _p(ptr), _p(ab), int(ab.shape[0]), ctypes.byref(bad))
    return st, bad.value


def _check(ctx, st):
    if st != RT_OK:
        msg = load().rt_last_error(ctx).decode() if ctx else ""
        raise RTError(st, msg)
    return st


def _torch_allocator():
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    return ALLOC_FN(_alloc), FREE_FN(_free)


def rt_create(systems: Sequence, params: rt_params, stream: Optional[int] = None, torch_memory: bool = True):
    """Returns (ctx handle, keep-alive list).  `systems` are objects with the
    fields of rt_system as numpy arrays (see RT)."""
    L = load()
    keep = []
    arr = (rt_system * len(systems))()
    for k, s in enumerate(systems):
        fs = _fill_system(arr[k], s)
        keep.extend(fs)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    if torch_memory:
        af, ff = _torch_allocator()
    else:
        af, ff = ALLOC_FN(), FREE_FN()
    keep.extend([af, ff])
    ctx = ctypes.c_void_p()
    st = L.rt_create(ctypes.byref(ctx), arr, len(systems), ctypes.byref(params), ctypes.c_void_p(stream), af, ff,
                     None)
    if st != RT_OK:
        raise RTError(st, "rt_create failed (reason printed on stderr)")
    return ctx, keep


def _fill_system(dst: rt_system, s):
    pos = np.ascontiguousarray(s.pos, dtype=np.float64)
    cell = None if s.cell is None else np.ascontiguousarray(s.cell, dtype=np.float64)
    bsize = np.ascontiguousarray(s.bsize, dtype=np.int32)
    srp = np.ascontiguousarray(s.s_rowptr, dtype=np.int32)
    scol = np.ascontiguousarray(s.s_col, dtype=np.int32)
    sval = np.ascontiguousarray(s.s_val, dtype=np.float64)
    hrp = np.ascontiguousarray(s.h_rowptr, dtype=np.int32)
    hcol = np.ascontiguousarray(s.h_col, dtype=np.int32)
    hval = np.ascontiguousarray(s.h_val, dtype=np.float64)
    d = [np.ascontiguousarray(x, dtype=np.float64) for x in s.d_val]
    dst.n_atoms = int(s.n_atoms)
    dst.pos = pos.ctypes.data
    dst.cell = cell.ctypes.data if cell is not None else None
    dst.bsize = bsize.ctypes.data
    dst.r_S = float(s.r_S)
    dst.r_H = float(s.r_H)
    dst.s_rowptr, dst.s_col, dst.s_val = srp.ctypes.data, scol.ctypes.data, sval.ctypes.data
    dst.h_rowptr, dst.h_col, dst.h_val = hrp.ctypes.data, hcol.ctypes.data, hval.ctypes.data
    for k in range(3):
        dst.d_val[k] = d[k].ctypes.data
    return [pos, cell, bsize, srp, scol, sval, hrp, hcol, hval] + d


def make_params(**kw) -> rt_params:
    p = rt_default_params()
    for k, v in kw.items():
        if k == "prop" and isinstance(v, str):
            v = {"em": RT_PROP_EM, "cn": RT_PROP_CN, "etrs": RT_PROP_ETRS, "m4": RT_PROP_M4}[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp64": RT_FP64, "fp32": RT_FP32}[v]
        setattr(p, k, v)
    return p


class RT:
    """One library context over one or more systems (same names as the C ABI)."""

    def __init__(self, systems, stream: Optional[int] = None, torch_memory: bool = True, **params):
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        self.systems = list(systems)
        self.params = make_params(**params)
        self.lib = load()
        self.ctx, self._keep = rt_create(self.systems, self.params, stream, torch_memory)

    # -- helpers
    def _c(self, st):
        return _check(self.ctx, st)

    def close(self):
        if self.ctx:
            self.lib.rt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI
    def set_field(self, kind=RT_FIELD_NONE, dir=0, E0=0.0, t0=0.0, sigma=1.0, omega=0.0):
        f = rt_field(kind, dir, E0, t0, sigma, omega)
        self._c(self.lib.rt_set_field(self.ctx, ctypes.byref(f)))

    def inverse(self, sys: int = -1):
        it = ctypes.c_int32()
        res = ctypes.c_double()
        st = self.lib.rt_inverse(self.ctx, sys, ctypes.byref(it), ctypes.byref(res))
        self._c(st)
        return it.value, res.value

    def pattern(self, sys: int, which: int):
        n = ctypes.c_int64()
        self._c(self.lib.rt_pattern_size(self.ctx, sys, which, ctypes.byref(n)))
        rowptr = np.zeros(self.systems[sys].n_atoms + 1, dtype=np.int32)
        col = np.zeros(max(n.value, 1), dtype=np.int32)
        self._c(self.lib.rt_get_pattern(self.ctx, sys, which, _p(rowptr), _p(col)))
        return rowptr, col[:n.value]

    def matrix(self, sys: int, which: int, kick: int = 0) -> np.ndarray:
        n = ctypes.c_int64()
        self._c(self.lib.rt_matrix_size(self.ctx, sys, which, ctypes.byref(n)))
        out = np.zeros(max(n.value, 2), dtype=np.float64)
        self._c(self.lib.rt_get_matrix(self.ctx, sys, kick, which, _p(out), n.value))
        return out[:n.value].view(np.complex128)

    def set_density(self, sys: int, kick: int, values: np.ndarray):
        v = np.ascontiguousarray(np.asarray(values, dtype=np.complex128)).view(np.float64)
        self._c(self.lib.rt_set_density(self.ctx, sys, kick, _p(v)))

    def set_density_dense(self, sys: int, kick: int, dense: np.ndarray):
        """Gathers the blocks of P_K from a dense n x n matrix (marshalling only)."""
        rowptr, col = self.pattern(sys, RT_PAT_K)
        bsize = np.asarray(self.systems[sys].bsize)
        foff = np.concatenate([[0], np.cumsum(bsize)])
        parts = []
        for i in range(len(bsize)):
            for q in range(rowptr[i], rowptr[i + 1]):
                j = col[q]
                parts.append(np.asarray(dense[foff[i]:foff[i + 1], foff[j]:foff[j + 1]]).reshape(-1))
        self.set_density(sys, kick, np.concatenate(parts).astype(np.complex128))

    def ground_state(self, sys: int, order: int, mu: float, kT: float, e_lo: float, e_hi: float):
        self._c(self.lib.rt_ground_state(self.ctx, sys, order, mu, kT, e_lo, e_hi))

    def kick(self, sys: int, kick: int, dir: int, kappa: float):
        self._c(self.lib.rt_kick(self.ctx, sys, kick, dir, kappa))

    def propagator(self, t: float = 0.0):
        self._c(self.lib.rt_propagator(self.ctx, t))

    def step(self, n: int = 1):
        self._c(self.lib.rt_step(self.ctx, n))

    def observables(self, sys: int = 0, kick: int = 0, max_steps: Optional[int] = None) -> np.ndarray:
        cap = max_steps or self.params.obs_capacity
        out = np.zeros((cap, RT_NOBS), dtype=np.float64)
        n = ctypes.c_int32()
        st = self.lib.rt_observables(self.ctx, sys, kick, _p(out), cap, ctypes.byref(n))
        if st not in (RT_OK, RT_ENUMERIC):
            self._c(st)
        res = out[:n.value].copy()
        if st == RT_ENUMERIC:
            raise RTError(st, "NaN/Inf in observables")
        return res

    def unitarity(self, sys: int = 0, metric_S: bool = True):
        mx, mn = ctypes.c_double(), ctypes.c_double()
        self._c(self.lib.rt_unitarity(self.ctx, sys, int(metric_S), ctypes.byref(mx), ctypes.byref(mn)))
        return mx.value, mn.value

    def step_work(self):
        f, b = ctypes.c_double(), ctypes.c_double()
        self._c(self.lib.rt_step_work(self.ctx, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def step_kernels(self) -> int:
        n = ctypes.c_int64()
        self._c(self.lib.rt_step_kernels(self.ctx, ctypes.byref(n)))
        return n.value

    def profile(self, enable: bool = True):
        self._c(self.lib.rt_profile(self.ctx, int(enable)))

    def profile_read(self):
        mx = 32
        n = ctypes.c_int32()
        la = np.zeros(mx, np.int64)
        ms, fl, by = np.zeros(mx), np.zeros(mx), np.zeros(mx)
        names = ctypes.create_string_buffer(32 * mx)
        self._c(self.lib.rt_profile_read(self.ctx, mx, ctypes.byref(n), _p(la), _p(ms), _p(fl), _p(by), names))
        out = {}
        raw = names.raw
        for i in range(n.value):
            nm = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = {"launches": int(la[i]), "ms": float(ms[i]), "flops": float(fl[i]), "bytes": float(by[i])}
        return out

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        self._c(self.lib.rt_get_state(self.ctx, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._c(self.lib.rt_get_state(self.ctx, buf, ctypes.byref(n)))
        return buf.raw

    def set_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._c(self.lib.rt_set_state(self.ctx, buf, len(data)))

    def synchronize(self):
        self._c(self.lib.rt_synchronize(self.ctx))

    # -- launch shapes of the grouped products (reference split, CUDA cores)
    STAGES = {0: "M, 13 functions", 1: "K', 13 functions", 2: "M, 4 functions", 3: "K', 4 functions"}

    def set_launch_shape(self, stage: int, stages: int, persistent: int):
        self._c(self.lib.rt_set_launch_shape(self.ctx, stage, stages, persistent))

    def get_launch_shape(self, stage: int):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        self._c(self.lib.rt_get_launch_shape(self.ctx, stage, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def _tune_key(self):
        try:
            import torch
            dev = torch.cuda.get_device_name()
        except Exception:  # the key only names the device
            dev = "cuda"
        sysk = [(int(s.n_atoms), int(np.sum(s.bsize)), int(np.max(s.bsize))) for s in self.systems]
        pk = self.params
        return json.dumps([dev, sysk, pk.n_kick, pk.r_U, pk.r_K, pk.r_M, pk.packed_fma, pk.precision])

    def autotune(self, reps: int = 3, cache: Optional[str] = None):
        """Picks the launch shape of every grouped product stage (rt_autotune)
        and returns {"source", "rows", "chosen"}.  With `cache` (a JSON file
        path), a shape tuned earlier for the same device, systems and
        parameters is applied without timing, and a new one is stored."""
        key = self._tune_key()
        store = {}
        if cache and os.path.exists(cache):
            try:
                with open(cache) as f:
                    store = json.load(f)
            except (OSError, ValueError):
                store = {}
        if key in store:
            for st, (ns, pers) in store[key].items():
                self.set_launch_shape(int(st), int(ns), int(pers))
            return {"source": "cache", "rows": [], "chosen": {int(k): tuple(v) for k, v in store[key].items()}}
        mx = 64
        n = ctypes.c_int32()
        rows = np.zeros((mx, 4), dtype=np.int32)
        ms = np.zeros(mx)
        self._c(self.lib.rt_autotune(self.ctx, reps, mx, ctypes.byref(n), _p(rows), _p(ms)))
        out_rows = [{"stage": int(r[0]), "what": self.STAGES[int(r[0])], "stages_per_warp": int(r[1]),
                     "persistent": int(r[2]), "chosen": bool(r[3]), "ms": float(t)}
                    for r, t in zip(rows[:min(n.value, mx)], ms[:min(n.value, mx)])]
        chosen = {r["stage"]: (r["stages_per_warp"], r["persistent"]) for r in out_rows if r["chosen"]}
        if cache:
            store[key] = {str(k): list(v) for k, v in chosen.items()}
            d = os.path.dirname(os.path.abspath(cache))
            os.makedirs(d, exist_ok=True)
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(store, f, indent=1)
            os.replace(tmp, cache)
        return {"source": "tuned", "rows": out_rows, "chosen": chosen}

    def debug_inject(self, flags: int):
        """Host-side fault injection (RT_FAULT_* flags) for tests."""
        self._c(self.lib.rt_debug_inject(self.ctx, flags))

    def debug_check(self) -> int:
        """Structural check of every pattern and triple list the context has
        built (rt_debug_check); returns the number of lists checked."""
        n = ctypes.c_int64(0)
        self._c(self.lib.rt_debug_check(self.ctx, ctypes.byref(n)))
        return n.value


def build(force: bool = False, verbose: bool = False) -> str:
    return _build.build(force=force, verbose=verbose)
