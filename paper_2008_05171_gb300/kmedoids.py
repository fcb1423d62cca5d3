"""Python binding of libkmedoids (include/kmedoids.h), argument marshalling only.

Every function here takes torch CUDA tensors, passes their device pointers,
sizes and the current CUDA stream to the C ABI of the same name, and turns
the result struct into a dict.  All of the method's arithmetic runs in the
library's kernels; there is no CPU fallback: if ``libkmedoids.so`` has not
been built, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# KMEDOIDS_BOUNDS_CHECK=1 selects the bounds-checking build of the library
LIB_PATH = os.path.join(HERE, "libkmedoids_bounds.so"
                        if os.environ.get("KMEDOIDS_BOUNDS_CHECK") == "1" else "libkmedoids.so")

KM_I32, KM_F32, KM_U16 = 0, 1, 2
VARIANTS = {"fastpam1": 0, "fastpam2": 1, "fasterpam": 2, "fastclarans": 3}
STATUS = {0: "KM_OK", 1: "KM_E_INVALID", 2: "KM_E_WORKSPACE", 3: "KM_E_CUDA",
          4: "KM_E_NOT_CONVERGED", 5: "KM_E_TIMEOUT", 6: "KM_E_NUMERIC",
          7: "KM_E_UNSUPPORTED", 8: "KM_E_BOUNDS"}
EXPORTS = ["km_default_options", "kmedoids_workspace_size", "kmedoids_build",
           "kmedoids_swap", "kmedoids_run", "kmedoids_eval_swaps",
           "kmedoids_cache", "kmedoids_last_error", "kmedoids_version",
           "kmedoids_eval_swaps_static", "kmedoids_gram_bf16",
           "kmedoids_features_workspace_size", "kmedoids_run_features",
           "kmedoids_swap_features", "kmedoids_batched_workspace_size",
           "kmedoids_batched_distances", "kmedoids_run_batched",
           "kmedoids_swap_batched", "kmedoids_clara_workspace_size", "kmedoids_clara",
           "kmedoids_geometry_info", "kmedoids_init_weighted",
           "kmedoids_init_lab", "kmedoids_wait_selftest", "kmedoids_build_features",
           "kmedoids_batched_geometry_info", "kmedoids_batched_autotune",
           "kmedoids_batched_clara_workspace_size", "kmedoids_run_batched_clara",
           "kmedoids_upload_matrix", "kmedoids_bounds_checked",
           "kmedoids_bichromatic_workspace_size", "kmedoids_run_bichromatic",
           "kmedoids_swap_bichromatic", "kmedoids_upload_rows"]


class KmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class km_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("tol", ctypes.c_double), ("fastpam2_tol", ctypes.c_double),
                ("rows_per_tile", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("trace_capacity", ctypes.c_int32),
                ("tune", ctypes.c_int32),
                ("trace_delta", ctypes.POINTER(ctypes.c_double)),
                ("trace_slot", ctypes.POINTER(ctypes.c_int32)),
                ("trace_cand", ctypes.POINTER(ctypes.c_int32)),
                ("trace_time_ns", ctypes.POINTER(ctypes.c_int64)),
                ("build_gains", ctypes.POINTER(ctypes.c_double)),
                ("draws", ctypes.c_void_p), ("draws_len", ctypes.c_int64),
                ("maxneighbor", ctypes.c_int64), ("check_input", ctypes.c_int32),
                ("build_full", ctypes.c_int32), ("wait_limit_ns", ctypes.c_int64),
                ("swap_full", ctypes.c_int32), ("gram_full", ctypes.c_int32)]


class km_result(ctypes.Structure):
    _fields_ = [("td", ctypes.c_double), ("td_i64", ctypes.c_int64),
                ("td_bookkept", ctypes.c_double),
                ("td_initial", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("swaps", ctypes.c_int32),
                ("status", ctypes.c_int32), ("build_steps", ctypes.c_int32),
                ("visited", ctypes.c_int64), ("build_ms", ctypes.c_double),
                ("swap_ms", ctypes.c_double), ("eval_ms", ctypes.c_double),
                ("eval_launches", ctypes.c_int32),
                ("build_launches", ctypes.c_int32),
                ("build_eval_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64),
                ("best_sample", ctypes.c_int32), ("swap_geometry", ctypes.c_int16),
                ("build_geometry", ctypes.c_int16), ("evaluated", ctypes.c_int64),
                ("build_rows", ctypes.c_int64), ("eval_ms_median", ctypes.c_double),
                ("eval_ms_first", ctypes.c_double)]


_LOCK = threading.Lock()
_LIB = None


def load(path: str = LIB_PATH):
    """Load libkmedoids.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(path):
            raise RuntimeError(
                "libkmedoids.so not found at %s: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')" % path)
        lib = ctypes.CDLL(path)
        P, i32, i64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                           ctypes.c_size_t)
        opt_p = ctypes.POINTER(km_options)
        res_p = ctypes.POINTER(km_result)
        lib.km_default_options.argtypes = [opt_p]
        lib.km_default_options.restype = None
        lib.kmedoids_workspace_size.argtypes = [i64, i32, i32, opt_p]
        lib.kmedoids_workspace_size.restype = sz
        for name in ("kmedoids_swap", "kmedoids_run"):
            f = getattr(lib, name)
            f.argtypes = [P, i32, i64, i64, i32, P, P, opt_p, res_p, P, sz, P]
            f.restype = i32
        lib.kmedoids_build.argtypes = [P, i32, i64, i64, i32, P, opt_p, res_p,
                                       P, sz, P]
        lib.kmedoids_build.restype = i32
        lib.kmedoids_eval_swaps.argtypes = [P, i32, i64, i64, i32, P, P, P,
                                            P, P, P, P, sz, P]
        lib.kmedoids_eval_swaps.restype = i32
        lib.kmedoids_cache.argtypes = [P, i32, i64, i64, i32, P, P, P, P, P,
                                       P, P, sz, P]
        lib.kmedoids_cache.restype = i32
        lib.kmedoids_eval_swaps_static.argtypes = [P, i32, i64, i64, i32, P,
                                                   P, P, P, P, P, P]
        lib.kmedoids_eval_swaps_static.restype = i32
        lib.kmedoids_gram_bf16.argtypes = [P, i64, i32, i64, P, i64, P, sz, P]
        lib.kmedoids_gram_bf16.restype = i32
        lib.kmedoids_features_workspace_size.argtypes = [i64, i32, i32, opt_p]
        lib.kmedoids_features_workspace_size.restype = sz
        for name in ("kmedoids_run_features", "kmedoids_swap_features",
                     "kmedoids_build_features"):
            f = getattr(lib, name)
            f.argtypes = [P, i64, i32, i64, i32, P, P, opt_p, res_p, P, sz, P]
            f.restype = i32
        lib.kmedoids_batched_workspace_size.argtypes = [i32]
        lib.kmedoids_batched_workspace_size.restype = sz
        lib.kmedoids_batched_distances.argtypes = [P, i32, P, P, i32, P, P]
        lib.kmedoids_batched_distances.restype = i32
        for f in (lib.kmedoids_run_batched, lib.kmedoids_swap_batched):
            f.argtypes = [P, P, i32, P, P, opt_p, P, sz, P]
            f.restype = i32
        lib.kmedoids_clara_workspace_size.argtypes = [i32, i32, i32]
        lib.kmedoids_clara_workspace_size.restype = sz
        lib.kmedoids_clara.argtypes = [P, i64, i32, i32, i32, i32, P, P, P, P,
                                       res_p, P, sz, P]
        lib.kmedoids_clara.restype = i32
        lib.kmedoids_geometry_info.argtypes = [i32, P, P, P]
        lib.kmedoids_geometry_info.restype = ctypes.c_int
        lib.kmedoids_init_weighted.argtypes = [P, i32, i64, i64, i32, P, P, P, sz, P]
        lib.kmedoids_init_weighted.restype = i32
        lib.kmedoids_init_lab.argtypes = [P, i32, i64, i64, i32, i32, P, P, P, P, sz,
                                          P]
        lib.kmedoids_init_lab.restype = i32
        lib.kmedoids_batched_geometry_info.argtypes = [i32, P, P]
        lib.kmedoids_batched_geometry_info.restype = i32
        lib.kmedoids_batched_autotune.argtypes = [P, P, i32, P, P, opt_p, P, sz, P, P, P]
        lib.kmedoids_batched_autotune.restype = i32
        lib.kmedoids_batched_clara_workspace_size.argtypes = [i32, i32, i32, i32]
        lib.kmedoids_batched_clara_workspace_size.restype = sz
        lib.kmedoids_run_batched_clara.argtypes = [P, P, i32, P, P, P, i64, i32, i32, i32, i32,
                                                   P, P, P, P, P, opt_p, P, sz, P]
        lib.kmedoids_run_batched_clara.restype = i32
        lib.kmedoids_wait_selftest.argtypes = [i32, i64, P, sz, P]
        lib.kmedoids_wait_selftest.restype = i32
        lib.kmedoids_upload_matrix.argtypes = [P, i64, i32, i64, P, i64, P]
        lib.kmedoids_upload_matrix.restype = i32
        lib.kmedoids_upload_rows.argtypes = [P, i64, i32, i64, i64, P, i64, P]
        lib.kmedoids_upload_rows.restype = i32
        lib.kmedoids_bichromatic_workspace_size.argtypes = [i64, i64, i32, i32, opt_p]
        lib.kmedoids_bichromatic_workspace_size.restype = sz
        for name in ("kmedoids_run_bichromatic", "kmedoids_swap_bichromatic"):
            f = getattr(lib, name)
            f.argtypes = [P, i32, i64, i64, i64, i32, P, P, opt_p, res_p, P, sz, P]
            f.restype = i32
        lib.kmedoids_bounds_checked.argtypes = []
        lib.kmedoids_bounds_checked.restype = i32
        lib.kmedoids_last_error.restype = ctypes.c_char_p
        lib.kmedoids_version.restype = ctypes.c_char_p
        _LIB = lib
    return _LIB


def _check(status: int):
    if status != 0:
        raise KmError(status, load().kmedoids_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libkmedoids needs a CUDA device; none is present")
    return torch


def _dtype_code(D) -> int:
    """int32 -> KM_I32, float32 -> KM_F32; uint16 (or int16, whose bits are
    read as unsigned) -> KM_U16, the compressed integer form."""
    torch = _torch()
    if D.dtype == torch.int32:
        return KM_I32
    if D.dtype == torch.float32:
        return KM_F32
    if D.dtype == torch.int16 or D.dtype == getattr(torch, "uint16", None):
        return KM_U16
    raise TypeError("D must be int32, float32 or 16-bit (got %s)" % D.dtype)


def _matrix(D, n):
    if D.dim() != 2 or not D.is_cuda or D.stride(1) != 1:
        raise ValueError("D must be a 2-D CUDA tensor with unit column stride")
    n = D.shape[0] if n is None else int(n)
    return n, D.stride(0)


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def options(variant="fastpam1", max_iter=0, tol=0.0, fastpam2_tol=0.0,
            rows_per_tile=0, profile=False, trace=0, tune=0, draws=None,
            maxneighbor=0, check_input=False, build_full=False, wait_limit_ns=0,
            swap_full=False, gram_full=False):
    """km_options.  draws: int32 CUDA tensor of candidate draws (FastCLARANS);
    the caller keeps it alive for the call.  build_full: every BUILD step
    streams all candidate rows instead of updating the gains
    incrementally.  wait_limit_ns: limit of the device waits (0 = 4 s).
    swap_full / gram_full (on-the-fly form): plain SWAP passes / every
    Gram tile in both orientations in the dense passes."""
    o = km_options()
    load().km_default_options(ctypes.byref(o))
    o.wait_limit_ns = int(wait_limit_ns)
    o.swap_full = 1 if swap_full else 0
    o.gram_full = 1 if gram_full else 0
    if draws is not None:
        o.draws = ctypes.c_void_p(draws.data_ptr())
        o.draws_len = int(draws.numel())
    o.maxneighbor = int(maxneighbor)
    o.check_input = 1 if check_input else 0
    o.build_full = 1 if build_full else 0
    o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    o.max_iter = int(max_iter)
    o.tol = float(tol)
    o.fastpam2_tol = float(fastpam2_tol)
    o.rows_per_tile = int(rows_per_tile)
    o.profile = 1 if profile else 0
    o.trace_capacity = int(trace)
    o.tune = int(tune)
    return o


def workspace_size(n, k, dtype_code, opts=None) -> int:
    return int(load().kmedoids_workspace_size(
        int(n), int(k), int(dtype_code),
        ctypes.byref(opts) if opts is not None else None))


def workspace(n, k, dtype_code, opts=None, device=None):
    """Allocate a device workspace (caller-owned torch tensor)."""
    torch = _torch()
    nbytes = workspace_size(n, k, dtype_code, opts)
    if nbytes == 0:
        raise KmError(1, "invalid sizes for a workspace")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def _result(res: km_result, o: km_options, k: int) -> dict:
    out = {f: getattr(res, f) for f, _ in km_result._fields_}
    return out


class _Trace:
    def __init__(self, o: km_options, cap: int, k: int, want_gains: bool):
        import numpy as np
        self.np = np
        self.d = np.zeros(max(cap, 1), np.float64)
        self.s = np.zeros(max(cap, 1), np.int32)
        self.c = np.zeros(max(cap, 1), np.int32)
        self.t = np.zeros(max(cap, 1), np.int64)
        self.g = np.zeros(max(k, 1), np.float64)
        if cap > 0:
            o.trace_delta = self.d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            o.trace_slot = self.s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            o.trace_cand = self.c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            o.trace_time_ns = self.t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        if want_gains:
            o.build_gains = self.g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def items(self, nswaps: int):
        m = min(nswaps, len(self.d))
        return [(float(self.d[i]), int(self.s[i]), int(self.c[i]))
                for i in range(m)]


def _call(fn_name, D, k, medoids, labels, n, ws, opts_kw, want_gains):
    torch = _torch()
    lib = load()
    n, ld = _matrix(D, n)
    code = _dtype_code(D)
    o = options(**opts_kw)
    tr = _Trace(o, o.trace_capacity, k, want_gains)
    if ws is None:
        ws = workspace(n, k, code, o, device=D.device)
    res = km_result()
    fn = getattr(lib, fn_name)
    if fn_name == "kmedoids_build":
        st = fn(ctypes.c_void_p(D.data_ptr()), code, n, ld, k,
                ctypes.c_void_p(medoids.data_ptr()), ctypes.byref(o),
                ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()),
                ws.numel(), _stream())
    else:
        st = fn(ctypes.c_void_p(D.data_ptr()), code, n, ld, k,
                ctypes.c_void_p(medoids.data_ptr()),
                ctypes.c_void_p(labels.data_ptr() if labels is not None else 0),
                ctypes.byref(o), ctypes.byref(res),
                ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream())
    if st not in (0, 4):
        _check(st)
    out = _result(res, o, k)
    out["status_name"] = STATUS.get(st, st)
    out["converged"] = st == 0
    out["medoids"] = medoids
    out["labels"] = labels
    out["trace"] = tr.items(res.swaps) if o.trace_capacity > 0 else []
    out["trace_time_ns"] = tr.t[:min(res.swaps, o.trace_capacity)].copy() \
        if o.trace_capacity > 0 else None
    if want_gains:
        out["build_gains"] = tr.g[:k].copy()
    return out


def run(D, k, n=None, labels=True, ws=None, **kw):
    """BUILD + SWAP (kmedoids_run).  kw: variant, max_iter, tol,
    fastpam2_tol, rows_per_tile, profile, trace."""
    torch = _torch()
    n_ = D.shape[0] if n is None else n
    med = torch.empty(k, dtype=torch.int32, device=D.device)
    lab = torch.empty(n_, dtype=torch.int32, device=D.device) if labels else None
    return _call("kmedoids_run", D, k, med, lab, n, ws, kw, True)


def build(D, k, n=None, ws=None, **kw):
    """PAM BUILD (kmedoids_build)."""
    torch = _torch()
    med = torch.empty(k, dtype=torch.int32, device=D.device)
    return _call("kmedoids_build", D, k, med, None, n, ws, kw, True)


def swap(D, medoids, n=None, labels=True, ws=None, **kw):
    """SWAP from the given medoids (kmedoids_swap); medoids are copied."""
    torch = _torch()
    med = torch.as_tensor(medoids, dtype=torch.int32).to(D.device).clone()
    n_ = D.shape[0] if n is None else n
    lab = torch.empty(n_, dtype=torch.int32, device=D.device) if labels else None
    return _call("kmedoids_swap", D, med.numel(), med, lab, n, ws, kw, False)


def eval_swaps(D, medoids, n=None, ws=None):
    """One FastPAM1 evaluation (kmedoids_eval_swaps): per-candidate best
    Delta and slot tensors, and the best (Delta, slot, candidate)."""
    torch = _torch()
    lib = load()
    n, ld = _matrix(D, n)
    code = _dtype_code(D)
    med = torch.as_tensor(medoids, dtype=torch.int32).to(D.device).contiguous()
    k = med.numel()
    if ws is None:
        ws = workspace(n, k, code, None, device=D.device)
    cd = torch.empty(n, dtype=torch.float64, device=D.device)
    cs = torch.empty(n, dtype=torch.int32, device=D.device)
    bd = ctypes.c_double()
    bs = ctypes.c_int32()
    bc = ctypes.c_int32()
    _check(lib.kmedoids_eval_swaps(
        ctypes.c_void_p(D.data_ptr()), code, n, ld, k,
        ctypes.c_void_p(med.data_ptr()), ctypes.c_void_p(cd.data_ptr()),
        ctypes.c_void_p(cs.data_ptr()), ctypes.byref(bd), ctypes.byref(bs),
        ctypes.byref(bc), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream()))
    return cd, cs, (bd.value, bs.value, bc.value)


def eval_swaps_static(D, medoids, n=None):
    """kmedoids_eval_swaps_static: the same evaluation pass with the
    library's fixed device scratch instead of a workspace (for callers that
    cannot allocate device memory; n <= 32768, k <= 512)."""
    torch = _torch()
    lib = load()
    n, ld = _matrix(D, n)
    code = _dtype_code(D)
    med = torch.as_tensor(medoids, dtype=torch.int32).to(D.device).contiguous()
    k = med.numel()
    cd = torch.empty(n, dtype=torch.float64, device=D.device)
    cs = torch.empty(n, dtype=torch.int32, device=D.device)
    bd = ctypes.c_double()
    bs = ctypes.c_int32()
    bc = ctypes.c_int32()
    _check(lib.kmedoids_eval_swaps_static(
        ctypes.c_void_p(D.data_ptr()), code, n, ld, k,
        ctypes.c_void_p(med.data_ptr()), ctypes.c_void_p(cd.data_ptr()),
        ctypes.c_void_p(cs.data_ptr()), ctypes.byref(bd), ctypes.byref(bs),
        ctypes.byref(bc), _stream()))
    return cd, cs, (bd.value, bs.value, bc.value)


def cache(D, medoids, n=None, ws=None):
    """Per-point cache (kmedoids_cache): near, sec, dn, ds, removal loss."""
    torch = _torch()
    lib = load()
    n, ld = _matrix(D, n)
    code = _dtype_code(D)
    med = torch.as_tensor(medoids, dtype=torch.int32).to(D.device).contiguous()
    k = med.numel()
    if ws is None:
        ws = workspace(n, k, code, None, device=D.device)
    near = torch.empty(n, dtype=torch.int32, device=D.device)
    sec = torch.empty(n, dtype=torch.int32, device=D.device)
    cdt = torch.int32 if code == KM_U16 else D.dtype  # the 16-bit form caches int32
    dn = torch.empty(n, dtype=cdt, device=D.device)
    ds = torch.empty(n, dtype=cdt, device=D.device)
    rl = torch.empty(k, dtype=torch.float64, device=D.device)
    _check(lib.kmedoids_cache(
        ctypes.c_void_p(D.data_ptr()), code, n, ld, k,
        ctypes.c_void_p(med.data_ptr()), ctypes.c_void_p(near.data_ptr()),
        ctypes.c_void_p(sec.data_ptr()), ctypes.c_void_p(dn.data_ptr()),
        ctypes.c_void_p(ds.data_ptr()), ctypes.c_void_p(rl.data_ptr()),
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()))
    return near, sec, dn, ds, rl


def init_weighted(D, k, u, n=None, ws=None):
    """Distance-weighted initialisation (kmedoids_init_weighted): u holds k
    uniform numbers in [0, 1) (array or CUDA float64 tensor).  Returns the
    k drawn medoids (int32 CUDA tensor, draw order)."""
    torch = _torch()
    lib = load()
    n, ld = _matrix(D, n)
    code = _dtype_code(D)
    u = torch.as_tensor(u, dtype=torch.float64).to(D.device).contiguous()
    if ws is None:
        ws = workspace(n, k, code, None, device=D.device)
    med = torch.empty(k, dtype=torch.int32, device=D.device)
    _check(lib.kmedoids_init_weighted(
        ctypes.c_void_p(D.data_ptr()), code, n, ld, int(k),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(med.data_ptr()),
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()))
    return med


def init_lab(D, k, ranks, n=None, ws=None):
    """LAB initialisation (kmedoids_init_lab): ranks (k x s, array or int32
    CUDA tensor) name each step's subsample among the current non-medoids.
    Returns (medoids int32 CUDA tensor, per-step gains as a numpy array)."""
    import numpy as np
    torch = _torch()
    lib = load()
    n, ld = _matrix(D, n)
    code = _dtype_code(D)
    r = torch.as_tensor(ranks, dtype=torch.int32).to(D.device).contiguous()
    if r.dim() != 2:
        raise ValueError("ranks must be k x s")
    if ws is None:
        ws = workspace(n, k, code, None, device=D.device)
    med = torch.empty(k, dtype=torch.int32, device=D.device)
    gains = np.zeros(max(int(k), 1), np.float64)
    _check(lib.kmedoids_init_lab(
        ctypes.c_void_p(D.data_ptr()), code, n, ld, int(k), int(r.shape[1]),
        ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(med.data_ptr()),
        gains.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(ws.data_ptr()),
        ws.numel(), _stream()))
    return med, gains[:k]


def gram_bf16(X):
    """kmedoids_gram_bf16: G = X X^T (FP32) of a bf16 CUDA tensor X (n x d)."""
    torch = _torch()
    lib = load()
    if X.dtype != torch.bfloat16 or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D bf16 CUDA tensor with unit column stride")
    n, d = X.shape
    n_pad = (n + 127) // 128 * 128
    ws = torch.empty(256 + n_pad * d * 2, dtype=torch.uint8, device=X.device)
    G = torch.empty((n, n), dtype=torch.float32, device=X.device)
    _check(lib.kmedoids_gram_bf16(
        ctypes.c_void_p(X.data_ptr()), n, d, X.stride(0),
        ctypes.c_void_p(G.data_ptr()), n, ctypes.c_void_p(ws.data_ptr()),
        ws.numel(), _stream()))
    return G


def _features_call(fn_name, X, k, med, labels, kw):
    torch = _torch()
    lib = load()
    if X.dtype != torch.bfloat16 or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D bf16 CUDA tensor with unit column stride")
    n, d = X.shape
    o = options(**kw)
    gains = fn_name in ("kmedoids_run_features", "kmedoids_build_features")
    tr = _Trace(o, o.trace_capacity, k, gains)
    nbytes = lib.kmedoids_features_workspace_size(n, d, k, ctypes.byref(o))
    if nbytes == 0:
        raise KmError(1, "invalid sizes for the feature form")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=X.device)
    res = km_result()
    st = getattr(lib, fn_name)(
        ctypes.c_void_p(X.data_ptr()), n, d, X.stride(0), k,
        ctypes.c_void_p(med.data_ptr()),
        ctypes.c_void_p(labels.data_ptr() if labels is not None else 0),
        ctypes.byref(o), ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()),
        ws.numel(), _stream())
    if st not in (0, 4):
        _check(st)
    out = _result(res, o, k)
    out["status_name"] = STATUS.get(st, st)
    out["converged"] = st == 0
    out["medoids"] = med
    out["labels"] = labels
    out["trace"] = tr.items(res.swaps) if o.trace_capacity > 0 else []
    if gains:
        out["build_gains"] = tr.g[:k].copy()
    return out


def run_features(X, k, labels=True, **kw):
    """BUILD + FastPAM1 on bf16 features with on-the-fly Euclidean distances
    (kmedoids_run_features)."""
    torch = _torch()
    med = torch.empty(k, dtype=torch.int32, device=X.device)
    lab = torch.empty(X.shape[0], dtype=torch.int32, device=X.device) \
        if labels else None
    return _features_call("kmedoids_run_features", X, k, med, lab, kw)


def build_features(X, k, labels=True, **kw):
    """BUILD alone on bf16 features (kmedoids_build_features): medoids in
    the order chosen, build_gains the gain of each step."""
    torch = _torch()
    med = torch.empty(k, dtype=torch.int32, device=X.device)
    lab = torch.empty(X.shape[0], dtype=torch.int32, device=X.device) \
        if labels else None
    return _features_call("kmedoids_build_features", X, k, med, lab, kw)


def swap_features(X, medoids, labels=True, **kw):
    """FastPAM1 on bf16 features from the given medoids
    (kmedoids_swap_features)."""
    torch = _torch()
    med = torch.as_tensor(medoids, dtype=torch.int32).to(X.device).clone()
    lab = torch.empty(X.shape[0], dtype=torch.int32, device=X.device) \
        if labels else None
    return _features_call("kmedoids_swap_features", X, med.numel(), med, lab, kw)


INSTANCE_DTYPE = [("offset", "<i8"), ("n", "<i4"), ("ld", "<i4"), ("k", "<i4"),
                  ("medoid_offset", "<i4")]
BATCH_RESULT_DTYPE = [("td", "<f8"), ("iterations", "<i4"), ("swaps", "<i4"),
                      ("status", "<i4"), ("pad", "<i4")]


def batch_layout(sizes):
    """Descriptor table for instances of (n, k): arena offsets with row
    stride ld = roundup(n, 4), concatenated medoid offsets.  Returns
    (numpy structured array, arena elements, total medoids)."""
    import numpy as np
    inst = np.zeros(len(sizes), dtype=INSTANCE_DTYPE)
    off = 0
    moff = 0
    for i, (n, k) in enumerate(sizes):
        ld = (n + 3) // 4 * 4
        inst[i] = (off, n, ld, k, moff)
        off += n * ld
        moff += k
    return inst, off, moff


def batched_distances(points, point_offsets, inst_dev, arena):
    """kmedoids_batched_distances: fill the arena from float32 points."""
    torch = _torch()
    lib = load()
    offs = torch.as_tensor(point_offsets, dtype=torch.int64).to(points.device)
    _check(lib.kmedoids_batched_distances(
        ctypes.c_void_p(points.data_ptr()), points.shape[1],
        ctypes.c_void_p(offs.data_ptr()), ctypes.c_void_p(inst_dev.data_ptr()),
        inst_dev.numel() // 24, ctypes.c_void_p(arena.data_ptr()), _stream()))


def run_batched(arena, inst_dev, total_medoids, **kw):
    """kmedoids_run_batched.  inst_dev: uint8 CUDA tensor holding the
    descriptor table.  Returns (medoids tensor, results uint8 tensor)."""
    torch = _torch()
    lib = load()
    count = inst_dev.numel() // 24
    med = torch.empty(total_medoids, dtype=torch.int32, device=arena.device)
    res = torch.empty(count * 24, dtype=torch.uint8, device=arena.device)
    ws = torch.empty(lib.kmedoids_batched_workspace_size(count),
                     dtype=torch.uint8, device=arena.device)
    o = options(**kw)
    _check(lib.kmedoids_run_batched(
        ctypes.c_void_p(arena.data_ptr()), ctypes.c_void_p(inst_dev.data_ptr()),
        count, ctypes.c_void_p(med.data_ptr()), ctypes.c_void_p(res.data_ptr()),
        ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()))
    return med, res


def swap_batched(arena, inst_dev, medoids, **kw):
    """kmedoids_swap_batched: medoids (int32 CUDA tensor, every instance's k
    starting medoids at its medoid_offset) is updated in place.  Returns
    (medoids, results uint8 tensor)."""
    torch = _torch()
    lib = load()
    count = inst_dev.numel() // 24
    res = torch.empty(count * 24, dtype=torch.uint8, device=arena.device)
    ws = torch.empty(lib.kmedoids_batched_workspace_size(count),
                     dtype=torch.uint8, device=arena.device)
    o = options(**kw)
    _check(lib.kmedoids_swap_batched(
        ctypes.c_void_p(arena.data_ptr()), ctypes.c_void_p(inst_dev.data_ptr()),
        count, ctypes.c_void_p(medoids.data_ptr()), ctypes.c_void_p(res.data_ptr()),
        ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()))
    return medoids, res


def clara(X, k, sample_idx):
    """kmedoids_clara: X float32 CUDA (n x d), sample_idx int32 CUDA
    (samples x sample_size).  Returns a dict with medoids, labels,
    sample_td (list), best_sample, td."""
    import numpy as np
    torch = _torch()
    lib = load()
    n, d = X.shape
    samples, s = sample_idx.shape
    ws = torch.empty(lib.kmedoids_clara_workspace_size(k, samples, s),
                     dtype=torch.uint8, device=X.device)
    med = torch.empty(k, dtype=torch.int32, device=X.device)
    lab = torch.empty(n, dtype=torch.int32, device=X.device)
    tds = np.zeros(samples, np.float64)
    res = km_result()
    _check(lib.kmedoids_clara(
        ctypes.c_void_p(X.data_ptr()), n, d, k, samples, s,
        ctypes.c_void_p(sample_idx.data_ptr()), ctypes.c_void_p(med.data_ptr()),
        ctypes.c_void_p(lab.data_ptr()),
        tds.ctypes.data_as(ctypes.c_void_p), ctypes.byref(res),
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()))
    return {"medoids": med, "labels": lab, "sample_td": tds.tolist(),
            "best_sample": res.best_sample, "td": res.td,
            "kernel_launches": res.kernel_launches}


CLARA_RESULT_DTYPE = [("td", "<f8"), ("best_sample", "<i4"), ("status", "<i4")]


def batched_geometry_info(geometry):
    """(warps per CTA, ring stages) of batched geometry 1..5."""
    w, st = ctypes.c_int32(), ctypes.c_int32()
    if load().kmedoids_batched_geometry_info(int(geometry), ctypes.byref(w), ctypes.byref(st)):
        raise KmError(1, "unknown batched geometry %d" % geometry)
    return w.value, st.value


def batched_autotune(arena, inst_dev, total_medoids, measure=True, **kw):
    """kmedoids_batched_autotune: times every geometry of the persistent
    kernel on this batch; returns (best geometry, per-geometry ms or None)."""
    import numpy as np
    torch = _torch()
    lib = load()
    count = inst_dev.numel() // 24
    med = torch.empty(total_medoids, dtype=torch.int32, device=arena.device)
    res = torch.empty(count * 24, dtype=torch.uint8, device=arena.device)
    ws = torch.empty(lib.kmedoids_batched_workspace_size(count),
                     dtype=torch.uint8, device=arena.device)
    o = options(**kw)
    g = ctypes.c_int32()
    ms = np.full(5, -1.0)
    _check(lib.kmedoids_batched_autotune(
        ctypes.c_void_p(arena.data_ptr()), ctypes.c_void_p(inst_dev.data_ptr()),
        count, ctypes.c_void_p(med.data_ptr()), ctypes.c_void_p(res.data_ptr()),
        ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(),
        ctypes.byref(g), ms.ctypes.data_as(ctypes.c_void_p) if measure else None))
    return g.value, (ms.tolist() if measure else None)


class BatchedClara:
    """Device buffers of one kmedoids_run_batched_clara configuration; call
    enqueue() to run it on the current stream (no host synchronisation, so
    it can be captured in a CUDA graph and replayed)."""

    def __init__(self, arena, inst_dev, total_medoids, X, k, sample_idx, labels=True, **kw):
        torch = _torch()
        lib = load()
        dev = X.device
        self.count = 0 if inst_dev is None else inst_dev.numel() // 24
        self.arena, self.inst, self.X, self.S = arena, inst_dev, X, sample_idx
        self.k = int(k)
        self.samples, self.s = sample_idx.shape
        self.medoids = torch.empty(max(1, total_medoids), dtype=torch.int32, device=dev)
        self.results = torch.empty(max(1, self.count) * 24, dtype=torch.uint8, device=dev)
        self.clara_medoids = torch.empty(self.k, dtype=torch.int32, device=dev)
        self.labels = torch.empty(X.shape[0], dtype=torch.int32, device=dev) if labels else None
        self.sample_td = torch.empty(self.samples, dtype=torch.float64, device=dev)
        self.clara_result = torch.empty(16, dtype=torch.uint8, device=dev)
        self.ws = torch.empty(lib.kmedoids_batched_clara_workspace_size(
            self.count, self.k, self.samples, self.s), dtype=torch.uint8, device=dev)
        self.opts = options(**kw)

    def enqueue(self):
        lib = load()
        n, d = self.X.shape
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
        _check(lib.kmedoids_run_batched_clara(
            ptr(self.arena), ptr(self.inst), self.count, ptr(self.medoids), ptr(self.results),
            ptr(self.X), n, d, self.k, self.samples, self.s, ptr(self.S),
            ptr(self.clara_medoids), ptr(self.labels), ptr(self.sample_td),
            ptr(self.clara_result), ctypes.byref(self.opts), ptr(self.ws), self.ws.numel(),
            _stream()))

    def clara_outcome(self):
        import numpy as np
        r = np.frombuffer(self.clara_result.cpu().numpy().tobytes(), dtype=CLARA_RESULT_DTYPE)[0]
        return {"td": float(r["td"]), "best_sample": int(r["best_sample"]),
                "status": int(r["status"])}


def geometry_info(geometry):
    """(rows, stages, ctas_per_sm) of a matrix-form geometry table entry."""
    r, st, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    if load().kmedoids_geometry_info(int(geometry), ctypes.byref(r), ctypes.byref(st),
                                     ctypes.byref(m)):
        raise KmError(1, "unknown geometry %d" % geometry)
    return r.value, st.value, m.value


def version() -> str:
    return load().kmedoids_version().decode()


def _bi_call(fn_name, D, k, n, medoids, labels, ws, kw):
    torch = _torch()
    lib = load()
    if D.dim() != 2 or not D.is_cuda or D.stride(1) != 1:
        raise ValueError("D must be a 2-D CUDA tensor with unit column stride")
    m, ld = D.shape[0], D.stride(0)
    code = _dtype_code(D)
    o = options(**kw)
    tr = _Trace(o, o.trace_capacity, k, True)
    if ws is None:
        nbytes = int(lib.kmedoids_bichromatic_workspace_size(m, int(n), int(k), code, ctypes.byref(o)))
        if nbytes == 0:
            raise KmError(1, "invalid sizes for a workspace")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=D.device)
    res = km_result()
    st = getattr(lib, fn_name)(
        ctypes.c_void_p(D.data_ptr()), code, m, int(n), ld, int(k),
        ctypes.c_void_p(medoids.data_ptr()),
        ctypes.c_void_p(labels.data_ptr() if labels is not None else 0),
        ctypes.byref(o), ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream())
    if st not in (0, 4):
        _check(st)
    out = _result(res, o, k)
    out["status_name"] = STATUS.get(st, st)
    out["converged"] = st == 0
    out["medoids"] = medoids
    out["labels"] = labels
    out["trace"] = tr.items(res.swaps) if o.trace_capacity > 0 else []
    out["build_gains"] = tr.g[:k].copy()
    return out


def run_bichromatic(D, k, n, labels=True, ws=None, **kw):
    """Bichromatic BUILD + SWAP (kmedoids_run_bichromatic): D holds m
    location rows of the distances to n consumers (columns); the medoids are
    location indices, the labels one slot per consumer."""
    torch = _torch()
    med = torch.empty(k, dtype=torch.int32, device=D.device)
    lab = torch.empty(int(n), dtype=torch.int32, device=D.device) if labels else None
    return _bi_call("kmedoids_run_bichromatic", D, k, n, med, lab, ws, kw)


def swap_bichromatic(D, medoids, n, labels=True, ws=None, **kw):
    """Bichromatic SWAP from the given locations (kmedoids_swap_bichromatic)."""
    torch = _torch()
    med = torch.as_tensor(medoids, dtype=torch.int32).to(D.device).clone()
    lab = torch.empty(int(n), dtype=torch.int32, device=D.device) if labels else None
    return _bi_call("kmedoids_swap_bichromatic", D, med.numel(), n, med, lab, ws, kw)


def upload(H, n=None, D=None, ld=None, device=None):
    """kmedoids_upload_rows: the rows of H (a CPU tensor with unit column
    stride, int32 / float32 / 16-bit; pinned memory is read by the SMs over
    the CPU-GPU link), n elements each (default: as many as H has rows, the
    square matrix), into the device tensor D (allocated with ld columns
    when None, ld defaulting to n rounded up to the library's alignment: 4
    elements, 8 for 16-bit).  Columns n .. ld-1 of D are set to zero.
    Returns D."""
    torch = _torch()
    if H.dim() != 2 or H.is_cuda or H.stride(1) != 1:
        raise ValueError("H must be a 2-D CPU tensor with unit column stride")
    code = _dtype_code(H)
    rows = H.shape[0]
    n = rows if n is None else int(n)
    if D is None:
        a = 8 if code == KM_U16 else 4
        ld = (n + a - 1) // a * a if ld is None else int(ld)
        D = torch.empty((rows, ld), dtype=H.dtype, device=device or "cuda")
    if D.dim() != 2 or not D.is_cuda or D.stride(1) != 1 or D.dtype != H.dtype or \
            D.shape[0] < rows:
        raise ValueError("D must be a 2-D CUDA tensor of H's dtype with unit column stride "
                         "and at least H's rows")
    with torch.cuda.device(D.device):
        _check(load().kmedoids_upload_rows(
            ctypes.c_void_p(H.data_ptr()), H.stride(0), code, rows, n,
            ctypes.c_void_p(D.data_ptr()), D.stride(0), _stream()))
    return D


def wait_selftest(kind, limit_ns, device=None):
    """kmedoids_wait_selftest: a kernel waits on something that never
    happens (kind 0 an mbarrier phase, 1 a consumer barrier, 2 the grid
    barrier) until limit_ns runs out.  Returns (status, message); the
    expected status is KM_E_TIMEOUT (5)."""
    torch = _torch()
    lib = load()
    ws = torch.zeros(512, dtype=torch.uint8, device=device or "cuda")
    st = lib.kmedoids_wait_selftest(int(kind), int(limit_ns), ctypes.c_void_p(ws.data_ptr()),
                                    ws.numel(), _stream())
    return st, lib.kmedoids_last_error().decode()
