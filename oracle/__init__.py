"""FP64 CPU oracle for the k-medoids hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  It wraps
``kmedoids_oracle.c`` (plain C, FP64) with ctypes; nothing here touches the
CUDA library and the CUDA library never touches this.

Every function follows a passage of Schubert & Rousseeuw, "Fast and Eager
k-Medoids Clustering" (arXiv 2008.05171):

* ``td``            -- Eq. (2) (TD objective), labels = lowest nearest slot;
                       ``td_points`` the same on feature vectors (FP64).
* ``cache``         -- the per-point cache nearest / d_n / d_s of Sec. 2.
* ``removal_loss``  -- Delta^{-m_i} of Eq. (7).
* ``pam_build``     -- Alg. 1 (PAM BUILD), self term included in each gain;
                       ``build_gains`` one step of it given a prefix.
* ``eval_swaps``    -- one SWAP evaluation: brute force (Eq. (2) recomputed),
                       PAM (Alg. 2 + Eq. (5)) or FastPAM1 (Alg. 3 + Eq. (7)).
* ``swap_delta``    -- Delta of one (slot, candidate) swap by Eq. (5).
* ``swap``          -- SWAP to convergence: PAM brute force / PAM cached /
                       FastPAM1 / FastPAM2 / FasterPAM (Alg. 4).
* ``clarans``       -- FastCLARANS (Sec. 3.4) over given candidate draws.
* ``init_weighted`` -- distance-weighted initialisation (Sec. 2.3 / 3.3) from
                       given uniform numbers.
* ``init_lab``      -- LAB, BUILD on a fresh subsample per medoid (Sec. 3.3),
                       from given subsample ranks.
* ``clara``         -- CLARA (Sec. 2.1, FastCLARA of Sec. 3.4) on given
                       samples; ``euclid_f32`` the FP64 -> float32 matrix.
* ``bi_*``          -- the bichromatic case of the Outlook (``bichromatic.c``):
                       medoids among m locations (rows), TD over n consumers
                       (columns); ``bi_td``, ``bi_build`` (Alg. 1, step 0 the
                       bichromatic medoid), ``bi_eval_swaps`` (brute force or
                       Eq. (7)), ``bi_swap`` / ``bi_run`` (FastPAM1, Alg. 3).

Parity unpinned: the reading of FastPAM2's additional swaps (the paper
describes FastPAM2 only in words, Sec. 3.2, and prints no values for it).
The tests pin the oracle to a brute-force replay of that reading.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmedoids_oracle.c")
_SRC_BI = os.path.join(_HERE, "bichromatic.c")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

VARIANTS = {"pam_bruteforce": 0, "pam": 1, "fastpam1": 2, "fastpam2": 3,
            "fasterpam": 4}
EVAL_METHODS = {"bruteforce": 0, "pam": 1, "fastpam1": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over candidates) in place."""
    if force or not os.path.exists(_SO) or \
            os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_BI)):
        tmp = _SO + ".tmp%d" % os.getpid()
        # -ffp-contract=off: no fused multiply-add unless the source asks for
        # one, so the results do not depend on the host architecture
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-fopenmp", "-o", tmp, _SRC, _SRC_BI, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_td.restype = f64
            lib.oracle_td.argtypes = [P, i32, i64, i64, P, i32, P]
            lib.oracle_cache.restype = None
            lib.oracle_cache.argtypes = [P, i32, i64, i64, P, i32, P, P, P, P]
            lib.oracle_removal_loss.restype = None
            lib.oracle_removal_loss.argtypes = [i64, i32, P, P, P, P]
            lib.oracle_build.restype = i32
            lib.oracle_build.argtypes = [P, i32, i64, i64, i32, P, P, P]
            lib.oracle_eval_swaps.restype = None
            lib.oracle_eval_swaps.argtypes = [P, i32, i64, i64, P, i32, i32,
                                              P, P, P, P, P]
            lib.oracle_swap_delta.restype = f64
            lib.oracle_swap_delta.argtypes = [P, i32, i64, i64, P, i32, i32,
                                              i64]
            lib.oracle_swap.restype = i32
            lib.oracle_swap.argtypes = [P, i32, i64, i64, i32, P, i32, i32,
                                        f64, f64, P, P, i32, P, P, P]
            lib.oracle_build_gains.restype = None
            lib.oracle_build_gains.argtypes = [P, i32, i64, i64, P, i32, P]
            lib.oracle_init_weighted.restype = i32
            lib.oracle_init_weighted.argtypes = [P, i32, i64, i64, i32, P, P]
            lib.oracle_td_points.restype = f64
            lib.oracle_td_points.argtypes = [P, i64, i32, P, i32, P]
            lib.oracle_init_lab.restype = i32
            lib.oracle_init_lab.argtypes = [P, i32, i64, i64, i32, i32, P, P, P]
            lib.oracle_fixed_shift.restype = i32
            lib.oracle_fixed_shift.argtypes = [P, i32, i64, i64]
            lib.oracle_clarans.restype = i32
            lib.oracle_clarans.argtypes = [P, i32, i64, i64, i32, P, P, i64, i64,
                                           f64, P, P, i32, P, P, P]
            lib.oracle_euclid_f32.restype = None
            lib.oracle_euclid_f32.argtypes = [P, i64, i32, P, i64, P]
            lib.oracle_clara.restype = i32
            lib.oracle_clara.argtypes = [P, i64, i32, i32, i32, i32, P, P, P,
                                         P, P]
            lib.oracle_bi_td.restype = f64
            lib.oracle_bi_td.argtypes = [P, i32, i64, i64, i64, P, i32, P]
            lib.oracle_bi_build.restype = i32
            lib.oracle_bi_build.argtypes = [P, i32, i64, i64, i64, i32, P, P, P]
            lib.oracle_bi_eval_swaps.restype = None
            lib.oracle_bi_eval_swaps.argtypes = [P, i32, i64, i64, i64, P, i32, i32,
                                                 P, P, P, P, P]
            lib.oracle_bi_swap.restype = i32
            lib.oracle_bi_swap.argtypes = [P, i32, i64, i64, i64, i32, P, i32, f64,
                                           P, P, i32, P, P, P]
            lib.oracle_num_threads.restype = i32
            lib.oracle_set_threads.argtypes = [i32]
            _LIB = lib
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mat(D: np.ndarray, n: int | None = None):
    """Return (array, dtype code, n, ld) for a C-contiguous (n, ld) matrix."""
    D = np.ascontiguousarray(D)
    if D.dtype == np.int32:
        code = 0
    elif D.dtype == np.float32:
        code = 1
    else:
        raise TypeError("oracle matrices are int32 or float32")
    rows, ld = D.shape
    n = rows if n is None else n
    if n > rows or n > ld:
        raise ValueError("n exceeds the matrix shape")
    return D, code, n, ld


def _med(medoids) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(medoids, dtype=np.int32))


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def set_threads(t: int) -> None:
    _lib().oracle_set_threads(int(t))


def td(D, medoids, n=None, return_labels=False):
    D, code, n, ld = _mat(D, n)
    med = _med(medoids)
    labels = np.empty(n, dtype=np.int32)
    v = _lib().oracle_td(_p(D), code, n, ld, _p(med), len(med), _p(labels))
    return (v, labels) if return_labels else v


def td_points(X, medoids, return_labels=False):
    """Eq. (2) for feature vectors: TD of the medoids (point indices) with
    Euclidean distances computed directly in FP64 (no matrix)."""
    X = np.ascontiguousarray(X, np.float32)
    med = _med(medoids)
    n, d = X.shape
    labels = np.empty(n, dtype=np.int32)
    v = _lib().oracle_td_points(_p(X), n, d, _p(med), len(med), _p(labels))
    return (v, labels) if return_labels else v


def cache(D, medoids, n=None):
    D, code, n, ld = _mat(D, n)
    med = _med(medoids)
    near = np.empty(n, np.int32)
    sec = np.empty(n, np.int32)
    dn = np.empty(n, np.float64)
    ds = np.empty(n, np.float64)
    _lib().oracle_cache(_p(D), code, n, ld, _p(med), len(med), _p(near),
                        _p(sec), _p(dn), _p(ds))
    return near, sec, dn, ds


def removal_loss(near, dn, ds, k):
    near = np.ascontiguousarray(near, np.int32)
    dn = np.ascontiguousarray(dn, np.float64)
    ds = np.ascontiguousarray(ds, np.float64)
    rl = np.empty(k, np.float64)
    _lib().oracle_removal_loss(len(near), k, _p(near), _p(dn), _p(ds), _p(rl))
    return rl


def pam_build(D, k, n=None):
    """Alg. 1 (BUILD). Returns (medoids int32[k], TD, step gains float64[k])."""
    D, code, n, ld = _mat(D, n)
    med = np.empty(k, np.int32)
    tdv = np.zeros(1, np.float64)
    steps = np.empty(k, np.float64)
    _lib().oracle_build(_p(D), code, n, ld, k, _p(med), _p(tdv), _p(steps))
    return med, float(tdv[0]), steps


def build_gains(D, prefix, n=None):
    """Gains of every candidate for the BUILD step after ``prefix`` (Alg. 1);
    with an empty prefix, the distance sums of step 0.  Medoids get +inf."""
    D, code, n, ld = _mat(D, n)
    med = _med(prefix) if len(prefix) else np.zeros(1, np.int32)
    g = np.empty(n, np.float64)
    _lib().oracle_build_gains(_p(D), code, n, ld, _p(med), len(prefix), _p(g))
    return g


def eval_swaps(D, medoids, method="fastpam1", n=None):
    """One SWAP evaluation. Returns (cand_delta[n], cand_slot[n], best)
    with best = (delta, slot, cand) the lexicographic minimum."""
    D, code, n, ld = _mat(D, n)
    med = _med(medoids)
    cd = np.empty(n, np.float64)
    cs = np.empty(n, np.int32)
    bd = np.zeros(1, np.float64)
    bs = np.zeros(1, np.int32)
    bc = np.zeros(1, np.int64)
    _lib().oracle_eval_swaps(_p(D), code, n, ld, _p(med), len(med),
                             EVAL_METHODS[method], _p(cd), _p(cs), _p(bd),
                             _p(bs), _p(bc))
    return cd, cs, (float(bd[0]), int(bs[0]), int(bc[0]))


def swap_delta(D, medoids, slot, cand, n=None):
    D, code, n, ld = _mat(D, n)
    med = _med(medoids)
    return float(_lib().oracle_swap_delta(_p(D), code, n, ld, _p(med),
                                          len(med), int(slot), int(cand)))


def swap(D, medoids, variant="fastpam1", max_iter=1000, tol=0.0,
         fastpam2_tol=0.0, n=None, trace_cap=None):
    """SWAP to convergence from ``medoids``.  Returns a dict with medoids,
    iterations, swaps, converged, visited, td_bookkept, td and the trace of
    applied swaps (delta, slot, cand)."""
    D, code, n, ld = _mat(D, n)
    med = _med(medoids).copy()
    k = len(med)
    cap = int(trace_cap if trace_cap is not None else max(16, 4 * k + 64))
    stats = np.zeros(4, np.int64)
    tdv = np.zeros(2, np.float64)
    tr_d = np.zeros(cap, np.float64)
    tr_i = np.zeros(cap, np.int32)
    tr_c = np.zeros(cap, np.int64)
    _lib().oracle_swap(_p(D), code, n, ld, k, _p(med), VARIANTS[variant],
                       int(max_iter), float(tol), float(fastpam2_tol),
                       _p(stats), _p(tdv), cap, _p(tr_d), _p(tr_i), _p(tr_c))
    ns = min(int(stats[1]), cap)
    return {
        "medoids": med, "iterations": int(stats[0]), "swaps": int(stats[1]),
        "converged": bool(stats[2]), "visited": int(stats[3]),
        "td_bookkept": float(tdv[0]), "td": float(tdv[1]),
        "trace": list(zip(tr_d[:ns].tolist(), tr_i[:ns].tolist(),
                          tr_c[:ns].tolist())),
    }


def init_weighted(D, k, u, n=None):
    """Distance-weighted initialisation (Sec. 2.3 / 3.3) driven by the given
    uniform numbers u (k values in [0, 1)): k distinct medoids in draw
    order."""
    D, code, n, ld = _mat(D, n)
    u = np.ascontiguousarray(u, np.float64)
    assert len(u) >= k
    med = np.empty(k, np.int32)
    if _lib().oracle_init_weighted(_p(D), code, n, ld, int(k), _p(u), _p(med)) != 0:
        raise ValueError("oracle_init_weighted: need 1 <= k <= n")
    return med


def lab_sample_size(n):
    """LAB's subsample size 10 + ceil(sqrt(n)) (Sec. 3.3)."""
    r = int(np.floor(np.sqrt(n)))
    while r * r < n:
        r += 1
    return 10 + r


def init_lab(D, k, ranks, n=None, gains=False):
    """LAB, Linear Approximative BUILD (Sec. 3.3): before each of the k
    choices, BUILD's gain over a subsample only.  ``ranks`` (k x s) name the
    subsample of step t as ranks among the n - t non-medoids in index order.
    Returns the k medoids in choice order (and each step's gain)."""
    D, code, n, ld = _mat(D, n)
    ranks = np.ascontiguousarray(ranks, np.int32)
    assert ranks.ndim == 2 and ranks.shape[0] >= k
    s = ranks.shape[1]
    med = np.empty(k, np.int32)
    g = np.empty(k, np.float64)
    if _lib().oracle_init_lab(_p(D), code, n, ld, int(k), int(s), _p(ranks), _p(med),
                              _p(g)) != 0:
        raise ValueError("oracle_init_lab: invalid sizes or ranks")
    return (med, g) if gains else med


def fixed_shift(D, n=None):
    """The fixed-point exponent f of the SWAP sums for this matrix."""
    D, code, n, ld = _mat(D, n)
    return int(_lib().oracle_fixed_shift(_p(D), code, n, ld))


def clarans(D, medoids, cand, maxneighbor, tol=0.0, n=None, trace_cap=None):
    """FastCLARANS (Sec. 3.4) from ``medoids`` over the given candidate draws
    ``cand``, stopping after ``maxneighbor`` consecutive failed draws.
    Returns a dict with medoids, consumed (draws used), swaps, stopped,
    evaluated, td_bookkept, td and the trace (delta, slot, cand)."""
    D, code, n, ld = _mat(D, n)
    med = _med(medoids).copy()
    k = len(med)
    cand = np.ascontiguousarray(cand, np.int32)
    cap = int(trace_cap if trace_cap is not None else max(16, 4 * k + 64))
    stats = np.zeros(4, np.int64)
    tdv = np.zeros(2, np.float64)
    tr_d = np.zeros(cap, np.float64)
    tr_i = np.zeros(cap, np.int32)
    tr_c = np.zeros(cap, np.int64)
    rc = _lib().oracle_clarans(_p(D), code, n, ld, k, _p(med), _p(cand), len(cand),
                               int(maxneighbor), float(tol), _p(stats), _p(tdv), cap,
                               _p(tr_d), _p(tr_i), _p(tr_c))
    if rc != 0:
        raise ValueError("oracle_clarans: need 2 <= k < n, maxneighbor >= 1")
    ns = min(int(stats[1]), cap)
    return {
        "medoids": med, "consumed": int(stats[0]), "swaps": int(stats[1]),
        "stopped": bool(stats[2]), "evaluated": int(stats[3]),
        "td_bookkept": float(tdv[0]), "td": float(tdv[1]),
        "trace": list(zip(tr_d[:ns].tolist(), tr_i[:ns].tolist(), tr_c[:ns].tolist())),
    }


def euclid_f32(X, idx=None, ld=None):
    """Euclidean matrix of float32 points computed in FP64, rounded once to
    float32 (rows padded to ld with zeros)."""
    X = np.ascontiguousarray(X, np.float32)
    m = X.shape[0] if idx is None else len(idx)
    ld = (m + 3) // 4 * 4 if ld is None else ld
    D = np.empty((m, ld), np.float32)
    ix = None if idx is None else np.ascontiguousarray(idx, np.int64)
    _lib().oracle_euclid_f32(_p(X), m, X.shape[1],
                             _p(ix) if ix is not None else None, ld, _p(D))
    return D


def clara(X, k, sample_idx):
    """CLARA (Sec. 2.1 / 3.4): PAM (BUILD + FastPAM1) on each given sample,
    full-data TD of each, best sample kept.  Returns (medoids, labels,
    sample_tds, best_sample)."""
    X = np.ascontiguousarray(X, np.float32)
    S = np.ascontiguousarray(sample_idx, np.int32)
    samples, s = S.shape
    n, d = X.shape
    med = np.empty(k, np.int32)
    lab = np.empty(n, np.int32)
    tds = np.empty(samples, np.float64)
    best = np.zeros(1, np.int32)
    _lib().oracle_clara(_p(X), n, d, k, samples, s, _p(S), _p(med), _p(lab),
                        _p(tds), _p(best))
    return med, lab, tds, int(best[0])


def run(D, k, variant="fastpam1", n=None, **kw):
    """BUILD followed by SWAP (the paper's full PAM / FastPAM1 / FasterPAM)."""
    med, td_build, _ = pam_build(D, k, n=n)
    out = swap(D, med, variant=variant, n=n, **kw)
    out["build_medoids"] = med
    out["td_build"] = td_build
    return out


# ------------------------------------------------------------ bichromatic
def _bimat(D: np.ndarray, n: int | None = None):
    """(array, dtype code, m, n, ld) of an (m locations, ld) matrix whose
    first n columns are the consumers: d(x_c, x_l) = D[l, c]."""
    D = np.ascontiguousarray(D)
    if D.dtype == np.int32:
        code = 0
    elif D.dtype == np.float32:
        code = 1
    else:
        raise TypeError("oracle matrices are int32 or float32")
    m, ld = D.shape
    n = ld if n is None else int(n)
    if n > ld:
        raise ValueError("n exceeds the row length")
    return D, code, m, n, ld


def bi_td(D, medoids, n=None, return_labels=False):
    """TD over the consumers (Eq. (2)) of medoid locations ``medoids``."""
    D, code, m, n, ld = _bimat(D, n)
    med = _med(medoids)
    labels = np.empty(n, np.int32)
    v = _lib().oracle_bi_td(_p(D), code, m, n, ld, _p(med), len(med), _p(labels))
    return (float(v), labels) if return_labels else float(v)


def bi_build(D, k, n=None):
    """BUILD over the locations (Alg. 1): (medoids, TD, gain per step)."""
    D, code, m, n, ld = _bimat(D, n)
    med = np.empty(k, np.int32)
    tdv = np.zeros(1, np.float64)
    steps = np.zeros(k, np.float64)
    if _lib().oracle_bi_build(_p(D), code, m, n, ld, int(k), _p(med), _p(tdv), _p(steps)) != 0:
        raise ValueError("oracle_bi_build: need 1 <= k <= m")
    return med, float(tdv[0]), steps


def bi_eval_swaps(D, medoids, method="fastpam1", n=None):
    """Every (slot, location) swap: (cand_delta[m], cand_slot[m], (best_delta,
    best_slot, best_location))."""
    D, code, m, n, ld = _bimat(D, n)
    med = _med(medoids)
    cd = np.zeros(m, np.float64)
    cs = np.zeros(m, np.int32)
    bd = np.zeros(1, np.float64)
    bs = np.zeros(1, np.int32)
    bc = np.zeros(1, np.int64)
    _lib().oracle_bi_eval_swaps(_p(D), code, m, n, ld, _p(med), len(med),
                                EVAL_METHODS[method], _p(cd), _p(cs), _p(bd), _p(bs), _p(bc))
    return cd, cs, (float(bd[0]), int(bs[0]), int(bc[0]))


def bi_swap(D, medoids, max_iter=1000, tol=0.0, n=None, trace_cap=None):
    """FastPAM1 SWAP to convergence over the locations (Alg. 3)."""
    D, code, m, n, ld = _bimat(D, n)
    med = _med(medoids).copy()
    k = len(med)
    cap = int(trace_cap if trace_cap is not None else max(16, 4 * k + 64))
    stats = np.zeros(3, np.int64)
    tdv = np.zeros(2, np.float64)
    tr_d = np.zeros(cap, np.float64)
    tr_i = np.zeros(cap, np.int32)
    tr_c = np.zeros(cap, np.int64)
    _lib().oracle_bi_swap(_p(D), code, m, n, ld, k, _p(med), int(max_iter), float(tol),
                          _p(stats), _p(tdv), cap, _p(tr_d), _p(tr_i), _p(tr_c))
    ns = min(int(stats[1]), cap)
    return {
        "medoids": med, "iterations": int(stats[0]), "swaps": int(stats[1]),
        "converged": bool(stats[2]), "td_bookkept": float(tdv[0]), "td": float(tdv[1]),
        "trace": list(zip(tr_d[:ns].tolist(), tr_i[:ns].tolist(), tr_c[:ns].tolist())),
    }


def bi_run(D, k, n=None, **kw):
    """BUILD then FastPAM1 SWAP in the bichromatic case."""
    med, td_build, _ = bi_build(D, k, n=n)
    out = bi_swap(D, med, n=n, **kw)
    out["build_medoids"] = med
    out["td_build"] = td_build
    return out
