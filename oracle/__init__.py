"""CPU FP64 oracle for mixed-precision Lloyd's k-means (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or calls it, and the two share
no code: the oracle's arithmetic lives in ``mpkm_oracle.c`` (plain C,
binary64, built with ``-ffp-contract=off``) plus the few numpy helpers
below, each citing the passage of Carson, Chen & Liu, "Computing k-means in
Mixed Precision" (arXiv 2407.12208) it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpkm_oracle.c")
_LIB = os.path.join(_HERE, "libmpkm_oracle.so")
_lock = threading.Lock()
_lib = None

FMT_FP16, FMT_BF16, FMT_E4M3 = 0, 1, 2

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over points, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.orc_unit_roundoff.restype = c.c_double
        lib.orc_unit_roundoff.argtypes = [c.c_int]
        lib.orc_round_to_format.restype = c.c_double
        lib.orc_round_to_format.argtypes = [c.c_double, c.c_int]
        lib.orc_quantize.restype = None
        lib.orc_quantize.argtypes = [_f32p, c.c_int64, c.c_int, _f32p]
        lib.orc_gamma.restype = c.c_double
        lib.orc_gamma.argtypes = [c.c_int, c.c_double]
        lib.orc_dist_labelled.restype = None
        lib.orc_dist_labelled.argtypes = [_f32p, c.c_int64, _f32p, c.c_int, c.c_int, _i32p, _f64p]
        lib.orc_dist_direct.restype = None
        lib.orc_dist_direct.argtypes = [_f32p, c.c_int64, _f32p, c.c_int, c.c_int, _f64p]
        lib.orc_assign.restype = None
        lib.orc_assign.argtypes = [_f32p, c.c_int64, _f32p, c.c_int, c.c_int, _i32p, _f64p, _f64p]
        lib.orc_update.restype = c.c_int
        lib.orc_update.argtypes = [_f32p, c.c_int64, c.c_int, _i32p, c.c_int, _f32p, c.c_int,
                                   c.c_void_p, _f32p, _i64p, c.POINTER(c.c_double)]
        lib.orc_lloyd.restype = c.c_int
        lib.orc_lloyd.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, _f32p, c.c_int, c.c_double,
                                  c.c_int, _f32p, _i32p, _f64p, c.POINTER(c.c_int)]
        lib.orc_mp_dist_paper.restype = c.c_int
        lib.orc_mp_dist_paper.argtypes = [_f32p, _f32p, c.c_int, c.c_double, c.c_double, c.c_int,
                                          c.POINTER(c.c_double), c.POINTER(c.c_double),
                                          c.POINTER(c.c_double)]
        lib.orc_dist_direct_fmt.restype = c.c_double
        lib.orc_dist_direct_fmt.argtypes = [_f32p, _f32p, c.c_int, c.c_int]
        lib.orc_mp_dist_fb.restype = c.c_int
        lib.orc_mp_dist_fb.argtypes = [_f32p, _f32p, c.c_int, c.c_double, c.c_double, c.c_int, c.c_int,
                                       c.POINTER(c.c_double), c.POINTER(c.c_double), c.POINTER(c.c_double)]
        lib.orc_tc_bound.restype = c.c_double
        lib.orc_tc_bound.argtypes = [c.c_double] * 7 + [c.c_int, c.c_int]
        lib.orc_row_quant_stats.restype = None
        lib.orc_row_quant_stats.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, c.c_int, _f32p,
                                            _f64p, _f64p, _f64p, _f64p, _f64p]
        lib.orc_expanded_quantised.restype = c.c_double
        lib.orc_kmeanspp.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, _f64p, c.c_void_p, _i64p, c.c_void_p]
        lib.orc_kmeanspp.restype = c.c_int
        lib.orc_expanded_quantised.argtypes = [_f32p, _f32p, c.c_int, c.c_double, c.c_double]
        _lib = lib
        return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


# --- Table 1.1 -------------------------------------------------------------
def unit_roundoff(fmt: int) -> float:
    """u of Table 1.1 (fmt 0 fp16, 1 bf16, 2 E4M3, 3 fp32, 4 fp64)."""
    return _load().orc_unit_roundoff(fmt)


def gamma(m: int, u: float) -> float:
    """gamma_m = m u / (1 - m u), Eq. (fpmode-vecprod)."""
    return _load().orc_gamma(int(m), float(u))


def round_to_format(v: float, fmt: int) -> float:
    return _load().orc_round_to_format(float(v), int(fmt))


def quantize(x, fmt: int) -> np.ndarray:
    x = _f32(x)
    out = np.empty_like(x)
    _load().orc_quantize(x.reshape(-1), x.size, int(fmt), out.reshape(-1))
    return out


# --- Eq. (dist-direct), Alg. 1 ---------------------------------------------
def dist_direct(X, C) -> np.ndarray:
    """All-pairs squared distances by Eq. (dist-direct) in binary64."""
    X, C = _f32(X), _f32(C)
    n, d = X.shape
    k = C.shape[0]
    D = np.empty((n, k), dtype=np.float64)
    _load().orc_dist_direct(X, n, C, k, d, D)
    return D


def dist_labelled(X, C, labels) -> np.ndarray:
    """Eq. (dist-direct) in binary64 between each x_i and c_{labels[i]}."""
    X, C = _f32(X), _f32(C)
    n, d = X.shape
    k = C.shape[0]
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    out = np.empty(n, dtype=np.float64)
    _load().orc_dist_labelled(X, n, C, k, d, lab, out)
    return out


def assign(X, C):
    """Alg. 1 assignment: (labels, best distance, second-best distance)."""
    X, C = _f32(X), _f32(C)
    n, d = X.shape
    k = C.shape[0]
    lab = np.empty(n, dtype=np.int32)
    d1 = np.empty(n, dtype=np.float64)
    d2 = np.empty(n, dtype=np.float64)
    _load().orc_assign(X, n, C, k, d, lab, d1, d2)
    return lab, d1, d2


def update(X, labels, C_old, empty_policy: int = 1, min_dist=None):
    """Eq. (center): (C_new fp32, counts, shift)."""
    X, C_old = _f32(X), _f32(C_old)
    n, d = X.shape
    k = C_old.shape[0]
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    Cn = np.empty_like(C_old)
    cnt = np.empty(k, dtype=np.int64)
    sh = ctypes.c_double(0.0)
    md = None
    md_ptr = None
    if min_dist is not None:
        md = np.ascontiguousarray(min_dist, dtype=np.float64)
        md_ptr = md.ctypes.data_as(ctypes.c_void_p)
    rc = _load().orc_update(X, n, d, lab, k, C_old, int(empty_policy), md_ptr, Cn, cnt,
                            ctypes.byref(sh))
    if rc != 0:
        raise ValueError("oracle update: invalid labels")
    return Cn, cnt, sh.value


def lloyd(X, C_init, max_iter: int, tau: float = 0.0, empty_policy: int = 1):
    """Alg. 1 with binary64 direct distances: (C, labels, sse[iters+1], iters)."""
    X, C0 = _f32(X), _f32(C_init)
    n, d = X.shape
    k = C0.shape[0]
    Cout = np.empty_like(C0)
    lab = np.empty(n, dtype=np.int32)
    sse = np.zeros(max_iter + 1, dtype=np.float64)
    it = ctypes.c_int(0)
    rc = _load().orc_lloyd(X, n, d, k, C0, int(max_iter), float(tau), int(empty_policy), Cout, lab,
                           sse, ctypes.byref(it))
    if rc != 0:
        raise ValueError("oracle lloyd: invalid arguments")
    return Cout, lab, sse[: it.value + 1], it.value


def kmeanspp(X, u, follow=None):
    """D^2-sampling seeds with the draws u (k values in [0, 1)): (indices,
    margins).  follow: continue each step from these indices instead of the
    oracle's own (margins are then those of the followed sequence)."""
    X = _f32(X)
    n, d = X.shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    k = len(u)
    idx = np.empty(k, dtype=np.int64)
    mg = np.empty(k, dtype=np.float64)
    fp = None
    if follow is not None:
        follow = np.ascontiguousarray(follow, dtype=np.int64)
        fp = follow.ctypes.data_as(ctypes.c_void_p)
    rc = _load().orc_kmeanspp(X, n, d, k, u, fp, idx, mg.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("oracle kmeanspp: invalid arguments")
    return idx, mg


# --- Alg. 2 ---------------------------------------------------------------
def mp_dist_paper(x, y, rho: float, fmt: int, c_A: float = 1.0):
    """Alg. 2 verbatim in emulated low precision.

    Returns (flag, d, dhat, E); flag is None when gamma^l_{r+2} is undefined.
    """
    x, y = _f32(x), _f32(y)
    dd, dh, E = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    f = _load().orc_mp_dist_paper(x, y, x.size, float(rho), float(c_A), int(fmt),
                                  ctypes.byref(dd), ctypes.byref(dh), ctypes.byref(E))
    if f < 0:
        return None, None, None, None
    return bool(f), dd.value, dh.value, E.value


def dist_direct_fmt(x, y, fmt: int) -> float:
    """Eq. (dist-direct) with every operation rounded to fmt (0 fp16, 1 bf16,
    3 fp32, 4 fp64): the fallback of Section 4.2 in that precision."""
    x, y = _f32(x), _f32(y)
    return _load().orc_dist_direct_fmt(x, y, x.size, int(fmt))


def mp_dist_fb(x, y, rho: float, fmt: int, fb_fmt: int, c_A: float = 1.0):
    """Alg. 2 (every low-precision op rounded; fmt 3 = binary32) with the
    fallback of Eq. (fallback-rule) in precision fb_fmt: (flag, d, dhat, E)."""
    x, y = _f32(x), _f32(y)
    dd, dh, E = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    f = _load().orc_mp_dist_fb(x, y, x.size, float(rho), float(c_A), int(fmt), int(fb_fmt),
                               ctypes.byref(dd), ctypes.byref(dh), ctypes.byref(E))
    if f < 0:
        return None, None, None, None
    return bool(f), dd.value, dh.value, E.value


def tc_bound(nrx, nc, nxq, nrc, ncq, p, q, d: int, fmt: int) -> float:
    """Error bound B of the tensor-core instantiation of Theorem 4.2."""
    return _load().orc_tc_bound(float(nrx), float(nc), float(nxq), float(nrc), float(ncq),
                                float(p), float(q), int(d), int(fmt))


def row_quant_stats(X, fmt: int, per_row_scale: bool = False):
    """Quantised rows and (p fp32-rounded, ||x||, ||x~||, ||x~-x||, scale)."""
    X = _f32(X)
    n, d = X.shape
    Xq = np.empty_like(X)
    p = np.empty(n); nx = np.empty(n); nq = np.empty(n); nr = np.empty(n); sc = np.empty(n)
    _load().orc_row_quant_stats(X, n, d, int(fmt), int(bool(per_row_scale)), Xq, p, nx, nq, nr, sc)
    return Xq, p, nx, nq, nr, sc


def tc_bound_matrix(X, C, fmt: int, per_row_scale: bool = False):
    """B_ij for all pairs (numpy broadcast of tc_bound's formula)."""
    d = X.shape[1]
    _, p, nx, nxq, nrx, _ = row_quant_stats(X, fmt, per_row_scale)
    _, q, nc, ncq, nrc, _ = row_quant_stats(C, fmt, per_row_scale)
    u32 = 2.0 ** -24
    uacc = 2.0 ** -13 if fmt == FMT_E4M3 else 2.0 ** -21
    kacc = 2.0 * gamma(d, uacc) + 4.0 * u32
    kn = 4.0 * u32
    return (2.0 * np.outer(nrx, nc) + 2.0 * np.outer(nxq, nrc) + kacc * np.outer(nxq, ncq)
            + kn * (p[:, None] + q[None, :]))


def predict_tc_flags(X, C, fmt: int, rho: float, test: str = "tc", c_A: float = 2.0,
                     per_row_scale: bool = False):
    """Flag prediction for the GPU's reliability test with a borderline band.

    The reference expanded value uses the exact cross term of the quantised
    data (a binary64 matmul of the quantised operands) and the fp32-rounded
    norms.  A pair whose reference value is further than the band from the
    threshold must be decided the same way by the GPU; inside the band either
    decision is valid (the GPU's fp32 accumulation moves d^ by at most the
    accumulation and rounding terms of B).  Returns (sure, maybe) boolean
    matrices: sure = flagged for certain, maybe = borderline.
    """
    X, C = _f32(X), _f32(C)
    d = X.shape[1]
    Xq, p, nx, nxq, nrx, _ = row_quant_stats(X, fmt, per_row_scale)
    Cq, q, nc, ncq, nrc, _ = row_quant_stats(C, fmt, per_row_scale)
    g = Xq.astype(np.float64) @ Cq.astype(np.float64).T
    dref = p[:, None] + q[None, :] - 2.0 * g
    u32 = 2.0 ** -24
    uacc = 2.0 ** -13 if fmt == FMT_E4M3 else 2.0 ** -21
    kacc = 2.0 * gamma(d, uacc) + 4.0 * u32
    B = tc_bound_matrix(X, C, fmt, per_row_scale)
    if test == "tc":
        thr = rho * B
    else:  # Alg. 2's E with the norms of the quantised data
        ul = unit_roundoff(fmt)
        thr = rho * c_A * gamma(d + 2, ul) * (nxq[:, None] ** 2 + ncq[None, :] ** 2)
    # band: accumulation + rounding of d^ plus a relative slack for the fp32
    # evaluation of the threshold on the GPU
    band = kacc * np.outer(nxq, ncq) + 4.0 * u32 * (p[:, None] + q[None, :]) + 1e-5 * np.abs(thr)
    sure = dref + band <= thr
    maybe = np.abs(dref - thr) < band
    return sure, maybe
