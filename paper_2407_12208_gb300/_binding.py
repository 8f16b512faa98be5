"""ctypes binding of libmpkm (include/mpkm.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch
provides device memory (tensors whose data_ptr() is passed) and streams.
There is no fallback: if the library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpkm.so")

KM_OK, KM_EINVAL, KM_ENOMEM, KM_ECUDA, KM_ETIMEOUT, KM_ENOTREADY, KM_ECANCELLED, KM_EUNSUPPORTED = range(8)
STATUS_NAMES = ["KM_OK", "KM_EINVAL", "KM_ENOMEM", "KM_ECUDA", "KM_ETIMEOUT", "KM_ENOTREADY",
                "KM_ECANCELLED", "KM_EUNSUPPORTED"]
FP64_DIRECT, FP32_DIRECT, FP16, BF16, E4M3, FP32 = range(6)
TEST_TC, TEST_PAPER, TEST_OFF = range(3)
EMPTY_KEEP, EMPTY_FARTHEST = range(2)
FB_FP64, FB_FP32, FB_LOW = range(3)
LOW_NAMES = {"fp64": FP64_DIRECT, "fp32": FP32_DIRECT, "fp16": FP16, "bf16": BF16, "e4m3": E4M3,
             "fp32x": FP32}  # fp32x: Alg. 2 with binary32 as the low precision (km_distances)
FALLBACK_NAMES = {"fp64": FB_FP64, "fp32": FB_FP32, "low": FB_LOW}
TEST_NAMES = {"tc": TEST_TC, "paper": TEST_PAPER, "off": TEST_OFF}

# Symbols declared in include/mpkm.h
EXPORTS = ["km_default_params", "km_init", "km_destroy", "km_last_error", "km_workspace_size",
           "km_distances", "km_assign", "km_update_centroids", "km_lloyd_run", "km_get_stats",
           "km_submit", "km_poll", "km_release", "km_cancel", "km_set_profiling", "km_get_phase_times",
           "km_get_launch_count", "km_assign_static", "km_lloyd_step", "km_host_workspace_size",
           "km_lloyd_step_host", "km_selftest_timeout", "km_quantize", "km_choose_low", "km_absmax",
           "km_update_partial", "km_update_finalize", "km_farthest_rows", "km_autotune",
           "km_set_screen_variant", "km_seed_pp", "km_lloyd_run_batch"]
SCREEN_VARIANTS = {"auto": -1, "full": 0, "half": 1, "c32": 2, "reg": 3}  # KM_SV_* of the C-ABI
STATIC_MAX_ROWS = 1048576  # KM_STATIC_MAX_ROWS of the C-ABI
PHASES = ["quantise", "screen", "refine", "fullrow", "update", "direct"]


class KmError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))


class Params(ctypes.Structure):
    _fields_ = [("low", ctypes.c_int32), ("test", ctypes.c_int32), ("rho", ctypes.c_double),
                ("paper_factor", ctypes.c_double), ("max_iter", ctypes.c_int32), ("empty", ctypes.c_int32),
                ("tau", ctypes.c_double), ("fallback", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("flagged", ctypes.c_uint64), ("fp32_evals", ctypes.c_uint64),
                ("fp64_evals", ctypes.c_uint64), ("ambiguous_rows", ctypes.c_uint64),
                ("overflow_rows", ctypes.c_uint64), ("sse", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


JOB_DEVICE_DATA = 1


class BatchJob(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32),
                ("C_init", ctypes.c_void_p), ("C_out", ctypes.c_void_p), ("labels", ctypes.c_void_p),
                ("sse_per_iter", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("scratch", ctypes.c_void_p)]


class Job(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32),
                ("C_init", ctypes.c_void_p), ("p", Params), ("kind", ctypes.c_int32), ("flags", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("sse", ctypes.c_double),
                ("eta", ctypes.c_double), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("C", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("message", ctypes.c_char_p)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads libmpkm.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libmpkm.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        c = ctypes
        vp, i64, i32, sz = c.c_void_p, c.c_int64, c.c_int, c.c_size_t
        P = c.POINTER(Params)
        lib.km_default_params.argtypes = [P]
        lib.km_default_params.restype = None
        lib.km_init.argtypes = [c.POINTER(vp), i32, vp, sz]
        lib.km_destroy.argtypes = [vp]
        lib.km_last_error.argtypes = [vp]
        lib.km_last_error.restype = c.c_char_p
        lib.km_workspace_size.argtypes = [vp, i64, i32, i32, P, c.POINTER(sz)]
        lib.km_distances.argtypes = [vp, vp, i64, vp, i32, i32, P, vp, vp, c.POINTER(c.c_uint64), vp, sz, vp]
        lib.km_assign.argtypes = [vp, vp, i64, vp, i32, i32, P, vp, vp, c.POINTER(c.c_uint64), vp, sz, vp]
        lib.km_update_centroids.argtypes = [vp, vp, i64, i32, vp, i32, vp, P, vp, vp, vp, c.POINTER(c.c_double),
                                            vp, sz, vp]
        lib.km_lloyd_run.argtypes = [vp, vp, i64, i32, i32, vp, P, vp, vp, vp, vp, c.POINTER(c.c_int), vp, sz, vp]
        lib.km_get_stats.argtypes = [vp, c.POINTER(Stats)]
        lib.km_submit.argtypes = [vp, c.POINTER(Job), c.POINTER(c.c_uint64)]
        lib.km_poll.argtypes = [vp, c.c_uint64, c.POINTER(Result)]
        lib.km_release.argtypes = [vp, c.c_uint64]
        lib.km_cancel.argtypes = [vp, c.c_uint64]
        lib.km_assign_static.argtypes = [vp, vp, i64, vp, i32, i32, vp, vp, vp]
        lib.km_lloyd_step.argtypes = [vp, vp, i64, i32, i32, vp, P, vp, vp, vp, vp, c.POINTER(c.c_double), vp, sz, vp]
        lib.km_host_workspace_size.argtypes = [vp, i64, i32, i32, P, c.POINTER(sz)]
        lib.km_lloyd_step_host.argtypes = [vp, vp, i64, i32, i32, vp, P, vp, vp, vp, vp, c.POINTER(c.c_double), vp,
                                           sz, vp]
        lib.km_selftest_timeout.argtypes = [vp, vp, sz, vp]
        lib.km_quantize.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, vp]
        lib.km_absmax.argtypes = [vp, vp, i64, c.POINTER(c.c_uint32), vp, sz, vp]
        lib.km_update_partial.argtypes = [vp, vp, i64, i32, vp, i32, c.c_uint32, i64, vp, vp, vp, sz, vp]
        lib.km_update_finalize.argtypes = [vp, vp, vp, i32, i32, c.c_uint32, i64, vp, vp, c.POINTER(c.c_double), vp, sz,
                                           vp]
        lib.km_farthest_rows.argtypes = [vp, vp, i64, i32, vp, vp, vp, sz, vp]
        lib.km_choose_low.argtypes = [vp, vp, i64, vp, i32, i32, c.c_double, c.POINTER(c.c_int32), vp, vp, sz, vp]
        lib.km_autotune.argtypes = [vp, vp, i64, vp, i32, i32, P, vp, c.POINTER(c.c_int32), vp, vp, sz, vp]
        lib.km_set_screen_variant.argtypes = [vp, i64, i32, i32, i32, i32]
        lib.km_seed_pp.argtypes = [vp, vp, i64, i32, i32, c.POINTER(c.c_double), vp, c.POINTER(c.c_int64), vp, sz,
                                   vp]
        lib.km_lloyd_run_batch.argtypes = [vp, c.POINTER(BatchJob), i32, P, vp]
        lib.km_set_profiling.argtypes = [vp, i32]
        lib.km_get_phase_times.argtypes = [vp, vp, vp]
        lib.km_get_launch_count.argtypes = [vp, c.POINTER(c.c_uint64)]
        for f in EXPORTS:
            fn = getattr(lib, f)
            if f not in ("km_default_params", "km_last_error"):
                fn.restype = c.c_int
        _lib = lib
        return lib


def params(low="bf16", test="tc", rho=5.0, paper_factor=2.0, max_iter=20, empty="farthest", tau=0.0,
           fallback="fp64") -> Params:
    p = Params()
    load().km_default_params(ctypes.byref(p))
    p.low = LOW_NAMES[low] if isinstance(low, str) else int(low)
    p.test = TEST_NAMES[test] if isinstance(test, str) else int(test)
    p.rho = float(rho)
    p.paper_factor = float(paper_factor)
    p.max_iter = int(max_iter)
    p.empty = {"keep": EMPTY_KEEP, "farthest": EMPTY_FARTHEST}[empty] if isinstance(empty, str) else int(empty)
    p.tau = float(tau)
    p.fallback = FALLBACK_NAMES[fallback] if isinstance(fallback, str) else int(fallback)
    return p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A libmpkm context on one GPU; optional serving arena (a torch tensor)."""

    def __init__(self, device: int = 0, arena_bytes: int = 0):
        import torch
        self.lib = load()
        self.device = device
        self._arena = None
        h = ctypes.c_void_p()
        arena_ptr, nbytes = None, 0
        if arena_bytes:
            self._arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda:%d" % device)
            arena_ptr, nbytes = ctypes.c_void_p(self._arena.data_ptr()), int(arena_bytes)
        rc = self.lib.km_init(ctypes.byref(h), device, arena_ptr, nbytes)
        if rc != KM_OK:
            raise KmError(rc, "km_init failed")
        self.h = h
        self._ws = None
        self._hws = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.km_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != KM_OK:
            raise KmError(rc, self.lib.km_last_error(self.h).decode())

    def workspace_size(self, n, d, k, p: Params) -> int:
        b = ctypes.c_size_t()
        self._check(self.lib.km_workspace_size(self.h, int(n), int(d), int(k), ctypes.byref(p), ctypes.byref(b)))
        return b.value

    def workspace(self, n, d, k, p: Params):
        """A cached device workspace large enough for (n, d, k, p)."""
        import torch
        need = self.workspace_size(n, d, k, p)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda:%d" % self.device)
        return self._ws

    def assign(self, X, C, p: Params, labels=None, min_dist=None, ws=None, stream=None, want_flagged=True):
        import torch
        n, d = X.shape
        k = C.shape[0]
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=X.device)
        if min_dist is None:
            min_dist = torch.empty(n, dtype=torch.float64, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p)
        nf = ctypes.c_uint64(0)
        self._check(self.lib.km_assign(self.h, _ptr(X), n, _ptr(C), k, d, ctypes.byref(p), _ptr(labels),
                                       _ptr(min_dist), ctypes.byref(nf) if want_flagged else None, _ptr(ws),
                                       ws.numel(), _stream(stream)))
        return labels, min_dist, (nf.value if want_flagged else None)

    def autotune(self, X, C, p: Params, ws=None, stream=None):
        """km_autotune: times the screening kernel's variants on this data and
        keeps the fastest for the shape class.  Returns (variant name, ms per
        call of full / half / c32, -1 where not timed)."""
        import torch
        n, d = X.shape
        k = C.shape[0]
        labels = torch.empty(n, dtype=torch.int32, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p)
        v = ctypes.c_int32(0)
        ms = (ctypes.c_float * 3)()
        self._check(self.lib.km_autotune(self.h, _ptr(X), n, _ptr(C), k, d, ctypes.byref(p), _ptr(labels),
                                         ctypes.byref(v), ms, _ptr(ws), ws.numel(), _stream(stream)))
        names = {val: key for key, val in SCREEN_VARIANTS.items() if val >= 0}  # -1: a direct format
        return names.get(v.value, "none"), [float(m) for m in ms]

    def set_screen_variant(self, n, d, k, low, variant):
        """km_set_screen_variant: pins ("full", "half", "c32") or clears ("auto")
        the screening variant of the shape class."""
        self._check(self.lib.km_set_screen_variant(self.h, n, d, k, LOW_NAMES[low] if isinstance(low, str) else int(low),
                                                   SCREEN_VARIANTS[variant]))

    def lloyd_run_batch(self, jobs, p: Params, stream=None):
        """km_lloyd_run_batch: Alg. 3 for every (X, C_init) pair of device
        tensors in one launch per 32 jobs of equal d.  Returns per job
        (C_out, labels, sse[:iters + 1], iters)."""
        import torch
        arr = (BatchJob * len(jobs))()
        keep = []
        for q, (X, C0) in enumerate(jobs):
            n, d = X.shape
            k = C0.shape[0]
            C = torch.empty_like(C0)
            lab = torch.empty(n, dtype=torch.int32, device=X.device)
            sse = torch.empty(p.max_iter + 1, dtype=torch.float64, device=X.device)
            it = torch.zeros(1, dtype=torch.int32, device=X.device)
            scr = torch.empty(n, dtype=torch.float64, device=X.device)
            arr[q] = BatchJob(_ptr(X), n, d, k, _ptr(C0), _ptr(C), _ptr(lab), _ptr(sse), _ptr(it), _ptr(scr))
            keep.append((C, lab, sse, it, scr))
        self._check(self.lib.km_lloyd_run_batch(self.h, arr, len(jobs), ctypes.byref(p), _stream(stream)))
        out = []
        for C, lab, sse, it, _ in keep:
            t = int(it.item())
            out.append((C, lab, sse[: t + 1].cpu().numpy(), t))
        return out

    def seed_pp(self, X, u, C_out=None, ws=None, stream=None):
        """km_seed_pp: k = len(u) initial centres by D^2 sampling with the
        draws u (in [0, 1)).  Returns (centres k x d on X's device, indices)."""
        import numpy as np
        import torch
        n, d = X.shape
        u = np.ascontiguousarray(u, dtype=np.float64)
        k = len(u)
        if C_out is None:
            C_out = torch.empty((k, d), dtype=torch.float32, device=X.device)
        if ws is None:
            ws = torch.empty(8 * n + 16 * k + 16 * min(n, 16384) + 1280, dtype=torch.uint8, device=X.device)
        idx = np.empty(k, dtype=np.int64)
        self._check(self.lib.km_seed_pp(self.h, _ptr(X), n, d, k, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        _ptr(C_out), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(ws),
                                        ws.numel(), _stream(stream)))
        return C_out, idx

    def quantize(self, X, low="bf16", stream=None):
        """km_quantize: (Xq as raw bytes n x (ldq * element size) uint8,
        stats n x 4 float32, scale n float32)."""
        import torch
        n, d = X.shape
        lowv = LOW_NAMES[low] if isinstance(low, str) else int(low)
        esz = 1 if lowv == E4M3 else 2
        ldq = (d + 15) // 16 * 16 if lowv == E4M3 else (d + 7) // 8 * 8
        Xq = torch.empty((n, ldq * esz), dtype=torch.uint8, device=X.device)
        stats = torch.empty((n, 4), dtype=torch.float32, device=X.device)
        scale = torch.empty(n, dtype=torch.float32, device=X.device)
        self._check(self.lib.km_quantize(self.h, _ptr(X), n, d, lowv, _ptr(Xq), _ptr(stats), _ptr(scale),
                                         _stream(stream)))
        return Xq, stats, scale

    def choose_low(self, X, C, max_overflow_share=0.01, ws=None, stream=None):
        """km_choose_low: (the chosen low format's name, {bf16/e4m3: mean
        candidates per row, predicted overflow share})."""
        import numpy as np
        n, d = X.shape
        k = C.shape[0]
        ws = ws if ws is not None else self.workspace(n, d, k, params("bf16"))
        low = ctypes.c_int32(0)
        st = np.zeros(4, dtype=np.float64)
        self._check(self.lib.km_choose_low(self.h, _ptr(X), n, _ptr(C), k, d, float(max_overflow_share),
                                           ctypes.byref(low), st.ctypes.data_as(ctypes.c_void_p), _ptr(ws), ws.numel(),
                                           _stream(stream)))
        name = {v: kk for kk, v in LOW_NAMES.items()}[low.value]
        return name, {"bf16": (float(st[0]), float(st[1])), "e4m3": (float(st[2]), float(st[3]))}

    # ---- row-sharded updates (the exchange of a data-parallel iteration)
    def absmax(self, X, stream=None) -> int:
        """km_absmax: max |x| of X as its binary32 bit pattern."""
        import torch
        ws = torch.empty(256, dtype=torch.uint8, device=X.device)
        b = ctypes.c_uint32(0)
        self._check(self.lib.km_absmax(self.h, _ptr(X), X.numel(), ctypes.byref(b), _ptr(ws), 256, _stream(stream)))
        return b.value

    def update_partial(self, X, labels, k, absmax_bits, n_total, p: Params = None, ws=None, stream=None):
        """km_update_partial: (sums k x d int64, counts k int64) of this shard."""
        import torch
        n, d = X.shape
        sums = torch.empty((k, d), dtype=torch.int64, device=X.device)
        counts = torch.empty(k, dtype=torch.int64, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p or params("bf16"))
        self._check(self.lib.km_update_partial(self.h, _ptr(X), n, d, _ptr(labels), int(k), ctypes.c_uint32(absmax_bits),
                                               int(n_total), _ptr(sums), _ptr(counts), _ptr(ws), ws.numel(),
                                               _stream(stream)))
        return sums, counts

    def update_finalize(self, sums, counts, C_old, absmax_bits, n_total, ws=None, stream=None):
        """km_update_finalize: (C_new, shift); empty clusters keep C_old's rows."""
        import torch
        k, d = C_old.shape
        C_new = torch.empty_like(C_old)
        ws = ws if ws is not None else self.workspace(1, d, k, params("bf16"))
        sh = ctypes.c_double(0.0)
        self._check(self.lib.km_update_finalize(self.h, _ptr(sums), _ptr(counts), k, d, ctypes.c_uint32(absmax_bits),
                                                int(n_total), _ptr(C_old), _ptr(C_new), ctypes.byref(sh), _ptr(ws),
                                                ws.numel(), _stream(stream)))
        return C_new, sh.value

    def farthest_rows(self, min_dist, e, k=None, ws=None, stream=None):
        """km_farthest_rows: (rows int64, min_dist values) of the e rows of
        largest min_dist, ties to the lowest index."""
        import torch
        n = min_dist.numel()
        rows = torch.empty(e, dtype=torch.int64, device=min_dist.device)
        vals = torch.empty(e, dtype=torch.float64, device=min_dist.device)
        ws = ws if ws is not None else self.workspace(n, 1, max(e, k or e), params("fp32"))
        self._check(self.lib.km_farthest_rows(self.h, _ptr(min_dist), n, int(e), _ptr(rows), _ptr(vals), _ptr(ws),
                                              ws.numel(), _stream(stream)))
        return rows, vals

    def assign_static(self, X, C, labels, min_dist, stream=None):
        """km_assign_static: the fp32 direct assignment with the library's
        static scratch (no workspace; the caller provides both outputs)."""
        n, d = X.shape
        k = C.shape[0]
        self._check(self.lib.km_assign_static(self.h, _ptr(X), n, _ptr(C), k, d, _ptr(labels), _ptr(min_dist),
                                              _stream(stream)))
        return labels, min_dist

    def distances(self, X, C, p: Params, D=None, flag_bits=None, ws=None, stream=None):
        import torch
        n, d = X.shape
        k = C.shape[0]
        if D is None:
            D = torch.empty((n, k), dtype=torch.float32, device=X.device)
        if flag_bits is None:
            flag_bits = torch.empty((n * k + 31) // 32, dtype=torch.int32, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p)
        nf = ctypes.c_uint64(0)
        self._check(self.lib.km_distances(self.h, _ptr(X), n, _ptr(C), k, d, ctypes.byref(p), _ptr(D),
                                          _ptr(flag_bits), ctypes.byref(nf), _ptr(ws), ws.numel(),
                                          _stream(stream)))
        return D, flag_bits, nf.value

    def lloyd_step(self, X, C_old, p: Params, labels=None, min_dist=None, C_new=None, counts=None, ws=None,
                   stream=None, want_shift=True):
        """km_lloyd_step: one assignment + centre update (Alg. 3's loop body)."""
        import torch
        n, d = X.shape
        k = C_old.shape[0]
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=X.device)
        if min_dist is None:
            min_dist = torch.empty(n, dtype=torch.float64, device=X.device)
        if C_new is None:
            C_new = torch.empty_like(C_old)
        if counts is None:
            counts = torch.empty(k, dtype=torch.int64, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p)
        sh = ctypes.c_double(0.0)
        self._check(self.lib.km_lloyd_step(self.h, _ptr(X), n, d, k, _ptr(C_old), ctypes.byref(p), _ptr(labels),
                                           _ptr(min_dist), _ptr(C_new), _ptr(counts),
                                           ctypes.byref(sh) if want_shift else None, _ptr(ws), ws.numel(),
                                           _stream(stream)))
        return labels, min_dist, C_new, counts, (sh.value if want_shift else None)

    def host_workspace(self, n, d, k, p: Params):
        """A cached device workspace for km_lloyd_step_host."""
        import torch
        b = ctypes.c_size_t()
        self._check(self.lib.km_host_workspace_size(self.h, int(n), int(d), int(k), ctypes.byref(p), ctypes.byref(b)))
        if self._hws is None or self._hws.numel() < b.value:
            self._hws = torch.empty(b.value, dtype=torch.uint8, device="cuda:%d" % self.device)
        return self._hws

    def lloyd_step_host(self, X, C_old, p: Params, labels=None, min_dist=None, C_new=None, counts=None, ws=None,
                        stream=None, want_shift=True):
        """km_lloyd_step_host: X, C_old and the outputs are CPU tensors (pin
        them for overlapped copies); returns when the outputs are written."""
        import torch
        assert X.device.type == "cpu" and C_old.device.type == "cpu"
        X = X.contiguous()
        C_old = C_old.contiguous()
        n, d = X.shape
        k = C_old.shape[0]
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32).pin_memory()
        if C_new is None:
            C_new = torch.empty((k, d), dtype=torch.float32).pin_memory()
        ws = ws if ws is not None else self.host_workspace(n, d, k, p)
        sh = ctypes.c_double(0.0)
        self._check(self.lib.km_lloyd_step_host(self.h, _ptr(X), n, d, k, _ptr(C_old), ctypes.byref(p), _ptr(labels),
                                                _ptr(min_dist), _ptr(C_new), _ptr(counts),
                                                ctypes.byref(sh) if want_shift else None, _ptr(ws), ws.numel(),
                                                _stream(stream)))
        return labels, min_dist, C_new, counts, (sh.value if want_shift else None)

    def update_centroids(self, X, labels, C_old, p: Params, min_dist=None, C_new=None, counts=None, ws=None,
                         stream=None, want_shift=True):
        import torch
        n, d = X.shape
        k = C_old.shape[0]
        if C_new is None:
            C_new = torch.empty_like(C_old)
        if counts is None:
            counts = torch.empty(k, dtype=torch.int64, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p)
        sh = ctypes.c_double(0.0)
        self._check(self.lib.km_update_centroids(self.h, _ptr(X), n, d, _ptr(labels), k, _ptr(C_old),
                                                 ctypes.byref(p), _ptr(min_dist), _ptr(C_new), _ptr(counts),
                                                 ctypes.byref(sh) if want_shift else None, _ptr(ws), ws.numel(),
                                                 _stream(stream)))
        return C_new, counts, (sh.value if want_shift else None)

    def lloyd_run(self, X, C_init, p: Params, C_out=None, labels=None, ws=None, stream=None):
        import numpy as np
        import torch
        n, d = X.shape
        k = C_init.shape[0]
        if C_out is None:
            C_out = torch.empty_like(C_init)
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=X.device)
        ws = ws if ws is not None else self.workspace(n, d, k, p)
        sse = np.zeros(p.max_iter + 1, dtype=np.float64)
        eta = np.zeros(p.max_iter + 1, dtype=np.float64)
        it = ctypes.c_int(0)
        self._check(self.lib.km_lloyd_run(self.h, _ptr(X), n, d, k, _ptr(C_init), ctypes.byref(p), _ptr(C_out),
                                          _ptr(labels), sse.ctypes.data_as(ctypes.c_void_p),
                                          eta.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it), _ptr(ws),
                                          ws.numel(), _stream(stream)))
        t = it.value
        return C_out, labels, sse[: t + 1], eta[: t + 1], t

    def selftest_timeout(self, stream=None) -> int:
        """km_selftest_timeout: the status of a bounded wait that runs out
        (KM_ETIMEOUT expected); raises nothing."""
        import torch
        ws = torch.empty(4096, dtype=torch.uint8, device="cuda:%d" % self.device)
        return int(self.lib.km_selftest_timeout(self.h, _ptr(ws), ws.numel(), _stream(stream)))

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.km_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def set_profiling(self, on: bool = True):
        self._check(self.lib.km_set_profiling(self.h, int(bool(on))))

    def phase_times(self):
        """{phase: (total ms, count)} since the previous read (synchronises)."""
        import numpy as np
        ms = np.zeros(len(PHASES), dtype=np.float64)
        cnt = np.zeros(len(PHASES), dtype=np.int64)
        self._check(self.lib.km_get_phase_times(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                                cnt.ctypes.data_as(ctypes.c_void_p)))
        return {ph: (float(ms[i]), int(cnt[i])) for i, ph in enumerate(PHASES)}

    def launch_count(self) -> int:
        v = ctypes.c_uint64(0)
        self._check(self.lib.km_get_launch_count(self.h, ctypes.byref(v)))
        return v.value

    # ---- serving
    def submit(self, X, C_init, p: Params, kind: int = 0) -> int:
        """X, C_init: C-contiguous float32 numpy arrays (host; copied before
        return) or CUDA tensors (resident: read in place, they must stay
        alive and unchanged until the job has finished)."""
        import numpy as np
        j = Job()
        if hasattr(X, "is_cuda") and X.is_cuda:
            assert X.is_contiguous() and C_init.is_contiguous() and C_init.is_cuda
            j.X, j.C_init = ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(C_init.data_ptr())
            j.n, j.d = X.shape
            j.k = C_init.shape[0]
            j.flags = JOB_DEVICE_DATA
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
            C = np.ascontiguousarray(C_init, dtype=np.float32)
            j.X = X.ctypes.data_as(ctypes.c_void_p)
            j.n, j.d = X.shape
            j.k = C.shape[0]
            j.C_init = C.ctypes.data_as(ctypes.c_void_p)
            j.flags = 0
        j.p = p
        j.kind = int(kind)
        jid = ctypes.c_uint64(0)
        self._check(self.lib.km_submit(self.h, ctypes.byref(j), ctypes.byref(jid)))
        return jid.value

    def poll(self, job_id: int):
        """None while running; else a dict (C / labels as device pointers)."""
        r = Result()
        rc = self.lib.km_poll(self.h, ctypes.c_uint64(job_id), ctypes.byref(r))
        if rc == KM_ENOTREADY:
            return None
        return {"status": rc, "iters": r.iters, "sse": r.sse, "eta": r.eta, "latency_ms": r.latency_ms,
                "queue_ms": r.queue_ms, "C": r.C, "labels": r.labels,
                "message": (r.message or b"").decode()}

    def release(self, job_id: int):
        self._check(self.lib.km_release(self.h, ctypes.c_uint64(job_id)))

    def cancel(self, job_id: int):
        self._check(self.lib.km_cancel(self.h, ctypes.c_uint64(job_id)))


def device_array(ptr: int, shape, dtype_str: str, device: int = 0):
    """A torch tensor viewing library-owned device memory (serving results)."""
    import torch

    class _CAI:
        def __init__(self):
            self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": dtype_str, "data": (ptr, False),
                                             "version": 3, "strides": None}

    return torch.as_tensor(_CAI(), device="cuda:%d" % device)
