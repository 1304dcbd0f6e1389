"""ctypes binding of libsaq.so (include/saq.h).  Argument marshalling only:
every step of the hot path runs in the library's CUDA kernels.  PyTorch
supplies device memory and the current CUDA stream.

The binding fails loudly if the compiled library is missing; there is no CPU
path.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsaq.so")

SAQ_PREC_FP32 = 0
SAQ_PREC_BF16 = 1
SAQ_PREC_FP8 = 2
SAQ_PREC_FP32_SIMT = 3
PRECISIONS = {"fp32": SAQ_PREC_FP32, "bf16": SAQ_PREC_BF16, "fp8": SAQ_PREC_FP8,
              "fp32_simt": SAQ_PREC_FP32_SIMT}

# every symbol include/saq.h declares
EXPORTS = [
    "saq_params_init", "saq_fit", "saq_model_create", "saq_model_free", "saq_code_bytes",
    "saq_factor_count", "saq_model_dim", "saq_model_kept_dim", "saq_model_num_segments",
    "saq_model_get_plan", "saq_model_get_mean", "saq_model_get_matrix",
    "saq_model_get_variances", "saq_model_set_precision", "saq_model_set_rounds",
    "saq_encode", "saq_encode_host", "saq_project", "saq_quantize_projected",
    "saq_estimate_dist", "saq_model_export", "saq_model_import", "saq_last_error",
    "saq_status_string", "saq_plan_search", "saq_kernel_launch_count",
    "saq_encode_noalloc", "saq_model_uses_tensor_cores", "saq_check_device",
    "saq_ingest_open", "saq_ingest_submit", "saq_ingest_poll", "saq_ingest_wait",
    "saq_ingest_get_stats", "saq_ingest_close", "saq_project_ex", "saq_quantize_projected_ex",
    "saq_kernel_timing", "saq_kernel_times", "saq_estimate_staged", "saq_model_set_basis",
    "saq_model_has_basis", "saq_quantize_step_ceiling", "saq_set_wait_limit",
]


class saq_ingest_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch_rows", ctypes.c_int32),
                ("slots", ctypes.c_int32)]


class saq_ingest_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rows_completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("max_latency_s", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("mixed_batches", ctypes.c_uint64), ("deferred_batches", ctypes.c_uint64),
                ("peak_bytes_in_flight", ctypes.c_size_t)]


class saq_params(ctypes.Structure):
    _fields_ = [("avg_bits", ctypes.c_double), ("max_bits", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("seg_granularity", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tie_frac", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class saq_segment(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int32), ("len", ctypes.c_int32), ("bits", ctypes.c_int32)]


class SaqError(RuntimeError):
    pass


_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsaq.so is not built (%s); run __graft_entry__.build() or "
                          "python paper_2509_12086_gb300/build.py" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    mp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "saq_params_init": (None, [ctypes.POINTER(saq_params)]),
        "saq_fit": (st, [vp, i64, i32, ctypes.POINTER(saq_params), ctypes.POINTER(mp), vp]),
        "saq_model_create": (st, [i32, dp, dp, ctypes.POINTER(saq_segment), i32, dp,
                                  ctypes.POINTER(saq_params), ctypes.POINTER(mp)]),
        "saq_model_free": (None, [mp]),
        "saq_code_bytes": (ctypes.c_size_t, [mp]),
        "saq_factor_count": (i32, [mp]),
        "saq_model_dim": (i32, [mp]),
        "saq_model_kept_dim": (i32, [mp]),
        "saq_model_num_segments": (i32, [mp]),
        "saq_model_get_plan": (st, [mp, ctypes.POINTER(saq_segment), i32]),
        "saq_model_get_mean": (st, [mp, dp]),
        "saq_model_get_matrix": (st, [mp, dp]),
        "saq_model_get_variances": (st, [mp, dp]),
        "saq_model_set_precision": (st, [mp, i32]),
        "saq_model_set_rounds": (st, [mp, i32]),
        "saq_encode": (st, [mp, vp, i64, vp, vp, vp]),
        "saq_encode_host": (st, [mp, vp, i64, vp, vp, vp]),
        "saq_project": (st, [mp, vp, i64, vp, vp, vp]),
        "saq_quantize_projected": (st, [mp, vp, vp, i64, vp, vp, vp]),
        "saq_estimate_dist": (st, [mp, vp, vp, i64, vp, i64, i32, vp, vp]),
        "saq_model_export": (st, [mp, vp, ctypes.POINTER(ctypes.c_size_t)]),
        "saq_model_import": (st, [vp, ctypes.c_size_t, ctypes.POINTER(mp)]),
        "saq_last_error": (ctypes.c_char_p, []),
        "saq_status_string": (ctypes.c_char_p, [st]),
        "saq_kernel_launch_count": (ctypes.c_uint64, []),
        "saq_kernel_timing": (st, [ctypes.c_int]),
        "saq_quantize_step_ceiling": (st, [i32, i32, ctypes.POINTER(ctypes.c_double)]),
        "saq_set_wait_limit": (st, [ctypes.c_uint64]),
        "saq_estimate_staged": (st, [mp, vp, vp, i64, vp, i64, ctypes.c_float, vp, vp]),
        "saq_model_set_basis": (st, [mp, ctypes.POINTER(ctypes.c_double)]),
        "saq_model_has_basis": (ctypes.c_int32, [mp]),
        "saq_kernel_times": (st, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.c_int]),
        "saq_encode_noalloc": (st, [mp, vp, i64, vp, vp, vp]),
        "saq_model_uses_tensor_cores": (i32, [mp]),
        "saq_check_device": (st, [mp, vp]),
        "saq_ingest_open": (st, [ctypes.POINTER(mp), i32, ctypes.POINTER(saq_ingest_params),
                                 ctypes.POINTER(vp)]),
        "saq_ingest_submit": (st, [vp, i32, vp, i64, vp, vp, ctypes.POINTER(ctypes.c_uint64)]),
        "saq_ingest_poll": (st, [vp, ctypes.c_uint64, ctypes.POINTER(i32)]),
        "saq_ingest_wait": (st, [vp, ctypes.c_uint64, i32, ctypes.POINTER(ctypes.c_double)]),
        "saq_ingest_get_stats": (st, [vp, ctypes.POINTER(saq_ingest_stats)]),
        "saq_ingest_close": (st, [vp]),
        "saq_project_ex": (st, [mp, vp, i64, vp, vp, i32, vp]),
        "saq_quantize_projected_ex": (st, [mp, vp, vp, i64, vp, vp, i32, vp]),
        "saq_plan_search": (st, [dp, i32, i32, i64, i32, ctypes.c_double,
                                 ctypes.POINTER(saq_segment), i32, ctypes.POINTER(i32), dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        lib = load()
        raise SaqError("%s: %s" % (lib.saq_status_string(rc).decode(),
                                   lib.saq_last_error().decode()))


def _dptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def params(avg_bits=4.0, max_bits=8, rounds=6, seg_granularity=64, precision="fp32",
           tie_frac=1e-3, seed=4) -> saq_params:
    p = saq_params()
    load().saq_params_init(ctypes.byref(p))
    p.avg_bits = avg_bits
    p.max_bits = max_bits
    p.rounds = rounds
    p.seg_granularity = seg_granularity
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.tie_frac = tie_frac
    p.seed = seed
    return p


class Model:
    """Owner of a saq_model handle."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        lib = load()
        self.d = lib.saq_model_dim(handle)
        self.d_kept = lib.saq_model_kept_dim(handle)
        self.code_bytes = int(lib.saq_code_bytes(handle))
        self.factor_count = lib.saq_factor_count(handle)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().saq_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries
    @property
    def plan(self) -> List[Tuple[int, int, int]]:
        lib = load()
        k = lib.saq_model_num_segments(self._h)
        arr = (saq_segment * k)()
        _check(lib.saq_model_get_plan(self._h, arr, k))
        return [(s.start, s.len, s.bits) for s in arr]

    @property
    def mean(self) -> np.ndarray:
        out = np.zeros(self.d)
        _check(load().saq_model_get_mean(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    @property
    def matrix(self) -> np.ndarray:
        out = np.zeros((self.d_kept, self.d))
        _check(load().saq_model_get_matrix(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    @property
    def variances(self) -> np.ndarray:
        out = np.zeros(self.d)
        _check(load().saq_model_get_variances(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    @property
    def tensor_cores(self) -> bool:
        return bool(load().saq_model_uses_tensor_cores(self._h))

    def check_device(self, stream=None):
        """Synchronise and raise if a bounded device wait gave up."""
        _check(load().saq_check_device(self._h, _stream(stream)))

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(load().saq_model_set_precision(self._h, p))

    def set_rounds(self, rounds: int):
        _check(load().saq_model_set_rounds(self._h, int(rounds)))

    # ---- hot path
    def alloc_outputs(self, n: int, device="cuda"):
        codes = torch.empty((n, max(self.code_bytes, 1)), dtype=torch.uint8, device=device)
        factors = torch.empty((n, self.factor_count), dtype=torch.float32, device=device)
        return codes, factors

    def encode(self, X: torch.Tensor, codes=None, factors=None, stream=None):
        assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
        n = X.shape[0]
        if codes is None:
            codes, factors = self.alloc_outputs(n, X.device)
        _check(load().saq_encode(self._h, _dptr(X), n, _dptr(codes), _dptr(factors), _stream(stream)))
        return codes[:, :self.code_bytes], factors

    def encode_host(self, X: torch.Tensor, codes=None, factors=None, stream=None):
        assert (not X.is_cuda) and X.dtype == torch.float32 and X.is_contiguous()
        n = X.shape[0]
        if codes is None:
            codes = torch.empty((n, max(self.code_bytes, 1)), dtype=torch.uint8).pin_memory()
            factors = torch.empty((n, self.factor_count), dtype=torch.float32).pin_memory()
        _check(load().saq_encode_host(self._h, ctypes.c_void_p(X.data_ptr()), n,
                                      ctypes.c_void_p(codes.data_ptr()),
                                      ctypes.c_void_p(factors.data_ptr()), _stream(stream)))
        return codes[:, :self.code_bytes], factors

    def project(self, X: torch.Tensor, stream=None):
        n = X.shape[0]
        O = torch.empty((n, max(self.d_kept, 1)), dtype=torch.float32, device=X.device)
        nrm = torch.empty((n,), dtype=torch.float32, device=X.device)
        _check(load().saq_project(self._h, _dptr(X), n, _dptr(O), _dptr(nrm), _stream(stream)))
        return O[:, :self.d_kept], nrm

    def quantize_projected(self, O: torch.Tensor, norms2: torch.Tensor, stream=None):
        assert O.is_contiguous() and O.shape[1] == self.d_kept
        n = O.shape[0]
        codes, factors = self.alloc_outputs(n, O.device)
        _check(load().saq_quantize_projected(self._h, _dptr(O), _dptr(norms2), n, _dptr(codes),
                                             _dptr(factors), _stream(stream)))
        return codes[:, :self.code_bytes], factors

    def project_interleaved(self, X: torch.Tensor, stream=None):
        """Projection into the encode's internal layout (groups of 32 rows)."""
        n = X.shape[0]
        O = torch.empty(((n + 31) // 32 * 32 * max(self.d_kept, 1),), dtype=torch.float32,
                        device=X.device)
        nrm = torch.empty((n,), dtype=torch.float32, device=X.device)
        _check(load().saq_project_ex(self._h, _dptr(X), n, _dptr(O), _dptr(nrm), 1,
                                     _stream(stream)))
        return O, nrm

    def quantize_interleaved(self, Oi: torch.Tensor, norms2: torch.Tensor, codes=None,
                             factors=None, stream=None):
        n = norms2.shape[0]
        if codes is None:
            codes, factors = self.alloc_outputs(n, Oi.device)
        _check(load().saq_quantize_projected_ex(self._h, _dptr(Oi), _dptr(norms2), n,
                                                _dptr(codes), _dptr(factors), 1, _stream(stream)))
        return codes[:, :self.code_bytes], factors

    def estimate_dist(self, codes: torch.Tensor, factors: torch.Tensor, Q: torch.Tensor,
                      prefix_bits: int = 0, stream=None):
        n, nq = factors.shape[0], Q.shape[0]
        if codes.shape[1] != self.code_bytes or not codes.is_contiguous():
            full = torch.zeros((n, max(self.code_bytes, 1)), dtype=torch.uint8, device=codes.device)
            full[:, :self.code_bytes] = codes
            codes = full
        dist = torch.empty((nq, n), dtype=torch.float32, device=Q.device)
        _check(load().saq_estimate_dist(self._h, _dptr(codes), _dptr(factors.contiguous()), n,
                                        _dptr(Q.contiguous()), nq, int(prefix_bits), _dptr(dist),
                                        _stream(stream)))
        return dist

    def estimate_staged(self, codes: torch.Tensor, factors: torch.Tensor, Q: torch.Tensor,
                        m_conf: float = 2.0, stream=None) -> torch.Tensor:
        """Sec. 4.3 multi-stage lower bounds, (nq, n, kept segments + 1)."""
        n, nq = factors.shape[0], Q.shape[0]
        if codes.shape[1] != self.code_bytes or not codes.is_contiguous():
            full = torch.zeros((n, max(self.code_bytes, 1)), dtype=torch.uint8, device=codes.device)
            full[:, :self.code_bytes] = codes
            codes = full
        k = self.factor_count // 2
        out = torch.empty((nq, n, k + 1), dtype=torch.float32, device=Q.device)
        _check(load().saq_estimate_staged(self._h, _dptr(codes), _dptr(factors.contiguous()), n,
                                          _dptr(Q.contiguous()), nq, float(m_conf), _dptr(out),
                                          _stream(stream)))
        return out

    def set_basis(self, Vt) -> None:
        Vt = _f64(Vt)
        _check(load().saq_model_set_basis(self._h, Vt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    @property
    def has_basis(self) -> bool:
        return bool(load().saq_model_has_basis(self._h))

    def export(self) -> bytes:
        lib = load()
        ln = ctypes.c_size_t(0)
        _check(lib.saq_model_export(self._h, None, ctypes.byref(ln)))
        buf = ctypes.create_string_buffer(ln.value)
        _check(lib.saq_model_export(self._h, buf, ctypes.byref(ln)))
        return buf.raw[:ln.value]


def saq_fit(X: torch.Tensor, avg_bits=4.0, max_bits=8, rounds=6, seg_granularity=64,
            precision="fp32", tie_frac=1e-3, seed=4, stream=None) -> Model:
    assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
    p = params(avg_bits, max_bits, rounds, seg_granularity, precision, tie_frac, seed)
    h = ctypes.c_void_p()
    _check(load().saq_fit(_dptr(X), X.shape[0], X.shape[1], ctypes.byref(p), ctypes.byref(h),
                          _stream(stream)))
    return Model(h)


def saq_model_create(d: int, mean, W, plan: Sequence[Tuple[int, int, int]], sig2=None,
                     rounds=6, precision="fp32", basis=None) -> Model:
    mean = _f64(mean)
    W = _f64(W) if W is not None else np.zeros((0, d))
    segs = (saq_segment * len(plan))(*[saq_segment(int(s), int(l), int(b)) for s, l, b in plan])
    s2 = _f64(sig2) if sig2 is not None else None
    p = params(rounds=rounds, precision=precision)
    h = ctypes.c_void_p()
    pd = ctypes.POINTER(ctypes.c_double)
    _check(load().saq_model_create(d, mean.ctypes.data_as(pd), W.ctypes.data_as(pd), segs,
                                   len(plan), s2.ctypes.data_as(pd) if s2 is not None else None,
                                   ctypes.byref(p), ctypes.byref(h)))
    m = Model(h)
    if basis is not None:
        m.set_basis(basis)
    return m


def saq_plan_search(sig2, quota_bits: int, g: int = 64, max_bits: int = 8,
                    tie_frac: float = 1e-3):
    """Library's plan search (host only); returns (segments, error)."""
    s2 = _f64(sig2)
    d = s2.shape[0]
    cap = (d + g - 1) // g
    out = (saq_segment * cap)()
    ns = ctypes.c_int32()
    err = ctypes.c_double()
    _check(load().saq_plan_search(s2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), d, g,
                                  int(quota_bits), max_bits, tie_frac, out, cap,
                                  ctypes.byref(ns), ctypes.byref(err)))
    return [(out[i].start, out[i].len, out[i].bits) for i in range(ns.value)], err.value


def saq_kernel_launch_count() -> int:
    return int(load().saq_kernel_launch_count())


KERNEL_KINDS = ("projection", "quantize_adjust_pack", "other")


def saq_quantize_step_ceiling(warps_per_sm: int = 32, bits: int = 4) -> float:
    """Lane-steps per second of the adjustment step on register-resident data
    (the quantize kernel's instruction ceiling at that occupancy)."""
    out = ctypes.c_double(0.0)
    _check(load().saq_quantize_step_ceiling(int(warps_per_sm), int(bits), ctypes.byref(out)))
    return float(out.value)


def saq_set_wait_limit(ns: int) -> None:
    """Bound (ns) of the projection's pipeline waits for later launches; 0
    restores the default (2 s)."""
    _check(load().saq_set_wait_limit(int(ns)))


def saq_kernel_timing(enable: bool) -> None:
    """Start (clearing the record) or stop (keeping it) per-launch device
    timing."""
    _check(load().saq_kernel_timing(1 if enable else 0))


def saq_kernel_times() -> dict:
    """{kind: (summed ms, launches)} of the launches recorded since timing
    was enabled."""
    ms = (ctypes.c_double * 3)()
    ln = (ctypes.c_int64 * 3)()
    _check(load().saq_kernel_times(ms, ln, 3))
    return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(KERNEL_KINDS)}


def saq_model_import(blob: bytes) -> Model:
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().saq_model_import(buf, len(blob), ctypes.byref(h)))
    return Model(h)


def saq_encode(model: Model, X, codes=None, factors=None, stream=None):
    return model.encode(X, codes, factors, stream)


def saq_estimate_dist(model: Model, codes, factors, Q, prefix_bits=0, stream=None):
    return model.estimate_dist(codes, factors, Q, prefix_bits, stream)


class Ingest:
    """Continuous-batching ingest service over resident collections
    (saq_ingest_* in include/saq.h).  Host buffers passed to submit must stay
    alive until the request completes; this wrapper keeps references."""

    def __init__(self, models: Sequence[Model], hbm_budget_bytes: int, max_batch_rows: int = 65536,
                 slots: int = 4):
        self._models = list(models)
        arr = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
        p = saq_ingest_params(hbm_budget_bytes, max_batch_rows, slots)
        h = ctypes.c_void_p()
        _check(load().saq_ingest_open(arr, len(models), ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, collection: int, X: torch.Tensor, codes: torch.Tensor = None,
               factors: torch.Tensor = None) -> int:
        assert (not X.is_cuda) and X.dtype == torch.float32 and X.is_contiguous()
        n = X.shape[0]
        # an out-of-range collection is rejected by the library itself
        m = self._models[collection] if 0 <= collection < len(self._models) else None
        cb = m.code_bytes if m is not None else 1
        if codes is None:
            # page-locked outputs when the rows are: copies to pageable memory
            # are synchronous and would serialise the service's batches
            pin = X.is_pinned()
            codes = torch.empty((n, max(cb, 1)), dtype=torch.uint8, pin_memory=pin)
            factors = torch.empty((n, m.factor_count if m is not None else 1), dtype=torch.float32,
                                  pin_memory=pin)
        t = ctypes.c_uint64()
        _check(load().saq_ingest_submit(self._h, collection, ctypes.c_void_p(X.data_ptr()), n,
                                        ctypes.c_void_p(codes.data_ptr()),
                                        ctypes.c_void_p(factors.data_ptr()), ctypes.byref(t)))
        self._keep[t.value] = (X, codes, factors, cb)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        lat = ctypes.c_double()
        _check(load().saq_ingest_wait(self._h, ticket, timeout_ms, ctypes.byref(lat)))
        X, codes, factors, cb = self._keep.pop(ticket)
        return codes[:, :cb], factors, lat.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        _check(load().saq_ingest_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def stats(self) -> dict:
        s = saq_ingest_stats()
        _check(load().saq_ingest_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in saq_ingest_stats._fields_}

    def close(self):
        if self._h:
            _check(load().saq_ingest_close(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
