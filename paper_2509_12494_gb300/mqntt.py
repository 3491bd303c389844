"""Thin Python binding of the C ABI in include/mqntt.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but convert
arguments: Python ints become two-word arrays, torch tensors become device pointers, a torch
stream (or None for the current stream) becomes a cudaStream_t.  All arithmetic runs in the CUDA
library ``libmqntt.so``; there is no fallback.  A non-zero status raises ``MqError`` carrying the
library's message.

Residue tensors are int64 tensors on the GPU holding the residues' bits: shape (..., ) for 64-bit
residues and (..., 2) -- low word first -- for 128-bit residues.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

MQ_OK = 0
MQ_ERR_ARG, MQ_ERR_MODULUS, MQ_ERR_ROOT, MQ_ERR_SIZE, MQ_ERR_ALIGN = -1, -2, -3, -4, -5
MQ_ERR_OOM, MQ_ERR_CUDA, MQ_ERR_TIMEOUT, MQ_ERR_RANGE, MQ_ERR_STATE = -6, -7, -8, -9, -10
MQ_ERR_CANCELLED = -11
MQ_W64, MQ_W128, MQ_W192, MQ_W256 = 1, 2, 3, 4
MQ_NEGACYCLIC, MQ_CYCLIC, MQ_ORDER_NATURAL, MQ_ORDER_BITREV = 0, 1, 0, 2
MQ_CHECK_INPUTS = 0x100   # plan flag, or OR-ed into a BLAS width: range-check the inputs first

_u64x2 = ctypes.c_uint64 * 2
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p
_lib = None


class MqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mqntt error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmqntt.so (compiled by __graft_entry__.build()).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c "
                               "'import __graft_entry__ as g; g.build()')")
        _build.build()
    L = ctypes.CDLL(path)
    sig = {
        "ntt_plan_create": [ctypes.POINTER(_vp), ctypes.c_uint, _u64p, _u64p, ctypes.c_int, ctypes.c_uint, _vp],
        "ntt_plan_destroy": [_vp],
        "ntt_forward": [_vp, _vp, ctypes.c_size_t, ctypes.c_size_t, _vp],
        "ntt_inverse": [_vp, _vp, ctypes.c_size_t, ctypes.c_size_t, _vp],
        "ntt_polymul": [_vp, _vp, _vp, _vp, ctypes.c_size_t, ctypes.c_size_t, _vp],
        "ntt_forward_noalloc": [_vp, _vp, ctypes.c_size_t, ctypes.c_size_t, _vp],
        "ntt_plan_info": [_vp, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint)],
        "mod_vadd": [_vp, _vp, _vp, ctypes.c_size_t, _u64p, ctypes.c_int, _vp],
        "mod_vsub": [_vp, _vp, _vp, ctypes.c_size_t, _u64p, ctypes.c_int, _vp],
        "mod_vmul": [_vp, _vp, _vp, ctypes.c_size_t, _u64p, ctypes.c_int, _vp],
        "mod_axpy": [_vp, _u64p, _vp, ctypes.c_size_t, _u64p, ctypes.c_int, _vp],
        "mq_probe_imad_rate": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), _vp],
        "mq_probe_mulmod": [ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _u64x2, _vp],
        "mq_probe_mulmod_rate": [ctypes.c_int, ctypes.c_int, _u64x2, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), _vp],
        "mq_batch_create": [ctypes.POINTER(_vp), _vp, ctypes.c_size_t, _vp, _vp],
        "mq_batch_update": [_vp, _vp, ctypes.c_size_t, _vp],
        "mq_batch_launch": [_vp, _vp],
        "mq_batch_status": [_vp],
        "mq_batch_info": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint),
                          ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
        "mq_batch_destroy": [_vp],
        "mq_autotune_batch": [_vp, ctypes.c_size_t, _vp, ctypes.c_char_p, _vp],
        "mq_server_create": [ctypes.POINTER(_vp), _vp],
        "mq_submit": [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)],
        "mq_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "mq_wait": [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_int)],
        "mq_server_drain": [_vp, ctypes.c_double],
        "mq_server_poisson": [_vp, _vp, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.POINTER(ctypes.c_double)],
        "mq_cancel": [_vp, ctypes.c_uint64],
        "mq_server_inject_alloc_failures": [_vp, ctypes.c_uint],
        "mq_server_stats": [_vp, _vp],
        "mq_server_reset_stats": [_vp],
        "mq_server_destroy": [_vp],
        "mq_last_error": [],
        "mq_version": [],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name in ("mq_last_error", "mq_version") else ctypes.c_int
    _lib = L
    return L


# ---------------------------------------------------------------------------------------- helpers

def words(v: int, width: int = 2) -> "ctypes.Array":
    """v as max(width, 2) 64-bit words, low first (the ABI's modulus / root / scalar arrays)."""
    v = int(v)
    n = max(width & 0xFF, 2)   # a width may carry MQ_CHECK_INPUTS
    if v < 0 or v >= 2 ** (64 * n):
        raise ValueError(f"value must be in [0, 2^{64 * n})")
    return (ctypes.c_uint64 * n)(*[(v >> (64 * k)) & (2**64 - 1) for k in range(n)])


def ptr(x) -> int:
    """Device pointer of a torch tensor, or an int passed through."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def stream_handle(stream=None) -> int:
    """cudaStream_t of a torch stream; None means torch's current stream."""
    if isinstance(stream, int):
        return stream
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(rc: int):
    if rc != MQ_OK:
        raise MqError(rc, (load().mq_last_error() or b"").decode())


def width_of(q: int) -> int:
    return MQ_W64 if q < 2**60 else MQ_W128 if q < 2**124 else MQ_W192 if q < 2**188 else MQ_W256


# ---------------------------------------------------------------------------------------- the ABI

class Plan:
    """Owns an ntt_plan* (freed by ntt_plan_destroy or on garbage collection)."""

    def __init__(self, handle: int, log2n: int, width: int, flags: int):
        self.handle, self.log2n, self.width, self.flags = handle, log2n, width, flags

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ntt_plan_destroy(self.handle)
            self.handle = None


def ntt_plan_create(log2n: int, q: int, root: int, width: int, flags: int = 0, stream=None) -> Plan:
    h = _vp()
    _check(load().ntt_plan_create(ctypes.byref(h), log2n, words(q, width), words(root, width), width, flags,
                                  stream_handle(stream)))
    return Plan(h.value, log2n, width, flags)


def ntt_plan_destroy(plan: Plan):
    if plan.handle:
        _check(load().ntt_plan_destroy(plan.handle))
        plan.handle = None


def ntt_forward(plan: Plan, data, batch: int = 1, stride: int = 0, stream=None):
    _check(load().ntt_forward(plan.handle, ptr(data), batch, stride, stream_handle(stream)))


def ntt_inverse(plan: Plan, data, batch: int = 1, stride: int = 0, stream=None):
    _check(load().ntt_inverse(plan.handle, ptr(data), batch, stride, stream_handle(stream)))


def ntt_polymul(plan: Plan, c, a, b, batch: int = 1, stride: int = 0, stream=None):
    """c = a * b mod (X^N + 1, q) (mod X^N - 1 for a cyclic plan), per polynomial."""
    _check(load().ntt_polymul(plan.handle, ptr(c), ptr(a), ptr(b), batch, stride, stream_handle(stream)))


MQ_NOALLOC_SCRATCH_BYTES = 16 << 20


def ntt_forward_noalloc(plan: Plan, data, batch: int = 1, stride: int = 0, stream=None):
    _check(load().ntt_forward_noalloc(plan.handle, ptr(data), batch, stride, stream_handle(stream)))


def ntt_plan_info(plan: Plan):
    a, b, c = ctypes.c_uint(), ctypes.c_int(), ctypes.c_uint()
    _check(load().ntt_plan_info(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def mod_vadd(c, a, b, n: int, q: int, width: int, stream=None):
    _check(load().mod_vadd(ptr(c), ptr(a), ptr(b), n, words(q, width), width, stream_handle(stream)))


def mod_vsub(c, a, b, n: int, q: int, width: int, stream=None):
    _check(load().mod_vsub(ptr(c), ptr(a), ptr(b), n, words(q, width), width, stream_handle(stream)))


def mod_vmul(c, a, b, n: int, q: int, width: int, stream=None):
    _check(load().mod_vmul(ptr(c), ptr(a), ptr(b), n, words(q, width), width, stream_handle(stream)))


def mod_axpy(y, a: int, x, n: int, q: int, width: int, stream=None):
    _check(load().mod_axpy(ptr(y), words(a, width), ptr(x), n, words(q, width), width, stream_handle(stream)))


MQ_PROBE_MAD_LO, MQ_PROBE_MAD_HI, MQ_PROBE_MAD_CC, MQ_PROBE_MAD_WIDE = 0, 1, 2, 3


def mq_probe_imad_rate(kind: int, iters: int, stream=None):
    """(thread-instructions per second, kernel ms) of the multiply-add probe."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().mq_probe_imad_rate(kind, iters, ctypes.byref(r), ctypes.byref(ms), stream_handle(stream)))
    return r.value, ms.value


MQ_MUL_SCHOOLBOOK, MQ_MUL_KARATSUBA = 0, 1


def mq_probe_mulmod(variant: int, c, a, b, n: int, q: int, stream=None):
    """c = a * b mod q (124-bit residues) with the schoolbook or the Karatsuba double-word product."""
    _check(load().mq_probe_mulmod(variant, ptr(c), ptr(a), ptr(b), n, words(q), stream_handle(stream)))


def mq_probe_mulmod_rate(variant: int, iters: int, q: int, stream=None):
    """(general 124-bit modular products per second, kernel ms) with the chosen product form."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().mq_probe_mulmod_rate(variant, iters, words(q), ctypes.byref(r), ctypes.byref(ms),
                                       stream_handle(stream)))
    return r.value, ms.value


def mq_last_error() -> str:
    return (load().mq_last_error() or b"").decode()


def mq_version() -> str:
    return load().mq_version().decode()


# ------------------------------------------------------------------------- batches (mqntt_batch.h)

MQ_JOB_NTT_FORWARD, MQ_JOB_NTT_INVERSE, MQ_JOB_VADD, MQ_JOB_VSUB, MQ_JOB_VMUL, MQ_JOB_AXPY = 1, 2, 3, 4, 5, 6
MQ_BATCH_NO_GRAPH, MQ_BATCH_TEST_DROP_ITEM = 1, 2
MQ_BATCH_FORM_SPLIT, MQ_BATCH_FORM_PREFETCH, MQ_BATCH_FORM_CALLS = 4, 8, 16


class mq_job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("after", ctypes.c_int), ("plan", _vp), ("data", _vp), ("a", _vp),
                ("b", _vp), ("n", ctypes.c_size_t), ("batch", ctypes.c_size_t), ("stride", ctypes.c_size_t),
                ("q", ctypes.c_uint64 * 2), ("scalar", ctypes.c_uint64 * 2), ("width", ctypes.c_int)]


class mq_batch_opts(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_uint), ("lag", ctypes.c_uint), ("blas_chunk", ctypes.c_uint),
                ("wait_timeout_s", ctypes.c_double), ("flags", ctypes.c_uint), ("split_shift", ctypes.c_int)]


def ntt_job(kind: int, plan: Plan, data, batch: int = 1, stride: int = 0, after: int = -1) -> mq_job:
    j = mq_job()
    j.kind, j.after, j.plan, j.data, j.batch, j.stride = kind, after, plan.handle, ptr(data), batch, stride
    return j


def blas_job(kind: int, data, a, b, n: int, q: int, width: int, scalar: int = 0, after: int = -1) -> mq_job:
    j = mq_job()
    j.kind, j.after, j.data, j.a, j.b, j.n, j.width = kind, after, ptr(data), ptr(a), ptr(b), n, width
    j.q = words(q)
    j.scalar = words(scalar)
    return j


def _job_array(jobs):
    arr = (mq_job * len(jobs))(*jobs)
    return arr


class Batch:
    """Owns an mq_batch* (freed by mq_batch_destroy or on garbage collection)."""

    def __init__(self, handle: int, njobs: int):
        self.handle, self.njobs = handle, njobs

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mq_batch_destroy(self.handle)
            self.handle = None


def mq_batch_create(jobs, opts: mq_batch_opts | None = None, stream=None) -> Batch:
    h = _vp()
    arr = _job_array(jobs)
    _check(load().mq_batch_create(ctypes.byref(h), ctypes.cast(arr, _vp), len(jobs),
                                  ctypes.cast(ctypes.byref(opts), _vp) if opts is not None else None,
                                  stream_handle(stream)))
    return Batch(h.value, len(jobs))


def mq_batch_update(batch: Batch, jobs, stream=None):
    arr = _job_array(jobs)
    _check(load().mq_batch_update(batch.handle, ctypes.cast(arr, _vp), len(jobs), stream_handle(stream)))


def mq_batch_launch(batch: Batch, stream=None):
    _check(load().mq_batch_launch(batch.handle, stream_handle(stream)))


def mq_batch_status(batch: Batch) -> int:
    """Returns the status code (0 or MQ_ERR_TIMEOUT, ...) without raising."""
    return load().mq_batch_status(batch.handle)


def mq_batch_info(batch: Batch):
    a, b, c, d = ctypes.c_size_t(), ctypes.c_uint(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().mq_batch_info(batch.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return {"items": a.value, "ctas": b.value, "ntt_items": c.value, "blas_items": d.value}


def mq_batch_destroy(batch: Batch):
    if batch.handle:
        _check(load().mq_batch_destroy(batch.handle))
        batch.handle = None


def mq_autotune_batch(jobs, cache_path: str | None = None, stream=None) -> mq_batch_opts:
    best = mq_batch_opts()
    arr = _job_array(jobs)
    _check(load().mq_autotune_batch(ctypes.cast(arr, _vp), len(jobs), ctypes.byref(best),
                                    cache_path.encode() if cache_path else None, stream_handle(stream)))
    return best


# ------------------------------------------------------------------------- serving (mqntt_serve.h)

MQ_SERVE_BATCHED, MQ_SERVE_PLAIN = 0, 1


class mq_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("slots", ctypes.c_uint), ("max_batch_jobs", ctypes.c_uint),
                ("linger_us", ctypes.c_double), ("wait_timeout_s", ctypes.c_double), ("mode", ctypes.c_int),
                ("reserve_bytes", ctypes.c_size_t)]


class mq_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("span_s", ctypes.c_double),
                ("jobs_per_s", ctypes.c_double), ("butterflies_per_s", ctypes.c_double),
                ("modmul_per_s", ctypes.c_double), ("mean_batch_jobs", ctypes.c_double),
                ("peak_inflight_bytes", ctypes.c_size_t), ("cancelled", ctypes.c_uint64),
                ("deferred", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Server:
    """Owns an mq_server* (freed by mq_server_destroy or on garbage collection)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mq_server_destroy(self.handle)
            self.handle = None


def mq_server_create(cfg: mq_server_cfg | None = None) -> Server:
    h = _vp()
    _check(load().mq_server_create(ctypes.byref(h), ctypes.cast(ctypes.byref(cfg), _vp) if cfg is not None else None))
    return Server(h.value)


def mq_submit(server: Server, job: mq_job) -> int:
    t = ctypes.c_uint64()
    _check(load().mq_submit(server.handle, ctypes.cast(ctypes.byref(job), _vp), ctypes.byref(t)))
    return t.value


def mq_cancel(server: Server, ticket: int):
    _check(load().mq_cancel(server.handle, ticket))


def mq_server_inject_alloc_failures(server: Server, n: int):
    _check(load().mq_server_inject_alloc_failures(server.handle, n))


def mq_poll(server: Server, ticket: int):
    done, st = ctypes.c_int(), ctypes.c_int()
    _check(load().mq_poll(server.handle, ticket, ctypes.byref(done), ctypes.byref(st)))
    return bool(done.value), st.value


def mq_wait(server: Server, ticket: int, timeout_s: float = 60.0) -> int:
    st = ctypes.c_int()
    _check(load().mq_wait(server.handle, ticket, timeout_s, ctypes.byref(st)))
    return st.value


def mq_server_drain(server: Server, timeout_s: float = 120.0):
    _check(load().mq_server_drain(server.handle, timeout_s))


def mq_server_poisson(server: Server, jobs, rate_per_s: float, n_requests: int, seed: int = 1) -> float:
    """Open-loop Poisson submission from a native thread; returns the achieved offered rate."""
    arr = _job_array(jobs)
    off = ctypes.c_double()
    _check(load().mq_server_poisson(server.handle, ctypes.cast(arr, _vp), len(jobs), rate_per_s, n_requests, seed,
                                    ctypes.byref(off)))
    return off.value


def mq_server_stats(server: Server) -> dict:
    st = mq_stats()
    _check(load().mq_server_stats(server.handle, ctypes.cast(ctypes.byref(st), _vp)))
    return st.as_dict()


def mq_server_reset_stats(server: Server):
    _check(load().mq_server_reset_stats(server.handle))


def mq_server_destroy(server: Server):
    if server.handle:
        _check(load().mq_server_destroy(server.handle))
        server.handle = None


# ------------------------------------------------------------------------- tensor marshalling

def to_device(a: np.ndarray, device="cuda"):
    """numpy uint64 residues -> int64 torch tensor with the same bits on the GPU."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def to_host(t) -> np.ndarray:
    """GPU int64 tensor -> numpy uint64 with the same bits."""
    return t.detach().cpu().numpy().view(np.uint64)
