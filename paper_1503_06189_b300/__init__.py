"""Python binding of libxe, the sm_103a X-engine library declared in include/xe.h.

Argument marshalling only: every step of the hot path runs in libxe's CUDA kernels. torch is used
for device memory and streams. The functions keep the C names; tensors are passed as torch CUDA
tensors (or raw integer device pointers where noted) and shapes as ``Shape(N, F, T)``.

There is no fallback: if libxe.so is missing or fails to load, the first call into the binding
raises ImportError (importing the package alone does not, so that its build module can run).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxe.so")

XE_OK, XE_EINVAL, XE_EOVERFLOW, XE_ENOMEM, XE_ECUDA, XE_ETIMEOUT, XE_EAGAIN = 0, -1, -2, -3, -4, -5, -6
XE_MAX_TIME = (1 << 24) - 1
XE_MAX_JOBS = 64
XE_ENGINE_AUTO, XE_ENGINE_UNPACKED, XE_ENGINE_FUSED, XE_ENGINE_UNPACKED_K, XE_ENGINE_FUSED_PAIR = 0, 1, 2, 3, 4
XE_ENGINE_LEGACY_S4, XE_ENGINE_LEGACY_S8 = 5, 6
XE_LAYOUT_AUTO, XE_LAYOUT_GRAM, XE_LAYOUT_GRAM_TWIN, XE_LAYOUT_GRAM_WIDE, XE_LAYOUT_FOLD = 0, 1, 2, 3, 4
XE_LAYOUT_FRAME_BLOCKS = 5
XE_LAYOUT_FOLD_SPLIT = 6
XE_TUNE_MAX_ENTRIES = 256
XE_TUNE_PACKETS, XE_TUNE_FRAMES = 0, 1

EXPORTED = [
    "xe_strerror", "xe_last_cuda_error", "xe_version", "xe_device_status", "xe_selftest_timeout",
    "xe_assemble_workspace_size", "xe_assemble", "xe_assemble_noalloc", "xe_unpack", "xe_correlate_workspace_size",
    "xe_correlate", "xe_correlate_batched_workspace_size", "xe_correlate_batched", "xe_tune_table_set",
    "xe_tune_table_get",
    "xe_correlate_packets_workspace_size", "xe_correlate_packets", "xe_correlate_packets_shifted",
    "xe_flag_counts_workspace_size",
    "xe_flag_counts", "xe_normalize", "xe_probe_mma_legacy", "xe_time_shift", "xe_time_shift_counts",
    "xe_stream_create", "xe_stream_submit", "xe_stream_submit_device", "xe_stream_flush", "xe_stream_poll", "xe_stream_release",
    "xe_stream_stats", "xe_stream_destroy",
]


class XeError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        L = lib()
        msg = L.xe_strerror(status).decode()
        if status == XE_ECUDA:
            msg += f" (cudaError {L.xe_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")


class Shape(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int32), ("n_chan", ctypes.c_int32), ("n_time", ctypes.c_int32)]

    def __init__(self, n_inputs=0, n_chan=0, n_time=0):
        super().__init__(int(n_inputs), int(n_chan), int(n_time))

    def __repr__(self):
        return f"Shape(N={self.n_inputs}, F={self.n_chan}, T={self.n_time})"


class Job(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_void_p), ("vis", ctypes.c_void_p), ("s", Shape), ("accumulate", ctypes.c_int32),
                ("max_strip", ctypes.c_int32)]


class Tune(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int32), ("max_strip", ctypes.c_int32), ("k_flush", ctypes.c_int32),
                ("n_ctas", ctypes.c_int32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int32), ("t_bucket", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("layout", ctypes.c_int32),
                ("pairs", ctypes.c_int32), ("odd_pairs", ctypes.c_int32), ("k_flush", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class StreamCfg(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("groups_per_stream", ctypes.c_int32), ("n_inputs", ctypes.c_int32),
                ("n_time", ctypes.c_int32), ("pkt_stride", ctypes.c_uint32), ("reorder_window", ctypes.c_int32),
                ("ring_frames", ctypes.c_int32), ("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("n_cuda_streams", ctypes.c_int32), ("hbm_budget", ctypes.c_uint64), ("batch_wait_us", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int32), ("slot", ctypes.c_int32), ("frame", ctypes.c_int64),
                ("out", ctypes.c_void_p), ("vis", ctypes.c_void_p), ("n", ctypes.c_void_p),
                ("lost", ctypes.c_void_p), ("stats", ctypes.c_void_p), ("packets", ctypes.c_uint32),
                ("batch", ctypes.c_uint32), ("latency_ns", ctypes.c_uint64), ("latency_submit_ns", ctypes.c_uint64)]


class StreamStats(ctypes.Structure):
    _fields_ = [("packets_submitted", ctypes.c_uint64), ("packets_late", ctypes.c_uint64),
                ("frames_closed", ctypes.c_uint64), ("frames_done", ctypes.c_uint64),
                ("frames_released", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("max_batch_seen", ctypes.c_uint64), ("latency_p50_us", ctypes.c_double),
                ("latency_p99_us", ctypes.c_double), ("latency_max_us", ctypes.c_double),
                ("device_bytes", ctypes.c_uint64), ("slots", ctypes.c_int32),
                ("latency_submit_p50_us", ctypes.c_double), ("latency_submit_p99_us", ctypes.c_double),
                ("latency_submit_max_us", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libxe.so not built at {LIB_PATH}; run `python -m paper_1503_06189_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, i32, u32, u64, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
    L.xe_strerror.restype = ctypes.c_char_p
    L.xe_strerror.argtypes = [ctypes.c_int]
    L.xe_last_cuda_error.restype = ctypes.c_int
    L.xe_version.restype = ctypes.c_int
    L.xe_device_status.argtypes = [ctypes.POINTER(ctypes.c_int), vp]
    L.xe_selftest_timeout.argtypes = [u64, vp]
    L.xe_probe_mma_legacy.argtypes = [i32, i32, i32, vp, vp]
    L.xe_assemble_workspace_size.restype = sz
    L.xe_assemble_workspace_size.argtypes = [Shape]
    L.xe_assemble.argtypes = [vp, u32, u32, u64, i32, Shape, vp, vp, vp, vp, vp, sz, vp]
    L.xe_assemble_noalloc.argtypes = [vp, u32, u32, u64, i32, Shape, vp, vp, vp, vp, vp]
    L.xe_unpack.argtypes = [vp, Shape, vp, i64, vp]
    L.xe_correlate_workspace_size.restype = sz
    L.xe_correlate_workspace_size.argtypes = [Shape]
    L.xe_correlate.argtypes = [vp, Shape, vp, ctypes.c_int, vp, sz, vp]
    L.xe_correlate_batched_workspace_size.restype = sz
    L.xe_correlate_batched_workspace_size.argtypes = [ctypes.POINTER(Job), i32, ctypes.POINTER(Tune)]
    L.xe_correlate_batched.argtypes = [ctypes.POINTER(Job), i32, ctypes.POINTER(Tune), vp, sz, vp]
    L.xe_tune_table_set.argtypes = [ctypes.POINTER(TuneEntry), i32]
    L.xe_tune_table_get.argtypes = [ctypes.POINTER(TuneEntry), i32]
    L.xe_correlate_packets_workspace_size.restype = sz
    L.xe_correlate_packets_workspace_size.argtypes = [Shape]
    L.xe_correlate_packets.argtypes = [vp, u32, u32, u64, i32, Shape, vp, ctypes.c_int, vp, vp, vp, vp, sz, vp]
    L.xe_correlate_packets_shifted.argtypes = [vp, u32, u32, u64, i32, Shape, vp, vp, ctypes.c_int, vp, vp, vp, vp,
                                               sz, vp]
    L.xe_flag_counts_workspace_size.restype = sz
    L.xe_flag_counts_workspace_size.argtypes = [Shape]
    L.xe_flag_counts.argtypes = [vp, u32, u32, u64, i32, Shape, vp, vp, vp, sz, vp]
    L.xe_normalize.argtypes = [vp, Shape, u32, vp, vp, vp, vp, vp, vp]
    L.xe_time_shift.argtypes = [vp, Shape, vp, vp, vp]
    L.xe_time_shift_counts.argtypes = [vp, Shape, vp, vp, vp]
    L.xe_stream_create.argtypes = [ctypes.POINTER(StreamCfg), ctypes.POINTER(vp)]
    L.xe_stream_submit.argtypes = [vp, i32, vp, u32]
    L.xe_stream_submit_device.argtypes = [vp, i32, vp, vp, u32]
    L.xe_stream_flush.argtypes = [vp]
    L.xe_stream_poll.argtypes = [vp, ctypes.POINTER(Result), i32]
    L.xe_stream_release.argtypes = [vp, ctypes.POINTER(Result)]
    L.xe_stream_stats.argtypes = [vp, ctypes.POINTER(StreamStats)]
    L.xe_stream_destroy.argtypes = [vp]
    for name in EXPORTED:
        getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
    return L


_lib = None


def lib():
    """The loaded libxe (loaded on first use; raises ImportError if it is missing)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


class _Lazy:
    def __getattr__(self, name):
        return getattr(lib(), name)


_L = _Lazy()


# ----------------------------------------------------------------------------- marshalling helpers

def _ptr(t):
    """Address of a dense buffer: an int (a raw address) passes through; a tensor must be contiguous,
    since every libxe buffer is a dense array in the layout include/xe.h states."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("libxe buffers are dense arrays: pass a contiguous tensor")
    return t.data_ptr()


def _dptr(t):
    """As _ptr, for the buffers libxe's kernels read or write: a tensor must live on a CUDA device."""
    if t is not None and not isinstance(t, int) and not t.is_cuda:
        raise ValueError("libxe device arguments must be CUDA tensors (or raw device addresses)")
    return _ptr(t)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, what: str):
    if st != XE_OK:
        raise XeError(st, what)


def _nbytes(t):
    return 0 if t is None else (t if isinstance(t, int) else t.numel() * t.element_size())


def npairs(n: int) -> int:
    return n * (n + 1) // 2


# ----------------------------------------------------------------------------- library

def xe_strerror(status: int) -> str:
    return _L.xe_strerror(status).decode()


def xe_last_cuda_error() -> int:
    return _L.xe_last_cuda_error()


def xe_version() -> int:
    return _L.xe_version()


def xe_device_status(stream=None) -> int:
    v = ctypes.c_int(0)
    _check(_L.xe_device_status(ctypes.byref(v), _stream(stream)), "xe_device_status")
    return v.value


def xe_selftest_timeout(timeout_ns: int, stream=None):
    _check(_L.xe_selftest_timeout(timeout_ns, _stream(stream)), "xe_selftest_timeout")


def xe_probe_mma_legacy(kind: int, blocks: int, iters: int, sink, stream=None):
    """Rate probe of the legacy mma.sync path: kind 0 = m16n8k64 s4, 1 = m16n8k32 s8."""
    _check(_L.xe_probe_mma_legacy(kind, blocks, iters, _dptr(sink), _stream(stream)), "xe_probe_mma_legacy")


# ----------------------------------------------------------------------------- A1

def xe_assemble_workspace_size(shape: Shape) -> int:
    return _L.xe_assemble_workspace_size(shape)


def xe_assemble(pkts, n_pkts: int, pkt_stride: int, seq0: int, groups_per_stream: int, shape: Shape,
                frame, filled, lost, stats, ws, stream=None):
    _check(_L.xe_assemble(_dptr(pkts), n_pkts, pkt_stride, seq0, groups_per_stream, shape, _dptr(frame),
                            _dptr(filled), _dptr(lost), _dptr(stats), _dptr(ws), _nbytes(ws), _stream(stream)),
           "xe_assemble")


XE_ASSEMBLE_NOALLOC_MAX_SLOTS = 1 << 18


def xe_assemble_noalloc(pkts, n_pkts: int, pkt_stride: int, seq0: int, groups_per_stream: int, shape: Shape,
                        frame, filled, lost, stats, stream=None):
    """xe_assemble without a workspace, for callers that cannot allocate device memory at this point
    (non-blocking real-time loops, hosts that own all device memory): the owner table is a fixed
    1 MiB array inside libxe shared by every call, so calls must not overlap on the GPU, and frames
    with (T/4)*(F/8) above XE_ASSEMBLE_NOALLOC_MAX_SLOTS are rejected (XE_ENOMEM)."""
    _check(_L.xe_assemble_noalloc(_dptr(pkts), n_pkts, pkt_stride, seq0, groups_per_stream, shape, _dptr(frame),
                                  _dptr(filled), _dptr(lost), _dptr(stats), _stream(stream)), "xe_assemble_noalloc")


# ----------------------------------------------------------------------------- A2..A4

def xe_unpack(frame, shape: Shape, y, ldy: int, stream=None):
    _check(_L.xe_unpack(_dptr(frame), shape, _dptr(y), ldy, _stream(stream)), "xe_unpack")


def xe_correlate_workspace_size(shape: Shape) -> int:
    return _L.xe_correlate_workspace_size(shape)


def xe_correlate(frame, shape: Shape, vis, accumulate: bool, ws, stream=None):
    _check(_L.xe_correlate(_dptr(frame), shape, _dptr(vis), 1 if accumulate else 0, _dptr(ws), _nbytes(ws),
                             _stream(stream)), "xe_correlate")


def _jobs(jobs):
    """jobs: (frame, vis, Shape, accumulate) or (frame, vis, Shape, accumulate, max_strip) tuples."""
    arr = (Job * len(jobs))()
    for k, j in enumerate(jobs):
        frame, vis, shape, acc = j[:4]
        ms = j[4] if len(j) > 4 else 0
        arr[k] = Job(_dptr(frame), _dptr(vis), shape, 1 if acc else 0, int(ms))
    return arr


def _tune(tune):
    if tune is None:
        return None
    if isinstance(tune, Tune):
        return ctypes.byref(tune)
    return ctypes.byref(Tune(**tune))


def xe_correlate_batched_workspace_size(jobs, tune=None) -> int:
    arr = _jobs(jobs)
    return _L.xe_correlate_batched_workspace_size(arr, len(jobs), _tune(tune))


def xe_correlate_batched(jobs, ws, tune=None, stream=None):
    """jobs: sequence of (frame, vis, Shape, accumulate)."""
    arr = _jobs(jobs)
    _check(_L.xe_correlate_batched(arr, len(jobs), _tune(tune), _dptr(ws), _nbytes(ws), _stream(stream)),
           "xe_correlate_batched")


def xe_tune_table_set(entries):
    """Replaces libxe's tuning table. entries: TuneEntry objects or dicts with TuneEntry's fields."""
    arr = (TuneEntry * max(1, len(entries)))()
    for k, e in enumerate(entries):
        arr[k] = e if isinstance(e, TuneEntry) else TuneEntry(**e)
    _check(_L.xe_tune_table_set(arr, len(entries)), "xe_tune_table_set")


def xe_tune_table_get():
    """The tuning table as a list of dicts."""
    n = _L.xe_tune_table_get(None, 0)
    arr = (TuneEntry * max(1, n))()
    n = _L.xe_tune_table_get(arr, n)
    return [arr[k].as_dict() for k in range(n)]


def xe_flag_counts_workspace_size(shape: Shape) -> int:
    return _L.xe_flag_counts_workspace_size(shape)


def xe_flag_counts(pkts, n_pkts: int, pkt_stride: int, seq0: int, groups_per_stream: int, shape: Shape,
                   flag_count, flag_pairs, ws, stream=None):
    """F-engine flags from the packets' footers: += per-input counts and pair intersections."""
    _check(_L.xe_flag_counts(_dptr(pkts), n_pkts, pkt_stride, seq0, groups_per_stream, shape, _dptr(flag_count),
                             _dptr(flag_pairs), _dptr(ws), _nbytes(ws), _stream(stream)), "xe_flag_counts")


def xe_correlate_packets_workspace_size(shape: Shape) -> int:
    return _L.xe_correlate_packets_workspace_size(shape)


def xe_correlate_packets(pkts, n_pkts: int, pkt_stride: int, seq0: int, groups_per_stream: int, shape: Shape,
                         vis, accumulate: bool, filled, lost, stats, ws, stream=None):
    """Zero-copy assembly + correlation: the result of xe_assemble then xe_correlate, without the frame."""
    _check(_L.xe_correlate_packets(_dptr(pkts), n_pkts, pkt_stride, seq0, groups_per_stream, shape, _dptr(vis),
                                   1 if accumulate else 0, _dptr(filled), _dptr(lost), _dptr(stats), _dptr(ws),
                                   _nbytes(ws), _stream(stream)), "xe_correlate_packets")


def xe_correlate_packets_shifted(pkts, n_pkts: int, pkt_stride: int, seq0: int, groups_per_stream: int,
                                 shape: Shape, delays, vis, accumulate: bool, filled, lost, stats, ws, stream=None):
    """xe_correlate_packets with input n read delays[n] samples late (host sequence of N ints, equal within
    each block of 16 inputs): the result of xe_assemble, xe_time_shift and xe_correlate, in one pass."""
    d = _host_delays(delays, shape.n_inputs)
    _check(_L.xe_correlate_packets_shifted(_dptr(pkts), n_pkts, pkt_stride, seq0, groups_per_stream, shape,
                                           d.ctypes.data, _dptr(vis), 1 if accumulate else 0, _dptr(filled),
                                           _dptr(lost), _dptr(stats), _dptr(ws), _nbytes(ws), _stream(stream)),
           "xe_correlate_packets_shifted")


# ----------------------------------------------------------------------------- time shift

def _host_delays(delays, n_inputs: int):
    import numpy as np

    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    if d.shape != (n_inputs,):
        raise ValueError("delays: one int32 per input")
    return d


def xe_time_shift(frame_in, shape: Shape, delays, frame_out, stream=None):
    """Delays input n of every channel by delays[n] samples (host sequence of N ints)."""
    d = _host_delays(delays, shape.n_inputs)
    _check(_L.xe_time_shift(_dptr(frame_in), shape, d.ctypes.data, _dptr(frame_out), _stream(stream)), "xe_time_shift")


def xe_time_shift_counts(delays, shape: Shape, flag_count, flag_pairs, stream=None):
    """Adds the shift's samples without data to xe_normalize's per-input counters."""
    d = _host_delays(delays, shape.n_inputs)
    _check(_L.xe_time_shift_counts(d.ctypes.data, shape, _dptr(flag_count), _dptr(flag_pairs), _stream(stream)),
           "xe_time_shift_counts")


# ----------------------------------------------------------------------------- A5

def xe_normalize(vis, shape: Shape, t_int: int, lost, out, n_out=None, flag_count=None, flag_pairs=None,
                 stream=None):
    _check(_L.xe_normalize(_dptr(vis), shape, t_int, _dptr(lost), _dptr(flag_count), _dptr(flag_pairs), _dptr(out),
                             _dptr(n_out), _stream(stream)), "xe_normalize")


# ----------------------------------------------------------------------------- A7

def xe_stream_create(cfg: StreamCfg):
    """Returns an opaque handle (int) to a serving runtime on the current device."""
    h = ctypes.c_void_p()
    _check(_L.xe_stream_create(ctypes.byref(cfg), ctypes.byref(h)), "xe_stream_create")
    return h.value


def xe_stream_submit(handle, stream_id: int, host_pkts, n_pkts: int) -> int:
    """host_pkts: a pointer (int) or a torch/numpy buffer in host memory. Returns XE_OK or XE_EAGAIN."""
    if hasattr(host_pkts, "ctypes"):
        ptr = host_pkts.ctypes.data
    else:
        ptr = _ptr(host_pkts)
    st = _L.xe_stream_submit(handle, stream_id, ptr, n_pkts)
    if st not in (XE_OK, XE_EAGAIN):
        raise XeError(st, "xe_stream_submit")
    return st


def xe_stream_submit_device(handle, stream_id: int, dev_pkts, host_headers, n_pkts: int) -> int:
    """dev_pkts: device records (CUDA tensor or address); host_headers: their 16-byte headers back to
    back in host memory (numpy/torch CPU buffer or address). Returns XE_OK or XE_EAGAIN."""
    hdr = host_headers.ctypes.data if hasattr(host_headers, "ctypes") else _ptr(host_headers)
    st = _L.xe_stream_submit_device(handle, stream_id, _dptr(dev_pkts), hdr, n_pkts)
    if st not in (XE_OK, XE_EAGAIN):
        raise XeError(st, "xe_stream_submit_device")
    return st


def xe_stream_flush(handle) -> int:
    """Closes every open frame; XE_EAGAIN if the queue of closed frames filled first (poll, release,
    call again)."""
    st = _L.xe_stream_flush(handle)
    if st not in (XE_OK, XE_EAGAIN):
        raise XeError(st, "xe_stream_flush")
    return st


def xe_stream_poll(handle, timeout_ms: int):
    """Next completed frame as a Result, or None on timeout."""
    r = Result()
    st = _L.xe_stream_poll(handle, ctypes.byref(r), timeout_ms)
    if st == XE_ETIMEOUT:
        return None
    _check(st, "xe_stream_poll")
    return r


def xe_stream_release(handle, result: Result):
    _check(_L.xe_stream_release(handle, ctypes.byref(result)), "xe_stream_release")


def xe_stream_stats(handle) -> StreamStats:
    o = StreamStats()
    _check(_L.xe_stream_stats(handle, ctypes.byref(o)), "xe_stream_stats")
    return o


def xe_stream_destroy(handle):
    _check(_L.xe_stream_destroy(handle), "xe_stream_destroy")
