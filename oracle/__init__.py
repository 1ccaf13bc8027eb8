"""CPU oracle of the X-engine hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the package smoke check and the CPU-baseline leg of ``bench.py`` may import this
module. The product library (``paper_1503_06189_b300``) never imports, loads or calls it, and it
imports nothing from the product. It wraps ``xe_oracle.c`` (plain C, int64 arithmetic, plain
loops) through ctypes; the C source is built by :func:`build` with gcc.

Function / paper passage:
  sample          one 4+4-bit byte -> (re, im)                       Sec. I
  correlate       V_f[i,j] = sum_t x_i conj(x_j), i <= j              Sec. I, Sec. II-B
  correlate_pairs the same for selected (i, j) of one channel          Sec. I, Sec. II-B
  assemble        packets -> frame, zero-fill, reorder, dedup         Sec. II-A.2
  counts_from_mask      n_ij by brute force over the sample mask      Sec. II-C
  counts_from_counters  n_ij by the loss / flag / intersection counters  Sec. II-C
  normalize       V / n_ij                                            Sec. II-C
  time_shift      per-input integer sample delay (reading)           Fig. 4 caption
  time_shift_counts     the delay's samples without data as counters  Fig. 4 caption, Sec. II-C
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EOVERFLOW = 0, -1, -2


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp build of an oracle C source into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
                           "-o", tmp, src])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile xe_oracle.c into liboracle.so if it is missing or stale. Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


class Oracle:
    """ctypes view of one build of xe_oracle.c (the default build, or a test's mutant build)."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.xo_correlate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.xo_assemble.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.xo_flag_counts.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p]
        L.xo_counts_from_mask.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p]
        L.xo_counts_from_counters.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.xo_normalize.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p]
        L.xo_time_shift.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p]
        L.xo_time_shift_counts.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p]
        L.xo_pidx.restype = ctypes.c_int64
        L.xo_pidx.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.xo_npairs.restype = ctypes.c_int64
        L.xo_npairs.argtypes = [ctypes.c_int]
        L.xo_sample.argtypes = [ctypes.c_uint8, P(ctypes.c_int), P(ctypes.c_int)]
        L.xo_correlate_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        self.L = L

    def threads(self) -> int:
        return int(self.L.xo_threads())

    def npairs(self, n: int) -> int:
        return int(self.L.xo_npairs(n))

    def pidx(self, i: int, j: int, n: int) -> int:
        return int(self.L.xo_pidx(i, j, n))

    def sample(self, b: int):
        re, im = ctypes.c_int(), ctypes.c_int()
        self.L.xo_sample(b, ctypes.byref(re), ctypes.byref(im))
        return re.value, im.value

    def correlate(self, frame: np.ndarray, f0: int = 0, nf: int | None = None):
        """frame uint8 [T][F][N] -> (int64 vis [nf][P][2], status); EOVERFLOW = exceeds int32."""
        frame = np.ascontiguousarray(frame, dtype=np.uint8)
        T, F, N = frame.shape
        nf = F - f0 if nf is None else nf
        vis = np.zeros((nf, self.npairs(N), 2), dtype=np.int64)
        st = self.L.xo_correlate(_ptr(frame), N, F, T, f0, nf, _ptr(vis))
        if st == EINVAL:
            raise ValueError("xo_correlate: invalid arguments")
        return vis, st

    def correlate_pairs(self, frame: np.ndarray, f: int, pairs) -> np.ndarray:
        """Visibilities of channel f for the given (i, j), i <= j, pairs: int64 [n][2] (re, im)."""
        frame = np.ascontiguousarray(frame, dtype=np.uint8)
        T, F, N = frame.shape
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        out = np.zeros((pr.shape[0], 2), dtype=np.int64)
        if self.L.xo_correlate_pairs(_ptr(frame), N, F, T, f, _ptr(pr), pr.shape[0], _ptr(out)) != OK:
            raise ValueError("xo_correlate_pairs: invalid arguments")
        return out

    def assemble(self, pkts: np.ndarray, seq0: int, gps: int, n_inputs: int, n_chan: int, n_time: int,
                 lost: np.ndarray | None = None, stats: np.ndarray | None = None):
        """pkts uint8 [n][stride] in arrival order -> (frame, filled, lost, stats)."""
        pkts = np.ascontiguousarray(pkts, dtype=np.uint8)
        n = pkts.shape[0] if pkts.ndim == 2 else 0
        stride = pkts.shape[1] if pkts.ndim == 2 and pkts.shape[0] else 16 + 32 * n_inputs
        frame = np.full((n_time, n_chan, n_inputs), 0xA5, dtype=np.uint8)   # must all be overwritten
        filled = np.zeros((n_time // 4, n_chan // 8), dtype=np.uint8)
        lost = np.zeros(n_chan, dtype=np.uint32) if lost is None else lost
        stats = np.zeros(5, dtype=np.uint32) if stats is None else stats
        st = self.L.xo_assemble(_ptr(pkts), n, stride, seq0, gps, n_inputs, n_chan, n_time,
                                _ptr(frame), _ptr(filled), _ptr(lost), _ptr(stats))
        if st != OK:
            raise ValueError("xo_assemble: invalid arguments")
        return frame, filled, lost, stats

    def flag_counts(self, pkts: np.ndarray, seq0: int, gps: int, n_inputs: int, n_chan: int, n_time: int,
                    flag_count: np.ndarray | None = None, flag_pairs: np.ndarray | None = None):
        """F-engine flags from the packets' footers (Sec. II-C) -> (flag_count [F][N], flag_pairs [F][P]),
        accumulated onto the given arrays."""
        pkts = np.ascontiguousarray(pkts, dtype=np.uint8)
        n = pkts.shape[0] if pkts.ndim == 2 else 0
        stride = pkts.shape[1] if pkts.ndim == 2 and pkts.shape[0] else 16 + 36 * n_inputs
        fc = np.zeros((n_chan, n_inputs), np.uint32) if flag_count is None else flag_count
        fp = np.zeros((n_chan, self.npairs(n_inputs)), np.uint32) if flag_pairs is None else flag_pairs
        st = self.L.xo_flag_counts(_ptr(pkts), n, stride, seq0, gps, n_inputs, n_chan, n_time, _ptr(fc), _ptr(fp))
        if st != OK:
            raise ValueError("xo_flag_counts: invalid arguments")
        return fc, fp

    def counts_from_mask(self, valid: np.ndarray) -> np.ndarray:
        valid = np.ascontiguousarray(valid, dtype=np.uint8)
        T, F, N = valid.shape
        n = np.zeros((F, self.npairs(N)), dtype=np.uint32)
        if self.L.xo_counts_from_mask(_ptr(valid), N, F, T, _ptr(n)) != OK:
            raise ValueError("xo_counts_from_mask: invalid arguments")
        return n

    def counts_from_counters(self, t_int: int, lost: np.ndarray, n_inputs: int, flag_count=None,
                             flag_pairs=None):
        lost = np.ascontiguousarray(lost, dtype=np.uint32)
        F = lost.shape[0]
        fc = None if flag_count is None else np.ascontiguousarray(flag_count, dtype=np.uint32)
        fp = None if flag_pairs is None else np.ascontiguousarray(flag_pairs, dtype=np.uint32)
        n = np.zeros((F, self.npairs(n_inputs)), dtype=np.uint32)
        if self.L.xo_counts_from_counters(t_int, _ptr(lost), _ptr(fc), _ptr(fp), n_inputs, F, _ptr(n)) != OK:
            raise ValueError("xo_counts_from_counters: invalid arguments")
        return n

    def normalize(self, vis: np.ndarray, n: np.ndarray) -> np.ndarray:
        vis = np.ascontiguousarray(vis, dtype=np.int64)
        n = np.ascontiguousarray(n, dtype=np.uint32)
        F, P, _ = vis.shape
        N = int((np.sqrt(8 * P + 1) - 1) // 2)
        out = np.zeros((F, P, 2), dtype=np.float32)
        if self.L.xo_normalize(_ptr(vis), _ptr(n), N, F, _ptr(out)) != OK:
            raise ValueError("xo_normalize: invalid arguments")
        return out

    def time_shift(self, frame: np.ndarray, delays) -> np.ndarray:
        """frame uint8 [T][F][N], delays int [N] (0 <= d <= T) -> the shifted frame."""
        frame = np.ascontiguousarray(frame, dtype=np.uint8)
        T, F, N = frame.shape
        d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
        out = np.full_like(frame, 0xA5)
        if d.shape != (N,) or self.L.xo_time_shift(_ptr(frame), N, F, T, _ptr(d), _ptr(out)) != OK:
            raise ValueError("xo_time_shift: invalid arguments")
        return out

    def time_shift_counts(self, delays, n_inputs: int, n_chan: int, flag_count=None, flag_pairs=None):
        """Adds the shift's samples without data to (flag_count [F][N], flag_pairs [F][P])."""
        d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
        c = np.zeros((n_chan, n_inputs), np.uint32) if flag_count is None else flag_count
        x = np.zeros((n_chan, self.npairs(n_inputs)), np.uint32) if flag_pairs is None else flag_pairs
        if d.shape != (n_inputs,) or self.L.xo_time_shift_counts(_ptr(d), n_inputs, n_chan, _ptr(c), _ptr(x)) != OK:
            raise ValueError("xo_time_shift_counts: invalid arguments")
        return c, x


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def threads() -> int:
    return default().threads()


def npairs(n: int) -> int:
    return default().npairs(n)


def pidx(i: int, j: int, n: int) -> int:
    return default().pidx(i, j, n)


def sample(b: int):
    return default().sample(b)


def correlate(frame, f0: int = 0, nf=None):
    return default().correlate(frame, f0, nf)


def correlate_pairs(frame, f, pairs):
    return default().correlate_pairs(frame, f, pairs)


def assemble(pkts, seq0, gps, n_inputs, n_chan, n_time, lost=None, stats=None):
    return default().assemble(pkts, seq0, gps, n_inputs, n_chan, n_time, lost, stats)


def flag_counts(pkts, seq0, gps, n_inputs, n_chan, n_time, flag_count=None, flag_pairs=None):
    return default().flag_counts(pkts, seq0, gps, n_inputs, n_chan, n_time, flag_count, flag_pairs)


def counts_from_mask(valid):
    return default().counts_from_mask(valid)


def counts_from_counters(t_int, lost, n_inputs, flag_count=None, flag_pairs=None):
    return default().counts_from_counters(t_int, lost, n_inputs, flag_count, flag_pairs)


def normalize(vis, n):
    return default().normalize(vis, n)


def time_shift(frame, delays):
    return default().time_shift(frame, delays)


def time_shift_counts(delays, n_inputs, n_chan, flag_count=None, flag_pairs=None):
    return default().time_shift_counts(delays, n_inputs, n_chan, flag_count, flag_pairs)
