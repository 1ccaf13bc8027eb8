"""The C-ABI library loads and exports every entry point include/xe.h declares (no GPU, no compute)."""
import ctypes
import os
import re

import pytest
import torch

import paper_1503_06189_b300 as xe

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "xe.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xe_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_functions():
    names = declared_functions()
    assert "xe_correlate" in names and "xe_assemble" in names and "xe_normalize" in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(xe.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(xe.EXPORTED) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(xe, n))


def test_host_only_calls():
    assert xe.xe_version() >= 10000
    assert "overflow" in xe.xe_strerror(xe.XE_EOVERFLOW) or "int32" in xe.xe_strerror(xe.XE_EOVERFLOW)
    assert xe.xe_correlate_workspace_size(xe.Shape(20, 1, 128)) == 0          # N % 16 != 0
    s = xe.Shape(256, 64, 16384)
    assert 0 < xe.xe_correlate_workspace_size(s) <= 4096          # fused default: work counter only
    jobs = [(0, 0, s, False)]
    unpacked = xe.xe_correlate_batched_workspace_size(jobs, dict(engine=xe.XE_ENGINE_UNPACKED, max_strip=0,
                                                                 k_flush=0, n_ctas=0))
    assert unpacked >= 64 * 512 * 16384                           # + the E5M2 operand in HBM
    assert xe.xe_assemble_workspace_size(xe.Shape(256, 1024, 4096)) == 1024 * 128 * 4


def test_binding_rejects_host_and_strided_buffers():
    """The binding passes raw addresses, so it refuses what would reach the library in the wrong
    place or layout: a host tensor where a device buffer is expected, and a non-contiguous view.
    Both are caught before the library is called."""
    with pytest.raises(ValueError, match="CUDA"):
        xe.xe_correlate(torch.zeros(16, dtype=torch.uint8), xe.Shape(16, 1, 1),
                        torch.zeros((1, xe.npairs(16), 2), dtype=torch.int32), False, None)
    with pytest.raises(ValueError, match="contiguous"):
        xe._ptr(torch.zeros((4, 8), dtype=torch.uint8).t())
    assert xe._ptr(1 << 20) == 1 << 20 and xe._dptr(None) is None


def test_shifted_packet_call_checks_delays_on_the_host():
    """xe_correlate_packets_shifted validates its host delays before it touches a device buffer:
    a delay out of [0, T] or one that differs within a block of 16 inputs is XE_EINVAL, and valid
    delays then fail only on the missing workspace (XE_ENOMEM)."""
    import numpy as np

    lib = xe.lib()
    N, F, T = 64, 8, 1024
    s = xe.Shape(N, F, T)

    def call(d):
        d = np.ascontiguousarray(np.asarray(d, dtype=np.int32))
        return lib.xe_correlate_packets_shifted(None, 0, 16 + 32 * N, 0, 1, s, d.ctypes.data, None, 0, None, None,
                                                None, None, 0, None)

    assert call(np.full(N, -1)) == xe.XE_EINVAL
    assert call(np.full(N, T + 1)) == xe.XE_EINVAL
    assert call(np.r_[np.zeros(N - 1, int), 1]) == xe.XE_EINVAL          # differs inside the last block
    assert call(np.repeat([0, T, 7, 300], 16)) == xe.XE_ENOMEM
