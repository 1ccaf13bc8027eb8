"""Parity of the CUDA path (called through the C ABI) with the CPU oracle, element by element.

Correlation and assembly must be bit-exact; normalisation must hold a relative tolerance of 1e-6
(the GPU rounds V and n to float and divides once in float: at most ~1.2e-7 relative).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def assert_vis_equal(got, want):
    got = got.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(got, want)


# ----------------------------------------------------------------------------- A2 unpack

@pytest.mark.parametrize("N,F,T", [(16, 2, 128), (48, 3, 300), (80, 1, 1), (256, 2, 4096)])
def test_unpack_codes(N, F, T):
    fr = synth.uniform_frame(N, F, T, 100 + N + T)
    want, R, ldy = X.e5m2_codes(fr)
    y = torch.full((F, ldy, R), 0x5A, dtype=torch.uint8, device="cuda")
    xe.xe_unpack(X.dev(fr), xe.Shape(N, F, T), y, ldy)
    np.testing.assert_array_equal(y.cpu().numpy(), want)


# ----------------------------------------------------------------------------- A3/A4 correlate

def test_correlate_tiny_config():
    """N=16, F=4, T=4096, i.i.d. uniform nibbles (seed 1): full bit-exact check."""
    fr = synth.uniform_frame(16, 4, 4096, 1)
    want, st = oracle.correlate(fr)
    assert st == oracle.OK
    assert_vis_equal(X.correlate(fr), want)


@pytest.mark.parametrize("N,F,T", [
    (16, 1, 1), (32, 3, 129), (48, 2, 1000), (64, 5, 256), (80, 2, 777), (144, 2, 640),
    (256, 3, 2048), (272, 2, 384), (512, 1, 512), (1024, 1, 256),
])
def test_correlate_shapes(N, F, T):
    """Several tiles, ragged inputs (N not a multiple of 64) and ragged time (T not a multiple of 128)."""
    fr = synth.uniform_frame(N, F, T, 7 * N + T)
    want, _ = oracle.correlate(fr)
    assert_vis_equal(X.correlate(fr), want)


def test_correlate_accumulate():
    """Integration across invocations (Sec. II-B): the second call adds to the first."""
    a = synth.signal_frame(64, 3, 1024, 3)
    b = synth.signal_frame(64, 3, 512, 4)
    va, _ = oracle.correlate(a)
    vb, _ = oracle.correlate(b)
    vis = X.correlate(a)
    X.correlate(b, vis=vis, accumulate=True)
    assert_vis_equal(vis, va + vb)


def test_correlate_zero_time():
    vis = X.correlate(np.zeros((0, 2, 16), np.uint8))
    assert not vis.any()


def test_correlate_worst_case_magnitudes():
    """Extreme samples (+-8, +-7) over a long frame: the largest partial sums the FP32 tensor-memory
    accumulator sees (|G| up to 64 * T = 2^22 at T = 65536) must stay exact."""
    rng = np.random.default_rng(5)
    T, F, N = 65536, 1, 32
    vals = np.array([0x88, 0x87, 0x78, 0x77, 0x80, 0x08], np.uint8)
    fr = vals[rng.integers(0, 6, (T, F, N))]
    fr[:, :, :4] = 0x88                    # four inputs at -8-8i: Re V = 128 T exactly
    want, _ = oracle.correlate(fr)
    assert_vis_equal(X.correlate(fr), want)


@pytest.mark.parametrize("engine", [xe.XE_ENGINE_FUSED_PAIR, xe.XE_ENGINE_LEGACY_S4, xe.XE_ENGINE_LEGACY_S8])
def test_correlate_int32_limit_closed_form(engine):
    """Every sample -8-8i over the longest integration the int32 output holds (T = 2^24 - 1): each
    visibility is T (-8-8i)(-8+8i) = 128 T = 2,147,483,520 + 0i, 128 below 2^31 (closed form)."""
    T, F, N = xe.XE_MAX_TIME, 1, 16
    frame = torch.full((T, F, N), 0x88, dtype=torch.uint8, device="cuda")
    (got,) = X.correlate_batched([frame], tune=dict(engine=engine, max_strip=0, k_flush=0, n_ctas=0))
    g = got.cpu().numpy().astype(np.int64)
    assert (g[..., 0] == 128 * T).all() and (g[..., 1] == 0).all()


@pytest.mark.parametrize("engine", [xe.XE_ENGINE_LEGACY_S4, xe.XE_ENGINE_LEGACY_S8])
def test_legacy_engine_accumulates(engine):
    """The legacy mma.sync engines add to the visibilities of an earlier call (Sec. II-B)."""
    a = synth.signal_frame(96, 3, 700, 11)
    b = synth.signal_frame(96, 3, 260, 12)
    va, _ = oracle.correlate(a)
    vb, _ = oracle.correlate(b)
    tune = dict(engine=engine, max_strip=0, k_flush=0, n_ctas=0)
    fa, fb = X.dev(a), X.dev(b)
    s_a, s_b = xe.Shape(96, 3, 700), xe.Shape(96, 3, 260)
    vis = torch.full((3, xe.npairs(96), 2), -5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_batched_workspace_size([(fa, vis, s_a, False)], tune), dtype=torch.uint8,
                     device="cuda")
    xe.xe_correlate_batched([(fa, vis, s_a, False)], ws, tune)
    xe.xe_correlate_batched([(fb, vis, s_b, True)], ws, tune)
    assert_vis_equal(vis, va + vb)


def test_correlate_overflow_bound_rejected():
    s = xe.Shape(16, 1, xe.XE_MAX_TIME + 1)
    vis = torch.zeros((1, xe.npairs(16), 2), dtype=torch.int32, device="cuda")
    frame = torch.zeros(16, dtype=torch.uint8, device="cuda")     # never read
    with pytest.raises(xe.XeError) as e:
        xe.xe_correlate(frame, s, vis, False, torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert e.value.status == xe.XE_EOVERFLOW


def test_correlate_invalid_shapes_rejected():
    for bad in (xe.Shape(20, 1, 128), xe.Shape(0, 1, 128), xe.Shape(16, 0, 128), xe.Shape(8192, 1, 128)):
        vis = torch.zeros(8, dtype=torch.int32, device="cuda")
        with pytest.raises(xe.XeError) as e:
            xe.xe_correlate(torch.zeros(16, dtype=torch.uint8, device="cuda"), bad, vis, False,
                            torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
        assert e.value.status == xe.XE_EINVAL


def test_correlate_workspace_too_small():
    fr = X.dev(synth.uniform_frame(16, 1, 128, 1))
    vis = torch.zeros((1, xe.npairs(16), 2), dtype=torch.int32, device="cuda")
    with pytest.raises(xe.XeError) as e:
        xe.xe_correlate(fr, xe.Shape(16, 1, 128), vis, False, torch.empty(64, dtype=torch.uint8, device="cuda"))
    assert e.value.status == xe.XE_ENOMEM


ENGINES = [xe.XE_ENGINE_FUSED, xe.XE_ENGINE_UNPACKED, xe.XE_ENGINE_UNPACKED_K, xe.XE_ENGINE_FUSED_PAIR,
           xe.XE_ENGINE_LEGACY_S4, xe.XE_ENGINE_LEGACY_S8]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("max_strip,k_flush", [(1, 128), (2, 256), (3, 384), (4, 128), (2, 0), (4, 0)])
def test_correlate_tunings_agree(engine, max_strip, k_flush):
    """Every engine, strip width and TMEM drain interval gives the same bits."""
    fr = synth.uniform_frame(272, 2, 1000, 9)
    want, _ = oracle.correlate(fr)
    (got,) = X.correlate_batched([fr], tune=dict(engine=engine, max_strip=max_strip, k_flush=k_flush, n_ctas=0))
    assert_vis_equal(got, want)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("N,F,T", [(16, 3, 200), (48, 2, 256), (80, 2, 300), (256, 4, 1024), (512, 1, 384)])
def test_correlate_engines_shapes(engine, N, F, T):
    """Small and ragged N (packed rows narrower than 64 bytes, partial 64-input blocks) per engine."""
    fr = synth.uniform_frame(N, F, T, 3 * N + T + engine)
    want, _ = oracle.correlate(fr)
    (got,) = X.correlate_batched([fr], tune=dict(engine=engine, max_strip=0, k_flush=0, n_ctas=0))
    assert_vis_equal(got, want)


@pytest.mark.parametrize("engine", ENGINES)
def test_correlate_few_ctas(engine):
    """Fewer persistent CTAs than work items: each CTA takes many items from the shared counter."""
    fr = synth.uniform_frame(256, 9, 512, 31)
    want, _ = oracle.correlate(fr)
    (got,) = X.correlate_batched([fr], tune=dict(engine=engine, max_strip=0, k_flush=0, n_ctas=3))
    assert_vis_equal(got, want)


def test_pair_engine_tiny():
    """CTA-pair engine on one small frame: one 256x256 block per channel (N=64)."""
    fr = synth.uniform_frame(64, 3, 384, 12)
    want, _ = oracle.correlate(fr)
    (got,) = X.correlate_batched([fr], tune=dict(engine=xe.XE_ENGINE_FUSED_PAIR, max_strip=0, k_flush=0, n_ctas=0))
    assert_vis_equal(got, want)


def test_pair_engine_accumulate_and_drain():
    """CTA-pair engine: off-diagonal blocks (N=384: 3 super-blocks), TMEM drains every 128 samples,
    and accumulation onto a previous result."""
    a = synth.signal_frame(384, 2, 640, 21)
    b = synth.signal_frame(384, 2, 256, 22)
    va, _ = oracle.correlate(a)
    vb, _ = oracle.correlate(b)
    tune = dict(engine=xe.XE_ENGINE_FUSED_PAIR, max_strip=0, k_flush=128, n_ctas=0)
    (got,) = X.correlate_batched([a], tune=tune)
    jobs = [(X.dev(b), got, xe.Shape(384, 2, 256), True)]
    ws = torch.empty(xe.xe_correlate_batched_workspace_size(jobs, tune), dtype=torch.uint8, device="cuda")
    xe.xe_correlate_batched(jobs, ws, tune)
    assert_vis_equal(got, va + vb)


def test_correlate_batched_uneven():
    """Jobs of different N, F and T in one persistent launch; each bit-exact."""
    shapes = [(64, 4, 1024), (128, 2, 384), (256, 3, 1280), (16, 5, 100), (512, 1, 256), (96, 2, 2000)]
    frames = [synth.signal_frame(N, F, T, 40 + k) for k, (N, F, T) in enumerate(shapes)]
    got = X.correlate_batched(frames)
    for fr, g in zip(frames, got):
        want, _ = oracle.correlate(fr)
        assert_vis_equal(g, want)


def test_correlate_maximum_inputs():
    """N = 4096, the largest input count the library accepts (8,390,656 visibilities per channel, 32
    blocks of 256 rows), with a ragged time tail, on the default engine and on the single-CTA and
    legacy engines."""
    N, F, T = 4096, 1, 300
    fr = synth.uniform_frame(N, F, T, 4096)
    want, st = oracle.correlate(fr)
    assert st == oracle.OK
    assert_vis_equal(X.correlate(fr), want)
    for engine in (xe.XE_ENGINE_FUSED, xe.XE_ENGINE_LEGACY_S8):
        (got,) = X.correlate_batched([fr], tune=dict(engine=engine, max_strip=0, k_flush=0, n_ctas=0))
        assert_vis_equal(got, want)


def test_correlate_batched_maximum_jobs():
    """XE_MAX_JOBS frames of different N, F and T in one launch, each bit-exact; one job more is
    rejected."""
    shapes = [(16 * (1 + k % 6), 1 + k % 3, 64 + 37 * k) for k in range(xe.XE_MAX_JOBS)]
    frames = [synth.uniform_frame(N, F, T, 900 + k) for k, (N, F, T) in enumerate(shapes)]
    got = X.correlate_batched(frames)
    for fr, g in zip(frames, got):
        want, _ = oracle.correlate(fr)
        assert_vis_equal(g, want)
    fr = X.dev(frames[0])
    vis = torch.zeros((fr.shape[1], xe.npairs(fr.shape[2]), 2), dtype=torch.int32, device="cuda")
    jobs = [(fr, vis, xe.Shape(fr.shape[2], fr.shape[1], fr.shape[0]), False)] * (xe.XE_MAX_JOBS + 1)
    with pytest.raises(xe.XeError) as e:
        xe.xe_correlate_batched(jobs, torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert e.value.status == xe.XE_EINVAL


def test_correlate_deterministic():
    fr = synth.uniform_frame(256, 2, 1024, 77)
    a = X.correlate(fr).cpu()
    b = X.correlate(fr).cpu()
    assert torch.equal(a, b)


def test_batched_launch_equals_plain_per_channel_launches():
    """All channels of a frame in one launch give exactly what one plain launch per channel gives
    (each channel's samples copied to a contiguous [T][1][N] frame first), and both match the
    oracle. N = 256 makes three 256x256 blocks per channel; T is ragged."""
    N, F, T = 256, 6, 1000
    fr = synth.signal_frame(N, F, T, 91)
    want, _ = oracle.correlate(fr)
    batched = X.correlate(fr)
    frame = X.dev(fr)
    s1 = xe.Shape(N, 1, T)
    ws = torch.empty(max(1, xe.xe_correlate_workspace_size(s1)), dtype=torch.uint8, device="cuda")
    per = torch.full_like(batched, 0x7EADBEEF)
    for f in range(F):
        xe.xe_correlate(frame[:, f:f + 1, :].contiguous(), s1, per[f], False, ws)
    torch.cuda.synchronize()
    assert torch.equal(per, batched)
    assert_vis_equal(per, want)


def test_correlate_pathfinder_frame_sampled():
    """Per-server Pathfinder frame: N=256, F=64, T=16384 (256 MiB), signal model. The oracle checks 6
    channels spread over the frame; all channels are compared against a second launch with a
    different strip width (bit-identical)."""
    N, F, T = 256, 64, 16384
    fr = synth.signal_frame_torch(N, F, T, 2, device="cuda")
    vis = X.correlate(fr)
    chans = [0, 1, 17, 31, 50, 63]
    host = fr.cpu().numpy()
    for f in chans:
        want, st = oracle.correlate(host, f, 1)
        assert st == oracle.OK
        assert_vis_equal(vis[f:f + 1], want)
    for engine, ms in ((xe.XE_ENGINE_UNPACKED, 4), (xe.XE_ENGINE_UNPACKED_K, 3), (xe.XE_ENGINE_FUSED, 1),
                       (xe.XE_ENGINE_FUSED_PAIR, 0)):
        (alt,) = X.correlate_batched([fr], tune=dict(engine=engine, max_strip=ms, k_flush=2048, n_ctas=0))
        assert torch.equal(alt, vis), (engine, ms)


# ----------------------------------------------------------------------------- A1 assemble

def _assemble_gpu(pk, seq0, gps, N, F, T, lost=None, stats=None):
    s = xe.Shape(N, F, T)
    frame = torch.full((T, F, N), 0xA5, dtype=torch.uint8, device="cuda")
    filled = torch.full((T // 4, F // 8), 7, dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda") if lost is None else lost
    stats = torch.zeros(5, dtype=torch.int32, device="cuda") if stats is None else stats
    ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
    pkd = X.dev(pk) if pk.shape[0] else torch.empty(16, dtype=torch.uint8, device="cuda")
    stride = pk.shape[1] if pk.ndim == 2 and pk.shape[0] else synth.packet_stride(N)
    xe.xe_assemble(pkd, pk.shape[0], stride, seq0, gps, s, frame, filled, lost, stats, ws)
    return frame.cpu().numpy(), filled.cpu().numpy(), lost.cpu().numpy().astype(np.uint32), stats.cpu().numpy().astype(np.uint32)


@pytest.mark.parametrize("p_drop,p_reorder,p_dup", [(0, 0, 0), (0.001, 0.005, 0), (0.05, 0.2, 0.05), (0.5, 0.5, 0.3)])
def test_assemble_matches_oracle(p_drop, p_reorder, p_dup):
    N, F, T, gps = 256, 64, 256, 2
    fr = synth.signal_frame(N, F, T + 64, 8)
    pk = synth.packet_stream(fr, 500, gps, seed=9, p_drop=p_drop, p_reorder=p_reorder, p_dup=p_dup)
    seq0 = 500 + 4                                   # 4 late slots before, 12 early slots after
    want = oracle.assemble(pk, seq0, gps, N, F, T)
    got = _assemble_gpu(pk, seq0, gps, N, F, T)
    for w, g in zip(want, got):
        np.testing.assert_array_equal(g, w)


def test_assemble_first_arrival_wins_and_invalid():
    N, F, T, gps = 16, 16, 32, 1
    fr = synth.uniform_frame(N, F, T, 12)
    pk = synth.packetize(fr, 0, gps)
    fake = pk[3].copy()
    fake[16:] = 0x11
    bad = pk[4].copy()
    bad[0:2] = np.frombuffer(np.uint16(5).tobytes(), np.uint8)
    arr = np.concatenate([pk[:10], fake[None], bad[None], pk[10:], pk[3:4]])
    want = oracle.assemble(arr, 0, gps, N, F, T)
    got = _assemble_gpu(arr, 0, gps, N, F, T)
    for w, g in zip(want, got):
        np.testing.assert_array_equal(g, w)
    assert got[3][1] == 2 and got[3][4] == 1


def test_assemble_empty_packet_set():
    N, F, T, gps = 16, 8, 16, 1
    pk = np.zeros((0, synth.packet_stride(N)), np.uint8)
    frame, filled, lost, stats = _assemble_gpu(pk, 0, gps, N, F, T)
    assert not frame.any() and not filled.any() and (lost == T).all() and not stats.any()


# ----------------------------------------------------------------------------- A5 normalise

def _rel_close(got, want):
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    assert np.all(err <= REL_TOL * np.abs(want.astype(np.float64)) + 1e-30), float(np.max(err / (np.abs(want) + 1e-30)))


def test_normalize_loss_only():
    N, F, T = 64, 8, 2048
    fr = synth.signal_frame(N, F, T, 13)
    vis64, _ = oracle.correlate(fr)
    rng = np.random.default_rng(14)
    lost = (rng.integers(0, 64, F) * 4).astype(np.uint32)
    lost[3] = T                                      # everything lost: n = 0 -> 0
    n = oracle.counts_from_counters(T, lost, N)
    want = oracle.normalize(vis64, n)
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device="cuda")
    n_out = torch.empty((F, xe.npairs(N)), dtype=torch.int32, device="cuda")
    xe.xe_normalize(X.dev(vis64.astype(np.int32)), xe.Shape(N, F, T), T, X.dev(lost.view(np.int32)), out, n_out)
    _rel_close(out.cpu().numpy(), want)
    np.testing.assert_array_equal(n_out.cpu().numpy().astype(np.uint32), n)


def test_normalize_with_flags():
    N, F, T = 48, 3, 400
    rng = np.random.default_rng(15)
    vis64 = rng.integers(-2**31 + 1, 2**31 - 1, (F, xe.npairs(N), 2)).astype(np.int64)
    present = np.repeat(rng.random((T // 4, F)) > 0.1, 4, axis=0)
    flags = (rng.random((T, F, N)) < 0.05) & present[:, :, None]
    lost = (T - present.sum(0)).astype(np.uint32)
    fc = flags.sum(0).astype(np.uint32)
    iu = np.triu_indices(N)
    fp = np.stack([(flags[:, f, :, None] & flags[:, f, None, :]).sum(0)[iu] for f in range(F)]).astype(np.uint32)
    n = oracle.counts_from_counters(T, lost, N, fc, fp)
    np.testing.assert_array_equal(n, oracle.counts_from_mask((present[:, :, None] & ~flags).astype(np.uint8)))
    want = oracle.normalize(vis64, n)
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device="cuda")
    n_out = torch.empty((F, xe.npairs(N)), dtype=torch.int32, device="cuda")
    xe.xe_normalize(X.dev(vis64.astype(np.int32)), xe.Shape(N, F, T), T, X.dev(lost.view(np.int32)), out, n_out,
                    flag_count=X.dev(fc.view(np.int32)), flag_pairs=X.dev(fp.view(np.int32)))
    _rel_close(out.cpu().numpy(), want)
    np.testing.assert_array_equal(n_out.cpu().numpy().astype(np.uint32), n)


# ----------------------------------------------------------------------------- end to end

def test_frame_pipeline_end_to_end():
    """Packets with loss -> assemble -> correlate (two frames accumulated) -> normalise, against the
    oracle's assembly, correlation and brute-force-mask sample counts."""
    N, F, T, gps = 128, 32, 512, 2
    s = xe.Shape(N, F, T)
    vis = torch.empty((F, xe.npairs(N), 2), dtype=torch.int32, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws_c = torch.empty(xe.xe_correlate_workspace_size(s), dtype=torch.uint8, device="cuda")
    want_vis = 0
    valid = []
    for k in range(2):
        fr = synth.signal_frame(N, F, T, 60 + k)
        pk = synth.packet_stream(fr, 1000 + k * T // 4, gps, seed=70 + k, p_drop=0.02, p_reorder=0.05, p_dup=0.01)
        frame_o, filled_o, _, _ = oracle.assemble(pk, 1000 + k * T // 4, gps, N, F, T)
        v, _ = oracle.correlate(frame_o)
        want_vis = want_vis + v
        valid.append(np.repeat(np.repeat(filled_o, 4, axis=0), 8, axis=1)[:, :, None].repeat(N, axis=2))
        frame = torch.empty((T, F, N), dtype=torch.uint8, device="cuda")
        filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
        ws_a = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
        xe.xe_assemble(X.dev(pk), pk.shape[0], pk.shape[1], 1000 + k * T // 4, gps, s, frame, filled, lost, stats, ws_a)
        xe.xe_correlate(frame, s, vis, k > 0, ws_c)
    assert_vis_equal(vis, want_vis)
    n = oracle.counts_from_mask(np.concatenate(valid).astype(np.uint8))
    want = oracle.normalize(want_vis, n)
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device="cuda")
    xe.xe_normalize(vis, xe.Shape(N, F, 2 * T), 2 * T, lost, out)
    _rel_close(out.cpu().numpy(), want)


# ----------------------------------------------------------------------------- failure detection

def test_bounded_wait_times_out_and_context_survives():
    assert xe.xe_device_status() == xe.XE_OK
    xe.xe_selftest_timeout(2_000_000)               # 2 ms wait on a flag nothing sets
    assert xe.xe_device_status() == xe.XE_ETIMEOUT
    assert xe.xe_device_status() == xe.XE_OK         # read clears it
    fr = synth.uniform_frame(16, 1, 256, 3)
    want, _ = oracle.correlate(fr)
    assert_vis_equal(X.correlate(fr), want)


def test_rate_probe_kinds():
    """The instruction-rate probe runs its three kinds (mma.sync s4, mma.sync s8, dp4a) and rejects
    any other."""
    sink = torch.zeros(2 * 256, dtype=torch.int32, device="cuda")
    for kind in (0, 1, 2):
        xe.xe_probe_mma_legacy(kind, 2, 3, sink)
    torch.cuda.synchronize()
    with pytest.raises(xe.XeError) as e:
        xe.xe_probe_mma_legacy(3, 2, 3, sink)
    assert e.value.status == xe.XE_EINVAL
