"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each ``pin_*`` function checks one fact and takes the oracle build to check, so the same pins can
be run against mutant builds with a planted mistake (test_oracle_mutants.py).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- helpers

def brute_full(frame):
    """Full-square V[f][i][j] = sum_t x_i conj(x_j) with Python complex integers (tiny inputs)."""
    T, F, N = frame.shape

    def dec(b):
        hi, lo = b >> 4, b & 15
        return complex(hi - 16 if hi >= 8 else hi, lo - 16 if lo >= 8 else lo)

    x = [[[dec(int(frame[t, f, n])) for n in range(N)] for f in range(F)] for t in range(T)]
    V = [[[0j] * N for _ in range(N)] for _ in range(F)]
    for f in range(F):
        for i in range(N):
            for j in range(N):
                s = 0j
                for t in range(T):
                    s += x[t][f][i] * x[t][f][j].conjugate()
                V[f][i][j] = s
    return V


def complex_samples(frame):
    """Decode bytes to complex int64 through integer arithmetic (independent of the oracle)."""
    b = frame.astype(np.int64)
    re = ((b >> 4) ^ 8) - 8
    im = ((b & 15) ^ 8) - 8
    return re, im


def unpack_triangle(vis, N):
    """[F][P][2] packed -> complex full upper triangle [F][N][N] (lower left zero), row-major walk."""
    F = vis.shape[0]
    out = np.zeros((F, N, N), dtype=np.complex128)
    p = 0
    for i in range(N):
        for j in range(i, N):
            out[:, i, j] = vis[:, p, 0] + 1j * vis[:, p, 1]
            p += 1
    return out


def assemble_by_definition(pkts, seq0, gps, N, F, T):
    """Assembly written out from its definition (Sec. II-A) with Python integers, one packet at a
    time in arrival order: header {u16 stream, u16 group, u32 reserved, u64 seq} little-endian, payload
    [4 t][8 channels][N]; a foreign stream or group is invalid, seq below the window late, at or past
    its end early; the first arrival of a (slot, group) is placed, later ones are duplicates; slots
    nothing filled stay zero and count 4 lost samples on each of the group's channels."""
    G, Q = F // 8, T // 4
    S = G // gps
    frame = np.zeros((T, F, N), np.uint8)
    filled = np.zeros((Q, G), np.uint8)
    stats = [0, 0, 0, 0, 0]                                          # ok, duplicate, late, early, invalid
    for rec in pkts:
        h = bytes(rec[:16])
        sid, grp = int.from_bytes(h[0:2], "little"), int.from_bytes(h[2:4], "little")
        seq = int.from_bytes(h[8:16], "little")
        if sid >= S or grp >= gps:
            stats[4] += 1
        elif seq < seq0:
            stats[2] += 1
        elif seq >= seq0 + Q:
            stats[3] += 1
        elif filled[seq - seq0, sid * gps + grp]:
            stats[1] += 1
        else:
            slot, g = seq - seq0, sid * gps + grp
            frame[4 * slot:4 * slot + 4, 8 * g:8 * g + 8, :] = np.asarray(rec[16:16 + 32 * N]).reshape(4, 8, N)
            filled[slot, g] = 1
            stats[0] += 1
    lost = np.zeros(F, np.uint32)
    for g in range(G):
        lost[8 * g:8 * g + 8] = 4 * (Q - int(filled[:, g].sum()))
    return frame, filled, lost, np.array(stats, np.uint32)


# ----------------------------------------------------------------------------- pins (take an oracle)

def pin_sample_decode(o):
    """Every byte decodes to the pair whose 4-bit two's complements re-pack to it; 0x88 = -8-8i."""
    seen = set()
    for b in range(256):
        re, im = o.sample(b)
        assert -8 <= re <= 7 and -8 <= im <= 7
        assert ((re & 15) << 4 | (im & 15)) == b
        seen.add((re, im))
    assert len(seen) == 256
    assert o.sample(0x88) == (-8, -8) and o.sample(0x7F) == (7, -1) and o.sample(0x10) == (1, 0)


def pin_pidx_bijection(o):
    for N in (1, 2, 5, 16, 33):
        p = [o.pidx(i, j, N) for i in range(N) for j in range(i, N)]
        assert p == list(range(N * (N + 1) // 2)) and o.npairs(N) == N * (N + 1) // 2


def pin_brute_force(o, seed=11):
    """Tiny random inputs (every byte value) against Python complex loops over the full square."""
    rng = np.random.default_rng(seed)
    for (N, F, T) in ((1, 1, 5), (3, 2, 17), (8, 2, 37)):
        fr = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
        fr[0, 0, 0] = 0x88
        vis, st = o.correlate(fr)
        assert st == oracle.OK
        V = brute_full(fr)
        full = unpack_triangle(vis, N)
        for f in range(F):
            for i in range(N):
                for j in range(i, N):
                    assert full[f, i, j] == V[f][i][j], (N, F, T, f, i, j)
                    assert V[f][j][i] == V[f][i][j].conjugate()          # Hermitian


def pin_library_gram(o, seed=12):
    """Mid-size inputs against numpy's int64 matrix product of the decoded samples."""
    fr = synth.uniform_frame(48, 3, 777, seed)
    vis, st = o.correlate(fr)
    assert st == oracle.OK
    re, im = complex_samples(fr)                  # [T][F][N]
    for f in range(3):
        a, b = re[:, f, :], im[:, f, :]
        Vre = a.T @ a + b.T @ b                   # sum_t a_i a_j + b_i b_j
        Vim = b.T @ a - a.T @ b                   # sum_t b_i a_j - a_i b_j
        iu = np.triu_indices(48)
        np.testing.assert_array_equal(vis[f, :, 0], Vre[iu])
        np.testing.assert_array_equal(vis[f, :, 1], Vim[iu])


def pin_pairs(o):
    """Selected pairs against Python complex brute force, and equal to the full triangle's entries."""
    rng = np.random.default_rng(17)
    fr = rng.integers(0, 256, (41, 3, 9), dtype=np.uint8)
    V = brute_full(fr)
    pairs = [(0, 0), (0, 8), (3, 5), (8, 8), (2, 7)]
    got = o.correlate_pairs(fr, 2, pairs)
    for (i, j), g in zip(pairs, got):
        assert complex(g[0], g[1]) == V[2][i][j]
    full, _ = o.correlate(synth.uniform_frame(32, 2, 300, 18))
    fr2 = synth.uniform_frame(32, 2, 300, 18)
    pr = [(i, j) for i in range(0, 32, 5) for j in range(i, 32, 7)]
    got = o.correlate_pairs(fr2, 1, pr)
    np.testing.assert_array_equal(got, full[1, [o.pidx(i, j, 32) for i, j in pr]])


def pin_subset_channels(o):
    fr = synth.uniform_frame(16, 6, 300, 13)
    full, _ = o.correlate(fr)
    part, _ = o.correlate(fr, 2, 3)
    np.testing.assert_array_equal(part, full[2:5])


def pin_autocorrelation(o):
    """Im V[i,i] = 0 and Re V[i,i] = sum |x_i|^2 >= 0."""
    fr = synth.signal_frame(32, 2, 512, 14)
    vis, _ = o.correlate(fr)
    re, im = complex_samples(fr)
    for i in range(32):
        p = o.pidx(i, i, 32)
        assert np.all(vis[:, p, 1] == 0)
        np.testing.assert_array_equal(vis[:, p, 0], (re[:, :, i] ** 2 + im[:, :, i] ** 2).sum(0))


def pin_constant_input(o):
    """x_n(t) = c_n for all t gives V = T c_i conj(c_j) exactly."""
    rng = np.random.default_rng(15)
    N, F, T = 10, 2, 999
    c = rng.integers(-8, 8, N) + 1j * rng.integers(-8, 8, N)
    c[0] = -8 - 8j
    c[1] = 3 - 5j
    fr = synth.constant_frame(c, F, T)
    vis, _ = o.correlate(fr)
    for i in range(N):
        for j in range(i, N):
            want = T * c[i] * np.conj(c[j])
            p = o.pidx(i, j, N)
            assert vis[0, p, 0] == want.real and vis[0, p, 1] == want.imag, (i, j)


def pin_single_source(o):
    """x_n(t) = g_n s(t) gives V = (sum_t |s(t)|^2) g_i conj(g_j)."""
    rng = np.random.default_rng(16)
    N, T = 12, 400
    g = rng.integers(-1, 2, N) + 1j * rng.integers(-1, 2, N)      # |Re, Im of g s| <= 6
    s = rng.integers(-2, 2, T) + 1j * rng.integers(-1, 2, T)
    x = s[:, None] * g[None, :]                   # components within [-8, 7]
    fr = synth.pack(x.real.astype(int), x.imag.astype(int)).reshape(T, 1, N)
    vis, _ = o.correlate(fr)
    S = int(np.sum(np.abs(s) ** 2))
    for i in range(N):
        for j in range(i, N):
            want = S * g[i] * np.conj(g[j])
            p = o.pidx(i, j, N)
            assert vis[0, p, 0] == want.real and vis[0, p, 1] == want.imag


def pin_overflow_bound(o):
    """All samples -8-8i: Re V[0,0] = 128 T. T = 2^24-1 is the last length that fits int32."""
    T = (1 << 24) - 1
    fr = np.full((T, 1, 2), 0x88, dtype=np.uint8)
    vis, st = o.correlate(fr)
    assert st == oracle.OK and vis[0, 0, 0] == 2147483520 and vis[0, 1, 0] == 2147483520
    assert vis[0, 1, 1] == 0
    fr = np.full((T + 1, 1, 1), 0x88, dtype=np.uint8)
    vis, st = o.correlate(fr)
    assert st == oracle.EOVERFLOW and vis[0, 0, 0] == 2147483648


def pin_assembly_basic(o):
    """Loss-free, in-order packets reproduce the frame; every stat is an ok packet."""
    N, F, T, gps = 16, 32, 64, 2
    fr = synth.uniform_frame(N, F, T, 21)
    pk = synth.packetize(fr, 1000, gps)
    out, filled, lost, stats = o.assemble(pk, 1000, gps, N, F, T)
    np.testing.assert_array_equal(out, fr)
    assert filled.all() and not lost.any()
    assert list(stats) == [pk.shape[0], 0, 0, 0, 0]


def pin_assembly_permutation(o):
    """A duplicate-free set of packets assembles the same frame in any arrival order."""
    N, F, T, gps = 16, 16, 64, 1
    fr = synth.uniform_frame(N, F, T, 22)
    pk = synth.packetize(fr, 7, gps)
    rng = np.random.default_rng(23)
    keep = rng.random(pk.shape[0]) > 0.1
    ref = o.assemble(pk[keep], 7, gps, N, F, T)
    for _ in range(3):
        perm = rng.permutation(np.flatnonzero(keep))
        got = o.assemble(pk[perm], 7, gps, N, F, T)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)


def pin_assembly_loss_and_dups(o):
    """Missing packets zero-filled, L = 4 x missing per channel; duplicates change nothing and the
    first arrival wins even when a later duplicate carries a different payload."""
    N, F, T, gps = 16, 16, 32, 2
    fr = synth.uniform_frame(N, F, T, 24)
    pk = synth.packetize(fr, 0, gps)
    n = pk.shape[0]
    drop = {3, 4, 9}
    order = [k for k in range(n) if k not in drop] + [5, 0]          # two byte-identical duplicates
    fake = pk[1].copy()
    fake[16:] = 0x77                                                 # a later duplicate that differs
    arr = np.concatenate([pk[order], fake[None]])
    out, filled, lost, stats = o.assemble(arr, 0, gps, N, F, T)
    assert list(stats) == [n - 3, 3, 0, 0, 0]
    G = F // 8
    want = fr.copy()
    want_lost = np.zeros(F, np.uint32)
    for k in drop:
        q, g = divmod(k, G)                                          # natural order: seq-major
        want[4 * q:4 * q + 4, 8 * g:8 * g + 8, :] = 0
        want_lost[8 * g:8 * g + 8] += 4
        assert filled[q, g] == 0
    np.testing.assert_array_equal(out, want)
    np.testing.assert_array_equal(lost, want_lost)
    assert filled.sum() == n - 3


def pin_assembly_window(o):
    """Packets before the window are late, at or after its end early, foreign stream/group invalid."""
    N, F, T, gps = 16, 16, 16, 1                                     # 2 streams x 1 group, Q = 4 slots
    fr = synth.uniform_frame(N, F, 3 * T, 25)
    pk = synth.packetize(fr, 100, gps)                               # k -> seq 100 + k//2, stream k%2
    bad = pk[8].copy()
    bad[0:2] = np.frombuffer(np.uint16(9).tobytes(), np.uint8)       # stream 9 does not exist
    bad2 = pk[9].copy()
    bad2[2:4] = np.frombuffer(np.uint16(1).tobytes(), np.uint8)      # group 1 >= gps
    arr = np.concatenate([pk[16:19], pk[0:5], bad[None], pk[8:14], bad2[None]])
    out, filled, lost, stats = o.assemble(arr, 104, gps, N, F, T)    # window seq 104..107
    assert list(stats) == [6, 0, 5, 3, 2]                            # ok, dup, late, early, invalid
    assert filled.sum() == 6 and not filled[3].any()
    np.testing.assert_array_equal(lost, np.full(F, 4, np.uint32))
    np.testing.assert_array_equal(out[:12], fr[16:28])
    assert not out[12:].any()


def pin_assembly_random_by_definition(o, cases=40):
    """Random packet sets assemble exactly as the definition written out packet by packet: valid,
    late, early, foreign-stream and foreign-group packets, and same-slot duplicates carrying different
    payloads, in random arrival order, with 64-bit sequence numbers."""
    rng = np.random.default_rng(26)
    for case in range(cases):
        N = int(rng.choice([16, 32]))
        gps, S, Q = int(rng.integers(1, 3)), int(rng.integers(1, 4)), int(rng.integers(1, 9))
        F, T = 8 * S * gps, 4 * Q
        seq0 = int(rng.integers(3, 1 << 40))
        n = int(rng.integers(0, 3 * Q * S * gps + 1))
        pk = synth.random_packet_set(260 + case, N, S, gps, Q, n, seq0)
        got = o.assemble(pk, seq0, gps, N, F, T)
        want = assemble_by_definition(pk, seq0, gps, N, F, T)
        for name, a, b in zip(("frame", "filled", "lost", "stats"), got, want):
            np.testing.assert_array_equal(a, b, err_msg=name)


def pin_counts_counters_equal_mask(o):
    """The paper's counter scheme (loss counter, per-input flag counts, pair intersections) gives the
    same per-visibility sample counts as brute force over the sample mask."""
    rng = np.random.default_rng(31)
    N, F, T = 9, 3, 200
    present = rng.random((T // 4, F)) > 0.15                         # per packet slot and channel
    present = np.repeat(present, 4, axis=0)                          # [T][F]
    flags = (rng.random((T, F, N)) < 0.08) & present[:, :, None]     # flags only on received data
    valid = present[:, :, None] & ~flags
    n_mask = o.counts_from_mask(valid.astype(np.uint8))
    lost = (T - present.sum(0)).astype(np.uint32)
    fc = flags.sum(0).astype(np.uint32)                              # [F][N]
    P = N * (N + 1) // 2
    fp = np.zeros((F, P), np.uint32)
    for f in range(F):
        p = 0
        for i in range(N):
            for j in range(i, N):
                fp[f, p] = np.sum(flags[:, f, i] & flags[:, f, j])
                p += 1
    n_cnt = o.counts_from_counters(T, lost, N, fc, fp)
    np.testing.assert_array_equal(n_cnt, n_mask)
    n_loss_only = o.counts_from_counters(T, lost, N)
    np.testing.assert_array_equal(n_loss_only, o.counts_from_mask(np.repeat(present[:, :, None], N, 2).astype(np.uint8)))


def pin_normalize(o):
    """No loss: V / T; n = 0 gives 0; values rounded once from the exact quotient."""
    fr = synth.signal_frame(8, 2, 100, 32)
    vis, _ = o.correlate(fr)
    n = np.full(vis.shape[:2], 100, np.uint32)
    out = o.normalize(vis, n)
    np.testing.assert_array_equal(out, (vis / 100.0).astype(np.float32))
    n[1, 3] = 0
    out = o.normalize(vis, n)
    assert out[1, 3, 0] == 0 and out[1, 3, 1] == 0
    v = np.array([[[2147483520, -7]]], np.int64)
    got = o.normalize(v, np.array([[3]], np.uint32))
    assert got[0, 0, 0] == np.float32(2147483520 / 3) and got[0, 0, 1] == np.float32(-7 / 3)


def pin_table1_geometry(o):
    """Table I / Sec. II-A figures: 8 KiB payload per packet, the link/host/system rates, packet rates,
    the ~9 kB wire packet, and the output size per 10 s integration (which pins the packed upper
    triangle *including* the diagonal at 8 bytes per visibility)."""
    g = json.load(open(os.path.join(GOLDEN, "table1.json")))
    N = g["n_inputs"]
    fs = g["band_mhz"] * 1e6 / g["channels_total"]                    # 390,625 samples/s/channel
    assert g["bytes_per_frequency_per_sample"] == N                   # one byte per 4+4-bit sample
    assert g["bytes_per_packet_sample_block"] == g["channels_per_link"] * N
    payload = synth.payload_bytes(N)
    assert payload == g["time_samples_per_packet"] * g["bytes_per_packet_sample_block"] == 8192
    link = g["channels_per_link"] * N * 8 * fs
    assert round(link / 1e9, 2) == g["sky_gbps"]["link"]
    assert round(link * g["links_per_server"] / 1e9, 1) == g["sky_gbps"]["host"]
    assert round(link * g["links_per_server"] * g["servers"] / 1e9, 1) == g["sky_gbps"]["system"]
    pps = link / 8 / payload
    assert pps * g["links_per_server"] == g["packets_per_second"]["host"]
    assert pps * g["links_per_server"] * g["servers"] == g["packets_per_second"]["system"]
    assert abs(pps - g["packets_per_second"]["link_as_printed"]) < 100   # printed value is a typo
    wire = g["sky_plus_headers_gbps"]["link"] * 1e9 / 8 / pps
    assert 9000 < wire < 9800                                          # "each UDP packet is ~9K"
    host_ch = g["channels_total"] // g["servers"]
    out_host = host_ch * o.npairs(N) * 8
    out_sys = g["channels_total"] * o.npairs(N) * 8
    assert out_host == 16_842_752 and out_sys == 269_484_032
    assert round(out_host / 1e6, 1) == g["output_per_10s"]["host"]
    assert round(out_sys / 1e6, 1) == g["output_per_10s"]["system"]


def _brute_flag_counts(flags):
    T, F, N = flags.shape
    c = flags.sum(0).astype(np.uint32)
    iu = np.triu_indices(N)
    x = np.stack([(flags[:, f, :, None] & flags[:, f, None, :]).sum(0)[iu] for f in range(F)]).astype(np.uint32)
    return c, x


def pin_flag_footer_layout(o):
    """Footer reading (Sec. II-C flags as packet bit fields): one flagged sample (t=6, f=11, n=13)
    sets exactly bit 13 % 8 of byte 13 / 8 of row (t % 4) * 8 + f % 8 of the footer of slot t / 4,
    group f / 8, and counts once for input 13 and once for the pair (13, 13). With the footer a
    packet is 16 + 36N bytes: 9,232 B at N = 256, the paper's ~9 kB packet."""
    N, F, T = 16, 16, 16
    fl = np.zeros((T, F, N), bool)
    fl[6, 11, 13] = True
    pk = synth.packetize(synth.uniform_frame(N, F, T, 3), 0, 1, fl)
    assert pk.shape[1] == 16 + 36 * N and 16 + 36 * 256 == 9232
    k = 1 * 2 + 1                                                    # slot 1, group 1 (2 groups)
    foot = pk[:, 16 + 32 * N:]
    row = (6 % 4) * 8 + 11 % 8
    assert foot[k, row * (N // 8) + 13 // 8] == 1 << (13 % 8) and foot.sum() == foot[k].sum() == 1 << (13 % 8)
    assert pk[k, 16 + row * N + 13] == 0                              # the flagged sample is zero in the data
    c, x = o.flag_counts(pk, 0, 1, N, F, T)
    assert c.sum() == 1 and c[11, 13] == 1
    assert x.sum() == 1 and x[11, o.pidx(13, 13, N)] == 1


def pin_flag_counts_brute_force(o):
    """Flag counts of a frame delivered with loss, reordering and duplicates equal the per-input
    sums and pair intersections of the flags of the samples that arrived (lost slots flag
    nothing), counted directly from the flag array."""
    N, F, T, gps = 24, 16, 64, 2
    fr = synth.signal_frame(N, F, T, 33)
    fl = synth.random_flags(T, F, N, 34, p_sample=0.03, p_burst=0.1, p_all=0.02)
    pk = synth.packet_stream(fr, 0, gps, 35, p_drop=0.1, p_reorder=0.2, p_dup=0.1, flags=fl)
    _, filled, _, _ = o.assemble(pk, 0, gps, N, F, T)
    present = np.repeat(np.repeat(filled.astype(bool), 4, axis=0), 8, axis=1)     # [T][F]
    c, x = o.flag_counts(pk, 0, gps, N, F, T)
    bc, bx = _brute_flag_counts(fl & present[:, :, None])
    np.testing.assert_array_equal(c, bc)
    np.testing.assert_array_equal(x, bx)
    assert c.sum() > 0 and (x.sum() > c.sum())                       # some pairs flagged together


def pin_flag_counts_give_mask_counts(o):
    """Sec. II-C end to end: loss counters from the assembly and flag counters from the footers,
    combined by the counter scheme, give the brute-force count of samples valid for both inputs."""
    N, F, T, gps = 16, 8, 128, 1
    fr = synth.signal_frame(N, F, T, 36)
    fl = synth.random_flags(T, F, N, 37, p_sample=0.02, p_burst=0.05, p_all=0.01)
    pk = synth.packet_stream(fr, 0, gps, 38, p_drop=0.05, p_reorder=0.1, flags=fl)
    _, filled, lost, _ = o.assemble(pk, 0, gps, N, F, T)
    c, x = o.flag_counts(pk, 0, gps, N, F, T)
    present = np.repeat(np.repeat(filled.astype(bool), 4, axis=0), 8, axis=1)
    valid = present[:, :, None] & ~fl
    np.testing.assert_array_equal(o.counts_from_counters(T, lost, N, c, x), o.counts_from_mask(valid.astype(np.uint8)))


def pin_time_shift_brute_force(o, seed=40):
    """Time shift (reading of the Fig. 4 stage): each output byte by its definition written out in
    Python; zero delays are the identity; the delay is a shift towards later samples."""
    rng = np.random.default_rng(seed)
    T, F, N = 37, 3, 16
    fr = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    d = rng.integers(0, T + 1, N)
    d[0], d[1] = 0, T
    got = o.time_shift(fr, d)
    want = np.zeros_like(fr)
    for t in range(T):
        for f in range(F):
            for n in range(N):
                if t >= d[n]:
                    want[t, f, n] = fr[t - d[n], f, n]
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(o.time_shift(fr, np.zeros(N, int)), fr)
    one = o.time_shift(fr, np.ones(N, int))
    np.testing.assert_array_equal(one[1:], fr[:-1])
    assert not one[0].any()


def pin_time_shift_constant_input(o):
    """A constant input shifted by d_n correlates to (T - max(d_i, d_j)) c_i conj(c_j) exactly."""
    rng = np.random.default_rng(41)
    N, F, T = 16, 2, 300
    c = rng.integers(-8, 8, N) + 1j * rng.integers(-8, 8, N)
    d = rng.integers(0, 120, N)
    v, st = o.correlate(o.time_shift(synth.constant_frame(c, F, T), d))
    assert st == oracle.OK
    for i in range(N):
        for j in range(i, N):
            want = (T - max(d[i], d[j])) * c[i] * np.conj(c[j])
            p = o.pidx(i, j, N)
            assert v[0, p, 0] == want.real and v[0, p, 1] == want.imag, (i, j)


def pin_time_shift_aligns_delayed_source(o):
    """The stage's purpose: a common signal s arriving at input n tau_n samples late
    (x_n(t) = g_n s(t - tau_n)) is re-aligned by delays d_n = D - tau_n (D = max tau): every input
    then carries g_n s(t - D), and V[i,j] = g_i conj(g_j) sum over t >= max(d_i, d_j) of |s(t - D)|^2."""
    rng = np.random.default_rng(42)
    N, T, D = 16, 400, 40
    tau = rng.integers(0, D + 1, N)
    tau[0] = D
    g = rng.integers(-1, 2, N) + 1j * rng.integers(-1, 2, N)      # |Re, Im of g s| <= 6
    s_t = rng.integers(-3, 4, T + D) + 1j * rng.integers(-3, 4, T + D)   # s(t) for t = -D .. T - 1
    x = np.stack([g[n] * s_t[D - tau[n]:D - tau[n] + T] for n in range(N)], axis=1)   # [T][N]
    fr = synth.pack(x.real.astype(np.int64), x.imag.astype(np.int64))[:, None, :]
    d = D - tau
    v, st = o.correlate(o.time_shift(fr, d))
    assert st == oracle.OK
    for i in range(N):
        for j in range(i, N):
            t0 = max(d[i], d[j])
            seg = s_t[t0:T]                                             # s(t - D) at t = t0 .. T - 1
            power = int(np.sum(seg.real.astype(np.int64) ** 2 + seg.imag.astype(np.int64) ** 2))
            want = g[i] * np.conj(g[j]) * power
            p = o.pidx(i, j, N)
            assert v[0, p, 0] == want.real and v[0, p, 1] == want.imag, (i, j)


def pin_time_shift_counts_give_mask_counts(o):
    """The shift's counters (c += d_n, x += min(d_i, d_j)), combined by the counter scheme with a
    channel's loss counter, give the brute-force count of samples valid for both inputs."""
    rng = np.random.default_rng(43)
    N, F, T = 16, 8, 96
    d = rng.integers(0, T + 1, N)
    lost = np.zeros(F, np.uint32)
    c, x = o.time_shift_counts(d, N, F)
    valid = (np.arange(T)[:, None, None] >= d[None, None, :]) & np.ones((T, F, N), bool)
    np.testing.assert_array_equal(o.counts_from_counters(T, lost, N, c, x), o.counts_from_mask(valid.astype(np.uint8)))
    c2, x2 = o.time_shift_counts(d, N, F, c.copy(), x.copy())      # the counters add up
    np.testing.assert_array_equal(c2, 2 * c)
    np.testing.assert_array_equal(x2, 2 * x)


PINS = [pin_sample_decode, pin_pidx_bijection, pin_brute_force, pin_pairs, pin_library_gram, pin_subset_channels,
        pin_autocorrelation, pin_constant_input, pin_single_source, pin_overflow_bound,
        pin_assembly_basic, pin_assembly_permutation, pin_assembly_loss_and_dups, pin_assembly_window,
        pin_assembly_random_by_definition,
        pin_counts_counters_equal_mask, pin_normalize, pin_table1_geometry, pin_flag_footer_layout,
        pin_flag_counts_brute_force, pin_flag_counts_give_mask_counts,
        pin_time_shift_brute_force, pin_time_shift_constant_input, pin_time_shift_aligns_delayed_source,
        pin_time_shift_counts_give_mask_counts]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin(oracle.default())
