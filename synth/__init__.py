"""Seeded synthetic inputs for the 4+4-bit X-engine.

This module is shared by the CPU oracle tests and by the CUDA-path tests and benchmark. It holds
none of the correlator's arithmetic: only random sample draws, the 4+4-bit packing of a quantised
complex value into one byte, and the UDP packet framing the F-engine would emit.

Sample format (one byte per complex sample): high nibble = real part, low nibble = imaginary part,
each a 4-bit two's-complement integer in [-8, 7] ("4+4-bit complex numbers", Sec. I).

Frame layout: ``uint8 [T][F][N]`` -- time-major, then frequency channel, then input, which is the
order in which the packets' data sections are concatenated (Sec. II-A: the data section "can be used
by the GPU without modification").

Packet layout (Fig. 3 is not legible in the paper; this is the reading used throughout): a 16-byte
little-endian header ``{u16 stream_id; u16 chan_group; u32 reserved; u64 seq}`` followed by a
payload of 4 time samples x 8 channels x N inputs, ``[t(4)][f(8)][n(N)]`` (Sec. II-A: 256 B per
frequency, 2 KB for 8 bands, 4 time samples per packet). ``seq`` counts packets, i.e. units of
4 time samples, and is array-synchronised.

Everything here draws from explicit seeds so that a test and the oracle see identical bytes.
"""
from __future__ import annotations

import math

import numpy as np

HEADER_BYTES = 16
SAMPLES_PER_PACKET = 4     # time samples per packet (Sec. II-A)
CHANNELS_PER_GROUP = 8     # frequency bands per packet (Sec. II-A)


def payload_bytes(n_inputs: int) -> int:
    return SAMPLES_PER_PACKET * CHANNELS_PER_GROUP * n_inputs


def packet_stride(n_inputs: int) -> int:
    return HEADER_BYTES + payload_bytes(n_inputs)


# ----------------------------------------------------------------------------- packing

def pack(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack integer re, im in [-8, 7] into 4+4-bit two's-complement bytes (high = re)."""
    re = np.asarray(re, dtype=np.int64)
    im = np.asarray(im, dtype=np.int64)
    if re.size and (re.min() < -8 or re.max() > 7 or im.min() < -8 or im.max() > 7):
        raise ValueError("4-bit components must lie in [-8, 7]")
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)


def _round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def _quantise(z: np.ndarray) -> np.ndarray:
    re = np.clip(_round_half_away(z.real), -8, 7)
    im = np.clip(_round_half_away(z.imag), -8, 7)
    return pack(re, im)


# ----------------------------------------------------------------------------- frames (host)

def uniform_frame(n_inputs: int, n_chan: int, n_time: int, seed: int) -> np.ndarray:
    """i.i.d. uniform nibbles on [-8, 7]: every byte value 0..255 equally likely. [T][F][N] u8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 256, size=(n_time, n_chan, n_inputs), dtype=np.uint8)


def signal_frame(n_inputs: int, n_chan: int, n_time: int, seed: int, sigma: float = 2.5,
                 n_src: int = 3, amp: float = 0.3) -> np.ndarray:
    """Gaussian noise plus common point sources, quantised to 4+4 bits. [T][F][N] u8.

    Per channel f, input n and sample t:
        x = w + sum_k amp*sigma * s_k(t) * exp(i*phi_{f,k,n})
    with w complex Gaussian (each component N(0, sigma^2)), s_k(t) a unit-power complex Gaussian
    common to all inputs, phi uniform on [0, 2pi) per (channel, source, input). Components are
    rounded half away from zero and clipped to [-8, 7].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n_time, n_chan, n_inputs), dtype=np.uint8)
    for f in range(n_chan):
        w = rng.normal(0.0, sigma, (n_time, n_inputs)) + 1j * rng.normal(0.0, sigma, (n_time, n_inputs))
        phi = rng.uniform(0.0, 2.0 * math.pi, (n_src, n_inputs))
        s = (rng.normal(0.0, math.sqrt(0.5), (n_time, n_src))
             + 1j * rng.normal(0.0, math.sqrt(0.5), (n_time, n_src)))
        x = w + (amp * sigma) * (s @ np.exp(1j * phi))
        out[:, f, :] = _quantise(x)
    return out


def constant_frame(values: np.ndarray, n_chan: int, n_time: int) -> np.ndarray:
    """x_n(t) = values[n] for every t and channel. values: complex ints in [-8, 7]."""
    v = np.asarray(values)
    row = pack(v.real.astype(np.int64), v.imag.astype(np.int64))
    return np.broadcast_to(row, (n_time, n_chan, row.size)).copy()


# ----------------------------------------------------------------------------- frames (torch)

def signal_frame_torch(n_inputs: int, n_chan: int, n_time: int, seed: int, device="cpu",
                       sigma: float = 2.5, n_src: int = 3, amp: float = 0.3, chunk: int = 64):
    """Same signal model as :func:`signal_frame`, drawn with torch's generator on ``device``.

    Used for the large (GiB-sized) workloads, which are generated directly in device memory. The
    byte stream differs from the numpy generator's; each test feeds the same bytes to both sides.
    Returns a uint8 tensor [T][F][N].
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((n_time, n_chan, n_inputs), dtype=torch.uint8, device=device)
    for f0 in range(0, n_chan, chunk):
        fc = min(chunk, n_chan - f0)
        w_re = torch.randn((n_time, fc, n_inputs), generator=g, device=device) * sigma
        w_im = torch.randn((n_time, fc, n_inputs), generator=g, device=device) * sigma
        phi = torch.rand((fc, n_src, n_inputs), generator=g, device=device) * (2.0 * math.pi)
        s_re = torch.randn((n_time, fc, n_src), generator=g, device=device) * math.sqrt(0.5)
        s_im = torch.randn((n_time, fc, n_src), generator=g, device=device) * math.sqrt(0.5)
        c, sn = torch.cos(phi), torch.sin(phi)
        # (s_re + i s_im)(c + i sn) summed over sources
        x_re = w_re + (amp * sigma) * (torch.einsum("tfk,fkn->tfn", s_re, c) - torch.einsum("tfk,fkn->tfn", s_im, sn))
        x_im = w_im + (amp * sigma) * (torch.einsum("tfk,fkn->tfn", s_re, sn) + torch.einsum("tfk,fkn->tfn", s_im, c))
        q_re = (torch.sign(x_re) * torch.floor(x_re.abs() + 0.5)).clamp_(-8, 7).to(torch.int32)
        q_im = (torch.sign(x_im) * torch.floor(x_im.abs() + 0.5)).clamp_(-8, 7).to(torch.int32)
        out[:, f0:f0 + fc, :] = (((q_re & 0xF) << 4) | (q_im & 0xF)).to(torch.uint8)
        del w_re, w_im, s_re, s_im, x_re, x_im, q_re, q_im
    return out


def uniform_frame_torch(n_inputs: int, n_chan: int, n_time: int, seed: int, device="cpu"):
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randint(0, 256, (n_time, n_chan, n_inputs), generator=g, device=device,
                         dtype=torch.int32).to(torch.uint8)


# ----------------------------------------------------------------------------- packets

def make_header(stream_id: int, chan_group: int, seq: int) -> np.ndarray:
    h = np.zeros(HEADER_BYTES, dtype=np.uint8)
    h[0:2] = np.frombuffer(np.uint16(stream_id).tobytes(), np.uint8)
    h[2:4] = np.frombuffer(np.uint16(chan_group).tobytes(), np.uint8)
    h[8:16] = np.frombuffer(np.uint64(seq).tobytes(), np.uint8)
    return h


def footer_bytes(n_inputs: int) -> int:
    """Flag footer of a packet: one bit per (sample, channel, input) = 4 x 8 x N bits."""
    return 4 * CHANNELS_PER_GROUP * n_inputs // 8


def packetize(frame: np.ndarray, seq0: int, groups_per_stream: int, flags: np.ndarray | None = None) -> np.ndarray:
    """Split a frame [T][F][N] into packets, in natural send order (seq, then stream, then group).

    Channel group G = stream_id * groups_per_stream + chan_group covers channels [8G, 8G+8).
    Returns uint8 [n_packets][16 + 32N]. With `flags` (bool [T][F][N], the F-engine's flags) the
    flagged samples are zeroed in the payload and each packet carries a footer of 4N bytes after
    it: [4 t][8 f][N/8], bit n % 8 of byte n / 8 set for a flagged input n; records are then
    16 + 36N bytes.
    """
    if flags is not None:
        flags = np.asarray(flags, dtype=bool)
        if flags.shape != frame.shape:
            raise ValueError("flags must have the frame's shape")
        frame = np.where(flags, np.uint8(0), frame)
    T, F, N = frame.shape
    G = F // CHANNELS_PER_GROUP
    if T % SAMPLES_PER_PACKET or F % CHANNELS_PER_GROUP or G % groups_per_stream:
        raise ValueError("frame shape incompatible with packet geometry")
    n_streams = G // groups_per_stream
    Q = T // SAMPLES_PER_PACKET
    pay = frame.reshape(Q, SAMPLES_PER_PACKET, n_streams, groups_per_stream, CHANNELS_PER_GROUP, N)
    pay = pay.transpose(0, 2, 3, 1, 4, 5).reshape(Q * G, payload_bytes(N))
    hdr = np.zeros((Q, n_streams, groups_per_stream, HEADER_BYTES), dtype=np.uint8)
    sid = np.arange(n_streams, dtype=np.uint16)[None, :, None]
    grp = np.arange(groups_per_stream, dtype=np.uint16)[None, None, :]
    seq = (np.uint64(seq0) + np.arange(Q, dtype=np.uint64))[:, None, None]
    hdr[..., 0:2] = np.broadcast_to(sid, (Q, n_streams, groups_per_stream)).astype("<u2")[..., None].view(np.uint8)
    hdr[..., 2:4] = np.broadcast_to(grp, (Q, n_streams, groups_per_stream)).astype("<u2")[..., None].view(np.uint8)
    hdr[..., 8:16] = np.broadcast_to(seq, (Q, n_streams, groups_per_stream)).astype("<u8")[..., None].view(np.uint8)
    parts = [hdr.reshape(Q * G, HEADER_BYTES), pay]
    if flags is not None:
        fl = flags.reshape(Q, SAMPLES_PER_PACKET, n_streams, groups_per_stream, CHANNELS_PER_GROUP, N)
        fl = fl.transpose(0, 2, 3, 1, 4, 5).reshape(Q * G, SAMPLES_PER_PACKET * CHANNELS_PER_GROUP, N)
        parts.append(np.packbits(fl, axis=2, bitorder="little").reshape(Q * G, footer_bytes(N)))
    return np.concatenate(parts, axis=1)


def network_order(n_packets: int, seed: int, p_drop: float = 0.0, p_reorder: float = 0.0,
                  p_dup: float = 0.0, max_disp: int = 64) -> np.ndarray:
    """Arrival order of packets sent in order 0..n-1 over a lossy UDP link.

    Each packet is independently dropped (p_drop), delayed by a uniform displacement in
    [1, max_disp] positions (p_reorder), and/or duplicated with the copy arriving up to max_disp
    positions later (p_dup). Returns the int64 indices of the arriving packets in arrival order.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.arange(n_packets, dtype=np.int64)
    key = idx.astype(np.float64)
    keep = rng.random(n_packets) >= p_drop
    moved = rng.random(n_packets) < p_reorder
    key = key + np.where(moved, rng.integers(1, max_disp + 1, n_packets) + 0.5, 0.0)
    dup = (rng.random(n_packets) < p_dup) & keep
    dkey = idx[dup] + rng.integers(1, max_disp + 1, int(dup.sum())) + 0.25
    all_idx = np.concatenate([idx[keep], idx[dup]])
    all_key = np.concatenate([key[keep], dkey])
    return all_idx[np.argsort(all_key, kind="stable")]


def packet_stream(frame: np.ndarray, seq0: int, groups_per_stream: int, seed: int,
                  p_drop: float = 0.0, p_reorder: float = 0.0, p_dup: float = 0.0,
                  max_disp: int = 64, flags: np.ndarray | None = None) -> np.ndarray:
    """Packets of ``frame`` as they arrive: natural send order perturbed by :func:`network_order`."""
    pk = packetize(frame, seq0, groups_per_stream, flags)
    order = network_order(pk.shape[0], seed, p_drop, p_reorder, p_dup, max_disp)
    return np.ascontiguousarray(pk[order])


def random_packet_set(seed: int, n_inputs: int, n_streams: int, groups_per_stream: int, n_slots: int,
                      n_packets: int, seq0: int) -> np.ndarray:
    """Packets with random headers and random payloads, in random arrival order: mostly valid
    (stream < n_streams, group < groups_per_stream, seq in [seq0, seq0 + n_slots)), some late
    (seq0 - 3 .. seq0 - 1) or early (up to seq0 + n_slots + 2), about 10 % from foreign streams (up to
    65535) and 5 % with a foreign group. Slots drawn twice become duplicates with different payloads.
    uint8 [n_packets][16 + 32 N]; requires seq0 >= 3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pk = np.zeros((n_packets, packet_stride(n_inputs)), dtype=np.uint8)
    for k in range(n_packets):
        sid = int(rng.integers(0, n_streams + 1)) if rng.random() < 0.9 else int(rng.integers(n_streams, 1 << 16))
        grp = int(rng.integers(0, groups_per_stream)) if rng.random() < 0.95 else groups_per_stream
        pk[k, :HEADER_BYTES] = make_header(sid, grp, seq0 + int(rng.integers(-3, n_slots + 3)))
        pk[k, HEADER_BYTES:] = rng.integers(0, 256, payload_bytes(n_inputs), dtype=np.uint8)
    return pk


def packetize_torch(frame, seq0: int, groups_per_stream: int):
    """Torch twin of :func:`packetize` (runs where ``frame`` lives). Returns uint8 [n][16+32N]."""
    import torch

    T, F, N = frame.shape
    G = F // CHANNELS_PER_GROUP
    if T % SAMPLES_PER_PACKET or F % CHANNELS_PER_GROUP or G % groups_per_stream:
        raise ValueError("frame shape incompatible with packet geometry")
    S = G // groups_per_stream
    Q = T // SAMPLES_PER_PACKET
    out = torch.empty((Q * G, packet_stride(N)), dtype=torch.uint8, device=frame.device)
    pay = frame.reshape(Q, SAMPLES_PER_PACKET, S, groups_per_stream, CHANNELS_PER_GROUP, N)
    out[:, HEADER_BYTES:] = pay.permute(0, 2, 3, 1, 4, 5).reshape(Q * G, payload_bytes(N))
    if int(seq0) < 0 or int(seq0) + Q > 0x7FFFFFFF:
        raise ValueError("packetize_torch supports 0 <= seq < 2^31")
    hdr = torch.zeros((Q, S, groups_per_stream, 4), dtype=torch.int32, device=frame.device)
    sid = torch.arange(S, dtype=torch.int32, device=frame.device)[None, :, None]
    grp = torch.arange(groups_per_stream, dtype=torch.int32, device=frame.device)[None, None, :]
    seq = int(seq0) + torch.arange(Q, dtype=torch.int32, device=frame.device)[:, None, None]
    hdr[..., 0] = sid | (grp << 16)
    hdr[..., 2] = seq          # low 32 bits of the little-endian u64; high word stays 0
    out[:, :HEADER_BYTES] = hdr.reshape(Q * G, 4).view(torch.uint8).reshape(Q * G, HEADER_BYTES)
    return out


def random_flags(n_time: int, n_chan: int, n_inputs: int, seed: int, p_sample: float = 0.002,
                 p_burst: float = 0.02, p_all: float = 0.002) -> np.ndarray:
    """F-engine flags, bool [T][F][N] (seeded): isolated flagged samples (p_sample per sample),
    bursts on one input (an input of a channel flagged for 16 consecutive samples, p_burst per input
    and channel), and samples in which every input of a channel is flagged (p_all per sample and
    channel: the dense case of the pair intersections)."""
    rng = np.random.default_rng(seed)
    fl = rng.random((n_time, n_chan, n_inputs)) < p_sample
    bursts = np.argwhere(rng.random((n_chan, n_inputs)) < p_burst)
    for f, n in bursts:
        t0 = int(rng.integers(0, max(1, n_time - 16)))
        fl[t0:t0 + 16, f, n] = True
    fl |= (rng.random((n_time, n_chan)) < p_all)[:, :, None]
    return fl


def config4_shapes(seed: int = 4, n_jobs: int = 24):
    """The uneven batch of 24 jobs: N from {64, 128, 256, 512, 1024, 2048}, F from {16, 64, 256},
    T log-uniform in [1024, 32768] rounded to a multiple of 128 (seeded). Returns [(N, F, T)]."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(n_jobs):
        N = int(rng.choice([64, 128, 256, 512, 1024, 2048]))
        F = int(rng.choice([16, 64, 256]))
        T = int(np.exp(rng.uniform(np.log(1024), np.log(32768))))
        T = max(128, (T + 64) // 128 * 128)
        shapes.append((N, F, T))
    return shapes
