// xe_correlate.cu -- A2 unpack and A3/A4 correlation (tcgen05 tensor cores, exact integers).
//
// Method (Sec. I, Sec. II-B): for every channel f, V_f[i,j] = sum_t x_i(t) conj(x_j(t)), i <= j.
// With x = a + ib and the real matrix Y_f whose row 2n is a_n(t) and row 2n+1 is b_n(t), the Gram
// matrix G = Y Y^T holds every real product sum, and
//     Re V[i,j] = G[2i,2j] + G[2i+1,2j+1],     Im V[i,j] = G[2i+1,2j] - G[2i,2j+1].
// G is computed on the tensor cores with tcgen05.mma kind::f8f6f4: the 4-bit integers are exact as
// FP8 E5M2 (the MN-major engines carry 16*a instead of a, also exact), their products and every
// partial sum below 2^24 (in units of the operand scales) are exact in the FP32 accumulator held in
// tensor memory, and the accumulator is drained to int32 at least every k_flush samples. Only
// 128x128 tiles of G on or above the block diagonal are computed.
//
// Single-CTA engines (one kernel template, one persistent CTA per SM):
//   UNPACKED_K  A2 unpack writes Y K-major [F][R][ldy]; TMA loads 128x128-byte swizzled tiles.
//   UNPACKED    A2 unpack writes Y MN-major [F][ldy][R] (an in-order byte expansion of the frame);
//               TMA loads 128 (t) x 128-byte tiles; MMAs read MN-major operands.
//   FUSED       no unpack: TMA loads packed [128 t][64 n] byte tiles of the frame and converter
//               warps expand them in shared memory into the MN-major operand layout.
// Roles: warp 0 = scheduler + TMA producer, warp 1 = TMEM owner + MMA issuer (one thread),
// warps 2..9 = epilogue (tcgen05.ld, FP32 -> int32, 2x2 Re/Im combine by shfl.xor, store or
// accumulate into the packed triangle), warps 10..17 = converters (FUSED only).
// Work items (job, channel, strip) are handed out dynamically (one atomic per item), channel by
// channel, so that the strips of a channel run together and share its data in L2.
// The default engine, FUSED_PAIR (correlate_pair_kernel, below), runs on CTA pairs with M = 256
// pair MMAs, converters loading samples straight into registers, from an assembled frame (frame
// mode) or from the packets through their index (packet mode, xe_correlate_packets). The legacy
// mma.sync baseline engine is in xe_legacy.cu.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "xe_device.cuh"
#include "xe_internal.h"

namespace xe {
namespace corr {

constexpr int kBlk = 128;                    // rows per operand block = MMA M
constexpr int kKtMax = 128;                  // time samples per pipeline stage (K-major engine)
constexpr int kKtMN = 128;                   // time samples per pipeline stage (MN-major engines)
constexpr int kPairKtFrame = 256;            // time samples per pipeline stage of the pair engine:
constexpr int kPairKtPackets = 128;          //   frame mode / packet mode
constexpr int kTmemCols = 512;
constexpr int kItemRing = 4;
constexpr int kSmemMax = 232448;             // 227 KiB opt-in limit per block
// TMEM drain interval: with at most 2^15 samples per drain every accumulated value, and every sum
// the epilogue forms from two of them, stays below 2^22 in magnitude (after the operand scales are
// removed), so FP32 holds them exactly and the 1.5 * 2^23 rounding trick converts them to int32.
constexpr int kDefaultKFlush = 1 << 15;
constexpr int kMaxKFlush = 1 << 15;
constexpr int kConvWarps = 8;

enum Engine { kUnpackedK = 0, kUnpackedMN = 1, kFusedMN = 2, kFusedPair = 3, kLegacyS4 = 4, kLegacyS8 = 5 };

struct Job {                 // 128-byte aligned through its CUtensorMap
    CUtensorMap tmap;        // operand map (unpacked engines) or packed frame map (fused)
    int32_t *vis;
    const uint8_t *frame;    // packed frame [T][F][N] (pair engine loads it directly)
    const uint8_t *pkts;     // packet mode: packets (16-byte header, payload [4 t][8 channels][N])
    const uint32_t *owner;   // packet mode: [F / 8][T / 4] packet of each (group, slot), ~0u = lost
    uint32_t pkt_stride;     // packet mode: bytes from one packet to the next
    int32_t n_inputs, n_chan, n_time, accumulate;
    int32_t nb;              // 128-row operand blocks (R / 128)
    int32_t strips;          // work items per channel (pair engine, packet mode: per channel pair)
    int32_t k_tiles;         // ceil(T / samples per stage)
    int32_t k_tiles_wide;    // packet mode: ceil(T / (2 x samples per stage)) (wide stages); else k_tiles
    int32_t item_begin;      // first global work-item index of this job
    int32_t pw;              // fused: bytes per packed row in shared memory (min(64, N))
    int32_t max_strip;       // tiles per work item along a row (1..4) for this job
    int32_t doubles;         // pair engine: double items per channel (0: every block a single item)
    int32_t offdiag;         // pair engine, packet mode: blocks (R, C >= R + 2) per channel
    int32_t twin;            // pair engine: 1 = packet-mode item layout (doubles, singles, twins)
    int32_t fold;            // pair engine, packet mode: 1 = fold layout (see decode_pair_item)
};

struct Params {
    Job jobs[XE_MAX_JOBS];
    int32_t n_jobs, n_items, k_flush_tiles;
    int32_t k_flush_tiles_wide;   // drain interval in wide stages (packet mode), else k_flush_tiles
    int32_t wide_diag;            // 1: single diagonal items run in wide stages (packet mode)
    int32_t op_stages, pk_stages, slots, n_acc;
    int32_t fold;                 // some job has the fold layout: three operand slots, transpose staging
    int32_t frame_rows;           // 128-sample kernel reading assembled frames (no owner tables)
    // balanced split (one job of fold items, one per channel): pair q takes stages
    // [q split_u, (q + 1) split_u) of the job's channel-major F x k_tiles stages, as up to
    // split_items items (pieces of consecutive channels); 0 = off
    int32_t split_u, split_pairs, split_items;
    // time-shifted packet calls (the kShift kernel, one job): the delay in samples of each block of
    // 16 inputs (inputs 16 b .. 16 b + 15 share delay16[b]); sample t of input n is read from row
    // t - delay16[n / 16] of the frame, zero before the frame's start
    int32_t delay16[XE_MAX_INPUTS / 16];
    int *status;
    int *counter;            // work-item counter, zero at launch
    uint64_t limit_ns;
};

// ----------------------------------------------------------------------------- work items
// A strip is a run of up to max_strip tiles along one block row rb, starting at column block
// cb0 >= rb. The diagonal strip of row rb starts at cb0 = rb (its A operand is its own first B
// block); further strips hold at most min(max_strip, 3) tiles so A plus the B blocks fit 4 slots.

__host__ __device__ inline int strips_in_row(int nb, int rb, int ms) {
    const int wd = min(ms, nb - rb);
    const int wo = min(ms, 3);
    const int rest = nb - rb - wd;
    return 1 + (rest + wo - 1) / wo;
}

__host__ __device__ inline int strips_per_channel(int nb, int ms) {
    int s = 0;
    for (int rb = 0; rb < nb; ++rb) s += strips_in_row(nb, rb, ms);
    return s;
}

__host__ __device__ inline void decode_strip(int s, int nb, int ms, int &rb, int &cb0, int &w) {
    for (rb = 0; rb < nb; ++rb) {
        const int n = strips_in_row(nb, rb, ms);
        if (s < n) {
            const int wd = min(ms, nb - rb);
            if (s == 0) {
                cb0 = rb;
                w = wd;
            } else {
                const int wo = min(ms, 3);
                cb0 = rb + wd + (s - 1) * wo;
                w = min(wo, nb - cb0);
            }
            return;
        }
        s -= n;
    }
    rb = cb0 = w = 0;
}

struct Item {
    int job, f, rb, cb0, w;
    int nblk;      // operand blocks per stage: the w B blocks, plus A when it is not among them
    int a_slot;    // stage slot holding the A block
};

// Operand block held in stage slot b: the B blocks cb0.. first, then A (off-diagonal strips).
__device__ __forceinline__ int block_of(const Item &it, int b) { return b < it.w ? it.cb0 + b : it.rb; }

// Channel-major order: all strips of one channel are consecutive item indices.
__device__ __forceinline__ Item decode_item(const Params &p, int g) {
    Item it;
    int j = 0;
    while (j + 1 < p.n_jobs && g >= p.jobs[j + 1].item_begin) ++j;
    const Job &jb = p.jobs[j];
    const int l = g - jb.item_begin;
    it.job = j;
    it.f = l / jb.strips;
    decode_strip(l % jb.strips, jb.nb, jb.max_strip, it.rb, it.cb0, it.w);
    const bool off_diag = it.rb < it.cb0;
    it.nblk = it.w + (off_diag ? 1 : 0);
    it.a_slot = off_diag ? it.w : 0;
    return it;
}

// ----------------------------------------------------------------------------- A2 unpack kernels

// K-major: grid (ldy/128, R/128, F), 256 threads; a 128-sample x 64-input byte tile is staged in
// shared memory and written as 128 rows (2n = Re, 2n+1 = Im) of 128 E5M2 codes (unscaled).
__global__ void __launch_bounds__(256) unpack_k_kernel(const uint8_t *__restrict__ frame, uint8_t *__restrict__ y,
                                                       int N, int F, int T, int R, int64_t ldy) {
    __shared__ uint32_t tile[128][17];
    const int t0 = blockIdx.x * 128;
    const int n0 = blockIdx.y * 64;
    const int f = blockIdx.z;
    for (int k = threadIdx.x; k < 512; k += 256) {
        const int tt = k >> 2, c = k & 3;
        const int t = t0 + tt, n = n0 + c * 16;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (t < T && n < N) v = __ldcs(reinterpret_cast<const uint4 *>(frame + ((size_t)t * F + f) * N + n));
        tile[tt][c * 4 + 0] = v.x;
        tile[tt][c * 4 + 1] = v.y;
        tile[tt][c * 4 + 2] = v.z;
        tile[tt][c * 4 + 3] = v.w;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 1024; k += 256) {
        const int row = k >> 3, c = k & 7;
        const int nl = row >> 1, comp = row & 1;
        const int shift = (nl & 3) * 8 + (comp ? 0 : 4);
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t nib = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) nib |= ((tile[c * 16 + q * 4 + u][nl >> 2] >> shift) & 0xFu) << (8 * u);
            w[q] = dev::nibbles_to_e5m2(nib);
        }
        *reinterpret_cast<uint4 *>(y + ((size_t)f * R + blockIdx.y * 128 + row) * ldy + t0 + c * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// MN-major: Y[f][t][0..R) = E5M2 codes in groups of four inputs (16 Re x_0..16 Re x_3, Im x_0..
// Im x_3, 16 Re x_4, ...), zero past 2N and past T.
// One thread per 32 output bytes (16 samples in): grid-stride over F * ldy * (R / 32).
__global__ void __launch_bounds__(256) unpack_mn_kernel(const uint8_t *__restrict__ frame, uint8_t *__restrict__ y,
                                                        int N, int F, int T, int R, int64_t ldy) {
    const int cpr = R / 32;                        // 32-byte chunks per output row
    const int64_t total = (int64_t)F * ldy * cpr;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % cpr);
        const int64_t row = q / cpr;               // f * ldy + t
        const int t = (int)(row % ldy);
        const int f = (int)(row / ldy);
        uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
        if (t < T && 16 * c < N) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(frame + ((size_t)t * F + f) * N + 16 * c));
            dev::expand16_e5m2(v, lo, hi);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(y + row * R + 32 * c);
        __stcs(dst, lo);
        __stcs(dst + 1, hi);
    }
}

// ----------------------------------------------------------------------------- epilogue

// Row (and column) order of the operand blocks. K-major engine: interleaved pairs, row 2n = Re x_n,
// row 2n+1 = Im x_n. MN-major engines: groups of four inputs, rows 8g..8g+3 = 16 Re x_{4g..4g+3},
// rows 8g+4..8g+7 = Im x_{4g..4g+3} (the order the byte expansion produces cheaply).
template <bool kMN>
struct Order {
    static __device__ __forceinline__ int input_of(int m) { return kMN ? 4 * (m >> 3) + (m & 3) : m >> 1; }
    static __device__ __forceinline__ int comp_of(int m) { return kMN ? (m >> 2) & 1 : m & 1; }
    static constexpr int kPartner = kMN ? 4 : 1;   // lane holding the other component of the same input
    // register (column within a 32-column chunk) of local output column jj (0..15), component c
    static __host__ __device__ constexpr int reg(int jj, int c) { return kMN ? 8 * (jj >> 2) + (jj & 3) + 4 * c : 2 * jj + c; }
};

// One 32-column chunk of this thread's TMEM lane (one row of G, 16 output columns j0..j0+15):
// the 2x2 Re/Im combine with the lane holding the other component of input i, in FP32 (exact: the
// operands are integers times powers of two below 2^22), then to int32 by adding 1.5 * 2^23 and
// subtracting its bit pattern. The Re-row lane produces j0..j0+7, the Im-row lane j0+8..j0+15:
// V = (G[re,re] + G[im,im]) + i (G[im,re] - G[re,im]). MN engines: G[re,re] carries 256, G[re,im]
// and G[im,re] 16, G[im,im] 1 (the operand holds 16 Re).
template <bool kMN>
__device__ __forceinline__ void combine_chunk(uint32_t taddr, bool im_row, int (&vr)[8], int (&vi)[8]) {
    using O = Order<kMN>;
    uint32_t r[32];
    dev::tmem_ld_32x32b_x32(taddr, r);
    dev::tmem_ld_wait();
    constexpr float kRR = kMN ? 1.0f / 256.0f : 1.0f;   // scale of G[re,re]
    constexpr float kRI = kMN ? 1.0f / 16.0f : 1.0f;    // scale of G[re,im] and G[im,re]
    constexpr float kMagic = 12582912.0f;               // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t s0 = im_row ? r[O::reg(k, 0)] : r[O::reg(8 + k, 0)];
        const uint32_t s1 = im_row ? r[O::reg(k, 1)] : r[O::reg(8 + k, 1)];
        const float r0 = __uint_as_float(__shfl_xor_sync(0xffffffffu, s0, O::kPartner));
        const float r1 = __uint_as_float(__shfl_xor_sync(0xffffffffu, s1, O::kPartner));
        float re, im;
        if (!im_row) {   // j = j0 + k: own G[re_i,re_j], G[re_i,im_j]; partner G[im_i,re_j], G[im_i,im_j]
            re = fmaf(__uint_as_float(r[O::reg(k, 0)]), kRR, r1);
            im = (r0 - __uint_as_float(r[O::reg(k, 1)])) * kRI;
        } else {         // j = j0 + 8 + k: own G[im_i,re_j], G[im_i,im_j]; partner G[re_i,re_j], G[re_i,im_j]
            re = fmaf(r0, kRR, __uint_as_float(r[O::reg(8 + k, 1)]));
            im = (__uint_as_float(r[O::reg(8 + k, 0)]) - r1) * kRI;
        }
        vr[k] = __float_as_int(re + kMagic) - kMagicBits;
        vi[k] = __float_as_int(im + kMagic) - kMagicBits;
    }
}

// Visibilities j = jb .. jb+7 of row i live at vis_f[2 (prow + j)]: valid for i <= j < N.
__device__ __forceinline__ void load_old(const int32_t *vis_f, int64_t prow, int i, int jb, int N, bool i_ok,
                                         int2 (&old)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int j = jb + k;
        old[k] = (i_ok && j >= i && j < N) ? *reinterpret_cast<const int2 *>(vis_f + 2 * (prow + j)) : make_int2(0, 0);
    }
}

__device__ __forceinline__ void store_vis(int32_t *vis_f, int64_t prow, int i, int jb, int N, bool i_ok,
                                          const int (&vr)[8], const int (&vi)[8], const int2 (&old)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int j = jb + k;
        if (i_ok && j >= i && j < N)
            *reinterpret_cast<int2 *>(vis_f + 2 * (prow + j)) = make_int2(vr[k] + old[k].x, vi[k] + old[k].y);
    }
}

// ----------------------------------------------------------------------------- GEMM kernel

constexpr int kEpiWarps = 8;                  // two per TMEM lane quarter
constexpr int kEpiWarp0 = 2;
constexpr int kConvWarp0 = kEpiWarp0 + kEpiWarps;

template <int kEngine>
struct Cfg {
    static constexpr bool kFused = kEngine == kFusedMN;
    static constexpr bool kMN = kEngine != kUnpackedK;
    static constexpr int kThreads = 32 * (kConvWarp0 + (kFused ? kConvWarps : 0));
    static constexpr int kKt = kMN ? kKtMN : kKtMax;    // samples per stage
    static constexpr int kOpSlotBytes = kBlk * kKt;     // one operand block for one stage
    static constexpr int kPkSlotBytes = 64 * kKt;       // 64 inputs x kKt samples, packed
};

__host__ __device__ constexpr int kt_of(int engine, bool packets = false) {
    return engine == kUnpackedK ? kKtMax : (engine == kFusedPair ? (packets ? kPairKtPackets : kPairKtFrame) : kKtMN);
}

template <int kEngine>
__global__ void __launch_bounds__(Cfg<kEngine>::kThreads, 1) correlate_kernel(const __grid_constant__ Params p) {
    using C = Cfg<kEngine>;
    constexpr int kKt = C::kKt;
    constexpr int kOpSlotBytes = C::kOpSlotBytes;
    constexpr int kPkSlotBytes = C::kPkSlotBytes;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int op_stage_bytes = p.slots * kOpSlotBytes;
    const int pk_stage_bytes = p.slots * kPkSlotBytes;
    uint8_t *op_ring = smem;
    uint8_t *pk_ring = smem + p.op_stages * op_stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(pk_ring + (C::kFused ? p.pk_stages * pk_stage_bytes : 0));
    uint64_t *op_full = bars;                       // [op_stages] operand ready (TMA or converters)
    uint64_t *op_empty = op_full + p.op_stages;     // [op_stages] MMA done reading
    uint64_t *pk_full = op_empty + p.op_stages;     // [pk_stages] packed tile landed (fused)
    uint64_t *pk_empty = pk_full + p.pk_stages;     // [pk_stages] packed tile consumed (fused)
    uint64_t *acc_full = pk_empty + p.pk_stages;    // [2] accumulator ready for the epilogue
    uint64_t *acc_empty = acc_full + 2;             // [2] accumulator drained
    uint64_t *item_full = acc_empty + 2;            // [kItemRing]
    uint64_t *item_empty = item_full + kItemRing;   // [kItemRing]
    uint64_t *done = item_empty + kItemRing;
    int *item_ring = reinterpret_cast<int *>(done + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(item_ring + kItemRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t op_base = dev::smem_u32(op_ring);
    const uint32_t pk_base = dev::smem_u32(pk_ring);
    const int n_item_consumers = 1 + kEpiWarps + (C::kFused ? kConvWarps : 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.op_stages; ++s) {
            dev::mbar_init(&op_full[s], C::kFused ? kConvWarps : 1);
            dev::mbar_init(&op_empty[s], 1);
        }
        for (int s = 0; s < p.pk_stages; ++s) {
            dev::mbar_init(&pk_full[s], 1);
            dev::mbar_init(&pk_empty[s], kConvWarps);
        }
        for (int a = 0; a < 2; ++a) {
            dev::mbar_init(&acc_full[a], 1);
            dev::mbar_init(&acc_empty[a], kEpiWarps);
        }
        for (int s = 0; s < kItemRing; ++s) {
            dev::mbar_init(&item_full[s], 1);
            dev::mbar_init(&item_empty[s], n_item_consumers);
        }
        dev::mbar_init(done, 1);
        *abort_flag = 0;
        dev::fence_mbar_init();
        for (int j = 0; j < p.n_jobs; ++j) dev::prefetch_tmap(&p.jobs[j].tmap);
    }
    if (warp == 1) {
        dev::tmem_alloc(tmem_slot, kTmemCols);
        dev::tmem_relinquish();
    }
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (dev::mbar_try_wait(bar, parity)) return true;
        const uint64_t t0 = dev::globaltimer_ns();
        for (uint32_t it = 1;; ++it) {
            if (dev::mbar_try_wait(bar, parity)) return true;
            if ((it & 127u) == 0) {
                if (*abort_flag) return false;
                if (dev::globaltimer_ns() - t0 > p.limit_ns) {
                    *abort_flag = 1;
                    atomicExch(p.status, XE_ETIMEOUT);
                    return false;
                }
            }
        }
    };

    // Next work item for a consumer role (one call per warp, or by the single MMA thread):
    // returns the item index, -1 when the list is exhausted, -2 on abort.
    uint32_t islot = 0, iphase = 0;
    auto next_item = [&](bool warp_role) -> int {
        if (!wait(&item_full[islot], iphase)) return -2;
        const int g = *reinterpret_cast<volatile int *>(&item_ring[islot]);
        if (warp_role) __syncwarp();
        if (!warp_role || lane == 0) dev::mbar_arrive(&item_empty[islot]);
        if (++islot == kItemRing) { islot = 0; iphase ^= 1; }
        return g;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------------- scheduler + TMA producer
            uint32_t s = 0, ph = 0;                 // op ring (unpacked) or packed ring (fused)
            uint32_t pslot = 0, pphase = 0;         // item ring
            uint32_t issued = 0, issued_parity = 0;
            const int n_stages = C::kFused ? p.pk_stages : p.op_stages;
            uint64_t *full = C::kFused ? pk_full : op_full;
            uint64_t *empty = C::kFused ? pk_empty : op_empty;
            bool ok = true;
            while (ok) {
                if (!wait(&item_empty[pslot], pphase ^ 1)) break;
                int g = atomicAdd(p.counter, 1);
                if (g >= p.n_items) g = -1;
                item_ring[pslot] = g;
                dev::mbar_arrive(&item_full[pslot]);
                if (++pslot == kItemRing) { pslot = 0; pphase ^= 1; }
                if (g < 0) break;
                const Item it = decode_item(p, g);
                const Job &jb = p.jobs[it.job];
                const uint32_t tx = C::kFused ? it.nblk * jb.pw * kKt : it.nblk * kOpSlotBytes;
                for (int kt = 0; kt < jb.k_tiles; ++kt) {
                    if (!wait(&empty[s], ph ^ 1)) { ok = false; break; }
                    dev::mbar_arrive_expect_tx(&full[s], tx);
                    for (int b = 0; b < it.nblk; ++b) {
                        if (C::kFused)
                            dev::tma_load_3d(pk_base + s * pk_stage_bytes + b * kPkSlotBytes, &jb.tmap, &full[s],
                                             block_of(it, b) * 64, it.f, kt * kKt);
                        else if (C::kMN)
                            dev::tma_load_3d(op_base + s * op_stage_bytes + b * kOpSlotBytes, &jb.tmap, &full[s],
                                             block_of(it, b) * kBlk, kt * kKt, it.f);
                        else
                            dev::tma_load_3d(op_base + s * op_stage_bytes + b * kOpSlotBytes, &jb.tmap, &full[s],
                                             kt * kKt, block_of(it, b) * kBlk, it.f);
                    }
                    issued |= 1u << s;
                    issued_parity = (issued_parity & ~(1u << s)) | (ph << s);
                    if (++s == (uint32_t)n_stages) { s = 0; ph ^= 1; }
                }
            }
            for (int q = 0; q < n_stages; ++q)
                if (issued & (1u << q)) dev::mbar_wait(&full[q], (issued_parity >> q) & 1u, p.limit_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------------------- MMA issuer
            uint32_t s = 0, ph = 0;
            uint32_t acc = 0, acc_ph = 0;            // bit a: phase parity of accumulator a
            bool ok = true;
            while (ok) {
                const int g = next_item(false);
                if (g < 0) break;
                const Item it = decode_item(p, g);
                const Job &jb = p.jobs[it.job];
                for (int k0 = 0; k0 < jb.k_tiles && ok; k0 += p.k_flush_tiles) {
                    const int k1 = min(jb.k_tiles, k0 + p.k_flush_tiles);
                    if (!wait(&acc_empty[acc], ((acc_ph >> acc) & 1u) ^ 1u)) { ok = false; break; }
                    dev::tc_fence_after();
                    const uint32_t d0 = tmem + acc * 256u;
                    for (int kt = k0; kt < k1; ++kt) {
                        if (!wait(&op_full[s], ph)) { ok = false; break; }
                        dev::tc_fence_after();
                        const uint32_t sb = op_base + s * op_stage_bytes;
#pragma unroll
                        for (int kk = 0; kk < kKt / 32; ++kk) {
                            const uint32_t accum = (kt > k0 || kk > 0) ? 1u : 0u;
                            for (int c = 0; c < it.w; c += 2) {
                                const bool wide = c + 1 < it.w;
                                uint64_t ad, bd;
                                uint32_t idesc;
                                if (C::kMN) {   // K step of 32 rows of 128 bytes = 4096 bytes
                                    ad = dev::sdesc_mn_sw128(sb + it.a_slot * kOpSlotBytes + kk * 4096, kOpSlotBytes);
                                    bd = dev::sdesc_mn_sw128(sb + c * kOpSlotBytes + kk * 4096, kOpSlotBytes);
                                    idesc = wide ? dev::idesc_e5m2_f32_mn(128, 256) : dev::idesc_e5m2_f32_mn(128, 128);
                                } else {        // K step of 32 bytes inside the 128-byte swizzled row
                                    ad = dev::sdesc_k_sw128(sb + it.a_slot * kOpSlotBytes + kk * 32);
                                    bd = dev::sdesc_k_sw128(sb + c * kOpSlotBytes + kk * 32);
                                    idesc = wide ? dev::idesc_e5m2_f32(128, 256) : dev::idesc_e5m2_f32(128, 128);
                                }
                                dev::mma_f8f6f4(d0 + c * kBlk, ad, bd, idesc, accum);
                            }
                        }
                        dev::tc_commit(&op_empty[s]);
                        if (++s == (uint32_t)p.op_stages) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    dev::tc_commit(&acc_full[acc]);
                    acc_ph ^= 1u << acc;
                    acc = (acc + 1 == (uint32_t)p.n_acc) ? 0u : acc + 1;
                }
            }
            dev::tc_commit(done);
            dev::mbar_wait(done, 0, p.limit_ns);
        }
    } else if (warp < kConvWarp0) {
        // -------------------------------------------------------------------- epilogue warps
        // Warp w reads TMEM lane quarter w % 4; the two warps of a quarter split the 32-column
        // chunks of an item between them. The accumulate-mode loads of the next chunk are issued
        // before the current chunk is combined, so their latency overlaps useful work.
        using O = Order<C::kMN>;
        const int q = warp & 3;
        const int half = (warp - kEpiWarp0) >> 2;
        const int m = q * 32 + lane;            // row of the 128-row tile
        const bool im_row = O::comp_of(m) != 0;
        uint32_t acc = 0, acc_ph = 0;
        bool ok = true;
        while (ok) {
            const int g = next_item(true);
            if (g < 0) break;
            const Item it = decode_item(p, g);
            const Job &jb = p.jobs[it.job];
            const int N = jb.n_inputs;
            const int i = it.rb * (kBlk / 2) + O::input_of(m);
            const bool i_ok = i < N;
            const int64_t prow = (int64_t)i * N - (int64_t)i * (i - 1) / 2 - i;   // p(i, j) = prow + j
            int32_t *vis_f = jb.vis + (size_t)it.f * (size_t)npairs(N) * 2;
            const int n_chunks = it.w * (kBlk / 32);
            for (int k0 = 0; k0 < jb.k_tiles; k0 += p.k_flush_tiles) {
                if (!wait(&acc_full[acc], (acc_ph >> acc) & 1u)) { ok = false; break; }
                dev::tc_fence_after();
                const bool add = jb.accumulate || k0 > 0;
                const uint32_t tb = tmem + acc * 256u + (uint32_t(q * 32) << 16);
                auto jb_of = [&](int ck) {           // first output column of chunk ck for this lane
                    return (it.cb0 * kBlk + ck * 32) / 2 + (im_row ? 8 : 0);
                };
                int2 old[8], nxt[8];
                int ck = half;
                if (add && ck < n_chunks) load_old(vis_f, prow, i, jb_of(ck), N, i_ok, old);
                else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) old[k] = make_int2(0, 0);
                }
#pragma unroll 1
                for (; ck < n_chunks; ck += 2) {
                    const bool more = ck + 2 < n_chunks;
                    if (add && more) load_old(vis_f, prow, i, jb_of(ck + 2), N, i_ok, nxt);
                    int vr[8], vi[8];
                    combine_chunk<C::kMN>(tb + ck * 32, im_row, vr, vi);
                    store_vis(vis_f, prow, i, jb_of(ck), N, i_ok, vr, vi, old);
                    if (add && more) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) old[k] = nxt[k];
                    }
                }
                dev::tc_fence_before();
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(&acc_empty[acc]);
                acc_ph ^= 1u << acc;
                acc = (acc + 1 == (uint32_t)p.n_acc) ? 0u : acc + 1;
            }
        }
    } else if constexpr (C::kFused) {
        // -------------------------------------------------------------------- converter warps
        // Packed tile [128 t][pw bytes] -> MN-major operand rows: row t of block b holds the 128
        // codes of inputs 64*blk .. 64*blk+63 at sample t in the grouped order, 16-byte chunks
        // swizzled as chunk ^ (t & 7) (the 128-byte swizzle the MMA descriptor names).
        // Each thread owns kTasks fixed (t, 16-byte chunk) positions of every block: kKt samples x
        // 4 chunks per block, spread over the 256 converter threads.
        constexpr int kTasks = kKt * 4 / (32 * kConvWarps);
        static_assert(kTasks * 32 * kConvWarps == kKt * 4, "conversion tasks divide evenly");
        const int ctid = threadIdx.x - 32 * kConvWarp0;
        uint32_t dst0[kTasks], dst1[kTasks];
#pragma unroll
        for (int u = 0; u < kTasks; ++u) {
            const int r = ctid + 32 * kConvWarps * u, t = r >> 2, c = r & 3;
            dst0[u] = t * 128 + (((2 * c) ^ (t & 7)) << 4);
            dst1[u] = t * 128 + (((2 * c + 1) ^ (t & 7)) << 4);
        }
        uint32_t ps = 0, pph = 0, os = 0, oph = 0;
        bool ok = true;
        while (ok) {
            const int g = next_item(true);
            if (g < 0) break;
            const Item it = decode_item(p, g);
            const Job &jb = p.jobs[it.job];
            uint32_t src[kTasks];
            bool have[kTasks];
#pragma unroll
            for (int u = 0; u < kTasks; ++u) {
                const int r = ctid + 32 * kConvWarps * u, t = r >> 2, c = r & 3;
                src[u] = t * jb.pw + 16 * c;
                have[u] = 16 * c < jb.pw;
            }
            for (int kt = 0; kt < jb.k_tiles; ++kt) {
                if (!wait(&pk_full[ps], pph)) { ok = false; break; }
                if (!wait(&op_empty[os], oph ^ 1)) { ok = false; break; }
                const uint32_t pk = pk_base + ps * pk_stage_bytes;
                const uint32_t op = op_base + os * op_stage_bytes;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if (b < it.nblk) {
#pragma unroll
                        for (int u = 0; u < kTasks; ++u) {
                            uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
                            if (have[u]) {
                                uint4 v;
                                asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                                             : "r"(pk + b * kPkSlotBytes + src[u]));
                                dev::expand16_e5m2(v, lo, hi);
                            }
                            const uint32_t row = op + b * kOpSlotBytes;
                            asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};"
                                         ::"r"(row + dst0[u]), "r"(lo.x), "r"(lo.y), "r"(lo.z), "r"(lo.w));
                            asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};"
                                         ::"r"(row + dst1[u]), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w));
                        }
                    }
                }
                dev::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    dev::mbar_arrive(&pk_empty[ps]);
                    dev::mbar_arrive(&op_full[os]);
                }
                if (++ps == (uint32_t)p.pk_stages) { ps = 0; pph ^= 1; }
                if (++os == (uint32_t)p.op_stages) { os = 0; oph ^= 1; }
            }
        }
    }

    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    if (warp == 1) dev::tmem_dealloc(tmem, kTmemCols);
}

// ----------------------------------------------------------------------------- pair engine (cta_group::2)
//
// FUSED_PAIR: a cluster of two CTAs on two SMs computes 256x256 blocks (R, C), C >= R, of a
// channel's Gram matrix with M = 256 tensor-core MMAs whose operands are split across the pair:
// CTA r holds A rows 256R + 128r .. +128 (operand block 2R + r) and B columns 256C + 128r .. +128
// (block 2C + r) in its own shared memory, and receives D rows 256R + 128r .. +128 x all 256
// columns in its own tensor memory. Each SM thus reads half of B per MAC and each converted block
// feeds twice the MACs of the single-CTA engine. On a diagonal block (R = C) the A and B halves of
// a CTA are the same block. Both CTAs walk the same static item sequence (item g = pair + k *
// pairs, channel-major); converters and epilogue warps of both CTAs arrive on the even CTA's
// barriers, and the even CTA's single MMA thread commits to both CTAs.
// Shared-memory bandwidth, not the tensor pipe, bounds this design when packed tiles are staged in
// shared memory (the MMAs alone read 32 KB of operands per stage and CTA), so the converters load
// their packed samples from global memory straight into registers, one stage ahead, and the
// converter forwarder keeps L2 warm with TMA prefetches a few stages further ahead; shared memory
// then only carries the converted operands.
// Every single-thread role (MMA issuer, the two forwarders) has a warp of its own: lanes of one
// warp on different roles run their branches in turn, and a lane suspended in an mbarrier wait
// would hold up the lane it waits for.

constexpr int kPairSlots = 2;                 // operand blocks per stage and CTA of Gram items: A, B (a twin: A
                                              // of channels f and f + 1; a wide stage: A, samples kKt further on)
constexpr int kFoldSlots = 3;                 // operand blocks per stage and CTA of fold items: S, A, B
constexpr int kFoldStageD = 32 * 128 * 4;     // fold epilogue: 32 rows of this CTA's diagonal quadrant
constexpr int kFoldStageX = 32 * 128 * 4;     // fold epilogue: 32 rows of the partner's off-diagonal quadrant
constexpr int kFoldStageBytes = kFoldStageD + kFoldStageX;   // leaves room for four operand stages
constexpr uint32_t kEpiBar = 1;               // named barrier of the four epilogue warps
constexpr int kPairEpiWarps = 4;              // one per TMEM lane quarter (accumulator double-buffered)
constexpr int kPairConvFwdWarp = 2;           // forwards converter completion, prefetches into L2
constexpr int kPairEpiFwdWarp = 3;            // forwards epilogue completion to the even CTA
constexpr int kPairEpiWarp0 = 4;
constexpr int kPairConvWarp0 = kPairEpiWarp0 + kPairEpiWarps;
// Converter shape per mode. A stage is kKt samples; 16 converter warps and two register buffers
// (one stage of samples in flight) in both kernels. Frame mode (the 256-sample kernel): 256-sample
// stages (half the per-stage bookkeeping of 128: 0.80 against 0.81 ms per full-band frame), two rows
// per thread; two buffers against three: 7.21 against 7.97 ms for N = 2048, 64 channels, T = 16384,
// 0.79 against 0.86 ms for N = 1024. Packet mode (the 128-sample kernel): one row per thread.
// Measured on the 8-frame full-band call shape (296 channels) and the one-frame call: 16 warps with
// two buffers 1.12 / 0.587 ms, with three 1.12 / 0.622, with four 1.67 / 0.90; 8 warps of two rows
// with four buffers 1.27 / 0.70, with three 1.22 / 0.65. The sample gathers in flight occupy L1,
// which the 196 KB of shared memory leaves at 60 KB per SM, and more warps rather than more stages
// in flight hide their latency. kRows sample rows per thread and block, kRowStep apart.
template <bool kPackets>
struct PairShape {
    static constexpr int kKt = kPackets ? kPairKtPackets : kPairKtFrame;
    static constexpr int kConvWarps = 16;
    static constexpr int kRows = kKt * 4 / (32 * kConvWarps);
    static constexpr int kRowStep = kKt / kRows;
    static constexpr int kBufs = 2;
    static constexpr int kThreads = 32 * (kPairConvWarp0 + kConvWarps);
    // registers per thread: at launch (the __launch_bounds__ limit), and after the split between
    // the role, epilogue and converter warpgroups, which hands out exactly the registers the
    // launch allocates. The 128-sample kernel: roles 48, fold epilogue 112, converters 80 (the
    // split with the fewest spills: 20 bytes of spill stores); the 256-sample kernel: roles 32, Gram
    // epilogue 96, converters (two rows) 88, without spills
    static constexpr int kRegsLaunch = 65536 / kThreads / 8 * 8;
    static constexpr int kRegsRoles = kPackets ? 48 : 32;
    static constexpr int kRegsEpi = kPackets ? 112 : 96;
    static constexpr int kRegsConv = (kRegsLaunch * kThreads - 128 * (kRegsRoles + kRegsEpi)) / (32 * kConvWarps) / 8 * 8;
    static_assert(kRegsConv >= 24 && kRegsConv <= 256, "a warpgroup holds 24 to 256 registers per thread");
    static_assert(128 * kRegsRoles + 128 * kRegsEpi + 32 * kConvWarps * kRegsConv <= kRegsLaunch * kThreads,
                  "the register split fits the launch's registers");
    static_assert(kRows * 32 * kConvWarps == kKt * 4, "conversion tasks divide evenly");
    static_assert(kRowStep % 8 == 0, "a thread's rows share their 128-byte swizzle phase");
};
constexpr int kPairMaxStages = 6;
constexpr int kPairSmemBudget = 196 * 1024;   // dynamic shared memory of a pair CTA (see run_batched)
// Packet mode: integrations of at least this many samples run the twin layout (see decode_pair_item)
constexpr int kTwinMinTime = 16384;
constexpr int kPairPrefetch = 4;              // L2 prefetch distance in stages

// One work item of the pair engine. Gram items compute a 256 x 256 block (R, C), C >= R, of the
// interleaved Gram matrix G = Y Y^T, in units of 256 Gram rows (128 inputs); fold items compute the
// folded product D = S S^T - 2 A B^T of the 256-input super-block R = C (inputs 256 R .. 256 R + 255).
struct PairItem {
    int job, f, R, C;
    bool dbl;    // fills both TMEM halves (a double or a twin)
    bool twin;   // the last diagonal blocks of channels f and f + 1
    bool wide;   // a single diagonal block in stages of 2 kKt samples
    bool fold;   // a fold item (fold layout only)
    bool empty;  // balanced split: no further item of this pair
    int kt0;     // balanced split: first stage of the piece (else 0)
    int kt_n;    // balanced split: stages of the piece (else -1: the job's whole integration)
};

// Work items of a frame-mode job: every 256x256 block (R, C >= R) of every channel its own item.
// Work items of a packet-mode job with at most 128 inputs (one 256-row block per channel): its
// diagonal block, by pairs of channels (2c, 2c + 1), which share a packet group:
// - each channel's doubles: the diagonal block (R, R) together with its right neighbour (R, R + 1),
//   R < S2 - 1, computed into the two TMEM halves from one operand stage (A = block R, B = block R
//   + 1) (none at N <= 128);
// - its singles (R, C >= R + 2);
// - then one twin: the last diagonal block (S2 - 1, S2 - 1) of both channels, channel 2c's block in
//   the A slot and channel 2c + 1's (N bytes further into the same packets) in the B slot, each
//   multiplied by itself into its own TMEM half.
// Integrations shorter than kTwinMinTime keep each channel's diagonal block as a wide single. Pairs
// take items pair, pair + pairs, ... (Frame mode, with 256-sample stages, runs every block as its own
// item: doubles make its stages MMA-bound, 0.80 -> 0.84 ms.)
// Work items of a packet-mode job with more than 128 inputs (the fold layout), channel by channel:
// - one fold item per whole 256-input super-block R: D = S S^T - 2 A B^T over its inputs, with
//   s = a + b; the visibilities of the super-block are Re V = (D + D^T) / 2, Im V = (D - D^T) / 2, so
//   its 2 x 2 Gram blocks (three of them on or above the diagonal) cost two block products;
// - a half super-block at the end (N mod 256 in (0, 128]) as a Gram diagonal single;
// - the Gram blocks between different super-blocks as singles (R, C) with R / 2 < C / 2.
// Each fold item and single fills one TMEM half, so consecutive items alternate halves.
// (kSplit: the 128-sample kernel, the only one that runs balanced splits)
template <bool kSplit>
__device__ __forceinline__ PairItem decode_pair_item(const Params &p, int g) {
    PairItem it;
    it.empty = false;
    it.kt0 = 0;
    it.kt_n = -1;
    if (kSplit && p.split_u > 0) {            // balanced split: piece k of pair q's stage range
        const Job &jb = p.jobs[0];
        const int q = g % p.split_pairs, k = g / p.split_pairs, K = jb.k_tiles;
        const int64_t total = (int64_t)jb.n_chan * K;
        const int64_t start = (int64_t)q * p.split_u, end = min(start + p.split_u, total);
        const int c = (int)(start / K) + k;
        const int64_t s0 = max(start, (int64_t)c * K), s1 = min(end, (int64_t)(c + 1) * K);
        it.job = 0;
        it.f = c;
        it.R = it.C = 0;
        it.dbl = it.twin = it.wide = false;
        it.fold = true;
        it.empty = c >= jb.n_chan || s0 >= s1;
        it.kt0 = (int)(s0 - (int64_t)c * K);
        it.kt_n = (int)(s1 - s0);
        return it;
    }
    int j = 0;
    while (j + 1 < p.n_jobs && g >= p.jobs[j + 1].item_begin) ++j;
    const Job &jb = p.jobs[j];
    int l = g - jb.item_begin;
    it.job = j;
    it.dbl = it.twin = it.wide = it.fold = false;
    const int S2 = jb.nb;                     // 256-row blocks (128 inputs each)
    int q;
    if (jb.fold) {
        it.f = l / jb.strips;
        q = l % jb.strips;
        const int n_fold = S2 / 2;
        if (q < n_fold) {                     // fold item of super-block q
            it.R = it.C = q;
            it.fold = true;
            return it;
        }
        q -= n_fold;
        if (S2 & 1) {                         // the last half super-block's diagonal block
            if (q == 0) {
                it.R = it.C = S2 - 1;
                return it;
            }
            --q;
        }
        for (it.R = 0; it.R < S2; ++it.R) {   // blocks of different super-blocks
            const int c0 = 2 * (it.R / 2 + 1), n = S2 - c0;
            if (n > 0) {
                if (q < n) {
                    it.C = c0 + q;
                    return it;
                }
                q -= n;
            }
        }
        it.R = it.C = 0;                      // not reached
        return it;
    }
    if (!jb.twin) {
        it.f = l / jb.strips;
        q = l % jb.strips;
        if (jb.doubles == 0 && !p.wide_diag) {   // frame mode: every block (R, C >= R) its own item
            for (it.R = 0; it.R < S2; ++it.R) {
                if (q < S2 - it.R) break;
                q -= S2 - it.R;
            }
            it.C = it.R + q;
            return it;
        }
        if (q < jb.doubles) {                 // packet mode, channel by channel: doubles,
            it.R = q;
            it.C = it.R + 1;
            it.dbl = true;
            return it;
        }
        q -= jb.doubles;                      // then singles, the last diagonal (wide) at the end
        for (it.R = 0; it.R < S2 - 1; ++it.R) {
            if (q < S2 - it.R - 2) break;
            q -= S2 - it.R - 2;
        }
        it.C = it.R < S2 - 1 ? it.R + 2 + q : it.R;
        it.wide = p.wide_diag && it.R == it.C;
        return it;
    }
    const int D = jb.doubles, per_ch = jb.doubles + jb.offdiag;
    const int per2 = jb.strips;               // 2 per_ch + 1 items per channel pair
    const int cp = l / per2;
    q = l % per2;
    if (cp < jb.n_chan / 2) {
        if (q == per2 - 1) {                  // the twin of channels 2 cp and 2 cp + 1
            it.f = 2 * cp;
            it.R = it.C = S2 - 1;
            it.dbl = it.twin = true;
            return it;
        }
        it.f = 2 * cp + q / per_ch;           // q < 2 per_ch, so per_ch > 0 here
        q %= per_ch;
    } else {                                  // the odd last channel: doubles, singles, its diagonal
        it.f = jb.n_chan - 1;
        q = l - (jb.n_chan / 2) * per2;
    }
    if (q < D) {
        it.R = q;
        it.C = it.R + 1;
        it.dbl = true;
        return it;
    }
    q -= D;
    for (it.R = 0; it.R < S2 - 1; ++it.R) {
        if (q < S2 - it.R - 2) break;
        q -= S2 - it.R - 2;
    }
    it.C = it.R < S2 - 1 ? it.R + 2 + q : it.R;
    it.wide = p.wide_diag && it.R == it.C;
    return it;
}

// stages of an item and its drain interval in stages
__device__ __forceinline__ void item_stages(const Params &p, const Job &jb, const PairItem &it, int &k_tiles,
                                            int &flush) {
    k_tiles = it.kt_n >= 0 ? it.kt_n : (it.wide ? jb.k_tiles_wide : jb.k_tiles);
    flush = it.wide ? p.k_flush_tiles_wide : p.k_flush_tiles;
}

// Walks the (item, k-tile) stages of one pair in order (frame mode: forwarder and L2 prefetch).
struct PairCursor {
    int g, kt, job, f, R, C, k_tiles;
    __device__ __forceinline__ void start(const Params &p, int g0) {
        g = g0;
        kt = 0;
        if (g < p.n_items) load(p);
    }
    __device__ __forceinline__ void load(const Params &p) {
        const PairItem it = decode_pair_item<false>(p, g);
        job = it.job;
        f = it.f;
        R = it.R;
        C = it.C;
        k_tiles = it.wide ? p.jobs[job].k_tiles_wide : p.jobs[job].k_tiles;
    }
    __device__ __forceinline__ bool valid(const Params &p) const { return g < p.n_items; }
    __device__ __forceinline__ void next(const Params &p, int n_pairs) {
        if (++kt < k_tiles) return;
        kt = 0;
        g += n_pairs;
        if (g < p.n_items) load(p);
    }
};

constexpr uint32_t kNoPacket = 0xFFFFFFFFu;

// One converter thread's walk over the stages of its pair. The thread converts inputs 16c ..
// 16c + 15 of the A block and (unless the item is a plain diagonal single) of the B slot's block,
// for samples t_row + r kRowStep (r < kRows) of each kKt-sample stage; a stage's address
// arithmetic is two 64-bit adds. A fold item's two loads are inputs 16c .. and 64 + 16c .. of the
// CTA's 128 inputs of the super-block (nblk = 3: they fill the S, A and B slots).
// Frame mode: sample t of these bytes sits at frame + (t F + f) N + column.
// Packet mode (the zero-copy path): sample t sits in packet o = owner[f / 8][t / 4] (the packet
// holding time slot t / 4 of this channel's group), at pkts + o * pkt_stride + 16 + ((t % 4) 8 +
// f % 8) N + column; a lost packet (o = ~0u) reads as zeros, as in an assembled frame. The
// kKt / 4 slots of a stage are looked up by coalesced loads, one per 32 slots and warp (lane l:
// slots l, l + 32, ...), and each thread takes the packets of its rows from those lanes by shfl.
template <bool kPackets, bool kShift = false>
struct PairLoader {
    using S = PairShape<kPackets>;
    static_assert(!kShift || (kPackets && S::kRows == 1), "the shifted reads run in the packet kernel");
    static constexpr int kOwn = S::kKt / 4 / 32;          // owner loads per lane and stage
    static constexpr int kOwnMax = kPackets ? 2 * kOwn : 1;   // a wide stage looks up twice as many
    int g, kt, k_tiles, nblk, t_left;         // t_left = T - (kt * S::kKt + t_row)
    bool va, vb;                              // columns of A / B inside the frame
    bool wide;                                // packet mode: a wide stage (B rows = the next kKt samples)
    const uint8_t *pa, *pb;                   // frame: sample kt * S::kKt + t_row; packets: in packet 0
    int64_t step, rstep;                      // frame: bytes per stage / between a thread's rows
    // packets: address of the owner entry of slot kt * S::kKt / 4 + lane; frame rows in the
    // 128-sample kernel (no owner table): 4 x that slot, which is then the "packet" itself
    uintptr_t own;
    int s_left;                               // T / 4 - (kt * S::kKt / 4 + lane)
    int64_t pstride;
    // time-shifted packets: the source slots of this thread's A and B rows in the current stage
    // (below 0 or from T / 4 on: outside the frame, read as zeros), the slots of the rows themselves
    // (from T / 4 on: past the frame's end, zeros too), and the owner entries of its channel group
    int sa, sb, ua, ub, q_slots;
    const uint32_t *orow;

    __device__ __forceinline__ void begin_item(const Params &p, uint32_t rank, int t_row, int c) {
        const PairItem it = decode_pair_item<kPackets>(p, g);
        if (it.empty) {                       // balanced split: this pair's pieces are done
            g = p.n_items;
            return;
        }
        const Job &jb = p.jobs[it.job];
        const int N = jb.n_inputs, F = jb.n_chan;
        kt = 0;
        wide = kPackets && it.wide;
        const bool twin = kPackets && it.twin;
        k_tiles = it.kt_n >= 0 ? it.kt_n : (wide ? jb.k_tiles_wide : jb.k_tiles);
        int ca, cb;
        if (kPackets && it.fold) {
            // odd rows take the CTA's second 64 inputs first: their first stores then go to chunks
            // 4..7 while even rows' go to chunks 0..3 (no shared-memory bank conflicts)
            nblk = 3;
            const int h = t_row & 1;
            ca = 256 * it.R + 128 * (int)rank + 64 * h + 16 * c;
            cb = 256 * it.R + 128 * (int)rank + 64 * (1 - h) + 16 * c;
        } else {
            nblk = it.R == it.C && !wide && !twin ? 1 : 2;
            ca = (2 * it.R + (int)rank) * 64 + 16 * c;
            cb = (2 * it.C + (int)rank) * 64 + 16 * c;
        }
        t_left = jb.n_time - t_row;
        va = ca < N;
        vb = nblk >= 2 && cb < N;
        const uint8_t *base;
        if constexpr (kPackets) {
            const int Q = jb.n_time / 4, lane = threadIdx.x & 31;
            if constexpr (kShift) {
                // row t of the shifted frame is row t - d of the frame: slot (t - d) / 4 (floor) and
                // row (t - d) mod 4 of that packet; a wide stage's B rows lie kKt samples further on
                const int da = va ? p.delay16[ca >> 4] : 0, db = vb ? p.delay16[cb >> 4] : 0;
                const int ta = t_row - da, tb = t_row - db + (wide ? S::kKt : 0);
                sa = ta >> 2;
                sb = tb >> 2;
                ua = t_row >> 2;
                ub = (t_row + (wide ? S::kKt : 0)) >> 2;
                q_slots = Q;
                orow = jb.owner + (size_t)(it.f / 8) * Q;
                pstride = jb.pkt_stride;
                pa = jb.pkts + 16 + ((size_t)(ta & 3) * 8 + it.f % 8) * N + ca;
                pb = jb.pkts + 16 + ((size_t)(tb & 3) * 8 + it.f % 8) * N + cb + (twin ? N : 0);
                base = nullptr;
            } else if (!p.frame_rows) {
                base = jb.pkts + 16 + ((size_t)(t_row & 3) * 8 + it.f % 8) * N;
                own = reinterpret_cast<uintptr_t>(jb.owner + (size_t)(it.f / 8) * Q + lane);
                pstride = jb.pkt_stride;
            } else {
                // an assembled frame read in the same 4-sample slots: slot s stands for a packet
                // whose rows 4 s .. 4 s + 3 lie 4 F N bytes on from those of slot s - 1
                base = jb.frame + ((size_t)(t_row & 3) * F + it.f) * N;
                own = (uintptr_t)lane * 4;
                pstride = (int64_t)4 * F * N;
            }
            s_left = Q - lane;
        } else {
            base = jb.frame + ((size_t)t_row * F + it.f) * N;
            step = (int64_t)S::kKt * F * N;
            rstep = (int64_t)S::kRowStep * F * N;
        }
        if (!kShift) {
            pa = base + ca;
            pb = base + cb + (twin ? N : 0);  // a twin's B block: channel f + 1, N bytes on
        }
        if constexpr (kPackets) {             // (the balanced split runs in this kernel only)
            if (it.kt0) {                     // a piece of a split integration starts kt0 stages in
                if constexpr (kShift) {
                    sa += it.kt0 * (S::kKt / 4);
                    sb += it.kt0 * (S::kKt / 4);
                    ua += it.kt0 * (S::kKt / 4);
                    ub += it.kt0 * (S::kKt / 4);
                } else {
                    own += (uintptr_t)it.kt0 * S::kKt;
                    s_left -= it.kt0 * (S::kKt / 4);
                }
            }
        }
    }
    __device__ __forceinline__ void start(const Params &p, int pair, uint32_t rank, int t_row, int c) {
        g = pair;
        if (g < p.n_items) begin_item(p, rank, t_row, c);
    }
    __device__ __forceinline__ bool valid(const Params &p) const { return g < p.n_items; }
    __device__ __forceinline__ void next(const Params &p, int n_pairs, uint32_t rank, int t_row, int c) {
        t_left -= S::kKt;
        if constexpr (kShift) {
            sa += (wide ? 2 : 1) * (S::kKt / 4);
            sb += (wide ? 2 : 1) * (S::kKt / 4);
            ua += (wide ? 2 : 1) * (S::kKt / 4);
            ub += (wide ? 2 : 1) * (S::kKt / 4);
        } else if constexpr (kPackets) {
            own += (wide ? 2 : 1) * S::kKt;       // kKt / 4 slots of 4 bytes
            s_left -= (wide ? 2 : 1) * (S::kKt / 4);
        } else {
            pa += step;
            pb += step;
        }
        if (++kt < k_tiles) return;
        g += n_pairs;
        if (g < p.n_items) begin_item(p, rank, t_row, c);
    }
    // packets: the packets of slots lane, lane + 32, ... of the current stage (a wide stage: then
    // those of slots kKt / 4 + lane, ... in o[kOwn ..])
    // Time-shifted packets: o[0] / o[1] the packets of this thread's A / B row of the stage.
    __device__ __forceinline__ void owners(const Params &p, uint32_t (&o)[kOwnMax]) const {
        if constexpr (kShift) {
            o[0] = o[1] = kNoPacket;
            if (sa >= 0 && sa < q_slots && ua < q_slots) asm("ld.global.nc.u32 %0, [%1];" : "=r"(o[0]) : "l"(orow + sa));
            if (sb >= 0 && sb < q_slots && ub < q_slots) asm("ld.global.nc.u32 %0, [%1];" : "=r"(o[1]) : "l"(orow + sb));
        } else {
#pragma unroll
            for (int q = 0; q < kOwnMax; ++q) {
                o[q] = kNoPacket;
                if constexpr (kPackets) {
                    if ((q < kOwn || wide) && s_left > 32 * q) {
                        if (!p.frame_rows) asm("ld.global.nc.u32 %0, [%1];" : "=r"(o[q]) : "l"(own + 128 * q));
                        else o[q] = (uint32_t)(own / 4) + 32 * q;       // frame rows: the slot itself
                    }
                }
            }
        }
    }
    // the current stage's samples of this thread (packet mode: o[r] / ob[r] the packet of row r of
    // the A / B slot; ob = o except in wide stages)
    __device__ __forceinline__ void load(const uint32_t (&o)[S::kRows], const uint32_t (&ob)[S::kRows],
                                         uint4 (&a)[S::kRows], uint4 (&b)[S::kRows]) const {
        const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int r = 0; r < S::kRows; ++r) {
            if constexpr (kPackets) {
                const bool ok = o[r] != kNoPacket, okb = ob[r] != kNoPacket;
                a[r] = ok && va ? dev::ld_stream_16(pa + (int64_t)o[r] * pstride) : z;
                b[r] = okb && vb ? dev::ld_stream_16(pb + (int64_t)ob[r] * pstride) : z;
            } else {
                const bool ok = t_left > r * S::kRowStep;
                const int64_t off = r * rstep;
                a[r] = ok && va ? dev::ld_stream_16(pa + off) : z;
                b[r] = ok && vb ? dev::ld_stream_16(pb + off) : z;
            }
        }
    }
};

template <bool kPackets, bool kShift = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PairShape<kPackets>::kThreads, 1)
    correlate_pair_kernel(const __grid_constant__ Params p) {
    using S = PairShape<kPackets>;
    constexpr int kPairConvWarps = S::kConvWarps;
    constexpr int kKt = S::kKt;
    constexpr int kOpSlotBytes = kBlk * kKt;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int op_stage_bytes = p.slots * kOpSlotBytes;
    uint8_t *op_ring = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(op_ring + p.op_stages * op_stage_bytes);
    uint64_t *op_full = bars;                       // [op_stages] even CTA: both CTAs' converters
    uint64_t *op_empty = op_full + p.op_stages;     // [op_stages] pair MMAs done (multicast commit)
    uint64_t *acc_full = op_empty + p.op_stages;    // [2] pair MMAs of a segment done (multicast)
    uint64_t *acc_empty = acc_full + 2;             // [2] even CTA: both CTAs' epilogues drained
    uint64_t *conv_done = acc_empty + 2;            // [op_stages] local: this CTA's converters finished
    uint64_t *epi_done = conv_done + p.op_stages;   // [2] local: this CTA's epilogue drained
    uint64_t *done = epi_done + 2;
    uint64_t *x_full = done + 1;                    // fold: the partner's epilogue filled this CTA's stage_x
    uint64_t *x_empty = x_full + 1;                 // fold: the partner's epilogue finished reading its stage_x
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(x_empty + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // fold epilogue staging (after the 1 KiB of barriers): stage_d = [32 rows][128 columns] of FP32
    // accumulator values of this CTA's diagonal quadrant, stage_x = [32 rows][128 columns] received
    // from the partner CTA; 16-byte chunks of a row are swizzled as chunk ^ (row & 7)
    uint8_t *stage_d_ptr = op_ring + p.op_stages * op_stage_bytes + 1024;
    const uint32_t stage_d = dev::smem_u32(stage_d_ptr);
    const uint32_t stage_x = stage_d + kFoldStageD;
    const float *stage_df = reinterpret_cast<const float *>(stage_d_ptr);
    const float *stage_xf = reinterpret_cast<const float *>(stage_d_ptr + kFoldStageD);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = dev::cluster_ctarank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
    const uint32_t op_base = dev::smem_u32(op_ring);

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.op_stages; ++s) {
            // one arrival per CTA of the pair (frame mode: the forwarders), or per converter warp
            dev::mbar_init(&op_full[s], kPackets ? 2 * kPairConvWarps : 2);
            dev::mbar_init(&op_empty[s], 1);
            dev::mbar_init(&conv_done[s], kPairConvWarps);
        }
        for (int a = 0; a < 2; ++a) {
            dev::mbar_init(&acc_full[a], 1);
            dev::mbar_init(&acc_empty[a], 2);
            dev::mbar_init(&epi_done[a], kPairEpiWarps);
        }
        dev::mbar_init(done, 1);
        dev::mbar_init(x_full, 1);                  // CTA 1: the sending warp of CTA 0
        dev::mbar_init(x_empty, kPairEpiWarps);     // CTA 0: the four epilogue warps of CTA 1
        *abort_flag = 0;
        dev::fence_mbar_init();
        if (!kPackets)
            for (int j = 0; j < p.n_jobs; ++j) dev::prefetch_tmap(&p.jobs[j].tmap);
    }
    if (warp == 1) {
        dev::tmem_alloc_pair(tmem_slot, kTmemCols);
        dev::tmem_relinquish_pair();
    }
    dev::tc_fence_before();
    __syncthreads();
    dev::cluster_sync();                            // barriers of both CTAs initialised
    dev::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // Bounded wait: suspended in the barrier between tries (up to 1 ms each; the thread resumes when
    // the phase completes), checking the abort flag and the time limit every 8 tries. Waiting warps
    // issue almost nothing, which leaves issue slots and power to the converters (0.3-0.8 % faster)
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (dev::mbar_try_wait(bar, parity)) return true;
        const uint64_t t0 = dev::globaltimer_ns();
        for (uint32_t it = 1;; ++it) {
            if (dev::mbar_try_wait_hint(bar, parity, 1000000u)) return true;
            if ((it & 7u) == 0) {
                if (*abort_flag) return false;
                if (dev::globaltimer_ns() - t0 > p.limit_ns) {
                    *abort_flag = 1;
                    atomicExch(p.status, XE_ETIMEOUT);
                    return false;
                }
            }
        }
    };
    // the same with cluster-scope acquire, for barriers guarding data the partner CTA wrote
    auto wait_cluster = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (dev::mbar_try_wait_cluster(bar, parity)) return true;
        const uint64_t t0 = dev::globaltimer_ns();
        for (uint32_t it = 1;; ++it) {
            if (dev::mbar_try_wait_cluster(bar, parity)) return true;
            if ((it & 127u) == 0) {
                if (*abort_flag) return false;
                if (dev::globaltimer_ns() - t0 > p.limit_ns) {
                    *abort_flag = 1;
                    atomicExch(p.status, XE_ETIMEOUT);
                    return false;
                }
            }
        }
    };

    // Roles by warpgroup, with the registers split between them (PairShape): the role warps (0-3)
    // need few, the epilogue (4-7) more than the launch's 80; the 128-sample kernel's converters
    // (8-23) keep 80 (128 x 48 + 128 x 112 + 512 x 80 = 768 x 80). Each warpgroup's whole role code
    // follows its split, so the compiler sizes that code for it (the epilogue's spills go away).
    if (warp < kPairEpiWarp0) {
    dev::setmaxnreg_dec<S::kRegsRoles>();
    if (warp == kPairConvFwdWarp) {
        if (!kPackets && lane == 0) {
            // ---------------------------------------------------------------- converter forwarder
            // frame mode: once all converter warps of this CTA finished a stage, tell the even CTA's
            // MMA thread (one arrival per CTA and stage), then prefetch a later stage's packed tiles
            // into L2. Packet mode has no tensor map to prefetch with: its converter warps arrive on
            // the even CTA's barrier themselves (the forwarder's hop measured 2-4 % of a call)
            auto prefetch = [&](const PairCursor &c) {
                const CUtensorMap *map = &p.jobs[c.job].tmap;
                dev::tma_prefetch_l2_3d(map, (2 * c.R + (int)rank) * 64, c.f, c.kt * kKt);
                if (c.R != c.C) dev::tma_prefetch_l2_3d(map, (2 * c.C + (int)rank) * 64, c.f, c.kt * kKt);
            };
            PairCursor cu, pf;
            cu.start(p, pair);
            pf.start(p, pair);
            for (int k = 0; k < kPairPrefetch && pf.valid(p); ++k) {
                prefetch(pf);
                pf.next(p, n_pairs);
            }
            uint32_t os = 0, oph = 0;
            for (; cu.valid(p); cu.next(p, n_pairs)) {
                if (!wait(&conv_done[os], oph)) break;
                dev::mbar_arrive_remote(&op_full[os], 0);
                if (++os == (uint32_t)p.op_stages) { os = 0; oph ^= 1; }
                if (pf.valid(p)) {
                    prefetch(pf);
                    pf.next(p, n_pairs);
                }
            }
        }
    } else if (warp == kPairEpiFwdWarp) {
        if (lane == 0) {
            // ---------------------------------------------------------------- epilogue forwarder
            uint32_t acc = 0, acc_ph = 0;
            bool ok = true;
            for (int g = pair; g < p.n_items && ok; g += n_pairs) {
                const PairItem it = decode_pair_item<kPackets>(p, g);
                if (it.empty) break;
                const bool dbl = kPackets && it.dbl;   // frame mode never runs doubles or twins
                int kt_n, fl;
                item_stages(p, p.jobs[it.job], it, kt_n, fl);
                for (int k0 = 0; k0 < kt_n && ok; k0 += fl) {
                    for (int sub = 0; sub < (dbl ? 2 : 1); ++sub) {   // a double fills both halves
                        if (*abort_flag || !wait(&epi_done[acc], (acc_ph >> acc) & 1u)) { ok = false; break; }
                        dev::mbar_arrive_remote(&acc_empty[acc], 0);
                        acc_ph ^= 1u << acc;
                        acc ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------------------------------------------------------- pair MMA issuer (even CTA)
            constexpr uint32_t idesc = dev::idesc_e5m2_f32_mn(256, 256);
            constexpr uint32_t idesc_s = dev::idesc_e4m3_f32_mn(256, 256);
            uint32_t s = 0, ph = 0, acc = 0, acc_ph = 0;
            bool ok = true;
            for (int g = pair; g < p.n_items && ok; g += n_pairs) {
                const PairItem it = decode_pair_item<kPackets>(p, g);
                if (it.empty) break;
                const bool dbl = kPackets && it.dbl;   // frame mode never runs doubles, twins or folds
                const bool twin = kPackets && it.twin;
                const bool fold = kPackets && it.fold;
                const Job &jb = p.jobs[it.job];
                // a single block multiplies A by B (B = A on the diagonal) into half acc; a double
                // multiplies A by A into half acc and A by B into the other half; a twin A by A and B
                // by B; a wide stage multiplies each slot by itself into half acc; a fold item adds
                // S S^T (E4M3) and A B^T (E5M2; the A codes carry -2 a) into half acc
                const bool wide = kPackets && it.wide;
                const uint32_t b_slot = it.R == it.C && !twin ? 0u : 1u;
                const uint32_t acc2 = acc ^ 1u;
                int kt_n, fl;
                item_stages(p, jb, it, kt_n, fl);
                for (int k0 = 0; k0 < kt_n && ok; k0 += fl) {
                    const int k1 = min(kt_n, k0 + fl);
                    if (*abort_flag || !wait(&acc_empty[acc], ((acc_ph >> acc) & 1u) ^ 1u)) { ok = false; break; }
                    if (dbl && !wait(&acc_empty[acc2], ((acc_ph >> acc2) & 1u) ^ 1u)) { ok = false; break; }
                    dev::tc_fence_after();
                    for (int kt = k0; kt < k1; ++kt) {
                        if (!wait(&op_full[s], ph)) { ok = false; break; }
                        dev::tc_fence_after();
                        const uint32_t sb = op_base + s * op_stage_bytes;
#pragma unroll
                        for (int kk = 0; kk < kKt / 32; ++kk) {
                            const uint64_t ad = dev::sdesc_mn_sw128(sb + kk * 4096, kOpSlotBytes);
                            const uint64_t bd = dev::sdesc_mn_sw128(sb + b_slot * kOpSlotBytes + kk * 4096, kOpSlotBytes);
                            const uint32_t accum = (kt > k0 || kk > 0) ? 1u : 0u;
                            if (fold) {
                                const uint64_t fa = dev::sdesc_mn_sw128(sb + kOpSlotBytes + kk * 4096, kOpSlotBytes);
                                const uint64_t fb = dev::sdesc_mn_sw128(sb + 2 * kOpSlotBytes + kk * 4096, kOpSlotBytes);
                                dev::mma_f8f6f4_pair(tmem + acc * 256u, ad, ad, idesc_s, accum);
                                dev::mma_f8f6f4_pair(tmem + acc * 256u, fa, fb, idesc, 1u);
                            } else if (dbl) {
                                dev::mma_f8f6f4_pair(tmem + acc * 256u, ad, ad, idesc, accum);
                                dev::mma_f8f6f4_pair(tmem + acc2 * 256u, twin ? bd : ad, bd, idesc, accum);
                            } else if (wide) {
                                const uint64_t ad1 = dev::sdesc_mn_sw128(sb + kOpSlotBytes + kk * 4096, kOpSlotBytes);
                                dev::mma_f8f6f4_pair(tmem + acc * 256u, ad, ad, idesc, accum);
                                dev::mma_f8f6f4_pair(tmem + acc * 256u, ad1, ad1, idesc, 1u);
                            } else {
                                dev::mma_f8f6f4_pair(tmem + acc * 256u, ad, bd, idesc, accum);
                            }
                        }
                        dev::tc_commit_pair_multicast(&op_empty[s], 3);
                        if (++s == (uint32_t)p.op_stages) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    dev::tc_commit_pair_multicast(&acc_full[acc], 3);
                    acc_ph ^= 1u << acc;
                    if (dbl) {
                        dev::tc_commit_pair_multicast(&acc_full[acc2], 3);
                        acc_ph ^= 1u << acc2;
                    } else {
                        acc ^= 1u;
                    }
                }
            }
            dev::tc_commit_pair_multicast(done, 1);
            dev::mbar_wait(done, 0, p.limit_ns);
        }
    }
    } else if (warp < kPairConvWarp0) {
        // -------------------------------------------------------------------- epilogue (both CTAs)
        if constexpr (S::kRegsEpi > S::kRegsLaunch) dev::setmaxnreg_inc<S::kRegsEpi>();
        else if constexpr (S::kRegsEpi < S::kRegsLaunch) dev::setmaxnreg_dec<S::kRegsEpi>();
        using O = Order<true>;
        constexpr int kPerQuarter = kPairEpiWarps / 4;
        constexpr float kMagic = 12582912.0f;               // 1.5 * 2^23
        constexpr int kMagicBits = 0x4B400000;
        const int q = warp & 3;
        const int half = (warp - kPairEpiWarp0) >> 2;
        const int m = q * 32 + lane;
        const bool im_row = O::comp_of(m) != 0;
        uint32_t acc = 0, acc_ph = 0, x_ph = 0;
        bool ok = true;
        // Fold items synchronise the four epilogue warps with a named barrier, so every warp walks
        // every item and leaves only together with the others: a warp that failed a wait skips the
        // work of Gram items and says so at the next fold item's first barrier, where all decide.
        for (int g = pair; g < p.n_items; g += n_pairs) {
            const PairItem it = decode_pair_item<kPackets>(p, g);
            if (it.empty) break;
            if (!ok && !(kPackets && it.fold)) continue;
            const bool dbl = kPackets && it.dbl;     // frame mode never runs doubles, twins or folds
            const bool twin = kPackets && it.twin;
            const Job &jb = p.jobs[it.job];
            const int N = jb.n_inputs;
            int32_t *vis_f = jb.vis + (size_t)it.f * (size_t)npairs(N) * 2;
            int kt_n, fl;
            item_stages(p, jb, it, kt_n, fl);
            if (kPackets && it.fold) {
                // ------------------------------------------------------------ fold item
                // This CTA holds rows 128 rank + m of D (scaled by 16) over the super-block's 256
                // inputs, all 256 columns. V[i][j] (i <= j) needs D[i][j] and D[j][i]:
                //   Re V = (D[i][j] + D[j][i]) / 32,  Im V = (D[i][j] - D[j][i]) / 32,
                // formed in FP32 (both sums exact: |2 x 16 V| < 2^28 with at most 23 significant bits)
                // and converted with the 1.5 * 2^23 trick (|V| <= 2^22 per drain segment). Every
                // visibility is written by the thread holding row j of D (column by column: a warp
                // writes 32 consecutive visibilities of one row), in four steps of 32 rows i: in step
                // s, warp s stages its rows of this CTA's diagonal quadrant in stage_d (D[i][j] for the
                // quadrant), and CTA 0's warp s sends its rows of the off-diagonal quadrant
                // (D[i][128 .. 255]) into CTA 1's stage_x; CTA 1 writes that quadrant's V[i][j].
                const int base = 256 * it.R;
                const uint32_t tb = tmem + (uint32_t(q * 32) << 16);
                auto prow_of = [N](int r) -> int32_t { return r * N - r * (r - 1) / 2 - r; };
                const int j = base + 128 * (int)rank + m;            // this thread's row of D
                // 16 visibilities V[ii0 + c][j], c < n_ok (one half of a 32-column TMEM chunk), from
                // D[ii0 + c][j] = stg[c][m] (staging rows r0 + c, whose swizzle phase is c & 7 as r0 is
                // a multiple of 16) and D[j][ii0 + c] = h16[c]. Positions advance row by row: V[ii + 1][j]
                // lies N - ii - 1 entries after V[ii][j]. Adding to existing values is left to L2
                // (red.add of Re and Im): the thread waits for no load, where loading the old values kept
                // the epilogue bound by their latency. Each visibility has one writer thread in every
                // drain, so the integer sums are exact and independent of order.
                auto chunk16 = [&](int ii0, const float *stg, int n_ok, const uint32_t (&h)[16], bool add) {
                    int32_t pos = prow_of(ii0) + j;
                    const int32_t step0 = N - ii0 - 1;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        if (c < n_ok) {
                            const float a = stg[c * 128 + (m ^ (4 * (c & 7)))];
                            const float b = __uint_as_float(h[c]);
                            const int re = __float_as_int(fmaf(a + b, 0.03125f, kMagic)) - kMagicBits;
                            const int im = __float_as_int(fmaf(a - b, 0.03125f, kMagic)) - kMagicBits;
                            int32_t *v = vis_f + 2 * pos;
                            if (add) {
                                dev::red_add(v, re);
                                dev::red_add(v + 1, im);
                            } else {
                                __stcg(reinterpret_cast<int2 *>(v), make_int2(re, im));
                            }
                        }
                        pos += step0 - c;
                    }
                };
                // word offset of (row, col) in a [32][128] staging tile
                auto off = [](int row, int col) -> int {
                    return row * 128 + ((((col >> 2) ^ row) & 7) | ((col >> 2) & ~7)) * 4 + (col & 3);
                };
                if (jb.accumulate) {
                    // the old values this item adds to go into L2 while its MMAs run: this warp writes
                    // columns c0 .. c0 + 31 of rows base .. c0 + 31 (CTA 0: its quadrant; CTA 1: the
                    // off-diagonal quadrant and its own), two 128-byte lines per row: lanes 0..15 take
                    // the first line of every 16th row, lanes 16..31 the second
                    const int c0 = base + 128 * (int)rank + 32 * q;
                    const int r_end = min(c0 + 31, N - 1);
                    if (c0 < N)
                        for (int r = base + (lane & 15); r <= r_end; r += 16)
                            dev::prefetch_l2(vis_f + 2 * (prow_of(r) + max(c0, r) + 16 * (lane >> 4)));
                }
                bool gone = false;
                for (int k0 = 0; k0 < kt_n; k0 += fl) {
                    const uint32_t ta = tb + acc * 256u;
                    // (every decision that guards a warp-wide tcgen05.ld is made uniform across the warp)
                    bool good = __all_sync(0xffffffffu, ok && !*abort_flag && wait(&acc_full[acc], (acc_ph >> acc) & 1u));
                    if (!dev::named_sync_and(kEpiBar, 32 * kPairEpiWarps, good)) { gone = true; break; }
                    dev::tc_fence_after();
                    const bool add = jb.accumulate || k0 > 0;
                    uint32_t d[32];
                    uint32_t h16[16];
                    const int qcol = 128 * (int)rank;                    // first TMEM column of the quadrant
                    for (int st = 0; st < 4; ++st) {
                        // the rows i = 32 st .. 32 st + 31 of this CTA (warp st's lanes)
                        if (good && q == st) {
                            if (rank == 0) {
                                // D[i][128 .. 255] -> CTA 1's stage_x, once it has read the last rows
                                good = __all_sync(0xffffffffu, wait_cluster(x_empty, x_ph ^ 1u));
                                if (good) {
                                    const uint32_t rx = dev::mapa(stage_x, 1);
#pragma unroll 1
                                    for (int k = 4; k < 8; ++k) {
                                        dev::tmem_ld_32x32b_x32(ta + 32 * k, d);
                                        dev::tmem_ld_wait();
#pragma unroll
                                        for (int c = 0; c < 32; c += 4)
                                            dev::st_cluster_v4(rx + 4 * off(lane, 32 * (k - 4) + c), d[c], d[c + 1], d[c + 2], d[c + 3]);
                                    }
                                }
                                asm volatile("fence.acq_rel.cluster;" ::: "memory");   // the stores above, then the arrival
                                __syncwarp();
                                if (lane == 0) dev::mbar_arrive_cluster(x_full, 1);
                            }
                            if (good) {                                  // the quadrant rows -> stage_d
#pragma unroll 1
                                for (int k = 0; k < 4; ++k) {
                                    dev::tmem_ld_32x32b_x32(ta + qcol + 32 * k, d);
                                    dev::tmem_ld_wait();
#pragma unroll
                                    for (int c = 0; c < 32; c += 4) {
                                        const uint32_t a = stage_d + 4 * off(lane, 32 * k + c);
                                        asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};"
                                                     ::"r"(a), "r"(d[c]), "r"(d[c + 1]), "r"(d[c + 2]), "r"(d[c + 3]));
                                    }
                                }
                            }
                        }
                        dev::named_sync(kEpiBar, 32 * kPairEpiWarps);
                        if (good && q >= st) {
                            // quadrant: V[i][j] for rows i = first + 32 st + r <= j; D[j][i] own (columns
                            // 32 st .. of the quadrant), D[i][j] = stage_d[r][m]
                            const bool j_ok = j < N;
#pragma unroll 1
                            for (int h = 0; h < 2; ++h) {
                                dev::tmem_ld_32x32b_x16(ta + qcol + 32 * st + 16 * h, h16);
                                dev::tmem_ld_wait();
                                const int il0 = 32 * st + 16 * h;      // rows il0 + c <= m of the quadrant
                                chunk16(base + 128 * (int)rank + il0, stage_df + 16 * h * 128,
                                        j_ok ? min(16, max(0, m - il0 + 1)) : 0, h16, add);
                            }
                        }
                        if (rank == 1) {
                            // off-diagonal quadrant: V[i][j] for CTA 0's rows i = base + 32 st + r;
                            // D[j][i] own (columns 32 st ..), D[i][j] = stage_x[r][m]
                            good = __all_sync(0xffffffffu, good && wait_cluster(x_full, x_ph));
                            if (good) {
                                const bool j_ok = j < N;
#pragma unroll 1
                                for (int h = 0; h < 2; ++h) {
                                    dev::tmem_ld_32x32b_x16(ta + 32 * st + 16 * h, h16);
                                    dev::tmem_ld_wait();
                                    chunk16(base + 32 * st + 16 * h, stage_xf + 16 * h * 128, j_ok ? 16 : 0, h16, add);
                                }
                            }
                            asm volatile("fence.acq_rel.cluster;" ::: "memory");   // the reads above, then the arrival
                            __syncwarp();
                            if (lane == 0) dev::mbar_arrive_cluster(x_empty, 0);
                        }
                        x_ph ^= 1u;
                        dev::named_sync(kEpiBar, 32 * kPairEpiWarps);     // stage_d free for the next rows
                    }
                    dev::tc_fence_before();
                    if (lane == 0) dev::mbar_arrive(&epi_done[acc]);
                    acc_ph ^= 1u << acc;
                    acc ^= 1u;
                    if (!dev::named_sync_and(kEpiBar, 32 * kPairEpiWarps, good)) { gone = true; break; }
                }
                if (gone) {                           // every epilogue warp leaves here together
                    *abort_flag = 1;
                    break;
                }
                continue;
            }
            const int rb = 2 * it.R + (int)rank;
            const int i = rb * (kBlk / 2) + O::input_of(m);
            const bool i_ok = i < N;
            const int64_t prow = (int64_t)i * N - (int64_t)i * (i - 1) / 2 - i;
            const int n_chunks = 2 * (kBlk / 32);
            if (kPackets && jb.accumulate && i_ok) {
                // packet mode: the old values this item adds to go into L2 while its MMAs run (the
                // drain of a half holds up the tensor core, a double item filling all of TMEM);
                // frame mode measured slower with the prefetch
                for (int sub = 0; sub < (dbl ? 2 : 1); ++sub) {
                    const int jc = (2 * (dbl && !twin ? it.R + sub : it.C) * kBlk) / 2 + (im_row ? 8 : 0);
                    const int32_t *vis_s = vis_f + (twin ? (size_t)sub * (size_t)npairs(N) * 2 : 0);
#pragma unroll 1
                    for (int ck = 0; ck < n_chunks; ++ck) {
                        const int j0 = max(jc + 16 * ck, i), j1 = min(jc + 16 * ck + 7, N - 1);
                        if (j0 > j1) continue;
                        dev::prefetch_l2(vis_s + 2 * (prow + j0));
                        dev::prefetch_l2(vis_s + 2 * (prow + j1));
                    }
                }
            }
            for (int k0 = 0; k0 < kt_n && ok; k0 += fl)
            for (int sub = 0; sub < (dbl ? 2 : 1); ++sub) {        // a double: block (R, R), then (R, R + 1)
                const int C = dbl && !twin ? it.R + sub : it.C;    // a twin: (R, R) of channel f, then f + 1
                const int cb0 = 2 * C;
                int32_t *vis_s = vis_f + (twin ? (size_t)sub * (size_t)npairs(N) * 2 : 0);
                if (*abort_flag || !wait(&acc_full[acc], (acc_ph >> acc) & 1u)) { ok = false; break; }
                dev::tc_fence_after();
                const bool add = jb.accumulate || k0 > 0;
                const uint32_t tb = tmem + acc * 256u + (uint32_t(q * 32) << 16);
                auto jb_of = [&](int ck) { return (cb0 * kBlk + ck * 32) / 2 + (im_row ? 8 : 0); };
                int2 old[8], nxt[8];
                int ck = half;
                if (add && ck < n_chunks) load_old(vis_s, prow, i, jb_of(ck), N, i_ok, old);
                else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) old[k] = make_int2(0, 0);
                }
                // frame mode reads the next chunk's old values after this chunk's store (a look-ahead
                // buffer would cost its 80-register converter warps); packet mode, whose epilogue drains
                // both halves of a double item, reads them ahead. (Adding through red.add in L2, as the
                // fold epilogue does, measured slower here: each warp instruction of this layout touches
                // 32 rows of the triangle.)
#pragma unroll 1
                for (; ck < n_chunks; ck += kPerQuarter) {
                    const bool more = ck + kPerQuarter < n_chunks;
                    if constexpr (kPackets) {
                        if (add && more) load_old(vis_s, prow, i, jb_of(ck + kPerQuarter), N, i_ok, nxt);
                    }
                    int vr[8], vi[8];
                    combine_chunk<true>(tb + ck * 32, im_row, vr, vi);
                    store_vis(vis_s, prow, i, jb_of(ck), N, i_ok, vr, vi, old);
                    if (add && more) {
                        if constexpr (kPackets) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) old[k] = nxt[k];
                        } else {
                            load_old(vis_s, prow, i, jb_of(ck + kPerQuarter), N, i_ok, old);
                        }
                    }
                }
                dev::tc_fence_before();
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(&epi_done[acc]);
                acc_ph ^= 1u << acc;
                acc ^= 1u;
            }
        }
    } else {
        // -------------------------------------------------------------------- converters (both CTAs)
        if constexpr (S::kRegsConv > S::kRegsLaunch) dev::setmaxnreg_inc<S::kRegsConv>();
        else if constexpr (S::kRegsConv < S::kRegsLaunch) dev::setmaxnreg_dec<S::kRegsConv>();
        // thread ctid converts inputs 16c .. 16c + 15 of samples t_row + r kRowStep (t_row = ctid / 4)
        // of each block: 16 packed bytes in, 32 E5M2 codes out into the two 16-byte chunks 2c and
        // 2c + 1 of those operand rows (128-byte swizzle; all of a thread's rows share its phase). A
        // fold item's two loads give 16 codes each for the S, A and B slots, at chunks c and 4 + c
        // (odd rows: 4 + c first).
        const int ctid = threadIdx.x - 32 * kPairConvWarp0;
        const int t_row = ctid >> 2, c = ctid & 3;
        const uint32_t dst0 = t_row * 128 + (((2 * c) ^ (t_row & 7)) << 4);
        const uint32_t dst1 = t_row * 128 + (((2 * c + 1) ^ (t_row & 7)) << 4);
        const uint32_t dsta = t_row * 128 + (((4 * (t_row & 1) + c) ^ (t_row & 7)) << 4);
        const uint32_t dstb = t_row * 128 + (((4 * (1 - (t_row & 1)) + c) ^ (t_row & 7)) << 4);
        constexpr uint32_t kRowBytes = S::kRowStep * 128;
        auto st16 = [](uint32_t a, const uint4 &v) {
            asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w));
        };
        auto convert = [&](uint32_t slot, const uint4 &v) {
            uint4 lo, hi;
            dev::expand16_e5m2(v, lo, hi);
            st16(slot + dst0, lo);
            st16(slot + dst1, hi);
        };
        auto convert_fold = [&](uint32_t row, uint32_t dst, const uint4 &v) {
            uint4 fs, fa, fb;
            dev::fold16(v, fs, fa, fb);
            st16(row + dst, fs);
            st16(row + kOpSlotBytes + dst, fa);
            st16(row + 2 * kOpSlotBytes + dst, fb);
        };
        constexpr int kOwn = PairLoader<kPackets, kShift>::kOwnMax;
        struct Buf {
            uint4 a[S::kRows], b[S::kRows];
            uint32_t own[kOwn];                       // packets of the stage this buffer receives next
            int nb;                                   // blocks of the stage it holds (0: none; 3: fold)
        };
        // samples of kBufs - 1 stages ahead are in flight while a stage is converted: kBufs buffers
        // in rotation (the loop is unrolled so that no buffer is copied); packet mode looks up a
        // stage's packets kBufs stages before its samples are loaded (right after the buffer that
        // will receive them issued its previous load)
        PairLoader<kPackets, kShift> ld, ow;
        ld.start(p, pair, rank, t_row, c);
        ow = ld;
        auto next_owners = [&](Buf &b) {
            if constexpr (kPackets) {
                if (!ow.valid(p)) return;
                ow.owners(p, b.own);
                ow.next(p, n_pairs, rank, t_row, c);
            }
        };
        auto issue = [&](Buf &b) {
            if (!ld.valid(p)) {
                b.nb = 0;
                return;
            }
            uint32_t o[S::kRows], ob[S::kRows];
#pragma unroll
            for (int r = 0; r < S::kRows; ++r) {
                o[r] = ob[r] = 0;
                if constexpr (kShift) {
                    o[r] = b.own[0];                  // this thread's own A and B row packets
                    ob[r] = b.own[1];
                } else if constexpr (kPackets) {
                    // slot (r kRowStep + t_row) / 4 of the stage: register (r kRowStep / 4) / 32,
                    // lane (r kRowStep / 4) % 32 + t_row / 4 (t_row / 4 < kRowStep / 4 <= 32); a wide
                    // stage's B rows: the same slot kKt / 4 further on (registers kOwn / 2 ..)
                    constexpr int kHalf = PairLoader<kPackets, kShift>::kOwn;
                    const int s0 = r * (S::kRowStep / 4);
                    o[r] = __shfl_sync(0xffffffffu, b.own[s0 / 32], s0 % 32 + (t_row >> 2));
                    ob[r] = o[r];
                    if (ld.wide) ob[r] = __shfl_sync(0xffffffffu, b.own[kHalf + s0 / 32], s0 % 32 + (t_row >> 2));
                }
            }
            ld.load(o, ob, b.a, b.b);
            b.nb = ld.nblk;
            ld.next(p, n_pairs, rank, t_row, c);
        };
        uint32_t os = 0, oph = 0;
        // look up the packets of lb's next stage, load the stage the rotation assigns to lb, then
        // convert stage i from cb. The lookup goes first into a register of its own: issued after
        // the sample loads into the owner register their shuffles read, it measured 8 % slower
        auto step = [&](Buf &lb, Buf &cb) -> bool {
            if (cb.nb == 0) return false;
            uint32_t nown[kOwn];
#pragma unroll
            for (int q = 0; q < kOwn; ++q) nown[q] = lb.own[q];
            if constexpr (kPackets) {
                if (ow.valid(p)) {
                    ow.owners(p, nown);
                    ow.next(p, n_pairs, rank, t_row, c);
                }
            }
            issue(lb);
#pragma unroll
            for (int q = 0; q < kOwn; ++q) lb.own[q] = nown[q];
            if (!wait(&op_empty[os], oph ^ 1)) return false;
            const uint32_t op = op_base + os * op_stage_bytes;
            if (kPackets && cb.nb == 3) {
#pragma unroll
                for (int r = 0; r < S::kRows; ++r) {
                    convert_fold(op + r * kRowBytes, dsta, cb.a[r]);
                    convert_fold(op + r * kRowBytes, dstb, cb.b[r]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < S::kRows; ++r) convert(op + r * kRowBytes, cb.a[r]);
                if (cb.nb == 2) {
#pragma unroll
                    for (int r = 0; r < S::kRows; ++r) convert(op + kOpSlotBytes + r * kRowBytes, cb.b[r]);
                }
            }
            dev::fence_proxy_async_smem();            // operand visible to the tensor core
            __syncwarp();
            if (lane == 0) {
                if constexpr (kPackets) dev::mbar_arrive_remote(&op_full[os], 0);
                else dev::mbar_arrive(&conv_done[os]);
            }
            if (++os == (uint32_t)p.op_stages) { os = 0; oph ^= 1; }
            return true;
        };
        static_assert(S::kBufs == 2, "the rotation below uses two buffers");
        Buf x, y;
#pragma unroll
        for (int q = 0; q < kOwn; ++q) x.own[q] = y.own[q] = kNoPacket;
        next_owners(x);                               // stages 0, 1
        next_owners(y);
        issue(x);
        next_owners(x);                               // stage 2
        for (;;) {
            if (!step(y, x)) break;
            if (!step(x, y)) break;
        }
    }

    dev::tc_fence_before();
    __syncthreads();
    dev::cluster_sync();                            // no CTA leaves while its pair may still signal it
    dev::tc_fence_after();
    if (warp == 1) dev::tmem_dealloc_pair(tmem, kTmemCols);
}

// ----------------------------------------------------------------------------- host side

struct JobGeom {
    int R, nb, k_tiles;
    int64_t ldy;
    size_t y_bytes;
};

static JobGeom geom(const xe_shape &s, int engine) {
    JobGeom g;
    const int kt = kt_of(engine);
    g.R = (int)round_up(2 * (int64_t)s.n_inputs, kBlk);
    g.nb = g.R / kBlk;
    g.ldy = round_up(std::max<int64_t>(s.n_time, 1), kKtMax);
    g.k_tiles = (int)((s.n_time + kt - 1) / kt);
    g.y_bytes = (engine == kFusedMN || engine == kFusedPair || engine == kLegacyS4 || engine == kLegacyS8)
                    ? 0 : (size_t)round_up((int64_t)s.n_chan * g.R * g.ldy, 1024);
    return g;
}

static int check_job(const xe_shape &s, const void *frame, const void *vis) {
    if (!valid_shape(s) || !vis || (!frame && s.n_time > 0)) return XE_EINVAL;   // T = 0 reads no frame
    if (s.n_time > XE_MAX_TIME) return XE_EOVERFLOW;
    if ((reinterpret_cast<uintptr_t>(frame) & 15) || (reinterpret_cast<uintptr_t>(vis) & 7)) return XE_EINVAL;
    return XE_OK;
}

static int engine_of(int api_engine) {
    switch (api_engine) {
        case XE_ENGINE_UNPACKED: return kUnpackedMN;
        case XE_ENGINE_FUSED: return kFusedMN;
        case XE_ENGINE_UNPACKED_K: return kUnpackedK;
        case XE_ENGINE_FUSED_PAIR: return kFusedPair;
        case XE_ENGINE_LEGACY_S4: return kLegacyS4;
        case XE_ENGINE_LEGACY_S8: return kLegacyS8;
        default: return -1;
    }
}

static void resolve_tune(const xe_tune *t, xe_tune &out) {
    out.engine = XE_ENGINE_FUSED_PAIR;
    out.max_strip = 4;
    out.k_flush = kDefaultKFlush;
    out.n_ctas = 0;
    if (!t) return;
    if (t->engine) out.engine = t->engine;
    if (t->max_strip) out.max_strip = t->max_strip;
    if (t->k_flush) out.k_flush = t->k_flush;
    out.n_ctas = t->n_ctas;
}

static int check_tune(const xe_tune &t) {
    if (engine_of(t.engine) < 0) return XE_EINVAL;
    if (t.max_strip < 1 || t.max_strip > 4) return XE_EINVAL;
    if (t.k_flush < kKtMax || t.k_flush % kKtMax || t.k_flush > kMaxKFlush) return XE_EINVAL;
    if (t.n_ctas < 0) return XE_EINVAL;
    return XE_OK;
}

// ----------------------------------------------------------------------------- tuning table

static std::mutex g_tune_mu;
static xe_tune_entry g_tune[XE_TUNE_MAX_ENTRIES];
static int g_tune_n = 0;

static int t_bucket_of(int t) {
    int b = 128;
    while (b < t && b < (1 << 30)) b <<= 1;
    return b;
}

// The table's entry for jobs of shape s, copied into *e; false if there is none. Caller holds g_tune_mu.
static bool tune_lookup(const xe_shape &s, int mode, xe_tune_entry *e) {
    const int b = t_bucket_of(s.n_time);
    for (int k = 0; k < g_tune_n; ++k)
        if (g_tune[k].n_inputs == s.n_inputs && g_tune[k].t_bucket == b && g_tune[k].mode == mode) {
            *e = g_tune[k];
            return true;
        }
    return false;
}

static constexpr size_t kWsHeader = 1024;   // work-item counter; operands start 1 KiB in

using PacketSrc = xe::packet_src;

// Packet mode needs whole 8-channel groups and whole 4-sample slots.
static bool s_chan_misfit(const xe_shape &s) { return s.n_chan % 8 != 0 || s.n_time % 4 != 0; }

static size_t batched_ws(const xe_job *jobs, int n, int engine) {
    size_t b = kWsHeader + 1024;   // + slack: the workspace is aligned up to 1 KiB inside
    for (int j = 0; j < n; ++j) b += geom(jobs[j].s, engine).y_bytes;
    return b;
}

static int launch_unpack(int engine, const uint8_t *frame, const xe_shape &s, uint8_t *y, int64_t ldy,
                         cudaStream_t st) {
    const int R = (int)round_up(2 * (int64_t)s.n_inputs, kBlk);
    if (engine == kUnpackedK) {
        dim3 grid((unsigned)(ldy / 128), (unsigned)(R / 128), (unsigned)s.n_chan);
        if (grid.x == 0 || grid.z > 65535u) return XE_EINVAL;
        unpack_k_kernel<<<grid, 256, 0, st>>>(frame, y, s.n_inputs, s.n_chan, s.n_time, R, ldy);
    } else {
        const int64_t chunks = (int64_t)s.n_chan * ldy * (R / 32);
        const int blocks = (int)std::min<int64_t>((chunks + 255) / 256, (int64_t)sm_count() * 16);
        unpack_mn_kernel<<<blocks, 256, 0, st>>>(frame, y, s.n_inputs, s.n_chan, s.n_time, R, ldy);
    }
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

template <int kEngine>
static int launch_gemm(const Params &hp, int ctas, int smem, cudaStream_t st) {
    static bool attr_set[64] = {};
    int dev = 0;
    XE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev >= 64) return XE_EINVAL;
    if (!attr_set[dev]) {
        XE_TRY_CUDA(cudaFuncSetAttribute(correlate_kernel<kEngine>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemMax));
        attr_set[dev] = true;
    }
    correlate_kernel<kEngine><<<ctas, Cfg<kEngine>::kThreads, smem, st>>>(hp);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

// Pair engine: as many 2-CTA clusters as can be resident at once (each CTA fills an SM), one per
// work item at most, at most n_ctas / 2 if n_ctas > 0.
template <bool kPackets, bool kShift = false>
static int pair_count(int items, int n_ctas, bool odd_pairs, bool keep_rounds, int *out) {
    static int max_pairs[64] = {};
    int dev = 0;
    XE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return XE_EINVAL;
    if (!max_pairs[dev]) {
        {
            // the kernel's register split (setmaxnreg) hands back exactly what it takes from the
            // registers a launch allocates; with any other allocation its increase could not be met
            cudaFuncAttributes fa{};
            XE_TRY_CUDA(cudaFuncGetAttributes(&fa, correlate_pair_kernel<kPackets, kShift>));
            if (fa.numRegs != PairShape<kPackets>::kRegsLaunch) return XE_ECUDA;
        }
        XE_TRY_CUDA(cudaFuncSetAttribute(correlate_pair_kernel<kPackets, kShift>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemMax));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * sm_count() / 2, 1, 1);
        cfg.blockDim = dim3(PairShape<kPackets>::kThreads, 1, 1);
        cfg.dynamicSmemBytes = kSmemMax;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        XE_TRY_CUDA(cudaOccupancyMaxActiveClusters(&n, correlate_pair_kernel<kPackets, kShift>, &cfg));
        max_pairs[dev] = std::max(1, n);
    }
    int pairs = std::min(items, max_pairs[dev]);
    const int rounds_all = (items + pairs - 1) / pairs;
    if (n_ctas > 0) pairs = std::max(1, std::min(pairs, n_ctas / 2));
    // a count from the tuning table was measured at the autotuner's probe size: where it adds a
    // round of work items at this launch's count, the launch takes the fewest pairs that keep the
    // rounds of a launch on all pairs instead (N = 2048, 64 channels: 68 pairs would run 128 rounds
    // of Gram blocks, 74 run 118)
    if (keep_rounds && (items + pairs - 1) / pairs > rounds_all) pairs = (items + rounds_all - 1) / rounds_all;
    // the packet-mode Gram layout interleaves doubles and singles channel by channel: an odd pair
    // count makes every pair alternate between the two kinds (fold items are all alike). One pair
    // fewer is not taken where it adds a round of work items: a full-band call of 1,024 fold items
    // runs 14 rounds on 74 pairs but 15 on 73 (4.76 against 4.4 ms)
    if (odd_pairs && pairs > 1 && pairs % 2 == 0) {
        const int rounds = (items + pairs - 1) / pairs, rounds_odd = (items + pairs - 2) / (pairs - 1);
        if (rounds_odd == rounds) --pairs;
    }
    *out = pairs;
    return XE_OK;
}

template <bool kPackets, bool kShift = false>
static int launch_pair(const Params &hp, int items, int n_ctas, int smem, bool odd_pairs, bool keep_rounds,
                       cudaStream_t st) {
    int pairs = 0;
    if (int e = pair_count<kPackets, kShift>(items, n_ctas, odd_pairs, keep_rounds, &pairs)) return e;
    correlate_pair_kernel<kPackets, kShift><<<2 * pairs, PairShape<kPackets>::kThreads, smem, st>>>(hp);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

// pk (packet mode, pair engine only): job j reads its samples from the packets pk[j] through the
// frame index pk[j].owner instead of from jobs[j].frame.
// delay16 (packet mode, one job only): the delay of each block of 16 inputs, HOST [N / 16], read
// here; the samples are read time-shifted (the kShift kernel).
static int run_batched(const xe_job *jobs, int n_jobs, const xe_tune *tune_in, void *ws, size_t ws_bytes,
                       cudaStream_t st, const PacketSrc *pk, const int32_t *delay16 = nullptr) {
    if (!jobs || n_jobs < 1 || n_jobs > XE_MAX_JOBS) return XE_EINVAL;
    if (delay16 && (!pk || n_jobs != 1)) return XE_EINVAL;
    xe_tune tune;
    resolve_tune(tune_in, tune);
    if (int e = check_tune(tune)) return e;
    const int engine = engine_of(tune.engine);
    if (pk && engine != kFusedPair) return XE_EINVAL;
    for (int j = 0; j < n_jobs; ++j) {
        const void *src = pk ? static_cast<const void *>(pk[j].pkts) : jobs[j].frame;
        if (int e = check_job(jobs[j].s, src, jobs[j].vis)) return e;
        if (pk && (!pk[j].owner || pk[j].pkt_stride % 16 || s_chan_misfit(jobs[j].s))) return XE_EINVAL;
    }
    if (engine == kLegacyS4 || engine == kLegacyS8) {   // the baseline paths: no workspace, no tcgen05
        if (!ws || ws_bytes < batched_ws(jobs, n_jobs, engine)) return XE_ENOMEM;
        return legacy::correlate_legacy(jobs, n_jobs, engine == kLegacyS8, st);
    }
    if (!ws || ws_bytes < batched_ws(jobs, n_jobs, engine)) return XE_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return XE_EINVAL;
    int *status = status_word();
    if (!status) return XE_ECUDA;

    // the tuning table's entries of the jobs (pair engine); the launch-wide choices come from the
    // entry of the job with the most work
    xe_tune_entry ent[XE_MAX_JOBS];
    bool has_ent[XE_MAX_JOBS] = {};
    xe_tune_entry launch_ent{};
    bool has_launch_ent = false;
    bool pairs_from_table = false;
    if (engine == kFusedPair) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        double best = -1.0;
        for (int j = 0; j < n_jobs; ++j) {
            has_ent[j] = tune_lookup(jobs[j].s, pk ? XE_TUNE_PACKETS : XE_TUNE_FRAMES, &ent[j]);
            const double w = (double)jobs[j].s.n_chan * (double)npairs(jobs[j].s.n_inputs) * (double)jobs[j].s.n_time;
            if (w > best) {
                best = w;
                has_launch_ent = has_ent[j];
                if (has_ent[j]) launch_ent = ent[j];
            }
        }
    }
    if (has_launch_ent) {
        if (!(tune_in && tune_in->k_flush) && launch_ent.k_flush) tune.k_flush = launch_ent.k_flush;
        if (!(tune_in && tune_in->n_ctas) && launch_ent.pairs) {
            tune.n_ctas = 2 * launch_ent.pairs;
            pairs_from_table = true;
        }
    }
    // The pair engine's 128-sample kernel (the packet-mode kernel) also reads assembled frames, in
    // 4-sample slots (whole slots only: T % 4 == 0), with every item layout. A frame launch takes it
    // when the table's entry of its largest job names one of its layouts; without an entry, when
    // that job has 129 to 256 inputs (one fold item per channel: measured 0.20 against 0.22 ms for
    // 64 channels of T = 16384, where at N = 1024 or 2048 the off-diagonal blocks' conversions make
    // it 1.6-1.9 times slower than the 256-sample kernel)
    bool rows128 = pk != nullptr;
    if (!pk && engine == kFusedPair) {
        if (has_launch_ent) {
            rows128 = launch_ent.layout != XE_LAYOUT_FRAME_BLOCKS;
        } else {
            int big = 0;
            double best = -1.0;
            for (int j = 0; j < n_jobs; ++j) {
                const double w = (double)jobs[j].s.n_chan * (double)npairs(jobs[j].s.n_inputs) * (double)jobs[j].s.n_time;
                if (w > best) { best = w; big = j; }
            }
            rows128 = jobs[big].s.n_inputs > 128 && jobs[big].s.n_inputs <= 256;
        }
        for (int j = 0; j < n_jobs; ++j) rows128 = rows128 && jobs[j].s.n_time % 4 == 0;
    }

    static Params hp;    // large; built under a lock
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    std::memset(&hp, 0, sizeof(hp));
    if (delay16) std::memcpy(hp.delay16, delay16, sizeof(int32_t) * (size_t)(jobs[0].s.n_inputs / 16));
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    int *counter = reinterpret_cast<int *>(base);
    uint8_t *ybase = base + kWsHeader;
    int items = 0, nj = 0, ms_max = 1;
    int job_layout[XE_MAX_JOBS] = {};
    for (int j = 0; j < n_jobs; ++j) {
        const xe_shape &s = jobs[j].s;
        const JobGeom g = geom(s, engine);
        uint8_t *y = ybase;
        ybase += g.y_bytes;
        if (s.n_time == 0) {     // empty integration: V = 0
            if (!jobs[j].accumulate)
                XE_TRY_CUDA(cudaMemsetAsync(jobs[j].vis, 0, (size_t)s.n_chan * npairs(s.n_inputs) * 8, st));
            continue;
        }
        Job &d = hp.jobs[nj++];
        int enc;
        if (pk) {
            d.pkts = pk[j].pkts;
            d.owner = pk[j].owner;
            d.pkt_stride = pk[j].pkt_stride;
            d.pw = 64;
            enc = XE_OK;
        } else if (rows128) {                   // frame rows through the 128-sample kernel
            hp.frame_rows = 1;
            d.pkts = nullptr;
            d.owner = nullptr;
            d.pkt_stride = 0;
            d.pw = 64;
            enc = XE_OK;
        } else if (engine == kFusedMN || engine == kFusedPair) {
            const uint32_t pw = (uint32_t)std::min(64, s.n_inputs);
            const uint64_t dims[3] = {(uint64_t)s.n_inputs, (uint64_t)s.n_chan, (uint64_t)s.n_time};
            const uint64_t strides[2] = {(uint64_t)s.n_inputs, (uint64_t)s.n_inputs * s.n_chan};
            const uint32_t box[3] = {pw, 1, (uint32_t)kt_of(engine)};
            enc = encode_tiled(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(jobs[j].frame), dims,
                               strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
            d.pw = (int)pw;
        } else {
            if (int e = launch_unpack(engine, jobs[j].frame, s, y, g.ldy, st)) return e;
            if (engine == kUnpackedMN) {
                const uint32_t box[3] = {kBlk, (uint32_t)kKtMN, 1};
                const uint64_t dims[3] = {(uint64_t)g.R, (uint64_t)g.ldy, (uint64_t)s.n_chan};
                const uint64_t strides[2] = {(uint64_t)g.R, (uint64_t)g.R * g.ldy};
                enc = encode_tiled(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, y, dims, strides, box,
                                   CU_TENSOR_MAP_SWIZZLE_128B);
            } else {
                const uint32_t box[3] = {(uint32_t)kKtMax, kBlk, 1};
                const uint64_t dims[3] = {(uint64_t)g.ldy, (uint64_t)g.R, (uint64_t)s.n_chan};
                const uint64_t strides[2] = {(uint64_t)g.ldy, (uint64_t)g.ldy * g.R};
                enc = encode_tiled(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, y, dims, strides, box,
                                   CU_TENSOR_MAP_SWIZZLE_128B);
            }
            d.pw = 64;
        }
        if (enc != XE_OK) return XE_EINVAL;
        d.vis = jobs[j].vis;
        d.frame = static_cast<const uint8_t *>(jobs[j].frame);
        d.n_inputs = s.n_inputs;
        d.n_chan = s.n_chan;
        d.n_time = s.n_time;
        d.accumulate = jobs[j].accumulate ? 1 : 0;
        int64_t job_items = 0;
        if (engine == kFusedPair) {             // 256x256 blocks on or above the diagonal
            d.nb = (g.nb + 1) / 2;
            d.fold = 0;
            int layout = has_ent[j] ? ent[j].layout : XE_LAYOUT_AUTO;
            if (layout == XE_LAYOUT_FRAME_BLOCKS) layout = XE_LAYOUT_AUTO;   // a job in a 128-sample launch
            job_layout[nj - 1] = layout;
            if (rows128 && d.nb >= 2 &&
                (layout == XE_LAYOUT_AUTO || layout == XE_LAYOUT_FOLD || layout == XE_LAYOUT_FOLD_SPLIT)) {
                // fold layout: per channel S2 / 2 fold items, a Gram diagonal single for an odd last
                // block, and the Gram blocks (R, C) between different super-blocks (R / 2 < C / 2)
                d.fold = 1;
                d.doubles = 0;
                d.offdiag = 0;
                d.twin = 0;
                int per_ch = d.nb / 2 + (d.nb & 1);
                for (int r = 0; r < d.nb; ++r) per_ch += std::max(0, d.nb - 2 * (r / 2 + 1));
                d.strips = per_ch;
                job_items = (int64_t)d.strips * s.n_chan;
            } else if (rows128) {
                // per channel S2 - 1 doubles and (S2 - 1)(S2 - 2) / 2 singles; then long
                // integrations take the last diagonal blocks of channel pairs as twins (an odd last
                // channel keeps its diagonal single), short ones each channel's as a wide single
                d.doubles = d.nb - 1;
                d.offdiag = (d.nb - 1) * (d.nb - 2) / 2;
                d.twin = layout == XE_LAYOUT_GRAM_TWIN ? 1
                         : layout == XE_LAYOUT_GRAM_WIDE ? 0
                         : (s.n_time >= kTwinMinTime ? 1 : 0);
                if (d.twin) {
                    d.strips = 2 * (d.doubles + d.offdiag) + 1;
                    job_items = (int64_t)(s.n_chan / 2) * d.strips + (s.n_chan % 2) * (d.doubles + d.offdiag + 1);
                } else {
                    d.strips = d.doubles + d.offdiag + 1;
                    job_items = (int64_t)d.strips * s.n_chan;
                }
            } else {
                d.doubles = 0;
                d.offdiag = 0;
                d.twin = 0;
                d.strips = d.nb * (d.nb + 1) / 2;
                job_items = (int64_t)d.strips * s.n_chan;
            }
            d.max_strip = 2;
        } else {
            d.nb = g.nb;
            d.max_strip = jobs[j].max_strip > 0 ? jobs[j].max_strip : tune.max_strip;
            if (d.max_strip > 4) return XE_EINVAL;
            ms_max = std::max(ms_max, d.max_strip);
            d.strips = strips_per_channel(g.nb, d.max_strip);
            job_items = (int64_t)d.strips * s.n_chan;
        }
        d.k_tiles = (int)((s.n_time + kt_of(engine, rows128) - 1) / kt_of(engine, rows128));
        // 128-sample kernel: single diagonal blocks run in stages of twice the samples
        const int kt_wide = 2 * kt_of(engine, rows128);
        d.k_tiles_wide = engine == kFusedPair && rows128 ? (int)((s.n_time + kt_wide - 1) / kt_wide) : d.k_tiles;
        d.item_begin = items;
        if (items + job_items > INT32_MAX / 2) return XE_EINVAL;
        items += (int)job_items;
    }
    if (nj == 0) return XE_OK;
    hp.n_jobs = nj;
    hp.n_items = items;
    // drain at least once per stage; a stage (<= 256 samples) never exceeds the exactness bound
    hp.k_flush_tiles = std::max(1, tune.k_flush / kt_of(engine, rows128));
    // wide stages (2 x 128 samples) stay within the exactness bound like any stage of <= 256 samples
    hp.wide_diag = engine == kFusedPair && rows128 ? 1 : 0;
    hp.k_flush_tiles_wide = hp.wide_diag ? std::max(1, tune.k_flush / (2 * kt_of(engine, true))) : hp.k_flush_tiles;
    hp.slots = ms_max == 1 ? 2 : (ms_max == 2 ? 3 : 4);     // operand blocks per stage for the widest strip
    hp.n_acc = ms_max <= 2 ? 2 : 1;                        // TMEM accumulators (each <= 256 columns)
    hp.status = status;
    hp.counter = counter;
    hp.limit_ns = wait_limit_ns();
    const int bar_bytes = 1024;
    const int avail = kSmemMax - 1024 - bar_bytes;
    const int op_slot = kBlk * kt_of(engine, rows128), pk_slot = 64 * kt_of(engine);
    int staging = 0;
    bool all_fold = nj > 0;
    for (int j = 0; j < nj; ++j) {
        hp.fold |= hp.jobs[j].fold;
        all_fold = all_fold && hp.jobs[j].fold;
    }
    if (engine == kFusedPair) {
        // fold items need three operand slots per stage and the epilogue's transpose staging. The
        // ring is as deep as fits in kPairSmemBudget: beyond it the SM takes its largest
        // shared-memory carve-out, and the L1 left over (28 instead of 60 KB) no longer holds the
        // converters' samples in flight (~48 KB per SM): measured 5.9 against 4.3 ms per
        // full-band 8-frame call with the same four stages (fold layout)
        hp.slots = hp.fold ? kFoldSlots : kPairSlots;
        staging = hp.fold ? kFoldStageBytes : 0;
        hp.n_acc = 2;
        hp.pk_stages = 0;
        hp.op_stages = std::min(kPairMaxStages, (kPairSmemBudget - 1024 - bar_bytes - staging) / (hp.slots * op_slot));
    } else if (engine == kFusedMN) {
        hp.pk_stages = 3;
        hp.op_stages = std::min(8, (avail - hp.pk_stages * hp.slots * pk_slot) / (hp.slots * op_slot));
    } else {
        hp.pk_stages = 0;
        hp.op_stages = std::min(8, avail / (hp.slots * op_slot));
    }
    if (hp.op_stages < 2) return XE_EINVAL;
    const int smem = 1024 + hp.op_stages * hp.slots * op_slot + hp.pk_stages * hp.slots * pk_slot + bar_bytes + staging;
    XE_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    if (engine == kFusedPair)
    {
        // the Gram layout's doubles and singles alternate best on an odd pair count; fold items are alike
        bool odd = rows128 && !all_fold;
        if (has_launch_ent && launch_ent.odd_pairs >= 0) odd = launch_ent.odd_pairs == 1;
        if (!rows128) return launch_pair<false>(hp, items, tune.n_ctas, smem, odd, pairs_from_table, st);
        // Balanced split: a launch of one job whose channels are one fold item each (129-256
        // inputs) hands every pair an equal share of the job's channel x stage range, as pieces of
        // consecutive channels, when whole items would leave more than a tenth of the last round's
        // pairs idle in a launch of two or more rounds, or always with XE_LAYOUT_FOLD_SPLIT. A
        // launch of one round takes one pair per item: configuration 2's 64 channels on 64 pairs
        // take 0.168 ms, split over all 74 pairs 0.178 ms (two drains per pair, reductions into
        // cleared visibilities). Pieces add their sums with L2 reductions, so a call that does not
        // accumulate first clears its visibilities.
        Job &d0 = hp.jobs[0];
        if (nj == 1 && d0.fold && d0.nb == 2) {
            const int64_t total = (int64_t)d0.n_chan * d0.k_tiles;
            int pairs = 0;
            if (int e = pair_count<true>(items, tune.n_ctas, false, pairs_from_table, &pairs)) return e;
            const int rounds = (items + pairs - 1) / pairs;
            const bool ragged = (double)items < 0.9 * (double)rounds * (double)pairs;
            if (job_layout[0] == XE_LAYOUT_FOLD_SPLIT || ragged) {
                hp.split_pairs = pairs;
                hp.split_u = (int)((total + pairs - 1) / pairs);
                hp.split_items = (hp.split_u + d0.k_tiles - 1) / d0.k_tiles + 1;
                if ((int64_t)pairs * hp.split_items > INT32_MAX / 2) return XE_EINVAL;
                hp.n_items = items = pairs * hp.split_items;
                if (!d0.accumulate) {
                    XE_TRY_CUDA(cudaMemsetAsync(d0.vis, 0, (size_t)d0.n_chan * npairs(d0.n_inputs) * 8, st));
                    d0.accumulate = 1;
                }
                if (delay16) return launch_pair<true, true>(hp, items, 2 * pairs, smem, false, false, st);
                return launch_pair<true>(hp, items, 2 * pairs, smem, false, false, st);
            }
        }
        if (delay16) return launch_pair<true, true>(hp, items, tune.n_ctas, smem, odd, pairs_from_table, st);
        return launch_pair<true>(hp, items, tune.n_ctas, smem, odd, pairs_from_table, st);
    }
    const int ctas = std::min(items, tune.n_ctas > 0 ? tune.n_ctas : sm_count());
    switch (engine) {
        case kUnpackedK: return launch_gemm<kUnpackedK>(hp, ctas, smem, st);
        case kUnpackedMN: return launch_gemm<kUnpackedMN>(hp, ctas, smem, st);
        default: return launch_gemm<kFusedMN>(hp, ctas, smem, st);
    }
}

}  // namespace corr
}  // namespace xe

int xe::correlate_packets_batched(const xe_job *jobs, const packet_src *src, int n_jobs, void *ws, size_t ws_bytes,
                                  cudaStream_t st) {
    if (!src) return XE_EINVAL;
    return corr::run_batched(jobs, n_jobs, nullptr, ws, ws_bytes, st, src);
}

using namespace xe;

extern "C" {

int xe_unpack(const uint8_t *frame, xe_shape s, uint8_t *y, int64_t ldy, void *stream) {
    if (!valid_shape(s) || !frame || !y || ldy < std::max(s.n_time, 1) || ldy % 128) return XE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(frame) & 15) || (reinterpret_cast<uintptr_t>(y) & 15)) return XE_EINVAL;
    return corr::launch_unpack(corr::kUnpackedMN, frame, s, y, ldy, static_cast<cudaStream_t>(stream));
}

size_t xe_correlate_workspace_size(xe_shape s) {
    if (!valid_shape(s)) return 0;
    xe_job j{nullptr, nullptr, s, 0, 0};
    return corr::batched_ws(&j, 1, corr::engine_of(XE_ENGINE_FUSED_PAIR));
}

int xe_correlate(const uint8_t *frame, xe_shape s, int32_t *vis, int accumulate, void *ws, size_t ws_bytes,
                 void *stream) {
    xe_job j{frame, vis, s, accumulate ? 1 : 0, 0};
    return corr::run_batched(&j, 1, nullptr, ws, ws_bytes, static_cast<cudaStream_t>(stream), nullptr);
}

int xe_tune_table_set(const xe_tune_entry *entries, int32_t n) {
    if (n < 0 || n > XE_TUNE_MAX_ENTRIES || (n > 0 && !entries)) return XE_EINVAL;
    for (int k = 0; k < n; ++k) {
        const xe_tune_entry &e = entries[k];
        const bool pow2 = e.t_bucket >= 128 && (e.t_bucket & (e.t_bucket - 1)) == 0;
        if (e.n_inputs < 16 || e.n_inputs > 4096 || e.n_inputs % 16 || !pow2 || e.mode < XE_TUNE_PACKETS ||
            e.mode > XE_TUNE_FRAMES || e.layout < XE_LAYOUT_AUTO ||
            e.layout > XE_LAYOUT_FOLD_SPLIT || (e.layout == XE_LAYOUT_FRAME_BLOCKS && e.mode != XE_TUNE_FRAMES) ||
            e.pairs < 0 || e.pairs > 4096 || e.odd_pairs < -1 || e.odd_pairs > 1 ||
            e.k_flush < 0 || e.k_flush > corr::kMaxKFlush || e.k_flush % corr::kKtMax)
            return XE_EINVAL;
        for (int k2 = 0; k2 < k; ++k2)
            if (entries[k2].n_inputs == e.n_inputs && entries[k2].t_bucket == e.t_bucket && entries[k2].mode == e.mode)
                return XE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(corr::g_tune_mu);
    for (int k = 0; k < n; ++k) corr::g_tune[k] = entries[k];
    corr::g_tune_n = n;
    return XE_OK;
}

int xe_tune_table_get(xe_tune_entry *out, int32_t cap) {
    std::lock_guard<std::mutex> lk(corr::g_tune_mu);
    if (out)
        for (int k = 0; k < std::min<int>(cap, corr::g_tune_n); ++k) out[k] = corr::g_tune[k];
    return corr::g_tune_n;
}

size_t xe_correlate_batched_workspace_size(const xe_job *jobs, int32_t n_jobs, const xe_tune *tune) {
    if (!jobs || n_jobs < 1 || n_jobs > XE_MAX_JOBS) return 0;
    for (int j = 0; j < n_jobs; ++j)
        if (!valid_shape(jobs[j].s)) return 0;
    xe_tune t;
    corr::resolve_tune(tune, t);
    const int e = corr::engine_of(t.engine);
    if (e < 0) return 0;
    return corr::batched_ws(jobs, n_jobs, e);
}

int xe_correlate_batched(const xe_job *jobs, int32_t n_jobs, const xe_tune *tune, void *ws, size_t ws_bytes,
                         void *stream) {
    return corr::run_batched(jobs, n_jobs, tune, ws, ws_bytes, static_cast<cudaStream_t>(stream), nullptr);
}

size_t xe_correlate_packets_workspace_size(xe_shape s) {
    if (!valid_shape(s) || s.n_time % 4 || s.n_chan % 8) return 0;
    xe_job j{nullptr, nullptr, s, 0, 0};
    const size_t owner_bytes = (size_t)round_up((int64_t)(s.n_time / 4) * (s.n_chan / 8) * 4, 1024);
    return 1024 + owner_bytes + corr::batched_ws(&j, 1, corr::engine_of(XE_ENGINE_FUSED_PAIR));
}

int xe_correlate_packets(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                         xe_shape s, int32_t *vis, int accumulate, uint8_t *filled, uint32_t *lost, uint32_t *stats,
                         void *ws, size_t ws_bytes, void *stream) {
    const size_t need = xe_correlate_packets_workspace_size(s);
    if (need == 0) return XE_EINVAL;
    if (!ws || ws_bytes < need) return XE_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    const size_t owner_bytes = (size_t)round_up((int64_t)(s.n_time / 4) * (s.n_chan / 8) * 4, 1024);
    uint32_t *owner = reinterpret_cast<uint32_t *>(base);
    if (int e = xe::index_streams(pkts, n_pkts, pkt_stride, seq0, gps, 0, s, filled, lost, stats, owner, st)) return e;
    // an empty packet buffer still yields a (zero) integration: point the gather at a valid address
    xe::packet_src src{n_pkts ? pkts : base, owner, pkt_stride};
    xe_job j{nullptr, vis, s, accumulate ? 1 : 0, 0};
    const size_t used = (size_t)(base - static_cast<uint8_t *>(ws)) + owner_bytes;
    return corr::run_batched(&j, 1, nullptr, base + owner_bytes, ws_bytes - used, st, &src);
}

int xe_correlate_packets_shifted(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                                 int32_t gps, xe_shape s, const int32_t *delays, int32_t *vis, int accumulate,
                                 uint8_t *filled, uint32_t *lost, uint32_t *stats, void *ws, size_t ws_bytes,
                                 void *stream) {
    const size_t need = xe_correlate_packets_workspace_size(s);
    if (need == 0 || !delays) return XE_EINVAL;
    // one delay per block of 16 inputs, within the frame
    int32_t d16[XE_MAX_INPUTS / 16];
    for (int b = 0; b < s.n_inputs / 16; ++b) {
        d16[b] = delays[16 * b];
        if (d16[b] < 0 || d16[b] > s.n_time) return XE_EINVAL;
        for (int k = 1; k < 16; ++k)
            if (delays[16 * b + k] != d16[b]) return XE_EINVAL;
    }
    if (!ws || ws_bytes < need) return XE_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    const size_t owner_bytes = (size_t)round_up((int64_t)(s.n_time / 4) * (s.n_chan / 8) * 4, 1024);
    uint32_t *owner = reinterpret_cast<uint32_t *>(base);
    if (int e = xe::index_streams(pkts, n_pkts, pkt_stride, seq0, gps, 0, s, filled, lost, stats, owner, st)) return e;
    xe::packet_src src{n_pkts ? pkts : base, owner, pkt_stride};
    xe_job j{nullptr, vis, s, accumulate ? 1 : 0, 0};
    const size_t used = (size_t)(base - static_cast<uint8_t *>(ws)) + owner_bytes;
    return corr::run_batched(&j, 1, nullptr, base + owner_bytes, ws_bytes - used, st, &src, d16);
}

}  // extern "C"
