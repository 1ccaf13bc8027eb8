// xe_correlate.cu -- A2 unpack and A3/A4 correlation (tcgen05 tensor cores, exact integers).
//
// Method (Sec. I, Sec. II-B): for every channel f, V_f[i,j] = sum_t x_i(t) conj(x_j(t)), i <= j.
// With x = a + ib and the real matrix Y_f whose row 2n is a_n(t) and row 2n+1 is b_n(t), the Gram
// matrix G = Y Y^T holds every real product sum, and
//     Re V[i,j] = G[2i,2j] + G[2i+1,2j+1],     Im V[i,j] = G[2i+1,2j] - G[2i,2j+1].
// G is computed on the tensor cores with tcgen05.mma kind::f8f6f4: the 4-bit integers -8..7 are
// exact as FP8 E5M2, their products (|p| <= 64) and every partial sum below 2^24 are exact in the
// FP32 accumulator held in tensor memory, and the accumulator is drained to int32 at least every
// k_flush samples. Only 128x128 tiles of G on or above the block diagonal are computed.
//
// Kernel roles (one persistent CTA per SM, 6 warps):
//   warp 0      TMA producer: 128x128-byte tiles of Y (one per 128-row block) into a 3-stage ring
//   warp 1      TMEM owner and MMA issuer (one thread): 4 MMAs of K=32 per block pair per stage
//   warps 2..5  epilogue: tcgen05.ld of the FP32 tile, FP32 -> int32, 2x2 Re/Im combine across
//               lane pairs with shfl.xor, store / accumulate into the packed triangle
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "xe_device.cuh"
#include "xe_internal.h"

namespace xe {
namespace corr {

constexpr int kBlk = 128;                         // rows per operand block = MMA M = N
constexpr int kKt = 128;                          // time samples per pipeline stage (128 B row)
constexpr int kTileBytes = kBlk * kKt;            // 16 KiB per operand block per stage
constexpr int kMaxBlocksPerStage = 4;
constexpr int kStageBytes = kTileBytes * kMaxBlocksPerStage;
constexpr int kStages = 3;
constexpr int kThreads = 192;
constexpr int kTmemCols = 512;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kDefaultKFlush = 1 << 17;           // samples; 64 * 2^17 = 2^23 < 2^24

struct Job {   // 128-byte aligned through its CUtensorMap
    CUtensorMap tmap;        // Y operand [F][R][ldy] bytes, box 128 x 128 x 1, 128-byte swizzle
    int32_t *vis;
    int32_t n_inputs, n_chan, n_time, accumulate;
    int32_t nb;              // 128-row operand blocks (R / 128)
    int32_t strips;          // work items per channel
    int32_t k_tiles;         // ceil(T / 128)
    int32_t item_begin;      // first global work-item index of this job
};

struct Params {
    Job jobs[XE_MAX_JOBS];
    int32_t n_jobs, n_items, max_strip, k_flush_tiles;
    int *status;
    uint64_t limit_ns;
};

// ----------------------------------------------------------------------------- work items
// A work item is (job, channel, strip); a strip is a run of up to max_strip tiles along one
// block row rb, starting at column block cb0 >= rb. The diagonal strip of row rb starts at
// cb0 = rb (its A operand is its own first B block); further strips hold at most 3 tiles so that
// A plus the B blocks fit the 4 operand slots of a stage.

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
};

__device__ __forceinline__ Item decode_item(const Params &p, int g) {
    Item it;
    int j = 0;
    while (j + 1 < p.n_jobs && g >= p.jobs[j + 1].item_begin) ++j;
    const Job &jb = p.jobs[j];
    const int l = g - jb.item_begin;
    it.job = j;
    it.f = l % jb.n_chan;
    decode_strip(l / jb.n_chan, jb.nb, p.max_strip, it.rb, it.cb0, it.w);
    return it;
}

// ----------------------------------------------------------------------------- A2 unpack

// grid (ldy/128, R/128, F), 256 threads: a 128-sample x 64-input byte tile of the frame is staged
// in shared memory, then written as 128 rows (2n = Re, 2n+1 = Im) of 128 E5M2 codes.
__global__ void __launch_bounds__(256) unpack_kernel(const uint8_t *__restrict__ frame,
                                                     uint8_t *__restrict__ y, int N, int F, int T,
                                                     int R, int64_t ldy) {
    __shared__ uint32_t tile[128][17];        // [t][n/4] packed bytes, padded row
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
        const int row = k >> 3, c = k & 7;    // out row 2*nl + comp, 16-sample chunk c
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

// ----------------------------------------------------------------------------- epilogue

// Drains 32 TMEM columns (16 column pairs j) of this thread's lane (one row of G) and writes the
// 8 complex visibilities this thread owns: even lanes (row 2i) take the first 8 j, odd lanes
// (row 2i+1) the last 8; each obtains the other row's two values per j from its lane partner.
__device__ __forceinline__ void drain_chunk(uint32_t taddr, int32_t *__restrict__ vis_f, int N, int i,
                                            bool odd, int j0, bool add) {
    uint32_t r[32];
    dev::tmem_ld_32x32b_x32(taddr, r);
    dev::tmem_ld_wait();
    int g[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) g[k] = __float2int_rn(__uint_as_float(r[k]));
    int vr[8], vi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int s0 = odd ? g[2 * k] : g[16 + 2 * k];
        const int s1 = odd ? g[2 * k + 1] : g[16 + 2 * k + 1];
        const int r0 = __shfl_xor_sync(0xffffffffu, s0, 1);
        const int r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
        if (!odd) {   // j = j0 + k: G[2i,2j] = g[2k], G[2i,2j+1] = g[2k+1]; partner row 2i+1: r0, r1
            vr[k] = g[2 * k] + r1;
            vi[k] = r0 - g[2 * k + 1];
        } else {      // j = j0 + 8 + k: G[2i+1,2j] = g[16+2k], G[2i+1,2j+1] = g[17+2k]; partner: r0, r1
            vr[k] = r0 + g[16 + 2 * k + 1];
            vi[k] = g[16 + 2 * k] - r1;
        }
    }
    if (i >= N) return;
    const int jb = j0 + (odd ? 8 : 0);
    const int64_t prow = (int64_t)i * N - (int64_t)i * (i - 1) / 2 - i;   // p(i, j) = prow + j
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int j = jb + k;
        if (j >= i && j < N) {
            int2 *dst = reinterpret_cast<int2 *>(vis_f + 2 * (prow + j));
            int2 v = make_int2(vr[k], vi[k]);
            if (add) {
                const int2 o = *dst;
                v.x += o.x;
                v.y += o.y;
            }
            *dst = v;
        }
    }
}

// ----------------------------------------------------------------------------- GEMM kernel

__global__ void __launch_bounds__(kThreads, 1) correlate_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *full = bars;                       // [kStages] TMA -> MMA
    uint64_t *empty = bars + kStages;            // [kStages] MMA -> TMA
    uint64_t *acc_full = bars + 2 * kStages;     // MMA -> epilogue
    uint64_t *acc_empty = acc_full + 1;          // epilogue -> MMA
    uint64_t *done = acc_full + 2;               // teardown
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t smem_base = dev::smem_u32(smem);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            dev::mbar_init(&full[s], 1);
            dev::mbar_init(&empty[s], 1);
        }
        dev::mbar_init(acc_full, 1);
        dev::mbar_init(acc_empty, 4);
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

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------------- TMA producer
            uint32_t stage = 0, phase = 0;
            uint32_t issued = 0, issued_parity = 0;   // per-stage bit masks
            bool ok = true;
            for (int g = blockIdx.x; g < p.n_items && ok; g += gridDim.x) {
                const Item it = decode_item(p, g);
                const Job &jb = p.jobs[it.job];
                int blk[4];
                int nblk = it.w;
                for (int c = 0; c < it.w; ++c) blk[c] = it.cb0 + c;
                if (it.rb < it.cb0) blk[nblk++] = it.rb;
                for (int kt = 0; kt < jb.k_tiles; ++kt) {
                    if (!wait(&empty[stage], phase ^ 1)) { ok = false; break; }
                    dev::mbar_arrive_expect_tx(&full[stage], nblk * kTileBytes);
                    for (int b = 0; b < nblk; ++b)
                        dev::tma_load_3d(smem_base + stage * kStageBytes + b * kTileBytes, &jb.tmap, &full[stage],
                                         kt * kKt, blk[b] * kBlk, it.f);
                    issued |= 1u << stage;
                    issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == kStages) { stage = 0; phase ^= 1; }
                }
            }
            // copies still in flight land before the CTA exits
            for (int s = 0; s < kStages; ++s)
                if (issued & (1u << s)) dev::mbar_wait(&full[s], (issued_parity >> s) & 1u, p.limit_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------------------- MMA issuer
            constexpr uint32_t idesc = dev::idesc_e5m2_f32(kBlk, kBlk);
            uint32_t stage = 0, phase = 0, acc_phase = 0;
            bool ok = true;
            for (int g = blockIdx.x; g < p.n_items && ok; g += gridDim.x) {
                const Item it = decode_item(p, g);
                const Job &jb = p.jobs[it.job];
                const int a_slot = it.rb < it.cb0 ? it.w : 0;
                for (int k0 = 0; k0 < jb.k_tiles && ok; k0 += p.k_flush_tiles) {
                    const int k1 = min(jb.k_tiles, k0 + p.k_flush_tiles);
                    if (!wait(acc_empty, acc_phase ^ 1)) { ok = false; break; }
                    dev::tc_fence_after();
                    for (int kt = k0; kt < k1; ++kt) {
                        if (!wait(&full[stage], phase)) { ok = false; break; }
                        dev::tc_fence_after();
                        const uint32_t sb = smem_base + stage * kStageBytes;
                        const uint64_t a0 = dev::sdesc_k_sw128(sb + a_slot * kTileBytes);
                        for (int c = 0; c < it.w; ++c) {
                            const uint64_t b0 = dev::sdesc_k_sw128(sb + c * kTileBytes);
#pragma unroll
                            for (int kk = 0; kk < kKt / 32; ++kk)   // K = 32 bytes per MMA: +2 in addr>>4
                                dev::mma_f8f6f4(tmem + c * kBlk, a0 + 2 * kk, b0 + 2 * kk, idesc,
                                                (kt > k0 || kk > 0) ? 1u : 0u);
                        }
                        dev::tc_commit(&empty[stage]);
                        if (++stage == kStages) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    dev::tc_commit(acc_full);
                    acc_phase ^= 1;
                }
            }
            dev::tc_commit(done);
            dev::mbar_wait(done, 0, p.limit_ns);
        }
    } else {
        // -------------------------------------------------------------------- epilogue warps
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int m = q * 32 + lane;            // row of the 128x128 tile
        const bool odd = (m & 1) != 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int g = blockIdx.x; g < p.n_items && ok; g += gridDim.x) {
            const Item it = decode_item(p, g);
            const Job &jb = p.jobs[it.job];
            const int N = jb.n_inputs;
            const int i = (it.rb * kBlk + m) >> 1;
            int32_t *vis_f = jb.vis + (size_t)it.f * (size_t)npairs(N) * 2;
            for (int k0 = 0; k0 < jb.k_tiles; k0 += p.k_flush_tiles) {
                if (!wait(acc_full, acc_phase)) { ok = false; break; }
                dev::tc_fence_after();
                const bool add = jb.accumulate || k0 > 0;
                for (int c = 0; c < it.w; ++c)
#pragma unroll 1
                    for (int ch = 0; ch < kBlk / 32; ++ch)
                        drain_chunk(tmem + (uint32_t(q * 32) << 16) + c * kBlk + ch * 32, vis_f, N, i, odd,
                                    ((it.cb0 + c) * kBlk + ch * 32) >> 1, add);
                dev::tc_fence_before();
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(acc_empty);
                acc_phase ^= 1;
            }
        }
    }

    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    if (warp == 1) dev::tmem_dealloc(tmem, kTmemCols);
}

// ----------------------------------------------------------------------------- host side

struct JobGeom {
    int R, nb, k_tiles;
    int64_t ldy;
    size_t y_bytes;
};

static JobGeom geom(const xe_shape &s) {
    JobGeom g;
    g.R = (int)round_up(2 * (int64_t)s.n_inputs, kBlk);
    g.nb = g.R / kBlk;
    g.ldy = round_up(std::max<int64_t>(s.n_time, 1), kKt);
    g.k_tiles = (int)((s.n_time + kKt - 1) / kKt);
    g.y_bytes = (size_t)round_up((int64_t)s.n_chan * g.R * g.ldy, 1024);
    return g;
}

static int check_job(const xe_shape &s, const void *frame, const void *vis) {
    if (!valid_shape(s) || !vis || (!frame && s.n_time > 0)) return XE_EINVAL;   // T = 0 reads no frame
    if (s.n_time > XE_MAX_TIME) return XE_EOVERFLOW;
    if ((reinterpret_cast<uintptr_t>(frame) & 15) || (reinterpret_cast<uintptr_t>(vis) & 7)) return XE_EINVAL;
    return XE_OK;
}

static void resolve_tune(const xe_tune *t, xe_tune &out) {
    out.engine = XE_ENGINE_UNPACKED;
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
    if (t.engine != XE_ENGINE_UNPACKED) return XE_EINVAL;
    if (t.max_strip < 1 || t.max_strip > 4) return XE_EINVAL;
    if (t.k_flush < kKt || t.k_flush % kKt || t.k_flush > (1 << 18)) return XE_EINVAL;
    if (t.n_ctas < 0) return XE_EINVAL;
    return XE_OK;
}

static size_t batched_ws(const xe_job *jobs, int n) {
    size_t b = 1024;     // slack: the operand base is aligned up to 1 KiB inside the workspace
    for (int j = 0; j < n; ++j) b += geom(jobs[j].s).y_bytes;
    return b;
}

static int launch_unpack(const uint8_t *frame, const xe_shape &s, uint8_t *y, int64_t ldy, cudaStream_t st) {
    const int R = (int)round_up(2 * (int64_t)s.n_inputs, kBlk);
    dim3 grid((unsigned)(ldy / 128), (unsigned)(R / 128), (unsigned)s.n_chan);
    if (grid.x == 0 || grid.z > 65535u) return XE_EINVAL;
    unpack_kernel<<<grid, 256, 0, st>>>(frame, y, s.n_inputs, s.n_chan, s.n_time, R, ldy);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

static int run_batched(const xe_job *jobs, int n_jobs, const xe_tune *tune_in, void *ws, size_t ws_bytes,
                       cudaStream_t st) {
    if (!jobs || n_jobs < 1 || n_jobs > XE_MAX_JOBS) return XE_EINVAL;
    xe_tune tune;
    resolve_tune(tune_in, tune);
    if (int e = check_tune(tune)) return e;
    for (int j = 0; j < n_jobs; ++j)
        if (int e = check_job(jobs[j].s, jobs[j].frame, jobs[j].vis)) return e;
    if (ws_bytes < batched_ws(jobs, n_jobs) || (!ws && batched_ws(jobs, n_jobs))) return XE_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return XE_EINVAL;
    int *status = status_word();
    if (!status) return XE_ECUDA;

    static Params hp;    // large; built under a lock
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    std::memset(&hp, 0, sizeof(hp));
    uint8_t *ybase = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    int items = 0, nj = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const xe_shape &s = jobs[j].s;
        const JobGeom g = geom(s);
        uint8_t *y = ybase;
        ybase += g.y_bytes;
        if (s.n_time == 0) {     // empty integration: V = 0
            if (!jobs[j].accumulate)
                XE_TRY_CUDA(cudaMemsetAsync(jobs[j].vis, 0, (size_t)s.n_chan * npairs(s.n_inputs) * 8, st));
            continue;
        }
        if (int e = launch_unpack(jobs[j].frame, s, y, g.ldy, st)) return e;
        Job &d = hp.jobs[nj++];
        const uint64_t dims[3] = {(uint64_t)g.ldy, (uint64_t)g.R, (uint64_t)s.n_chan};
        const uint64_t strides[2] = {(uint64_t)g.ldy, (uint64_t)g.ldy * g.R};
        const uint32_t box[3] = {kKt, kBlk, 1};
        if (encode_tiled(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, y, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != XE_OK)
            return XE_EINVAL;
        d.vis = jobs[j].vis;
        d.n_inputs = s.n_inputs;
        d.n_chan = s.n_chan;
        d.n_time = s.n_time;
        d.accumulate = jobs[j].accumulate ? 1 : 0;
        d.nb = g.nb;
        d.strips = strips_per_channel(g.nb, tune.max_strip);
        d.k_tiles = g.k_tiles;
        d.item_begin = items;
        const int64_t add = (int64_t)d.strips * s.n_chan;
        if (items + add > INT32_MAX / 2) return XE_EINVAL;
        items += (int)add;
    }
    if (nj == 0) return XE_OK;
    hp.n_jobs = nj;
    hp.n_items = items;
    hp.max_strip = tune.max_strip;
    hp.k_flush_tiles = tune.k_flush / kKt;
    hp.status = status;
    hp.limit_ns = wait_limit_ns();

    static bool attr_set[64] = {};
    int dev = 0;
    XE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !attr_set[dev]) {
        XE_TRY_CUDA(cudaFuncSetAttribute(correlate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        attr_set[dev] = true;
    }
    const int ctas = std::min(items, tune.n_ctas > 0 ? tune.n_ctas : sm_count());
    correlate_kernel<<<ctas, kThreads, kSmemBytes, st>>>(hp);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

}  // namespace corr
}  // namespace xe

using namespace xe;

extern "C" {

int xe_unpack(const uint8_t *frame, xe_shape s, uint8_t *y, int64_t ldy, void *stream) {
    if (!valid_shape(s) || !frame || !y || ldy < std::max(s.n_time, 1) || ldy % 128) return XE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(frame) & 15) || (reinterpret_cast<uintptr_t>(y) & 15)) return XE_EINVAL;
    return corr::launch_unpack(frame, s, y, ldy, static_cast<cudaStream_t>(stream));
}

size_t xe_correlate_workspace_size(xe_shape s) {
    if (!valid_shape(s)) return 0;
    return corr::geom(s).y_bytes + 1024;
}

int xe_correlate(const uint8_t *frame, xe_shape s, int32_t *vis, int accumulate, void *ws, size_t ws_bytes,
                 void *stream) {
    xe_job j{frame, vis, s, accumulate ? 1 : 0};
    return corr::run_batched(&j, 1, nullptr, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

size_t xe_correlate_batched_workspace_size(const xe_job *jobs, int32_t n_jobs, const xe_tune *) {
    if (!jobs || n_jobs < 1 || n_jobs > XE_MAX_JOBS) return 0;
    for (int j = 0; j < n_jobs; ++j)
        if (!valid_shape(jobs[j].s)) return 0;
    return corr::batched_ws(jobs, n_jobs);
}

int xe_correlate_batched(const xe_job *jobs, int32_t n_jobs, const xe_tune *tune, void *ws, size_t ws_bytes,
                         void *stream) {
    return corr::run_batched(jobs, n_jobs, tune, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
