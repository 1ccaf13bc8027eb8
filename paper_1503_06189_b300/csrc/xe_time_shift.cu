// xe_time_shift.cu -- the time-shift stage between assembly and correlation.
//
// Fig. 4's caption names "time shifting" among the optional GPU stages that may run between a
// frame's transfer and its correlation, and defines it no further. Reading used here: every input
// n of every channel is delayed by an integer number of samples d[n], 0 <= d[n] <= T:
//     out[t][f][n] = in[t - d[n]][f][n] for t >= d[n], 0 (no data) for t < d[n].
// The delays are few (one per input) and come from the host; they travel in the launch's parameter
// block. Both kernels are bound by device memory (a byte in and a byte out per sample; 4 bytes per
// visibility for the counters).
//
// The shift runs in tiles of 128 output rows x 128 inputs of one channel. A tile's source rows lie
// in a window of 128 + spread rows (spread: the largest minus the smallest delay of its 128 inputs),
// which TMA brings into shared memory in boxes of 128 rows; rows before the frame's start come in as
// zeros, the "no data" of the shifted frame. Each thread then assembles 16-byte output vectors: one
// 16-byte shared-memory read where 16 inputs share a delay, 16 byte reads otherwise. Frames whose
// spread exceeds kMaxSpread take a gather kernel that reads each byte from its own row in global
// memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "xe_device.cuh"
#include "xe_internal.h"

namespace xe {
namespace shift {

struct Delays {
    int32_t d[4096];           // per input
    uint8_t uniform[256];      // 1 where the 16 inputs of block b share one delay
    int32_t dmax[32];          // per 128 inputs: the largest delay
    int32_t dmin[32];          // per 128 inputs: the smallest delay
    int32_t spread;            // max over the 128-input blocks of dmax - dmin
};

constexpr int kThreads = 256;
constexpr int kTileRows = 128;                         // output rows of a window tile
constexpr int kBoxRows = 128;                          // rows of one TMA box
constexpr int kMaxSpread = 256;                        // window kernel: at most this delay spread per block
constexpr int kMaxBoxes = (kTileRows + kMaxSpread + kBoxRows - 1) / kBoxRows;
constexpr int kWinBytes = kMaxBoxes * kBoxRows * 128;  // 48 KB: four tiles per SM

// Window kernel: CTAs walk the tiles (channel f, 128-input block b, row tile) of the frame. Thread
// (v = tid % 8, r0 = tid / 8) writes the 16 inputs 128 b + 16 v of rows r0, r0 + 32, ... of the
// tile. A window row w holds source row t0 - dmax_b + w, so output row t0 + r of input n reads
// window row r + dmax_b - d[n].
__global__ void __launch_bounds__(kThreads) shift_window_kernel(const __grid_constant__ CUtensorMap map,
                                                                 uint8_t *__restrict__ out, int N, int F, int T,
                                                                 int box_x, const __grid_constant__ Delays dl,
                                                                 uint64_t limit_ns, int *status) {
    extern __shared__ __align__(1024) uint8_t win[];
    __shared__ __align__(8) uint64_t bar;
    // per input: its window row offset e[n] = dmax of its block - d[n] (0 .. kMaxSpread), and per 16
    // inputs the one-delay flag, copied once per CTA: the parameter block is read through the constant
    // cache, which serialises lanes that read different addresses
    uint16_t *se = reinterpret_cast<uint16_t *>(win + kWinBytes);
    uint8_t *su = win + kWinBytes + 2 * N;
    const int nb = (N + 127) / 128, n_tt = (T + kTileRows - 1) / kTileRows;
    const int64_t tiles = (int64_t)F * nb * n_tt;
    const int v = threadIdx.x & 7, r0 = threadIdx.x >> 3;
    for (int n = threadIdx.x; n < N; n += kThreads) se[n] = (uint16_t)(dl.dmax[n / 128] - dl.d[n]);
    for (int g = threadIdx.x; g < N / 16; g += kThreads) su[g] = dl.uniform[g];
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int tt = (int)(tile % n_tt);
        const int64_t fb = tile / n_tt;
        const int b = (int)(fb % nb), f = (int)(fb / nb);
        const int t0 = tt * kTileRows, rows = min(kTileRows, T - t0);
        const int dmax = dl.dmax[b];
        const int boxes = (rows + dmax - dl.dmin[b] + kBoxRows - 1) / kBoxRows;
        if (threadIdx.x == 0) {
            dev::mbar_arrive_expect_tx(&bar, (uint32_t)(boxes * kBoxRows * box_x));
            for (int k = 0; k < boxes; ++k)
                dev::tma_load_3d(dev::smem_u32(win + k * kBoxRows * box_x), &map, &bar, 128 * b, f,
                                 t0 - dmax + k * kBoxRows);
        }
        const bool ok = dev::mbar_wait(&bar, phase, limit_ns);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {               // every thread leaves together
            if (threadIdx.x == 0) atomicExch(status, XE_ETIMEOUT);
            return;
        }
        const int n0 = 128 * b + 16 * v;
        if (16 * v < box_x && n0 < N) {
            uint8_t *dst = out + ((size_t)t0 * F + f) * N + n0;
            const size_t rstride = (size_t)F * N;
            if (su[n0 / 16]) {
                const int e = se[n0];
                for (int r = r0; r < rows; r += kThreads / 8) {
                    const uint4 x = *reinterpret_cast<const uint4 *>(win + (r + e) * box_x + 16 * v);
                    __stcs(reinterpret_cast<uint4 *>(dst + r * rstride), x);
                }
            } else {
                // Byte j of the loop reads input 16 v + k with k = (j + 4 rl) mod 16, rl = this lane's
                // row within its warp: the 32 lanes of a warp then read 32 different banks (with
                // k = j for all lanes they shared 8 banks, four rows apart). The words are assembled
                // in that rotated order and rotated back by rl words before the store.
                const int rl = r0 & 3;
                int base[16];                       // window offset of loop byte j at tile row 0
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int k = (j + 4 * rl) & 15;
                    base[j] = se[n0 + k] * box_x + 16 * v + k;
                }
                for (int r = r0; r < rows; r += kThreads / 8) {
                    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < 16; ++j) w[j >> 2] |= (uint32_t)win[base[j] + r * box_x] << (8 * (j & 3));
                    // rotated word i holds inputs 4 ((i + rl) mod 4) ..: output word o = w[(o - rl) mod 4]
                    uint32_t o[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int s0 = (i - rl) & 3;
                        o[i] = s0 == 0 ? w[0] : s0 == 1 ? w[1] : s0 == 2 ? w[2] : w[3];
                    }
                    __stcs(reinterpret_cast<uint4 *>(dst + r * rstride), make_uint4(o[0], o[1], o[2], o[3]));
                }
            }
        }
        __syncthreads();                            // the window is free for the next tile
    }
}

// Gather kernel (delay spreads beyond kMaxSpread): one thread per output vector of 16 inputs at one
// (t, f); a block of inputs with one delay copies a 16-byte vector from row t - d, otherwise each
// byte comes from its own row.
__global__ void __launch_bounds__(kThreads) shift_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                                         int N, int F, int T, const __grid_constant__ Delays dl) {
    const int NB = N / 16;
    const int64_t total = (int64_t)T * F * NB;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(q % NB);
        const int64_t tf = q / NB;
        const int f = (int)(tf % F), t = (int)(tf / F);
        const int n0 = 16 * b;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (dl.uniform[b]) {
            const int src = t - dl.d[n0];
            if (src >= 0) v = __ldcs(reinterpret_cast<const uint4 *>(in + ((size_t)src * F + f) * N + n0));
        } else {
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int src = t - dl.d[n0 + k];
                const uint32_t byte = src >= 0 ? __ldg(in + ((size_t)src * F + f) * N + n0 + k) : 0u;
                w[k >> 2] |= byte << (8 * (k & 3));
            }
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        __stcs(reinterpret_cast<uint4 *>(out + ((size_t)t * F + f) * N + n0), v);
    }
}

// One warp per (f, i) row of the triangle: flag_pairs[f][p(i, j)] += min(d[i], d[j]) for j >= i,
// flag_count[f][i] += d[i].
__global__ void __launch_bounds__(kThreads) counts_kernel(uint32_t *count, uint32_t *pairs, int N, int F,
                                                          const __grid_constant__ Delays dl) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = (int64_t)F * N;
    const int64_t P = npairs(N);
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < rows;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int f = (int)(w / N), i = (int)(w % N);
        const int di = dl.d[i];
        const int64_t prow = (int64_t)f * P + (int64_t)i * N - (int64_t)i * (i - 1) / 2 - i;
        for (int j = i + lane; j < N; j += 32) pairs[prow + j] += (uint32_t)min(di, dl.d[j]);
        if (lane == 0) count[(size_t)f * N + i] += (uint32_t)di;
    }
}

static int make_delays(const int32_t *host, const xe_shape &s, Delays &dl) {
    if (!host) return XE_EINVAL;
    for (int n = 0; n < s.n_inputs; ++n) {
        if (host[n] < 0 || host[n] > s.n_time) return XE_EINVAL;
        dl.d[n] = host[n];
    }
    for (int b = 0; b < s.n_inputs / 16; ++b) {
        bool u = true;
        for (int k = 1; k < 16; ++k) u = u && host[16 * b + k] == host[16 * b];
        dl.uniform[b] = u ? 1 : 0;
    }
    dl.spread = 0;
    for (int b = 0; b < (s.n_inputs + 127) / 128; ++b) {
        const int n1 = std::min(s.n_inputs, 128 * b + 128);
        dl.dmax[b] = *std::max_element(host + 128 * b, host + n1);
        dl.dmin[b] = *std::min_element(host + 128 * b, host + n1);
        dl.spread = std::max(dl.spread, dl.dmax[b] - dl.dmin[b]);
    }
    return XE_OK;
}

static int grid_of(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + kThreads - 1) / kThreads, (int64_t)sm_count() * 8));
}

}  // namespace shift
}  // namespace xe

using namespace xe;

extern "C" {

int xe_time_shift(const uint8_t *in, xe_shape s, const int32_t *delays, uint8_t *out, void *stream) {
    if (!valid_shape(s) || !in || !out) return XE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) return XE_EINVAL;
    const size_t bytes = (size_t)s.n_time * s.n_chan * s.n_inputs;
    if (in < out + bytes && out < in + bytes && bytes) return XE_EINVAL;     // the buffers must not overlap
    static shift::Delays dl;       // 16 KB: built on the host for each call
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (int e = shift::make_delays(delays, s, dl)) return e;
    if (s.n_time == 0) return XE_OK;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dl.spread <= shift::kMaxSpread) {
        int *status = status_word();
        if (!status) return XE_ECUDA;
        const int box_x = std::min(128, s.n_inputs);
        CUtensorMap map;
        const uint64_t dims[3] = {(uint64_t)s.n_inputs, (uint64_t)s.n_chan, (uint64_t)s.n_time};
        const uint64_t strides[2] = {(uint64_t)s.n_inputs, (uint64_t)s.n_inputs * s.n_chan};
        const uint32_t box[3] = {(uint32_t)box_x, 1, (uint32_t)shift::kBoxRows};
        if (encode_tiled(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(in), dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_NONE) != XE_OK)
            return XE_EINVAL;
        // dynamic shared memory: the window, then the per-input offsets and the one-delay flags
        const int smem = shift::kWinBytes + 2 * s.n_inputs + s.n_inputs / 16;
        static bool attr_set[64] = {};
        int dev = 0;
        XE_TRY_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return XE_EINVAL;
        if (!attr_set[dev]) {
            XE_TRY_CUDA(cudaFuncSetAttribute(shift::shift_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             shift::kWinBytes + 2 * 4096 + 4096 / 16));
            attr_set[dev] = true;
        }
        int per_sm = 0;
        XE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shift::shift_window_kernel, shift::kThreads,
                                                                  smem));
        const int64_t tiles = (int64_t)s.n_chan * ((s.n_inputs + 127) / 128) *
                              ((s.n_time + shift::kTileRows - 1) / shift::kTileRows);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count() * std::max(1, per_sm)));
        shift::shift_window_kernel<<<grid, shift::kThreads, smem, st>>>(
            map, out, s.n_inputs, s.n_chan, s.n_time, box_x, dl, wait_limit_ns(), status);
    } else {
        const int64_t work = (int64_t)s.n_time * s.n_chan * (s.n_inputs / 16);
        shift::shift_kernel<<<shift::grid_of(work), shift::kThreads, 0, st>>>(in, out, s.n_inputs, s.n_chan,
                                                                             s.n_time, dl);
    }
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

int xe_time_shift_counts(const int32_t *delays, xe_shape s, uint32_t *flag_count, uint32_t *flag_pairs, void *stream) {
    if (!valid_shape(s) || !flag_count || !flag_pairs) return XE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(flag_count) | reinterpret_cast<uintptr_t>(flag_pairs)) & 3) return XE_EINVAL;
    static shift::Delays dl;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (int e = shift::make_delays(delays, s, dl)) return e;
    const int64_t work = (int64_t)s.n_chan * s.n_inputs * 32;
    shift::counts_kernel<<<shift::grid_of(work), shift::kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        flag_count, flag_pairs, s.n_inputs, s.n_chan, dl);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

}  // extern "C"
