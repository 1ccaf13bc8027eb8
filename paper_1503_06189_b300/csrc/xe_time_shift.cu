// xe_time_shift.cu -- the time-shift stage between assembly and correlation.
//
// Fig. 4's caption names "time shifting" among the optional GPU stages that may run between a
// frame's transfer and its correlation, and defines it no further. Reading used here: every input
// n of every channel is delayed by an integer number of samples d[n], 0 <= d[n] <= T:
//     out[t][f][n] = in[t - d[n]][f][n] for t >= d[n], 0 (no data) for t < d[n].
// The delays are few (one per input) and come from the host; they travel in the launch's parameter
// block. Both kernels are bound by device memory (a byte in and a byte out per sample; 4 bytes per
// visibility for the counters).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "xe_internal.h"

namespace xe {
namespace shift {

struct Delays {
    int32_t d[4096];           // per input
    uint8_t uniform[256];      // 1 where the 16 inputs of block b share one delay
};

constexpr int kThreads = 256;

// One thread per output vector of 16 inputs at one (t, f): a block of inputs with one delay copies
// a 16-byte vector from row t - d; otherwise each byte comes from its own row.
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
    const int64_t work = (int64_t)s.n_time * s.n_chan * (s.n_inputs / 16);
    shift::shift_kernel<<<shift::grid_of(work), shift::kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        in, out, s.n_inputs, s.n_chan, s.n_time, dl);
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
