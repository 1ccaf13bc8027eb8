// xe_normalize.cu -- A5: normalisation of the integrated matrix by per-visibility sample counts
// (Sec. II-C). Packet loss is one counter per channel applied to every point of the matrix;
// F-engine flags are counted per input and channel; pairs flagged in the same sample were
// subtracted twice and are added back once: n_ij = t_int - L_f - c_i - c_j + x_ij.
// out = (float)V / (float)n_ij with IEEE division. HBM-bound: 8 B read + 12 B written per point.
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_internal.h"

namespace xe {
namespace norm {

// Row i of the packed triangle that holds position p: start(i) = i*N - i*(i-1)/2 <= p < start(i+1).
__device__ __forceinline__ int row_of(int64_t p, int N) {
    const float b = 2.0f * N + 1.0f;
    const float disc = fmaxf(b * b - 8.0f * (float)p, 0.0f);
    int i = (int)((b - sqrtf(disc)) * 0.5f);
    i = max(0, min(N - 1, i));
    auto start = [N](int r) { return (int64_t)r * N - (int64_t)r * (r - 1) / 2; };
    while (i > 0 && start(i) > p) --i;
    while (i + 1 < N && start(i + 1) <= p) ++i;
    return i;
}

// Points per thread: its loads are all issued before the first store, so each thread keeps
// kUnroll * 8 B in flight (one 8-byte load per thread leaves HBM half idle at full occupancy).
constexpr int kUnroll = 4;
constexpr int kThreads = 256;

// grid (x: chunks of kThreads * kUnroll points, y: channel); thread t of chunk b handles points
// b * kThreads * kUnroll + u * kThreads + t, u < kUnroll (coalesced per warp for every u).
__global__ void __launch_bounds__(kThreads) normalize_kernel(const int2 *__restrict__ vis, int N, int64_t P,
                                                             uint32_t t_int, const uint32_t *__restrict__ lost,
                                                             const uint32_t *__restrict__ fc,
                                                             const uint32_t *__restrict__ fp, float2 *__restrict__ out,
                                                             uint32_t *__restrict__ n_out) {
    const int f = blockIdx.y;
    const int64_t base = (int64_t)f * P;
    const int64_t c0 = (int64_t)t_int - lost[f];
    const int64_t p0 = (int64_t)blockIdx.x * (kThreads * kUnroll) + threadIdx.x;
    int2 v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int64_t p = p0 + u * kThreads;
        v[u] = p < P ? __ldcs(vis + base + p) : make_int2(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int64_t p = p0 + u * kThreads;
        if (p >= P) break;
        int64_t c = c0;
        if (fc) {
            const int i = row_of(p, N);
            const int j = i + (int)(p - ((int64_t)i * N - (int64_t)i * (i - 1) / 2));
            if (i == j) c -= fc[(int64_t)f * N + i];
            else c -= (int64_t)fc[(int64_t)f * N + i] + fc[(int64_t)f * N + j] - fp[base + p];
        }
        float2 o = make_float2(0.0f, 0.0f);
        if (c > 0) {
            const float d = (float)c;
            o.x = __fdiv_rn((float)v[u].x, d);
            o.y = __fdiv_rn((float)v[u].y, d);
        }
        __stcs(out + base + p, o);
        if (n_out) __stcs(n_out + base + p, c > 0 ? (uint32_t)c : 0u);
    }
}

}  // namespace norm
}  // namespace xe

using namespace xe;

extern "C" int xe_normalize(const int32_t *vis, xe_shape s, uint32_t t_int, const uint32_t *lost,
                            const uint32_t *flag_count, const uint32_t *flag_pairs, float *out, uint32_t *n_out,
                            void *stream) {
    if (!valid_shape(s) || !vis || !lost || !out || (!flag_count) != (!flag_pairs)) return XE_EINVAL;
    if (s.n_chan > 65535) return XE_EINVAL;
    if (t_int > XE_MAX_TIME) return XE_EOVERFLOW;
    if ((reinterpret_cast<uintptr_t>(vis) | reinterpret_cast<uintptr_t>(out)) & 7) return XE_EINVAL;
    const int64_t P = npairs(s.n_inputs);
    const int64_t per_block = norm::kThreads * norm::kUnroll;
    dim3 grid((unsigned)((P + per_block - 1) / per_block), (unsigned)s.n_chan);
    norm::normalize_kernel<<<grid, norm::kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const int2 *>(vis), s.n_inputs, P, t_int, lost, flag_count, flag_pairs,
        reinterpret_cast<float2 *>(out), n_out);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}
