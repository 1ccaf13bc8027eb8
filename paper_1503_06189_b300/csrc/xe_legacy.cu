// xe_legacy.cu -- A3/A4 on the legacy warp-level tensor path: mma.sync m16n8k64 with 4-bit signed
// operands, straight on the packed samples (no unpack, no tcgen05), and its m16n8k32 s8 variant on
// samples unpacked in shared memory. Baselines for the tcgen05 engines, measured beside them.
//
// Method (Sec. I, Sec. II-B): V_f[i,j] = sum_t x_i(t) conj(x_j(t)), i <= j, x = re + i im. A sample
// byte is re << 4 | im, so four consecutive samples of one input, as one 32-bit register, are the
// eight 4-bit values (im_t, re_t, im_t+1, re_t+1, ...) along K. With A the packed rows of inputs i,
// B those of inputs j, B' the same bytes with their nibbles swapped (re, im) and A' the bytes of A
// with the Re nibble cleared (im, 0):
//     A B^T   = sum_t re_i re_j + im_i im_j             = Re V
//     A B'^T  = sum_t im_i re_j + re_i im_j             = S
//     A' B'^T = sum_t im_i re_j                         = X
//     Im V = X - (S - X) = 2 X - S = sum_t im_i re_j - re_i im_j.
// Three m16n8k64 MMAs per 16 x 8 tile and 32 samples, int32 accumulators (exact: |Re V| <= 128 T,
// |2 X| <= 128 T, below 2^31 for T <= 2^24 - 1).
//
// Tiling: one CTA per (channel, 64 x 64 block pair I <= J), 8 warps each with a 16 x 32 tile. The
// packed frame [T][F][N] is read 128 samples at a time and transposed in registers into shared
// rows [64 inputs][128 samples] (4 words of padding per row: the fragment loads of a warp hit 32
// distinct banks).
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_internal.h"

namespace xe {
namespace legacy {

constexpr int kTile = 64;          // inputs per block
constexpr int kKt = 128;           // samples per stage: 128 bytes = 32 words per input row
constexpr int kRowWords = 36;      // 32 words + 4 of padding
constexpr int kThreads = 256;

__device__ __forceinline__ void mma_s4(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k64.row.col.s32.s4.s4.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (re, im) nibbles of every byte swapped
__device__ __forceinline__ uint32_t swap_nibbles(uint32_t b) {
    return ((b >> 4) & 0x0F0F0F0Fu) | ((b << 4) & 0xF0F0F0F0u);
}

__global__ void __launch_bounds__(kThreads) correlate_s4_kernel(const uint8_t *__restrict__ frame, int N, int F,
                                                                int T, int32_t *__restrict__ vis, int accumulate) {
    __shared__ uint32_t sa[kTile * kRowWords];
    __shared__ uint32_t sb[kTile * kRowWords];
    const int nbk = (N + kTile - 1) / kTile;
    int q = blockIdx.x, I = 0;
    while (q >= nbk - I) {
        q -= nbk - I;
        ++I;
    }
    const int J = I + q;
    const bool diag = I == J;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = warp & 3, wj = warp >> 2;      // rows 16 wi .. +15, columns 32 wj .. +31 of the block
    const int g = lane >> 2, tq = lane & 3;
    const int tb = threadIdx.x & 31, ng = threadIdx.x >> 5;   // loader: samples 4 tb .. +3, inputs 8 ng .. +7
    const int64_t P = (int64_t)N * (N + 1) / 2;

    for (int f = blockIdx.y; f < F; f += gridDim.y) {
        int acc_re[4][4] = {}, acc_s[4][4] = {}, acc_x[4][4] = {};
        for (int t0 = 0; t0 < T; t0 += kKt) {
            __syncthreads();                      // the previous stage's fragments are read
            for (int which = 0; which < (diag ? 1 : 2); ++which) {
                const int n0 = (which ? J : I) * kTile + ng * 8;
                uint32_t w[4][2];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int t = t0 + tb * 4 + s;
                    uint2 v = make_uint2(0u, 0u);
                    if (t < T && n0 < N) v = *reinterpret_cast<const uint2 *>(frame + ((size_t)t * F + f) * N + n0);
                    w[s][0] = v.x;
                    w[s][1] = v.y;
                }
                uint32_t *dst = which ? sb : sa;
#pragma unroll
                for (int k = 0; k < 8; ++k) {     // input n0 + k: its bytes of samples 4 tb .. 4 tb + 3
                    const int h = k >> 2, b = k & 3;
                    const uint32_t sel = (uint32_t)(b | ((b + 4) << 4));
                    const uint32_t lo = __byte_perm(w[0][h], w[1][h], sel);
                    const uint32_t hi = __byte_perm(w[2][h], w[3][h], sel);
                    dst[(ng * 8 + k) * kRowWords + tb] = __byte_perm(lo, hi, 0x5410);
                }
            }
            __syncthreads();
            const uint32_t *sB = diag ? sa : sb;
#pragma unroll
            for (int kk = 0; kk < kKt / 32; ++kk) {   // 32 samples = 64 nibbles = 8 words per step
                const int kw = kk * 8;
                const uint32_t *ra = sa + (wi * 16 + g) * kRowWords + kw + tq;
                uint32_t a[4], am[4];
                a[0] = ra[0];
                a[1] = ra[8 * kRowWords];
                a[2] = ra[4];
                a[3] = ra[8 * kRowWords + 4];
#pragma unroll
                for (int r = 0; r < 4; ++r) am[r] = a[r] & 0x0F0F0F0Fu;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const uint32_t *rb = sB + (wj * 32 + nt * 8 + g) * kRowWords + kw + tq;
                    const uint32_t b0 = rb[0], b1 = rb[4];
                    const uint32_t s0 = swap_nibbles(b0), s1 = swap_nibbles(b1);
                    mma_s4(acc_re[nt], a, b0, b1);
                    mma_s4(acc_s[nt], a, s0, s1);
                    mma_s4(acc_x[nt], am, s0, s1);
                }
            }
        }
        // epilogue: D rows g, g + 8 (c0 c1 / c2 c3), columns 2 tq, 2 tq + 1 of each 8-column tile
        int32_t *vis_f = vis + (size_t)f * (size_t)P * 2;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = I * kTile + wi * 16 + g + (r >> 1) * 8;
                const int j = J * kTile + wj * 32 + nt * 8 + 2 * tq + (r & 1);
                if (i >= N || j >= N || j < i) continue;
                const int64_t p = (int64_t)i * N - (int64_t)i * (i - 1) / 2 + (j - i);
                const int re = acc_re[nt][r];
                const int im = (int)(2u * (uint32_t)acc_x[nt][r] - (uint32_t)acc_s[nt][r]);
                int2 *o = reinterpret_cast<int2 *>(vis_f) + p;
                if (accumulate) {
                    const int2 v = *o;
                    *o = make_int2((int)((uint32_t)v.x + (uint32_t)re), (int)((uint32_t)v.y + (uint32_t)im));
                } else {
                    *o = make_int2(re, im);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ s8 variant (XE_ENGINE_LEGACY_S8)
// The same method on int8 operands, m16n8k32 (16 samples per MMA): the loader unpacks every sample
// once, into shared rows of (re, im) int8 pairs [64 inputs][2 x 128 samples]; B' swaps the bytes of
// each pair (im, re) and A' clears the re bytes (0, im). Three MMAs per 16 x 8 tile and 16 samples.
constexpr int kRowWords8 = 68;     // 64 words of (re, im) pairs + 4 of padding

__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Two packed samples (the low 16 bits of h: bytes re << 4 | im) -> int8 bytes (re0, im0, re1, im1).
// Each byte's nibble v in [0, 15] becomes v - 16 [v >= 8]: OR in 0xF0 where bit 3 is set; (v & 8) x 30
// = 240 stays inside its byte, so one multiply fills all four.
__device__ __forceinline__ uint32_t unpack2_s8(uint32_t h) {
    const uint32_t x = __byte_perm(h, 0, 0x1100);                     // (p0, p0, p1, p1)
    const uint32_t v = ((x >> 4) & 0x000F000Fu) | (x & 0x0F000F00u);   // (re0, im0, re1, im1) as nibbles
    return v | ((v & 0x08080808u) * 0x1Eu);
}

__global__ void __launch_bounds__(kThreads) correlate_s8_kernel(const uint8_t *__restrict__ frame, int N, int F,
                                                                int T, int32_t *__restrict__ vis, int accumulate) {
    __shared__ uint32_t sa[kTile * kRowWords8];
    __shared__ uint32_t sb[kTile * kRowWords8];
    const int nbk = (N + kTile - 1) / kTile;
    int q = blockIdx.x, I = 0;
    while (q >= nbk - I) {
        q -= nbk - I;
        ++I;
    }
    const int J = I + q;
    const bool diag = I == J;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = warp & 3, wj = warp >> 2;
    const int g = lane >> 2, tq = lane & 3;
    const int tb = threadIdx.x & 31, ng = threadIdx.x >> 5;
    const int64_t P = (int64_t)N * (N + 1) / 2;

    for (int f = blockIdx.y; f < F; f += gridDim.y) {
        int acc_re[4][4] = {}, acc_s[4][4] = {}, acc_x[4][4] = {};
        for (int t0 = 0; t0 < T; t0 += kKt) {
            __syncthreads();
            for (int which = 0; which < (diag ? 1 : 2); ++which) {
                const int n0 = (which ? J : I) * kTile + ng * 8;
                uint32_t w[4][2];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int t = t0 + tb * 4 + s;
                    uint2 v = make_uint2(0u, 0u);
                    if (t < T && n0 < N) v = *reinterpret_cast<const uint2 *>(frame + ((size_t)t * F + f) * N + n0);
                    w[s][0] = v.x;
                    w[s][1] = v.y;
                }
                uint32_t *dst = which ? sb : sa;
#pragma unroll
                for (int k = 0; k < 8; ++k) {     // input n0 + k, samples 4 tb .. 4 tb + 3 -> words 2 tb, 2 tb + 1
                    const int h = k >> 2, b = k & 3;
                    const uint32_t sel = (uint32_t)(b | ((b + 4) << 4));
                    const uint32_t lo = __byte_perm(w[0][h], w[1][h], sel);     // samples 0, 1 in bytes 0, 1
                    const uint32_t hi = __byte_perm(w[2][h], w[3][h], sel);     // samples 2, 3
                    uint2 o = make_uint2(unpack2_s8(lo), unpack2_s8(hi));
                    *reinterpret_cast<uint2 *>(&dst[(ng * 8 + k) * kRowWords8 + 2 * tb]) = o;
                }
            }
            __syncthreads();
            const uint32_t *sB = diag ? sa : sb;
#pragma unroll
            for (int kk = 0; kk < kKt / 16; ++kk) {   // 16 samples = 32 int8 = 8 words per step
                const int kw = kk * 8;
                const uint32_t *ra = sa + (wi * 16 + g) * kRowWords8 + kw + tq;
                uint32_t a[4], am[4];
                a[0] = ra[0];
                a[1] = ra[8 * kRowWords8];
                a[2] = ra[4];
                a[3] = ra[8 * kRowWords8 + 4];
#pragma unroll
                for (int r = 0; r < 4; ++r) am[r] = a[r] & 0xFF00FF00u;   // (0, im) pairs
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const uint32_t *rb = sB + (wj * 32 + nt * 8 + g) * kRowWords8 + kw + tq;
                    const uint32_t b0 = rb[0], b1 = rb[4];
                    const uint32_t s0 = __byte_perm(b0, 0, 0x2301), s1 = __byte_perm(b1, 0, 0x2301);   // (im, re)
                    mma_s8(acc_re[nt], a, b0, b1);
                    mma_s8(acc_s[nt], a, s0, s1);
                    mma_s8(acc_x[nt], am, s0, s1);
                }
            }
        }
        int32_t *vis_f = vis + (size_t)f * (size_t)P * 2;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = I * kTile + wi * 16 + g + (r >> 1) * 8;
                const int j = J * kTile + wj * 32 + nt * 8 + 2 * tq + (r & 1);
                if (i >= N || j >= N || j < i) continue;
                const int64_t p = (int64_t)i * N - (int64_t)i * (i - 1) / 2 + (j - i);
                const int re = acc_re[nt][r];
                const int im = (int)(2u * (uint32_t)acc_x[nt][r] - (uint32_t)acc_s[nt][r]);
                int2 *o = reinterpret_cast<int2 *>(vis_f) + p;
                if (accumulate) {
                    const int2 v = *o;
                    *o = make_int2((int)((uint32_t)v.x + (uint32_t)re), (int)((uint32_t)v.y + (uint32_t)im));
                } else {
                    *o = make_int2(re, im);
                }
            }
        }
    }
}

int correlate_legacy(const xe_job *jobs, int n_jobs, bool s8, cudaStream_t st) {
    for (int j = 0; j < n_jobs; ++j) {
        const xe_shape &s = jobs[j].s;
        if (s.n_time == 0) {                      // empty integration: V = 0, or unchanged when adding
            if (!jobs[j].accumulate) {
                const size_t bytes = (size_t)s.n_chan * (size_t)((int64_t)s.n_inputs * (s.n_inputs + 1) / 2) * 8;
                if (cudaError_t e = cudaMemsetAsync(jobs[j].vis, 0, bytes, st)) return cuda_fail(e);
            }
            continue;
        }
        const int nbk = (s.n_inputs + kTile - 1) / kTile;
        dim3 grid((unsigned)(nbk * (nbk + 1) / 2), (unsigned)(s.n_chan < 65535 ? s.n_chan : 65535), 1);
        const uint8_t *fr = static_cast<const uint8_t *>(jobs[j].frame);
        if (s8)
            correlate_s8_kernel<<<grid, kThreads, 0, st>>>(fr, s.n_inputs, s.n_chan, s.n_time, jobs[j].vis,
                                                           jobs[j].accumulate ? 1 : 0);
        else
            correlate_s4_kernel<<<grid, kThreads, 0, st>>>(fr, s.n_inputs, s.n_chan, s.n_time, jobs[j].vis,
                                                           jobs[j].accumulate ? 1 : 0);
        if (cudaError_t e = cudaGetLastError()) return cuda_fail(e);
    }
    return XE_OK;
}

// Rate probe: every warp issues chains of independent mma.sync on register operands (8 chains, so
// the pipe never waits for a result); kind 0 = m16n8k64 s4 (16,384 int ops per instruction),
// kind 1 = m16n8k32 s8 (8,192); kind 2 = the CUDA-core 4-way int8 dot product dp4a (8 int ops per
// thread and instruction, 256 per warp instruction), in 8 independent chains per thread.
__global__ void __launch_bounds__(kThreads) mma_probe_kernel(int kind, int iters, int32_t *sink) {
    uint32_t a[4] = {threadIdx.x * 0x01010101u, threadIdx.x ^ 0x5A5A5A5Au, blockIdx.x * 0x11111111u, 0x12345678u};
    const uint32_t b0 = threadIdx.x * 0x9E3779B9u, b1 = blockIdx.x ^ 0xA5A5A5A5u;
    int acc[8][4] = {};
    if (kind == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) mma_s4(acc[k], a, b0 + k, b1);
        }
    } else if (kind == 2) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("dp4a.s32.s32 %0, %1, %2, %0;" : "+r"(acc[k][0]) : "r"(a[k & 3]), "r"(b0 + k));
        }
    } else {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                             "{%0,%1,%2,%3};"
                             : "+r"(acc[k][0]), "+r"(acc[k][1]), "+r"(acc[k][2]), "+r"(acc[k][3])
                             : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0 + k), "r"(b1));
        }
    }
    int x = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) x += acc[k][0] + acc[k][1] + acc[k][2] + acc[k][3];
    sink[blockIdx.x * kThreads + threadIdx.x] = x;
}

}  // namespace legacy
}  // namespace xe

extern "C" int xe_probe_mma_legacy(int32_t kind, int32_t blocks, int32_t iters, int32_t *sink, void *stream) {
    if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !sink) return XE_EINVAL;
    xe::legacy::mma_probe_kernel<<<blocks, xe::legacy::kThreads, 0, static_cast<cudaStream_t>(stream)>>>(kind, iters,
                                                                                                         sink);
    if (cudaError_t e = cudaGetLastError()) return xe::cuda_fail(e);
    return XE_OK;
}
