/*
 * A plain-C user of the libxe C ABI (include/xe.h), with no Python or torch involved: it allocates
 * its own device buffers, correlates a constant frame (every input holds one complex value for the
 * whole frame), normalises it, and checks both results against their closed forms:
 *   V[i,j] = T x_i conj(x_j), i.e. Re = T (a_i a_j + b_i b_j), Im = T (b_i a_j - a_i b_j),
 *   out = V / T and n = T (no loss, no flags).
 * Built and run by tests/test_c_abi.py. Exit status: 0 = every value matched, 1 = a mismatch,
 * 2 = a CUDA error, 3 = a libxe error.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "xe.h"

#define CHECK_CUDA(call)                                                                    \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));                     \
            return 2;                                                                       \
        }                                                                                   \
    } while (0)
#define CHECK_XE(call)                                                                      \
    do {                                                                                    \
        int s_ = (call);                                                                    \
        if (s_ != XE_OK) {                                                                  \
            fprintf(stderr, "%s: %s\n", #call, xe_strerror(s_));                            \
            return 3;                                                                       \
        }                                                                                   \
    } while (0)

enum { N = 64, F = 3, T = 1000 };

/* The constant value of input n in channel f: re, im in [-8, 7]. */
static int value_re(int f, int n) { return (3 * n + f) % 16 - 8; }
static int value_im(int f, int n) { return (5 * n + 2 * f + 1) % 16 - 8; }

static int run(void) {
    const int64_t P = (int64_t)N * (N + 1) / 2;
    const size_t frame_bytes = (size_t)T * F * N, vis_count = (size_t)F * P * 2;
    uint8_t *frame_h = malloc(frame_bytes);
    int32_t *vis_h = malloc(vis_count * sizeof(int32_t));
    float *out_h = malloc(vis_count * sizeof(float));
    uint32_t *n_h = malloc((size_t)F * P * sizeof(uint32_t));
    if (!frame_h || !vis_h || !out_h || !n_h) return 2;
    for (int t = 0; t < T; ++t)
        for (int f = 0; f < F; ++f)
            for (int n = 0; n < N; ++n)
                frame_h[((size_t)t * F + f) * N + n] =
                    (uint8_t)(((value_re(f, n) & 15) << 4) | (value_im(f, n) & 15));

    xe_shape s;
    s.n_inputs = N;
    s.n_chan = F;
    s.n_time = T;
    const size_t ws_bytes = xe_correlate_workspace_size(s);
    uint8_t *frame_d;
    int32_t *vis_d;
    float *out_d;
    uint32_t *n_d, *lost_d;
    void *ws_d;
    cudaStream_t st;
    CHECK_CUDA(cudaStreamCreate(&st));
    CHECK_CUDA(cudaMalloc((void **)&frame_d, frame_bytes));
    CHECK_CUDA(cudaMalloc((void **)&vis_d, vis_count * sizeof(int32_t)));
    CHECK_CUDA(cudaMalloc((void **)&out_d, vis_count * sizeof(float)));
    CHECK_CUDA(cudaMalloc((void **)&n_d, (size_t)F * P * sizeof(uint32_t)));
    CHECK_CUDA(cudaMalloc((void **)&lost_d, F * sizeof(uint32_t)));
    CHECK_CUDA(cudaMalloc(&ws_d, ws_bytes > 0 ? ws_bytes : 1));
    CHECK_CUDA(cudaMemcpyAsync(frame_d, frame_h, frame_bytes, cudaMemcpyHostToDevice, st));
    CHECK_CUDA(cudaMemsetAsync(lost_d, 0, F * sizeof(uint32_t), st));

    CHECK_XE(xe_correlate(frame_d, s, vis_d, 0, ws_d, ws_bytes, (void *)st));
    CHECK_XE(xe_normalize(vis_d, s, T, lost_d, NULL, NULL, out_d, n_d, (void *)st));
    CHECK_CUDA(cudaMemcpyAsync(vis_h, vis_d, vis_count * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CHECK_CUDA(cudaMemcpyAsync(out_h, out_d, vis_count * sizeof(float), cudaMemcpyDeviceToHost, st));
    CHECK_CUDA(cudaMemcpyAsync(n_h, n_d, (size_t)F * P * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CHECK_CUDA(cudaStreamSynchronize(st));
    int device_status = XE_OK;                      /* expired bounded waits, if any */
    CHECK_XE(xe_device_status(&device_status, (void *)st));
    CHECK_XE(device_status);

    long bad = 0;
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                const int64_t p = (int64_t)i * N - (int64_t)i * (i - 1) / 2 + (j - i);
                const size_t k = ((size_t)f * P + p) * 2;
                const int ai = value_re(f, i), bi = value_im(f, i), aj = value_re(f, j), bj = value_im(f, j);
                const int32_t re = T * (ai * aj + bi * bj), im = T * (bi * aj - ai * bj);
                const double out_re = (double)re / T, out_im = (double)im / T;
                if (vis_h[k] != re || vis_h[k + 1] != im || n_h[(size_t)f * P + p] != T ||
                    fabs(out_h[k] - out_re) > 1e-6 * fabs(out_re) || fabs(out_h[k + 1] - out_im) > 1e-6 * fabs(out_im)) {
                    if (bad < 5)
                        fprintf(stderr, "f=%d i=%d j=%d: vis (%d, %d) want (%d, %d), out (%g, %g), n %u\n", f, i, j,
                                vis_h[k], vis_h[k + 1], re, im, out_h[k], out_h[k + 1], n_h[(size_t)f * P + p]);
                    ++bad;
                }
            }
    cudaFree(frame_d);
    cudaFree(vis_d);
    cudaFree(out_d);
    cudaFree(n_d);
    cudaFree(lost_d);
    cudaFree(ws_d);
    cudaStreamDestroy(st);
    free(frame_h);
    free(vis_h);
    free(out_h);
    free(n_h);
    if (bad) {
        fprintf(stderr, "%ld mismatches\n", bad);
        return 1;
    }
    printf("ok: %d channels x %lld visibilities match the closed form\n", F, (long long)P);
    return 0;
}

int main(void) { return run(); }
