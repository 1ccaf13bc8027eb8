// xe_internal.h -- host-side helpers shared by the libxe translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe.h"

namespace xe {

// Records a failing CUDA runtime status for xe_last_cuda_error() and maps it to XE_ECUDA.
int cuda_fail(cudaError_t e);

#define XE_TRY_CUDA(call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ::xe::cuda_fail(e_);  \
    } while (0)

// Device address of the library's status word on the current device (nullptr on failure).
int *status_word();

// Wall-clock limit of every bounded device-side wait, in nanoseconds.
uint64_t wait_limit_ns();

// SM count of the current device (cached per device).
int sm_count();

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda needed).
int encode_tiled(CUtensorMap *map, CUtensorMapDataType dtype, uint32_t rank, void *base,
                 const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box,
                 CUtensorMapSwizzle swizzle);

#ifdef __CUDACC__
#define XE_HD __host__ __device__
#else
#define XE_HD
#endif

XE_HD inline int64_t npairs(int64_t n) { return n * (n + 1) / 2; }
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// xe_assemble with header stream ids offset by stream_base (see xe_assemble.cu).
int assemble_streams(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                     uint32_t stream_base, xe_shape s, uint8_t *frame, uint8_t *filled, uint32_t *lost,
                     uint32_t *stats, void *ws, size_t ws_bytes, cudaStream_t st);

// The assembly's index without its payload copy (see xe_assemble.cu): owner[F / 8][T / 4], the
// packet holding each (channel group, time slot), 0xFFFFFFFF where none arrived.
int index_streams(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                  uint32_t stream_base, xe_shape s, uint8_t *filled, uint32_t *lost, uint32_t *stats,
                  uint32_t *owner, cudaStream_t st);

// Samples of one frame read in place from its packets through its index (zero-copy correlation).
struct packet_src {
    const uint8_t *pkts;
    const uint32_t *owner;       // index_streams output for this frame
    uint32_t pkt_stride;
};

// xe_correlate_batched with job j's samples read from src[j] instead of jobs[j].frame (pair engine).
int correlate_packets_batched(const xe_job *jobs, const packet_src *src, int n_jobs, void *ws, size_t ws_bytes,
                              cudaStream_t st);

namespace legacy {
// XE_ENGINE_LEGACY_S4 / _S8: the jobs (checked by the caller) on the mma.sync 4-bit path or its int8
// variant (s8), one launch per job.
int correlate_legacy(const xe_job *jobs, int n_jobs, bool s8, cudaStream_t st);
}  // namespace legacy

inline bool valid_shape(const xe_shape &s) {
    return s.n_inputs >= 16 && s.n_inputs <= XE_MAX_INPUTS && s.n_inputs % 16 == 0 && s.n_chan >= 1 &&
           s.n_time >= 0;
}

}  // namespace xe
