// xe_core.cu -- status codes, CUDA error plumbing, the device status word, tensor-map encoding and
// the failure-detection self test.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "xe_device.cuh"
#include "xe_internal.h"

namespace xe {

// Device status word: kernels store XE_ETIMEOUT here when a bounded wait expires.
__device__ int g_status;

static thread_local int t_last_cuda = 0;

int cuda_fail(cudaError_t e) {
    t_last_cuda = static_cast<int>(e);
    return XE_ECUDA;
}

static constexpr int kMaxDevices = 64;

int *status_word() {
    static int *addr[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<int *>(p);
    }
    return addr[dev];
}

uint64_t wait_limit_ns() {
    static const uint64_t v = [] {
        const char *e = std::getenv("XE_WAIT_LIMIT_MS");
        const long ms = e ? std::atol(e) : 2000;
        return static_cast<uint64_t>(ms > 0 ? ms : 2000) * 1000000ull;
    }();
    return v;
}

int sm_count() {
    static int cache[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 148;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_tiled(CUtensorMap *map, CUtensorMapDataType dtype, uint32_t rank, void *base,
                 const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box,
                 CUtensorMapSwizzle swizzle) {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    if (!fn) return XE_ECUDA;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], es[5];
    for (uint32_t i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) st[i] = strides_bytes[i];
    }
    const CUresult r = fn(map, dtype, rank, base, d, st, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? XE_OK : XE_EINVAL;
}

// Waits on an mbarrier that nothing ever arrives at, for at most limit_ns, then records the
// timeout. Exercises the same bounded-wait path as the pipeline kernels.
__global__ void selftest_timeout_kernel(uint64_t limit_ns, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !dev::mbar_wait(&bar, 0, limit_ns)) atomicExch(status, XE_ETIMEOUT);
}

}  // namespace xe

extern "C" {

const char *xe_strerror(int status) {
    switch (status) {
        case XE_OK: return "ok";
        case XE_EINVAL: return "invalid argument (shape, pointer, alignment or option)";
        case XE_EOVERFLOW: return "integration length beyond the int32 bound (T > 2^24 - 1)";
        case XE_ENOMEM: return "workspace too small or device-memory budget exceeded";
        case XE_ECUDA: return "CUDA call failed (see xe_last_cuda_error)";
        case XE_ETIMEOUT: return "bounded wait expired";
        case XE_EAGAIN: return "no free slot; retry";
        default: return "unknown status";
    }
}

int xe_last_cuda_error(void) { return xe::t_last_cuda; }

int xe_version(void) { return 10100; }

int xe_device_status(int *status_out, void *stream) {
    if (!status_out) return XE_EINVAL;
    int *w = xe::status_word();
    if (!w) return XE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    XE_TRY_CUDA(cudaMemcpyAsync(&v, w, sizeof(int), cudaMemcpyDeviceToHost, s));
    XE_TRY_CUDA(cudaStreamSynchronize(s));
    const int zero = 0;
    XE_TRY_CUDA(cudaMemcpyAsync(w, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    XE_TRY_CUDA(cudaStreamSynchronize(s));
    *status_out = v;
    return XE_OK;
}

int xe_selftest_timeout(uint64_t timeout_ns, void *stream) {
    if (timeout_ns == 0 || timeout_ns > 10ull * 1000000000ull) return XE_EINVAL;
    int *w = xe::status_word();
    if (!w) return XE_ECUDA;
    xe::selftest_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(timeout_ns, w);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

}  // extern "C"
