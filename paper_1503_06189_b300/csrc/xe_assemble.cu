// xe_assemble.cu -- A1: UDP packets -> frame (Sec. II-A).
//
// Sec. II-A.2: sequence numbers place each packet's data section in the frame; lost packets leave
// zeros in their place; out-of-order packets land by sequence number; duplicates are ignored.
// Sec. II-A.3: the data section is moved with non-temporal (streaming) loads and stores.
//
// Three launches, all HBM-bound and independent of thread timing:
//   1. init   owner[group][slot] = none (group-major: one group's slots are contiguous)
//   2. claim  every in-window packet k does owner = min(owner, k): the first arrival wins
//   3. copy   packet k copies its payload iff owner == k (else it is a duplicate); every slot that
//             no packet owns is zero-filled and its 8 channels' lost counters grow by 4 samples.
// The zero-copy path (xe_correlate_packets) runs 1 and 2 and a tally (the counts of 3 without
// moving any payload, from the owner table alone): the owner table is then the frame's index,
// through which the correlator reads the packets in place.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "xe_internal.h"

namespace xe {
namespace asmb {

constexpr uint32_t kNone = 0xFFFFFFFFu;

struct Geo {
    uint64_t seq0;
    uint32_t n_pkts, stride;
    int32_t N, F, Q, G, gps, S;
    uint32_t stream_base = 0;    // header stream ids [stream_base, stream_base + S) map to this frame
};

enum Class { kOk = 0, kLate = 2, kEarly = 3, kInvalid = 4 };

// Owner table entry of (time slot, channel group).
__device__ __forceinline__ size_t oidx(const Geo &g, int slot, int grp) { return (size_t)grp * g.Q + slot; }

__device__ __forceinline__ int classify(const uint8_t *pkts, const Geo &g, uint32_t k, int &slot, int &grp) {
    const uint4 h = __ldg(reinterpret_cast<const uint4 *>(pkts + (size_t)k * g.stride));
    const uint32_t sid = (h.x & 0xFFFFu) - g.stream_base, cg = h.x >> 16;
    const uint64_t seq = (static_cast<uint64_t>(h.w) << 32) | h.z;
    if (sid >= (uint32_t)g.S || cg >= (uint32_t)g.gps) return kInvalid;
    if (seq < g.seq0) return kLate;
    if (seq - g.seq0 >= (uint64_t)g.Q) return kEarly;
    slot = (int)(seq - g.seq0);
    grp = (int)(sid * g.gps + cg);
    return kOk;
}

constexpr int kIndexThreads = 512;           // claim / tally block size (one counter atomic per block)

__global__ void init_kernel(uint32_t *owner, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        owner[i] = kNone;
}

// Adds this block's counts v[0..n) (one value per thread, summed per warp, then per block in shared
// memory) to dst[0..n): one global atomic per counter and block, as the counters are single words
// every block adds to. All threads of the block must call it.
template <int n>
__device__ __forceinline__ void block_add(const uint32_t (&v)[n], uint32_t *const (&dst)[n]) {
    __shared__ uint32_t part[n];
    if (threadIdx.x < n) part[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < n; ++c) {
        const uint32_t w = __reduce_add_sync(0xffffffffu, v[c]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&part[c], w);
    }
    __syncthreads();
    if (threadIdx.x < n && part[threadIdx.x] && dst[threadIdx.x]) atomicAdd(dst[threadIdx.x], part[threadIdx.x]);
}

// count_in_window (the zero-copy path): stats[1] also grows by every in-window packet; the tally
// then moves the owners among them from stats[1] to stats[0], leaving the duplicates in stats[1].
__global__ void claim_kernel(const uint8_t *__restrict__ pkts, Geo g, uint32_t *owner, uint32_t *stats,
                             int count_in_window) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    int cls = -1, slot = 0, grp = 0;
    if (k < g.n_pkts) {
        cls = classify(pkts, g, k, slot, grp);
        if (cls == kOk) atomicMin(&owner[oidx(g, slot, grp)], k);
    }
    const uint32_t v[4] = {cls == kOk ? 1u : 0u, cls == kLate ? 1u : 0u, cls == kEarly ? 1u : 0u,
                           cls == kInvalid ? 1u : 0u};
    uint32_t *const dst[4] = {count_in_window ? &stats[1] : nullptr, &stats[2], &stats[3], &stats[4]};
    block_add(v, dst);
}

// Tally only (the zero-copy path), one thread per (slot, group): filled, lost, and the ok count.
// Every filled slot has exactly one owner, an in-window packet, so ok = filled slots and the
// duplicates are the in-window packets the claim counted into stats[1] less the owners: no packet
// header is read again.
__global__ void tally_kernel(Geo g, const uint32_t *__restrict__ owner, uint8_t *__restrict__ filled, uint32_t *lost,
                             uint32_t *stats) {
    const uint64_t sg = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    bool have = false;
    if (sg < (uint64_t)g.Q * g.G) {
        const int grp = (int)(sg % g.G);
        have = owner[oidx(g, (int)(sg / g.G), grp)] != kNone;
        filled[sg] = have ? 1 : 0;
        if (!have) {
            for (int c = 0; c < 8; ++c) atomicAdd(&lost[8 * grp + c], 4u);
        }
    }
    // ok += n, dup -= n (modulo 2^32: adding the two's complement subtracts)
    const uint32_t v[2] = {have ? 1u : 0u, have ? 0xFFFFFFFFu : 0u};
    uint32_t *const dst[2] = {&stats[0], &stats[1]};
    block_add(v, dst);
}

// F-engine flags (Sec. II-C): one warp per packet; a packet that owns its slot adds the flags of its
// footer (at byte `footer`: [4 t][8 f][N/8] bytes, bit n % 8 of byte n / 8 = input n flagged) to the
// per-input counts count[f][n] and the pair intersections pairs[f][p(i,j)], i <= j. A row with E
// flagged inputs costs E (E + 1) / 2 atomic adds, spread over the warp; rows without flags are
// skipped after one warp vote.
constexpr int kFlagThreads = 128;

__global__ void __launch_bounds__(kFlagThreads) flags_kernel(const uint8_t *__restrict__ pkts, Geo g,
                                                            const uint32_t *__restrict__ owner, uint32_t footer,
                                                            uint32_t *count, uint32_t *pairs) {
    __shared__ uint16_t list[kFlagThreads / 32][4096];
    __shared__ int n_set[kFlagThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t k = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    if (k >= g.n_pkts) return;
    int slot = 0, grp = 0;
    if (classify(pkts, g, (uint32_t)k, slot, grp) != kOk) return;
    if (owner[oidx(g, slot, grp)] != (uint32_t)k) return;          // duplicate: its first arrival counts
    const int N = g.N, NB = N / 8;
    const int64_t P = npairs(N);
    const uint8_t *foot = pkts + (size_t)k * g.stride + footer;
    for (int row = 0; row < 32; ++row) {                             // (t % 4, f % 8) = (row / 8, row % 8)
        const uint8_t *bits = foot + (size_t)row * NB;
        int any = 0;
        for (int b = lane; b < NB; b += 32) any |= bits[b];
        if (!__any_sync(0xffffffffu, any)) continue;
        const int f = 8 * grp + (row & 7);
        if (lane == 0) n_set[w] = 0;
        __syncwarp();
        for (int b = lane; b < NB; b += 32) {
            for (uint32_t v = bits[b]; v; v &= v - 1) {
                const int i = 8 * b + __ffs(v) - 1;
                list[w][atomicAdd(&n_set[w], 1)] = (uint16_t)i;
                atomicAdd(&count[(size_t)f * N + i], 1u);
            }
        }
        __syncwarp();
        const int E = n_set[w];
        for (int a = 0; a < E; ++a) {
            const int ia = list[w][a];
            for (int b = a + lane; b < E; b += 32) {
                const int ib = list[w][b];
                const int i = min(ia, ib), j = max(ia, ib);
                atomicAdd(&pairs[(size_t)f * P + (int64_t)i * N - (int64_t)i * (i - 1) / 2 + (j - i)], 1u);
            }
        }
        __syncwarp();
    }
}

// One warp per packet (warps [0, n_pkts)) and one warp per (slot, group) (the warps after them).
// Blocks of 128 threads: small enough to run beside the correlation kernel on the same SM, so the
// assembly of one frame can overlap the correlation of the previous one.
constexpr int kCopyThreads = 128;

__global__ void __launch_bounds__(kCopyThreads) copy_kernel(const uint8_t *__restrict__ pkts, Geo g,
                                                   const uint32_t *__restrict__ owner, uint8_t *__restrict__ frame,
                                                   uint8_t *__restrict__ filled, uint32_t *lost, uint32_t *stats) {
    const uint64_t wid = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int row_vec = g.N / 2;                  // 16-byte vectors in one 8-channel row (8N bytes)
    if (wid < g.n_pkts) {
        const uint32_t k = (uint32_t)wid;
        int slot = 0, grp = 0;
        if (classify(pkts, g, k, slot, grp) != kOk) return;
        const bool mine = owner[oidx(g, slot, grp)] == k;
        if (lane == 0) atomicAdd(&stats[mine ? 0 : 1], 1u);
        if (!mine) return;
        const uint4 *src = reinterpret_cast<const uint4 *>(pkts + (size_t)k * g.stride + 16);
        for (int tt = 0; tt < 4; ++tt) {
            uint4 *dst = reinterpret_cast<uint4 *>(frame + ((size_t)(4 * slot + tt) * g.F + 8 * grp) * g.N);
            for (int v = lane; v < row_vec; v += 32) __stcs(dst + v, __ldcs(src + tt * row_vec + v));
        }
        return;
    }
    const uint64_t sg = wid - g.n_pkts;
    if (sg >= (uint64_t)g.Q * g.G) return;
    const int slot = (int)(sg / g.G), grp = (int)(sg % g.G);
    const bool have = owner[oidx(g, slot, grp)] != kNone;
    if (lane == 0) filled[sg] = have ? 1 : 0;
    if (have) return;
    if (lane < 8) atomicAdd(&lost[8 * grp + lane], 4u);
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int tt = 0; tt < 4; ++tt) {
        uint4 *dst = reinterpret_cast<uint4 *>(frame + ((size_t)(4 * slot + tt) * g.F + 8 * grp) * g.N);
        for (int v = lane; v < row_vec; v += 32) __stcs(dst + v, z);
    }
}

}  // namespace asmb
}  // namespace xe

using namespace xe;

extern "C" {

size_t xe_assemble_workspace_size(xe_shape s) {
    if (!valid_shape(s) || s.n_time % 4 || s.n_chan % 8) return 0;
    return (size_t)round_up((int64_t)(s.n_time / 4) * (s.n_chan / 8) * 4, 256);
}

int xe_assemble(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                xe_shape s, uint8_t *frame, uint8_t *filled, uint32_t *lost, uint32_t *stats, void *ws,
                size_t ws_bytes, void *stream) {
    return xe::assemble_streams(pkts, n_pkts, pkt_stride, seq0, gps, 0, s, frame, filled, lost, stats, ws, ws_bytes,
                                static_cast<cudaStream_t>(stream));
}

size_t xe_flag_counts_workspace_size(xe_shape s) {
    if (!valid_shape(s) || s.n_time % 4 || s.n_chan % 8) return 0;
    return (size_t)round_up((int64_t)(s.n_time / 4) * (s.n_chan / 8), 64) * 4 + 256;
}

int xe_flag_counts(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps, xe_shape s,
                   uint32_t *flag_count, uint32_t *flag_pairs, void *ws, size_t ws_bytes, void *stream) {
    if (!valid_shape(s) || s.n_time < 4 || s.n_time % 4 || s.n_chan % 8 || gps < 1 || (s.n_chan / 8) % gps)
        return XE_EINVAL;
    if (!flag_count || !flag_pairs || (n_pkts && !pkts)) return XE_EINVAL;
    const uint32_t footer = 16u + 32u * (uint32_t)s.n_inputs;
    if (pkt_stride % 16 || pkt_stride < footer + 4u * (uint32_t)s.n_inputs) return XE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(pkts) & 15) || (reinterpret_cast<uintptr_t>(ws) & 3) ||
        (reinterpret_cast<uintptr_t>(flag_count) & 3) || (reinterpret_cast<uintptr_t>(flag_pairs) & 3))
        return XE_EINVAL;
    if (!ws || ws_bytes < xe_flag_counts_workspace_size(s)) return XE_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    asmb::Geo g;
    g.seq0 = seq0;
    g.n_pkts = n_pkts;
    g.stride = pkt_stride;
    g.N = s.n_inputs;
    g.F = s.n_chan;
    g.Q = s.n_time / 4;
    g.G = s.n_chan / 8;
    g.gps = gps;
    g.S = g.G / gps;
    uint32_t *owner = static_cast<uint32_t *>(ws);
    const int64_t slots = (int64_t)g.Q * g.G;
    uint32_t *scratch = owner + round_up(slots, 64);             // the claim's late / early counters
    XE_TRY_CUDA(cudaMemsetAsync(scratch, 0, 32, st));
    asmb::init_kernel<<<(unsigned)std::min<int64_t>((slots + 255) / 256, 4096), 256, 0, st>>>(owner, slots);
    XE_TRY_CUDA(cudaGetLastError());
    if (n_pkts) {
        asmb::claim_kernel<<<(n_pkts + 255) / 256, 256, 0, st>>>(pkts, g, owner, scratch, 0);
        XE_TRY_CUDA(cudaGetLastError());
        const uint64_t blocks = ((uint64_t)n_pkts * 32 + asmb::kFlagThreads - 1) / asmb::kFlagThreads;
        if (blocks > 0x7FFFFFFFull) return XE_EINVAL;
        asmb::flags_kernel<<<(unsigned)blocks, asmb::kFlagThreads, 0, st>>>(pkts, g, owner, footer, flag_count,
                                                                             flag_pairs);
        XE_TRY_CUDA(cudaGetLastError());
    }
    return XE_OK;
}

}  // extern "C"

namespace xe {
namespace asmb {

// Checks the arguments shared by every assembly form and fills the geometry.
static int make_geo(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                    uint32_t stream_base, const xe_shape &s, const uint8_t *filled, const uint32_t *lost,
                    const uint32_t *stats, Geo &g) {
    if (!valid_shape(s) || s.n_time < 4 || s.n_time % 4 || s.n_chan % 8 || gps < 1 || (s.n_chan / 8) % gps)
        return XE_EINVAL;
    if (!filled || !lost || !stats || (n_pkts && !pkts)) return XE_EINVAL;
    if (pkt_stride % 16 || pkt_stride < 16u + 32u * (uint32_t)s.n_inputs) return XE_EINVAL;
    if (reinterpret_cast<uintptr_t>(pkts) & 15) return XE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(lost) | reinterpret_cast<uintptr_t>(stats)) & 3) return XE_EINVAL;
    g.stream_base = stream_base;
    g.seq0 = seq0;
    g.n_pkts = n_pkts;
    g.stride = pkt_stride;
    g.N = s.n_inputs;
    g.F = s.n_chan;
    g.Q = s.n_time / 4;
    g.G = s.n_chan / 8;
    g.gps = gps;
    g.S = g.G / gps;
    return XE_OK;
}

// init, claim and copy (kCopy) or tally (!kCopy) on stream st.
template <bool kCopy>
static int launch(const uint8_t *pkts, const Geo &g, uint32_t *owner, uint8_t *frame, uint8_t *filled, uint32_t *lost,
                  uint32_t *stats, cudaStream_t st) {
    const int64_t slots = (int64_t)g.Q * g.G;
    init_kernel<<<(unsigned)std::min<int64_t>((slots + 255) / 256, 4096), 256, 0, st>>>(owner, slots);
    XE_TRY_CUDA(cudaGetLastError());
    if (g.n_pkts) {
        claim_kernel<<<(g.n_pkts + kIndexThreads - 1) / kIndexThreads, kIndexThreads, 0, st>>>(pkts, g, owner, stats,
                                                                                              kCopy ? 0 : 1);
        XE_TRY_CUDA(cudaGetLastError());
    }
    if (!kCopy) {
        const uint64_t blocks = ((uint64_t)slots + kIndexThreads - 1) / kIndexThreads;
        if (blocks > 0x7FFFFFFFull) return XE_EINVAL;
        tally_kernel<<<(unsigned)blocks, kIndexThreads, 0, st>>>(g, owner, filled, lost, stats);
        XE_TRY_CUDA(cudaGetLastError());
        return XE_OK;
    }
    const uint64_t warps = (uint64_t)g.n_pkts + (uint64_t)slots;
    const uint64_t blocks = (warps + kCopyThreads / 32 - 1) / (kCopyThreads / 32);
    if (blocks > 0x7FFFFFFFull) return XE_EINVAL;
    copy_kernel<<<(unsigned)blocks, kCopyThreads, 0, st>>>(pkts, g, owner, frame, filled, lost, stats);
    XE_TRY_CUDA(cudaGetLastError());
    return XE_OK;
}

}  // namespace asmb
}  // namespace xe

// xe_assemble for the frame of some streams: packets whose header stream id is stream_base + s map
// to the frame's stream s (the serving loop assembles each F-engine stream into its own frame).
int xe::assemble_streams(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                         uint32_t stream_base, xe_shape s, uint8_t *frame, uint8_t *filled, uint32_t *lost,
                         uint32_t *stats, void *ws, size_t ws_bytes, cudaStream_t st) {
    asmb::Geo g;
    if (int e = asmb::make_geo(pkts, n_pkts, pkt_stride, seq0, gps, stream_base, s, filled, lost, stats, g)) return e;
    if (!frame || (reinterpret_cast<uintptr_t>(frame) & 15)) return XE_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) & 3) return XE_EINVAL;
    if (!ws || ws_bytes < xe_assemble_workspace_size(s)) return XE_ENOMEM;
    return asmb::launch<true>(pkts, g, static_cast<uint32_t *>(ws), frame, filled, lost, stats, st);
}

// The frame's index without its payload: owner[group * T/4 + slot] = the packet that supplies samples
// 4 slot .. 4 slot + 3 of channels 8 group .. 8 group + 7, or 0xFFFFFFFF (lost: zeros); filled,
// lost and stats exactly as xe_assemble gives them.
int xe::index_streams(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int32_t gps,
                      uint32_t stream_base, xe_shape s, uint8_t *filled, uint32_t *lost, uint32_t *stats,
                      uint32_t *owner, cudaStream_t st) {
    asmb::Geo g;
    if (int e = asmb::make_geo(pkts, n_pkts, pkt_stride, seq0, gps, stream_base, s, filled, lost, stats, g)) return e;
    if (!owner || (reinterpret_cast<uintptr_t>(owner) & 3)) return XE_EINVAL;
    return asmb::launch<false>(pkts, g, owner, nullptr, filled, lost, stats, st);
}

// ---------------------------------------------------------------------------- allocation-free variant
// xe_assemble_noalloc runs the same three kernels as xe_assemble, but its owner table lives in a
// fixed-size array compiled into the library instead of in caller-provided workspace. It exists
// for callers that cannot obtain device memory at the point where they assemble frames (see the
// declaration in xe.h). Every call on a device shares this one array.

namespace xe {
namespace asmb {

static __device__ __align__(256) uint32_t g_noalloc_owner[XE_ASSEMBLE_NOALLOC_MAX_SLOTS];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Identity of the current device's context (0 if there is none yet). A context id is unique for the
// life of the process, so a context created after a device reset gets a new one.
static unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_owner on the current device. In host code the symbol itself is only a
// host-side stand-in, so the kernels must be given this address. It is looked up with the device
// current on the first call in each of the device's contexts (the first call after cudaDeviceReset
// looks it up again: the array then lives at a new address) and cached against the context's id.
static uint32_t *noalloc_owner(int *status) {
    struct Entry {
        unsigned long long ctx = 0;
        uint32_t *addr = nullptr;
    };
    static Entry cache[64];
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *status = cuda_fail(e); return nullptr; }
    if (dev < 0 || dev >= 64) { *status = XE_EINVAL; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    unsigned long long ctx = current_ctx_id();
    if (ctx != 0 && cache[dev].ctx == ctx && cache[dev].addr) return cache[dev].addr;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_owner);       // creates the context if there is none yet
    if (e != cudaSuccess || !p) { *status = cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol); return nullptr; }
    if (ctx == 0) ctx = current_ctx_id();
    cache[dev].ctx = ctx;
    cache[dev].addr = static_cast<uint32_t *>(p);
    return cache[dev].addr;
}

}  // namespace asmb
}  // namespace xe

extern "C" int xe_assemble_noalloc(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                                   int32_t gps, xe_shape s, uint8_t *frame, uint8_t *filled, uint32_t *lost,
                                   uint32_t *stats, void *stream) {
    asmb::Geo g;
    if (int e = asmb::make_geo(pkts, n_pkts, pkt_stride, seq0, gps, 0, s, filled, lost, stats, g)) return e;
    if (!frame || (reinterpret_cast<uintptr_t>(frame) & 15)) return XE_EINVAL;
    const int64_t slots = (int64_t)g.Q * g.G;
    if (slots > XE_ASSEMBLE_NOALLOC_MAX_SLOTS) return XE_ENOMEM;    // frame larger than the static table
    int status = XE_OK;
    uint32_t *owner = asmb::noalloc_owner(&status);
    if (!owner) return status;
    // the table keeps whatever the previous call left in it: launch() first resets the slots this
    // frame uses (init), then claims and copies exactly as xe_assemble does
    return asmb::launch<true>(pkts, g, owner, frame, filled, lost, stats, static_cast<cudaStream_t>(stream));
}
