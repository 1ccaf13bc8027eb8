// xe_device.cuh -- inline-PTX building blocks for sm_103a: mbarriers, TMA tensor loads and
// 5th-generation tensor-core (tcgen05) MMA with tensor-memory accumulators.
#pragma once

#include <cstdint>
#include <cuda.h>

namespace xe {
namespace dev {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ mbarrier

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// As mbar_try_wait, but a thread whose phase has not completed may stay suspended for up to
// hint_ns; it resumes as soon as the phase completes, so waiting warps issue no spin instructions.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits until the phase with the given parity has completed, for at most `limit_ns`.
// Returns false when the limit expired (the caller records a timeout and unwinds).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// ------------------------------------------------------------------ clusters (CTA pairs)

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of all CTAs of the cluster; orders prior memory operations at cluster scope.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrives (release, cluster scope) on the mbarrier at the same shared-memory offset in CTA `rank`.
__device__ __forceinline__ void mbar_arrive_cluster(uint64_t *bar, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

// Arrive on the mbarrier at the same offset in CTA `rank` with the default (release, CTA-scope)
// semantics; the producer of the guarded data has already fenced it for its consumer.
__device__ __forceinline__ void mbar_arrive_remote(uint64_t *bar, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

// Named barrier among `nthreads` threads (multiple of 32) of the CTA.
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ANDs a predicate over its `nthreads` participants: every thread gets the
// same result, so a group of warps can take a decision together.
__device__ __forceinline__ bool named_sync_and(uint32_t id, uint32_t nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred ? 1u : 0u), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// try_wait with cluster-scope acquire (for barriers other CTAs of the cluster arrive on).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Address of the shared-memory location `saddr` (a shared::cta address) in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(saddr), "r"(rank));
    return remote;
}

// Stores into another CTA's shared memory (a shared::cluster address from mapa).
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// ------------------------------------------------------------------ proxies / TMA

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// 3-D tiled tensor load global -> shared, completion counted on `bar` in bytes.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t c0, int32_t c1, int32_t c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)),
          "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Prefetches a 3-D tile of a tensor map into L2 (no shared memory, no completion signal).
// Out-of-range parts of the box are ignored.
__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap *map, int32_t c0, int32_t c1, int32_t c2) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

// 16-byte global load cached in L2 only (streamed operand data: each byte is used once per SM).
__device__ __forceinline__ uint4 ld_stream_16(const uint8_t *ptr) {
    uint4 v;
    asm("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr));
    return v;
}

// Adds v to *ptr in L2 (relaxed, device scope) without returning the old value: the thread does not
// wait for the line, so an epilogue that adds into existing visibilities keeps no loads in flight.
__device__ __forceinline__ void red_add(int32_t *ptr, int32_t v) {
    asm volatile("red.global.add.s32 [%0], %1;" ::"l"(ptr), "r"(v));
}

// Hint: bring the 128-byte line holding ptr into L2 (no register result, no fault on the address).
__device__ __forceinline__ void prefetch_l2(const void *ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// ------------------------------------------------------------------ tcgen05 (TMEM + MMA)

// Allocates `ncols` TMEM columns (power of two >= 32); the base address is written to smem.
// Executed by one full warp.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Arrives once on `bar` when every tcgen05 operation issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

// TMEM allocation shared by a CTA pair (cta_group::2): one warp of EACH CTA of the pair executes it.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(ncols) : "memory");
}
// Register split between warpgroups (all four warps of a warpgroup execute it): dec hands registers
// back to the CTA's pool, inc waits until the pool holds enough. The counts must add up to at most
// the launch's registers per thread x threads, which the host checks before the launch.
template <uint32_t kRegs>
__device__ __forceinline__ void setmaxnreg_dec() {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegs));
}
template <uint32_t kRegs>
__device__ __forceinline__ void setmaxnreg_inc() {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegs));
}
__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Pair MMA (issued by one thread of the pair's even CTA): D (M = 256 rows, half in each CTA's TMEM)
// (+)= A (128 rows from each CTA's shared memory) * B (N/2 columns from each CTA's shared memory).
__device__ __forceinline__ void mma_f8f6f4_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                                uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrives once on the mbarrier at this offset in every CTA of `mask` when the pair MMAs issued so
// far by this thread have completed.
__device__ __forceinline__ void tc_commit_pair_multicast(uint64_t *bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(smem_u32(bar)), "h"(mask) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, 8-bit float operands, FP32 accumulate. `acc` = 0 overwrites.
__device__ __forceinline__ void mma_f8f6f4(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                           uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the 128-byte swizzle:
// rows of 128 bytes, 8-row (1024-byte) swizzle atoms stacked along M/N.
//   bits  0-13  start address >> 4
//   bits 16-29  leading byte offset >> 4 (not used by swizzled K-major layouts; 1)
//   bits 32-45  stride byte offset >> 4 (1024 bytes between 8-row groups)
//   bits 46-47  descriptor version 1
//   bits 61-63  layout: 2 = 128-byte swizzle
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(1u) << 16;
    d |= static_cast<uint64_t>(1024u >> 4) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(2u) << 61;
    return d;
}

// Instruction descriptor of kind::f8f6f4 with E5M2 x E5M2 -> F32, both operands K-major.
//   bits 4-5 D format (1 = F32), 7-9 A format, 10-12 B format (1 = E5M2),
//   15/16 A/B major (0 = K), 17-22 N >> 3, 24-28 M >> 4
__host__ __device__ constexpr uint32_t idesc_e5m2_f32(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// 32 lanes x 32 consecutive 32-bit TMEM columns -> 32 registers per thread (thread = lane).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
// 32 lanes x 16 consecutive 32-bit TMEM columns -> 16 registers per thread (thread = lane).
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of an MN-major operand tile with the 128-byte swizzle: one row
// of 128 bytes (128 values along M or N) per K index, 8-row (1024-byte) swizzle atoms stacked
// along K (stride byte offset 1024); `lbo` is the byte distance between consecutive 128-value
// atoms along M/N (used when the operand spans more than 128 values, e.g. N = 256).
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>(1024u >> 4) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(2u) << 61;
    return d;
}

// Same as idesc_e5m2_f32 with both operands MN-major (transpose bits 15 and 16 set).
__host__ __device__ constexpr uint32_t idesc_e5m2_f32_mn(uint32_t m, uint32_t n) {
    return idesc_e5m2_f32(m, n) | (1u << 15) | (1u << 16);
}

// Same as idesc_e5m2_f32_mn with E4M3 x E4M3 operands (format code 0 in both type fields).
__host__ __device__ constexpr uint32_t idesc_e4m3_f32_mn(uint32_t m, uint32_t n) {
    return (1u << 4) | ((n >> 3) << 17) | ((m >> 4) << 24) | (1u << 15) | (1u << 16);
}

// ------------------------------------------------------------------ 4-bit -> E5M2

// Four packed 4-bit two's-complement values (one per byte, in bits 0-3 of each byte) to four
// E5M2 codes. v = u - 8 with u = nibble ^ 8 in [0, 15]: the half-precision number with bits
// 0x6400 | u equals 1024 + u exactly, and subtracting 1032 leaves v exactly. For |v| <= 8 the low
// eight bits of the half are zero, so its high byte is the E5M2 code of v.
__device__ __forceinline__ uint32_t nibbles_to_e5m2(uint32_t lo_nibbles) {
    const uint32_t u = (lo_nibbles & 0x0F0F0F0Fu) ^ 0x08080808u;
    // bytes u0 u1 u2 u3 -> halves (0x64|u0, 0x64|u1) and (0x64|u2, 0x64|u3)
    const uint32_t h01 = __byte_perm(u, 0x64646464u, 0x4140);
    const uint32_t h23 = __byte_perm(u, 0x64646464u, 0x4342);
    uint32_t d01, d23;
    const uint32_t k = 0x64086408u;   // (1032, 1032) as half2
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d01) : "r"(h01), "r"(k));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d23) : "r"(h23), "r"(k));
    return __byte_perm(d01, d23, 0x7531);
}

// Four packed samples x_0..x_3 (bytes re<<4 | im, 4-bit two's complement) -> eight E5M2 codes,
// returned as wre = (16 re_0, 16 re_1, 16 re_2, 16 re_3) and wim = (im_0, .., im_3). Per
// half-precision lane, (x & 0x000F) ^ 0x6408 has the bits of 1024 + (im ^ 8) = 1032 + im and
// (x & 0x00F0) ^ 0x6480 those of 1024 + 16 (re ^ 8) = 1152 + 16 re; subtracting 1032 resp. 1152 is
// exact and leaves im resp. 16 re, whose low bytes are zero, so their high bytes are the E5M2 codes.
// One shift and four three-input logic operations with both constants as immediates (written out:
// left to the compiler the mask-and-flip took more instructions), four half2 subtractions and two
// byte permutes for eight codes.
__device__ __forceinline__ void expand4_e5m2(uint32_t x, uint32_t &wre, uint32_t &wim) {
    uint32_t x8, im02, im13, re02, re13;
    asm("shr.b32 %0, %1, 8;" : "=r"(x8) : "r"(x));
    // lut 0x6A: (a & b) ^ c
    asm("lop3.b32 %0, %1, 0x000F000F, 0x64086408, 0x6A;" : "=r"(im02) : "r"(x));
    asm("lop3.b32 %0, %1, 0x000F000F, 0x64086408, 0x6A;" : "=r"(im13) : "r"(x8));
    asm("lop3.b32 %0, %1, 0x00F000F0, 0x64806480, 0x6A;" : "=r"(re02) : "r"(x));
    asm("lop3.b32 %0, %1, 0x00F000F0, 0x64806480, 0x6A;" : "=r"(re13) : "r"(x8));
    const uint32_t k_im = 0x64086408u, k_re = 0x64806480u;
    asm("sub.rn.f16x2 %0, %0, %1;" : "+r"(im02) : "r"(k_im));
    asm("sub.rn.f16x2 %0, %0, %1;" : "+r"(im13) : "r"(k_im));
    asm("sub.rn.f16x2 %0, %0, %1;" : "+r"(re02) : "r"(k_re));
    asm("sub.rn.f16x2 %0, %0, %1;" : "+r"(re13) : "r"(k_re));
    // the codes sit in bytes 1 and 3 of each word: (w02.b1, w13.b1, w02.b3, w13.b3)
    wre = __byte_perm(re02, re13, 0x7351);
    wim = __byte_perm(im02, im13, 0x7351);
}

// 16 packed samples -> 32 E5M2 codes in groups of four inputs: (16 re_0..16 re_3, im_0..im_3,
// 16 re_4.., im_4.., ...). This is the operand row order of the MN-major engines.
__device__ __forceinline__ void expand16_e5m2(const uint4 &in, uint4 &lo, uint4 &hi) {
    expand4_e5m2(in.x, lo.x, lo.y);
    expand4_e5m2(in.y, lo.z, lo.w);
    expand4_e5m2(in.z, hi.x, hi.y);
    expand4_e5m2(in.w, hi.z, hi.w);
}

// Operands of the folded product D = S S^T - 2 A B^T (a = Re x, b = Im x, s = a + b), scaled so that
// D carries a factor 16: four packed samples (bytes re<<4 | im) -> ws = E4M3 codes of 4s, wa = E5M2
// codes of -8a, wb = E5M2 codes of 4b (one code per sample, samples 0..3 in bytes 0..3); then
// S S^T = 16 s s and A B^T = -32 a b.
// Per half-precision lane: (x & 0x00F0) ^ 0x6080 has the bits of 512 + 8 (a ^ 8) = 576 + 8a, and
// (x & 0x000F) ^ 0x6C08 those of 4096 + 4 (b ^ 8) = 4128 + 4b; 576 - (.) and (.) - 4128 are exact
// and leave -8a and 4b, whose at most three significant bits sit in the high byte of the half: that
// byte is the E5M2 code. -0.5 (-8a) + 4b = 4s is exact too; |4s| <= 64 with at most four
// significant bits, so its E4M3 conversion is exact.
__device__ __forceinline__ void fold4(uint32_t x, uint32_t &ws, uint32_t &wa, uint32_t &wb) {
    uint32_t x8, re02, re13, im02, im13;
    asm("shr.b32 %0, %1, 8;" : "=r"(x8) : "r"(x));
    // lut 0x6A: (a & b) ^ c
    asm("lop3.b32 %0, %1, 0x00F000F0, 0x60806080, 0x6A;" : "=r"(re02) : "r"(x));
    asm("lop3.b32 %0, %1, 0x00F000F0, 0x60806080, 0x6A;" : "=r"(re13) : "r"(x8));
    asm("lop3.b32 %0, %1, 0x000F000F, 0x6C086C08, 0x6A;" : "=r"(im02) : "r"(x));
    asm("lop3.b32 %0, %1, 0x000F000F, 0x6C086C08, 0x6A;" : "=r"(im13) : "r"(x8));
    // 576, 4128, -0.5 as half pairs
    const uint32_t k_re = 0x60806080u, k_im = 0x6C086C08u, k_half = 0xB800B800u;
    uint32_t na02, na13, b02, b13, s02, s13;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(na02) : "r"(k_re), "r"(re02));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(na13) : "r"(k_re), "r"(re13));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(b02) : "r"(im02), "r"(k_im));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(b13) : "r"(im13), "r"(k_im));
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(s02) : "r"(na02), "r"(k_half), "r"(b02));
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(s13) : "r"(na13), "r"(k_half), "r"(b13));
    wa = __byte_perm(na02, na13, 0x7351);
    wb = __byte_perm(b02, b13, 0x7351);
    // E4M3 pairs (samples 0, 2) and (1, 3), each half's code in the byte of the same position
    uint32_t c;
    asm("{\n\t.reg .b16 l, h;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 l, %1;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 h, %2;\n\t"
        "mov.b32 %0, {l, h};\n\t}"
        : "=r"(c) : "r"(s02), "r"(s13));
    ws = __byte_perm(c, 0, 0x3120);
}

// 16 packed samples -> 16 codes each of 4s (E4M3), -8a and 4b (E5M2), in input order.
__device__ __forceinline__ void fold16(const uint4 &in, uint4 &s, uint4 &a, uint4 &b) {
    fold4(in.x, s.x, a.x, b.x);
    fold4(in.y, s.y, a.y, b.y);
    fold4(in.z, s.z, a.z, b.z);
    fold4(in.w, s.w, a.w, b.w);
}

}  // namespace dev
}  // namespace xe
