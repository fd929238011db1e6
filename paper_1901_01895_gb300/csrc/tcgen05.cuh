// Device helpers shared by the tensor-core kernels: mbarriers with bounded waits,
// bulk (TMA) copies, tcgen05 descriptors, MMA issue and commit, TMEM loads, BF16 splits.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace mmf {
namespace tc {

constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;   // every mbarrier wait gives up after 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the phase
// completes or about 2 us pass, instead of spinning on the issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(2000u)
        : "memory");
    return ok != 0;
}
// try_wait with cluster-scope acquire, for barriers that the peer CTA of a pair arrives on
// (release.cluster): the peer's writes before its arrival are visible after the wait.
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(2000u)
        : "memory");
    return ok != 0;
}
// Bounded wait for completion of the phase with the given parity; false on timeout.
// CL: cluster-scope acquire (the barrier receives arrivals from the peer CTA).
// The waiting part of mbar_wait, out of line: kernels wait in many places, and one copy of
// the polling loop keeps their code small.
template <bool CL>
__device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t parity, int* err, int code) {
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (CL ? mbar_try_wait_cl(b, parity) : mbar_try_wait_sleep(b, parity)) return true;
        if ((it & 15) == 0) {
            if (globaltimer() - t0 > WAIT_LIMIT_NS) {
                atomicCAS(err, 0, code);
                return false;
            }
            if (*(volatile int*)err != 0) return false;
        }
    }
}
// Bounded wait for completion of the phase with the given parity; false on timeout.
// CL: cluster-scope acquire (the barrier receives arrivals from the peer CTA).
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, int code) {
    if (CL ? mbar_try_wait_cl(b, parity) : mbar_try_wait(b, parity)) return true;
    return mbar_wait_slow<CL>(b, parity, err, code);
}
// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, int* err, int code) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(b, parity, err, code) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}
// One lane of the (converged) warp is elected: the warp's uniform values stay in uniform
// registers around the single-thread tcgen05 and bulk-copy instructions.
__device__ __forceinline__ bool elect_one() {
    uint32_t pred = 0;
    asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.u32 %0, 1, 0, P;\n\t}" : "=r"(pred));
    return pred != 0;
}
// Bounded wait polled by lane 0 of a converged warp; the outcome is a warp vote (uniform).
template <bool CL = false>
__device__ __forceinline__ bool warp_wait_u(uint64_t* b, uint32_t parity, int* err, int code) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait<CL>(b, parity, err, code);
    return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor for a K-major tile with SW-byte swizzled rows:
// start address, leading offset (unused for swizzled K-major, 16 B), 8-row group stride
// 8*SW bytes, descriptor version 1, swizzle mode (128 B: 2, 64 B: 4, 32 B: 6).
template <int SW>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
    constexpr uint64_t mode = SW == 128 ? 2 : (SW == 64 ? 4 : 6);
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((8 * SW) >> 4) << 32) |
           ((uint64_t)1 << 46) | (mode << 61);
}
// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// ---- CTA pairs (thread-block clusters of two, tcgen05 cta_group::2) ----
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of both CTAs arrives, then waits (release/acquire at cluster scope).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared::cluster address of the variable at local shared address saddr in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// Arrive on an mbarrier of another CTA of the cluster (shared::cluster address).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// Instruction descriptor of a pair MMA: BF16 x BF16 -> FP32, K-major, M = 256 (128 rows per
// CTA), N = n (each CTA holds n/2 rows of B).
__device__ __forceinline__ uint32_t idesc_bf16_pair(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Instruction descriptor of a pair MMA with TF32 operands (kind::tf32): FP32 accumulate,
// K-major, M = 256, N = n.
__device__ __forceinline__ uint32_t idesc_tf32_pair(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
template <bool TF>
__device__ __forceinline__ uint32_t idesc_pair(int n) { return TF ? idesc_tf32_pair(n) : idesc_bf16_pair(n); }
template <bool TF>
__device__ __forceinline__ void mma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (TF) mma_tf32_pair(d_tmem, a, b, idesc, acc);
    else mma_bf16_pair(d_tmem, a, b, idesc, acc);
}
// Completion of the pair's MMAs issued so far arrives on the barrier at the same shared
// offset in every CTA of ctamask.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t ctamask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(ctamask)
        : "memory");
}
// Issue a 32-lane x 16-column TMEM load (results valid only after tmem_wait16 on them).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// Wait for the outstanding TMEM loads; the registers are tied to the wait so no use of
// them can be scheduled before it.
__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}
// The same for 4 and 12 registers.
__device__ __forceinline__ void tmem_wait4(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
}
__device__ __forceinline__ void tmem_wait12(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
                 :
                 : "memory");
}
// Wait for the outstanding TMEM loads into r[0..7]; the eight registers are tied to the wait
// so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait8(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}
// Two floats -> packed BF16 pair (first in the low half), round to nearest even.
__device__ __forceinline__ uint32_t pack_bf16(float first, float second) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(first, second);
    return *reinterpret_cast<const uint32_t*>(&h);
}
// TF32 (FP32 bit pattern, low 13 mantissa bits zero) of x, rounded to nearest, ties away.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// hi = TF32(x); lo = TF32 of the remainder x - hi (exact in FP32).
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}
// hi = BF16(first, second) packed; lo = BF16 of the remainders (first - hi, second - hi).
__device__ __forceinline__ void split_bf16(float first, float second, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16(first, second);
    // (first - h0, second - h1) as one packed fma(h, -1, x): the same rounding as the scalar
    // subtractions
    const float2 h = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xFFFF0000u));
    const float2 r = __ffma2_rn(h, make_float2(-1.f, -1.f), make_float2(first, second));
    lo = pack_bf16(r.x, r.y);
}


// TMEM loads of exactly NS (1..16) consecutive columns of the warp's 32 lanes: the
// power-of-two pieces of NS, so that no column beyond the requested ones is touched.
__device__ __forceinline__ void tmem_ld1(uint32_t a, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[0]) : "r"(a));
}
__device__ __forceinline__ void tmem_ld2(uint32_t a, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void tmem_ld4(uint32_t a, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void tmem_ld8(uint32_t a, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(a));
}
template <int NS>
__device__ __forceinline__ void tmem_ld_n(uint32_t a, uint32_t* r) {
    static_assert(NS >= 1 && NS <= 16, "1..16 columns");
    constexpr int o8 = NS & 16, o4 = o8 + (NS & 8), o2 = o4 + (NS & 4), o1 = o2 + (NS & 2);
    if constexpr ((NS & 16) != 0) tmem_ld16(a, r);
    if constexpr ((NS & 8) != 0) tmem_ld8(a + o8, r + o8);
    if constexpr ((NS & 4) != 0) tmem_ld4(a + o4, r + o4);
    if constexpr ((NS & 2) != 0) tmem_ld2(a + o2, r + o2);
    if constexpr ((NS & 1) != 0) tmem_ld1(a + o1, r + o1);
}
__device__ __forceinline__ void named_bar_sync(int id, int n_threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n_threads) : "memory");
}

}  // namespace tc
}  // namespace mmf
