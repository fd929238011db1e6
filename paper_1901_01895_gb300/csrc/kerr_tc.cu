// Kerr term of Eq. 1 as a pair contraction on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands in shared memory, S tiles by TMA).
//
// Same factorisation as the CUDA-core path (kerr_pairs.cu):
//   u_ij = c_ij Re sum_a A_ia conj(A_ja),  v_ij = c_ij sum_a A_ia A_ja      (pairs i <= j)
//   W_pl = sum_(ij) S_plij u_ij,           Z_pl = sum_(ij) S_plij v_ij
//   K_(p,a) = (i gamma h / 3)[2 sum_l W_pl A_la + sum_l Z_pl conj(A_la)]   (2 pol; 1 pol: Z term only)
// evaluated per tile of 128 time samples as GEMMs D[s][n] = sum_k X[s][k] B[n][k]:
//   rows s      = 128 samples of the tile (the MMA M dimension, one TMEM lane each),
//   K           = the input pairs (ij) of one parity class, 64 per chunk,
//   columns n   = output pairs (p, l) of that class with p in a group G of modes and l
//                 running over the modes whose parity completes the class (N <= 160),
//   X rows      = u, Re v, Im v (two polarisations) or Re v, Im v (one): one accumulator each,
//   B[n][k]     = S_pair[(p l),(ij)] = S_plij, stored on the device already in the
//                 canonical 128-byte-swizzled K-major tile layout so one bulk TMA copy
//                 moves a tile.
// BF16X3 splits both operands x = hi + lo in BF16 and accumulates hi*hi + hi*lo + lo*hi in
// FP32; BF16 uses hi*hi only.
//
// Warp roles (288 threads, one CTA per SM, persistent over (sample tile, mode group)):
//   warps 0-7  form the pair products of a chunk (thread = sample, warps w and w+4 split
//              the 64 pairs), then run the epilogue (thread = sample, w < 4 polarisation 0,
//              w >= 4 polarisation 1): tcgen05.ld of its TMEM lane, contraction with
//              A_l(t) into per-(p, pol) shared accumulators, final store.
//   warp 8     one thread issues the TMA bulk copies of the S tiles (double-buffered) and
//              the tcgen05.mma instructions, and commits completion to mbarriers.
// Every mbarrier wait gives up after one second, records an error code in k.err and
// lets the kernel wind down (TMEM is always released).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace mmf {
namespace {

constexpr int TS = 128;              // samples per tile (MMA M)
constexpr int KCH = 64;              // input pairs per K chunk (one 128-byte swizzle row)
constexpr int NMAX = 160;            // max output columns per (group, class)
constexpr int NPROD_WARPS = 8;
constexpr int NTHREADS = (NPROD_WARPS + 1) * 32;
constexpr int A_TILE = TS * 128;     // bytes of one [128 x 64] bf16 operand tile
constexpr int B_TILE = NMAX * 128;   // bytes of one [160 x 64] bf16 operand tile
constexpr int GMAX = 16;             // max modes per group
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;

enum : int { ERR_NONE = 0, ERR_TIMEOUT_A_EMPTY = 1, ERR_TIMEOUT_A_FULL, ERR_TIMEOUT_B_EMPTY, ERR_TIMEOUT_B_FULL,
             ERR_TIMEOUT_ACC_FULL, ERR_TIMEOUT_ACC_EMPTY, ERR_TIMEOUT_DRAIN };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
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
// Bounded wait for the phase with the given parity; false on timeout (error recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, int code) {
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(b, parity)) {
        if (globaltimer() - t0 > WAIT_LIMIT_NS) {
            atomicCAS(err, 0, code);
            return false;
        }
        if (*(volatile int*)err != 0) return false;
    }
    return true;
}
// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, int* err, int code) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(b, parity, err, code) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
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

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TS >> 4) << 24);
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

// Byte offset of element (row, k) in a [rows x 64] bf16 K-major tile with 128-byte swizzle.
__host__ __device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
    const int chunk = k >> 3;
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
    const __nv_bfloat16 a = __float2bfloat16_rn(lo_elem), b = __float2bfloat16_rn(hi_elem);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// x = hi + lo split: returns hi as float, stores the BF16 remainder value in lo.
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <int NPOL>
__global__ void __launch_bounds__(NTHREADS, 1) kerr_tc_kernel(KerrTC k, const cf* __restrict__ x, cf* __restrict__ out,
                                                              float scale, int N) {
    constexpr int ROWS = NPOL == 2 ? 3 : 2;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned carve-up
    uint8_t* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int nsplit = k.x3 ? 2 : 1;
    uint8_t* A_s = base;                                               // [ROWS][nsplit][A_TILE]
    uint8_t* B_s = A_s + ROWS * 2 * A_TILE;                            // [2 stages][nsplit][B_TILE]
    float* sacc = reinterpret_cast<float*>(B_s + 2 * 2 * B_TILE);      // [GMAX][NPOL][2][TS]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sacc + GMAX * NPOL * 2 * TS);
    uint64_t* a_full = bars + 0;
    uint64_t* a_empty = bars + 1;
    uint64_t* b_full = bars + 2;      // [2]
    uint64_t* b_empty = bars + 4;     // [2]
    uint64_t* acc_full = bars + 6;
    uint64_t* acc_empty = bars + 7;
    uint64_t* mma_drain = bars + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(a_full, NPROD_WARPS);
        mbar_init(a_empty, 1);
        mbar_init(b_full, 1);
        mbar_init(b_full + 1, 1);
        mbar_init(b_empty, 1);
        mbar_init(b_empty + 1, 1);
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, NPROD_WARPS);
        mbar_init(mma_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int n_tiles = (N + TS - 1) / TS;
    const int n_work = n_tiles * k.n_group;
    bool abort_ = false;

    if (warp == NPROD_WARPS) {
        // ------------------------------------------------ TMA + MMA issuer ----
        if (lane == 0) {
            uint32_t a_full_n = 0, acc_empty_n = 0, b_use[2] = {0, 0}, b_full_n[2] = {0, 0};
            int bstage = 0;
            for (int w = blockIdx.x; w < n_work && !abort_; w += gridDim.x) {
                const int g = w % k.n_group;
                for (int c = 0; c < k.n_class && !abort_; ++c) {
                    const int gc = g * k.n_class + c;
                    const int npad = k.gc_npad[gc];
                    const int nc = k.cls_off[c + 1] - k.cls_off[c];
                    if (npad == 0 || nc == 0) continue;
                    const int nkc = (nc + KCH - 1) / KCH;
                    const uint32_t idesc = idesc_bf16(npad);
                    const uint32_t tile_bytes = (uint32_t)npad * 128;
                    for (int kc = 0; kc < nkc && !abort_; ++kc) {
                        const int s = bstage;
                        // S tiles of this chunk -> B stage s
                        if (!mbar_wait(b_empty + s, (b_use[s] & 1) ^ 1, k.err, ERR_TIMEOUT_B_EMPTY)) { abort_ = true; break; }
                        ++b_use[s];
                        const uint8_t* src = k.B + k.gc_boff[gc] + (int64_t)kc * nsplit * tile_bytes;
                        mbar_expect_tx(b_full + s, tile_bytes * nsplit);
                        bulk_g2s(B_s + (s * 2 + 0) * B_TILE, src, tile_bytes, b_full + s);
                        if (k.x3) bulk_g2s(B_s + (s * 2 + 1) * B_TILE, src + tile_bytes, tile_bytes, b_full + s);
                        // pair products of this chunk
                        if (!mbar_wait(a_full, a_full_n & 1, k.err, ERR_TIMEOUT_A_FULL)) { abort_ = true; break; }
                        ++a_full_n;
                        if (kc == 0) {
                            if (!mbar_wait(acc_empty, (acc_empty_n & 1) ^ 1, k.err, ERR_TIMEOUT_ACC_EMPTY)) { abort_ = true; break; }
                            ++acc_empty_n;
                        }
                        if (!mbar_wait(b_full + s, b_full_n[s] & 1, k.err, ERR_TIMEOUT_B_FULL)) { abort_ = true; break; }
                        ++b_full_n[s];
                        tc_fence_after();
                        const uint32_t b_hi = smem_u32(B_s + (s * 2 + 0) * B_TILE);
                        const uint32_t b_lo = smem_u32(B_s + (s * 2 + 1) * B_TILE);
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            const uint32_t d = tmem + (uint32_t)(r * NMAX);
                            const uint32_t a_hi = smem_u32(A_s + (r * 2 + 0) * A_TILE);
                            const uint32_t a_lo = smem_u32(A_s + (r * 2 + 1) * A_TILE);
#pragma unroll
                            for (int ks = 0; ks < KCH / 16; ++ks) {
                                const uint32_t off = ks * 32;
                                mma_bf16(d, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                                if (k.x3) {
                                    mma_bf16(d, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
                                    mma_bf16(d, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
                                }
                            }
                        }
                        mma_commit(a_empty);
                        mma_commit(b_empty + s);
                        if (kc == nkc - 1) mma_commit(acc_full);
                        bstage ^= 1;
                    }
                }
            }
            // drain: wait (bounded) for the MMAs and copies still in flight before leaving
            mma_commit(mma_drain);
            mbar_wait(mma_drain, 0, k.err, ERR_TIMEOUT_DRAIN);
            for (int s = 0; s < 2; ++s)
                if (b_use[s] > b_full_n[s]) mbar_wait(b_full + s, b_full_n[s] & 1, k.err, ERR_TIMEOUT_DRAIN);
        }
    } else {
        // --------------------------------------- producers and epilogue -------
        const int srow = (warp & 3) * 32 + lane;   // sample row = TMEM lane
        const int half = warp >> 2;
        uint32_t a_empty_n = 0, acc_full_n = 0;
        for (int w = blockIdx.x; w < n_work && !abort_; w += gridDim.x) {
            const int tile = w / k.n_group, g = w % k.n_group;
            const int t = tile * TS + srow;
            const bool tvalid = t < N;
            const int gbeg = k.grp_off[g], gsize = k.grp_off[g + 1] - gbeg;
            // clear this thread's accumulators (its sample, its polarisation)
            if (half < NPOL)
                for (int pi = 0; pi < gsize; ++pi) {
                    sacc[((pi * NPOL + half) * 2 + 0) * TS + srow] = 0.f;
                    sacc[((pi * NPOL + half) * 2 + 1) * TS + srow] = 0.f;
                }
            for (int c = 0; c < k.n_class && !abort_; ++c) {
                const int gc = g * k.n_class + c;
                const int npad = k.gc_npad[gc];
                const int pbeg = k.cls_off[c], nc = k.cls_off[c + 1] - pbeg;
                if (npad == 0 || nc == 0) continue;
                const int nkc = (nc + KCH - 1) / KCH;
                for (int kc = 0; kc < nkc && !abort_; ++kc) {
                    if (!warp_wait(a_empty, (a_empty_n & 1) ^ 1, k.err, ERR_TIMEOUT_A_EMPTY)) { abort_ = true; break; }
                    ++a_empty_n;
                    // pairs kc*64 + 32*half + [0, 32) for sample srow
#pragma unroll 1
                    for (int q8 = 0; q8 < 4; ++q8) {
                        float hv[ROWS][8], lv[ROWS][8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int pidx = kc * KCH + half * 32 + q8 * 8 + q;
                            float u = 0.f, vr = 0.f, vi = 0.f;
                            if (pidx < nc && tvalid) {
                                const int2 ij = __ldg(k.pair_ij + pbeg + pidx);
                                const float cij = __ldg(k.pair_c + pbeg + pidx);
#pragma unroll
                                for (int a = 0; a < NPOL; ++a) {
                                    const cf ai = __ldg(x + (size_t)(ij.x * NPOL + a) * N + t);
                                    const cf aj = __ldg(x + (size_t)(ij.y * NPOL + a) * N + t);
                                    if (NPOL == 2) u = fmaf(ai.x, aj.x, fmaf(ai.y, aj.y, u));
                                    vr = fmaf(ai.x, aj.x, fmaf(-ai.y, aj.y, vr));
                                    vi = fmaf(ai.x, aj.y, fmaf(ai.y, aj.x, vi));
                                }
                                u *= cij; vr *= cij; vi *= cij;
                            }
                            const float vals[3] = {u, vr, vi};
#pragma unroll
                            for (int r = 0; r < ROWS; ++r) {
                                const float v = vals[r + (NPOL == 2 ? 0 : 1)];
                                const float h = bf16_round(v);
                                hv[r][q] = v;
                                lv[r][q] = v - h;
                            }
                        }
                        const int chunk = half * 4 + q8;
                        const uint32_t off = (uint32_t)((srow >> 3) * 1024 + (srow & 7) * 128 + ((chunk ^ (srow & 7)) << 4));
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            uint4 hi;
                            hi.x = pack_bf16(hv[r][0], hv[r][1]);
                            hi.y = pack_bf16(hv[r][2], hv[r][3]);
                            hi.z = pack_bf16(hv[r][4], hv[r][5]);
                            hi.w = pack_bf16(hv[r][6], hv[r][7]);
                            *reinterpret_cast<uint4*>(A_s + (r * 2 + 0) * A_TILE + off) = hi;
                            if (k.x3) {
                                uint4 lo;
                                lo.x = pack_bf16(lv[r][0], lv[r][1]);
                                lo.y = pack_bf16(lv[r][2], lv[r][3]);
                                lo.z = pack_bf16(lv[r][4], lv[r][5]);
                                lo.w = pack_bf16(lv[r][6], lv[r][7]);
                                *reinterpret_cast<uint4*>(A_s + (r * 2 + 1) * A_TILE + off) = lo;
                            }
                        }
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(a_full);
                }
                if (abort_) break;
                // epilogue of this class: contract the accumulators with A_l(t)
                if (!warp_wait(acc_full, acc_full_n & 1, k.err, ERR_TIMEOUT_ACC_FULL)) { abort_ = true; break; }
                ++acc_full_n;
                tc_fence_after();
                const int* meta = k.col_meta + k.gc_coff[gc];
                const int ncol = k.gc_ncol[gc];
                const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
                for (int n0 = 0; n0 < npad; n0 += 16) {
                    uint32_t dr[ROWS][16];
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) tmem_ld16(lane_base + (uint32_t)(r * NMAX + n0), dr[r]);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) tmem_wait16(dr[r]);
                    float dv[ROWS][16];
#pragma unroll
                    for (int r = 0; r < ROWS; ++r)
#pragma unroll
                        for (int j = 0; j < 16; ++j) dv[r][j] = __uint_as_float(dr[r][j]);
                    if (half < NPOL && tvalid) {
                        int lprev = -1;
                        cf Al = make_float2(0.f, 0.f);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int n = n0 + j;
                            if (n >= ncol) break;
                            const int m = __ldg(meta + n);
                            const int pi = m >> 16, l = m & 0xFFFF;
                            if (l != lprev) {
                                Al = __ldg(x + (size_t)(l * NPOL + half) * N + t);
                                lprev = l;
                            }
                            const float W = NPOL == 2 ? 2.f * dv[0][j] : 0.f;
                            const float Zr = dv[ROWS - 2][j], Zi = dv[ROWS - 1][j];
                            float* accp = sacc + ((pi * NPOL + half) * 2) * TS + srow;
                            accp[0] += fmaf(W, Al.x, fmaf(Zr, Al.x, Zi * Al.y));
                            accp[TS] += fmaf(W, Al.y, fmaf(Zi, Al.x, -Zr * Al.y));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
            }
            if (abort_) break;
            if (half < NPOL && tvalid) {
                const float sc = NPOL == 2 ? scale / 3.f : scale;
                for (int pi = 0; pi < gsize; ++pi) {
                    const int p = k.grp_modes[gbeg + pi];
                    const float kr = sacc[((pi * NPOL + half) * 2 + 0) * TS + srow];
                    const float ki = sacc[((pi * NPOL + half) * 2 + 1) * TS + srow];
                    out[(size_t)(p * NPOL + half) * N + t] = make_float2(-sc * ki, sc * kr);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

size_t kerr_tc_smem_bytes(int n_pol) {
    const int rows = n_pol == 2 ? 3 : 2;
    return 1024 + (size_t)rows * 2 * A_TILE + 2 * 2 * B_TILE + (size_t)GMAX * n_pol * 2 * TS * 4 + 9 * 8 + 16;
}

cudaError_t kerr_tc_launch(const KerrTC& k, const float2* x, float2* out, float scale, int N, int n_sm, cudaStream_t s) {
    const size_t smem = kerr_tc_smem_bytes(k.n_pol);
    const int n_work = ((N + TS - 1) / TS) * k.n_group;
    const int grid = n_work < n_sm ? n_work : n_sm;
    if (k.n_pol == 2) {
        cudaError_t e = cudaFuncSetAttribute(kerr_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kerr_tc_kernel<2><<<grid, NTHREADS, smem, s>>>(k, x, out, scale, N);
    } else {
        cudaError_t e = cudaFuncSetAttribute(kerr_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kerr_tc_kernel<1><<<grid, NTHREADS, smem, s>>>(k, x, out, scale, N);
    }
    return cudaGetLastError();
}

// x = in0 + c * in1 (stage input of the Runge-Kutta step)
__global__ void axpy_kernel(const cf* __restrict__ a, const cf* __restrict__ b, float c, cf* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const cf u = a[i], v = b[i];
        y[i] = make_float2(fmaf(c, v.x, u.x), fmaf(c, v.y, u.y));
    }
}

cudaError_t axpy_launch(const float2* a, const float2* b, float c, float2* y, size_t n, cudaStream_t s) {
    axpy_kernel<<<152 * 8, 256, 0, s>>>(a, b, c, y, n);
    return cudaGetLastError();
}

}  // namespace mmf
