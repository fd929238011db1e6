// Kerr term of Eq. 1 as a pair contraction on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands in shared memory, S tiles by TMA).
//
// Same factorisation as the CUDA-core path (kerr_pairs.cu):
//   u_ij = c_ij Re sum_a A_ia conj(A_ja),  v_ij = c_ij sum_a A_ia A_ja      (pairs i <= j)
//   W_pl = sum_(ij) S_plij u_ij,           Z_pl = sum_(ij) S_plij v_ij
//   K_(p,a) = (i gamma h / 3)[2 sum_l W_pl A_la + sum_l Z_pl conj(A_la)]   (2 pol; 1 pol: Z term only)
// evaluated per tile of 128 time samples as GEMMs D[s][n] = sum_k X[s][k] B[n][k]:
//   rows s      = the 128 samples of the tile (MMA M; one TMEM lane each),
//   K           = the input pairs (ij) of one parity class, KCH = SW/2 per chunk,
//   columns n   = output pairs (p, l) of that class, p in a group of modes, l running over
//                 the modes whose parity completes the class, l-major (N <= 160),
//   X rows      = u, Re v, Im v (two polarisations) or Re v, Im v (one): one accumulator each,
//   B[n][k]     = S_plij, stored on the device already in the canonical K-major swizzled
//                 tile layout (SW-byte rows), so one bulk TMA copy moves a tile.
// BF16X3 splits both operands x = hi + lo in BF16 and accumulates hi*hi + hi*lo + lo*hi in
// FP32; BF16 uses hi*hi only.
//
// Warp roles (288 threads, one CTA per SM, persistent over (sample tile, mode group)):
//   warps 0-7  producers: stage the tile's fields in shared memory (when they fit), form
//              the pair products of each chunk into a double-buffered A stage (thread =
//              sample, warps w and w+4 take different 16-byte chunks of the row), then the
//              epilogue of each class (thread = sample, w < 4 polarisation 0, w >= 4
//              polarisation 1): tcgen05.ld of its TMEM lane and contraction with A_l(t)
//              into per-(p, pol) shared accumulators.  The epilogue of a class is deferred
//              until the first chunk of the next class has been formed, so it overlaps
//              that chunk's MMAs.
//   warp 8     one thread: TMA bulk copies of the S tiles one chunk ahead (double-buffered)
//              and the tcgen05.mma issue, completion committed to mbarriers.
// Every wait (mbarriers, and the producer-wide synchronisation, which is an mbarrier too)
// gives up after one second, records an error code in k.err and lets the kernel wind
// down; in-flight MMAs and copies are drained and TMEM is released.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mmf {
namespace {

using namespace tc;

constexpr int TS = 128;              // samples per tile (MMA M)
constexpr int NMAX = 160;            // max output columns per (group, class)
constexpr int NEPI_WARPS = 4;       // epilogue warps (one per TMEM lane quarter)
constexpr int NFORM_WARPS = 8;      // pair-product formation warps (two per row quarter)
constexpr int FSTRIDE = NFORM_WARPS / 4;   // formation warps sharing one row quarter
constexpr int NTHREADS = (NEPI_WARPS + NFORM_WARPS + 1) * 32;
constexpr int GMAX = KerrTC::GMAX;   // max modes per group
constexpr int NSB = 3;            // S-tile (B operand) stages
constexpr int NBARS = 19;

enum : int { ERR_TIMEOUT_A_EMPTY = 1, ERR_TIMEOUT_A_FULL, ERR_TIMEOUT_B_EMPTY, ERR_TIMEOUT_B_FULL,
             ERR_TIMEOUT_ACC_FULL, ERR_TIMEOUT_ACC_EMPTY, ERR_TIMEOUT_DRAIN, ERR_TIMEOUT_PSYNC };

// The small per-(group, class) tables, copied to shared memory at kernel start (the L1
// left beside the operand stages is too small to keep them, and the serial paths --
// the MMA issuer and the epilogue -- would otherwise wait on L2 for every lookup).
struct Tabs {
    int* cls_off;      // [n_class+1]
    int* npad;         // [G*C]
    int* ncol;         // [G*C]
    int* coff;         // [G*C]
    int64_t* boff;     // [G*C]
    int* grp_off;      // [G+1]
    int* grp_modes;    // [M]
};
__host__ __device__ __forceinline__ size_t tabs_bytes(int M, int G, int C) {
    return (size_t)G * C * 8 + ((size_t)(C + 1) + 3 * (size_t)G * C + (G + 1) + M) * 4 + 16;
}

// Position in the sequence of K chunks a CTA processes: work items w (sample tile, mode
// group), classes c with a nonempty (group, class) block, chunks kc.
struct ChunkIt {
    int w, c, kc, nkc;
    bool valid;
};
__device__ __forceinline__ bool class_active(const KerrTC& k, const Tabs& T, int g, int c, int* nkc, int kch) {
    const int npad = T.npad[g * k.n_class + c];
    const int nc = T.cls_off[c + 1] - T.cls_off[c];
    *nkc = (nc + kch - 1) / kch;
    return npad > 0 && nc > 0;
}
__device__ __forceinline__ void it_first_class(const KerrTC& k, const Tabs& T, ChunkIt& it, int c0, int n_work, int kch) {
    for (; it.w < n_work; it.w += gridDim.x, c0 = 0) {
        const int g = it.w % k.n_group;
        for (int c = c0; c < k.n_class; ++c)
            if (class_active(k, T, g, c, &it.nkc, kch)) {
                it.c = c;
                it.kc = 0;
                it.valid = true;
                return;
            }
    }
    it.valid = false;
}
__device__ __forceinline__ void it_advance(const KerrTC& k, const Tabs& T, ChunkIt& it, int n_work, int kch) {
    if (++it.kc < it.nkc) return;
    it_first_class(k, T, it, it.c + 1, n_work, kch);
}

template <int NPOL, int SW, bool FS, bool X3>
__global__ void __launch_bounds__(NTHREADS, 1) kerr_tc_kernel(KerrTC k, const cf* __restrict__ x, cf* __restrict__ out,
                                                              float scale, int N, int nsa) {
    constexpr int ROWS = NPOL == 2 ? 3 : 2;
    constexpr int KCH = SW / 2;                 // pairs per chunk
    constexpr int NSPLIT = X3 ? 2 : 1;
    constexpr int A_TILE = TS * SW;
    constexpr int B_TILE = NMAX * SW;
    constexpr int SWS = SW == 128 ? 0 : (SW == 64 ? 1 : 2);
    constexpr int CPR = SW / 16;                // 16-byte chunks per tile row (8 pairs each)
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int P = k.M * NPOL;
    const int n_pairs = k.n_pairs;
    uint8_t* A_s = base;                                            // [nsa][ROWS][NSPLIT][A_TILE]
    uint8_t* B_s = A_s + (size_t)nsa * ROWS * NSPLIT * A_TILE;      // [NSB][NSPLIT][B_TILE]
    cf* sF = reinterpret_cast<cf*>(B_s + NSB * NSPLIT * B_TILE);    // [M][TS][NPOL] when FS
    uint16_t* sP = reinterpret_cast<uint16_t*>(FS ? (uint8_t*)(sF + (size_t)P * TS) : (uint8_t*)sF);  // pairs i | j<<8
    const int GC = k.n_group * k.n_class;
    Tabs T;
    T.boff = reinterpret_cast<int64_t*>(((uintptr_t)(sP + n_pairs) + 15) & ~(uintptr_t)15);
    T.cls_off = reinterpret_cast<int*>(T.boff + GC);
    T.npad = T.cls_off + k.n_class + 1;
    T.ncol = T.npad + GC;
    T.coff = T.ncol + GC;
    T.grp_off = T.coff + GC;
    T.grp_modes = T.grp_off + k.n_group + 1;
    int* s_meta = reinterpret_cast<int*>(((uintptr_t)(T.grp_modes + k.M) + 15) & ~(uintptr_t)15);  // [NEPI_WARPS][NMAX]
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_meta + NEPI_WARPS * NMAX);
    uint64_t* a_full = bars + 0;      // [3]
    uint64_t* a_empty = bars + 3;     // [3]
    uint64_t* b_full = bars + 6;      // [NSB <= 4]
    uint64_t* b_empty = bars + 10;    // [NSB <= 4]
    uint64_t* acc_full = bars + 14;
    uint64_t* acc_empty = bars + 15;
    uint64_t* mma_drain = bars + 16;
    uint64_t* f_ready = bars + 17;    // fields of the work item staged
    uint64_t* f_free = bars + 18;     // epilogue of the work item done with the staged fields
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBARS);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 3; ++s) {
            mbar_init(a_full + s, NFORM_WARPS);
            mbar_init(a_empty + s, 1);
        }
        for (int s = 0; s < NSB; ++s) {
            mbar_init(b_full + s, 1);
            mbar_init(b_empty + s, 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, NEPI_WARPS);
        mbar_init(mma_drain, 1);
        mbar_init(f_ready, NFORM_WARPS);
        mbar_init(f_free, NEPI_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = threadIdx.x; q < n_pairs; q += NTHREADS) {
        const int4 pk = __ldg(k.pair_pk + q);
        sP[q] = (uint16_t)(pk.x | (pk.y << 8));
    }
    for (int q = threadIdx.x; q < GC; q += NTHREADS) {
        T.npad[q] = k.gc_npad[q];
        T.ncol[q] = k.gc_ncol[q];
        T.coff[q] = k.gc_coff[q];
        T.boff[q] = k.gc_boff[q];
    }
    for (int q = threadIdx.x; q <= k.n_class; q += NTHREADS) T.cls_off[q] = k.cls_off[q];
    for (int q = threadIdx.x; q <= k.n_group; q += NTHREADS) T.grp_off[q] = k.grp_off[q];
    for (int q = threadIdx.x; q < k.M; q += NTHREADS) T.grp_modes[q] = k.grp_modes[q];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_work = ((N + TS - 1) / TS) * k.n_group;
    // both polarisations of mode m at the tile's sample: staged (FS) or read from HBM/L2
    auto load_mode = [&](int m, int srow_, int tcl, cf* a) {
        if constexpr (FS) {
            if constexpr (NPOL == 2) {
                const float4 v = reinterpret_cast<const float4*>(sF)[m * TS + srow_];
                a[0] = make_float2(v.x, v.y);
                a[1] = make_float2(v.z, v.w);
            } else {
                a[0] = sF[m * TS + srow_];
            }
        } else {
#pragma unroll
            for (int q = 0; q < NPOL; ++q) a[q] = __ldg(x + (size_t)(m * NPOL + q) * N + tcl);
        }
    };

    if (warp == NEPI_WARPS + NFORM_WARPS) {
        // ------------------------------------------------ TMA + MMA issuer ----
        if (lane == 0) {
            bool abort_ = false;
            ChunkIt im = {(int)blockIdx.x, 0, 0, 0, false}, il;
            it_first_class(k, T, im, 0, n_work, KCH);
            il = im;
            uint32_t jl = 0, jm = 0, e = 0;
            // S-tile copy of chunk jl into stage jl % NSB once the MMAs of chunk jl - NSB are done
            auto issue_load = [&](const ChunkIt& it, bool block) -> int {
                const int s = (int)(jl % NSB);
                const uint32_t ph = ((jl / NSB) & 1) ^ 1;
                if (block) {
                    if (!mbar_wait(b_empty + s, ph, k.err, ERR_TIMEOUT_B_EMPTY)) return -1;
                } else if (!mbar_test_wait(b_empty + s, ph)) {
                    return 0;
                }
                const int gc = (it.w % k.n_group) * k.n_class + it.c;
                const uint32_t tile_bytes = (uint32_t)T.npad[gc] * SW;
                const uint8_t* src = k.B + T.boff[gc] + (int64_t)it.kc * NSPLIT * tile_bytes;
                mbar_expect_tx(b_full + s, tile_bytes * NSPLIT);
                bulk_g2s(B_s + (s * NSPLIT + 0) * B_TILE, src, tile_bytes, b_full + s);
                if (X3) bulk_g2s(B_s + (s * NSPLIT + 1) * B_TILE, src + tile_bytes, tile_bytes, b_full + s);
                ++jl;
                return 1;
            };
            while (im.valid && !abort_) {
                // keep up to NSB copies in flight; block only when the chunk to multiply has none
                while (il.valid && jl < jm + NSB) {
                    const int r = issue_load(il, jl == jm);
                    if (r < 0) { abort_ = true; break; }
                    if (r == 0) break;
                    it_advance(k, T, il, n_work, KCH);
                }
                if (abort_) break;
                const int sa = (int)(jm % (uint32_t)nsa), sb = (int)(jm % NSB);
                if (!mbar_wait(a_full + sa, (jm / nsa) & 1, k.err, ERR_TIMEOUT_A_FULL)) { abort_ = true; break; }
                if (im.kc == 0) {
                    if (!mbar_wait(acc_empty, (e & 1) ^ 1, k.err, ERR_TIMEOUT_ACC_EMPTY)) { abort_ = true; break; }
                    ++e;
                }
                if (!mbar_wait(b_full + sb, (jm / NSB) & 1, k.err, ERR_TIMEOUT_B_FULL)) { abort_ = true; break; }
                tc_fence_after();
                const int gc = (im.w % k.n_group) * k.n_class + im.c;
                const uint32_t idesc = idesc_bf16(T.npad[gc]);
                const uint32_t b_hi = smem_u32(B_s + (sb * NSPLIT + 0) * B_TILE);
                const uint32_t b_lo = smem_u32(B_s + (sb * NSPLIT + (NSPLIT - 1)) * B_TILE);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const uint32_t d = tmem + (uint32_t)(r * NMAX);
                    const uint32_t a_hi = smem_u32(A_s + ((size_t)(sa * ROWS + r) * NSPLIT + 0) * A_TILE);
                    const uint32_t a_lo = smem_u32(A_s + ((size_t)(sa * ROWS + r) * NSPLIT + (NSPLIT - 1)) * A_TILE);
#pragma unroll
                    for (int ks = 0; ks < KCH / 16; ++ks) {
                        const uint32_t off = ks * 32;
                        mma_bf16(d, sw_desc<SW>(a_hi + off), sw_desc<SW>(b_hi + off), idesc,
                                 (im.kc > 0 || ks > 0) ? 1u : 0u);
                        if (X3) {
                            mma_bf16(d, sw_desc<SW>(a_hi + off), sw_desc<SW>(b_lo + off), idesc, 1u);
                            mma_bf16(d, sw_desc<SW>(a_lo + off), sw_desc<SW>(b_hi + off), idesc, 1u);
                        }
                    }
                }
                mma_commit(a_empty + sa);
                mma_commit(b_empty + sb);
                if (im.kc == im.nkc - 1) mma_commit(acc_full);
                ++jm;
                it_advance(k, T, im, n_work, KCH);
            }
            // drain: the MMAs and the copies still in flight complete before the CTA exits
            mma_commit(mma_drain);
            mbar_wait(mma_drain, 0, k.err, ERR_TIMEOUT_DRAIN);
            for (uint32_t j = jm; j < jl; ++j) mbar_wait(b_full + (j % NSB), (j / NSB) & 1, k.err, ERR_TIMEOUT_DRAIN);
        }
    } else if (warp >= NEPI_WARPS) {
        // -------------------------------------------------- formation ---------
        const int fw = warp - NEPI_WARPS;
        const int srow = (fw & 3) * 32 + lane;
        const int part = fw >> 2;                  // which 16-byte chunks of the row (stride FSTRIDE)
        uint32_t j = 0, wi = 0;
        bool abort_ = false;
        for (int w = blockIdx.x; w < n_work && !abort_; w += gridDim.x, ++wi) {
            const int tile = w / k.n_group, g = w % k.n_group;
            const int t = tile * TS + srow;
            const bool tvalid = t < N;
            const int tc = tvalid ? t : N - 1;
            if constexpr (FS) {
                if (!warp_wait(f_free, (wi & 1) ^ 1, k.err, ERR_TIMEOUT_PSYNC)) { abort_ = true; break; }
                for (int m = part; m < k.M; m += FSTRIDE) {
                    if constexpr (NPOL == 2) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (tvalid) {
                            const cf a0 = __ldg(x + (size_t)(2 * m) * N + t), a1 = __ldg(x + (size_t)(2 * m + 1) * N + t);
                            v = make_float4(a0.x, a0.y, a1.x, a1.y);
                        }
                        reinterpret_cast<float4*>(sF)[m * TS + srow] = v;
                    } else {
                        sF[m * TS + srow] = tvalid ? __ldg(x + (size_t)m * N + t) : make_float2(0.f, 0.f);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(f_ready);
                if (!warp_wait(f_ready, wi & 1, k.err, ERR_TIMEOUT_PSYNC)) { abort_ = true; break; }
            }
            for (int c = 0; c < k.n_class && !abort_; ++c) {
                int nkc;
                if (!class_active(k, T, g, c, &nkc, KCH)) continue;
                const int pbeg = T.cls_off[c], nc = T.cls_off[c + 1] - pbeg;
                for (int kc = 0; kc < nkc && !abort_; ++kc, ++j) {
                    const int s = (int)(j % (uint32_t)nsa);
                    if (!warp_wait(a_empty + s, ((j / nsa) & 1) ^ 1, k.err, ERR_TIMEOUT_A_EMPTY)) { abort_ = true; break; }
                    uint8_t* As = A_s + (size_t)s * ROWS * NSPLIT * A_TILE;
#pragma unroll 1
                    for (int cidx = part; cidx < CPR; cidx += FSTRIDE) {
                        int pi_[8], pj_[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            // beyond the class the S tile rows are zero; any valid pair will do
                            const int pidx = kc * KCH + cidx * 8 + q;
                            const uint32_t ij = sP[pbeg + (pidx < nc ? pidx : nc - 1)];
                            pi_[q] = ij & 0xFF;
                            pj_[q] = ij >> 8;
                        }
                        // all field loads of the 8 pairs first (independent), then the arithmetic
                        cf ai[8][NPOL], aj[8][NPOL];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            load_mode(pi_[q], srow, tc, ai[q]);
                            load_mode(pj_[q], srow, tc, aj[q]);
                        }
                        float vals[ROWS][8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            float u = 0.f, vr = 0.f, vi = 0.f;
#pragma unroll
                            for (int a = 0; a < NPOL; ++a) {
                                if (NPOL == 2) u = fmaf(ai[q][a].x, aj[q][a].x, fmaf(ai[q][a].y, aj[q][a].y, u));
                                vr = fmaf(ai[q][a].x, aj[q][a].x, fmaf(-ai[q][a].y, aj[q][a].y, vr));
                                vi = fmaf(ai[q][a].x, aj[q][a].y, fmaf(ai[q][a].y, aj[q][a].x, vi));
                            }
                            if constexpr (NPOL == 2) {
                                vals[0][q] = u;
                                vals[1][q] = vr;
                                vals[2][q] = vi;
                            } else {
                                vals[0][q] = vr;
                                vals[1][q] = vi;
                            }
                        }
                        const uint32_t off = (uint32_t)((srow >> 3) * 8 * SW + (srow & 7) * SW +
                                                        ((cidx ^ ((srow & 7) >> SWS)) << 4));
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            uint4 hi, lo;
                            if constexpr (X3) {
                                split_bf16(vals[r][0], vals[r][1], hi.x, lo.x);
                                split_bf16(vals[r][2], vals[r][3], hi.y, lo.y);
                                split_bf16(vals[r][4], vals[r][5], hi.z, lo.z);
                                split_bf16(vals[r][6], vals[r][7], hi.w, lo.w);
                                *reinterpret_cast<uint4*>(As + (r * NSPLIT + 1) * A_TILE + off) = lo;
                            } else {
                                hi.x = pack_bf16(vals[r][0], vals[r][1]);
                                hi.y = pack_bf16(vals[r][2], vals[r][3]);
                                hi.z = pack_bf16(vals[r][4], vals[r][5]);
                                hi.w = pack_bf16(vals[r][6], vals[r][7]);
                            }
                            *reinterpret_cast<uint4*>(As + (r * NSPLIT + 0) * A_TILE + off) = hi;
                        }
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(a_full + s);
                }
            }
        }
    } else {
        // --------------------------------------------------- epilogue ---------
        // One warp per TMEM lane quarter; each thread keeps the group's sums of both
        // polarisations for its sample in registers.
        const int srow = warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        int* meta = s_meta + warp * NMAX;
        uint32_t e = 0, wi = 0;
        bool abort_ = false;
        for (int w = blockIdx.x; w < n_work && !abort_; w += gridDim.x, ++wi) {
            const int tile = w / k.n_group, g = w % k.n_group;
            const int t = tile * TS + srow;
            const bool tvalid = t < N;
            const int tc = tvalid ? t : N - 1;
            const int gbeg = T.grp_off[g], gsize = T.grp_off[g + 1] - gbeg;
            float sum[GMAX][NPOL][2];
#pragma unroll
            for (int q = 0; q < GMAX; ++q)
#pragma unroll
                for (int a = 0; a < NPOL; ++a) sum[q][a][0] = sum[q][a][1] = 0.f;
            if constexpr (FS) {
                if (!warp_wait(f_ready, wi & 1, k.err, ERR_TIMEOUT_PSYNC)) { abort_ = true; break; }
            }
            for (int c = 0; c < k.n_class && !abort_; ++c) {
                int nkc;
                if (!class_active(k, T, g, c, &nkc, KCH)) continue;
                const int gc = g * k.n_class + c;
                const int ncol = T.ncol[gc], npad = T.npad[gc];
                // this warp's copy of the class's column list, fetched while the MMAs finish
                for (int n = lane; n < ncol; n += 32) meta[n] = __ldg(k.col_meta + T.coff[gc] + n);
                __syncwarp();
                if (!warp_wait(acc_full, e & 1, k.err, ERR_TIMEOUT_ACC_FULL)) { abort_ = true; break; }
                ++e;
                tc_fence_after();
                // columns are p-major: accumulate a run of equal p, then add it to that p's sum
                int pcur = -1;
                float run[NPOL][2];
                auto flush = [&]() {
#pragma unroll
                    for (int q = 0; q < GMAX; ++q)
                        if (q == pcur) {
#pragma unroll
                            for (int a = 0; a < NPOL; ++a) {
                                sum[q][a][0] += run[a][0];
                                sum[q][a][1] += run[a][1];
                            }
                        }
                };
                for (int n0 = 0; n0 < npad; n0 += 16) {
                    uint32_t dr[ROWS][16];
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) tmem_ld16(lane_base + (uint32_t)(r * NMAX + n0), dr[r]);
                    int mm[16];
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) mm[jj] = (n0 + jj < ncol) ? meta[n0 + jj] : -1;
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) tmem_wait16(dr[r]);
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) {
                        cf Al[8][NPOL];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int m = mm[h8 * 8 + q];
                            load_mode(m >= 0 ? (m & 0xFFFF) : 0, srow, tc, Al[q]);
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int jj = h8 * 8 + q;
                            const int m = mm[jj];
                            if (m < 0) break;
                            const int pi = m >> 16;
                            if (pi != pcur) {
                                if (pcur >= 0) flush();
                                pcur = pi;
#pragma unroll
                                for (int a = 0; a < NPOL; ++a) run[a][0] = run[a][1] = 0.f;
                            }
                            const float W = NPOL == 2 ? 2.f * __uint_as_float(dr[0][jj]) : 0.f;
                            const float Zr = __uint_as_float(dr[ROWS - 2][jj]), Zi = __uint_as_float(dr[ROWS - 1][jj]);
#pragma unroll
                            for (int a = 0; a < NPOL; ++a) {
                                // 2 W A + Z conj(A)
                                run[a][0] += fmaf(W, Al[q][a].x, fmaf(Zr, Al[q][a].x, Zi * Al[q][a].y));
                                run[a][1] += fmaf(W, Al[q][a].y, fmaf(Zi, Al[q][a].x, -Zr * Al[q][a].y));
                            }
                        }
                    }
                }
                if (pcur >= 0) flush();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
            }
            if (abort_) break;
            if constexpr (FS) {
                __syncwarp();
                if (lane == 0) mbar_arrive(f_free);
            }
            if (tvalid) {
                const float sc = NPOL == 2 ? scale / 3.f : scale;
#pragma unroll
                for (int q = 0; q < GMAX; ++q)
                    if (q < gsize) {
                        const int p = T.grp_modes[gbeg + q];
#pragma unroll
                        for (int a = 0; a < NPOL; ++a)
                            out[(size_t)(p * NPOL + a) * N + t] = make_float2(-sc * sum[q][a][1], sc * sum[q][a][0]);
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

template <int NPOL, int SW, bool FS, bool X3>
cudaError_t launch_tc(const KerrTC& k, const float2* x, float2* out, float scale, int N, int grid, size_t smem,
                      cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kerr_tc_kernel<NPOL, SW, FS, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kerr_tc_kernel<NPOL, SW, FS, X3><<<grid, NTHREADS, smem, s>>>(k, x, out, scale, N, k.a_stages);
    return cudaGetLastError();
}

template <int NPOL, int SW>
cudaError_t launch_tc_fs(const KerrTC& k, const float2* x, float2* out, float scale, int N, int grid, size_t smem,
                         cudaStream_t s) {
    if (k.x3)
        return k.fields_smem ? launch_tc<NPOL, SW, true, true>(k, x, out, scale, N, grid, smem, s)
                             : launch_tc<NPOL, SW, false, true>(k, x, out, scale, N, grid, smem, s);
    return k.fields_smem ? launch_tc<NPOL, SW, true, false>(k, x, out, scale, N, grid, smem, s)
                         : launch_tc<NPOL, SW, false, false>(k, x, out, scale, N, grid, smem, s);
}

}  // namespace

size_t kerr_tc_smem_bytes(int n_pol, int sw, int P, int n_pairs, int a_stages, bool fields_smem, int n_group,
                          int n_class, bool x3) {
    const int rows = n_pol == 2 ? 3 : 2;
    const int M = P / n_pol;
    const int nsplit = x3 ? 2 : 1;
    return 1024 + (size_t)a_stages * rows * nsplit * TS * sw + (size_t)NSB * nsplit * NMAX * sw +
           (fields_smem ? (size_t)P * TS * 8 : 0) + (size_t)n_pairs * 2 + 16 + tabs_bytes(M, n_group, n_class) + 16 +
           (size_t)NEPI_WARPS * NMAX * 4 + NBARS * 8 + 16;
}

cudaError_t kerr_tc_launch(const KerrTC& k, const float2* x, float2* out, float scale, int N, int n_sm, cudaStream_t s) {
    const int P = k.M * k.n_pol;
    const size_t smem = kerr_tc_smem_bytes(k.n_pol, k.sw, P, k.n_pairs, k.a_stages, k.fields_smem != 0, k.n_group, k.n_class,
                                           k.x3 != 0);
    const int n_work = ((N + TS - 1) / TS) * k.n_group;
    const int grid = n_work < n_sm ? n_work : n_sm;
    if (k.sw != 32 && k.sw != 64) return cudaErrorInvalidValue;
    if (k.n_pol == 2)
        return k.sw == 32 ? launch_tc_fs<2, 32>(k, x, out, scale, N, grid, smem, s)
                          : launch_tc_fs<2, 64>(k, x, out, scale, N, grid, smem, s);
    return k.sw == 32 ? launch_tc_fs<1, 32>(k, x, out, scale, N, grid, smem, s)
                      : launch_tc_fs<1, 64>(k, x, out, scale, N, grid, smem, s);
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
