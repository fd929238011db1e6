// Kerr term of Eq. 1 in the form the paper prints, on the 5th-generation tensor cores:
//   out_f(t) = i * scale * phi_f(t) * x_f(t),   phi_f(t) = sum_g kappa_fg q_g(t),  q_g = |x_g|^2,
// x = in0 + c1 * in1 (the Runge-Kutta stage input, formed on load).
//
// phi = Q kappa^T is a real GEMM per tile of QM = 128 samples:
//   rows (M)    the tile's samples, one TMEM lane each;
//   K           the field rows g, in chunks of 32 (one 64-byte row of BF16, swizzled);
//   columns (N) the output rows f, all of them in one MMA (N = P rounded up to 16, <= 256);
//   A[t][g]     q_g(t), formed by the formation warps straight from the fields in HBM;
//   B[f][g]     kappa_fg, stored on the device already in the canonical K-major 64-byte
//               swizzled layout, one bulk copy per chunk (the same for every tile, so it comes
//               from L2).
// Both operands are split x = hi + lo in BF16 and the MMAs accumulate hi*hi + hi*lo + lo*hi in
// FP32 (BF16x3).  Every product q_g kappa_fg is non-negative, so the sum has no cancellation.
// Two accumulators of N columns let the epilogue of one tile overlap the MMAs of the next.
//
// Warp roles (one CTA per SM, persistent over sample tiles):
//   warp 0      bulk copies of the kappa chunks into the stage ring; allocates TMEM;
//   warp 1      MMA issue (one elected lane) and commits;
//   QNF warps   formation: thread (sample s, half h) loads x_g(t) for 16 rows g of a chunk,
//               forms q, splits it and stores two 16-byte atoms of each split;
//   QNE warps   epilogue: two warps per TMEM lane quarter (lane = sample), each taking every
//               other group of 16 columns f: phi from TMEM, x reloaded (the tile is still in
//               L2), out_f(t) written; lanes are consecutive samples, so every access is coalesced.
// Every wait is bounded (one second); on timeout the kernel records a code in k.err, winds down,
// waits for its copies and MMAs in flight and releases TMEM.
#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mmf {
namespace {

using namespace tc;

constexpr int QM = 128;                    // samples per tile (MMA M, TMEM lanes)
constexpr int QKC = 32;                    // rows g per K chunk
constexpr int QROWB = 64;                  // bytes per swizzled row of a chunk
constexpr int QKSTEPS = QROWB / 32;        // MMA k-steps per chunk
constexpr int QNS = 4;                     // stages of the ring
constexpr int QNF = 8;                     // formation warps: two per sample
constexpr int QNE = 8;                     // epilogue warps: two per TMEM lane quarter
constexpr int QNTH = (2 + QNF + QNE) * 32;
constexpr int Q_ASPLIT = QM * QROWB;       // one split of an A stage (8 KB)
constexpr int Q_ACC = 256;                 // TMEM columns per accumulator

enum : int { QERR_FULL = 31, QERR_DONE, QERR_ACC_FULL, QERR_ACC_EMPTY, QERR_DRAIN };

struct QLayout {
    size_t a, b, bars, total;
};
__host__ __device__ inline QLayout q_layout(int NP) {
    QLayout L;
    L.a = 0;
    L.b = L.a + (size_t)QNS * 2 * Q_ASPLIT;
    L.bars = L.b + (size_t)QNS * 2 * NP * QROWB;
    L.total = L.bars + 16 * 8;
    return L;
}

__global__ void __launch_bounds__(QNTH, 1)
    kerr_kappa_tc_kernel(KappaTC k, const cf* __restrict__ in0, const cf* __restrict__ in1, float c1,
                         cf* __restrict__ out, float scale, int N) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int P = k.P, NP = k.NP, NKC = k.nkc;
    const QLayout L = q_layout(NP);
    uint8_t* A_s = base + L.a;   // [QNS][hi, lo][QM rows x 64 B]
    uint8_t* B_s = base + L.b;   // [QNS][hi, lo][NP rows x 64 B]
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bars);
    uint64_t* full = bars + 0;        // [QNS] chunk's q formed (QNF warps) and kappa copied (tx)
    uint64_t* done = bars + 4;        // [QNS] chunk's MMAs complete: the stage is free
    uint64_t* acc_full = bars + 8;    // [2]
    uint64_t* acc_empty = bars + 10;  // [2]
    uint64_t* drain = bars + 12;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 14);
    const uint32_t bsplit = (uint32_t)NP * QROWB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (N + QM - 1) / QM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < QNS; ++s) {
            mbar_init(full + s, QNF + 1);
            mbar_init(done + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, QNE);
        }
        mbar_init(drain, 1);
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

    if (warp == 0) {
        // ------------------------------------------------ kappa chunk copies ------
        if (lane == 0) {
            uint32_t j = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                for (int kc = 0; kc < NKC; ++kc, ++j) {
                    const uint32_t s = j % QNS;
                    if (j >= (uint32_t)QNS && !mbar_wait(done + s, ((j / QNS) - 1) & 1, k.err, QERR_DONE)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full + s, 2 * bsplit);
                    bulk_g2s(B_s + (size_t)s * 2 * bsplit, k.B + (size_t)kc * 2 * bsplit, 2 * bsplit, full + s);
                }
            }
            // copies still in flight land before the CTA exits
            for (uint32_t q = j > (uint32_t)QNS ? j - QNS : 0u; q < j; ++q)
                mbar_wait(full + q % QNS, (q / QNS) & 1, k.err, QERR_DRAIN);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issue --------
        const uint32_t idesc = idesc_bf16(NP);
        const uint64_t dA0 = sw_desc<QROWB>(smem_u32(A_s)), dB0 = sw_desc<QROWB>(smem_u32(B_s));
        constexpr uint32_t A_STEP = (2 * Q_ASPLIT) >> 4, A_LO = Q_ASPLIT >> 4;
        const uint32_t B_STEP = (2 * bsplit) >> 4, B_LO = bsplit >> 4;
        uint32_t j = 0, e = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++e) {
            const uint32_t buf = e & 1;
            if (!warp_wait_u(acc_empty + buf, ((e >> 1) & 1) ^ 1, k.err, QERR_ACC_EMPTY)) break;
            tc_fence_after();
            const uint32_t d = tmem + buf * Q_ACC;
            for (int kc = 0; kc < NKC; ++kc, ++j) {
                const uint32_t s = j % QNS;
                if (!warp_wait_u(full + s, (j / QNS) & 1, k.err, QERR_FULL)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ah = dA0 + s * A_STEP, bh = dB0 + s * B_STEP;
                if (elect_one()) {
#pragma unroll
                    for (int ks = 0; ks < QKSTEPS; ++ks) {
                        const uint32_t o = ks * 2;   // 32 bytes further along K
                        mma_bf16(d, ah + o, bh + o, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                        mma_bf16(d, ah + o, bh + B_LO + o, idesc, 1u);
                        mma_bf16(d, ah + A_LO + o, bh + o, idesc, 1u);
                    }
                    mma_commit(done + s);
                    if (kc == NKC - 1) mma_commit(acc_full + buf);
                }
                __syncwarp();
            }
        }
        // the MMAs in flight complete before TMEM is released
        if (j > 0) {
            if (elect_one()) mma_commit(drain);
            __syncwarp();
            warp_wait_u(drain, 0, k.err, QERR_DRAIN);
        }
    } else if (warp < 2 + QNF) {
        // ------------------------------------------------------- formation --------
        const int ft = threadIdx.x - 64;
        const int r = ft % QM, h = ft / QM;   // sample row of the tile, half of the chunk's rows g
        const uint32_t sw = (uint32_t)((r & 7) >> 1);
        const uint32_t row_off = (uint32_t)((r >> 3) * 8 * QROWB + (r & 7) * QROWB);
        const uint32_t at0 = row_off + ((((uint32_t)(2 * h)) ^ sw) << 4), at1 = row_off + ((((uint32_t)(2 * h + 1)) ^ sw) << 4);
        uint32_t j = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            const int t = tile * QM + r;
            const bool tv = t < N;
            for (int kc = 0; kc < NKC; ++kc, ++j) {
                const int g0 = kc * QKC + 16 * h;
                float q[16];
                // loads first: their latency runs while the stage's previous chunk is consumed
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int g = g0 + i;
                    cf x = make_float2(0.f, 0.f);
                    if (tv && g < P) {
                        x = in0[(size_t)g * N + t];
                        if (in1) {
                            const cf y = in1[(size_t)g * N + t];
                            x = __ffma2_rn(make_float2(c1, c1), y, x);
                        }
                    }
                    q[i] = fmaf(x.x, x.x, x.y * x.y);
                }
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) split_bf16(q[2 * i], q[2 * i + 1], hi[i], lo[i]);
                const uint32_t s = j % QNS;
                if (j >= (uint32_t)QNS && !warp_wait(done + s, ((j / QNS) - 1) & 1, k.err, QERR_DONE)) {
                    ok = false;
                    break;
                }
                uint8_t* As = A_s + (size_t)s * 2 * Q_ASPLIT;
                *reinterpret_cast<uint4*>(As + at0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(As + at1) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                *reinterpret_cast<uint4*>(As + Q_ASPLIT + at0) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<uint4*>(As + Q_ASPLIT + at1) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full + s);
            }
        }
    } else {
        // -------------------------------------------------------- epilogue --------
        const int ew = warp - 2 - QNF;            // 0 .. QNE-1
        const int qw = warp & 3, half = ew >> 2;  // TMEM lane quarter (warp % 4), column half
        const int r = 32 * qw + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * qw) << 16);
        const int ngrp = (P + 15) / 16;
        uint32_t e = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++e) {
            const uint32_t buf = e & 1;
            if (!warp_wait(acc_full + buf, (e >> 1) & 1, k.err, QERR_ACC_FULL)) break;
            tc_fence_after();
            const int t = tile * QM + r;
            const bool tv = t < N;
            for (int grp = half; grp < ngrp; grp += 2) {
                const int f0 = grp * 16;
                uint32_t v[16];
                tmem_ld16(lane_base + buf * Q_ACC + (uint32_t)f0, v);
                cf x[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int f = f0 + i;
                    x[i] = make_float2(0.f, 0.f);
                    if (tv && f < P) {
                        x[i] = in0[(size_t)f * N + t];
                        if (in1) x[i] = __ffma2_rn(make_float2(c1, c1), in1[(size_t)f * N + t], x[i]);
                    }
                }
                tmem_wait16(v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int f = f0 + i;
                    if (tv && f < P) {
                        const float a = scale * __uint_as_float(v[i]);
                        out[(size_t)f * N + t] = make_float2(-a * x[i].y, a * x[i].x);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + buf);
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

size_t kerr_kappa_tc_smem_bytes(int NP) { return 1024 + q_layout(NP).total; }

cudaError_t kerr_kappa_tc_launch(const KappaTC& k, const float2* in0, const float2* in1, float c1, float2* out,
                                 float scale, int N, int n_sm, cudaStream_t s) {
    if (k.P < 1 || k.NP < 16 || k.NP > 256 || (k.NP & 15) != 0 || k.NP < k.P || k.nkc != (k.P + QKC - 1) / QKC)
        return cudaErrorInvalidValue;
    const size_t smem = kerr_kappa_tc_smem_bytes(k.NP);
    cudaError_t e = cudaFuncSetAttribute(kerr_kappa_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int n_tiles = (N + QM - 1) / QM;
    const int grid = n_tiles < n_sm ? n_tiles : (n_sm > 0 ? n_sm : 1);
    kerr_kappa_tc_kernel<<<grid, QNTH, smem, s>>>(k, in0, in1, c1, out, scale, N);
    return cudaGetLastError();
}

}  // namespace mmf
