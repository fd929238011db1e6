// Kerr term of Eq. 1 as a pair contraction (FP32, CUDA cores).
//
// For a fully symmetric real overlap tensor S and the isotropic two-polarisation
// tensor, the sum over (l b)(m c)(n d) of Sfull A A conj(A) factors through pair
// quantities of the spatial modes (i <= j, c_ij = 2 off the diagonal, 1 on it):
//   u_ij = c_ij Re sum_a A_ia conj(A_ja),   v_ij = c_ij sum_a A_ia A_ja,
//   W_pl = sum_(ij) S_plij u_ij,            Z_pl = sum_(ij) S_plij v_ij,
//   K_(p,a) = (i gamma h / 3) [ 2 sum_l W_pl A_la + sum_l Z_pl conj(A_la) ],
// and for one polarisation K_p = i gamma h sum_l Z_pl conj(A_l).  S_pair[(pl),(ij)] = S_plij
// is block diagonal over the parity classes of the pairs (class(i,j) = par(i) ^ par(j)).
//
// Per CTA: TS time samples.  The fields of the tile are staged in shared memory
// (the Runge-Kutta stage input x = in0 + c*in1 is formed on the way in).  For each
// class and each tile of NO output pairs the CTA runs a register-blocked GEMM
//   Y[row][s][o] = sum_k X[row][s][k] S_pair[o][k]     (rows: u, Re v, Im v)
// over K chunks of KC input pairs whose X values are formed in shared memory from
// the staged fields; the epilogue contracts Y with A (or conj A) into a shared
// accumulator K[f][s] (shared-memory atomics), written once at the end.
#include "common.cuh"
#include "kernels.h"

namespace mmf {
namespace {

constexpr int NO = 64;     // output pairs per tile
constexpr int KC = 32;     // input pairs per K chunk
constexpr int NTH = 256;

template <int TS, int NPOL>
__global__ void __launch_bounds__(NTH) kerr_pairs_simt_kernel(KerrPairs k, KerrIO io, float scale, int N) {
    constexpr int ROWS = NPOL == 2 ? 3 : 2;
    constexpr int SPT = TS / 16;          // samples per thread (4 or 2)
    extern __shared__ float4 smem_raw[];
    const int P = k.M * NPOL;
    cf* sA = reinterpret_cast<cf*>(smem_raw);                  // [P][TS]
    cf* sK = sA + (size_t)P * TS;                              // [P][TS]
    float* Xs = reinterpret_cast<float*>(sK + (size_t)P * TS); // [ROWS][KC][TS]
    float* Ss = Xs + ROWS * KC * TS;                           // [KC][NO]
    const int tid = threadIdx.x;
    const int t0 = blockIdx.x * TS;
    if (!tile_live(io.slot_steps, io.slot_len, t0, TS, N)) return;

    for (int e = tid; e < P * TS; e += NTH) {
        const int f = e / TS, s = e % TS, t = t0 + s;
        cf x = make_float2(0.f, 0.f);
        if (t < N) {
            const size_t g = (size_t)f * N + t;
            x = io.in0[g];
            if (io.in1) {
                const cf y = io.in1[g];
                x.x = fmaf(io.in1_coef, y.x, x.x);
                x.y = fmaf(io.in1_coef, y.y, x.y);
            }
        }
        sA[e] = x;
        sK[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();

    // thread tile: samples sg*SPT .. +SPT, outputs og*4 .. +4
    const int warp = tid >> 5, lane = tid & 31;
    const int sg = (warp & 1) * 8 + (lane & 7);
    const int og = (warp >> 1) * 4 + (lane >> 3);

    for (int c = 0; c < k.n_class; ++c) {
        const int pbeg = k.cls_off[c], nc = k.cls_off[c + 1] - pbeg;
        if (nc == 0) continue;
        const float* Sc = k.S_pair + k.S_off[c];
        for (int ot = 0; ot < nc; ot += NO) {
            float acc[ROWS][SPT][4];
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
#pragma unroll
                for (int i = 0; i < SPT; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[r][i][j] = 0.f;
            for (int kc = 0; kc < nc; kc += KC) {
                // pair products of this chunk: X[row][kk][s]
                for (int e = tid; e < KC * TS; e += NTH) {
                    const int kk = e / TS, s = e % TS;
                    float u = 0.f, vr = 0.f, vi = 0.f;
                    if (kc + kk < nc) {
                        const int2 ij = k.pair_ij[pbeg + kc + kk];
                        const float cij = k.pair_c[pbeg + kc + kk];
#pragma unroll
                        for (int a = 0; a < NPOL; ++a) {
                            const cf ai = sA[(ij.x * NPOL + a) * TS + s], aj = sA[(ij.y * NPOL + a) * TS + s];
                            if (NPOL == 2) u = fmaf(ai.x, aj.x, fmaf(ai.y, aj.y, u));
                            vr = fmaf(ai.x, aj.x, fmaf(-ai.y, aj.y, vr));
                            vi = fmaf(ai.x, aj.y, fmaf(ai.y, aj.x, vi));
                        }
                        u *= cij; vr *= cij; vi *= cij;
                    }
                    if (NPOL == 2) {
                        Xs[(0 * KC + kk) * TS + s] = u;
                        Xs[(1 * KC + kk) * TS + s] = vr;
                        Xs[(2 * KC + kk) * TS + s] = vi;
                    } else {
                        Xs[(0 * KC + kk) * TS + s] = vr;
                        Xs[(1 * KC + kk) * TS + s] = vi;
                    }
                }
                // S chunk (S_pair is symmetric: row kc+kk, columns ot..ot+NO)
                for (int e = tid; e < KC * NO; e += NTH) {
                    const int kk = e / NO, o = e % NO;
                    float v = 0.f;
                    if (kc + kk < nc && ot + o < nc) v = __ldg(Sc + (size_t)(kc + kk) * nc + ot + o);
                    Ss[kk * NO + o] = v;
                }
                __syncthreads();
#pragma unroll 4
                for (int kk = 0; kk < KC; ++kk) {
                    const float4 sv = *reinterpret_cast<const float4*>(Ss + kk * NO + og * 4);
                    const float s4[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        float xv[SPT];
                        if constexpr (SPT == 4) {
                            const float4 x4 = *reinterpret_cast<const float4*>(Xs + (r * KC + kk) * TS + sg * 4);
                            xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
                        } else {
                            const float2 x2 = *reinterpret_cast<const float2*>(Xs + (r * KC + kk) * TS + sg * 2);
                            xv[0] = x2.x; xv[1] = x2.y;
                        }
#pragma unroll
                        for (int i = 0; i < SPT; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) acc[r][i][j] = fmaf(xv[i], s4[j], acc[r][i][j]);
                    }
                }
                __syncthreads();
            }
            // epilogue: contract with A into K
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = ot + og * 4 + j;
                if (o >= nc) continue;
                const int2 pl = k.pair_ij[pbeg + o];
#pragma unroll
                for (int i = 0; i < SPT; ++i) {
                    const int s = sg * SPT + i;
                    const float W = NPOL == 2 ? 2.f * acc[0][i][j] : 0.f;
                    const float Zr = acc[ROWS - 2][i][j], Zi = acc[ROWS - 1][i][j];
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        if (side == 1 && pl.x == pl.y) break;
                        const int dst = side == 0 ? pl.x : pl.y, src = side == 0 ? pl.y : pl.x;
#pragma unroll
                        for (int a = 0; a < NPOL; ++a) {
                            const cf A = sA[(src * NPOL + a) * TS + s];
                            // W A + Z conj(A)
                            const float re = fmaf(W, A.x, fmaf(Zr, A.x, Zi * A.y));
                            const float im = fmaf(W, A.y, fmaf(Zi, A.x, -Zr * A.y));
                            cf* d = sK + (dst * NPOL + a) * TS + s;
                            atomicAdd(&d->x, re);
                            atomicAdd(&d->y, im);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const float sc = NPOL == 2 ? scale / 3.f : scale;
    for (int e = tid; e < P * TS; e += NTH) {
        const int f = e / TS, s = e % TS, t = t0 + s;
        if (t < N) {
            const cf v = sK[e];
            io.out[(size_t)f * N + t] = make_float2(-sc * v.y, sc * v.x);   // i * scale * K
        }
    }
}

template <int TS, int NPOL>
cudaError_t launch_pairs(const KerrPairs& k, const KerrIO& io, float scale, int N, cudaStream_t s) {
    constexpr int ROWS = NPOL == 2 ? 3 : 2;
    const int P = k.M * NPOL;
    const size_t smem = (size_t)2 * P * TS * sizeof(cf) + (size_t)ROWS * KC * TS * 4 + (size_t)KC * NO * 4;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kerr_pairs_simt_kernel<TS, NPOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kerr_pairs_simt_kernel<TS, NPOL><<<(N + TS - 1) / TS, NTH, smem, s>>>(k, io, scale, N);
    return cudaGetLastError();
}

}  // namespace

cudaError_t kerr_pairs_simt_launch(const KerrPairs& k, const KerrIO& io, float scale, int N, cudaStream_t s) {
    const int P = k.M * k.n_pol;
    // 64 samples per CTA while the staged fields and accumulator fit, else 32
    const bool wide = (size_t)2 * P * 64 * sizeof(cf) + 3 * KC * 64 * 4 + KC * NO * 4 <= 200 * 1024;
    if (k.n_pol == 2) return wide ? launch_pairs<64, 2>(k, io, scale, N, s) : launch_pairs<32, 2>(k, io, scale, N, s);
    return wide ? launch_pairs<64, 1>(k, io, scale, N, s) : launch_pairs<32, 1>(k, io, scale, N, s);
}

}  // namespace mmf
