// Kerr term of Eq. 1 in the form the paper prints (self- and cross-phase only, every row a
// spatial or polarisation mode):
//   out_f(t) = i * scale * phi_f(t) * x_f(t),   phi_f(t) = sum_g kappa_fg |x_g(t)|^2,
// x = in0 + c1 * in1 (the Runge-Kutta stage input, formed on load).  kappa is symmetric and
// kept as its packed upper triangle (row f holds kappa_f,f .. kappa_f,P-1), the storage the
// paper describes (Section 4.4): P(P+1)/2 values, 113 KiB in FP32 at P = 240.
//
// Persistent CTAs of 512 threads (16 warps: one CTA per SM, held by its shared memory): each
// stages the packed kappa in shared memory once, then walks sample tiles of TS = 64.  Per
// tile |x|^2 is staged in shared memory, every thread accumulates an 8-row x 4-sample block of
// phi = kappa |x|^2, and writes i * scale * phi * x with x read again (the tile is still in
// L2).  Per kappa column: eight kappa loads, one 16-byte |x|^2 load, four register moves and
// 16 packed FP32 FMAs (fma.rn.f32x2 on row pairs) for 32 multiply-adds.  Work per
// field-sample: 2P flops against 16 bytes of HBM traffic (field in, Kerr term out).
#include "common.cuh"
#include "kernels.h"

namespace mmf {
namespace {

constexpr int KTS = 64;    // samples per tile
constexpr int KNT = 512;   // threads: one 8-row x 4-sample output block each (P <= 256)
constexpr int RB = 8;      // rows per block

// MODE 0: out = i * scale * phi(x) * x,  x = in0 + c1 in1          (Kerr term)
// MODE 1: ph.phi_out = phi(y),            y = in0                    (phase store)
// MODE 2: out = u * exp(i * scale * (ph.phi0 + phi(y)) / 2),  y = in0, u = ph.u   (rotation)
template <int MODE>
__global__ void __launch_bounds__(KNT) kerr_kappa_kernel(KerrKappa k, KerrIO io, KappaPhase ph, float scale, int N) {
    extern __shared__ float4 smem_raw[];
    const int P = k.P;
    const int nU = P * (P + 1) / 2;
    float* sU = reinterpret_cast<float*>(smem_raw);                       // packed upper triangle
    float* sQ = sU + ((nU + 3) & ~3);                                     // [P][KTS] |x|^2
    const int tid = threadIdx.x;
    for (int q = tid; q < nU; q += KNT) sU[q] = __ldg(k.U + q);

    // this thread's block: rows f0 .. f0+7, samples 4 sb .. 4 sb + 3
    const int nfb = (P + RB - 1) / RB;
    const int fb = tid / (KTS / 4), sb = tid % (KTS / 4);
    const bool active = fb < nfb;
    const int f0 = fb * RB;
    const int n_tiles = (N + KTS - 1) / KTS;
    auto rowoff = [P](int r) { return r * P - r * (r - 1) / 2; };   // start of row r in the triangle
    auto load_x = [&](size_t gi) {
        cf x = io.in0[gi];
        if (io.in1) {
            const cf y = io.in1[gi];
            x.x = fmaf(io.in1_coef, y.x, x.x);
            x.y = fmaf(io.in1_coef, y.y, x.y);
        }
        return x;
    };

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int t0 = tile * KTS;
        if (!tile_live(io.slot_steps, io.slot_len, t0, KTS, N)) continue;   // uniform over the CTA
        __syncthreads();   // kappa staged / the previous tile's |x|^2 no longer read
        // |x|^2 of the tile, in batches of SU elements per thread whose loads are all issued
        // before the first is used
        constexpr int SU = 4;
        for (int e0 = tid; e0 < P * KTS; e0 += SU * KNT) {
            float qv[SU];
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int e = e0 + u * KNT;
                const int f = e / KTS, t = t0 + e % KTS;
                qv[u] = 0.f;
                if (e < P * KTS && t < N) {
                    const cf x = load_x((size_t)f * N + t);
                    qv[u] = fmaf(x.x, x.x, x.y * x.y);
                }
            }
#pragma unroll
            for (int u = 0; u < SU; ++u)
                if (e0 + u * KNT < P * KTS) sQ[e0 + u * KNT] = qv[u];
        }
        __syncthreads();
        if (!active) continue;
        // acc[r][j] = (phi of row f0 + 2r, phi of row f0 + 2r + 1) at sample t0 + 4 sb + j
        float2 acc[RB / 2][4];
#pragma unroll
        for (int r = 0; r < RB / 2; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[r][j] = make_float2(0.f, 0.f);
        const float4* Q4 = reinterpret_cast<const float4*>(sQ) + sb;   // row g at Q4[g * KTS/4]
        auto fma_block = [&](const float* kv, int g) {
            const float4 q = Q4[g * (KTS / 4)];
            const float2 qq[4] = {make_float2(q.x, q.x), make_float2(q.y, q.y), make_float2(q.z, q.z),
                                  make_float2(q.w, q.w)};
#pragma unroll
            for (int r = 0; r < RB / 2; ++r) {
                const float2 kk = make_float2(kv[2 * r], kv[2 * r + 1]);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[r][j] = __ffma2_rn(kk, qq[j], acc[r][j]);
            }
        };
        // g < f0: kappa_(f0+i) g = U[rowoff(g) + f0 + i - g], RB consecutive values of row g
        int base = f0;   // rowoff(g) - g + f0 for g = 0
#pragma unroll 4
        for (int g = 0; g < f0; ++g) {
            float kv[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) kv[i] = sU[base + i];
            fma_block(kv, g);
            base += P - g - 1;
        }
        // the diagonal block f0 <= g < f0 + RB (rows beyond P carry zero)
        for (int g = f0; g < f0 + RB && g < P; ++g) {
            float kv[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int f = f0 + i;
                kv[i] = f >= P ? 0.f : (f <= g ? sU[rowoff(f) + g - f] : sU[rowoff(g) + f - g]);
            }
            fma_block(kv, g);
        }
        // g >= f0 + RB: kappa_(f0+i) g = U[rowoff(f0+i) + g - (f0+i)], one value from each row
        {
            int rb[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) rb[i] = f0 + i < P ? rowoff(f0 + i) - (f0 + i) : rowoff(f0) - f0;
#pragma unroll 4
            for (int g = f0 + RB; g < P; ++g) {
                float kv[RB];
#pragma unroll
                for (int i = 0; i < RB; ++i) kv[i] = sU[rb[i] + g];
                fma_block(kv, g);
            }
        }
        // phi of row f0 + i at sample t0 + 4 sb + j
        auto phi = [&](int i, int j) { return (i & 1) ? acc[i >> 1][j].y : acc[i >> 1][j].x; };
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int f = f0 + i;
            if (f >= P) break;
            const int t = t0 + sb * 4;
            const size_t gi = (size_t)f * N + t;
            if constexpr (MODE == 1) {
                float* dst = ph.phi_out + gi;
                if (t + 3 < N) {
                    *reinterpret_cast<float4*>(dst) = make_float4(phi(i, 0), phi(i, 1), phi(i, 2), phi(i, 3));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (t + j < N) dst[j] = phi(i, j);
                }
            } else if constexpr (MODE == 2) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (t + j < N) {
                        float sn, cs;
                        sincosf(0.5f * scale * (ph.phi0[gi + j] + phi(i, j)), &sn, &cs);
                        const cf u = ph.u[gi + j];
                        io.out[gi + j] = make_float2(u.x * cs - u.y * sn, u.x * sn + u.y * cs);
                    }
            } else {
                // out = i * scale * phi * x, x re-read (the tile is still in L2)
                cf* dst = io.out + gi;
                if (t + 3 < N) {
                    cf o[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const cf x = load_x(gi + j);
                        const float a = scale * phi(i, j);
                        o[j] = make_float2(-a * x.y, a * x.x);
                    }
                    reinterpret_cast<float4*>(dst)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                    reinterpret_cast<float4*>(dst)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (t + j < N) {
                            const cf x = load_x(gi + j);
                            const float a = scale * phi(i, j);
                            dst[j] = make_float2(-a * x.y, a * x.x);
                        }
                }
            }
        }
    }
}

// out = u * exp(i * scale * phi0), elementwise (the first estimate of the iterative step)
__global__ void phase_rotate_kernel(const cf* __restrict__ u, const float* __restrict__ phi0, float scale, cf* out,
                                    size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float sn, cs;
        sincosf(scale * phi0[i], &sn, &cs);
        const cf a = u[i];
        out[i] = make_float2(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
    }
}

template <int MODE>
cudaError_t launch_kappa(const KerrKappa& k, const KerrIO& io, const KappaPhase& ph, float scale, int N, int n_sm,
                         cudaStream_t s) {
    if (k.P < 1 || k.P > 256) return cudaErrorInvalidValue;
    const size_t smem = kerr_kappa_smem_bytes(k.P);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kerr_kappa_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kerr_kappa_kernel<MODE>, KNT, smem);
    if (e != cudaSuccess) return e;
    const int n_tiles = (N + KTS - 1) / KTS;
    const int cap = n_sm * (per_sm > 0 ? per_sm : 1);
    kerr_kappa_kernel<MODE><<<n_tiles < cap ? n_tiles : cap, KNT, smem, s>>>(k, io, ph, scale, N);
    return cudaGetLastError();
}

}  // namespace

size_t kerr_kappa_smem_bytes(int P) {
    const size_t nU = (size_t)P * (P + 1) / 2;
    return ((nU + 3) & ~(size_t)3) * 4 + (size_t)P * KTS * 4;
}

cudaError_t kerr_kappa_launch(const KerrKappa& k, const KerrIO& io, float scale, int N, int n_sm, cudaStream_t s) {
    return launch_kappa<0>(k, io, KappaPhase{}, scale, N, n_sm, s);
}

cudaError_t kappa_phi_launch(const KerrKappa& k, const float2* y, float* phi_out, int N, int n_sm, cudaStream_t s) {
    KerrIO io = {};
    io.in0 = y;
    KappaPhase ph = {};
    ph.phi_out = phi_out;
    return launch_kappa<1>(k, io, ph, 0.f, N, n_sm, s);
}

cudaError_t kappa_rotate_launch(const KerrKappa& k, const float2* y, const float2* u, const float* phi0, float scale,
                                float2* out, int N, int n_sm, const int* slot_steps, int slot_len, cudaStream_t s) {
    KerrIO io = {};
    io.in0 = y;
    io.out = out;
    io.slot_steps = slot_steps;
    io.slot_len = slot_len;
    KappaPhase ph = {};
    ph.u = u;
    ph.phi0 = phi0;
    return launch_kappa<2>(k, io, ph, scale, N, n_sm, s);
}

cudaError_t phase_rotate_launch(const float2* u, const float* phi0, float scale, float2* out, size_t n,
                                cudaStream_t s) {
    const size_t blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
    phase_rotate_kernel<<<(unsigned)blocks, 256, 0, s>>>(u, phi0, scale, out, n);
    return cudaGetLastError();
}

}  // namespace mmf
