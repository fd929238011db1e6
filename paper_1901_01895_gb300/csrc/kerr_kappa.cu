// Kerr term of Eq. 1 in the form the paper prints (self- and cross-phase only, every row a
// spatial or polarisation mode):
//   out_f(t) = i * scale * phi_f(t) * x_f(t),   phi_f(t) = sum_g kappa_fg |x_g(t)|^2,
// x = in0 + c1 * in1 (the Runge-Kutta stage input, formed on load).  kappa is symmetric and
// kept as its packed upper triangle (row f holds kappa_f,f .. kappa_f,P-1), the storage the
// paper describes (Section 4.4): P(P+1)/2 values, 113 KiB in FP32 at P = 240.
//
// Persistent CTAs: each stages the packed kappa in shared memory once, then walks sample
// tiles of TS = 32.  Per tile the fields x and |x|^2 are staged in shared memory, every
// thread accumulates a 4-field x 4-sample block of phi = kappa |x|^2 (P multiply-adds per
// output), and writes i * scale * phi * x.  Work per field-sample: 2P flops against 16 bytes
// of HBM traffic (field in, Kerr term out).
#include "common.cuh"
#include "kernels.h"

namespace mmf {
namespace {

constexpr int KTS = 32;    // samples per tile
constexpr int KNT = 512;   // threads: one 4x4 output block each (P <= 256)

__global__ void __launch_bounds__(KNT) kerr_kappa_kernel(KerrKappa k, KerrIO io, float scale, int N) {
    extern __shared__ float4 smem_raw[];
    const int P = k.P;
    const int nU = P * (P + 1) / 2;
    float* sU = reinterpret_cast<float*>(smem_raw);                       // packed upper triangle
    float* sQ = sU + ((nU + 3) & ~3);                                     // [P][KTS] |x|^2
    cf* sX = reinterpret_cast<cf*>(sQ + (size_t)P * KTS);                 // [P][KTS] x
    const int tid = threadIdx.x;
    for (int q = tid; q < nU; q += KNT) sU[q] = __ldg(k.U + q);

    // this thread's block: fields f0 .. f0+3, samples 4 sb .. 4 sb + 3
    const int nfb = (P + 3) / 4;
    const int fb = tid / (KTS / 4), sb = tid % (KTS / 4);
    const bool active = fb < nfb;
    const int f0 = fb * 4;
    const int n_tiles = (N + KTS - 1) / KTS;
    auto rowoff = [P](int r) { return r * P - r * (r - 1) / 2; };   // start of row r in the triangle

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int t0 = tile * KTS;
        if (!tile_live(io.slot_steps, io.slot_len, t0, KTS, N)) continue;   // uniform over the CTA
        __syncthreads();   // kappa staged / the previous tile's x and |x|^2 no longer read
        for (int e = tid; e < P * KTS; e += KNT) {
            const int f = e / KTS, s = e % KTS, t = t0 + s;
            cf x = make_float2(0.f, 0.f);
            if (t < N) {
                const size_t gi = (size_t)f * N + t;
                x = io.in0[gi];
                if (io.in1) {
                    const cf y = io.in1[gi];
                    x.x = fmaf(io.in1_coef, y.x, x.x);
                    x.y = fmaf(io.in1_coef, y.y, x.y);
                }
            }
            sX[e] = x;
            sQ[e] = fmaf(x.x, x.x, x.y * x.y);
        }
        __syncthreads();
        if (!active) continue;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        const float4* Q4 = reinterpret_cast<const float4*>(sQ) + sb;   // row g at Q4[g * KTS/4]
        auto fma_block = [&](const float* kv, const float4 q) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fmaf(kv[i], q.x, acc[i][0]);
                acc[i][1] = fmaf(kv[i], q.y, acc[i][1]);
                acc[i][2] = fmaf(kv[i], q.z, acc[i][2]);
                acc[i][3] = fmaf(kv[i], q.w, acc[i][3]);
            }
        };
        // g < f0: kappa_(f0+i) g = U[rowoff(g) + f0 + i - g], four consecutive values of row g
        int base = f0;   // rowoff(g) - g + f0 for g = 0
        for (int g = 0; g < f0; ++g) {
            const float kv[4] = {sU[base], sU[base + 1], sU[base + 2], sU[base + 3]};
            fma_block(kv, Q4[g * (KTS / 4)]);
            base += P - g - 1;
        }
        // the diagonal block f0 <= g < f0 + 4 (rows beyond P carry zero)
        for (int g = f0; g < f0 + 4 && g < P; ++g) {
            float kv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int f = f0 + i;
                kv[i] = f >= P ? 0.f : (f <= g ? sU[rowoff(f) + g - f] : sU[rowoff(g) + f - g]);
            }
            fma_block(kv, Q4[g * (KTS / 4)]);
        }
        // g >= f0 + 4: kappa_(f0+i) g = U[rowoff(f0+i) + g - (f0+i)], one value from each row
        {
            const float* r0 = sU + rowoff(f0) - f0;
            const float* r1 = f0 + 1 < P ? sU + rowoff(f0 + 1) - (f0 + 1) : r0;
            const float* r2 = f0 + 2 < P ? sU + rowoff(f0 + 2) - (f0 + 2) : r0;
            const float* r3 = f0 + 3 < P ? sU + rowoff(f0 + 3) - (f0 + 3) : r0;
            for (int g = f0 + 4; g < P; ++g) {
                const float kv[4] = {r0[g], r1[g], r2[g], r3[g]};
                fma_block(kv, Q4[g * (KTS / 4)]);
            }
        }
        // out = i * scale * phi * x
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int f = f0 + i;
            if (f >= P) break;
            const cf* xr = sX + (size_t)f * KTS + sb * 4;
            cf o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float a = scale * acc[i][j];
                o[j] = make_float2(-a * xr[j].y, a * xr[j].x);
            }
            const int t = t0 + sb * 4;
            cf* dst = io.out + (size_t)f * N + t;
            if (t + 3 < N) {
                reinterpret_cast<float4*>(dst)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                reinterpret_cast<float4*>(dst)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (t + j < N) dst[j] = o[j];
            }
        }
    }
}

}  // namespace

size_t kerr_kappa_smem_bytes(int P) {
    const size_t nU = (size_t)P * (P + 1) / 2;
    return ((nU + 3) & ~(size_t)3) * 4 + (size_t)P * KTS * 4 + (size_t)P * KTS * 8;
}

cudaError_t kerr_kappa_launch(const KerrKappa& k, const KerrIO& io, float scale, int N, int n_sm, cudaStream_t s) {
    if (k.P < 1 || k.P > 256) return cudaErrorInvalidValue;
    const size_t smem = kerr_kappa_smem_bytes(k.P);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kerr_kappa_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kerr_kappa_kernel, KNT, smem);
    if (e != cudaSuccess) return e;
    const int n_tiles = (N + KTS - 1) / KTS;
    const int grid = n_tiles < n_sm * (per_sm > 0 ? per_sm : 1) ? n_tiles : n_sm * (per_sm > 0 ? per_sm : 1);
    kerr_kappa_kernel<<<grid, KNT, smem, s>>>(k, io, scale, N);
    return cudaGetLastError();
}

}  // namespace mmf
