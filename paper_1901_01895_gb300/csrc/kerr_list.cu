// Kerr term of Eq. 1 in its general overlap-tensor form, evaluated as a sum over the
// nonzero entries of the polarisation-resolved tensor (any real S, including the
// kappa form printed in Eq. 1).  The term is pointwise in t: one thread per time
// sample, its P field values staged in shared memory (one column per thread, so no
// synchronisation), the term list read with warp-uniform addresses (broadcast).
//
//   out_f(t) = i * scale * sum_{l <= m, n} c_{f l m n} A_l(t) A_m(t) conj(A_n(t))
//   c_{f l m n} = Sfull_{f l m n} + Sfull_{f m l n}   (l < m),   Sfull_{f l l n}   (l = m)
#include "common.cuh"
#include "kernels.h"

namespace mmf {
namespace {

__device__ __forceinline__ cf load_input(const KerrIO& io, size_t idx) {
    cf x = io.in0[idx];
    if (io.in1) {
        const cf y = io.in1[idx];
        x.x = fmaf(io.in1_coef, y.x, x.x);
        x.y = fmaf(io.in1_coef, y.y, x.y);
    }
    return x;
}

template <int NT>
__global__ void __launch_bounds__(NT) kerr_list_kernel(KerrList k, KerrIO io, float scale, int N) {
    extern __shared__ float4 smem_raw[];
    cf* sA = reinterpret_cast<cf*>(smem_raw);   // [P][NT]
    const int t = blockIdx.x * NT + threadIdx.x;
    if (t >= N || !tile_live(io.slot_steps, io.slot_len, t, 1, N)) return;
    for (int f = 0; f < k.P; ++f) sA[f * NT + threadIdx.x] = load_input(io, (size_t)f * N + t);
    const cf* col = sA + threadIdx.x;
    for (int f = 0; f < k.P; ++f) {
        float ar = 0.f, ai = 0.f;
        const int e1 = __ldg(k.term_off + f + 1);
        for (int e = __ldg(k.term_off + f); e < e1; ++e) {
            const uint32_t id = __ldg(k.idx + e);
            const float c = __ldg(k.coef + e);
            const cf al = col[(id & 1023u) * NT], am = col[((id >> 10) & 1023u) * NT], an = col[(id >> 20) * NT];
            // q = c * al * am, then acc += q * conj(an)
            const float qr = c * (al.x * am.x - al.y * am.y);
            const float qi = c * (al.x * am.y + al.y * am.x);
            ar = fmaf(qr, an.x, fmaf(qi, an.y, ar));
            ai = fmaf(qi, an.x, fmaf(-qr, an.y, ai));
        }
        io.out[(size_t)f * N + t] = make_float2(-scale * ai, scale * ar);   // i * scale * acc
    }
}

}  // namespace

cudaError_t kerr_list_launch(const KerrList& k, const KerrIO& io, float scale, int N, cudaStream_t s) {
    constexpr int NT = 128;
    const size_t smem = (size_t)k.P * NT * sizeof(cf);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kerr_list_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kerr_list_kernel<NT><<<(N + NT - 1) / NT, NT, smem, s>>>(k, io, scale, N);
    return cudaGetLastError();
}

// ------------------------------------------------------------- energy ------

namespace {
constexpr int ENT = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < ENT / 32; ++w) s += red[w];
    return s;
}

// part[row][blk] = sum over this block's samples of |A|^2 (FP64, fixed order)
__global__ void __launch_bounds__(ENT) energy_partial_kernel(const cf* __restrict__ A, int N, int nblk, double* part) {
    __shared__ double red[ENT / 32];
    const int row = blockIdx.y, blk = blockIdx.x;
    const cf* r = A + (size_t)row * N;
    double s = 0.0;
    for (int t = blk * ENT + threadIdx.x; t < N; t += nblk * ENT) {
        const cf v = r[t];
        s = fma((double)v.x, (double)v.x, s);
        s = fma((double)v.y, (double)v.y, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(size_t)row * nblk + blk] = s;
}

__global__ void energy_final_kernel(const double* __restrict__ part, int P, int nblk, double dt, double* out) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= P) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)row * nblk + b];
    out[row] = s * dt;
}
}  // namespace

int energy_blocks(int N) {
    int nblk = N / (ENT * 8);
    if (nblk < 1) nblk = 1;
    if (nblk > 64) nblk = 64;
    return nblk;
}

cudaError_t energy_launch(const float2* A, int P, int N, double dt, double* scratch, int nblk, double* out,
                          cudaStream_t s) {
    energy_partial_kernel<<<dim3(nblk, P), ENT, 0, s>>>(A, N, nblk, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<(P + 127) / 128, 128, 0, s>>>(scratch, P, nblk, dt, out);
    return cudaGetLastError();
}

}  // namespace mmf
