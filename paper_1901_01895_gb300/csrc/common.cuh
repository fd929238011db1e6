// Device helpers shared by the RK4IP kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mmf {

// Complex value as interleaved FP32 (matches the complex64 field layout).
typedef float2 cf;

// A unit-modulus constant stored as a double-float pair: value = hi + lo with hi the
// FP32 rounding of the FP64 value and lo the FP32 rounding of the remainder.  Used
// for FFT twiddles and for the propagator table: with plain FP32 constants the
// rounding error of each constant is the same at every application and the error
// grows linearly with the number of steps; with hi+lo it is random and grows as
// the square root.
typedef float4 cdf;   // (hi.re, hi.im, lo.re, lo.im)

// Request batches lay slots of slot_len samples side by side on the time axis.  A sample
// tile [t0, t0 + ts) is live when any slot it touches still has steps to run.
__device__ __forceinline__ bool tile_live(const int* slot_steps, int slot_len, int t0, int ts, int N) {
    if (!slot_steps) return true;
    const int last = (t0 + ts < N ? t0 + ts : N) - 1;
    for (int b = t0 / slot_len; b <= last / slot_len; ++b)
        if (__ldg(slot_steps + b) > 0) return true;
    return false;
}

// Complex add, subtract and real scale on packed FP32 pairs (add/fma/mul.rn.f32x2): one
// instruction per complex operation, each half rounded exactly as the scalar operation
// (a - b is fma(b, -1, a), exact product then one rounding).
__device__ __forceinline__ cf cadd(cf a, cf b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ cf csub(cf a, cf b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ cf cscale(cf a, float s) { return __fmul2_rn(a, make_float2(s, s)); }

// b * (w.hi + w.lo) with one rounding per FMA; INV multiplies by the conjugate.
template <bool INV>
__device__ __forceinline__ cf cmul_df(cf b, cdf w) {
    const float wr = w.x, wi = INV ? -w.y : w.y, lr = w.z, li = INV ? -w.w : w.w;
    const float tr = fmaf(b.x, lr, -(b.y * li));
    const float ti = fmaf(b.x, li, b.y * lr);
    return make_float2(fmaf(b.x, wr, fmaf(-b.y, wi, tr)), fmaf(b.x, wi, fmaf(b.y, wr, ti)));
}

// Multiply by -i (forward) or +i (inverse): exact.
template <bool INV>
__device__ __forceinline__ cf mul_mi(cf a) { return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

// Radix-2 and radix-4 DFT butterflies in registers (exact multiplications by +-1, +-i).
template <bool INV>
__device__ __forceinline__ void dft2(cf& a, cf& b) {
    cf t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
template <bool INV>
__device__ __forceinline__ void dft4(cf& x0, cf& x1, cf& x2, cf& x3) {
    cf a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_mi<INV>(csub(x1, x3));
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
}

// R-point DFT (R = 2, 4, 8, 16) of v[0..R) in registers, natural order in and out.
// The internal rotations W_R^m are read from the length-N twiddle table tw (W_N^j at j).
// R = R1 * R2 with R1 = 4: n = R2*n1 + n2, k = k1 + 4*k2.
template <int R, bool INV>
__device__ __forceinline__ void dft(cf* v, const cdf* __restrict__ tw, int N) {
    if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else {
        constexpr int R2 = R / 4;
        // step 1: 4-point DFTs over n1 for each n2
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) dft4<INV>(v[n2], v[R2 + n2], v[2 * R2 + n2], v[3 * R2 + n2]);
        // step 2: rotate y[n2][k1] (stored at v[k1*R2 + n2]) by W_R^{n2*k1}
#pragma unroll
        for (int n2 = 1; n2 < R2; ++n2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) {
                const int e = n2 * k1;               // exponent of W_R
                if ((4 * e) % R == 0) {               // multiple of a quarter turn: exact
                    const int q = (4 * e / R) & 3;
                    cf& x = v[k1 * R2 + n2];
                    if (q == 1) x = mul_mi<INV>(x);
                    else if (q == 2) x = make_float2(-x.x, -x.y);
                    else if (q == 3) x = mul_mi<!INV>(x);
                } else {
                    v[k1 * R2 + n2] = cmul_df<INV>(v[k1 * R2 + n2], __ldg(tw + e * (N / R)));
                }
            }
        // step 3: R2-point DFTs over n2 for each k1; output X[k1 + 4*k2]
        cf t[R];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            if constexpr (R2 == 2) {
                cf a = v[k1 * 2], b = v[k1 * 2 + 1];
                dft2<INV>(a, b);
                t[k1] = a; t[k1 + 4] = b;
            } else {
                cf a = v[k1 * 4], b = v[k1 * 4 + 1], c = v[k1 * 4 + 2], d = v[k1 * 4 + 3];
                dft4<INV>(a, b, c, d);
                t[k1] = a; t[k1 + 4] = b; t[k1 + 8] = c; t[k1 + 12] = d;
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = t[i];
    }
}

// Shared-memory index with one pad slot per 16 elements (bank-conflict-free for the
// strided Stockham stores).
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

}  // namespace mmf
