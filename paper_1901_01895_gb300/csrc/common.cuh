// Device helpers shared by the RK4IP kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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

// Compile-time loop: f(std::integral_constant<int, i>) for i = B .. E-1, so that i can serve as a
// template argument or in a constant expression inside f.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// cos(2 pi e / 32) and sin(2 pi e / 32) for any integer e, from cos(k pi / 16), k = 0..8.
__host__ __device__ constexpr double cos_pi16(int k) {
    return k == 0 ? 1.0
         : k == 1 ? 0.98078528040323044912618223613424
         : k == 2 ? 0.92387953251128675612818318939679
         : k == 3 ? 0.83146961230254523707878837761791
         : k == 4 ? 0.70710678118654752440084436210485
         : k == 5 ? 0.55557023301960222474283081394853
         : k == 6 ? 0.38268343236508977172845998403040
         : k == 7 ? 0.19509032201612826784828486847702
         : 0.0;
}
__host__ __device__ constexpr double cos32(int e) {
    e &= 31;
    return e <= 8 ? cos_pi16(e) : e <= 16 ? -cos_pi16(16 - e) : e <= 24 ? -cos_pi16(e - 16) : cos_pi16(32 - e);
}
__host__ __device__ constexpr double sin32(int e) { return cos32(8 - e); }

// x * W_R^E (W_R = exp(-2 pi i / R), conjugated for INV) for R dividing 32, with the constant as
// a compile-time double-float: quarter turns are exact swaps, eighth turns (c = +-s) take one
// rounded add per component and a double-float scale, the rest the full double-float product.
template <int R, int E, bool INV>
__device__ __forceinline__ cf rotc(cf x) {
    constexpr int e = ((E * (32 / R)) % 32 + 32) % 32;   // exponent of W_32
    if constexpr (e == 0) {
        return x;
    } else if constexpr (e == 8) {
        return mul_mi<INV>(x);
    } else if constexpr (e == 16) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (e == 24) {
        return mul_mi<!INV>(x);
    } else {
        constexpr double c = cos32(e), s = INV ? sin32(e) : -sin32(e);   // W = c + i s
        if constexpr (e % 8 == 4) {
            // c = sc h, s = ss h with h = 1/sqrt(2): x W = h ((sc x.r - ss x.i) + i (ss x.r + sc x.i))
            constexpr float sc = c > 0 ? 1.f : -1.f, ss = s > 0 ? 1.f : -1.f;
            constexpr double h = 0.70710678118654752440084436210485;
            constexpr float hh = (float)h, hl = (float)(h - (double)hh);
            const float p = fmaf(-ss, x.y, sc * x.x), q = fmaf(ss, x.x, sc * x.y);
            return make_float2(fmaf(p, hh, p * hl), fmaf(q, hh, q * hl));
        } else {
            constexpr float ch = (float)c, sh = (float)s;
            constexpr float cl = (float)(c - (double)ch), sl = (float)(s - (double)sh);
            return cmul_df<false>(x, make_float4(ch, sh, cl, sl));
        }
    }
}

// R-point DFT (R = 2, 4, 8, 16, 32) of v[0..R) in registers, natural order in and out, with
// compile-time rotations.  R = 4 * R2: n = R2*n1 + n2, k = k1 + 4*k2.
template <int R, bool INV>
__device__ __forceinline__ void dftc(cf* v) {
    if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else {
        constexpr int R2 = R / 4;
        // 4-point DFTs over n1 for each n2: y[k1][n2] at v[k1*R2 + n2]
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) dft4<INV>(v[n2], v[R2 + n2], v[2 * R2 + n2], v[3 * R2 + n2]);
        // rotations W_R^{n2 k1}
        static_for<1, R2>([&](auto n2) {
            static_for<1, 4>([&](auto k1) {
                constexpr int i = decltype(k1)::value * R2 + decltype(n2)::value;
                v[i] = rotc<R, decltype(n2)::value * decltype(k1)::value, INV>(v[i]);
            });
        });
        // R2-point DFTs over n2 for each k1: X[k1 + 4*k2]
        cf t[R];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            dftc<R2, INV>(v + k1 * R2);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) t[k1 + 4 * k2] = v[k1 * R2 + k2];
        }
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = t[i];
    }
}

// Shared-memory index with one pad slot per 16 elements (bank-conflict-free for the
// strided Stockham stores).
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

}  // namespace mmf
