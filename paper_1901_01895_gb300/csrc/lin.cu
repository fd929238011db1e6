// Fused linear step of the RK4IP scheme: out = IFFT(E * FFT(in)) per field row, with
// E_f(omega_k) = exp(h/2 * D_f(omega_k)) (Eq. 1 linear operator, Eq. 4 uses it four
// times per step), together with the Runge-Kutta stage combines that feed it and
// consume it.
//
// Rows of up to 2^14 samples: one CTA per row holds the row in shared memory, one HBM read
// and one write per field sample.  Its FFT is Stockham radix-16 passes (radix 2/4/8 for the
// remainder) in registers with shared-memory transposes; the last forward pass, the
// propagator multiply and the first inverse pass touch the same 16 values per butterfly and
// run fused in registers.  The inverse mirrors the forward path.
//
// Longer rows (2^15 .. 2^17 samples, N = C*L with slices of L = 2^13) take three passes over a
// scratch row: with n = L*n1 + n2 and k = k1 + C*k2 the DFT splits into C-point DFTs over n1
// (read straight from HBM, one element of each of the C segments) and a twiddle W_N^{n2 k1}
// (pass A), an L-point FFT, the propagator and the L-point inverse per slice k1 (pass B), and
// the inverse of pass A (pass C).
//
// Twiddles are double-float (hi + lo) values.  The rotations inside the radix-2..32 DFTs are
// compile-time constants; the twiddles between passes come from small shared-memory tables.
#include "common.cuh"
#include "kernels.h"

namespace mmf {

namespace {

constexpr int TW1K = 1024;   // entries of the W_1024 table
constexpr int TLO = 64;      // entries of the W_L low-factor table
// The tables are read at strides k*r (k consecutive over a warp): with power-of-two r the
// 16-byte entries of a warp would fall into the same banks.  One pad entry per eight breaks
// that pattern.
__host__ __device__ constexpr int tpad(int m) { return m + (m >> 3); }
constexpr int TW1K_P = tpad(TW1K), TLO_P = tpad(TLO);

// Shared twiddle tables of one CTA.
struct Tw {
    const cdf* w1k;   // W_1024^m (or W_N^m for N <= 1024, then nfull = N)
    const cdf* wl;    // W_L^m, m < 64
    int nfull;        // 1024, or N when N <= 1024 (then w1k is the whole W_N table)
};

// x * W_D^m for a denominator D dividing Dbig (Dbig = L with the W_L low-factor table, or
// N with the W_N one).  Small D read the W_1024 table; otherwise with m' = m*Dbig/D,
// W_D^m = W_Dbig^{m'} = W_Dbig^{m' mod nlo} * W_{Dbig/nlo}^{m' / nlo} (two factors).
template <bool INV>
__device__ __forceinline__ cf tw_apply_big(cf x, const Tw& t, const cdf* lo, int nlo, int Dbig, int D, int m) {
    if (D <= t.nfull) return cmul_df<INV>(x, t.w1k[tpad(m * (t.nfull / D))]);
    const int mm = m * (Dbig / D);
    const int mlo = mm & (nlo - 1), mhi = mm / nlo;
    x = cmul_df<INV>(x, lo[tpad(mlo)]);
    return cmul_df<INV>(x, t.w1k[tpad(mhi * (t.nfull / (Dbig / nlo)))]);
}

template <int LOGL>
struct Plan {
    static constexpr int L = 1 << LOGL;
    static constexpr int Q = LOGL / 4;             // radix-16 passes
    static constexpr int REM = 1 << (LOGL % 4);    // remainder radix (1 = none)
    static constexpr int NT = L / 16 < 1024 ? L / 16 : 1024;   // 16 values per thread
    static constexpr int EPT = L / NT;             // 16 or 32 values per thread
    static constexpr int NB16 = EPT / 16;          // radix-16 butterflies per thread
};

// One Stockham pass of radix R over the L-point row in shared memory (the twiddle
// denominator Ns*R is at most 1024, except in the last inverse pass where it is L):
// butterfly j reads in[j + r*L/R], applies W_{Ns R}^{k r} (k = j mod Ns), an R-point DFT,
// and writes out[(j - k)*R + k + r*Ns].  The pass is in place: only the stores wait for
// every thread's loads, so the twiddles and the DFT run before that barrier.
template <int LOGL, int R, bool INV>
__device__ __forceinline__ void stockham_pass(cf* buf, int Ns, const Tw& t) {
    using PL = Plan<LOGL>;
    constexpr int L = PL::L, NT = PL::NT;
    constexpr int NB = (L / R) / NT;
    static_assert(NB * R == PL::EPT, "pass shape");
    cf v[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = threadIdx.x + b * NT;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = buf[spad(j + r * (L / R))];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = threadIdx.x + b * NT;
        const int k = j & (Ns - 1);
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[b][r] = tw_apply_big<INV>(v[b][r], t, t.wl, TLO, L, Ns * R, k * r);
        }
        dftc<R, INV>(v[b]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = threadIdx.x + b * NT;
        const int k = j & (Ns - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[spad(base + r * Ns)] = v[b][r];
    }
    __syncthreads();
}

// Forward passes before the fused middle: [REM (if > 1), 16 x (Q-1)].
template <int LOGL>
__device__ __forceinline__ void forward_head(cf* buf, const Tw& t) {
    using PL = Plan<LOGL>;
    int Ns = 1;
    if constexpr (PL::REM > 1) {
        stockham_pass<LOGL, PL::REM, false>(buf, Ns, t);
        Ns *= PL::REM;
    }
#pragma unroll 1
    for (int q = 0; q < PL::Q - 1; ++q) {
        stockham_pass<LOGL, 16, false>(buf, Ns, t);
        Ns *= 16;
    }
}

// Inverse passes after the fused middle: [16 x (Q-1), REM (if > 1)], Ns starting at 16.
template <int LOGL>
__device__ __forceinline__ void inverse_tail(cf* buf, const Tw& t) {
    using PL = Plan<LOGL>;
    int Ns = 16;
#pragma unroll 1
    for (int q = 0; q < PL::Q - 1; ++q) {
        stockham_pass<LOGL, 16, true>(buf, Ns, t);
        Ns *= 16;
    }
    if constexpr (PL::REM > 1) stockham_pass<LOGL, PL::REM, true>(buf, Ns, t);
}

// Last forward radix-16 pass (Ns = L/16), propagator multiply, first inverse radix-16
// pass (Ns = 1), on the 16 values butterfly j holds at positions j + r*L/16 (position p is
// frequency p).
template <int LOGL>
__device__ __forceinline__ void fused_middle(cf* buf, const Tw& t, const cdf* __restrict__ Erow) {
    using PL = Plan<LOGL>;
    constexpr int L = PL::L, NT = PL::NT;
    cf v[PL::NB16][16];
#pragma unroll
    for (int b = 0; b < PL::NB16; ++b) {
        const int j = threadIdx.x + b * NT;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[b][r] = buf[spad(j + r * (L / 16))];
    }
    // everything up to the stores runs before the barrier (the pass is in place)
#pragma unroll
    for (int b = 0; b < PL::NB16; ++b) {
        const int j = threadIdx.x + b * NT;
        if (L > 16 && j != 0) {
#pragma unroll
            for (int r = 1; r < 16; ++r) v[b][r] = tw_apply_big<false>(v[b][r], t, t.wl, TLO, L, L, j * r);
        }
        dftc<16, false>(v[b]);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[b][r] = cmul_df<false>(v[b][r], __ldg(Erow + j + r * (L / 16)));
        dftc<16, true>(v[b]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < PL::NB16; ++b) {
        const int j = threadIdx.x + b * NT;
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[spad(j * 16 + r)] = v[b][r];
    }
    __syncthreads();
}

__device__ __forceinline__ cf load_combined(const LinArgs& a, size_t idx) {
    cf v = a.in[0][idx];
    if (a.coef[0] != 1.0f) v = cscale(v, a.coef[0]);
#pragma unroll
    for (int i = 1; i < LinArgs::MAX_IN; ++i) {
        if (i < a.n_in) {
            v = __ffma2_rn(make_float2(a.coef[i], a.coef[i]), a.in[i][idx], v);
        }
    }
    return v;
}

// Output stores of K values per thread, out = v + add_coef * add: the added row is read in full
// before the first store (add never aliases out), so that the K reads overlap instead of
// waiting one by one behind stores the compiler cannot move past them.
template <int K, int STRIDE>
__device__ __forceinline__ void store_combined_k(const LinArgs& a, size_t idx0, const cf* v) {
    if (a.add) {
        cf ad[K];
#pragma unroll
        for (int i = 0; i < K; ++i) ad[i] = a.add[idx0 + (size_t)i * STRIDE];
        const float2 c = make_float2(a.add_coef, a.add_coef);
#pragma unroll
        for (int i = 0; i < K; ++i) a.out[idx0 + (size_t)i * STRIDE] = __ffma2_rn(c, ad[i], v[i]);
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) a.out[idx0 + (size_t)i * STRIDE] = v[i];
    }
}

// Propagator row of row r = f * e_batch + b: ((r / e_batch) >> e_shift) * e_batch + b.
__device__ __forceinline__ int e_row(const LinArgs& a, int r) {
    const int f = r / a.e_batch, b = r - f * a.e_batch;
    return (f >> a.e_shift) * a.e_batch + b;
}

// Fill the CTA's twiddle tables from the global W_N table (N entries, double-float).
__device__ __forceinline__ Tw load_twiddles(cdf* st, const cdf* __restrict__ tw, int N, int L, int nthreads) {
    Tw t;
    cdf* w1k = st;
    cdf* wl = st + TW1K_P;
    t.nfull = N <= TW1K ? N : TW1K;
    for (int m = threadIdx.x; m < t.nfull; m += nthreads) w1k[tpad(m)] = __ldg(tw + m * (N / t.nfull));
    for (int m = threadIdx.x; m < TLO; m += nthreads) wl[tpad(m)] = __ldg(tw + (size_t)(m % L) * (N / L));
    t.w1k = w1k;
    t.wl = wl;
    return t;
}
constexpr int TW_SMEM = (TW1K_P + TLO_P) * (int)sizeof(cdf);

// Single-CTA rows (C = 1): N = L <= 2^14.
template <int LOGL>
__global__ void __launch_bounds__(Plan<LOGL>::NT) lin_kernel_c1(LinArgs a) {
    using PL = Plan<LOGL>;
    extern __shared__ float4 smem_raw[];
    cdf* st = reinterpret_cast<cdf*>(smem_raw);
    cf* buf = reinterpret_cast<cf*>(st + TW1K_P + TLO_P);
    const int row = blockIdx.x;
    if (a.slot_steps && __ldg(a.slot_steps + row % a.e_batch) <= 0) return;
    const size_t base = (size_t)row * PL::L;
    const cdf* Erow = a.E + (size_t)e_row(a, row) * PL::L;
    const Tw t = load_twiddles(st, a.tw, PL::L, PL::L, PL::NT);
#pragma unroll
    for (int i = 0; i < PL::EPT; ++i) {
        const int n = threadIdx.x + i * PL::NT;
        buf[spad(n)] = load_combined(a, base + n);
    }
    __syncthreads();
    forward_head<LOGL>(buf, t);
    fused_middle<LOGL>(buf, t, Erow);
    inverse_tail<LOGL>(buf, t);
    cf v[PL::EPT];
#pragma unroll
    for (int i = 0; i < PL::EPT; ++i) v[i] = buf[spad(threadIdx.x + i * PL::NT)];
    store_combined_k<PL::EPT, PL::NT>(a, base + threadIdx.x, v);
}

// Rows of N = C * L samples, 2^15 .. 2^17 (C = 4, 8, 16 slices of L = 2^13), in three passes
// through a scratch row in global memory:
//   A  y[k1][n2] = W_N^{n2 k1} sum_n1 W_C^{n1 k1} x[L n1 + n2]   (C-point DFTs, one column a thread)
//   B  per slice k1: L-point FFT, propagator, L-point IFFT, in place (one CTA a slice)
//   C  x[L n1 + n2] = sum_k1 W_C^{-n1 k1} W_N^{-n2 k1} z[k1][n2]  (C-point inverse DFTs, combines)
// A row in one thread-block cluster exchanging through distributed shared memory would save
// the two scratch round trips, but large clusters place badly (eight-CTA clusters of one CTA
// per SM left 32 of the 152 SMs idle).  Slices of 2^13 (92 KB of shared memory) let two CTAs
// share an SM, so that one CTA's HBM reads and writes overlap the other's FFT passes.
// The twiddles of A and C, W_N^{n2 k1} with n2 = 32 nh + nl, are two factors:
// TA2[k1][nl] = W_N^{nl k1} from a shared table (a warp reads 32 consecutive entries) and
// W_{N/32}^{nh k1}, the same for the whole warp, read from the W_N table at stride 32.  Both
// passes run a persistent grid, one table fill per CTA.
constexpr int SPLIT_NT = 256;
constexpr int SPLIT_TA = 16 * 32;

__device__ __forceinline__ void split_table(cdf* TA2, const cdf* __restrict__ tw) {
    for (int i = threadIdx.x; i < SPLIT_TA; i += SPLIT_NT) TA2[i] = __ldg(tw + (i & 31) * (i >> 5));
    __syncthreads();
}

// x * W_N^{n2 k1} (conjugate for INV) for k1 = 1 .. C-1.
template <int C, int LOGL, bool INV>
__device__ __forceinline__ void split_twiddles(cf* x, const cdf* TA2, const cdf* __restrict__ tw, int n2) {
    const int nl = n2 & 31, nh = n2 >> 5;
#pragma unroll
    for (int k1 = 1; k1 < C; ++k1) {
        const cdf hi = __ldg(tw + (size_t)(nh * k1) * 32);   // W_{N/32}^{nh k1}: one address per warp
        x[k1] = cmul_df<INV>(cmul_df<INV>(x[k1], TA2[k1 * 32 + nl]), hi);
    }
}

template <int C, int LOGL, int NIN>
__global__ void __launch_bounds__(SPLIT_NT, 3) lin_split_a(LinArgs a, int rows) {
    constexpr int L = 1 << LOGL, N = C * L;
    __shared__ cdf TA2[SPLIT_TA];
    split_table(TA2, a.tw);
    const size_t total = (size_t)rows * L;
    for (size_t idx = blockIdx.x * (size_t)SPLIT_NT + threadIdx.x; idx < total; idx += (size_t)gridDim.x * SPLIT_NT) {
        const int row = (int)(idx / L), n2 = (int)(idx % L);
        if (a.slot_steps && __ldg(a.slot_steps + row % a.e_batch) <= 0) continue;
        const size_t base = (size_t)row * N + n2;
        cf x[C];
        // x = c0 in0 + c1 in1 + ... in this order of roundings (the scale only when c0 != 1)
#pragma unroll
        for (int n1 = 0; n1 < C; ++n1) x[n1] = a.in[0][base + (size_t)n1 * L];
        if (a.coef[0] != 1.0f) {
#pragma unroll
            for (int n1 = 0; n1 < C; ++n1) x[n1] = cscale(x[n1], a.coef[0]);
        }
#pragma unroll
        for (int i = 1; i < NIN; ++i) {
            const float2 c = make_float2(a.coef[i], a.coef[i]);
#pragma unroll
            for (int n1 = 0; n1 < C; ++n1) x[n1] = __ffma2_rn(c, a.in[i][base + (size_t)n1 * L], x[n1]);
        }
        dftc<C, false>(x);
        split_twiddles<C, LOGL, false>(x, TA2, a.tw, n2);
#pragma unroll
        for (int k1 = 0; k1 < C; ++k1) a.scratch[base + (size_t)k1 * L] = x[k1];
    }
}

// Pass B for slices of L = 2^13 samples: FFT, propagator and IFFT of each slice, one slice at a
// time per persistent CTA of 256 threads.  The forward FFT is three self-sorting (Stockham)
// passes of radix 32, 16, 16: pass (R, Ns) takes butterfly j, loads in[j + r L/R], multiplies
// by the twiddle W_{Ns R}^{k r} (k = j mod Ns), does an R-point DFT and stores
// out[(j - k) R + k + r Ns].  The inverse is the conjugate transpose of the same three passes in
// reverse order (the DFT matrix is symmetric, so its inverse is conj(F^T)/N): each transposed
// pass loads where the forward pass stored, does the conjugate DFT, multiplies by the conjugate
// twiddle after it and stores where the forward pass loaded.  Hence
//   pass 3 (forward, the propagator, transposed inverse) reads and writes the positions
//          j + 512 r of its own butterflies only: no barrier inside it;
//   the last inverse pass (radix 32, Ns = 1) has no twiddles;
//   the first forward pass reads the slice from the scratch row and the last inverse pass
//          writes it back (unit stride over the threads): four shared-memory round trips, plus
//          the middle pass's read-modify-write of its own positions for its conjugate twiddles.
// Radix-16 passes give each thread butterflies t and t + 256.  Twiddle tables are indexed
// [r][lane] so that a warp reads consecutive entries: T2[r][k] = W_512^{k r} (k = t mod 32)
// for pass 2 and its transpose, and W_8192^{j r} = TA[r][j mod 64] * W_128^{(j / 64) r}, the second factor the
// same for a whole warp.  Rotations inside the DFTs are compile-time constants.
namespace s13 {
constexpr int L = 1 << 13;
constexpr int NT = 256;
constexpr int N_T2 = 16 * 32, N_TA = 16 * 64, N_W128 = 128;
constexpr size_t SMEM = (size_t)(N_T2 + N_TA + N_W128) * sizeof(cdf) + (size_t)L * sizeof(cf);
// Swizzled shared-memory index (8-byte units): bits 0-3 XORed with bits 4-7 and 5-8.  Every
// access of these passes over 16 consecutive threads (unit stride; stride 16, whose swizzle is
// the Gray code of the thread; stride 32) then falls on 16 different bank pairs, with no padding.
__device__ __forceinline__ int sw(int a) { return a ^ (((a >> 4) ^ (a >> 5)) & 15); }
}  // namespace s13

template <int C>
__global__ void __launch_bounds__(s13::NT, 2) lin_slice13(LinArgs a, int rows) {
    using namespace s13;
    constexpr int N = C * L;
    extern __shared__ float4 smem_raw[];
    cdf* T2 = reinterpret_cast<cdf*>(smem_raw);   // [r][k]  = W_512^{k r}
    cdf* TA = T2 + N_T2;                           // [r][jl] = W_8192^{jl r}
    cdf* W128 = TA + N_TA;                         // [m]     = W_128^m
    cf* buf = reinterpret_cast<cf*>(W128 + N_W128);
    const int t = threadIdx.x;
    for (int i = t; i < N_T2; i += NT) T2[i] = __ldg(a.tw + (((i & 31) * (i >> 5)) & 511) * (N / 512));
    for (int i = t; i < N_TA; i += NT) TA[i] = __ldg(a.tw + (i & 63) * (i >> 6) * (N / L));
    if (t < N_W128) W128[t] = __ldg(a.tw + t * (N / 128));
    // (the first barrier of the slice loop orders these stores before any table read)

    for (int sl = blockIdx.x; sl < rows * C; sl += gridDim.x) {
        const int row = sl / C, k1 = sl % C;
        if (a.slot_steps && __ldg(a.slot_steps + row % a.e_batch) <= 0) continue;
        cf* slice = a.scratch + (size_t)row * N + (size_t)k1 * L;
        // entry (k1, p) of the propagator row is frequency k1 + C p of the full row
        const cdf* __restrict__ Es = a.E + (size_t)e_row(a, row) * N + (size_t)k1 * L;
        // the propagator slice (128 KB) is read in pass 3: start bringing it into L2 now
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(Es) + (size_t)(t + NT * i) * 128));

        // pass 1: radix 32, Ns = 1 (no twiddles), straight from the scratch row
        {
            cf v[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = slice[t + 256 * r];
            dftc<32, false>(v);
            __syncthreads();   // the previous slice's last loads from buf are done
#pragma unroll
            for (int r = 0; r < 32; ++r) buf[sw(32 * t + r)] = v[r];
        }
        __syncthreads();

        // the next slice of this CTA is read at the start of its pass 1: bring it into L2 now,
        // two 128-byte lines per thread
        if (sl + (int)gridDim.x < rows * C) {
            const int nrow = (sl + gridDim.x) / C, nk1 = (sl + gridDim.x) % C;
            const char* nx = reinterpret_cast<const char*>(a.scratch + (size_t)nrow * N + (size_t)nk1 * L);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + (size_t)t * 128));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + (size_t)(t + NT) * 128));
        }

        // pass 2: radix 16, Ns = 32, butterflies t and t + 256 (same k = t mod 32, same twiddles)
        const int k = t & 31;
        {
            cf v[2][16];
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int r = 0; r < 16; ++r) v[b][r] = buf[sw(t + 256 * b + 512 * r)];
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                const cdf w = T2[r * 32 + k];
                v[0][r] = cmul_df<false>(v[0][r], w);
                v[1][r] = cmul_df<false>(v[1][r], w);
            }
            dftc<16, false>(v[0]);
            dftc<16, false>(v[1]);
            __syncthreads();
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int base = (t + 256 * b - k) * 16 + k;
#pragma unroll
                for (int r = 0; r < 16; ++r) buf[sw(base + 32 * r)] = v[b][r];
            }
        }
        __syncthreads();

        // pass 3: radix 16, Ns = 512 (twiddle W_8192^{j r}), the propagator at frequency
        // j + 512 r, and its transpose (conjugate DFT, conjugate twiddle) back to the same positions;
        // one butterfly at a time (both at once hold two propagator slices and spill)
#pragma unroll 1
        for (int b = 0; b < 2; ++b) {
            const int j = t + 256 * b, jl = j & 63, jh = j >> 6;
            cf v[16];
            cdf e[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = buf[sw(j + 512 * r)];
#pragma unroll
            for (int r = 0; r < 16; ++r) e[r] = __ldg(Es + j + 512 * r);
#pragma unroll
            for (int r = 1; r < 16; ++r)
                v[r] = cmul_df<false>(cmul_df<false>(v[r], TA[r * 64 + jl]), W128[(jh * r) & 127]);
            dftc<16, false>(v);
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = cmul_df<false>(v[r], e[r]);
            dftc<16, true>(v);
#pragma unroll
            for (int r = 0; r < 16; ++r) buf[sw(j + 512 * r)] = v[r];
            // the conjugate twiddles as a read-modify-write of the thread's own positions: applied
            // in registers, the compiler hoists all thirty table loads next to the sixteen values and
            // spills
            asm volatile("" ::: "memory");
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                const int p = sw(j + 512 * r);
                buf[p] = cmul_df<true>(cmul_df<true>(buf[p], TA[r * 64 + jl]), W128[(jh * r) & 127]);
            }
        }
        __syncthreads();

        // pass 2 transposed: loads where pass 2 stored, conjugate DFT, conjugate twiddle, stores
        // where pass 2 loaded
        {
            cf v[2][16];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int base = (t + 256 * b - k) * 16 + k;
#pragma unroll
                for (int r = 0; r < 16; ++r) v[b][r] = buf[sw(base + 32 * r)];
            }
            dftc<16, true>(v[0]);
            dftc<16, true>(v[1]);
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                const cdf w = T2[r * 32 + k];
                v[0][r] = cmul_df<true>(v[0][r], w);
                v[1][r] = cmul_df<true>(v[1][r], w);
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int r = 0; r < 16; ++r) buf[sw(t + 256 * b + 512 * r)] = v[b][r];
        }
        __syncthreads();

        // pass 1 transposed: radix 32, no twiddles, straight back to the scratch row
        {
            cf v[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = buf[sw(32 * t + r)];
            dftc<32, true>(v);
#pragma unroll
            for (int r = 0; r < 32; ++r) slice[t + 256 * r] = v[r];
        }
    }
}

template <int C, int LOGL>
__global__ void __launch_bounds__(SPLIT_NT, 3) lin_split_c(LinArgs a, int rows) {
    constexpr int L = 1 << LOGL, N = C * L;
    __shared__ cdf TA2[SPLIT_TA];
    split_table(TA2, a.tw);
    const size_t total = (size_t)rows * L;
    for (size_t idx = blockIdx.x * (size_t)SPLIT_NT + threadIdx.x; idx < total; idx += (size_t)gridDim.x * SPLIT_NT) {
        const int row = (int)(idx / L), n2 = (int)(idx % L);
        if (a.slot_steps && __ldg(a.slot_steps + row % a.e_batch) <= 0) continue;
        const size_t base = (size_t)row * N + n2;
        cf x[C];
#pragma unroll
        for (int k1 = 0; k1 < C; ++k1) x[k1] = a.scratch[base + (size_t)k1 * L];
        split_twiddles<C, LOGL, true>(x, TA2, a.tw, n2);
        dftc<C, true>(x);
        store_combined_k<C, L>(a, base, x);
    }
}

template <int LOGL>
cudaError_t launch_c1(const LinArgs& a, int rows, cudaStream_t s) {
    using PL = Plan<LOGL>;
    const size_t smem = TW_SMEM + (size_t)(PL::L + PL::L / 16) * sizeof(cf);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(lin_kernel_c1<LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    lin_kernel_c1<LOGL><<<rows, PL::NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int C, int LOGL>
cudaError_t launch_split(const LinArgs& a, int rows, cudaStream_t s) {
    using PL = Plan<LOGL>;
    const size_t cols = (size_t)rows * PL::L;
    const size_t cap = (size_t)(a.n_sm > 0 ? a.n_sm : 1) * 3;   // persistent: 3 CTAs of 256 threads per SM
    const unsigned gridc = (unsigned)((cols + SPLIT_NT - 1) / SPLIT_NT < cap ? (cols + SPLIT_NT - 1) / SPLIT_NT : cap);
    switch (a.n_in) {
        case 1: lin_split_a<C, LOGL, 1><<<gridc, SPLIT_NT, 0, s>>>(a, rows); break;
        case 2: lin_split_a<C, LOGL, 2><<<gridc, SPLIT_NT, 0, s>>>(a, rows); break;
        case 3: lin_split_a<C, LOGL, 3><<<gridc, SPLIT_NT, 0, s>>>(a, rows); break;
        case 4: lin_split_a<C, LOGL, 4><<<gridc, SPLIT_NT, 0, s>>>(a, rows); break;
        case 5: lin_split_a<C, LOGL, 5><<<gridc, SPLIT_NT, 0, s>>>(a, rows); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static_assert(LOGL == 13, "pass B is written for slices of 2^13 samples");
    if ((e = cudaFuncSetAttribute(lin_slice13<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s13::SMEM)) !=
        cudaSuccess)
        return e;
    const int slices = rows * C, gridb = slices < 2 * a.n_sm ? slices : 2 * (a.n_sm > 0 ? a.n_sm : 1);
    lin_slice13<C><<<gridb, s13::NT, s13::SMEM, s>>>(a, rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    lin_split_c<C, LOGL><<<gridc, SPLIT_NT, 0, s>>>(a, rows);
    return cudaGetLastError();
}

// FP64 tables: twiddles W_N^j and the propagator exp(z D_f(omega_k)) / N.
__global__ void twiddle_table_kernel(cdf* tw, int N) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)j / (double)N, &s, &c);
        const double re = c, im = -s;
        const float hr = (float)re, hi = (float)im;
        tw[j] = make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
    }
}

// Entry (row, q) with q = k1*L + p holds frequency k = k1 + C*p (C slices of L samples per
// row), so that each slice reads a contiguous part.  L is the whole row up to 2^14 samples
// (C = 1), and 2^13 for the three-pass rows (2^15 .. 2^17).
__global__ void propagator_table_kernel(cdf* E, const double* __restrict__ betas, int rows, int row_stride,
                                        int N, double dt, double alpha, double z, size_t out_pitch) {
    const size_t total = (size_t)rows * N;
    const int L = lin_needs_scratch(N) ? (1 << 13) : N, C = N / L;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(idx / N), q = (int)(idx % N);
        const int k = (q / L) + C * (q % L);
        const double* b = betas + (size_t)row * row_stride * 4;
        const int ks = (k < N / 2) ? k : k - N;
        const double w = 2.0 * 3.14159265358979323846 * (double)ks / ((double)N * dt);
        const double phase = z * (b[0] - b[1] * w + b[2] * w * w / 2.0 - b[3] * w * w * w / 6.0);
        const double mag = exp(-alpha * z / 2.0) / (double)N;
        double s, c;
        sincos(phase, &s, &c);
        const double re = mag * c, im = mag * s;
        const float hr = (float)re, hi = (float)im;
        E[(size_t)row * out_pitch + q] = make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
    }
}

// Amplifier of a multi-span link: A = g * A + noise (noise may be NULL), g = sqrt(power gain).
__global__ void amplify_kernel(cf* A, float g, const cf* __restrict__ noise, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cf a = A[i];
        a.x *= g;
        a.y *= g;
        if (noise) {
            const cf w = noise[i];
            a.x += w.x;
            a.y += w.y;
        }
        A[i] = a;
    }
}

__global__ void slot_tick_kernel(int* steps, int n) {
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        if (steps[b] > 0) steps[b] -= 1;
}

}  // namespace

cudaError_t lin_launch(const LinArgs& a, int rows, int N, cudaStream_t s) {
    switch (N) {
        case 1 << 4: return launch_c1<4>(a, rows, s);
        case 1 << 5: return launch_c1<5>(a, rows, s);
        case 1 << 6: return launch_c1<6>(a, rows, s);
        case 1 << 7: return launch_c1<7>(a, rows, s);
        case 1 << 8: return launch_c1<8>(a, rows, s);
        case 1 << 9: return launch_c1<9>(a, rows, s);
        case 1 << 10: return launch_c1<10>(a, rows, s);
        case 1 << 11: return launch_c1<11>(a, rows, s);
        case 1 << 12: return launch_c1<12>(a, rows, s);
        case 1 << 13: return launch_c1<13>(a, rows, s);
        case 1 << 14: return launch_c1<14>(a, rows, s);
        case 1 << 15: return a.scratch ? launch_split<4, 13>(a, rows, s) : cudaErrorInvalidValue;
        case 1 << 16: return a.scratch ? launch_split<8, 13>(a, rows, s) : cudaErrorInvalidValue;
        case 1 << 17: return a.scratch ? launch_split<16, 13>(a, rows, s) : cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t twiddle_table_launch(cdf* tw, int N, cudaStream_t s) {
    twiddle_table_kernel<<<(N + 255) / 256, 256, 0, s>>>(tw, N);
    return cudaGetLastError();
}

cudaError_t propagator_table_launch(cdf* E, const double* betas_dev, int rows, int row_stride, int N,
                                    double dt, double alpha, double z, size_t out_pitch, cudaStream_t s) {
    const size_t total = (size_t)rows * N;
    const int blocks = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    propagator_table_kernel<<<blocks, 256, 0, s>>>(E, betas_dev, rows, row_stride, N, dt, alpha, z, out_pitch);
    return cudaGetLastError();
}

cudaError_t amplify_launch(float2* A, float gain, const float2* noise, size_t n, cudaStream_t s) {
    const size_t blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
    amplify_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, s>>>(A, gain, noise, n);
    return cudaGetLastError();
}

cudaError_t slot_tick_launch(int* slot_steps, int n_slots, cudaStream_t s) {
    slot_tick_kernel<<<1, 128, 0, s>>>(slot_steps, n_slots);
    return cudaGetLastError();
}

}  // namespace mmf
