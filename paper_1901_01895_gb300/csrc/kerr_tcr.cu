// Kerr term of Eq. 1 on the 5th-generation tensor cores, one TMEM lane per (sample,
// pair quantity).
//
// Factorisation (exact for a fully symmetric S_plmn and the isotropic polarisation tensor):
//   u_ij = c_ij Re sum_a A_ia conj(A_ja),  v_ij = c_ij sum_a A_ia A_ja      (pairs i <= j, c = 2 off-diagonal)
//   W_pl = sum_(ij) S_plij u_ij,           Z_pl = sum_(ij) S_plij v_ij
//   K_(p,a) = (i gamma h / 3)[2 sum_l W_pl A_la + sum_l Z_pl conj(A_la)]   (2 pol)
//   K_p     = i gamma h sum_l Z_pl conj(A_l)                                (1 pol)
// S is block-diagonal over the parity classes par(i)^par(j) of the pairs.  Per sample tile
// and class this is one GEMM D[r][n] = sum_k X[r][k] B[n][k] with
//   rows r     = (sample, quantity): 3 rows per sample (u, Re v, Im v) for two
//                polarisations, 2 (Re v, Im v) for one.  A 32-row TMEM lane quarter holds 10
//                (or 16) samples, quantity-major (row_lane below); two rows of a quarter are
//                zero padding (2 pol),
//   K          = the input pairs (ij) of the class, 32 per chunk (64-byte swizzled rows),
//   columns n  = the output pairs of the class as UNORDERED pairs {p, l}: W and Z are
//                symmetric (S_plij = S_lpij), so one column serves both K_p (with A_l) and
//                K_l (with A_p), half the columns and MMAs of ordered pairs.  Columns are cut
//                into passes of at most 256; a pass is a list of segments {p in a p-list} x
//                {l in an l-list of at most 8 modes}, p-major,
//   B[n][k]    = S_plij c_ij w_pl, with w_pl = 1/2 on the columns of a square segment that
//                holds both orders of its pairs (and its diagonal), else 1; stored on the
//                device already in the canonical K-major 64-byte swizzled tile layout, one
//                bulk copy per (pass, chunk).
// Because each column needs one TMEM column (not one per quantity), a pass can be 256
// columns wide and two passes' accumulators fit in the 512 TMEM columns: the epilogue of
// one pass overlaps the MMAs of the next.
// BF16X3 splits both operands x = hi + lo in BF16 and accumulates hi*hi + hi*lo + lo*hi in
// FP32; BF16 uses hi*hi only.
//
// Warp roles (one CTA per SM, persistent over sample tiles):
//   epilogue    one or (two polarisations) two groups of four warps, warp w of a group = TMEM
//               lane quarter w.  Lane (s', q) reads its row of a segment's columns with
//               tcgen05.ld and contracts them with A(t) transformed for its quantity q: by rows
//               (over the l-list, held in registers, into K_p for each p of the p-list) and by
//               columns (over the p-list into K_l for each l, register sums).  Each mode's sums
//               of a pass belong to one group (the plan assigns the row and column sweeps of the
//               segments accordingly, the two groups doing about equal work), so the groups share
//               one accumulator K[p][t] in shared memory with a single writer per address; they
//               meet between passes.  The lanes of one sample are summed with shuffles and the
//               sum is added to the accumulator.  At the end of the tile the warps write
//               i * scale * K to HBM.
//   formation   per (pass, chunk) one thread per (sample, 16-byte atom of 8
//               pairs) forms the pair quantities from the staged fields, splits them into
//               BF16 hi/lo and stores them into the swizzled A stage.
//   MMA warp    one thread: waits for a chunk's pair products and S tile, issues the
//               tcgen05.mma instructions and commits their completion to mbarriers.
//   TMA warp    one thread: bulk copies of the S tiles, up to nb chunks ahead of the MMAs.
//               Keeping the copies off the MMA thread matters: tcgen05 instructions cost the
//               issuing thread ~100 cycles each, and with both duties on one thread the
//               tensor pipe waited on copy issue between chunks.
//   loader warp stages the next tile's fields x = in0 + c1 in1 in shared memory (two buffers
//               when they fit) while the current tile is contracted.
// Every wait is bounded (one second of %globaltimer); on timeout the kernel records a code
// in k.err, winds down, drains the MMAs and copies in flight and releases TMEM.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mmf {
namespace {

using namespace tc;

constexpr int KC_MAX = 32;             // pairs per K chunk: 32 BF16 or 16 TF32 values fill a row
constexpr int ROWB = 64;               // bytes per tile row, 64-byte swizzle
constexpr int KSTEPS = ROWB / 32;      // MMA k-steps per chunk (32 bytes of K each)
constexpr int A_TILE = 128 * ROWB;     // one 128-row split tile of a stage
constexpr int NEPI = 4;                // epilogue warps of a group (one per TMEM lane quarter)
constexpr int ACC_COLS = 256;          // TMEM columns per accumulator buffer
constexpr int BU_ROWS = 256;           // columns of the widest pass (one N <= 256 MMA per k-step)
constexpr int BH_ROWS = BU_ROWS / 2;   // rows of an S-tile stage: each CTA of a pair holds half of N
constexpr int NB_MAX = 4;              // S-tile stages
constexpr int NFB_MAX = 3;             // field buffers
constexpr int NDONE = 4;               // ring of chunk-done barriers (>= pair-product and S-tile stages)
static_assert((NDONE & (NDONE - 1)) == 0, "the issue loop indexes the ring with a mask");

template <int NPOL>
struct Geo {
    static constexpr int R = NPOL == 2 ? 3 : 2;        // rows per sample
    static constexpr int SPW = NPOL == 2 ? 10 : 16;    // samples per 32-lane quarter
    static constexpr int TS = 4 * SPW;                 // samples per tile
};
// Warp roles.  For two polarisations two epilogue groups of four warps share each pass: every
// mode's sums of the pass belong to one group (the plan's ownership), which sweeps the
// segments' rows or columns that produce them.
template <int NPOL, bool KG>
struct Roles {
    static constexpr int NGRP = NPOL == 2 ? 2 : 1;                       // epilogue groups
    static constexpr int NE = NEPI * NGRP;                               // epilogue warps
    static constexpr int NF = NPOL == 2 ? 5 : 8;                         // formation warps: TS * 4 units
    static constexpr int NTH = (NE + NF + 3) * 32;   // + MMA, S-tile producer and field loader warps
};

enum : int { ERR_A_EMPTY = 11, ERR_A_FULL, ERR_B_EMPTY, ERR_B_FULL, ERR_ACC_FULL, ERR_ACC_EMPTY, ERR_DRAIN,
             ERR_F_FULL, ERR_F_FREE, ERR_E_SYNC, ERR_PEER };

// Shared-memory carve-up (offsets from a 1024-byte aligned base); the host sizes the
// launch with the same function.
struct TcrLayout {
    size_t a, b, f, kacc, pairs, cls, pass, boff, seg, list, bars, total;
};
__host__ __device__ inline TcrLayout tcr_layout(int M, int n_pol, bool x3, bool kacc_global, int na, int nb, int nfb,
                                                int np_max, int n_pairs, int n_class, int n_pass, int n_seg, int n_list) {
    auto al = [](size_t v, size_t a) -> size_t { return (v + a - 1) / a * a; };
    const int nsplit = x3 ? 2 : 1;
    const int ts = n_pol == 2 ? Geo<2>::TS : Geo<1>::TS;
    const size_t fv = n_pol == 2 ? 16 : 8;
    TcrLayout L;
    L.a = 0;
    L.b = L.a + (size_t)na * nsplit * A_TILE;
    L.f = L.b + (size_t)nb * nsplit * BH_ROWS * ROWB;
    L.kacc = L.f + (size_t)nfb * M * ts * fv;
    L.pairs = L.kacc + (kacc_global ? 0 : (size_t)M * ts * fv);
    L.cls = al(L.pairs + (size_t)(n_pairs + n_class * (KC_MAX - 1)) * 2, 16);   // classes padded to whole chunks
    L.pass = al(L.cls + (size_t)(n_class + 1) * 4, 16);
    L.boff = L.pass + (size_t)n_pass * 16;
    L.seg = al(L.boff + (size_t)n_pass * 8, 16);
    L.list = L.seg + (size_t)n_seg * 16;
    L.bars = al(L.list + (size_t)n_list, 16);
    L.total = L.bars + 64 * 8 + 16;
    return L;
}

template <int NPOL>
using FV = typename std::conditional<NPOL == 2, float4, float2>::type;

// A_l(t) transformed for the lane's quantity q, so that every lane accumulates
// K += D[q] * At (four or two FMAs, no branch on q):
//   2 pol, A = (a0r, a0i, a1r, a1i): q=0 (W):  2 (a0r, a0i, a1r, a1i)
//                                    q=1 (Zr):   (a0r, -a0i, a1r, -a1i)
//                                    q=2 (Zi):   (a0i, a0r, a1i, a1r)
//   1 pol, A = (ar, ai):             q=0 (Zr):   (ar, -ai);  q=1 (Zi): (ai, ar)
struct LaneCoef {
    float al, be, ga, de;   // At.x = al*re + be*im, At.y = ga*im + de*re
};
__device__ __forceinline__ float4 xform(const float4& v, const LaneCoef& c) {
    return make_float4(fmaf(c.al, v.x, c.be * v.y), fmaf(c.ga, v.y, c.de * v.x), fmaf(c.al, v.z, c.be * v.w),
                       fmaf(c.ga, v.w, c.de * v.z));
}
__device__ __forceinline__ float2 xform(const float2& v, const LaneCoef& c) {
    return make_float2(fmaf(c.al, v.x, c.be * v.y), fmaf(c.ga, v.y, c.de * v.x));
}
// TMEM lane (row within the 32-row quarter w) of quantity q of the quarter's sample sp:
// quantity-major, rotated by 2w for two polarisations, so that the row is congruent mod 8 to
// the sample's index in the tile plus 2q.  Eight consecutive samples then sit on eight
// different rows mod 8, and the formation's 16-byte stores of eight consecutive samples
// into the 64-byte swizzled pair-product tile fall on eight different bank groups (with
// three rows per sample side by side they fell on as few as six).
template <int NPOL>
__device__ __forceinline__ int row_lane(int sp, int q, int w) {
    if constexpr (NPOL == 2) return (sp + 10 * q + 2 * w) & 31;
    else return sp + 16 * q;
}
// Sum of the quantities' contributions of a sample, left on its q = 0 lane, in two halves:
// lane_shuf issues the shuffles and lane_comb adds what they return, so that independent work
// (the previous output's store, the next accumulator load) can be placed between them.
template <int NPOL>
struct LaneShuf;
template <>
struct LaneShuf<2> {
    float2 a1, a2, b1, b2;
};
template <>
struct LaneShuf<1> {
    float x, y;
};
template <int NPOL>
__device__ __forceinline__ LaneShuf<NPOL> lane_shuf(const FV<NPOL>& k) {
    LaneShuf<NPOL> r;
    const unsigned m = 0xffffffffu;
    if constexpr (NPOL == 2) {
        // the sample's q = 1 and q = 2 rows are 10 and 20 lanes further on (mod 32)
        const int lane = threadIdx.x & 31, l1 = (lane + 10) & 31, l2 = (lane + 20) & 31;
        r.a1 = make_float2(__shfl_sync(m, k.x, l1), __shfl_sync(m, k.y, l1));
        r.a2 = make_float2(__shfl_sync(m, k.x, l2), __shfl_sync(m, k.y, l2));
        r.b1 = make_float2(__shfl_sync(m, k.z, l1), __shfl_sync(m, k.w, l1));
        r.b2 = make_float2(__shfl_sync(m, k.z, l2), __shfl_sync(m, k.w, l2));
    } else {
        r.x = __shfl_down_sync(m, k.x, 16);
        r.y = __shfl_down_sync(m, k.y, 16);
    }
    return r;
}
template <int NPOL>
__device__ __forceinline__ void lane_comb(FV<NPOL>& k, const LaneShuf<NPOL>& r) {
    if constexpr (NPOL == 2) {
        const float2 xy = __fadd2_rn(make_float2(k.x, k.y), __fadd2_rn(r.a1, r.a2));
        const float2 zw = __fadd2_rn(make_float2(k.z, k.w), __fadd2_rn(r.b1, r.b2));
        k = make_float4(xy.x, xy.y, zw.x, zw.y);
    } else {
        k.x += r.x;
        k.y += r.y;
    }
}
__device__ __forceinline__ void add_to(float4& a, const float4& b) {
    const float2 xy = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 zw = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
    a = make_float4(xy.x, xy.y, zw.x, zw.y);
}
__device__ __forceinline__ void add_to(float2& a, const float2& b) {
    a.x += b.x;
    a.y += b.y;
}
template <int NPOL>
__device__ __forceinline__ FV<NPOL> fv_zero() {
    if constexpr (NPOL == 2) return make_float4(0.f, 0.f, 0.f, 0.f);
    else return make_float2(0.f, 0.f);
}

__device__ __forceinline__ void red_add2(cf* p, float a, float b) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
// Shared-memory accesses by 32-bit shared address.  The field reads are plain loads (the
// buffer does not change while a segment is swept); the accumulator reads and writes are
// volatile, so that they stay in program order.
template <int NPOL>
__device__ __forceinline__ FV<NPOL> lds_field(uint32_t a) {
    FV<NPOL> v;
    if constexpr (NPOL == 2) asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    else asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
template <int NPOL>
__device__ __forceinline__ FV<NPOL> lds_acc(uint32_t a) {
    FV<NPOL> v;
    if constexpr (NPOL == 2)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    else asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
template <int NPOL>
__device__ __forceinline__ void sts_acc(uint32_t a, const FV<NPOL>& v) {
    if constexpr (NPOL == 2)
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
    else asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

// Where the epilogue adds a sample's contribution to K_p: the tile accumulator in shared
// memory (load, add, store), or (KG) i * sc * K_p straight into the output in global memory
// with vector reductions.  Within a pass each mode belongs to one epilogue group, and the
// groups meet between passes, so each address has one writer lane at a time, which adds in
// program order: either way the sum is formed in a fixed order.
template <int NPOL, bool KG>
struct EpiOut {
    uint32_t kacc;    // shared address of the lane's K[0][s] in the [M][TS] accumulator
    cf* out;          // (KG) &out[0][t], t the lane's sample
    int N;
    float sc;
    bool tvalid;
    __device__ __forceinline__ FV<NPOL> load(int p) const {
        if constexpr (!KG) return lds_acc<NPOL>(kacc + (uint32_t)(p * Geo<NPOL>::TS) * (uint32_t)sizeof(FV<NPOL>));
        else return fv_zero<NPOL>();
    }
    __device__ __forceinline__ void store(int p, FV<NPOL> old, const FV<NPOL>& kk) const {
        if constexpr (!KG) {
            add_to(old, kk);
            sts_acc<NPOL>(kacc + (uint32_t)(p * Geo<NPOL>::TS) * (uint32_t)sizeof(FV<NPOL>), old);
        } else if (tvalid) {
            if constexpr (NPOL == 2) {
                red_add2(out + (size_t)(2 * p) * N, -sc * kk.y, sc * kk.x);
                red_add2(out + (size_t)(2 * p + 1) * N, -sc * kk.w, sc * kk.z);
            } else {
                red_add2(out + (size_t)p * N, -sc * kk.y, sc * kk.x);
            }
        }
    }
};

// TMEM wait tied to the W (a multiple of 4, at most 24) registers of a segment row.
template <int W>
__device__ __forceinline__ void tmem_wait_w(uint32_t* r) {
    static_assert(W % 4 == 0 && W <= 24, "block registers");
    if constexpr (W >= 16) {
        tmem_wait16(r);
        if constexpr (W - 16 == 8) tmem_wait8(r + 16);
        else if constexpr (W - 16 == 4) tmem_wait4(r + 16);
    } else if constexpr (W == 12) {
        tmem_wait12(r);
    } else if constexpr (W == 8) {
        tmem_wait8(r);
    } else {
        tmem_wait4(r);
    }
}

// The two sweeps of a segment {p-list} x {l-list}: columns col .. col + n_p*NS - 1, p-major,
// l over the NS (<= 12) modes of the l-list.  Column (p, l) holds D = W_pl or Z_pl of the
// lane's quantity, symmetric in (p, l), and adds to both outputs:
//   rows:    K_p += sum_l D[p][l] T(A_l)   for each p of the p-list,
//   columns: K_l += T(sum_p D[p][l] A_p)   for each l of the l-list,
// T the lane's quantity transform (linear, so it is applied to the l-list's fields when the
// row sweep starts and to the column sums when the column sweep ends).  Each sweep reads the
// segment's TMEM columns once; a square segment (its p-list is its l-list, half weights) is
// swept both ways by one group.  All arithmetic is on packed FP32 pairs (fma.rn.f32x2) whose
// operands need no moves: columns 2h and 2h+1 of a TMEM load land in adjacent registers, and
// the l-list's fields and the column sums are held as pairs (component of l = 2h, of 2h+1).
// The TMEM load of the next p is issued before the arithmetic of the current.  (One
// instantiation per list length, fully unrolled.)
template <int NPOL, bool KG, int NS>
__device__ __noinline__ void epi_rows(uint32_t taddr, const uint8_t* __restrict__ ll, int n_p, uint32_t fs,
                                  EpiOut<NPOL, KG> eo, bool writer, LaneCoef lc) {
    constexpr int TS = Geo<NPOL>::TS;
    constexpr int NC = NPOL == 2 ? 4 : 2;        // float components of A(t)
    constexpr int NH = (NS + 1) / 2;             // pairs of l (an odd list's last pair padded with zero)
    constexpr int W = (NS + 3) / 4 * 4;          // registers of a TMEM row
    float2 Ap[NC][NH];                           // T(A_l), pairs over l
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const FV<NPOL> a = xform(lds_field<NPOL>(fs + (uint32_t)((int)ll[2 * h] * TS) * (uint32_t)sizeof(FV<NPOL>)), lc);
        const FV<NPOL> b = 2 * h + 1 < NS
                               ? xform(lds_field<NPOL>(fs + (uint32_t)((int)ll[2 * h + 1] * TS) * (uint32_t)sizeof(FV<NPOL>)), lc)
                               : fv_zero<NPOL>();
        Ap[0][h] = make_float2(a.x, b.x);
        Ap[1][h] = make_float2(a.y, b.y);
        if constexpr (NPOL == 2) {
            Ap[2 % NC][h] = make_float2(a.z, b.z);
            Ap[3 % NC][h] = make_float2(a.w, b.w);
        }
    }
    const uint8_t* pl = ll + NS;
    uint32_t d0[W], d1[W];                       // columns beyond NS stay zero
#pragma unroll
    for (int j = 0; j < W; ++j) d0[j] = d1[j] = 0u;
    // software pipeline over p: the shuffles of output ip are in flight while output ip - 1 is
    // stored and the accumulator of ip is read; ip's sum is stored after the FMAs of ip + 1
    FV<NPOL> kprev = fv_zero<NPOL>(), oprev = fv_zero<NPOL>();
    int pprev = 0;
    auto step = [&](const uint32_t* d, int ip) {
        float2 acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const float2 dd = make_float2(__uint_as_float(d[2 * h]), __uint_as_float(d[2 * h + 1]));
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = __ffma2_rn(dd, Ap[c][h], acc[c]);
        }
        FV<NPOL> kk;
        if constexpr (NPOL == 2)
            kk = make_float4(acc[0].x + acc[0].y, acc[1].x + acc[1].y, acc[2 % NC].x + acc[2 % NC].y,
                             acc[3 % NC].x + acc[3 % NC].y);
        else
            kk = make_float2(acc[0].x + acc[0].y, acc[1].x + acc[1].y);
        const LaneShuf<NPOL> sh = lane_shuf<NPOL>(kk);
        if (ip > 0 && writer) eo.store(pprev, oprev, kprev);
        const int p = (int)pl[ip];
        oprev = eo.load(p);
        lane_comb<NPOL>(kk, sh);
        kprev = kk;
        pprev = p;
    };
    tmem_ld_n<NS>(taddr, d0);
    tmem_wait_w<W>(d0);
    for (int ip = 0; ip < n_p; ip += 2) {
        const bool has1 = ip + 1 < n_p, has2 = ip + 2 < n_p;
        if (has1) tmem_ld_n<NS>(taddr + (uint32_t)((ip + 1) * NS), d1);
        step(d0, ip);
        if (has1) {
            tmem_wait_w<W>(d1);
            if (has2) tmem_ld_n<NS>(taddr + (uint32_t)((ip + 2) * NS), d0);
            step(d1, ip + 1);
            if (has2) tmem_wait_w<W>(d0);
        }
    }
    if (n_p > 0 && writer) eo.store(pprev, oprev, kprev);
}

template <int NPOL, bool KG, int NS>
__device__ __noinline__ void epi_cols(uint32_t taddr, const uint8_t* __restrict__ ll, int n_p, uint32_t fs,
                                  EpiOut<NPOL, KG> eo, bool writer, LaneCoef lc) {
    constexpr int TS = Geo<NPOL>::TS;
    constexpr int NC = NPOL == 2 ? 4 : 2;
    constexpr int NH = (NS + 1) / 2;
    constexpr int W = (NS + 3) / 4 * 4;
    float2 Lc[NC][NH];                           // sum_p D[p][l] A_p (untransformed), pairs over l
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int c = 0; c < NC; ++c) Lc[c][h] = make_float2(0.f, 0.f);
    const uint8_t* pl = ll + NS;
    uint32_t d0[W], d1[W];
#pragma unroll
    for (int j = 0; j < W; ++j) d0[j] = d1[j] = 0u;
    auto step = [&](const uint32_t* d, int ip) {
        const FV<NPOL> ap = lds_field<NPOL>(fs + (uint32_t)((int)pl[ip] * TS) * (uint32_t)sizeof(FV<NPOL>));
        float2 bc[NC];
        bc[0] = make_float2(ap.x, ap.x);
        bc[1] = make_float2(ap.y, ap.y);
        if constexpr (NPOL == 2) {
            bc[2 % NC] = make_float2(ap.z, ap.z);
            bc[3 % NC] = make_float2(ap.w, ap.w);
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const float2 dd = make_float2(__uint_as_float(d[2 * h]), __uint_as_float(d[2 * h + 1]));
#pragma unroll
            for (int c = 0; c < NC; ++c) Lc[c][h] = __ffma2_rn(dd, bc[c], Lc[c][h]);
        }
    };
    tmem_ld_n<NS>(taddr, d0);
    tmem_wait_w<W>(d0);
    for (int ip = 0; ip < n_p; ip += 2) {
        const bool has1 = ip + 1 < n_p, has2 = ip + 2 < n_p;
        if (has1) tmem_ld_n<NS>(taddr + (uint32_t)((ip + 1) * NS), d1);
        step(d0, ip);
        if (has1) {
            tmem_wait_w<W>(d1);
            if (has2) tmem_ld_n<NS>(taddr + (uint32_t)((ip + 2) * NS), d0);
            step(d1, ip + 1);
            if (has2) tmem_wait_w<W>(d0);
        }
    }
    // the NS outputs, two at a time: both pairs of shuffles and accumulator reads are in
    // flight together (the l-list's modes are distinct, so the reads and stores of one pair
    // touch different accumulators)
    auto raw = [&](int j) -> FV<NPOL> {
        if constexpr (NPOL == 2)
            return (j & 1) ? make_float4(Lc[0][j / 2].y, Lc[1][j / 2].y, Lc[2 % NC][j / 2].y, Lc[3 % NC][j / 2].y)
                           : make_float4(Lc[0][j / 2].x, Lc[1][j / 2].x, Lc[2 % NC][j / 2].x, Lc[3 % NC][j / 2].x);
        else
            return (j & 1) ? make_float2(Lc[0][j / 2].y, Lc[1][j / 2].y) : make_float2(Lc[0][j / 2].x, Lc[1][j / 2].x);
    };
#pragma unroll
    for (int j = 0; j < NS; j += 2) {
        const bool two = j + 1 < NS;
        FV<NPOL> ka = xform(raw(j), lc), kb = two ? xform(raw(j + 1), lc) : fv_zero<NPOL>();
        const LaneShuf<NPOL> sa = lane_shuf<NPOL>(ka);
        LaneShuf<NPOL> sb;
        if (two) sb = lane_shuf<NPOL>(kb);
        const int la = (int)ll[j], lb = two ? (int)ll[j + 1] : 0;
        const FV<NPOL> oa = eo.load(la);
        const FV<NPOL> ob = two ? eo.load(lb) : fv_zero<NPOL>();
        lane_comb<NPOL>(ka, sa);
        if (two) lane_comb<NPOL>(kb, sb);
        if (writer) {
            eo.store(la, oa, ka);
            if (two) eo.store(lb, ob, kb);
        }
    }
}

template <int NPOL, bool KG>
__device__ __forceinline__ void epi_dispatch(bool rows, int ns, uint32_t taddr, const uint8_t* ll, int n_p, uint32_t fs,
                                             const EpiOut<NPOL, KG>& eo, bool writer, const LaneCoef& lc) {
#define MMF_EPI_CASE(n)                                                     \
    case n:                                                                 \
        if (rows) epi_rows<NPOL, KG, n>(taddr, ll, n_p, fs, eo, writer, lc); \
        else epi_cols<NPOL, KG, n>(taddr, ll, n_p, fs, eo, writer, lc);      \
        break;
    switch (ns) {
        MMF_EPI_CASE(1) MMF_EPI_CASE(2) MMF_EPI_CASE(3) MMF_EPI_CASE(4) MMF_EPI_CASE(5) MMF_EPI_CASE(6)
        MMF_EPI_CASE(7) MMF_EPI_CASE(8) MMF_EPI_CASE(9) MMF_EPI_CASE(10) MMF_EPI_CASE(11) MMF_EPI_CASE(12)
        default: break;
    }
#undef MMF_EPI_CASE
}

// PREC: 0 BF16, 1 BF16x3, 2 TF32x3 (operands split into hi + lo, three products).
template <int NPOL, int PREC, bool KG>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Roles<NPOL, KG>::NTH, 1)
    kerr_tcr_kernel(KerrTCR k, const cf* __restrict__ in0, const cf* __restrict__ in1, float c1, cf* __restrict__ out,
                    float scale, int N) {
    using G = Geo<NPOL>;
    using V = FV<NPOL>;
    using RL = Roles<NPOL, KG>;
    constexpr int R = G::R, SPW = G::SPW, TS = G::TS, NF = RL::NF, NE = RL::NE, NGRP = RL::NGRP;
    constexpr bool X3 = PREC != 0, TF = PREC == 2;
    constexpr int NSPLIT = X3 ? 2 : 1;
    constexpr int KC = TF ? 16 : 32;                     // pairs per chunk (a 64-byte row of K)
    constexpr int PPA = KC / 4;                          // pairs per 16-byte atom of a row
    using CodeT = typename std::conditional<PPA == 8, uint4, uint2>::type;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int M = k.M, na = k.na, nb = k.nb, nfb = k.nfb;
    const TcrLayout L = tcr_layout(M, NPOL, X3, KG, na, nb, nfb, k.np_max, k.n_pairs, k.n_class, k.n_pass, k.n_seg,
                                   k.n_list);
    const uint32_t bslot = (uint32_t)BH_ROWS * ROWB;     // bytes of one split of an S-tile stage
    // CTA pairs: rank 0 (the leader) issues the pair's MMAs (M = 256: its 128 rows and the
    // peer's), each CTA stages its own sample tile's pair products and half of each S tile
    const uint32_t rank = cluster_ctarank();
    const int pair = (int)(blockIdx.x >> 1), n_pairs_grid = (int)(gridDim.x >> 1);
    uint8_t* A_s = base + L.a;                           // [na][NSPLIT][A_TILE]
    uint8_t* B_s = base + L.b;                           // [nb][NSPLIT][bslot]
    V* sF = reinterpret_cast<V*>(base + L.f);            // [nfb][M][TS]
    V* sK = reinterpret_cast<V*>(base + L.kacc);         // [M][TS] (not with KG)
    uint16_t* sP = reinterpret_cast<uint16_t*>(base + L.pairs);   // pair codes i | j << 8, classes padded to KC
    int* s_cls = reinterpret_cast<int*>(base + L.cls);
    int4* s_pass = reinterpret_cast<int4*>(base + L.pass);
    int64_t* s_boff = reinterpret_cast<int64_t*>(base + L.boff);
    int4* s_seg = reinterpret_cast<int4*>(base + L.seg);
    uint8_t* s_list = base + L.list;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bars);
    uint64_t* a_full = bars + 0;      // [4] the CTA's pair products formed and its S-tile half copied
    uint64_t* peer_full = bars + 30;  // [4] (leader) the same for the peer CTA, relayed by its MMA warp
    uint64_t* done = bars + 4;        // [NDONE] chunk c's MMAs complete: frees its A and S stages
    uint64_t* acc_full = bars + 16;   // [2]
    uint64_t* acc_empty = bars + 18;  // [2]
    uint64_t* f_full = bars + 34;     // [NFB_MAX] fields of a tile staged
    uint64_t* f_free = bars + 38;     // [NFB_MAX] formation and epilogue done with a field buffer
    uint64_t* drain = bars + 24;
    uint64_t* e_sync = bars + 25;     // the four epilogue warps
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 48);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 4; ++s) {
            mbar_init(a_full + s, NF + 1);   // the formation warps and the S-tile copy
            mbar_init(done + s, 1);
            mbar_init(peer_full + s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full + s, 1);
            mbar_init(acc_empty + s, 2 * NE);   // both CTAs' epilogue warps (the leader's copy is used)
        }
        for (int s = 0; s < NFB_MAX; ++s) {
            mbar_init(f_full + s, 1);
            mbar_init(f_free + s, NF + NE);
        }
        mbar_init(drain, 1);
        mbar_init(e_sync, NE);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // tables, zeroed A stages (the padding rows are never written) and accumulators
    // each class's pair list padded to a whole number of chunks with copies of its last pair
    // (their S rows are zero), so that a thread's eight codes are one aligned 16-byte load
    for (int c = 0, pbase = 0; c < k.n_class; ++c) {
        const int pb = k.cls_off[c], nc = k.cls_off[c + 1] - pb, npad = (nc + KC - 1) / KC * KC;
        for (int q = threadIdx.x; q < npad; q += RL::NTH) sP[pbase + q] = k.pairs[pb + (q < nc ? q : nc - 1)];
        pbase += npad;
    }
    for (int q = threadIdx.x; q <= k.n_class; q += RL::NTH) s_cls[q] = k.cls_off[q];
    for (int q = threadIdx.x; q < k.n_pass; q += RL::NTH) {
        s_pass[q] = k.passes[q];
        s_boff[q] = k.pass_boff[q];
    }
    for (int q = threadIdx.x; q < k.n_seg; q += RL::NTH) s_seg[q] = k.segs[q];
    for (int q = threadIdx.x; q < k.n_list; q += RL::NTH) s_list[q] = k.lists[q];
    {
        uint4* a4 = reinterpret_cast<uint4*>(A_s);
        const int n4 = na * NSPLIT * A_TILE / 16;
        for (int q = threadIdx.x; q < n4; q += RL::NTH) a4[q] = make_uint4(0u, 0u, 0u, 0u);
        if constexpr (!KG)
            for (int q = threadIdx.x; q < M * TS; q += RL::NTH) {
                if constexpr (NPOL == 2) sK[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                else sK[q] = make_float2(0.f, 0.f);
            }
    }
    fence_proxy_async();
    if (warp == 0) {
        // one warp of each CTA of the pair: the same 512 columns in both SMs' tensor memory
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist and TMEM is allocated before any signal crosses the pair
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_tiles = (N + TS - 1) / TS;
    const int n_ptiles = (n_tiles + 1) / 2;   // pair-tile pt: tile 2 pt for the leader, 2 pt + 1 for the peer
    const int n_pass = k.n_pass;
    // the pair's next pair-tile at or after pt that touches a request slot with steps left
    // (every pair-tile when the launch is not a request batch); all warp roles of both CTAs walk
    // the same list.  A tile beyond the last (odd tile count) is formed from zero fields and
    // writes nothing.
    auto live1 = [&](int t) { return t < n_tiles && tile_live(k.slot_steps, k.slot_len, t * TS, TS, N); };
    auto live_from = [&](int pt) {
        while (pt < n_ptiles && !live1(2 * pt) && !live1(2 * pt + 1)) pt += n_pairs_grid;
        return pt;
    };
    auto nkc_of = [&](int pass) {
        const int c = s_pass[pass].x;
        return (s_cls[c + 1] - s_cls[c] + KC - 1) / KC;
    };

    // chunks: (tile, pass, chunk kc); the MMA thread and the producer walk the same sequence
    struct It {
        int tile, pass, kc, nkc;
        bool valid;
    };
    auto it_init = [&](It& it) {
        it.tile = live_from(pair);
        it.pass = 0;
        it.kc = 0;
        it.valid = it.tile < n_ptiles;
        it.nkc = it.valid ? nkc_of(0) : 0;
    };
    auto it_next = [&](It& it) {
        if (++it.kc < it.nkc) return;
        it.kc = 0;
        if (++it.pass == n_pass) {
            it.pass = 0;
            it.tile = live_from(it.tile + n_pairs_grid);
            if (it.tile >= n_ptiles) {
                it.valid = false;
                return;
            }
        }
        it.nkc = nkc_of(it.pass);
    };

    if (warp == NE + NF + 1) {
        // ------------------------------------------- S-tile producer (TMA) ----
        // chunk jl's S tile (hi and, for BF16x3, lo split) goes to stage jl % nb once the MMAs
        // of chunk jl - nb, the stage's previous reader, are complete
        if (lane == 0) {
            It il;
            it_init(il);
            uint32_t jl = 0;
            while (il.valid) {
                const int s = (int)(jl % (uint32_t)nb);
                const int c = (int)jl - nb;
                if (c >= 0 && !mbar_wait(done + (c % NDONE), (uint32_t)(c / NDONE) & 1, k.err, ERR_B_EMPTY)) break;
                // a chunk's tiles are stored [rank][split][npad/2 rows]: this CTA's half, hi then lo
                const uint32_t half_bytes = (uint32_t)(s_pass[il.pass].y / 2) * ROWB;
                const uint8_t* src = k.B + s_boff[il.pass] + (int64_t)il.kc * 2 * NSPLIT * half_bytes +
                                     (int64_t)rank * NSPLIT * half_bytes;
                mbar_expect_tx(a_full + s, half_bytes * NSPLIT);
                bulk_g2s(B_s + (size_t)(s * NSPLIT + 0) * bslot, src, half_bytes, a_full + s);
                if (X3) bulk_g2s(B_s + (size_t)(s * NSPLIT + 1) * bslot, src + half_bytes, half_bytes, a_full + s);
                ++jl;
                it_next(il);
            }
            // copies still in flight land before the CTA exits (the last use of each stage)
            for (uint32_t j = jl > (uint32_t)nb ? jl - nb : 0u; j < jl; ++j)
                mbar_wait(a_full + (j % (uint32_t)nb), (j / nb) & 1, k.err, ERR_DRAIN);
        }
    } else if (warp == NE + NF) {
        // ---------------------------------------------------- MMA issuer ------
        // The whole warp runs the issue loop converged (its descriptors and counters are
        // warp-uniform values) and one elected lane issues each tcgen05 instruction.
        if (rank == 0) {
            It im;
            it_init(im);
            // The issue loop runs once per chunk next to the tensor pipe's work, so it avoids
            // divisions and rebuilds no descriptor: stage indices and phase bits advance
            // incrementally, and a stage's descriptor is the first stage's plus a constant
            // stride (the start-address field holds addr >> 4 in 14 bits, which every
            // shared-memory address fits).  The pair MMAs read A and B at the same shared
            // offsets in both CTAs.
            const uint64_t dA0 = sw_desc<ROWB>(smem_u32(A_s)), dB0 = sw_desc<ROWB>(smem_u32(B_s));
            constexpr uint32_t A_STEP = (NSPLIT * A_TILE) >> 4, A_LO = ((NSPLIT - 1) * A_TILE) >> 4;
            const uint32_t B_STEP = (NSPLIT * bslot) >> 4, B_LO = ((NSPLIT - 1) * bslot) >> 4;
            // jm: chunks consumed, e: passes done; (sa, pa): stage and phase parity (the
            // pair-product and S-tile rings have the same depth and advance together)
            uint32_t jm = 0, e = 0, sa = 0, pa = 0, idesc = 0;
            while (im.valid) {
                const uint32_t buf = e & 1;
                if (!warp_wait_u(a_full + sa, pa, k.err, ERR_A_FULL)) break;
                if (im.kc == 0) {
                    if (!warp_wait_u<true>(acc_empty + buf, ((e >> 1) & 1) ^ 1, k.err, ERR_ACC_EMPTY)) break;
                    idesc = idesc_pair<TF>(s_pass[im.pass].y);
                }
                if (!warp_wait_u<true>(peer_full + sa, pa, k.err, ERR_PEER)) break;
                tc_fence_after();
                const uint32_t d = tmem + buf * ACC_COLS;
                const uint64_t ah = dA0 + sa * A_STEP, bh = dB0 + sa * B_STEP;
                const bool last = im.kc == im.nkc - 1;
                if (elect_one()) {
#pragma unroll
                    for (int ks = 0; ks < KSTEPS; ++ks) {
                        const uint32_t o = ks * 2;   // 32 bytes further along K
                        mma_pair<TF>(d, ah + o, bh + o, idesc, (im.kc > 0 || ks > 0) ? 1u : 0u);
                        if (X3) {
                            mma_pair<TF>(d, ah + o, bh + B_LO + o, idesc, 1u);
                            mma_pair<TF>(d, ah + A_LO + o, bh + o, idesc, 1u);
                        }
                    }
                    // one commit, to both CTAs, frees the chunk's pair-product and S-tile stages
                    mma_commit_pair(done + (jm & (NDONE - 1)), 3);
                    if (last) mma_commit_pair(acc_full + buf, 3);
                }
                __syncwarp();
                if (last) ++e;
                ++jm;
                if (++sa == (uint32_t)na) sa = 0, pa ^= 1;
                it_next(im);
            }
            // drain: the MMAs in flight complete before TMEM is released
            if (jm > 0) {
                if (elect_one()) mma_commit_pair(drain, 1);
                __syncwarp();
                warp_wait_u(drain, 0, k.err, ERR_DRAIN);
            }
        } else if (lane == 0) {
            // peer: relay "this CTA's pair products and S half of the chunk are staged" to the
            // leader's peer_full barrier of the same stage (both CTAs walk the same chunks; a
            // stage is reused only after the leader's MMAs of its previous chunk completed, so
            // phases do not mix).  One thread relays: a release at cluster scope is costly, and
            // from every formation warp it slowed the kernel down.
            It im;
            it_init(im);
            const uint32_t peer_full0 = mapa_shared(smem_u32(peer_full), 0);
            uint32_t sa = 0, pa = 0;
            while (im.valid) {
                if (!mbar_wait(a_full + sa, pa, k.err, ERR_A_FULL)) break;
                mbar_arrive_remote(peer_full0 + 8u * sa);
                if (++sa == (uint32_t)na) sa = 0, pa ^= 1;
                it_next(im);
            }
        }
    } else if (warp == NE + NF + 2) {
        // ---------------------------------------------------- field loader ----
        // stages x = in0 + c1 in1 of the CTA's next tile in a free field buffer while the
        // formation and epilogue warps work on the current one; a late buffer stalls the
        // formation of the tile's first chunk, so the loads are 16 bytes wide where the
        // pointers allow and issued in batches
        const bool vec16 = (N & 1) == 0 && ((reinterpret_cast<uintptr_t>(in0) | reinterpret_cast<uintptr_t>(in1) |
                                              reinterpret_cast<uintptr_t>(out)) & 15) == 0;
        uint32_t ti = 0;
        for (int pt = live_from(pair); pt < n_ptiles; pt = live_from(pt + n_pairs_grid), ++ti) {
            const int tile = 2 * pt + (int)rank;
            const int fb = (int)(ti % (uint32_t)nfb);
            if (!warp_wait(f_free + fb, ((ti / nfb) & 1) ^ 1, k.err, ERR_F_FREE)) break;
            V* F = sF + (size_t)fb * M * TS;
            const int t0 = tile * TS;
            if (vec16) {
                // sample pairs (t, t + 1), t even: one 16-byte load per row and input, batches of
                // SU pairs per lane with all loads of a batch issued before the first is used
                constexpr int SU = 8, TS2 = TS / 2;
#pragma unroll 1
                for (int idx0 = lane; idx0 < M * TS2; idx0 += SU * 32) {
                    float4 v0[SU], v1[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int idx = idx0 + u * 32;
                        const int m = idx / TS2, t = t0 + 2 * (idx - m * TS2);
                        v0[u] = v1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (idx < M * TS2 && t < N) {   // N is even, so t + 1 < N too
                            const int r0 = NPOL == 2 ? 2 * m : m;
                            v0[u] = __ldg(reinterpret_cast<const float4*>(in0 + (size_t)r0 * N + t));
                            if constexpr (NPOL == 2) v1[u] = __ldg(reinterpret_cast<const float4*>(in0 + (size_t)(r0 + 1) * N + t));
                            if (in1) {
                                const float4 b0 = __ldg(reinterpret_cast<const float4*>(in1 + (size_t)r0 * N + t));
                                const float2 cc = make_float2(c1, c1);
                                float2 lo = __ffma2_rn(cc, make_float2(b0.x, b0.y), make_float2(v0[u].x, v0[u].y));
                                float2 hi = __ffma2_rn(cc, make_float2(b0.z, b0.w), make_float2(v0[u].z, v0[u].w));
                                v0[u] = make_float4(lo.x, lo.y, hi.x, hi.y);
                                if constexpr (NPOL == 2) {
                                    const float4 b1 = __ldg(reinterpret_cast<const float4*>(in1 + (size_t)(r0 + 1) * N + t));
                                    lo = __ffma2_rn(cc, make_float2(b1.x, b1.y), make_float2(v1[u].x, v1[u].y));
                                    hi = __ffma2_rn(cc, make_float2(b1.z, b1.w), make_float2(v1[u].z, v1[u].w));
                                    v1[u] = make_float4(lo.x, lo.y, hi.x, hi.y);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int idx = idx0 + u * 32;
                        if (idx >= M * TS2) break;
                        const int m = idx / TS2, tt = 2 * (idx - m * TS2), t = t0 + tt;
                        if constexpr (NPOL == 2) {
                            F[m * TS + tt] = make_float4(v0[u].x, v0[u].y, v1[u].x, v1[u].y);
                            F[m * TS + tt + 1] = make_float4(v0[u].z, v0[u].w, v1[u].z, v1[u].w);
                        } else {
                            F[m * TS + tt] = make_float2(v0[u].x, v0[u].y);
                            F[m * TS + tt + 1] = make_float2(v0[u].z, v0[u].w);
                        }
                        if constexpr (KG) {
                            if (t < N) {
                                const int r0 = NPOL == 2 ? 2 * m : m;
                                *reinterpret_cast<float4*>(out + (size_t)r0 * N + t) = make_float4(0.f, 0.f, 0.f, 0.f);
                                if constexpr (NPOL == 2)
                                    *reinterpret_cast<float4*>(out + (size_t)(r0 + 1) * N + t) = make_float4(0.f, 0.f, 0.f, 0.f);
                            }
                        }
                    }
                }
            } else {
                // batches of SU elements per lane, all loads of a batch issued before the first is
                // used (one global-memory latency per batch, not per element)
                constexpr int SU = 8;
#pragma unroll 1
                for (int idx0 = lane; idx0 < M * TS; idx0 += SU * 32) {
                    V v[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int idx = idx0 + u * 32;
                        const int m = idx / TS, t = t0 + idx - m * TS;
                        const bool ok = idx < M * TS && t < N;
                        if constexpr (NPOL == 2) {
                            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (ok) {
                                cf a0 = __ldg(in0 + (size_t)(2 * m) * N + t), a1 = __ldg(in0 + (size_t)(2 * m + 1) * N + t);
                                if (in1) {
                                    const cf b0 = __ldg(in1 + (size_t)(2 * m) * N + t),
                                             b1 = __ldg(in1 + (size_t)(2 * m + 1) * N + t);
                                    a0 = make_float2(fmaf(c1, b0.x, a0.x), fmaf(c1, b0.y, a0.y));
                                    a1 = make_float2(fmaf(c1, b1.x, a1.x), fmaf(c1, b1.y, a1.y));
                                }
                                v[u] = make_float4(a0.x, a0.y, a1.x, a1.y);
                            }
                        } else {
                            v[u] = make_float2(0.f, 0.f);
                            if (ok) {
                                v[u] = __ldg(in0 + (size_t)m * N + t);
                                if (in1) {
                                    const cf b = __ldg(in1 + (size_t)m * N + t);
                                    v[u] = make_float2(fmaf(c1, b.x, v[u].x), fmaf(c1, b.y, v[u].y));
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int idx = idx0 + u * 32;
                        if (idx >= M * TS) break;
                        F[idx] = v[u];
                        if constexpr (KG) {
                            const int m = idx / TS, t = t0 + idx - m * TS;
                            if (t < N) {
                                if constexpr (NPOL == 2) {
                                    out[(size_t)(2 * m) * N + t] = make_float2(0.f, 0.f);
                                    out[(size_t)(2 * m + 1) * N + t] = make_float2(0.f, 0.f);
                                } else {
                                    out[(size_t)m * N + t] = make_float2(0.f, 0.f);
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(f_full + fb);
        }
    } else if (warp >= NE) {
        // -------------------------------------------------- formation ---------
        // one thread per (sample s, 16-byte atom of 8 pairs)
        static_assert(TS * 4 == NF * 32, "one formation thread per (sample, atom)");
        const int ft = threadIdx.x - NE * 32;
        const int s = ft % TS, atom = ft / TS;
        const int qw = s / SPW, sp = s % SPW;
        uint32_t roff[R];   // byte offset of the thread's atom in the row of quantity q (swizzled tile)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int r = 32 * qw + row_lane<NPOL>(sp, q, qw);
            roff[q] = (uint32_t)((r >> 3) * 8 * ROWB + (r & 7) * ROWB + ((atom ^ ((r & 7) >> 1)) << 4));
        }
        uint32_t j = 0, ti = 0;
        bool abort_ = false;
        for (int pt = live_from(pair); pt < n_ptiles && !abort_; pt = live_from(pt + n_pairs_grid), ++ti) {
            const int fb = (int)(ti % (uint32_t)nfb);
            if (!warp_wait(f_full + fb, (ti / nfb) & 1, k.err, ERR_F_FULL)) break;
            const V* F = sF + (size_t)fb * M * TS;
            for (int pass = 0; pass < n_pass && !abort_; ++pass) {
                const int c = s_pass[pass].x;
                const int nkc = (s_cls[c + 1] - s_cls[c] + KC - 1) / KC;
                int cbase = 0;   // start of class c in the padded code table
                for (int c2 = 0; c2 < c; ++c2) cbase += (s_cls[c2 + 1] - s_cls[c2] + KC - 1) / KC * KC;
                const CodeT* codes = reinterpret_cast<const CodeT*>(sP + cbase) + atom;
#pragma unroll 1
                for (int kc = 0; kc < nkc; ++kc, ++j) {
                    const int slot = (int)(j % (uint32_t)na);
                    const int c = (int)j - na;   // the stage's previous chunk
                    if (c >= 0 && !warp_wait(done + (c % NDONE), (uint32_t)(c / NDONE) & 1, k.err, ERR_A_EMPTY)) {
                        abort_ = true;
                        break;
                    }
                    uint8_t* As = A_s + (size_t)slot * NSPLIT * A_TILE;
                    const CodeT cw = codes[kc * 4];
                    uint32_t cv[PPA / 2];
                    if constexpr (PPA == 8) {
                        cv[0] = cw.x; cv[1] = cw.y; cv[2 % (PPA / 2)] = cw.z; cv[3 % (PPA / 2)] = cw.w;
                    } else {
                        cv[0] = cw.x; cv[1] = cw.y;
                    }
                    int pi_[PPA], pj_[PPA];
#pragma unroll
                    for (int q = 0; q < PPA; ++q) {
                        const uint32_t ij = cv[q >> 1] >> ((q & 1) * 16);
                        pi_[q] = ij & 0xFF;
                        pj_[q] = (ij >> 8) & 0xFF;
                    }
                    float vals[R][PPA];
                    // pairs are ordered by i, so consecutive pairs mostly share A_i: it is
                    // read again only when i changes (fewer shared-memory wavefronts)
                    V ai = F[pi_[0] * TS + s];
#pragma unroll
                    for (int q = 0; q < PPA; ++q) {
                        if (q > 0 && pi_[q] != pi_[q - 1]) ai = F[pi_[q] * TS + s];
                        const V aj = F[pj_[q] * TS + s];
                        if constexpr (NPOL == 2) {
                            // (sum of the real-part products, sum of the imaginary-part products)
                            // over the two polarisations, on packed pairs: u is their sum, Re v
                            // their difference
                            const float2 pp = __ffma2_rn(make_float2(ai.x, ai.y), make_float2(aj.x, aj.y),
                                                         __fmul2_rn(make_float2(ai.z, ai.w), make_float2(aj.z, aj.w)));
                            vals[0][q] = pp.x + pp.y;
                            vals[1][q] = pp.x - pp.y;
                            vals[2][q] = fmaf(ai.x, aj.y, fmaf(ai.y, aj.x, fmaf(ai.z, aj.w, ai.w * aj.z)));
                        } else {
                            vals[0][q] = fmaf(ai.x, aj.x, -ai.y * aj.y);
                            vals[1][q] = fmaf(ai.x, aj.y, ai.y * aj.x);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        uint4 hi, lo;
                        if constexpr (TF) {
                            split_tf32(vals[q][0], hi.x, lo.x);
                            split_tf32(vals[q][1], hi.y, lo.y);
                            split_tf32(vals[q][2 % PPA], hi.z, lo.z);
                            split_tf32(vals[q][3 % PPA], hi.w, lo.w);
                            *reinterpret_cast<uint4*>(As + A_TILE + roff[q]) = lo;
                        } else if constexpr (X3) {
                            split_bf16(vals[q][0], vals[q][1], hi.x, lo.x);
                            split_bf16(vals[q][2], vals[q][3], hi.y, lo.y);
                            split_bf16(vals[q][4 % PPA], vals[q][5 % PPA], hi.z, lo.z);
                            split_bf16(vals[q][6 % PPA], vals[q][7 % PPA], hi.w, lo.w);
                            *reinterpret_cast<uint4*>(As + A_TILE + roff[q]) = lo;
                        } else {
                            hi.x = pack_bf16(vals[q][0], vals[q][1]);
                            hi.y = pack_bf16(vals[q][2], vals[q][3]);
                            hi.z = pack_bf16(vals[q][4 % PPA], vals[q][5 % PPA]);
                            hi.w = pack_bf16(vals[q][6 % PPA], vals[q][7 % PPA]);
                        }
                        *reinterpret_cast<uint4*>(As + roff[q]) = hi;
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(a_full + slot);
                }
            }
            if (abort_) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(f_free + fb);
        }
    } else {
        // --------------------------------------------------- epilogue ---------
        // the lane's (sample, quantity): the inverse of row_lane; the two padding lanes of a
        // two-polarisation quarter (rows of zeros) act as q = 0 lanes that never write
        const int qw = warp & 3, grp = warp >> 2;   // TMEM lane quarter, epilogue group
        int sp, q;
        if constexpr (NPOL == 2) {
            const int t = (lane - 2 * qw) & 31;
            sp = t < 30 ? t % 10 : SPW;
            q = t < 30 ? t / 10 : 0;
        } else {
            sp = lane & 15;
            q = lane >> 4;
        }
        const bool writer = q == 0 && sp < SPW;
        const int s = qw * SPW + (sp < SPW ? sp : SPW - 1);
        const uint32_t lane_base = tmem + ((uint32_t)(qw * 32) << 16);
        LaneCoef lc;
        if constexpr (NPOL == 2) {
            const float be = q == 2 ? 1.f : 0.f;
            lc = {q == 0 ? 2.f : (q == 1 ? 1.f : 0.f), be, q == 0 ? 2.f : (q == 1 ? -1.f : 0.f), be};
        } else {
            lc = q == 0 ? LaneCoef{1.f, 0.f, -1.f, 0.f} : LaneCoef{0.f, 1.f, 0.f, 1.f};
        }
        const float sc = NPOL == 2 ? scale / 3.f : scale;
        uint32_t e = 0, ti = 0, es = 0;
        bool abort_ = false;
        auto epi_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) mbar_arrive(e_sync);
            const bool ok = warp_wait(e_sync, es & 1, k.err, ERR_E_SYNC);
            ++es;
            return ok;
        };
        const uint32_t acc_empty0 = mapa_shared(smem_u32(acc_empty), 0);   // the leader's ring
        for (int pt = live_from(pair); pt < n_ptiles && !abort_; pt = live_from(pt + n_pairs_grid), ++ti) {
            const int tile = 2 * pt + (int)rank;
            const int fb = (int)(ti % (uint32_t)nfb);
            if (!warp_wait(f_full + fb, (ti / nfb) & 1, k.err, ERR_F_FULL)) break;
            const V* F = sF + (size_t)fb * M * TS;
            const int t_s = tile * TS + s;
            const EpiOut<NPOL, KG> eo = {smem_u32(sK + s), out + (t_s < N ? t_s : 0), N, sc, t_s < N && sp < SPW};
            const uint32_t fs = smem_u32(F + s);   // the lane's sample of field row 0
            for (int pass = 0; pass < n_pass; ++pass) {
                const uint32_t buf = e & 1;
                // a mode's sums may change owner from one pass to the next: both groups finish a
                // pass before either starts the next (at a tile's first pass the tile-end
                // synchronisation has done this, except with KG)
                if (NGRP > 1 && e > 0 && (KG || pass > 0) && !epi_sync()) {
                    abort_ = true;
                    break;
                }
                if (!warp_wait(acc_full + buf, (e >> 1) & 1, k.err, ERR_ACC_FULL)) {
                    abort_ = true;
                    break;
                }
                tc_fence_after();
                const int4 ps = s_pass[pass];
                const uint32_t tb = lane_base + buf * ACC_COLS;
                for (int g = ps.z; g < ps.w; ++g) {
                    const int4 sg = s_seg[g];
                    const int ns = sg.y & 0xFF;
                    if (((sg.y >> 8) & (NGRP - 1)) == grp)
                        epi_dispatch<NPOL, KG>(true, ns, tb + (uint32_t)sg.x, s_list + sg.w, sg.z, fs, eo, writer, lc);
                    if (((sg.y >> 9) & (NGRP - 1)) == grp)
                        epi_dispatch<NPOL, KG>(false, ns, tb + (uint32_t)sg.x, s_list + sg.w, sg.z, fs, eo, writer, lc);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(acc_empty0 + 8u * buf);   // the leader waits for both CTAs
                ++e;
            }
            if (abort_) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(f_free + fb);
            if constexpr (KG) continue;
            // every epilogue warp's sums are in sK: write i * sc * K and clear it for the next tile
            if (!epi_sync()) break;
            const int t0 = tile * TS;
#pragma unroll 1
            for (int idx = threadIdx.x; idx < M * TS; idx += NE * 32) {
                const int m = idx / TS, t = t0 + idx - m * TS;
                const V v = sK[idx];
                if constexpr (NPOL == 2) {
                    sK[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (t < N) {
                        out[(size_t)(2 * m) * N + t] = make_float2(-sc * v.y, sc * v.x);
                        out[(size_t)(2 * m + 1) * N + t] = make_float2(-sc * v.w, sc * v.z);
                    }
                } else {
                    sK[idx] = make_float2(0.f, 0.f);
                    if (t < N) out[(size_t)m * N + t] = make_float2(-sc * v.y, sc * v.x);
                }
            }
            if (!epi_sync()) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    // the leader's MMAs have drained, and neither CTA reads or signals the other any more
    cluster_sync();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

template <int NPOL, int PREC, bool KG>
cudaError_t launch_tcr(const KerrTCR& k, const float2* in0, const float2* in1, float c1, float2* out, float scale,
                       int N, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kerr_tcr_kernel<NPOL, PREC, KG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kerr_tcr_kernel<NPOL, PREC, KG><<<grid, Roles<NPOL, KG>::NTH, smem, s>>>(k, in0, in1, c1, out, scale, N);
    return cudaGetLastError();
}

}  // namespace

int kerr_tcr_tile_samples(int n_pol) { return n_pol == 2 ? Geo<2>::TS : Geo<1>::TS; }

size_t kerr_tcr_smem_bytes(const KerrTCR& k) {
    return 1024 + tcr_layout(k.M, k.n_pol, k.x3 != 0, k.kacc_global != 0, k.na, k.nb, k.nfb, k.np_max, k.n_pairs, k.n_class, k.n_pass,
                             k.n_seg, k.n_list)
                      .total;
}

cudaError_t kerr_tcr_launch(const KerrTCR& k, const float2* in0, const float2* in1, float c1, float2* out, float scale,
                            int N, int n_sm, cudaStream_t s) {
    if (k.na < 2 || k.na > NDONE || k.nb != k.na || k.nb > NB_MAX || k.nfb < 1 || k.nfb > NFB_MAX || k.np_max < 16 ||
        k.np_max > BU_ROWS)
        return cudaErrorInvalidValue;
    const size_t smem = kerr_tcr_smem_bytes(k);
    const int TS = kerr_tcr_tile_samples(k.n_pol);
    const int n_tiles = (N + TS - 1) / TS;
    const int n_ptiles = (n_tiles + 1) / 2;
    const int n_pairs = n_sm / 2 > 0 ? n_sm / 2 : 1;
    const int grid = 2 * (n_ptiles < n_pairs ? n_ptiles : n_pairs);   // clusters of two CTAs
#define MMF_TCR_LAUNCH(NP_, P_, KG_) launch_tcr<NP_, P_, KG_>(k, in0, in1, c1, out, scale, N, grid, smem, s)
#define MMF_TCR_KG(NP_, P_) (k.kacc_global ? MMF_TCR_LAUNCH(NP_, P_, true) : MMF_TCR_LAUNCH(NP_, P_, false))
    const int prec = k.tf32 ? 2 : (k.x3 ? 1 : 0);
    if (k.tf32 && !k.x3) return cudaErrorInvalidValue;
    if (k.n_pol == 2) return prec == 2 ? MMF_TCR_KG(2, 2) : prec == 1 ? MMF_TCR_KG(2, 1) : MMF_TCR_KG(2, 0);
    return prec == 2 ? MMF_TCR_KG(1, 2) : prec == 1 ? MMF_TCR_KG(1, 1) : MMF_TCR_KG(1, 0);
#undef MMF_TCR_KG
#undef MMF_TCR_LAUNCH
}

}  // namespace mmf
