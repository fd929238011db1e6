// C ABI of the RK4IP propagator (declared in include/mmf.h).
//
// One RK4IP step (Eq. 4a-4f) is eight launches over six field-sized scratch buffers:
//   Lin : A_I = Lin(A)                                       (4a)
//   Kerr: T   = Kerr(A)                 [T = h N(A)]
//   Lin : k1  = Lin(T)                                        (4b)
//   Kerr: k2  = Kerr(A_I + k1/2)                              (4c)
//   Kerr: k3  = Kerr(A_I + k2/2)                              (4d)
//   Lin : v   = Lin(A_I + k3)
//   Kerr: T   = Kerr(v)                 [= k4]                (4e)
//   Lin : A   = Lin(A_I + k1/6 + k2/3 + k3/3) + T/6           (4f)
// where Lin(x) = IFFT(exp(h/2 D) FFT(x)) and Kerr(x) = i gamma h sum Sfull x_l x_m conj(x_n).
// The stage combines are folded into the loads and stores of the kernels that
// consume or produce them.  A step is captured once per (fields pointer, h) as a
// CUDA graph and replayed n_steps times.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mmf.h"
#include "ctx.h"
#include "kernels.h"

using namespace mmf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(MMF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

}  // namespace

void mmf::set_last_error(const std::string& msg) { g_last_error = msg; }


namespace {

// Coefficients of the polarisation-resolved tensor: T = 1 (one polarisation) or
// (d_ab d_cd + d_ac d_bd + d_ad d_bc)/3 (two, isotropic).
double pol_tensor(int n_pol, int a, int b, int c, int d) {
    if (n_pol == 1) return 1.0;
    return ((a == b && c == d) + (a == c && b == d) + (a == d && b == c)) / 3.0;
}

// Build the folded (l <= m) term list of the Kerr sum per output field.
int build_term_list(mmf_ctx* h, const double* S) {
    const int M = h->M, np = h->n_pol, P = h->P;
    std::vector<int> off(P + 1, 0);
    std::vector<uint32_t> idx;
    std::vector<float> coef;
    std::vector<double> acc((size_t)P * P * P);
    for (int f = 0; f < P; ++f) {
        const int p = f / np, a = f % np;
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int l = 0; l < M; ++l)
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < M; ++n) {
                    const double s = S[(((size_t)p * M + l) * M + m) * M + n];
                    if (s == 0.0) continue;
                    for (int b = 0; b < np; ++b)
                        for (int c = 0; c < np; ++c)
                            for (int d = 0; d < np; ++d) {
                                const double T = pol_tensor(np, a, b, c, d);
                                if (T == 0.0) continue;
                                int lf = l * np + b, mf = m * np + c;
                                const int nf = n * np + d;
                                if (lf > mf) std::swap(lf, mf);
                                acc[((size_t)lf * P + mf) * P + nf] += s * T;
                            }
                }
        for (int lf = 0; lf < P; ++lf)
            for (int mf = lf; mf < P; ++mf)
                for (int nf = 0; nf < P; ++nf) {
                    const double v = acc[((size_t)lf * P + mf) * P + nf];
                    if (v == 0.0) continue;
                    idx.push_back((uint32_t)lf | ((uint32_t)mf << 10) | ((uint32_t)nf << 20));
                    coef.push_back((float)v);
                }
        off[f + 1] = (int)idx.size();
    }
    h->n_terms = (int)idx.size();
    CK(cudaMalloc(&h->d_term_off, sizeof(int) * (P + 1)));
    CK(cudaMalloc(&h->d_idx, sizeof(uint32_t) * std::max<size_t>(1, idx.size())));
    CK(cudaMalloc(&h->d_coef, sizeof(float) * std::max<size_t>(1, coef.size())));
    CK(cudaMemcpy(h->d_term_off, off.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    if (!idx.empty()) {
        CK(cudaMemcpy(h->d_idx, idx.data(), sizeof(uint32_t) * idx.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->d_coef, coef.data(), sizeof(float) * coef.size(), cudaMemcpyHostToDevice));
    }
    h->scratch_bytes += sizeof(int) * (P + 1) + (sizeof(uint32_t) + sizeof(float)) * idx.size();
    return MMF_OK;
}

// True if S is invariant under the transpositions (p l), (l m), (m n), which generate
// all 24 index permutations (relative tolerance 1e-12 of the largest entry).
bool fully_symmetric(const double* S, int M) {
    const size_t M4 = (size_t)M * M * M * M;
    double mx = 0.0;
    for (size_t i = 0; i < M4; ++i) mx = std::max(mx, std::fabs(S[i]));
    const double tol = 1e-12 * mx;
    auto at = [&](int p, int l, int m, int n) { return S[(((size_t)p * M + l) * M + m) * M + n]; };
    for (int p = 0; p < M; ++p)
        for (int l = 0; l < M; ++l)
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < M; ++n) {
                    const double v = at(p, l, m, n);
                    if (std::fabs(v - at(l, p, m, n)) > tol || std::fabs(v - at(p, m, l, n)) > tol ||
                        std::fabs(v - at(p, l, n, m)) > tol)
                        return false;
                }
    return true;
}

// Pair tables of the factored contraction: pairs (i <= j) grouped by the parity class
// par(i) ^ par(j), and per class the dense block S_pair[a][b] = S[i_a, j_a, i_b, j_b].
int build_pairs(mmf_ctx* h, const double* S, const int32_t* parity) {
    const int M = h->M;
    std::vector<int> par(M, 0);
    if (parity)
        for (int i = 0; i < M; ++i) par[i] = parity[i];
    std::vector<int> keys;
    for (int i = 0; i < M; ++i)
        for (int j = i; j < M; ++j) {
            const int c = par[i] ^ par[j];
            if (std::find(keys.begin(), keys.end(), c) == keys.end()) keys.push_back(c);
        }
    std::sort(keys.begin(), keys.end());
    h->n_class = (int)keys.size();
    h->cls_off.assign(h->n_class + 1, 0);
    h->pair_ij.clear();
    std::vector<float> pc;
    for (int ci = 0; ci < h->n_class; ++ci) {
        for (int i = 0; i < M; ++i)
            for (int j = i; j < M; ++j)
                if ((par[i] ^ par[j]) == keys[ci]) {
                    h->pair_ij.push_back(make_int2(i, j));
                    pc.push_back(i == j ? 1.f : 2.f);
                }
        h->cls_off[ci + 1] = (int)h->pair_ij.size();
    }
    h->S_off.assign(h->n_class, 0);
    int64_t total = 0;
    for (int ci = 0; ci < h->n_class; ++ci) {
        h->S_off[ci] = total;
        const int64_t nc = h->cls_off[ci + 1] - h->cls_off[ci];
        total += nc * nc;
    }
    std::vector<float> Sp((size_t)std::max<int64_t>(total, 1));
    for (int ci = 0; ci < h->n_class; ++ci) {
        const int b0 = h->cls_off[ci], nc = h->cls_off[ci + 1] - b0;
        float* blk = Sp.data() + h->S_off[ci];
        for (int a = 0; a < nc; ++a) {
            const int2 pa = h->pair_ij[b0 + a];
            for (int b = 0; b < nc; ++b) {
                const int2 pb = h->pair_ij[b0 + b];
                blk[(size_t)a * nc + b] = (float)S[(((size_t)pa.x * M + pa.y) * M + pb.x) * M + pb.y];
            }
        }
    }
    const size_t np = h->pair_ij.size();
    CK(cudaMalloc(&h->d_cls_off, sizeof(int) * (h->n_class + 1)));
    CK(cudaMalloc(&h->d_pair_ij, sizeof(int2) * np));
    CK(cudaMalloc(&h->d_pair_c, sizeof(float) * np));
    CK(cudaMalloc(&h->d_S_pair, sizeof(float) * Sp.size()));
    CK(cudaMalloc(&h->d_S_off, sizeof(int64_t) * h->n_class));
    CK(cudaMemcpy(h->d_cls_off, h->cls_off.data(), sizeof(int) * (h->n_class + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_pair_ij, h->pair_ij.data(), sizeof(int2) * np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_pair_c, pc.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_S_pair, Sp.data(), sizeof(float) * Sp.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_S_off, h->S_off.data(), sizeof(int64_t) * h->n_class, cudaMemcpyHostToDevice));
    h->scratch_bytes += sizeof(float) * Sp.size() + (sizeof(int2) + sizeof(float)) * np;
    return MMF_OK;
}

uint16_t bf16_bits(double v) {
    float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
// Byte offset of (row, k) in a [rows x sw/esz] tile of esz-byte elements, K-major with rows of
// sw bytes swizzled the canonical way: the 16-byte chunk index is XORed with (row mod 8) >>
// log2(128/sw) (address bits [4, 4+log2(sw/16)) XOR bits [7, ...)); 8-row groups 8*sw bytes apart.
size_t sw_byte(int sw, int row, int k, int esz) {
    const int shift = sw == 128 ? 0 : (sw == 64 ? 1 : 2), per = 16 / esz;
    return (size_t)(row >> 3) * 8 * sw + (row & 7) * sw + (size_t)(((k / per) ^ ((row & 7) >> shift)) << 4) +
           (size_t)(k % per) * esz;
}
// TF32 bit pattern of v (FP32 with the low 13 mantissa bits cleared), rounded to nearest with
// ties away from zero on the FP32 value; finite inputs only.
uint32_t tf32_bits(double v) {
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u + 0x1000u) & 0xFFFFE000u;
}
double tf32_value(uint32_t b) {
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

// Column plan of the row-triplet tensor-core path for pass width np_max.  W_pl and Z_pl are
// symmetric in (p, l) (S_plij = S_lpij), so every unordered output pair is one column and the
// epilogue adds its contribution to both K_p (with A_l) and K_l (with A_p).  Per class c:
//   - bucket pairs (X, Y), X < Y, X ^ Y = key(c): segments {p in X} x {l in a sub-list of Y of
//     at most 8 modes}, every column once;
//   - a bucket paired with itself (key 0): the bucket cut into sub-lists L_1..L_k of at most 8
//     modes; segment b is {p in L_1 .. L_b} x {l in L_b}, in which the square L_b x L_b holds
//     both orders of its pairs and its diagonal, so those columns carry half weight;
// segments cut to at most np_max columns and packed first-fit (widest first) into passes.
struct TcrPlan {
    std::vector<int4> passes;                 // {class, npad, seg_begin, seg_end}
    std::vector<int4> segs;                   // {col, n_l | own_p << 8 | own_l << 9, n_p, list_off}
    std::vector<uint8_t> lists;
    std::vector<std::vector<int2>> cols;      // per pass: (p, l) of each column
    std::vector<std::vector<float>> colw;     // per pass: weight of each column (1 or 1/2)
};
constexpr int TCR_NS_MAX = 12;                // l-list length of a segment (epilogue registers)
// Passes and segments of the tensor-core Kerr.  The epilogue's two warp groups share one
// accumulator per (mode, sample); within a pass every mode's sums belong to one group (its
// owner), so each address has a single writer and a fixed order of additions.  A segment
// {p-list} x {l-list} is swept by rows (K_p for the p-list) by the owner of its p-list and by
// columns (K_l for the l-list) by the owner of its l-list:
//   - a block of two different parity buckets X x Y: X owned by group 0, Y by group 1, so the
//     row and column sweeps of every segment (the same work) go to different groups;
//   - a diagonal block X x X: X (from 8 modes on) cut into k >= 2 sub-lists L_1..L_k with
//     alternating owners, one segment per (L_j, L_i), j <= i; the square ones (j = i, half
//     weights) are swept both ways by their owner.
TcrPlan plan_tcr(int M, const std::vector<int>& par, const std::vector<int>& ckey, int np_max) {
    std::vector<int> keys;
    for (int i = 0; i < M; ++i)
        if (std::find(keys.begin(), keys.end(), par[i]) == keys.end()) keys.push_back(par[i]);
    std::sort(keys.begin(), keys.end());
    auto bucket = [&](int pv) {
        std::vector<int> b;
        for (int i = 0; i < M; ++i)
            if (par[i] == pv) b.push_back(i);
        return b;
    };
    auto split_k = [](const std::vector<int>& v, int k) {
        std::vector<std::vector<int>> out;
        const int n = (int)v.size();
        for (int i = 0; i < k; ++i)
            out.emplace_back(v.begin() + (size_t)i * n / k, v.begin() + (size_t)(i + 1) * n / k);
        return out;
    };
    struct Seg {
        std::vector<int> ls, ps;
        int width, own_p, own_l;
    };
    TcrPlan pl;
    for (int c = 0; c < (int)ckey.size(); ++c) {
        std::vector<Seg> sg;
        auto add_segs = [&](const std::vector<int>& ps_all, const std::vector<int>& ls, int own_p, int own_l) {
            const int maxp = std::max(1, np_max / (int)ls.size());
            for (size_t p0 = 0; p0 < ps_all.size(); p0 += maxp) {
                Seg g;
                g.ls = ls;
                g.ps.assign(ps_all.begin() + p0, ps_all.begin() + std::min(ps_all.size(), p0 + maxp));
                g.width = (int)(g.ls.size() * g.ps.size());
                g.own_p = own_p;
                g.own_l = own_l;
                sg.push_back(g);
            }
        };
        int diag = 0;
        for (int q : keys) {
            const int qp = q ^ ckey[c];
            if (std::find(keys.begin(), keys.end(), qp) == keys.end() || qp < q) continue;
            const std::vector<int> X = bucket(q), Y = bucket(qp);
            if (qp != q) {
                const int k = ((int)Y.size() + TCR_NS_MAX - 1) / TCR_NS_MAX;
                for (const auto& ls : split_k(Y, k)) add_segs(X, ls, 0, 1);
            } else {
                // small buckets stay whole: one square segment, swept both ways by one group (the
                // owners alternate between diagonal blocks); tiny segments cost more than they balance
                const int k = std::max((int)X.size() >= 8 ? 2 : 1, ((int)X.size() + TCR_NS_MAX - 1) / TCR_NS_MAX);
                const auto L = split_k(X, k);
                for (int i = 0; i < k; ++i)
                    for (int j = 0; j <= i; ++j) add_segs(L[j], L[i], (j + diag) & 1, (i + diag) & 1);
                ++diag;
            }
        }
    std::stable_sort(sg.begin(), sg.end(), [](const Seg& a, const Seg& b) { return a.width > b.width; });
        std::vector<std::vector<int>> bins;
        std::vector<int> used;
        for (int g = 0; g < (int)sg.size(); ++g) {
            size_t b = 0;
            while (b < bins.size() && used[b] + sg[g].width > np_max) ++b;
            if (b == bins.size()) {
                bins.emplace_back();
                used.push_back(0);
            }
            bins[b].push_back(g);
            used[b] += sg[g].width;
        }
        for (size_t b = 0; b < bins.size(); ++b) {
            const int seg0 = (int)pl.segs.size();
            std::vector<int2> cols;
            std::vector<float> w;
            for (int g : bins[b]) {
                const Seg& S_ = sg[g];
                pl.segs.push_back(make_int4((int)cols.size(), (int)S_.ls.size() | S_.own_p << 8 | S_.own_l << 9,
                                            (int)S_.ps.size(), (int)pl.lists.size()));
                for (int l : S_.ls) pl.lists.push_back((uint8_t)l);
                for (int p : S_.ps) pl.lists.push_back((uint8_t)p);
                for (int p : S_.ps) {
                    const bool in_ls = std::find(S_.ls.begin(), S_.ls.end(), p) != S_.ls.end();
                    for (int l : S_.ls) {
                        cols.push_back(make_int2(p, l));
                        w.push_back(in_ls ? 0.5f : 1.0f);
                    }
                }
            }
            const int npad = ((int)cols.size() + 15) / 16 * 16;
            pl.passes.push_back(make_int4(c, npad, seg0, (int)pl.segs.size()));
            pl.cols.push_back(cols);
            pl.colw.push_back(w);
        }
    }
    // Pass order: the passes of the diagonal class (square segments, swept both ways by one
    // group: the most epilogue work per column) between the others, so that the epilogue,
    // which runs one pass behind the MMAs, catches up during a lighter pass.
    std::vector<int> zq, oq, order;
    for (int q = 0; q < (int)pl.passes.size(); ++q) (ckey[pl.passes[q].x] == 0 ? zq : oq).push_back(q);
    for (size_t iz = 0, io = 0; iz < zq.size() || io < oq.size();) {
        if (io < oq.size()) order.push_back(oq[io++]);
        if (iz < zq.size()) order.push_back(zq[iz++]);
    }
    TcrPlan out;
    out.segs = std::move(pl.segs);
    out.lists = std::move(pl.lists);
    for (int q : order) {
        out.passes.push_back(pl.passes[q]);
        out.cols.push_back(std::move(pl.cols[q]));
        out.colw.push_back(std::move(pl.colw[q]));
    }
    return out;
}

// Tables of the row-triplet tensor-core pair contraction (needs build_pairs first).
int build_tcr(mmf_ctx* h, const double* S, const int32_t* parity, bool x3, bool tf32) {
    const int M = h->M, C = h->n_class, KCH = tf32 ? 16 : 32, ESZ = tf32 ? 4 : 2;
    const int n_pairs = (int)h->pair_ij.size();
    if (M > 255) return fail(MMF_EINVAL, "the tensor-core Kerr path supports at most 255 spatial modes");
    std::vector<int> par(M, 0);
    if (parity)
        for (int i = 0; i < M; ++i) par[i] = parity[i];
    std::vector<int> ckey(C);
    for (int c = 0; c < C; ++c) {
        const int2 pr = h->pair_ij[h->cls_off[c]];
        ckey[c] = par[pr.x] ^ par[pr.y];
    }
    // Stage counts and pass width: the widest pass that fits (fewer formations of the pair
    // products), then the deepest rings that fit: a chunk's round trip (formation, hand-over to
    // the MMA thread, MMAs, completion back to both CTAs) is ~5k cycles, so two stages leave
    // the tensor pipe idle (measured at 45 modes, BF16x3: two stages 1.30 ms, three 1.16 ms,
    // four 1.13 ms; with 16-byte field loads two field buffers are enough).  The pair-product
    // and S-tile rings have the same depth: one barrier per stage collects both.  Each CTA of
    // a pair holds half of every S tile (8 KB per split); the fields of a 40-sample tile
    // (M x 640 B per buffer) decide what fits.
    KerrTCR k = {};
    k.M = M;
    k.n_pol = h->n_pol;
    k.n_class = C;
    k.n_pairs = n_pairs;
    k.x3 = x3 ? 1 : 0;
    k.tf32 = tf32 ? 1 : 0;
    TcrPlan plan;
    bool found = false;
    struct Cand {
        int na, nb, nfb, kg;
    };
    const Cand cands[] = {{4, 4, 3, 0}, {4, 4, 2, 0}, {3, 3, 3, 0}, {3, 3, 2, 0}, {2, 2, 3, 0}, {2, 2, 2, 0},
                          {4, 4, 2, 1}, {3, 3, 2, 1}, {2, 2, 2, 1}, {4, 4, 1, 0}, {3, 3, 1, 0}, {2, 2, 1, 0},
                          {4, 4, 1, 1}, {3, 3, 1, 1}, {2, 2, 1, 1}};
    const int np_floor[] = {256, 192, 128, 64, 16};
    for (int fl : np_floor) {
        for (const Cand& cd : cands) {
            for (int np = 256; np >= fl && !found; np -= 16) {
                TcrPlan p = plan_tcr(M, par, ckey, np);
                k.na = cd.na;
                k.nb = cd.nb;
                k.nfb = cd.nfb;
                k.kacc_global = cd.kg;
                k.np_max = np;
                k.n_pass = (int)p.passes.size();
                k.n_seg = (int)p.segs.size();
                k.n_list = (int)p.lists.size();
                if (kerr_tcr_smem_bytes(k) <= 227 * 1024) {
                    plan = std::move(p);
                    found = true;
                }
            }
            if (found) break;
        }
        if (found) break;
    }
    if (!found) return fail(MMF_EINVAL, "tensor-core Kerr: the fields of a sample tile do not fit in shared memory");
    const int nsplit = x3 ? 2 : 1;
    std::vector<int64_t> boff(plan.passes.size());
    int64_t bbytes = 0;
    for (size_t q = 0; q < plan.passes.size(); ++q) {
        const int c = plan.passes[q].x, npad = plan.passes[q].y;
        const int nkc = (h->cls_off[c + 1] - h->cls_off[c] + KCH - 1) / KCH;
        boff[q] = bbytes;
        bbytes += (int64_t)nkc * nsplit * npad * 64;
    }
    // per (pass, chunk) the S tile is stored [rank][split][npad/2 rows x 64 B]: CTA rank r of a
    // pair holds columns r*npad/2 .. (r+1)*npad/2 - 1 of the pass (the N half of the pair MMA)
    std::vector<uint8_t> B((size_t)std::max<int64_t>(bbytes, 16), 0);
    for (size_t q = 0; q < plan.passes.size(); ++q) {
        const int c = plan.passes[q].x, npad = plan.passes[q].y;
        const int pb = h->cls_off[c], nc = h->cls_off[c + 1] - pb;
        const size_t half = (size_t)(npad / 2) * 64;
        for (size_t n = 0; n < plan.cols[q].size(); ++n) {
            const int p = plan.cols[q][n].x, l = plan.cols[q][n].y;
            const int rk = (int)n / (npad / 2), row = (int)n % (npad / 2);
            const double wcol = plan.colw[q][n];
            for (int kidx = 0; kidx < nc; ++kidx) {
                const int2 ij = h->pair_ij[pb + kidx];
                // the pair fold factor c_ij (2 off the diagonal) and the column weight (1/2 where
                // both orders of (p, l) are columns) are carried by the S tile
                const double v =
                    S[(((size_t)p * M + l) * M + ij.x) * M + ij.y] * (ij.x == ij.y ? 1.0 : 2.0) * wcol;
                uint8_t* t0 = B.data() + boff[q] + (size_t)(kidx / KCH) * 2 * nsplit * half + (size_t)rk * nsplit * half;
                const size_t o = sw_byte(64, row, kidx % KCH, ESZ);
                if (tf32) {
                    const uint32_t hb = tf32_bits(v), lb = tf32_bits(v - tf32_value(hb));
                    std::memcpy(t0 + o, &hb, 4);
                    if (x3) std::memcpy(t0 + half + o, &lb, 4);
                } else {
                    const uint16_t hb = bf16_bits(v), lb = bf16_bits(v - bf16_value(hb));
                    std::memcpy(t0 + o, &hb, 2);
                    if (x3) std::memcpy(t0 + half + o, &lb, 2);
                }
            }
        }
    }
    std::vector<uint16_t> pk(n_pairs);
    for (int q = 0; q < n_pairs; ++q) pk[q] = (uint16_t)(h->pair_ij[q].x | (h->pair_ij[q].y << 8));
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_cls = 0, o_pairs = o_cls + al(sizeof(int) * (C + 1));
    const size_t o_pass = o_pairs + al(2 * std::max(1, n_pairs));
    const size_t o_boff = o_pass + al(sizeof(int4) * plan.passes.size());
    const size_t o_seg = o_boff + al(sizeof(int64_t) * boff.size());
    const size_t o_list = o_seg + al(sizeof(int4) * plan.segs.size());
    const size_t o_B = o_list + al(std::max<size_t>(1, plan.lists.size()));
    const size_t total = o_B + al(B.size());
    if (cudaMalloc(&h->d_tc_blob, total) != cudaSuccess) return fail(MMF_ENOMEM, "tensor-core table allocation failed");
    uint8_t* d = (uint8_t*)h->d_tc_blob;
    CK(cudaMemcpy(d + o_cls, h->cls_off.data(), sizeof(int) * (C + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d + o_pairs, pk.data(), 2 * (size_t)n_pairs, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d + o_pass, plan.passes.data(), sizeof(int4) * plan.passes.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d + o_boff, boff.data(), sizeof(int64_t) * boff.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d + o_seg, plan.segs.data(), sizeof(int4) * plan.segs.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d + o_list, plan.lists.data(), plan.lists.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d + o_B, B.data(), B.size(), cudaMemcpyHostToDevice));
    h->scratch_bytes += total;
    k.cls_off = (const int*)(d + o_cls);
    k.pairs = (const uint16_t*)(d + o_pairs);
    k.passes = (const int4*)(d + o_pass);
    k.pass_boff = (const int64_t*)(d + o_boff);
    k.segs = (const int4*)(d + o_seg);
    k.lists = d + o_list;
    k.B = d + o_B;
    k.err = h->d_err;
    h->tcr = k;
    return MMF_OK;
}

void free_ctx(mmf_ctx* h) {
    if (!h) return;
    if (h->device >= 0) cudaSetDevice(h->device);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->io_stream) {
        cudaStreamDestroy(h->io_stream);
        for (cudaEvent_t ev : h->io_ev) if (ev) cudaEventDestroy(ev);
        for (cudaEvent_t ev : h->io_ev_out) if (ev) cudaEventDestroy(ev);
    }
    cudaFree(h->d_betas);
    cudaFree(h->d_tw);
    cudaFree(h->d_E);
    cudaFree(h->d_Elin);
    for (auto& b : h->buf) cudaFree(b);
    cudaFree(h->d_linscratch);
    cudaFree(h->d_io);
    cudaFree(h->d_term_off);
    cudaFree(h->d_idx);
    cudaFree(h->d_coef);
    cudaFree(h->d_cls_off);
    cudaFree(h->d_pair_ij);
    cudaFree(h->d_pair_c);
    cudaFree(h->d_S_pair);
    cudaFree(h->d_S_off);
    cudaFree(h->d_tc_blob);
    cudaFree(h->d_kappa);
    cudaFree(h->d_kappa_tc);
    cudaFree(h->d_err);
    cudaFree(h->d_epart);
    cudaFree(h->d_eout);
    delete h;
}

int ensure_E(mmf_ctx* h, float4** table, double* table_z, double z) {
    if (*table_z == z) return MMF_OK;
    if (!*table) {
        cudaError_t e = cudaMalloc(table, sizeof(float4) * (size_t)h->e_rows * h->N);
        if (e != cudaSuccess) return fail(MMF_ENOMEM, "propagator table allocation failed");
    }
    CK(propagator_table_launch(*table, h->d_betas, h->e_rows, 1 << h->e_shift, h->N, h->dt, h->alpha, z, (size_t)h->N,
                               h->stream));
    *table_z = z;
    return MMF_OK;
}

cudaError_t kerr_eval(mmf_ctx* h, const float2* in0, const float2* in1, float in1_coef, float2* out, float scale,
                      cudaStream_t s) {
    KerrIO io = {};
    io.in0 = in0;
    io.in1 = in1;
    io.in1_coef = in1_coef;
    io.out = out;
    io.slot_steps = h->d_slot_steps;
    io.slot_len = h->N;
    if (h->kerr_path == 0) {
        KerrList k = {h->d_term_off, h->d_idx, h->d_coef, h->P};
        return kerr_list_launch(k, io, scale, h->Nk, s);
    }
    if (h->kerr_path == 4) {
        KerrKappa k = {h->P, h->d_kappa};
        return kerr_kappa_launch(k, io, scale, h->Nk, h->n_sm, s);
    }
    if (h->kerr_path == 5) return kerr_kappa_tc_launch(h->ktc, in0, in1, in1_coef, out, scale, h->Nk, h->n_sm, s);
    if (h->kerr_path == 3) {
        KerrTCR k = h->tcr;
        k.slot_steps = h->d_slot_steps;
        k.slot_len = h->N;
        return kerr_tcr_launch(k, in0, in1, in1_coef, out, scale, h->Nk, h->n_sm, s);
    }
    KerrPairs k = {h->M, h->n_pol, h->n_class, h->d_cls_off, h->d_pair_ij, h->d_pair_c, h->d_S_pair, h->d_S_off};
    return kerr_pairs_simt_launch(k, io, scale, h->Nk, s);
}

LinArgs lin_args(mmf_ctx* h, const float4* E) {
    LinArgs a = {};
    a.E = E;
    a.e_shift = h->e_shift;
    a.tw = h->d_tw;
    a.e_batch = h->batch;
    a.slot_steps = h->d_slot_steps;
    a.scratch = h->d_linscratch;
    a.n_sm = h->n_sm;
    return a;
}

// One symmetric split step with a classic RK4 nonlinear step (SSFM-RK4, Section 3.1):
//   u = E A;  k1 = h N(u);  k2 = h N(u + k1/2);  k3 = h N(u + k2/2);  k4 = h N(u + k3);
//   A = E (u + k1/6 + k2/3 + k3/3 + k4/6),   E = exp(h/2 L).
// Six launches: the final combine is folded into the load of the second linear step.
cudaError_t enqueue_ssfm_rk4_step(mmf_ctx* h, float2* A, double hstep, cudaStream_t s) {
    float2 *u = h->buf[0], *k1 = h->buf[1], *k2 = h->buf[2], *k3 = h->buf[3], *k4 = h->buf[5];
    const float ksc = (float)(h->gamma * hstep);
    const int P = h->P * h->batch, N = h->N;
    cudaError_t e;
    LinArgs a = lin_args(h, h->d_E);
    a.in[0] = A; a.coef[0] = 1.f; a.n_in = 1; a.add = nullptr; a.out = u;
    if ((e = lin_launch(a, P, N, s)) != cudaSuccess) return e;
    if ((e = kerr_eval(h, u, nullptr, 0.f, k1, ksc, s)) != cudaSuccess) return e;
    if ((e = kerr_eval(h, u, k1, 0.5f, k2, ksc, s)) != cudaSuccess) return e;
    if ((e = kerr_eval(h, u, k2, 0.5f, k3, ksc, s)) != cudaSuccess) return e;
    if ((e = kerr_eval(h, u, k3, 1.f, k4, ksc, s)) != cudaSuccess) return e;
    a.in[0] = u; a.coef[0] = 1.f;
    a.in[1] = k1; a.coef[1] = 1.f / 6.f;
    a.in[2] = k2; a.coef[2] = 1.f / 3.f;
    a.in[3] = k3; a.coef[3] = 1.f / 3.f;
    a.in[4] = k4; a.coef[4] = 1.f / 6.f;
    a.n_in = 5;
    a.out = A;
    return lin_launch(a, P, N, s);
}

// One symmetric split step with the iterative nonlinear step (SSFM-Agrawal, Section 3.1),
// kappa form only.  The kappa-form nonlinear flow keeps |A| and rotates A_f by
// exp(i gamma int phi_f dz), phi_f = sum_g kappa_fg |A_g|^2; the integral is the trapezoid of
// phi at the two ends of the step, phi(z+h) estimated from the step's own result:
//   phi0 = phi(A);  u = E A;  A1 = E [u exp(i gamma h phi0)];
//   A_{k+1} = E [u exp(i gamma h (phi0 + phi(A_k)) / 2)]   (k = 1, 2);   A(z+h) = A_3.
// Eight launches.
constexpr int AGRAWAL_REFINE = 2;
cudaError_t enqueue_ssfm_agrawal_step(mmf_ctx* h, float2* A, double hstep, cudaStream_t s) {
    float2 *u = h->buf[0], *v = h->buf[1], *est = h->buf[3];
    float* phi0 = reinterpret_cast<float*>(h->buf[2]);
    const float ksc = (float)(h->gamma * hstep);
    const int P = h->P * h->batch, N = h->N;
    const KerrKappa kk = {h->P, h->d_kappa};
    cudaError_t e;
    if ((e = kappa_phi_launch(kk, A, phi0, h->Nk, h->n_sm, s)) != cudaSuccess) return e;
    LinArgs a = lin_args(h, h->d_E);
    a.in[0] = A; a.coef[0] = 1.f; a.n_in = 1; a.add = nullptr; a.out = u;
    if ((e = lin_launch(a, P, N, s)) != cudaSuccess) return e;
    if ((e = phase_rotate_launch(u, phi0, ksc, v, (size_t)h->P * h->Nk, s)) != cudaSuccess) return e;
    for (int k = 0; k <= AGRAWAL_REFINE; ++k) {
        a.in[0] = v;
        a.out = k == AGRAWAL_REFINE ? A : est;
        if ((e = lin_launch(a, P, N, s)) != cudaSuccess) return e;
        if (k == AGRAWAL_REFINE) break;
        if ((e = kappa_rotate_launch(kk, est, u, phi0, ksc, v, h->Nk, h->n_sm, h->d_slot_steps, h->N, s)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// Enqueue one RK4IP step (Eq. 4a-4f) on stream s (or the handle's other method).
// One RK4IP step (Eq. 4a-4f) in three parts.  The linear step acts on every row on its own,
// so the first part (4a) and the last (4f) can run on a range of rows [r0, r1) at a time; the
// middle couples all rows through the Kerr term.  r0 and r1 are multiples of the rows that
// share a propagator row (1 << e_shift), so that the range's E rows are contiguous.
LinArgs lin_rows(mmf_ctx* h, int r0) {
    LinArgs a = lin_args(h, h->d_E + (size_t)(r0 >> h->e_shift) * h->N);
    if (a.scratch) a.scratch += (size_t)r0 * h->N;
    return a;
}

// (4a) A_I = Lin(A) on rows [r0, r1)
cudaError_t step_head(mmf_ctx* h, float2* A, int r0, int r1, cudaStream_t s) {
    const size_t o = (size_t)r0 * h->N;
    LinArgs a = lin_rows(h, r0);
    a.in[0] = A + o; a.coef[0] = 1.f; a.n_in = 1; a.add = nullptr; a.out = h->buf[0] + o;
    return lin_launch(a, r1 - r0, h->N, s);
}

// T = h N(A); (4b) k1 = Lin(T); (4c) k2 = h N(A_I + k1/2); (4d) k3 = h N(A_I + k2/2);
// v = Lin(A_I + k3); (4e) k4 = h N(v) -> T
cudaError_t step_middle(mmf_ctx* h, float2* A, double hstep, cudaStream_t s) {
    float2 *AI = h->buf[0], *k1 = h->buf[1], *k2 = h->buf[2], *k3 = h->buf[3], *T = h->buf[4], *v = h->buf[5];
    const float ksc = (float)(h->gamma * hstep);
    const int P = h->P * h->batch, N = h->N;
    cudaError_t e;
    LinArgs a = lin_args(h, h->d_E);
    if ((e = kerr_eval(h, A, nullptr, 0.f, T, ksc, s)) != cudaSuccess) return e;
    a.in[0] = T; a.coef[0] = 1.f; a.n_in = 1; a.add = nullptr; a.out = k1;
    if ((e = lin_launch(a, P, N, s)) != cudaSuccess) return e;
    if ((e = kerr_eval(h, AI, k1, 0.5f, k2, ksc, s)) != cudaSuccess) return e;
    if ((e = kerr_eval(h, AI, k2, 0.5f, k3, ksc, s)) != cudaSuccess) return e;
    a.in[0] = AI; a.coef[0] = 1.f; a.in[1] = k3; a.coef[1] = 1.f; a.n_in = 2; a.out = v;
    if ((e = lin_launch(a, P, N, s)) != cudaSuccess) return e;
    return kerr_eval(h, v, nullptr, 0.f, T, ksc, s);
}

// (4f) A = Lin(A_I + k1/6 + k2/3 + k3/3) + k4/6 on rows [r0, r1)
cudaError_t step_tail(mmf_ctx* h, float2* A, int r0, int r1, cudaStream_t s) {
    const size_t o = (size_t)r0 * h->N;
    LinArgs a = lin_rows(h, r0);
    a.in[0] = h->buf[0] + o; a.coef[0] = 1.f;
    a.in[1] = h->buf[1] + o; a.coef[1] = 1.f / 6.f;
    a.in[2] = h->buf[2] + o; a.coef[2] = 1.f / 3.f;
    a.in[3] = h->buf[3] + o; a.coef[3] = 1.f / 3.f;
    a.n_in = 4;
    a.add = h->buf[4] + o; a.add_coef = 1.f / 6.f;
    a.out = A + o;
    return lin_launch(a, r1 - r0, h->N, s);
}

// Eight launches over six scratch buffers (A_I, k1, k2, k3, T, v), each stage combine folded
// into a neighbouring kernel.
cudaError_t enqueue_step(mmf_ctx* h, float2* A, double hstep, cudaStream_t s) {
    if (((h->flags >> 7) & 3u) == 1u) return enqueue_ssfm_rk4_step(h, A, hstep, s);
    if (((h->flags >> 7) & 3u) == 2u) return enqueue_ssfm_agrawal_step(h, A, hstep, s);
    const int P = h->P * h->batch;
    cudaError_t e;
    if ((e = step_head(h, A, 0, P, s)) != cudaSuccess) return e;
    if ((e = step_middle(h, A, hstep, s)) != cudaSuccess) return e;
    return step_tail(h, A, 0, P, s);
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

cudaError_t mmf::ctx_enqueue_step(mmf_ctx* h, float2* A, double hstep, cudaStream_t s) {
    return enqueue_step(h, A, hstep, s);
}
void mmf::ctx_free(mmf_ctx* h) { free_ctx(h); }
int mmf::ctx_fail(int code, const std::string& msg) { return fail(code, msg); }

// Packed upper triangle of a symmetric kappa (FP32) for the kappa-form kernel.
int build_kappa(mmf_ctx* h, const double* kappa) {
    const int P = h->P;
    double mx = 0.0;
    for (size_t i = 0; i < (size_t)P * P; ++i) mx = std::max(mx, std::fabs(kappa[i]));
    for (int f = 0; f < P; ++f)
        for (int g = f + 1; g < P; ++g)
            if (std::fabs(kappa[(size_t)f * P + g] - kappa[(size_t)g * P + f]) > 1e-12 * mx)
                return fail(MMF_EINVAL, "kappa must be symmetric");
    // one 4-row x 4-sample block per thread of a 512-thread CTA covers 256 rows
    if (P > 256 || kerr_kappa_smem_bytes(P) > 227 * 1024) return fail(MMF_EINVAL, "the kappa form supports at most 256 rows");
    std::vector<float> U;
    U.reserve((size_t)P * (P + 1) / 2);
    for (int f = 0; f < P; ++f)
        for (int g = f; g < P; ++g) U.push_back((float)kappa[(size_t)f * P + g]);
    if (cudaMalloc(&h->d_kappa, sizeof(float) * U.size()) != cudaSuccess) return fail(MMF_ENOMEM, "kappa allocation failed");
    CK(cudaMemcpy(h->d_kappa, U.data(), sizeof(float) * U.size(), cudaMemcpyHostToDevice));
    h->scratch_bytes += sizeof(float) * U.size();
    return MMF_OK;
}

// kappa as the B operand of the tensor-core kappa kernel: per chunk of 32 rows g, the hi and lo
// BF16 splits of kappa_f,g (f < P; rows up to NP and g beyond P zero) in the K-major 64-byte
// swizzled layout of the MMA, [chunk][split][NP rows x 64 B].
int build_kappa_tc(mmf_ctx* h, const double* kappa) {
    const int P = h->P, NP = (P + 15) / 16 * 16, nkc = (P + 31) / 32;
    if (NP > 256 || kerr_kappa_tc_smem_bytes(NP) > 227 * 1024)
        return fail(MMF_EINVAL, "the tensor-core kappa form supports at most 256 rows");
    const size_t split = (size_t)NP * 64, bytes = (size_t)nkc * 2 * split;
    std::vector<uint8_t> B(bytes, 0);
    for (int kc = 0; kc < nkc; ++kc)
        for (int f = 0; f < P; ++f)
            for (int k = 0; k < 32 && kc * 32 + k < P; ++k) {
                const double v = kappa[(size_t)f * P + kc * 32 + k];
                const uint16_t hb = bf16_bits(v), lb = bf16_bits(v - bf16_value(hb));
                uint8_t* t0 = B.data() + (size_t)kc * 2 * split;
                const size_t o = sw_byte(64, f, k, 2);
                std::memcpy(t0 + o, &hb, 2);
                std::memcpy(t0 + split + o, &lb, 2);
            }
    if (cudaMalloc(&h->d_kappa_tc, bytes) != cudaSuccess) return fail(MMF_ENOMEM, "kappa tile allocation failed");
    CK(cudaMemcpy(h->d_kappa_tc, B.data(), bytes, cudaMemcpyHostToDevice));
    h->scratch_bytes += bytes;
    h->ktc = {P, NP, nkc, h->d_kappa_tc, h->d_err};
    return MMF_OK;
}

int mmf::ctx_create(mmf_ctx** out, int n_modes, int n_pol, const double* S_plmn, const int32_t* parity_class,
                    const double* betas, double alpha, double gamma, int64_t N_t, double dt, unsigned flags,
                    void* stream, int batch, int e_shift_in, const double* kappa) {
    if (!out) return fail(MMF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_modes < 1) return fail(MMF_EINVAL, "n_modes must be >= 1");
    if (n_pol != 1 && n_pol != 2) return fail(MMF_EINVAL, "n_pol must be 1 or 2");
    if (n_modes * n_pol > 1023) return fail(MMF_EINVAL, "at most 1023 fields");
    if (batch < 1) return fail(MMF_EINVAL, "batch must be >= 1");
    if (kappa && (n_pol != 1 || (flags & ~((3u << 7) | 3u)) != 0 || ((flags & 3u) != MMF_KERR_FP32 && (flags & 3u) != MMF_KERR_BF16X3)))
        return fail(MMF_EINVAL, "the kappa form takes one row per field and FP32 or BF16x3 Kerr arithmetic");
    if (kappa && (flags & 3u) == MMF_KERR_BF16X3 && (((flags >> 7) & 3u) == 2u || batch != 1))
        return fail(MMF_EINVAL, "the kappa form's BF16x3 tensor-core Kerr serves RK4IP and SSFM-RK4 on one request");
    if (kappa) {
        S_plmn = nullptr;
        parity_class = nullptr;
    }
    if ((!S_plmn && !kappa) || (!betas && batch == 1)) return fail(MMF_EINVAL, "S_plmn (or kappa) and betas must not be NULL");
    if (!is_pow2(N_t) || N_t < 16 || N_t > (1 << 17)) return fail(MMF_EINVAL, "N_t must be a power of two in [16, 131072]");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(MMF_EINVAL, "dt must be positive");
    if (!std::isfinite(alpha) || !std::isfinite(gamma)) return fail(MMF_EINVAL, "alpha and gamma must be finite");
    if (((flags >> 7) & 3u) > 2u) return fail(MMF_EINVAL, "unknown method flag");
    if ((flags >> 5) & 3u) return fail(MMF_EINVAL, "flags bits 5-6 are reserved");
    if (((flags >> 7) & 3u) == 2u && !kappa)
        return fail(MMF_EINVAL, "MMF_METHOD_SSFM_AGRAWAL needs the kappa form (mmf_create_kappa)");
    const int M = n_modes, P = n_modes * n_pol;
    if (kappa) {
        for (size_t i = 0; i < (size_t)P * P; ++i)
            if (!std::isfinite(kappa[i])) return fail(MMF_EINVAL, "kappa has a non-finite entry");
    } else {
        const size_t M4 = (size_t)M * M * M * M;
        for (size_t i = 0; i < M4; ++i)
            if (!std::isfinite(S_plmn[i])) return fail(MMF_EINVAL, "S_plmn has a non-finite entry");
    }
    if (betas)
        for (int i = 0; i < 4 * P; ++i)
            if (!std::isfinite(betas[i])) return fail(MMF_EINVAL, "betas has a non-finite entry");
    if ((int64_t)P * batch * N_t > ((int64_t)1 << 31) - 1)
        return fail(MMF_EINVAL, "fields x slots x samples must stay below 2^31");
    if (parity_class) {
        for (int p = 0; p < M; ++p)
            for (int l = 0; l < M; ++l)
                for (int m = 0; m < M; ++m)
                    for (int n = 0; n < M; ++n) {
                        const int x = parity_class[p] ^ parity_class[l] ^ parity_class[m] ^ parity_class[n];
                        if (x != 0 && S_plmn[(((size_t)p * M + l) * M + m) * M + n] != 0.0)
                            return fail(MMF_EINVAL, "S_plmn is nonzero across parity classes");
                    }
    }
    mmf_ctx* h = new (std::nothrow) mmf_ctx();
    if (!h) return fail(MMF_ENOMEM, "host allocation failed");
    int rc = MMF_OK;
    auto bail = [&](int code) {
        free_ctx(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(MMF_ECUDA, "no CUDA device"));
    h->stream = (cudaStream_t)stream;
    h->M = M; h->n_pol = n_pol; h->P = P; h->N = (int)N_t;
    h->batch = batch;
    h->Nk = (int)N_t * batch;
    h->dt = dt; h->alpha = alpha; h->gamma = gamma; h->flags = flags;
    if (betas) h->betas.assign(betas, betas + 4 * P);
    // polarisation rows with identical betas share one propagator row
    h->e_shift = 0;
    if (e_shift_in >= 0) {
        h->e_shift = (P % 2 == 0 && e_shift_in > 0) ? 1 : 0;
    } else if (P % 2 == 0) {
        // rows 2i and 2i+1 (the two polarisations of a mode) with identical betas share a row
        bool same = true;
        for (int i = 0; i < P / 2 && same; ++i)
            same = std::memcmp(betas + 8 * i, betas + 8 * i + 4, 4 * sizeof(double)) == 0;
        h->e_shift = same ? 1 : 0;
    }
    h->e_rows = P >> h->e_shift;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess) return bail(cuda_fail(e, "stream"));
    const size_t fbytes = sizeof(float2) * (size_t)P * N_t * batch;
    if (cudaMalloc(&h->d_betas, sizeof(double) * 4 * P * batch) != cudaSuccess ||
        cudaMalloc(&h->d_tw, sizeof(float4) * (size_t)N_t) != cudaSuccess)
        return bail(fail(MMF_ENOMEM, "device allocation failed"));
    for (auto& b : h->buf)
        if (cudaMalloc(&b, fbytes) != cudaSuccess) return bail(fail(MMF_ENOMEM, "scratch allocation failed"));
    h->scratch_bytes = 6 * fbytes + sizeof(float4) * (size_t)N_t * (1 + (size_t)h->e_rows * batch);
    if (lin_needs_scratch(N_t)) {
        // rows of more than 2^14 samples go through the linear step in three passes over a scratch row
        if (cudaMalloc(&h->d_linscratch, fbytes) != cudaSuccess)
            return bail(fail(MMF_ENOMEM, "linear-step scratch allocation failed"));
        h->scratch_bytes += fbytes;
    }
    if (betas) {
        if ((e = cudaMemcpy(h->d_betas, betas, sizeof(double) * 4 * P, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(cuda_fail(e, "copy betas"));
    } else if ((e = cudaMemset(h->d_betas, 0, sizeof(double) * 4 * P * batch)) != cudaSuccess) {
        return bail(cuda_fail(e, "clear betas"));
    }
    if (batch > 1) {
        // request batches: per-slot propagator rows [e_rows][batch][N_t], written per admission;
        // the fields and scratch start cleared so that idle slots hold finite values
        if (cudaMalloc(&h->d_E, sizeof(float4) * (size_t)h->e_rows * batch * N_t) != cudaSuccess)
            return bail(fail(MMF_ENOMEM, "propagator table allocation failed"));
        for (auto& b : h->buf)
            if ((e = cudaMemset(b, 0, fbytes)) != cudaSuccess) return bail(cuda_fail(e, "clear scratch"));
    }
    if ((e = twiddle_table_launch(h->d_tw, (int)N_t, h->stream)) != cudaSuccess) return bail(cuda_fail(e, "twiddles"));
    h->e_nblk = energy_blocks((int)N_t);
    if (cudaMalloc(&h->d_epart, sizeof(double) * P * h->e_nblk) != cudaSuccess ||
        cudaMalloc(&h->d_eout, sizeof(double) * P) != cudaSuccess)
        return bail(fail(MMF_ENOMEM, "energy scratch allocation failed"));
    const unsigned algo = flags & (3u << 3), prec = flags & 3u;
    if ((e = cudaMalloc(&h->d_err, sizeof(int))) != cudaSuccess) return bail(fail(MMF_ENOMEM, "status allocation failed"));
    if ((e = cudaMemset(h->d_err, 0, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "status init"));
    if ((e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
        return bail(cuda_fail(e, "SM count"));
    if (kappa) {
        h->kerr_path = 4;
        if ((rc = build_kappa(h, kappa)) != MMF_OK) return bail(rc);
        if (prec == MMF_KERR_BF16X3) {
            int major = 0;
            cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
            if (major != 10) return bail(fail(MMF_EINVAL, "the tensor-core Kerr path needs an sm_10x (Blackwell) GPU"));
            if ((rc = build_kappa_tc(h, kappa)) != MMF_OK) return bail(rc);
            h->kerr_path = 5;
        }
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(e, "create sync"));
        *out = h;
        return MMF_OK;
    }
    const bool sym = algo != MMF_KERR_LIST && fully_symmetric(S_plmn, M);
    if (algo == MMF_KERR_PAIRS && !sym) return bail(fail(MMF_EINVAL, "MMF_KERR_PAIRS needs a fully symmetric S_plmn"));
    if (prec != MMF_KERR_FP32 && !sym)
        return bail(fail(MMF_EINVAL, "the BF16 Kerr paths need a fully symmetric S_plmn (pair contraction)"));
    if (sym) {
        h->kerr_path = 1;
        if ((rc = build_pairs(h, S_plmn, parity_class)) != MMF_OK) return bail(rc);
    } else {
        h->kerr_path = 0;
        if (P > 64) return bail(fail(MMF_EINVAL, "the general list path supports at most 64 fields"));
        if ((rc = build_term_list(h, S_plmn)) != MMF_OK) return bail(rc);
    }
    if (prec != MMF_KERR_FP32) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device);
        if (major != 10) return bail(fail(MMF_EINVAL, "the tensor-core Kerr path needs an sm_10x (Blackwell) GPU"));
        const bool x3 = prec != MMF_KERR_BF16, tf32 = prec == MMF_KERR_TF32X3;
        if ((rc = build_tcr(h, S_plmn, parity_class, x3, tf32)) != MMF_OK) return bail(rc);
        h->kerr_path = 3;
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(e, "create sync"));
    *out = h;
    return MMF_OK;
}

extern "C" {

const char* mmf_last_error(void) { return g_last_error.c_str(); }

int mmf_create(mmf_handle* out, int n_modes, int n_pol, const double* S_plmn, const int32_t* parity_class,
               const double* betas, double alpha, double gamma, int64_t N_t, double dt, unsigned flags,
               void* stream) {
    g_last_error.clear();
    return ctx_create(out, n_modes, n_pol, S_plmn, parity_class, betas, alpha, gamma, N_t, dt, flags, stream, 1, -1);
}

int mmf_create_kappa(mmf_handle* out, int n_fields, const double* kappa, const double* betas, double alpha,
                     double gamma, int64_t N_t, double dt, unsigned flags, void* stream) {
    g_last_error.clear();
    if (!kappa) return fail(MMF_EINVAL, "kappa is NULL");
    return ctx_create(out, n_fields, 1, nullptr, nullptr, betas, alpha, gamma, N_t, dt, flags, stream, 1, -1, kappa);
}

int mmf_device_status(mmf_handle h, int* code) {
    if (!h || !code) return fail(MMF_EINVAL, "NULL argument");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(code, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    if (*code != 0) return fail(MMF_ETIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(*code) + ")");
    return MMF_OK;
}

int mmf_destroy(mmf_handle h) {
    if (!h) return MMF_OK;
    free_ctx(h);
    return MMF_OK;
}

int mmf_info(mmf_handle h, int* P, int64_t* N_t, int* kerr_path, size_t* scratch_bytes) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (P) *P = h->P;
    if (N_t) *N_t = h->N;
    if (kerr_path) *kerr_path = h->kerr_path;
    if (scratch_bytes) *scratch_bytes = h->scratch_bytes;
    return MMF_OK;
}

namespace {

// The step graph for (fields, h), captured on first use and whenever either changes.
int ensure_step_graph(mmf_ctx* h, void* fields, double hs) {
    if (h->graph && h->graph_fields == fields && h->graph_h == hs) return MMF_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_step(h, (float2*)fields, hs, h->cap);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "capture RK4IP step");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(e, "instantiate step graph");
    }
    h->graph_fields = fields;
    h->graph_h = hs;
    return MMF_OK;
}

}  // namespace

int mmf_propagate(mmf_handle h, void* fields, double L, int n_steps) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!fields) return fail(MMF_EINVAL, "fields is NULL");
    if (n_steps < 0) return fail(MMF_EINVAL, "n_steps must be >= 0");
    if (!std::isfinite(L)) return fail(MMF_EINVAL, "L must be finite");
    if (n_steps == 0) return MMF_OK;
    CK(cudaSetDevice(h->device));
    const double hs = L / n_steps;
    int rc = ensure_E(h, &h->d_E, &h->E_z, hs / 2);
    if (rc != MMF_OK) return rc;
    if ((rc = ensure_step_graph(h, fields, hs)) != MMF_OK) return rc;
    for (int i = 0; i < n_steps; ++i) CK(cudaGraphLaunch(h->graph, h->stream));
    return MMF_OK;
}

// Host buffers in and out.  The linear step acts on each row on its own, so the copies are cut
// into row chunks on a second stream: the first step's (4a) runs on each chunk as soon as it
// has arrived, and the last step's (4f) hands each chunk to its copy back as soon as it is
// done.  The Kerr evaluations between them couple all rows and wait for the whole upload.
// Same kernels on the same rows as mmf_propagate: the results are the same bits.
int mmf_propagate_host(mmf_handle h, const void* fields_in, void* fields_out, double L, int n_steps) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!fields_in || !fields_out) return fail(MMF_EINVAL, "host buffers must not be NULL");
    if (n_steps < 0) return fail(MMF_EINVAL, "n_steps must be >= 0");
    if (!std::isfinite(L)) return fail(MMF_EINVAL, "L must be finite");
    CK(cudaSetDevice(h->device));
    const int P = h->P;
    const size_t row_bytes = sizeof(float2) * (size_t)h->N, bytes = row_bytes * P;
    if (!h->d_io) {
        if (cudaMalloc(&h->d_io, bytes) != cudaSuccess) return fail(MMF_ENOMEM, "staging allocation failed");
        h->scratch_bytes += bytes;
    }
    const char* src = (const char*)fields_in;
    char* dst = (char*)fields_out;
    float2* A = h->d_io;
    // chunks of whole propagator-row groups (polarisation pairs when they share E)
    const int unit = 1 << h->e_shift, units = P / unit;
    const int nch = units < MMF_IO_CHUNKS ? units : MMF_IO_CHUNKS;
    const bool split = n_steps > 0 && nch > 1 && ((h->flags >> 7) & 3u) == 0u && h->batch == 1;
    if (!split) {
        CK(cudaMemcpyAsync(h->d_io, fields_in, bytes, cudaMemcpyHostToDevice, h->stream));
        int rc = mmf_propagate(h, h->d_io, L, n_steps);
        if (rc != MMF_OK) return rc;
        CK(cudaMemcpyAsync(fields_out, h->d_io, bytes, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return MMF_OK;
    }
    if (!h->io_stream) {
        CK(cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking));
        for (int c = 0; c <= MMF_IO_CHUNKS; ++c) CK(cudaEventCreateWithFlags(&h->io_ev[c], cudaEventDisableTiming));
        for (int c = 0; c < MMF_IO_CHUNKS; ++c) CK(cudaEventCreateWithFlags(&h->io_ev_out[c], cudaEventDisableTiming));
    }
    const double hs = L / n_steps;
    int rc = ensure_E(h, &h->d_E, &h->E_z, hs / 2);
    if (rc != MMF_OK) return rc;
    if (n_steps > 2 && (rc = ensure_step_graph(h, h->d_io, hs)) != MMF_OK) return rc;
    auto row0 = [&](int c) { return (int)((int64_t)c * units / nch) * unit; };
    // the upload starts after whatever the caller's stream has queued
    CK(cudaEventRecord(h->io_ev[MMF_IO_CHUNKS], h->stream));
    CK(cudaStreamWaitEvent(h->io_stream, h->io_ev[MMF_IO_CHUNKS], 0));
    for (int c = 0; c < nch; ++c) {
        const int r0 = row0(c), r1 = row0(c + 1);
        CK(cudaMemcpyAsync((char*)A + r0 * row_bytes, src + r0 * row_bytes, (r1 - r0) * row_bytes,
                           cudaMemcpyHostToDevice, h->io_stream));
        CK(cudaEventRecord(h->io_ev[c], h->io_stream));
    }
    // first step: (4a) chunk by chunk as the rows arrive
    for (int c = 0; c < nch; ++c) {
        CK(cudaStreamWaitEvent(h->stream, h->io_ev[c], 0));
        CK(step_head(h, A, row0(c), row0(c + 1), h->stream));
    }
    CK(step_middle(h, A, hs, h->stream));
    if (n_steps > 1) {
        CK(step_tail(h, A, 0, P, h->stream));
        for (int i = 1; i < n_steps - 1; ++i) CK(cudaGraphLaunch(h->graph, h->stream));
        CK(step_head(h, A, 0, P, h->stream));
        CK(step_middle(h, A, hs, h->stream));
    }
    // last step: (4f) chunk by chunk, each chunk copied back as soon as it is done
    for (int c = 0; c < nch; ++c) {
        const int r0 = row0(c), r1 = row0(c + 1);
        CK(step_tail(h, A, r0, r1, h->stream));
        CK(cudaEventRecord(h->io_ev_out[c], h->stream));
        CK(cudaStreamWaitEvent(h->io_stream, h->io_ev_out[c], 0));
        CK(cudaMemcpyAsync(dst + r0 * row_bytes, (const char*)A + r0 * row_bytes, (r1 - r0) * row_bytes,
                           cudaMemcpyDeviceToHost, h->io_stream));
    }
    CK(cudaStreamSynchronize(h->io_stream));
    CK(cudaStreamSynchronize(h->stream));
    return MMF_OK;
}

int mmf_energy(mmf_handle h, const void* fields, double* out_per_field) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!fields || !out_per_field) return fail(MMF_EINVAL, "NULL pointer");
    CK(cudaSetDevice(h->device));
    CK(energy_launch((const float2*)fields, h->P, h->N, h->dt, h->d_epart, h->e_nblk, h->d_eout, h->stream));
    CK(cudaMemcpyAsync(out_per_field, h->d_eout, sizeof(double) * h->P, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MMF_OK;
}

int mmf_kerr(mmf_handle h, const void* in, void* out, double scale) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!in || !out || in == out) return fail(MMF_EINVAL, "in and out must be distinct device pointers");
    CK(cudaSetDevice(h->device));
    CK(kerr_eval(h, (const float2*)in, nullptr, 0.f, (float2*)out, (float)(h->gamma * scale), h->stream));
    return MMF_OK;
}

int mmf_kerr_stage(mmf_handle h, const void* in0, const void* in1, double c1, void* out, double scale) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!in0 || !out || in0 == out || in1 == out) return fail(MMF_EINVAL, "out must be distinct from in0 and in1");
    if (!std::isfinite(c1) || !std::isfinite(scale)) return fail(MMF_EINVAL, "c1 and scale must be finite");
    CK(cudaSetDevice(h->device));
    CK(kerr_eval(h, (const float2*)in0, (const float2*)in1, (float)c1, (float2*)out, (float)(h->gamma * scale),
                 h->stream));
    return MMF_OK;
}

int mmf_linear_stage(mmf_handle h, int n_in, const void* const* in, const double* coef, const void* add,
                     double add_coef, void* out, double z) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (n_in < 1 || n_in > LinArgs::MAX_IN) return fail(MMF_EINVAL, "n_in must be in 1..5");
    if (!in || !coef || !out) return fail(MMF_EINVAL, "NULL pointer");
    if (!std::isfinite(z) || !std::isfinite(add_coef)) return fail(MMF_EINVAL, "z and add_coef must be finite");
    for (int i = 0; i < n_in; ++i) {
        if (!in[i]) return fail(MMF_EINVAL, "NULL input");
        if (i > 0 && in[i] == out) return fail(MMF_EINVAL, "out may alias in[0] only");
        if (!std::isfinite(coef[i])) return fail(MMF_EINVAL, "coef must be finite");
    }
    if (add && add == out) return fail(MMF_EINVAL, "out must not alias add");
    CK(cudaSetDevice(h->device));
    int rc = ensure_E(h, &h->d_Elin, &h->Elin_z, z);
    if (rc != MMF_OK) return rc;
    LinArgs a = lin_args(h, h->d_Elin);
    for (int i = 0; i < n_in; ++i) {
        a.in[i] = (const float2*)in[i];
        a.coef[i] = (float)coef[i];
    }
    a.n_in = n_in;
    a.add = (const float2*)add;
    a.add_coef = (float)add_coef;
    a.out = (float2*)out;
    CK(lin_launch(a, h->P, h->N, h->stream));
    return MMF_OK;
}

int mmf_amplify(mmf_handle h, void* fields, double power_gain, const void* noise) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!fields) return fail(MMF_EINVAL, "fields is NULL");
    if (!(power_gain >= 0) || !std::isfinite(power_gain)) return fail(MMF_EINVAL, "power_gain must be finite and >= 0");
    CK(cudaSetDevice(h->device));
    CK(amplify_launch((float2*)fields, (float)std::sqrt(power_gain), (const float2*)noise, (size_t)h->P * h->N,
                      h->stream));
    return MMF_OK;
}

int mmf_linear(mmf_handle h, const void* in, void* out, double z) {
    if (!h) return fail(MMF_EINVAL, "NULL handle");
    if (!in || !out) return fail(MMF_EINVAL, "NULL pointer");
    if (!std::isfinite(z)) return fail(MMF_EINVAL, "z must be finite");
    CK(cudaSetDevice(h->device));
    int rc = ensure_E(h, &h->d_Elin, &h->Elin_z, z);
    if (rc != MMF_OK) return rc;
    LinArgs a = lin_args(h, h->d_Elin);
    a.in[0] = (const float2*)in;
    a.coef[0] = 1.f;
    a.n_in = 1;
    a.out = (float2*)out;
    CK(lin_launch(a, h->P, h->N, h->stream));
    return MMF_OK;
}

}  // extern "C"
