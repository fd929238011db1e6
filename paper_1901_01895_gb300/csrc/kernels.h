// Internal launch interface between the C ABI (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace mmf {

// out = Lin(sum_i coef[i] * in[i]) + add_coef * add    (add may be NULL)
// Lin(x) = IFFT(E * FFT(x)) row by row.  Rows are r = f * e_batch + b (field f, request
// slot b; e_batch = 1 outside a request batch) and use E row
// ((r / e_batch) >> e_shift) * e_batch + r % e_batch.  With slot_steps != NULL a row whose
// slot has no steps left (slot_steps[b] <= 0) is skipped: neither read nor written.
struct LinArgs {
    static constexpr int MAX_IN = 5;
    const float2* in[MAX_IN];
    float coef[MAX_IN];
    int n_in;
    const float2* add;
    float add_coef;
    float2* out;
    const float4* E;    // [rows >> e_shift][N] double-float propagator
    int e_shift;
    const float4* tw;   // [N] double-float W_N^j
    int e_batch;        // request slots per field (1 outside a request batch)
    const int* slot_steps;   // [e_batch] steps left per slot, or NULL
    float2* scratch;    // [rows][N] for rows of 2^17 samples (three-pass path), or NULL
    int n_sm;           // SMs of the device (sizes the grid-stride passes)
};

cudaError_t lin_launch(const LinArgs& a, int rows, int N, cudaStream_t s);
// Rows of more than 2^14 samples go through the linear step in three launches over a scratch
// row of the same size as the fields (slices of 2^13 samples); shorter rows in one launch.
__host__ __device__ inline bool lin_needs_scratch(int64_t N) { return N > (1 << 14); }
cudaError_t twiddle_table_launch(float4* tw, int N, cudaStream_t s);
// E row i (i < rows) at E + i * out_pitch, from betas_dev + i * row_stride * 4.
cudaError_t propagator_table_launch(float4* E, const double* betas_dev, int rows, int row_stride, int N,
                                    double dt, double alpha, double z, size_t out_pitch, cudaStream_t s);
// A = g * A + noise over n complex values (noise may be NULL): a flat-gain amplifier.
cudaError_t amplify_launch(float2* A, float gain, const float2* noise, size_t n, cudaStream_t s);
// One tick of a request batch: slot_steps[b] -= 1 where it is positive.
cudaError_t slot_tick_launch(int* slot_steps, int n_slots, cudaStream_t s);

// Kerr input x = in0 + in1_coef * in1 (in1 may be NULL); the kernels write
//   k = scale * Kerr(x)                         to out (scale = i*gamma*h folded in),
// and, when acc != NULL, also acc_out = acc + acc_coef * k  and  nxt = base + nxt_coef * k.
// With slot_steps != NULL the time axis holds request slots of slot_len samples each and
// sample tiles that touch only slots without steps left are skipped.
struct KerrIO {
    const float2* in0;
    const float2* in1;
    float in1_coef;
    float2* out;
    const float2* acc;
    float acc_coef;
    float2* acc_out;
    const float2* base;
    float nxt_coef;
    float2* nxt;
    const int* slot_steps;
    int slot_len;
};

// General nonzero-list Kerr sum (any real S, either polarisation model).
// Terms grouped by output field: term_off[f] .. term_off[f+1]-1 index into idx/coef;
// idx packs (l, m, n) field indices (10 bits each), coef already includes the l<->m fold.
struct KerrList {
    const int* term_off;      // [P+1]
    const uint32_t* idx;      // [n_terms]
    const float* coef;        // [n_terms]
    int P;
};
cudaError_t kerr_list_launch(const KerrList& k, const KerrIO& io, float scale, int N, cudaStream_t s);

// Factored pair contraction (S fully symmetric; isotropic two-polarisation or scalar):
//   u_(ij) = c_ij Re sum_a A_ia conj(A_ja),  v_(ij) = c_ij sum_a A_ia A_ja   (i <= j, c = 2 off-diagonal)
//   W_(pl) = sum S_pair[(pl),(ij)] u_(ij),   Z_(pl) = sum S_pair[(pl),(ij)] v_(ij)   (per parity class)
//   K_(p,a) = (i gamma h / 3) [2 sum_l W_pl A_la + sum_l Z_pl conj(A_la)]   (two polarisations)
//   K_p     = i gamma h sum_l Z_pl conj(A_l)                                 (one polarisation)
struct KerrPairs {
    int M;                   // spatial modes
    int n_pol;
    int n_class;             // parity classes present
    const int* cls_off;      // [n_class+1] pair offsets per class (pairs sorted by class)
    const int2* pair_ij;     // [n_pairs] (i, j), i <= j, in class order
    const float* pair_c;     // [n_pairs] fold factor c_ij (1 or 2)
    const float* S_pair;     // per class c: dense [n_c][n_c] row-major at S_off[c]
    const int64_t* S_off;    // [n_class]
};
cudaError_t kerr_pairs_simt_launch(const KerrPairs& k, const KerrIO& io, float scale, int N, cudaStream_t s);

// Pair contraction on the tensor cores with one TMEM lane per (sample, pair quantity)
// (kerr_tcr.cu).  Per parity class c the output pairs (p, l) are cut into passes of at most
// np_max columns; a pass is a list of segments {p-list} x {l-list of <= 12 modes}, p-major.
//   passes[q]   = {class, npad (columns, multiple of 16), first segment, end segment}
//   pass_boff[q]= byte offset into B of the pass's tiles [n_chunk][split][npad x 64 B]
//   segs[g]     = {first column in the pass, l-list length | own_p << 8 | own_l << 9,
//                  p-list length, list offset}; own_p / own_l: the epilogue group that sweeps
//                  the segment by rows (K_p) / by columns (K_l)
//   lists       = per segment the l-list then the p-list (mode indices, one byte each)
//   pairs       = i | j << 8 of the input pairs in class order, cls_off the class offsets
struct KerrTCR {
    int M, n_pol, n_class, n_pass, n_seg, n_list, n_pairs;
    int np_max;              // widest pass = rows of a B stage
    int na, nb, nfb;         // pair-product stages, S-tile stages, field buffers
    int kacc_global;         // epilogue adds into the output in global memory (no shared accumulator)
    const int* cls_off;
    const uint16_t* pairs;
    const int4* passes;
    const int64_t* pass_boff;
    const int4* segs;
    const uint8_t* lists;
    const uint8_t* B;
    int x3;                  // three-term split (hi*hi + hi*lo + lo*hi)
    int tf32;                // operands in TF32 (16 pairs per chunk) instead of BF16 (32 pairs)
    int* err;
    const int* slot_steps;   // request slots along the time axis (skip tiles without steps left), or NULL
    int slot_len;
};
int kerr_tcr_tile_samples(int n_pol);
size_t kerr_tcr_smem_bytes(const KerrTCR& k);
// out = scale * Kerr(in0 + c1 * in1)   (in1 may be NULL)
cudaError_t kerr_tcr_launch(const KerrTCR& k, const float2* in0, const float2* in1, float c1, float2* out, float scale,
                            int N, int n_sm, cudaStream_t s);

// Kerr term in the kappa form of Eq. 1 (kerr_kappa.cu): out_f = i * scale * (sum_g kappa_fg |x_g|^2) x_f
// with kappa symmetric, U its packed upper triangle in FP32 (row f: kappa_f,f .. kappa_f,P-1).
struct KerrKappa {
    int P;
    const float* U;
};
// Phase of the kappa form's nonlinear flow (the flow keeps |A| and rotates A_f by
// exp(i gamma int phi_f dz), phi_f = sum_g kappa_fg |A_g|^2), for the iterative split step.
struct KappaPhase {
    const float2* u;     // field to rotate
    const float* phi0;   // [P][N] phase rate at the start of the step
    float* phi_out;      // [P][N] phase rate written by kappa_phi_launch
};
size_t kerr_kappa_smem_bytes(int P);
// The same Kerr term on the tensor cores (kerr_kappa_tc.cu): phi = kappa |x|^2 as a BF16x3 GEMM
// per tile of 128 samples.  B: the kappa chunks [nkc][hi, lo][NP rows x 64 B], chunk c holding
// kappa_f,g for g = 32c .. 32c + 31 in the K-major 64-byte swizzled layout (zero beyond P).
struct KappaTC {
    int P;                 // rows
    int NP;                // P rounded up to 16 (the MMA's N, <= 256)
    int nkc;               // chunks of 32 rows g
    const uint8_t* B;
    int* err;              // device status word (bounded waits that time out)
};
size_t kerr_kappa_tc_smem_bytes(int NP);
cudaError_t kerr_kappa_tc_launch(const KappaTC& k, const float2* in0, const float2* in1, float c1, float2* out,
                                 float scale, int N, int n_sm, cudaStream_t s);
cudaError_t kerr_kappa_launch(const KerrKappa& k, const KerrIO& io, float scale, int N, int n_sm, cudaStream_t s);
// phi_out = kappa |y|^2
cudaError_t kappa_phi_launch(const KerrKappa& k, const float2* y, float* phi_out, int N, int n_sm, cudaStream_t s);
// out = u exp(i scale (phi0 + kappa |y|^2) / 2)
cudaError_t kappa_rotate_launch(const KerrKappa& k, const float2* y, const float2* u, const float* phi0, float scale,
                                float2* out, int N, int n_sm, const int* slot_steps, int slot_len, cudaStream_t s);
// out = u exp(i scale phi0), elementwise over n values
cudaError_t phase_rotate_launch(const float2* u, const float* phi0, float scale, float2* out, size_t n,
                                cudaStream_t s);

// FP64 per-field energies: partial sums into scratch [P][nblk], then a fixed-order
// reduction into out[P] (device).
cudaError_t energy_launch(const float2* A, int P, int N, double dt, double* scratch, int nblk,
                          double* out, cudaStream_t s);
int energy_blocks(int N);

// Sets the thread's message returned by mmf_last_error().
void set_last_error(const std::string& msg);

}  // namespace mmf
