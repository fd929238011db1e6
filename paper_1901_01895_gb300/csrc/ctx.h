// Internal state of a propagator handle (shared by the C ABI in api.cu and the request
// server in server.cu).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"

using mmf::KerrTCR;

// Row chunks of mmf_propagate_host's copies (each overlapped with the linear step of the
// chunk before or after it).
constexpr int MMF_IO_CHUNKS = 8;

struct mmf_ctx {
    int device = -1;
    cudaStream_t stream = nullptr;     // caller's stream
    cudaStream_t cap = nullptr;        // private stream used for graph capture
    int M = 0, n_pol = 0, P = 0;
    int N = 0;                         // samples per field row (the FFT length N_t)
    int batch = 1;                     // request slots side by side on the time axis
    int Nk = 0;                        // samples per field seen by the Kerr kernels: batch * N
    const int* d_slot_steps = nullptr; // [batch] steps left per slot (request batches only; not owned)
    double dt = 0, alpha = 0, gamma = 0;
    unsigned flags = 0;
    int kerr_path = 0;                 // 0 list, 1 pairs SIMT, 3 pairs tensor core (one TMEM lane
                                       // per sample quantity), 4 kappa form (self- and cross-phase
                                       // matrix), 5 kappa form on the tensor cores; 2 is retired
    float* d_kappa = nullptr;          // packed upper triangle of kappa (kappa form)
    uint8_t* d_kappa_tc = nullptr;     // kappa's BF16 hi/lo chunks (kappa form, tensor cores)
    mmf::KappaTC ktc = {};
    std::vector<double> betas;         // [P][4]
    double* d_betas = nullptr;
    int e_shift = 0, e_rows = 0;
    float4* d_tw = nullptr;            // [N]
    float4* d_E = nullptr;             // [e_rows][N] for z = E_z
    double E_z = NAN;
    float4* d_Elin = nullptr;          // table for mmf_linear
    double Elin_z = NAN;
    float2* buf[6] = {};               // AI, k1, k2, k3, T, v
    float2* d_linscratch = nullptr;    // the linear step's scratch rows above N_t = 2^14
    float2* d_io = nullptr;            // device staging for mmf_propagate_host
    cudaStream_t io_stream = nullptr;  // mmf_propagate_host: row-chunk copies beside the compute
    cudaEvent_t io_ev[MMF_IO_CHUNKS + 1] = {};    // chunk c uploaded; [MMF_IO_CHUNKS]: caller's queue
    cudaEvent_t io_ev_out[MMF_IO_CHUNKS] = {};    // chunk c's last linear step done
    // Kerr: nonzero list
    int* d_term_off = nullptr;
    uint32_t* d_idx = nullptr;
    float* d_coef = nullptr;
    int n_terms = 0;
    // Kerr: pair contraction
    int n_class = 0;
    int* d_cls_off = nullptr;
    int2* d_pair_ij = nullptr;
    float* d_pair_c = nullptr;
    float* d_S_pair = nullptr;
    int64_t* d_S_off = nullptr;
    std::vector<int> cls_off;          // host copies (tensor-core path tables)
    std::vector<int2> pair_ij;
    std::vector<int64_t> S_off;
    // Kerr: tensor-core tables
    KerrTCR tcr = {};
    int n_sm = 0;
    void* d_tc_blob = nullptr;         // all tensor-core tables in one allocation
    int* d_err = nullptr;              // device status word
    // energy
    int e_nblk = 0;
    double* d_epart = nullptr;
    double* d_eout = nullptr;
    // graph of one step
    cudaGraphExec_t graph = nullptr;
    const void* graph_fields = nullptr;
    double graph_h = NAN;
    size_t scratch_bytes = 0;
};

namespace mmf {

// Creates a handle for n_modes x n_pol fields of N_t samples and `batch` request slots:
// field rows are laid out [P][batch][N_t] and the Kerr kernels see batch * N_t samples per
// field.  batch == 1 with e_shift < 0 is mmf_create; for batch > 1 betas may be NULL (the
// per-slot betas are written later) and e_shift (0 or 1) is given by the caller.
// With kappa != NULL the handle evaluates the kappa form of Eq. 1 instead of the overlap
// tensor: n_modes is then the number of rows P (n_pol = 1), kappa is host [P][P] symmetric and
// S_plmn / parity_class are ignored.
int ctx_create(mmf_ctx** out, int n_modes, int n_pol, const double* S_plmn, const int32_t* parity_class,
               const double* betas, double alpha, double gamma, int64_t N_t, double dt, unsigned flags, void* stream,
               int batch, int e_shift, const double* kappa = nullptr);
void ctx_free(mmf_ctx* h);
// Enqueues one RK4IP step (Eq. 4a-4f) of all rows on stream s (h's propagator table d_E
// must hold exp(hstep/2 D)).
cudaError_t ctx_enqueue_step(mmf_ctx* h, float2* A, double hstep, cudaStream_t s);
int ctx_fail(int code, const std::string& msg);

}  // namespace mmf
