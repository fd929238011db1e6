/*
 * mmf.h -- C ABI of the GB300 RK4IP propagator for the coupled multimode NLSE.
 *
 * The library advances optical fields A_f(t) (f = spatial mode x polarisation,
 * t = time sample) along a fiber with the fourth-order Runge-Kutta method in the
 * interaction picture (RK4IP, Section 3.2, Eq. 4a-4f of Brehler et al.,
 * arXiv:1901.01895) applied to
 *
 *   dA_f/dz = Lhat A_f + Nhat_f(A)                                       (Eq. 1)
 *   Lhat    = -alpha/2 + i sum_n (i^n/n!) beta_{n,f} d^n/dt^n
 *   Nhat_f  = i gamma sum_{l,m,n} Sfull_{f l m n} A_l A_m conj(A_n)
 *
 * Eq. 1 prints the nonlinear operator with a coupling matrix kappa; this library
 * takes the general overlap tensor S_plmn, of which the kappa form is the special
 * case S_pppp = kappa_pp, S_ppbb = S_pbpb = kappa_pb/2.  With two polarisations
 * the polarisation-resolved tensor is the isotropic one:
 *   Sfull_{(p a)(l b)(m c)(n d)} = S_plmn (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 3.
 *
 * Conventions shared by every call:
 *  - fields: complex64 (interleaved float re, im), row-major [P][N_t], P = n_modes*n_pol,
 *    field index f = mode*n_pol + pol, units sqrt(W); rows contiguous (Section 4).
 *  - Fourier convention: forward FFT exp(-2 pi i k t/N), omega_k = 2 pi k/(N dt) with
 *    k in [-N/2, N/2); the linear operator is then diagonal,
 *    D_f(omega) = -alpha/2 + i (beta0 - beta1 omega + beta2 omega^2/2 - beta3 omega^3/6).
 *  - Every call returns MMF_OK (0) or a negative MMF_E* code; mmf_last_error()
 *    gives a message for the calling thread.  No call aborts the process.
 *  - A handle is bound to one CUDA device and one stream and is not thread-safe.
 *    Device pointers passed in are owned by the caller; the library owns only the
 *    scratch it allocates in mmf_create and frees in mmf_destroy.
 */
#ifndef MMF_H
#define MMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mmf_ctx* mmf_handle;

enum {
    MMF_OK = 0,
    MMF_EINVAL = -1,    /* bad argument (shape, NULL pointer, tensor that violates parity, ...) */
    MMF_ENOMEM = -2,    /* device or host allocation failed                                    */
    MMF_ECUDA = -3,     /* a CUDA call failed; message from cudaGetErrorString                 */
    MMF_ETIMEOUT = -4,  /* a bounded device-side wait gave up                                  */
    MMF_EBUSY = -5      /* resource budget exhausted (serving admission)                       */
};

/* Kerr evaluation precision (flags bits 0-1).  All accumulate in FP32. */
enum {
    MMF_KERR_FP32 = 0,     /* FP32 operands (CUDA cores)                                    */
    MMF_KERR_BF16X3 = 1,   /* tensor cores, operands split x = hi + lo in BF16, three terms  */
    MMF_KERR_BF16 = 2,     /* tensor cores, plain BF16 operands                              */
    MMF_KERR_TF32X3 = 3    /* tensor cores, operands split x = hi + lo in TF32, three terms
                              (about FP32 precision)                                         */
};
/* Kerr algorithm (flags bits 3-4). */
enum {
    MMF_KERR_AUTO = 0 << 3,     /* factored pair contraction when S is fully symmetric, else list */
    MMF_KERR_LIST = 1 << 3,     /* general nonzero-list sum over the polarisation-resolved tensor */
    MMF_KERR_PAIRS = 2 << 3     /* require the factored pair contraction (EINVAL if S is not symmetric) */
};
/* Flags bits 5-6 are reserved and must be zero (MMF_EINVAL otherwise). */

/* Step method (flags bits 7-8). */
enum {
    MMF_METHOD_RK4IP = 0 << 7,     /* RK4 in the interaction picture (Section 3.2, Eq. 4a-4f), global O(h^4) */
    MMF_METHOD_SSFM_RK4 = 1 << 7,  /* symmetric split step, classic RK4 nonlinear step (Section 3.1), O(h^2):
                                      exp(h/2 L) . RK4 of dA/dz = N(A) over h . exp(h/2 L) */
    MMF_METHOD_SSFM_AGRAWAL = 2 << 7  /* symmetric split step with the iterative nonlinear step (Section 3.1),
                                         kappa form only: the phase exp(i gamma int phi dz) by the trapezoid of
                                         phi = kappa |A|^2 at both ends, the end estimate refined twice */
};

/*
 * mmf_create -- validate and copy the fiber description, allocate device scratch.
 *
 * n_modes, n_pol   spatial modes (>= 1) and polarisations (1 or 2); P = n_modes*n_pol.
 * S_plmn           host, float64 [n_modes]^4 row-major [p][l][m][n], 1/m^2; copied.
 * parity_class     host, int32 [n_modes] or NULL.  If given, S_plmn must vanish unless
 *                  the four classes XOR to 0 (checked: EINVAL otherwise); used to skip
 *                  the zero blocks.  NULL treats every mode as class 0 (dense).
 * betas            host, float64 [P][4]: beta0 rad/m, beta1 s/m, beta2 s^2/m, beta3 s^3/m
 *                  (Eq. 1's Taylor coefficients per field); copied.
 * alpha            power attenuation, 1/m (the field decays as exp(-alpha z / 2)).
 * gamma            n2 omega0 / c0, m/W (gamma * S is the nonlinear coefficient, 1/(W m)).
 * N_t              time samples, a power of two in [16, 131072].
 * dt               sample spacing, s.
 * flags            MMF_KERR_* precision | MMF_KERR_* algorithm | MMF_TC_* layout | MMF_METHOD_*.
 * stream           cudaStream_t (as void*) on which every later call of this handle
 *                  runs; NULL = legacy default stream.  The current CUDA device at
 *                  creation is the handle's device.
 * Device memory: about 6 field copies of scratch (6*P*N_t*8 bytes; a seventh above
 * N_t = 2^14, the linear step's scratch row) plus the Kerr coefficient tables and the
 * propagator table (n_modes or P rows of N_t*16 bytes).
 */
int mmf_create(mmf_handle* out, int n_modes, int n_pol, const double* S_plmn,
               const int32_t* parity_class, const double* betas, double alpha, double gamma,
               int64_t N_t, double dt, unsigned flags, void* stream);

/*
 * mmf_create_kappa -- the same propagator with the Kerr term in the form Eq. 1 prints:
 *   Nhat_f = i gamma (kappa_ff |A_f|^2 + sum_{g != f} kappa_fg |A_g|^2) A_f,
 * self- and cross-phase modulation only, every row f one spatial or polarisation mode
 * (Section 2; the paper's own interaction matrix, Section 4.4).
 * n_fields  rows P, 1..256.
 * kappa     host float64 [P][P], symmetric (checked to 1e-12 of its largest entry, else
 *           MMF_EINVAL), 1/m^2 like S_plmn (gamma * kappa in 1/(W m)); copied and kept on the
 *           device as its packed upper triangle in FP32 (P(P+1)/2 values).
 * betas, alpha, gamma, N_t, dt, stream  as for mmf_create (betas [P][4]).
 * flags     MMF_KERR_FP32 (phi = kappa |A|^2 on the CUDA cores) or MMF_KERR_BF16X3 (phi as a
 *           GEMM on the tensor cores, both operands split hi + lo in BF16, FP32 accumulation;
 *           kappa also kept as BF16 hi/lo tiles; not with MMF_METHOD_SSFM_AGRAWAL, whose phase
 *           kernels stay FP32) | MMF_METHOD_*.
 * Every other call (mmf_propagate, mmf_kerr, mmf_energy, ...) works on the handle unchanged.
 */
int mmf_create_kappa(mmf_handle* out, int n_fields, const double* kappa, const double* betas, double alpha,
                     double gamma, int64_t N_t, double dt, unsigned flags, void* stream);

/*
 * mmf_propagate -- advance the fields in place over length L with n_steps fixed RK4IP
 * steps, h = L / n_steps (Eq. 4a-4f per step).  fields: device pointer, complex64
 * [P][N_t].  Asynchronous on the handle's stream (returns after enqueueing; errors
 * from the launches are reported).  Restartable: two calls of L/2 equal one of L
 * when n_steps splits evenly.
 */
int mmf_propagate(mmf_handle h, void* fields, double L, int n_steps);

/*
 * mmf_propagate_host -- same as mmf_propagate for HOST buffers: copies fields_in
 * (host, complex64 [P][N_t]) to the device, propagates, copies the result to
 * fields_out (host; may equal fields_in) and synchronises the stream.  Pinned host
 * memory gives asynchronous full-bandwidth copies; pageable memory works too.
 * For the RK4IP method the copies are cut into up to eight row chunks on a private
 * stream: the first step's linear step (Eq. 4a) starts on each chunk as it arrives and
 * the last step's (Eq. 4f) hands each chunk to its copy back as soon as it is done.  The
 * work queued on the handle's stream before the call runs first; the results are the
 * same bits as mmf_propagate on the same fields.  The call allocates a staging field
 * copy on first use.
 */
int mmf_propagate_host(mmf_handle h, const void* fields_in, void* fields_out, double L, int n_steps);

/*
 * mmf_energy -- per-field energy E_f = sum_t |A_f(t)|^2 dt in W s, accumulated in
 * FP64 on the device in a fixed order (bitwise reproducible).  fields: device
 * pointer complex64 [P][N_t]; out_per_field: host float64 [P].  Synchronises the stream.
 */
int mmf_energy(mmf_handle h, const void* fields, double* out_per_field);

/*
 * mmf_kerr -- one evaluation of the Kerr term alone (the operator that Eq. 4 calls
 * four times per step): out = i * scale * gamma * sum Sfull A_l A_m conj(A_n) at every
 * sample.  in, out: device complex64 [P][N_t], distinct.  For tests and profiling.
 */
int mmf_kerr(mmf_handle h, const void* in, void* out, double scale);

/*
 * mmf_linear -- one application of exp(z * Lhat) (the linear propagator of Eq. 1,
 * exact in the frequency domain) to every field: out = IFFT(exp(z D) FFT(in)).
 * in, out: device complex64 [P][N_t]; may alias.  For tests and profiling.
 */
int mmf_linear(mmf_handle h, const void* in, void* out, double z);

/*
 * mmf_kerr_stage -- the Kerr evaluation as it runs inside a step (Eq. 4c, 4d): the
 * Runge-Kutta stage input is formed on the load,
 *   out = i * scale * gamma * Kerr(in0 + c1 * in1)      (in1 may be NULL: Eq. 4b, 4e),
 * with the same kernel, tiles and precision as mmf_propagate.  in0, in1, out: device
 * complex64 [P][N_t]; out must alias neither input.  Asynchronous on the handle's stream.
 * For composing other Runge-Kutta schemes from the library's stages, and for timing the
 * two-input variant that the step launches twice.
 */
int mmf_kerr_stage(mmf_handle h, const void* in0, const void* in1, double c1, void* out, double scale);

/*
 * mmf_linear_stage -- the linear step as it runs inside a step (Eq. 4a, 4b, 4f), with
 * the stage combines folded into its load and store:
 *   out = exp(z Lhat) [sum_{i < n_in} coef[i] * in[i]] + add_coef * add     (add may be NULL)
 * n_in in 1..5; in[i], add, out: device complex64 [P][N_t]; out may alias in[0] only.
 * coef: host, n_in values.  Asynchronous on the handle's stream.  Eq. 4f is
 * n_in = 4 (A_I, k1, k2, k3 with 1, 1/6, 1/3, 1/3) and add = k4 with add_coef = 1/6.
 */
int mmf_linear_stage(mmf_handle h, int n_in, const void* const* in, const double* coef, const void* add,
                     double add_coef, void* out, double z);

/*
 * mmf_amplify -- the noiseless flat-gain amplifier of a multi-span link (Section 6), plus
 * optional added white noise: fields = sqrt(power_gain) * fields + noise on every field and
 * sample.  fields: device complex64 [P][N_t], in place; noise: device complex64 [P][N_t] or
 * NULL.  Asynchronous on the handle's stream.  MMF_EINVAL for a negative or non-finite gain.
 */
int mmf_amplify(mmf_handle h, void* fields, double power_gain, const void* noise);

/* mmf_info -- P, N_t and the Kerr path chosen (0 list, 1 pairs SIMT, 3 pairs tensor core
 * row-triplet layout, 4 kappa form). */
int mmf_info(mmf_handle h, int* P, int64_t* N_t, int* kerr_path, size_t* scratch_bytes);

/*
 * mmf_energy_noalloc -- the per-field energies of mmf_energy for callers that cannot
 * allocate device memory (the paper has no counterpart; this is an interface choice).
 * Such callers run where device memory is already claimed by another framework's
 * caching allocator, or in loops where cudaMalloc/cudaFree are not allowed because
 * they synchronise the whole device.  No handle is needed and nothing is allocated:
 * the FP64 partial sums go to a buffer compiled into the library, a __device__ array of
 * MMF_NOALLOC_ENERGY_MAX doubles (128 KiB) that every GPU loading the library keeps
 * until the process exits.
 *   fields   device, complex64 [P][N_t] (N_t a power of two in [16, 131072]).
 *   out_dev  device, float64 [P]: E_f = sum_t |A_f(t)|^2 dt, W s.
 *   stream   cudaStream_t as void* (NULL = legacy default stream); asynchronous.
 * Returns MMF_EINVAL when P times the number of partial sums per field (N_t/2048,
 * clamped to 1..64) exceeds MMF_NOALLOC_ENERGY_MAX, e.g. P > 256 at N_t = 2^17.
 * The first call on a device looks up the buffer's device address (with that device
 * current) and remembers it with the device's current context; a call that finds another
 * context current (after cudaDeviceReset, or a torn-down and re-created primary context)
 * looks it up again.  Such a first call should come before any stream capture.  All calls share the one
 * buffer: calls that overlap on the GPU race on it and must be ordered by the caller.
 * Each call rewrites every partial it reads, so nothing needs clearing between calls.
 */
#define MMF_NOALLOC_ENERGY_MAX 16384
int mmf_energy_noalloc(const void* fields, int P, int64_t N_t, double dt, double* out_dev, void* stream);

/*
 * mmf_device_status -- synchronise the handle's stream and report the device status
 * word: *code = 0 when every bounded device-side wait of the handle's kernels completed,
 * else the code of the first wait that gave up (the call then returns MMF_ETIMEOUT).
 * The word is cleared by the call.
 */
int mmf_device_status(mmf_handle h, int* code);

/* mmf_destroy -- free the handle's device memory; NULL is accepted. */
int mmf_destroy(mmf_handle h);

/* mmf_last_error -- message of the last failing call on this thread ("" if none). */
const char* mmf_last_error(void);

/* ------------------------------------------------------------------------------------
 * Request server: continuous batching of many independent RK4IP propagations (a design
 * sweep over launch power, length, mode count and N_t; the paper runs one link at a time,
 * Section 5, and has no serving counterpart -- this is the method's use in many-link
 * studies).  Each request is the RK4IP of Eq. 4a-4f on its own fields with its own
 * betas, loss, dt, length and step count; requests share a registered fiber type (mode
 * count, polarisations, S_plmn, gamma, Kerr flags).
 *
 * Requests of the same shape (fiber type, N_t, step size h = L/n_steps, and whether both
 * polarisations of every mode share betas) run as slots of one device-resident pool:
 * their fields sit side by side on the time axis ([P][B][N_t]), one CUDA graph of K
 * RK4IP steps advances every occupied slot, and a step counter per slot in device memory
 * makes every kernel skip the slots that have finished.  A worker thread admits pending
 * requests whenever a slot of their pool frees up, creates pools for new shapes while
 * the HBM budget allows (freeing idle pools of other shapes to make room), keeps two
 * graphs in flight per pool, and copies finished slots out while the next graph runs.
 * A result is bitwise the same whether its request ran alone or among others: every
 * kernel computes each (field, slot) row and each time sample independently.
 * ------------------------------------------------------------------------------------ */
typedef struct mmf_server* mmf_server_handle;

/* One propagation request (all pointers host or device; UVA copies). */
typedef struct {
    int fiber;                 /* id from mmf_server_add_fiber                                 */
    const double* betas;       /* host float64 [P][4], as for mmf_create; copied at submit     */
    double alpha;              /* power attenuation, 1/m                                        */
    int64_t N_t;               /* power of two in [16, 131072]                                   */
    double dt;                 /* sample spacing, s                                              */
    double L;                  /* length, m                                                      */
    int n_steps;               /* fixed RK4IP steps (>= 1), h = L / n_steps                     */
    const void* fields_in;     /* complex64 [P][N_t]; read when the request is admitted          */
    void* fields_out;          /* complex64 [P][N_t]; written when it finishes (may equal in)   */
} mmf_request;

/* Aggregate counters of a server. */
typedef struct {
    uint64_t completed, failed;
    uint64_t pending;           /* submitted, not yet admitted                                   */
    int running, peak_running;  /* requests holding a slot now / at most so far                  */
    int pools;
    size_t bytes_in_use;        /* device memory held by the pools                               */
    double field_sample_steps;  /* sum over completed requests of P * N_t * n_steps              */
    uint64_t graph_launches;    /* graphs of K steps launched                                    */
    uint64_t kernel_launches;   /* kernels launched by those graphs and by admissions           */
} mmf_server_stats_t;

/*
 * mmf_server_create -- start a server on the current CUDA device.
 * hbm_budget_bytes  device memory the pools may hold (0 = 90 % of the free memory now).
 * max_slots         most requests running at once over all pools (0 = no limit); also
 *                   caps the slots of one pool.
 * Each pool holds B slots of 7 field copies (P*N_t*8 bytes each) plus per-slot propagator
 * rows (P or P/2 rows of N_t*16 bytes); B is chosen so that B*P*N_t is about 2^23
 * (2 <= B <= 64).  Returns MMF_ENOMEM if the worker thread cannot start.
 */
int mmf_server_create(mmf_server_handle* out, size_t hbm_budget_bytes, int max_slots);

/*
 * mmf_server_add_fiber -- register a fiber type; S_plmn (host float64 [n_modes]^4),
 * parity_class (host int32 [n_modes] or NULL) are copied; gamma and flags as for
 * mmf_create.  The tensor is validated when the first pool of the type is built: a
 * request whose pool cannot be built fails with that error.  *fiber_id receives the id.
 */
int mmf_server_add_fiber(mmf_server_handle s, int n_modes, int n_pol, const double* S_plmn,
                         const int32_t* parity_class, double gamma, unsigned flags, int* fiber_id);

/*
 * mmf_server_submit -- queue one request; returns at once with *id.  The caller keeps
 * req->fields_in readable until the request is running (mmf_server_poll state >= 1) and
 * req->fields_out writable until it is done.  Pinned host memory or device memory gives
 * asynchronous copies.  EINVAL for bad shapes or an unknown fiber.
 */
int mmf_server_submit(mmf_server_handle s, const mmf_request* req, uint64_t* id);

/*
 * mmf_server_poll -- *state = 0 pending, 1 running, 2 done, 3 failed; *latency_ms (may be
 * NULL) = submit-to-result time of a finished request (host clock), else -1.  Returns the
 * request's error code (and message) when it failed, MMF_EINVAL for an unknown id.
 */
int mmf_server_poll(mmf_server_handle s, uint64_t id, int* state, double* latency_ms);

/* mmf_server_wait -- block until the request is done or failed (timeout_s < 0: no limit;
 * MMF_ETIMEOUT when the limit passes first). */
int mmf_server_wait(mmf_server_handle s, uint64_t id, double timeout_s, double* latency_ms);

/* mmf_server_release -- forget a finished request (MMF_EBUSY while it is pending/running). */
int mmf_server_release(mmf_server_handle s, uint64_t id);

/* mmf_server_stats -- counters; returns the server's fatal error code (0 if none). */
int mmf_server_stats(mmf_server_handle s, mmf_server_stats_t* out);

/* mmf_server_destroy -- stop the worker after the graphs in flight, free every pool;
 * requests not finished are dropped.  NULL is accepted. */
int mmf_server_destroy(mmf_server_handle s);

#ifdef __cplusplus
}
#endif
#endif /* MMF_H */
