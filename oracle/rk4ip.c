/*
 * FP64 CPU oracle for the RK4IP step of the coupled multimode NLSE.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code with the CUDA
 * path and is deliberately plain and slow: every quantity is FP64, the FFT is a
 * textbook recursive radix-2 Cooley-Tukey with twiddles from cos/sin, the Kerr
 * term is a loop over the nonzero entries of the overlap tensor, and each
 * Runge-Kutta stage is computed separately in the order the paper gives it.
 *
 * Model (Section 2, Eq. 1; Kerr term in the general overlap-tensor form):
 *   dA_f/dz = Lhat A_f + Nhat_f(A),
 *   Lhat    = -alpha/2 + i sum_n (i^n / n!) beta_{n,f} d^n/dt^n          (Eq. 1)
 *   Nhat_f  = i gamma sum_{l,m,n} Sfull_{f l m n} A_l A_m conj(A_n)
 * Fields are indexed f = mode * n_pol + pol.  The polarisation-resolved tensor is
 *   Sfull_{(p a)(l b)(m c)(n d)} = S_plmn * T_abcd,
 *   T = 1                                                   for one polarisation,
 *   T_abcd = (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 3          for two (isotropic Kerr).
 *
 * Fourier convention: X_k = sum_t x_t exp(-2 pi i k t / N), x_t = (1/N) sum_k X_k exp(+2 pi i k t / N),
 * omega_k = 2 pi k / (N dt) with k in [-N/2, N/2) (the Nyquist bin is negative).
 * Then d/dt -> i omega and Eq. 1's linear operator becomes the diagonal
 *   D_f(omega) = -alpha/2 + i (beta0 - beta1 omega + beta2 omega^2 / 2 - beta3 omega^3 / 6).
 *
 * RK4IP (Section 3.2, Eq. 4a-4f), with E = exp(h/2 Lhat) applied in the frequency domain:
 *   A_I = E A
 *   k1  = E [h Nhat(A)]
 *   k2  = h Nhat(A_I + k1/2)
 *   k3  = h Nhat(A_I + k2/2)
 *   k4  = h Nhat(E (A_I + k3))
 *   A(z+h) = E (A_I + k1/6 + k2/3 + k3/3) + k4/6
 * Eq. 4b is printed with misplaced brackets; it is read as the Kerr term of A(z)
 * propagated by E, and "Nhat(X) X" in Eq. 4c-4e as the Kerr term evaluated at X.
 *
 * The symmetric split-step method with a classic RK4 nonlinear step (SSFM-RK4, Section 3.1)
 * is also provided: A(z+h) = E [RK4 of dA/dz = Nhat(A) over h] E A, E = exp(h/2 Lhat).
 *
 * For the kappa form, the split step with Agrawal's iterative nonlinear step (SSFM-Agrawal,
 * Section 3.1) is provided as well: the kappa-form nonlinear flow keeps every |A_g| constant,
 * so over a step it is the phase rotation exp(i gamma int phi dz') with phi_f = sum_g
 * kappa_fg |A_g|^2; the integral is taken by the trapezoidal rule with phi at both ends of
 * the step, phi(z+h) estimated from the step's own result and refined twice.
 *
 * The kappa form printed in Eq. 1 (SPM/XPM only, every row a spatial or polarisation
 * mode) is also provided:  Nhat_f = i gamma (sum_g kappa_fg |A_g|^2) A_f  (orc_kerr_kappa,
 * orc_propagate_kappa), with the same RK4IP.
 *
 * Parity pins (tests/test_oracle_*.py): FFT vs an O(N^2) DFT and Parseval;
 * gamma = 0 against the exact linear solution; the pure-beta1 circular shift; the
 * Gaussian-pulse beta2 broadening law; the exp(-alpha z) energy decay; the
 * dispersion-free SPM/XPM closed forms with observed 4th-order convergence (Section
 * 3.2: local error O(h^5), global O(h^4)); the fundamental soliton; pointwise
 * power conservation of the Kerr flow; dense brute-force Kerr vs the nonzero list.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------- FFT ---- */

/* Recursive radix-2 decimation-in-time DFT of length n (a power of two), in place.
 * sign = -1: forward, X_k = sum x_t e^{-2 pi i k t/n}; sign = +1: unnormalised inverse. */
static void fft_rec(cplx *x, int64_t n, int sign, cplx *tmp) {
    if (n == 1) return;
    int64_t h = n / 2;
    for (int64_t i = 0; i < h; ++i) {
        tmp[i] = x[2 * i];
        tmp[h + i] = x[2 * i + 1];
    }
    memcpy(x, tmp, (size_t)n * sizeof(cplx));
    fft_rec(x, h, sign, tmp);          /* even samples */
    fft_rec(x + h, h, sign, tmp);      /* odd samples  */
    for (int64_t k = 0; k < h; ++k) {
        double ang = sign * 2.0 * M_PI * (double)k / (double)n;
        cplx w = cos(ang) + I * sin(ang);
        cplx e = x[k], o = w * x[h + k];
        tmp[k] = e + o;
        tmp[k + h] = e - o;
    }
    memcpy(x, tmp, (size_t)n * sizeof(cplx));
}

/* In-place DFT of one row; returns 0 or -1 on a bad length / allocation failure. */
int orc_fft(cplx *x, int64_t n, int sign) {
    if (n < 1 || (n & (n - 1))) return -1;
    cplx *tmp = (cplx *)malloc((size_t)n * sizeof(cplx));
    if (!tmp) return -1;
    fft_rec(x, n, sign, tmp);
    free(tmp);
    return 0;
}

/* ------------------------------------------------- linear operator (Eq. 1) */

static double omega_of(int64_t k, int64_t n, double dt) {
    int64_t ks = (k < n / 2) ? k : k - n;     /* Nyquist bin k = n/2 maps to -n/2 */
    return 2.0 * M_PI * (double)ks / ((double)n * dt);
}

/* D_f(omega) of Eq. 1 for beta = (beta0, beta1, beta2, beta3). */
static cplx dispersion(const double *beta, double alpha, double w) {
    double im = beta[0] - beta[1] * w + beta[2] * w * w / 2.0 - beta[3] * w * w * w / 6.0;
    return -alpha / 2.0 + I * im;
}

/* out_f = IFFT( exp(z D_f(omega)) FFT(in_f) ) for every field f: the exact solution of
 * the linear part of Eq. 1 over a distance z.  in and out may alias. */
int orc_lin(int P, int64_t Nt, double dt, const double *betas /*[P][4]*/, double alpha,
            double z, const cplx *in, cplx *out) {
    int err = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : err)
    for (int f = 0; f < P; ++f) {
        cplx *row = out + (size_t)f * Nt;
        if (row != in + (size_t)f * Nt) memcpy(row, in + (size_t)f * Nt, (size_t)Nt * sizeof(cplx));
        err |= orc_fft(row, Nt, -1);
        for (int64_t k = 0; k < Nt; ++k) row[k] *= cexp(z * dispersion(betas + 4 * f, alpha, omega_of(k, Nt, dt)));
        err |= orc_fft(row, Nt, +1);
        for (int64_t k = 0; k < Nt; ++k) row[k] /= (double)Nt;
    }
    return err ? -1 : 0;
}

/* ---------------------------------------------------------- Kerr term ---- */

/* Nonzero entries of the spatial overlap tensor S[p][l][m][n] (row-major M^4). */
typedef struct {
    int M, n_pol;
    int64_t nnz;
    int32_t *idx;     /* 4 per entry: p, l, m, n */
    double *val;
} orc_kerr_list;

orc_kerr_list *orc_kerr_build(int M, int n_pol, const double *S) {
    if (M < 1 || (n_pol != 1 && n_pol != 2)) return NULL;
    int64_t total = (int64_t)M * M * M * M, nnz = 0;
    for (int64_t i = 0; i < total; ++i) nnz += (S[i] != 0.0);
    orc_kerr_list *L = (orc_kerr_list *)calloc(1, sizeof(orc_kerr_list));
    if (!L) return NULL;
    L->M = M; L->n_pol = n_pol; L->nnz = nnz;
    L->idx = (int32_t *)malloc((size_t)(4 * nnz + 4) * sizeof(int32_t));
    L->val = (double *)malloc((size_t)(nnz + 1) * sizeof(double));
    if (!L->idx || !L->val) { free(L->idx); free(L->val); free(L); return NULL; }
    int64_t e = 0;
    for (int p = 0; p < M; ++p)
        for (int l = 0; l < M; ++l)
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < M; ++n) {
                    double s = S[(((int64_t)p * M + l) * M + m) * M + n];
                    if (s == 0.0) continue;
                    L->idx[4 * e + 0] = p; L->idx[4 * e + 1] = l;
                    L->idx[4 * e + 2] = m; L->idx[4 * e + 3] = n;
                    L->val[e] = s;
                    ++e;
                }
    return L;
}

void orc_kerr_free(orc_kerr_list *L) {
    if (!L) return;
    free(L->idx); free(L->val); free(L);
}

int64_t orc_kerr_nnz(const orc_kerr_list *L) { return L ? L->nnz : -1; }

/* Kerr term at one time sample: a[f] are the P = M*n_pol field values, out[f] receives
 * i * scale * sum_{l,m,n} Sfull_{f l m n} a_l a_m conj(a_n).
 * For two polarisations the isotropic tensor T_abcd is summed out explicitly:
 *   sum_{b,c,d} T_abcd a_{l b} a_{m c} conj(a_{n d})
 *     = ( a_{l a} (a_m . conj a_n) + a_{m a} (a_l . conj a_n) + conj(a_{n a}) (a_l . a_m) ) / 3,
 * with (x . y) = sum over polarisations of x_c y_c. */
static void kerr_sample(const orc_kerr_list *L, const cplx *a, double scale, cplx *out) {
    int np = L->n_pol, P = L->M * np;
    for (int f = 0; f < P; ++f) out[f] = 0.0;
    for (int64_t e = 0; e < L->nnz; ++e) {
        int p = L->idx[4 * e], l = L->idx[4 * e + 1], m = L->idx[4 * e + 2], n = L->idx[4 * e + 3];
        double s = L->val[e];
        if (np == 1) {
            out[p] += s * a[l] * a[m] * conj(a[n]);
        } else {
            const cplx *al = a + 2 * l, *am = a + 2 * m, *an = a + 2 * n;
            cplx mn = am[0] * conj(an[0]) + am[1] * conj(an[1]);
            cplx ln = al[0] * conj(an[0]) + al[1] * conj(an[1]);
            cplx lm = al[0] * am[0] + al[1] * am[1];
            for (int pa = 0; pa < 2; ++pa)
                out[2 * p + pa] += s * (al[pa] * mn + am[pa] * ln + conj(an[pa]) * lm) / 3.0;
        }
    }
    for (int f = 0; f < P; ++f) out[f] *= I * scale;
}

/* out[f][t] = i*scale*sum Sfull A_l A_m conj(A_n) for all fields and samples (scale = gamma*h). */
int orc_kerr(const orc_kerr_list *L, int64_t Nt, double scale, const cplx *A, cplx *out) {
    if (!L) return -1;
    int P = L->M * L->n_pol;
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        cplx *a = (cplx *)malloc((size_t)P * sizeof(cplx));
        cplx *o = (cplx *)malloc((size_t)P * sizeof(cplx));
        if (!a || !o) err = 1;
        else {
#pragma omp for schedule(static)
            for (int64_t t = 0; t < Nt; ++t) {
                for (int f = 0; f < P; ++f) a[f] = A[(size_t)f * Nt + t];
                kerr_sample(L, a, scale, o);
                for (int f = 0; f < P; ++f) out[(size_t)f * Nt + t] = o[f];
            }
        }
        free(a); free(o);
    }
    return err ? -1 : 0;
}

/* Kerr term at selected samples only (the term is pointwise in t): out[f][j] for
 * t = samples[j], j < n_samples.  Lets large-P cases be checked at full N_t. */
int orc_kerr_at(const orc_kerr_list *L, int64_t Nt, double scale, const cplx *A,
                const int64_t *samples, int64_t n_samples, cplx *out) {
    if (!L) return -1;
    int P = L->M * L->n_pol;
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        cplx *a = (cplx *)malloc((size_t)P * sizeof(cplx));
        cplx *o = (cplx *)malloc((size_t)P * sizeof(cplx));
        if (!a || !o) err = 1;
        else {
#pragma omp for schedule(dynamic)
            for (int64_t j = 0; j < n_samples; ++j) {
                int64_t t = samples[j];
                for (int f = 0; f < P; ++f) a[f] = A[(size_t)f * Nt + t];
                kerr_sample(L, a, scale, o);
                for (int f = 0; f < P; ++f) out[(size_t)f * n_samples + j] = o[f];
            }
        }
        free(a); free(o);
    }
    return err ? -1 : 0;
}

/* Brute force over all P^4 field index combinations with the polarisation tensor
 * written as its Kronecker deltas; for small P only (pins the nonzero-list form). */
int orc_kerr_dense(int M, int n_pol, const double *S, int64_t Nt, double scale,
                   const cplx *A, cplx *out) {
    int P = M * n_pol;
    for (int64_t t = 0; t < Nt; ++t)
        for (int f = 0; f < P; ++f) {
            cplx acc = 0.0;
            int p = f / n_pol, a = f % n_pol;
            for (int fl = 0; fl < P; ++fl)
                for (int fm = 0; fm < P; ++fm)
                    for (int fn = 0; fn < P; ++fn) {
                        int l = fl / n_pol, b = fl % n_pol;
                        int m = fm / n_pol, c = fm % n_pol;
                        int n = fn / n_pol, d = fn % n_pol;
                        double T;
                        if (n_pol == 1) T = 1.0;
                        else T = ((a == b && c == d) + (a == c && b == d) + (a == d && b == c)) / 3.0;
                        double s = S[(((int64_t)p * M + l) * M + m) * M + n];
                        acc += s * T * A[(size_t)fl * Nt + t] * A[(size_t)fm * Nt + t] * conj(A[(size_t)fn * Nt + t]);
                    }
            out[(size_t)f * Nt + t] = I * scale * acc;
        }
    return 0;
}

/* Kerr term in the kappa form of Eq. 1: out_f(t) = i*scale*(sum_g kappa_fg |A_g(t)|^2) A_f(t),
 * kappa [P][P] row-major (the diagonal carries the intramodal kappa_aa). */
int orc_kerr_kappa(int P, int64_t Nt, const double *kappa, double scale, const cplx *A, cplx *out) {
    int err = 0;
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * P);
        if (!q) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(static)
            for (int64_t t = 0; t < Nt; ++t) {
                for (int g = 0; g < P; ++g) {
                    const cplx a = A[(size_t)g * Nt + t];
                    q[g] = creal(a) * creal(a) + cimag(a) * cimag(a);
                }
                for (int f = 0; f < P; ++f) {
                    double phi = 0.0;
                    for (int g = 0; g < P; ++g) phi += kappa[(size_t)f * P + g] * q[g];
                    out[(size_t)f * Nt + t] = I * scale * phi * A[(size_t)f * Nt + t];
                }
            }
            free(q);
        }
    }
    return err ? -1 : 0;
}

/* ---------------------------------------------------- RK4IP (Eq. 4) ---- */

typedef struct {
    int P;
    int64_t Nt;
    double dt, alpha, gamma;
    const double *betas;          /* [P][4] */
    const orc_kerr_list *kerr;    /* overlap-tensor form, or NULL for the kappa form */
    const double *kappa;          /* [P][P] (kappa form) */
    int method;                   /* 0 RK4IP (Eq. 4), 1 SSFM-RK4, 2 SSFM-Agrawal (Section 3.1) */
} fiber_t;

static int nhat(const fiber_t *F, double scale, const cplx *in, cplx *out) {
    if (F->kerr) return orc_kerr(F->kerr, F->Nt, scale, in, out);
    return orc_kerr_kappa(F->P, F->Nt, F->kappa, scale, in, out);
}

static int lin(const fiber_t *F, double z, const cplx *in, cplx *out) {
    return orc_lin(F->P, F->Nt, F->dt, F->betas, F->alpha, z, in, out);
}

/* One step of Eq. 4a-4f, in place on A (P*Nt values); work holds 5 arrays of P*Nt. */
static int rk4ip_step(const fiber_t *F, double h, cplx *A, cplx *work) {
    size_t n = (size_t)F->P * F->Nt;
    cplx *AI = work, *k1 = work + n, *k2 = work + 2 * n, *k3 = work + 3 * n, *k4 = work + 4 * n;
    int err = 0;
    err |= lin(F, h / 2, A, AI);                                   /* (4a) A_I = E A          */
    err |= nhat(F, F->gamma * h, A, k1);                                  /* h N(A)                  */
    err |= lin(F, h / 2, k1, k1);                                  /* (4b) k1 = E [h N(A)]    */
    for (size_t i = 0; i < n; ++i) k4[i] = AI[i] + k1[i] / 2.0;
    err |= nhat(F, F->gamma * h, k4, k2);                                 /* (4c) k2 = h N(A_I+k1/2) */
    for (size_t i = 0; i < n; ++i) k4[i] = AI[i] + k2[i] / 2.0;
    err |= nhat(F, F->gamma * h, k4, k3);                                 /* (4d) k3 = h N(A_I+k2/2) */
    for (size_t i = 0; i < n; ++i) A[i] = AI[i] + k3[i];
    err |= lin(F, h / 2, A, A);                                    /*      E (A_I + k3)       */
    err |= nhat(F, F->gamma * h, A, k4);                                  /* (4e) k4 = h N(...)      */
    for (size_t i = 0; i < n; ++i) A[i] = AI[i] + k1[i] / 6.0 + k2[i] / 3.0 + k3[i] / 3.0;
    err |= lin(F, h / 2, A, A);                                    /* (4f) E (A_I + ...)      */
    for (size_t i = 0; i < n; ++i) A[i] += k4[i] / 6.0;            /*      + k4/6             */
    return err ? -1 : 0;
}

/* One symmetric split step (Section 3.1): half a linear step, the nonlinear flow
 * dA/dz = Nhat(A) over h by the classic fourth-order Runge-Kutta method, half a linear step. */
static int ssfm_rk4_step(const fiber_t *F, double h, cplx *A, cplx *work) {
    size_t n = (size_t)F->P * F->Nt;
    cplx *u = work, *k1 = work + n, *k2 = work + 2 * n, *k3 = work + 3 * n, *y = work + 4 * n;
    int err = 0;
    err |= lin(F, h / 2, A, u);                                  /* exp(h/2 L) A            */
    err |= nhat(F, F->gamma * h, u, k1);                         /* k1 = h N(u)             */
    for (size_t i = 0; i < n; ++i) y[i] = u[i] + k1[i] / 2.0;
    err |= nhat(F, F->gamma * h, y, k2);                         /* k2 = h N(u + k1/2)      */
    for (size_t i = 0; i < n; ++i) y[i] = u[i] + k2[i] / 2.0;
    err |= nhat(F, F->gamma * h, y, k3);                         /* k3 = h N(u + k2/2)      */
    for (size_t i = 0; i < n; ++i) y[i] = u[i] + k3[i];
    err |= nhat(F, F->gamma * h, y, A);                          /* k4 = h N(u + k3) -> A   */
    for (size_t i = 0; i < n; ++i) y[i] = u[i] + k1[i] / 6.0 + k2[i] / 3.0 + k3[i] / 3.0 + A[i] / 6.0;
    err |= lin(F, h / 2, y, A);                                  /* exp(h/2 L) (...)        */
    return err ? -1 : 0;
}

/* phi_f(t) = sum_g kappa_fg |A_g(t)|^2 (kappa form), stored in the real parts of phi. */
static void kappa_phi(const fiber_t *F, const cplx *A, cplx *phi) {
    const int P = F->P;
    const int64_t Nt = F->Nt;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < Nt; ++t)
        for (int f = 0; f < P; ++f) {
            double s = 0.0;
            for (int g = 0; g < P; ++g) {
                const cplx a = A[(size_t)g * Nt + t];
                s += F->kappa[(size_t)f * P + g] * (creal(a) * creal(a) + cimag(a) * cimag(a));
            }
            phi[(size_t)f * Nt + t] = s;
        }
}

#define AGRAWAL_REFINE 2   /* refinements of the end-of-step phase after the first estimate */

/* One symmetric split step with the iterative nonlinear step (kappa form only):
 *   u = E A(z);  A(z+h) = E [u exp(i gamma h (phi(z) + phi(z+h)) / 2)],
 * phi(z+h) first taken equal to phi(z), then recomputed from the result AGRAWAL_REFINE times. */
static int ssfm_agrawal_step(const fiber_t *F, double h, cplx *A, cplx *work) {
    if (!F->kappa) return -1;
    size_t n = (size_t)F->P * F->Nt;
    cplx *u = work, *v = work + n, *phi0 = work + 2 * n, *phi1 = work + 3 * n;
    int err = 0;
    kappa_phi(F, A, phi0);
    err |= lin(F, h / 2, A, u);
    memcpy(phi1, phi0, n * sizeof(cplx));
    for (int it = 0; it <= AGRAWAL_REFINE && !err; ++it) {
        for (size_t i = 0; i < n; ++i) v[i] = u[i] * cexp(I * F->gamma * h * 0.5 * (creal(phi0[i]) + creal(phi1[i])));
        err |= lin(F, h / 2, v, A);
        if (it < AGRAWAL_REFINE) kappa_phi(F, A, phi1);
    }
    return err ? -1 : 0;
}

static int propagate_fiber(const fiber_t *F, cplx *A, double L, int n_steps) {
    cplx *work = (cplx *)malloc((size_t)5 * F->P * F->Nt * sizeof(cplx));
    if (!work) return -1;
    double h = L / n_steps;
    int err = 0;
    for (int s = 0; s < n_steps && !err; ++s)
        err = F->method == 2 ? ssfm_agrawal_step(F, h, A, work)
                             : (F->method == 1 ? ssfm_rk4_step(F, h, A, work) : rk4ip_step(F, h, A, work));
    free(work);
    return err;
}

/* Either Kerr form and either method: kappa != NULL selects the kappa form (P rows, S and
 * n_pol ignored), else the overlap-tensor form over M modes x n_pol; method 0 RK4IP, 1 SSFM-RK4. */
int orc_propagate_method(int method, int M, int n_pol, const double *S, const double *kappa,
                         const double *betas, double alpha, double gamma, int64_t Nt, double dt, cplx *A,
                         double L, int n_steps) {
    if (M < 1 || n_steps < 1 || Nt < 1 || (Nt & (Nt - 1)) || method < 0 || method > 2) return -1;
    if (method == 2 && !kappa) return -1;   /* the iterative step is defined for the kappa form */
    orc_kerr_list *K = NULL;
    int P = M;
    if (!kappa) {
        K = orc_kerr_build(M, n_pol, S);
        if (!K) return -1;
        P = M * n_pol;
    }
    fiber_t F = {P, Nt, dt, alpha, gamma, betas, K, kappa, method};
    int err = propagate_fiber(&F, A, L, n_steps);
    if (K) orc_kerr_free(K);
    return err;
}

/* Propagate A ([P][Nt] complex, sqrt(W)) over length L with n_steps fixed steps h = L/n_steps. */
int orc_propagate(int M, int n_pol, const double *S, const double *betas, double alpha,
                  double gamma, int64_t Nt, double dt, cplx *A, double L, int n_steps) {
    if (M < 1 || n_steps < 1 || Nt < 1 || (Nt & (Nt - 1))) return -1;
    orc_kerr_list *K = orc_kerr_build(M, n_pol, S);
    if (!K) return -1;
    fiber_t F = {M * n_pol, Nt, dt, alpha, gamma, betas, K, NULL, 0};
    int err = propagate_fiber(&F, A, L, n_steps);
    orc_kerr_free(K);
    return err;
}

/* The same propagation with the kappa form of Eq. 1 (P rows, kappa [P][P]). */
int orc_propagate_kappa(int P, const double *kappa, const double *betas, double alpha, double gamma,
                        int64_t Nt, double dt, cplx *A, double L, int n_steps) {
    if (P < 1 || n_steps < 1 || Nt < 1 || (Nt & (Nt - 1))) return -1;
    fiber_t F = {P, Nt, dt, alpha, gamma, betas, NULL, kappa, 0};
    return propagate_fiber(&F, A, L, n_steps);
}

/* Energy per field, E_f = sum_t |A_f(t)|^2 dt  [W s]. */
void orc_energy(int P, int64_t Nt, double dt, const cplx *A, double *out) {
    for (int f = 0; f < P; ++f) {
        double s = 0.0;
        for (int64_t t = 0; t < Nt; ++t) {
            cplx v = A[(size_t)f * Nt + t];
            s += creal(v) * creal(v) + cimag(v) * cimag(v);
        }
        out[f] = s * dt;
    }
}
