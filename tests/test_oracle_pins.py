"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each case is chosen so that a plausible mistake (a dropped term, a sign flip, a
wrong or conjugated index, a wrong Runge-Kutta weight) fails at least one of them:
closed-form solutions of special cases of Eq. 1, invariants of the Kerr flow, the
4th-order convergence the paper states for RK4IP (Section 3.2), brute force on tiny
inputs, and numbers printed in the paper (tests/golden/paper_numbers.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from workloads import hg_modes, overlap_tensor, gamma_from_n2, alpha_from_db_per_km, kappa_from_overlap, kappa_hg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)
W0 = 10e-6


def rng_fields(P, N, seed, scale=1.0):
    r = np.random.default_rng(seed)
    return (r.standard_normal((P, N)) + 1j * r.standard_normal((P, N))) * scale


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def zero_betas(P):
    return np.zeros((P, 4))


def smooth_fields(P, N, seed, scale, keep=8):
    """Random fields low-pass filtered to |k| < N/(2*keep): resolved by few RK4IP steps."""
    X = np.fft.fft(rng_fields(P, N, seed), axis=1)
    k = np.abs(np.fft.fftfreq(N)) * N
    X[:, k >= N / (2 * keep)] = 0
    x = np.fft.ifft(X, axis=1)
    return x * scale / np.sqrt(np.mean(abs(x) ** 2))


# ------------------------------------------------------------------ FFT ----

@pytest.mark.parametrize("N", [1, 2, 4, 8, 64, 256])
def test_fft_matches_direct_dft(N):
    x = rng_fields(1, N, N)[0]
    t = np.arange(N)
    W = np.exp(-2j * np.pi * np.outer(t, t) / N)        # textbook O(N^2) DFT matrix
    np.testing.assert_allclose(oracle.fft(x, -1), W @ x, rtol=0, atol=1e-12 * N * np.abs(x).max())
    np.testing.assert_allclose(oracle.fft(x, +1), W.conj() @ x, rtol=0, atol=1e-12 * N * np.abs(x).max())


def test_fft_large_against_numpy_and_parseval():
    x = rng_fields(1, 4096, 7)[0]
    X = oracle.fft(x, -1)
    assert relerr(X, np.fft.fft(x)) < 1e-13
    assert abs(np.sum(abs(X) ** 2) / x.size - np.sum(abs(x) ** 2)) / np.sum(abs(x) ** 2) < 1e-13
    assert relerr(oracle.fft(X, +1) / x.size, x) < 1e-14


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12), -1)


# ------------------------------------------------ linear part of Eq. 1 ----

def test_beta0_gives_pure_phase_and_loss_gives_exp_decay():
    # Eq. 1 with only beta0 and alpha: dA/dz = (-alpha/2 + i beta0) A.
    x = rng_fields(2, 64, 1)
    betas = np.array([[3.0, 0, 0, 0], [-7.5, 0, 0, 0]])
    a = alpha_from_db_per_km(0.2)
    z = 123.0
    y = oracle.lin(x, betas, a, 1e-12, z)
    expect = x * np.exp((-a / 2 + 1j * betas[:, :1]) * z)
    assert relerr(y, expect) < 1e-13


def test_beta1_is_an_exact_delay():
    # dA/dz = -beta1 dA/dt: a delay of beta1*z; chosen to be an integer number of samples.
    N, dt = 256, 1e-12
    x = rng_fields(1, N, 3)
    z = 1000.0
    shift = 5
    beta1 = shift * dt / z
    y = oracle.lin(x, np.array([[0, beta1, 0, 0]]), 0.0, dt, z)
    assert relerr(y, np.roll(x, shift, axis=1)) < 1e-12


def test_beta2_gaussian_broadening_law():
    # Textbook: an unchirped Gaussian exp(-t^2/(2 T0^2)) keeps its shape with width
    # T(z) = T0 sqrt(1 + (z/L_D)^2), L_D = T0^2/|beta2| (either sign of beta2).
    N, dt, T0 = 4096, 0.1e-12, 2e-12
    t = (np.arange(N) - N // 2) * dt
    x = np.exp(-t ** 2 / (2 * T0 ** 2))[None, :].astype(complex)
    beta2 = -21.7e-27
    LD = T0 ** 2 / abs(beta2)
    for z in (0.5 * LD, 2.0 * LD):
        y = oracle.lin(x, np.array([[0, 0, beta2, 0]]), 0.0, dt, z)[0]
        p = abs(y) ** 2
        rms = math.sqrt(np.sum(p * t ** 2) / np.sum(p))      # rms of |A|^2 is T/sqrt(2)
        assert abs(rms * math.sqrt(2) / (T0 * math.sqrt(1 + (z / LD) ** 2)) - 1) < 1e-9


def test_beta2_chirp_sign():
    # For beta2 < 0 (anomalous dispersion) the high-frequency (blue) components travel
    # faster: after propagation the leading edge (t < 0) carries the positive
    # instantaneous frequency -d(phase)/dt > 0 with the exp(-i omega t) carrier convention
    # used by Eq. 1's i^n d^n/dt^n form; equivalently the phase curvature is negative.
    N, dt, T0 = 4096, 0.1e-12, 2e-12
    t = (np.arange(N) - N // 2) * dt
    x = np.exp(-t ** 2 / (2 * T0 ** 2))[None, :].astype(complex)
    beta2 = -21.7e-27
    z = T0 ** 2 / abs(beta2)
    y = oracle.lin(x, np.array([[0, 0, beta2, 0]]), 0.0, dt, z)[0]
    ph = np.unwrap(np.angle(y))
    c = N // 2
    curvature = ph[c + 10] - 2 * ph[c] + ph[c - 10]
    # Closed form: A(z,t) ~ exp(-t^2 / (2 T0^2 (1 - i beta2 z / T0^2)));
    # phase = -t^2 (beta2 z / T0^2) / (2 T0^2 (1 + (beta2 z/T0^2)^2)): curvature sign = -sign(beta2 z)
    assert np.sign(curvature) == -np.sign(beta2 * z)


def test_beta3_airy_tail_trails():
    # Textbook third-order dispersion: for beta3 > 0 the oscillatory Airy tail forms on
    # the trailing edge (t > 0); flipping beta3 mirrors it.
    N, dt, T0 = 8192, 0.02e-12, 0.2e-12
    t = (np.arange(N) - N // 2) * dt
    x = np.exp(-t ** 2 / (2 * T0 ** 2))[None, :].astype(complex)
    beta3 = 0.1e-39 * 1e3            # 0.1 ps^3/km in s^3/m
    z = 5 * T0 ** 3 / beta3
    for sgn in (+1, -1):
        y = oracle.lin(x, np.array([[0, 0, 0, sgn * beta3]]), 0.0, dt, z)[0]
        p = abs(y) ** 2
        tail_after = p[t > 3 * T0].sum()
        tail_before = p[t < -3 * T0].sum()
        assert (tail_after > 5 * tail_before) if sgn > 0 else (tail_before > 5 * tail_after)


def test_gamma_zero_rk4ip_is_the_exact_linear_solution():
    # With gamma = 0 every k_i vanishes and Eq. 4 reduces to A(z+h) = E E A (exact).
    M, npol, N = 2, 2, 256
    S = overlap_tensor(hg_modes(1)[:M], W0)
    r = np.random.default_rng(5)
    betas = np.zeros((M * npol, 4))
    betas[:, 0] = r.uniform(-50, 50, M * npol)
    betas[:, 1] = r.uniform(-0.5e-15, 0.5e-15, M * npol)
    betas[:, 2] = -21.7e-27
    betas[:, 3] = 0.1e-39
    x = rng_fields(M * npol, N, 6, 1e-2)
    a = alpha_from_db_per_km(0.2)
    L, dt = 2000.0, 1e-12
    y = oracle.propagate(S, npol, betas, a, 0.0, dt, x, L, 7)
    X = np.fft.fft(x, axis=1)
    w = 2 * np.pi * np.fft.fftfreq(N, dt)
    D = -a / 2 + 1j * (betas[:, :1] - betas[:, 1:2] * w + betas[:, 2:3] * w ** 2 / 2 - betas[:, 3:4] * w ** 3 / 6)
    # (independent check: numpy's FFT, not the oracle's)
    expect = np.fft.ifft(X * np.exp(D * L), axis=1)
    # beta0*L reaches 1e5 rad; FP64 rounding of such a phase is ~1e-11 rad
    assert relerr(y, expect) < 1e-10


# --------------------------------------------------------- Kerr term ----

def _kappa_tensor(kappa):
    """Overlap tensor realising the paper's kappa form (Eq. 1): S_pppp = kappa_pp,
    S_ppbb = S_pbpb = kappa_pb / 2 for b != p, all other entries zero."""
    M = kappa.shape[0]
    S = np.zeros((M,) * 4)
    for p in range(M):
        S[p, p, p, p] = kappa[p, p]
        for b in range(M):
            if b != p:
                S[p, p, b, b] = kappa[p, b] / 2
                S[p, b, p, b] = kappa[p, b] / 2
    return S


@pytest.mark.parametrize("M,npol", [(2, 1), (3, 1), (2, 2), (3, 2)])
def test_kerr_list_matches_dense_brute_force(M, npol):
    S = overlap_tensor(hg_modes(2)[:M], W0)
    x = rng_fields(M * npol, 16, 11 + M + npol, 0.3)
    K = oracle.KerrList(S, npol)
    a = K(x, 0.7)
    b = oracle.kerr_dense(S, npol, x, 0.7)
    assert relerr(a, b) < 1e-13
    samples = np.array([3, 0, 15, 7])
    assert relerr(K.at(x, 0.7, samples), a[:, samples]) < 1e-15


def test_kerr_kappa_form_is_spm_plus_xpm():
    # Eq. 1's own nonlinear operator: N_a = i gamma (kappa_aa |A_a|^2 + sum_b kappa_ab |A_b|^2) A_a.
    kappa = np.array([[1.0, 0.6, 0.3], [0.6, 0.8, 0.45], [0.3, 0.45, 0.7]]) * 5e9
    x = rng_fields(3, 32, 2, 0.1)
    got = oracle.KerrList(_kappa_tensor(kappa), 1)(x, 2.0)
    expect = 1j * 2.0 * (kappa @ (abs(x) ** 2)) * x
    assert relerr(got, expect) < 1e-14


def test_kappa_oracle_matches_the_tensor_route():
    # orc_kerr_kappa (a P x P matrix-vector product per sample) against the overlap-tensor
    # list evaluating the same operator through S_ppbb = S_pbpb = kappa_pb / 2, S_pppp = kappa_pp;
    # also for a non-symmetric kappa, which the kappa-form oracle does not assume symmetric
    r = np.random.default_rng(12)
    for sym in (True, False):
        k = r.uniform(0.2, 1.0, (5, 5)) * 4e9
        if sym:
            k = (k + k.T) / 2
        x = rng_fields(5, 48, 13, 0.2)
        got = oracle.kerr_kappa(k, x, 3.0)
        ref = oracle.KerrList(_kappa_tensor(k), 1)(x, 3.0)
        assert relerr(got, ref) < 1e-14


def test_kappa_from_hg_overlaps_textbook_factors():
    # one spatial mode, two polarisations: self-phase S_0000, orthogonal-polarisation
    # cross-phase 2/3 of it (Agrawal's XPM factor for linear polarisations)
    S1 = overlap_tensor(hg_modes(0), W0)
    k = kappa_from_overlap(S1, 2)
    s0 = 1.0 / (math.pi * W0 ** 2)
    assert np.allclose(k, s0 * np.array([[1.0, 2.0 / 3.0], [2.0 / 3.0, 1.0]]), rtol=1e-12)
    # HG00 and HG10, one polarisation: cross-phase twice the overlap, S(10,10,00,00) = S_0000 / 2
    S2 = overlap_tensor(hg_modes(1)[:2], W0)
    k2 = kappa_from_overlap(S2, 1)
    assert np.isclose(k2[0, 1], s0, rtol=1e-12) and np.isclose(k2[1, 0], s0, rtol=1e-12)
    assert np.isclose(k2[1, 1], 0.75 * s0, rtol=1e-12)


def test_kappa_hg_equals_kappa_from_the_full_tensor():
    for order, npol in ((3, 2), (4, 1)):
        ms = hg_modes(order)
        assert np.allclose(kappa_hg(ms, W0, npol), kappa_from_overlap(overlap_tensor(ms, W0), npol), rtol=1e-13, atol=0)


def test_kappa_from_overlap_keeps_the_spm_xpm_part_of_the_tensor_form():
    # with the four-wave-mixing phases averaged out, the tensor form reduces to the kappa form:
    # for two fields with independent random phases the phase-averaged Kerr term of field f
    # is i gamma (sum_g kappa_fg |A_g|^2) A_f; check it by averaging over many phases
    S = overlap_tensor(hg_modes(1), W0)
    k = kappa_from_overlap(S, 1)
    r = np.random.default_rng(3)
    amp = np.array([0.7, 1.1, 0.9])
    acc = np.zeros(3, complex)
    n = 4000
    for _ in range(n):
        ph = np.exp(2j * np.pi * r.random(3))
        x = (amp * ph)[:, None]
        kt = oracle.KerrList(S, 1)(x, 1.0)[:, 0]
        acc += kt / ph                       # phase of A_f removed: the XPM part survives the average
    expect = 1j * (k @ amp ** 2) * amp
    assert np.allclose(acc / n, expect, rtol=0.05, atol=0.05 * np.abs(expect).max())


def test_isotropic_polarisation_tensor_textbook_cases():
    # Single spatial mode, two polarisations, isotropic Kerr medium (textbook):
    #   N_x = i g (|A_x|^2 + 2/3 |A_y|^2) A_x + i g/3 A_y^2 conj(A_x),
    # so linear polarisation sees the full SPM coefficient and circular polarisation 2/3 of it.
    S = np.full((1, 1, 1, 1), 4e9)
    K = oracle.KerrList(S, 2)
    r = np.random.default_rng(9)
    ax = r.standard_normal(8) + 1j * r.standard_normal(8)
    ay = r.standard_normal(8) + 1j * r.standard_normal(8)
    x = np.stack([ax, ay])
    got = K(x, 1.0)
    nx = 1j * 4e9 * ((abs(ax) ** 2 + 2 / 3 * abs(ay) ** 2) * ax + ay ** 2 * ax.conj() / 3)
    ny = 1j * 4e9 * ((abs(ay) ** 2 + 2 / 3 * abs(ax) ** 2) * ay + ax ** 2 * ay.conj() / 3)
    assert relerr(got, np.stack([nx, ny])) < 1e-14
    circ = np.stack([ax / math.sqrt(2), 1j * ax / math.sqrt(2)])
    got = K(circ, 1.0)
    assert relerr(got, 1j * 4e9 * (2 / 3) * abs(ax) ** 2 * circ) < 1e-14


def test_kerr_power_flow_is_conservative_pointwise():
    # For a real, fully symmetric S the Kerr flow conserves sum_f |A_f(t)|^2 at every t:
    # sum_f Re(conj(A_f) N_f) = 0 sample by sample.
    S = overlap_tensor(hg_modes(2), W0)
    for npol in (1, 2):
        x = rng_fields(S.shape[0] * npol, 64, 4 + npol, 0.2)
        nl = oracle.KerrList(S, npol)(x, 1.0)
        flow = np.real(np.sum(x.conj() * nl, axis=0))
        scale = np.sum(abs(x.conj() * nl), axis=0)
        assert np.max(abs(flow) / scale) < 1e-13


# ----------------------------------------------------- RK4IP (Eq. 4) ----

def _xpm_case():
    kappa = np.array([[1.0, 0.6, 0.3], [0.6, 0.8, 0.45], [0.3, 0.45, 0.7]]) * 1.0 / (math.pi * W0 ** 2)
    S = _kappa_tensor(kappa)
    x = rng_fields(3, 16, 21, 1.0)          # ~2 W per field: order-1 radian nonlinear phase
    L = 2000.0
    exact = x * np.exp(1j * GAMMA * (kappa @ abs(x) ** 2) * L)
    return S, x, L, exact


def test_rk4ip_xpm_closed_form_and_fourth_order():
    # Dispersion-free kappa-form: |A_b| is invariant, so A_a(z) = A_a(0) exp(i gamma sum_b kappa_ab |A_b(0)|^2 z).
    S, x, L, exact = _xpm_case()
    errs = []
    for n in (16, 32, 64):
        y = oracle.propagate(S, 1, zero_betas(3), 0.0, GAMMA, 1e-12, x, L, n)
        errs.append(relerr(y, exact))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-5
    for o in orders:
        assert 3.8 < o < 4.2, (errs, orders)


def test_rk4ip_kappa_form_closed_form_and_fourth_order():
    # the kappa-form propagator: dispersion-free solution A_f(z) = A_f(0) exp(i gamma sum_g kappa_fg |A_g(0)|^2 z)
    kappa = np.array([[1.0, 0.6, 0.3], [0.6, 0.8, 0.45], [0.3, 0.45, 0.7]]) * 1.0 / (math.pi * W0 ** 2)
    x = rng_fields(3, 16, 21, 1.0)
    L = 2000.0
    exact = x * np.exp(1j * GAMMA * (kappa @ abs(x) ** 2) * L)
    errs = [relerr(oracle.propagate_kappa(kappa, zero_betas(3), 0.0, GAMMA, 1e-12, x, L, n), exact)
            for n in (16, 32, 64)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-5
    for o in orders:
        assert 3.8 < o < 4.2, (errs, orders)


def test_rk4ip_kappa_form_matches_tensor_route_with_dispersion():
    # the same RK4IP with the two Kerr evaluations: kappa matrix vs its overlap-tensor realisation
    kappa = kappa_from_overlap(overlap_tensor(hg_modes(1), W0), 2)
    P = kappa.shape[0]
    b = np.zeros((P, 4))
    b[:, 1] = np.repeat([0.0, 0.3e-15, -0.2e-15], 2)
    b[:, 2] = -21.7e-27
    x = smooth_fields(P, 256, 5, 0.3)
    a = oracle.propagate_kappa(kappa, b, 1e-5, GAMMA, 1e-12, x, 300.0, 6)
    r = oracle.propagate(_kappa_tensor(kappa), 1, b, 1e-5, GAMMA, 1e-12, x, 300.0, 6)
    assert relerr(a, r) < 1e-13


def test_ssfm_rk4_gamma_zero_is_the_exact_linear_solution():
    # two half linear steps per step compose to exp(h Lhat): exact for any step count
    P, N = 3, 256
    b = np.zeros((P, 4))
    b[:, 0] = [3.0, -2.0, 0.5]
    b[:, 1] = [0.4e-15, -0.1e-15, 0.0]
    b[:, 2] = -21.7e-27
    x = smooth_fields(P, N, 8, 0.1)
    exact = oracle.lin(x, b, 2e-5, 1e-12, 700.0)
    y = oracle.propagate(np.zeros((P, P, P, P)), 1, b, 2e-5, 0.0, 1e-12, x, 700.0, 7, method="ssfm-rk4")
    assert relerr(y, exact) < 1e-12


def test_ssfm_rk4_without_dispersion_is_classic_rk4_like_rk4ip():
    # with Lhat = 0 both methods are the classic RK4 of dA/dz = Nhat(A): identical up to rounding
    S, x, L, exact = _xpm_case()
    a = oracle.propagate(S, 1, zero_betas(3), 0.0, GAMMA, 1e-12, x, L, 32, method="ssfm-rk4")
    r = oracle.propagate(S, 1, zero_betas(3), 0.0, GAMMA, 1e-12, x, L, 32)
    assert relerr(a, r) < 1e-13
    assert relerr(a, exact) < 1e-4


def test_ssfm_rk4_is_second_order_rk4ip_fourth_with_dispersion():
    # Section 3.1: the symmetric split step has a global error O(h^2) (splitting error);
    # RK4IP is O(h^4).  Walk-off (beta1) and dispersion against cross-phase modulation.
    kappa = np.array([[1.0, 0.7], [0.7, 0.9]]) / (math.pi * W0 ** 2)
    b = np.zeros((2, 4))
    b[:, 1] = [2.0e-15, -2.0e-15]
    b[:, 2] = -21.7e-27
    x = smooth_fields(2, 256, 17, 0.3, keep=16)
    dt, L = 2e-12, 2000.0
    ref = oracle.propagate_kappa(kappa, b, 0.0, GAMMA, dt, x, L, 2048)
    e_ss = [relerr(oracle.propagate_kappa(kappa, b, 0.0, GAMMA, dt, x, L, n, method="ssfm-rk4"), ref)
            for n in (16, 32, 64)]
    e_ip = [relerr(oracle.propagate_kappa(kappa, b, 0.0, GAMMA, dt, x, L, n), ref) for n in (16, 32)]
    o_ss = [math.log2(e_ss[i] / e_ss[i + 1]) for i in range(2)]
    o_ip = math.log2(e_ip[0] / e_ip[1])
    assert all(1.8 < o < 2.2 for o in o_ss), (e_ss, o_ss)
    assert 3.6 < o_ip < 4.4, (e_ip, o_ip)
    assert e_ip[0] < e_ss[0] / 10     # the paper's reason to prefer RK4IP at equal step size


def test_ssfm_agrawal_limits_and_second_order():
    # kappa form: with no dispersion the trapezoidal phase of a constant phi is exact;
    # with gamma = 0 the two half steps compose to the exact linear solution; with both,
    # the splitting error makes it globally second order (Section 3.1)
    kappa = np.array([[1.0, 0.7], [0.7, 0.9]]) / (math.pi * W0 ** 2)
    x = smooth_fields(2, 256, 17, 0.3, keep=16)
    exact = x * np.exp(1j * GAMMA * (kappa @ abs(x) ** 2) * 2000.0)
    y = oracle.propagate_kappa(kappa, zero_betas(2), 0.0, GAMMA, 2e-12, x, 2000.0, 3, method="ssfm-agrawal")
    assert relerr(y, exact) < 1e-13
    b = np.zeros((2, 4))
    b[:, 1] = [2.0e-15, -2.0e-15]
    b[:, 2] = -21.7e-27
    lin_exact = oracle.lin(x, b, 1e-5, 2e-12, 2000.0)
    y = oracle.propagate_kappa(kappa, b, 1e-5, 0.0, 2e-12, x, 2000.0, 5, method="ssfm-agrawal")
    assert relerr(y, lin_exact) < 1e-12
    ref = oracle.propagate_kappa(kappa, b, 0.0, GAMMA, 2e-12, x, 2000.0, 2048)
    e = [relerr(oracle.propagate_kappa(kappa, b, 0.0, GAMMA, 2e-12, x, 2000.0, n, method="ssfm-agrawal"), ref)
         for n in (16, 32, 64)]
    o = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(1.8 < v < 2.2 for v in o), (e, o)


def test_rk4ip_spm_modulus_and_phase():
    # Single HG00 mode, no dispersion: |A| constant, phase gamma S_0000 |A|^2 z.
    S = overlap_tensor(hg_modes(0), W0)
    assert abs(GAMMA * S[0, 0, 0, 0] * 1e3 - 0.3355) < 1e-3      # 0.3355 1/(W km) at w = 10 um
    x = rng_fields(1, 32, 8, 0.3)          # up to ~1.5 W: ~0.5 rad nonlinear phase over 1 km
    L = 1000.0
    y = oracle.propagate(S, 1, zero_betas(1), 0.0, GAMMA, 1e-12, x, L, 64)
    exact = x * np.exp(1j * GAMMA * S[0, 0, 0, 0] * abs(x) ** 2 * L)
    assert relerr(y, exact) < 1e-7
    assert np.max(abs(abs(y) - abs(x)) / abs(x)) < 1e-7


def test_rk4ip_fundamental_soliton():
    # N = 1 soliton: sqrt(P0) sech(t/T0) with P0 = |beta2| / (gamma S T0^2) keeps its shape
    # and gains the phase gamma S P0 z / 2 (textbook; needs beta2 < 0 and the 1/2 of Eq. 1's n = 2 term).
    S = overlap_tensor(hg_modes(0), W0)
    gS = GAMMA * S[0, 0, 0, 0]
    T0, beta2 = 1e-12, -21.7e-27
    P0 = abs(beta2) / (gS * T0 ** 2)
    N, dt = 2048, 0.05e-12
    t = (np.arange(N) - N // 2) * dt
    x = (math.sqrt(P0) / np.cosh(t / T0))[None, :].astype(complex)
    L = 2 * T0 ** 2 / abs(beta2)
    y = oracle.propagate(S, 1, np.array([[0, 0, beta2, 0]]), 0.0, GAMMA, dt, x, L, 400)
    exact = x * np.exp(1j * gS * P0 * L / 2)
    assert relerr(y, exact) < 1e-6
    # the wrong sign of beta2 destroys the soliton
    y_bad = oracle.propagate(S, 1, np.array([[0, 0, -beta2, 0]]), 0.0, GAMMA, dt, x, L, 400)
    assert relerr(y_bad, exact) > 0.1


def test_rk4ip_dispersive_fwm_fourth_order_and_energy():
    # Full multimode case (dispersion + intermodal four-wave mixing, two polarisations):
    # global error O(h^4) against a fine-step run, and total energy conserved (lossless).
    S = overlap_tensor(hg_modes(1), W0)
    M, npol, N = 3, 2, 128
    r = np.random.default_rng(12)
    betas = np.zeros((M * npol, 4))
    betas[:, 0] = np.repeat(r.uniform(-0.005, 0.005, M), npol)   # phase-matched FWM is resolved
    betas[:, 1] = np.repeat(r.uniform(-0.5e-15, 0.5e-15, M), npol)
    betas[:, 2] = -21.7e-27
    dt = 0.5e-12
    x = smooth_fields(M * npol, N, 13, 1.0)                          # ~1 W: order-1 rad over L
    L = 500.0
    ref = oracle.propagate(S, npol, betas, 0.0, GAMMA, dt, x, L, 1024)
    errs = [relerr(oracle.propagate(S, npol, betas, 0.0, GAMMA, dt, x, L, n), ref) for n in (32, 64, 128)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for o in orders:
        assert 3.7 < o < 4.3, (errs, orders)
    e0, e1 = oracle.energy(x, dt).sum(), oracle.energy(ref, dt).sum()
    assert abs(e1 / e0 - 1) < 1e-9


def test_loss_energy_decay_with_kerr():
    # d/dz sum|A|^2 = -alpha sum|A|^2 exactly (the Kerr flow is conservative).
    S = overlap_tensor(hg_modes(1), W0)
    betas = np.zeros((6, 4)); betas[:, 2] = -21.7e-27
    a = alpha_from_db_per_km(0.2)
    x = smooth_fields(6, 64, 14, 0.1)
    L = 5000.0
    y = oracle.propagate(S, 2, betas, a, GAMMA, 1e-12, x, L, 50)
    ratio = oracle.energy(y, 1e-12).sum() / oracle.energy(x, 1e-12).sum()
    assert abs(ratio / math.exp(-a * L) - 1) < 1e-8


def test_energy_absolute_scale_closed_forms():
    # The pulse energy int |A(t)|^2 dt in W*s, not only its ratios: a sampled sum over a
    # wide window of smooth, fast-decaying pulses equals the integral to rounding.
    #   sech:      int P0 sech^2(t/T0) dt = 2 P0 T0
    #   Gaussian:  int P0 exp(-t^2/T0^2) dt = sqrt(pi) P0 T0
    # A dropped or doubled dt, a missing square or a sum over the wrong axis fails here.
    N, dt = 1 << 14, 0.125e-12
    t = (np.arange(N) - N // 2) * dt
    P0, T0 = 2.5e-3, 3.0e-12
    sech = np.sqrt(P0) / np.cosh(t / T0)
    gauss = np.sqrt(P0) * np.exp(-t ** 2 / (2 * T0 ** 2)) * np.exp(1j * 0.3 * t / T0)
    e = oracle.energy(np.stack([sech, gauss, 2 * gauss]), dt)
    assert abs(e[0] / (2 * P0 * T0) - 1) < 1e-12
    assert abs(e[1] / (math.sqrt(math.pi) * P0 * T0) - 1) < 1e-12
    assert abs(e[2] / (4 * math.sqrt(math.pi) * P0 * T0) - 1) < 1e-12


# --------------------------------------------- inputs and paper numbers ----

def test_hg_overlap_closed_forms():
    modes = hg_modes(1)
    S = overlap_tensor(modes, W0)
    S0 = 1 / (math.pi * W0 ** 2)                                  # Int exp(-4r^2/w^2) / (Int exp(-2r^2/w^2))^2
    assert abs(S[0, 0, 0, 0] / S0 - 1) < 1e-13
    assert abs(S[1, 1, 1, 1] / S0 - 0.75) < 1e-13                 # HG10: 3/4
    assert abs(S[1, 1, 0, 0] / S0 - 0.5) < 1e-13                  # HG10,HG10,HG00,HG00: 1/2
    assert S[1, 0, 0, 0] == 0 and S[1, 2, 0, 0] == 0              # odd parity vanishes
    assert [len(hg_modes(g)) for g in (1, 4, 8, 14)] == [3, 15, 45, 120]
    big = overlap_tensor(hg_modes(6), W0)
    for perm in [(1, 0, 2, 3), (0, 2, 1, 3), (3, 1, 2, 0), (2, 3, 0, 1)]:
        assert np.max(abs(big - big.transpose(perm))) <= 1e-12 * big.max()
    assert 0.24 < np.mean(big != 0) < 0.27


def test_paper_printed_numbers():
    g = json.load(open(GOLDEN))
    ge = g["gamma_example"]
    f0 = 0.5 * (ge["f_low_THz"] + ge["f_high_THz"]) * 1e12
    lam = 299792458.0 / f0
    gamma = gamma_from_n2(ge["n2_m2_per_W"], lam) / (ge["A_eff_um2"] * 1e-12) * 1e3
    assert round(gamma, ge["printed_digits"]) == ge["gamma_per_W_km"]
    sm = g["signal_matrix_bytes"]
    N = sm["N_s"] * sm["N_sps"]
    assert sm["rows"] * N * 16 / 2 ** 20 == sm["MiB_complex_fp64"]
    assert sm["rows"] * N * 8 / 2 ** 20 == sm["MiB_abs2_fp64"]
    for sps, span in g["spectral_range"]["cases"]:
        assert sps * g["spectral_range"]["baud"] == span
    k = g["kappa_upper_triangle"]
    assert (2 * k["M"]) ** 2 // 2 + k["M"] == k["count"]
