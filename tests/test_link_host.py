"""The multi-span link's receiver and noise conventions on the host (no GPU): back-to-back
recovery, the Q^2 of white noise at a known OSNR, the OSNR definition itself, and the exact
undoing of the linear part that stands for perfect dispersion compensation."""
import numpy as np

import oracle
from paper_1901_01895_gb300.link import B_REF, noise_variance, receive, white_noise
from workloads import wdm_fields_symbols
from workloads.configs import draw_betas

BAUD, SPACING = 32e9, 50e9


def test_back_to_back_recovers_the_symbols():
    for n_ch, sps in ((1, 4), (3, 8)):
        x, s = wdm_fields_symbols(2, 2, 512 * sps, sps, n_ch, BAUD, SPACING, 0.0, 5)
        q = receive(x, s, sps, BAUD, SPACING, 1.0 / (sps * BAUD))["q2_db"]
        assert q.min() > 45.0, q


def test_white_noise_q2_matches_the_osnr():
    # per polarisation, the matched filter sees SNR = P_ch/2 / (sigma^2 R_s / f_s) = OSNR * B_ref / R_s
    sps, osnr = 4, 20.0
    dt = 1.0 / (sps * BAUD)
    x, s = wdm_fields_symbols(1, 2, 4096 * sps, sps, 1, BAUD, SPACING, -1.0, 6)
    p_ch = 10 ** (-1.0 / 10) * 1e-3
    y = x + white_noise(x.shape, noise_variance(p_ch, osnr, 1.0 / dt, 2), 7)
    q = receive(y, s, sps, BAUD, SPACING, dt)["q2_db"]
    expect = 10 * np.log10(10 ** (osnr / 10) * B_REF / BAUD)
    assert np.all(np.abs(q - expect) < 0.3), (q, expect)


def test_noise_variance_is_the_osnr_definition():
    # measure the noise of both polarisations in 12.5 GHz against the channel power
    N, dt = 1 << 16, 1.0 / (8 * BAUD)
    p_ch = 2e-4
    n = white_noise((2, N), noise_variance(p_ch, 17.0, 1.0 / dt, 2), 8).astype(np.complex128)
    f = np.fft.fftfreq(N, dt)
    band = np.abs(f) < B_REF / 2
    p_noise = sum(np.sum(np.abs(np.fft.fft(n[k])[band]) ** 2) / N ** 2 for k in range(2))
    assert abs(10 * np.log10(p_ch / p_noise) - 17.0) < 0.1


def test_linear_part_is_undone_exactly():
    x, s = wdm_fields_symbols(3, 2, 1024, 8, 3, BAUD, SPACING, 0.0, 9)
    b = draw_betas(3, 2, 10)
    dt = 1.0 / (8 * BAUD)
    y = oracle.lin(oracle.lin(x, b, 0.0, dt, 160e3), b, 0.0, dt, -160e3)
    assert np.linalg.norm(y - x) / np.linalg.norm(x) < 1e-12
    assert receive(y, s, 8, BAUD, SPACING, dt)["q2_db"].min() > 45.0
