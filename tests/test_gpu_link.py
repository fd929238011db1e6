"""Multi-span link (Section 6) through the GPU path vs the same link with every span propagated
by the FP64 oracle: fields and Q^2 per mode and channel."""
import numpy as np
import pytest

import oracle
import paper_1901_01895_gb300 as mmf
from paper_1901_01895_gb300.link import Link, noise_variance, receive, white_noise
from workloads import hg_modes, kappa_hg, gamma_from_n2, alpha_from_db_per_km, wdm_fields_symbols
from workloads.configs import draw_betas

from gpu_util import torch, require_gpu, to_dev, to_host, relerr, stream_ptr

pytestmark = pytest.mark.gpu
BAUD, SPACING = 32e9, 50e9
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)
ALPHA = alpha_from_db_per_km(0.23)


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def oracle_link(kappa, betas, x, dt, span, n_spans, steps, noise):
    y = x.astype(np.complex128)
    g = np.exp(ALPHA * span / 2)
    for k in range(n_spans):
        y = oracle.propagate_kappa(kappa, betas, ALPHA, GAMMA, dt, y, span, steps) * g
    y = y + noise.astype(np.complex128)
    return oracle.lin(y, betas, 0.0, dt, -span * n_spans)


@pytest.mark.parametrize("power_dbm,osnr", [(-1.0, 20.0), (6.0, None)])
def test_link_gpu_matches_oracle_link(power_dbm, osnr):
    modes = hg_modes(1)
    M, npol, sps, nsym = len(modes), 2, 8, 256
    N, dt = nsym * sps, 1.0 / (sps * BAUD)
    kappa = kappa_hg(modes, 10e-6, npol)
    betas = draw_betas(M, npol, 21)
    x, syms = wdm_fields_symbols(M, npol, N, sps, 3, BAUD, SPACING, power_dbm, 22)
    span, n_spans, steps = 20e3, 2, 40
    sigma2 = 0.0 if osnr is None else noise_variance(10 ** (power_dbm / 10) * 1e-3, osnr, 1 / dt, npol)
    noise = white_noise(x.shape, sigma2, 23)
    link = Link(span, n_spans, steps, kappa=kappa, n_pol=npol, betas=betas, alpha=ALPHA, gamma=GAMMA, N_t=N, dt=dt,
                stream=stream_ptr())
    xd, nd = to_dev(x), to_dev(noise)
    link.transmit(xd.data_ptr(), nd.data_ptr())
    y = to_host(xd)
    link.close()
    ref = oracle_link(kappa, betas, x.astype(np.complex64), dt, span, n_spans, steps, noise)
    err = relerr(y, ref)
    q = receive(y, syms, sps, BAUD, SPACING, dt)["q2_db"]
    q_ref = receive(ref, syms, sps, BAUD, SPACING, dt)["q2_db"]
    print(f"link {power_dbm} dBm, OSNR {osnr}: fields rel {err:.2e}, Q2 {q.mean():.2f} dB "
          f"(oracle {q_ref.mean():.2f}), max |dQ2| {np.abs(q - q_ref).max():.3f} dB")
    assert err < 2e-5
    assert np.abs(q - q_ref).max() < 0.05


def test_link_linear_is_transparent_and_power_degrades_q2():
    modes = hg_modes(1)
    M, npol, sps, nsym = len(modes), 2, 8, 512
    N, dt = nsym * sps, 1.0 / (sps * BAUD)
    kappa = kappa_hg(modes, 10e-6, npol)
    betas = draw_betas(M, npol, 31)
    q = {}
    for p_dbm, gamma in ((0.0, 0.0), (0.0, GAMMA), (8.0, GAMMA)):
        x, syms = wdm_fields_symbols(M, npol, N, sps, 3, BAUD, SPACING, p_dbm, 32)
        link = Link(40e3, 2, 80, kappa=kappa, n_pol=npol, betas=betas, alpha=ALPHA, gamma=gamma, N_t=N, dt=dt,
                    stream=stream_ptr())
        xd = to_dev(x)
        link.transmit(xd.data_ptr())
        q[(p_dbm, gamma)] = receive(to_host(xd), syms, sps, BAUD, SPACING, dt)["q2_db"]
        link.close()
    print({k: round(float(v.mean()), 2) for k, v in q.items()})
    assert q[(0.0, 0.0)].min() > 40.0                          # no nonlinearity: only FP32 round-off
    assert q[(8.0, GAMMA)].mean() < q[(0.0, GAMMA)].mean() - 3  # Kerr impairment grows with power


def test_amplify_validates_and_scales():
    modes = hg_modes(0)
    f = mmf.Fiber(1, 2, np.ones((1, 1, 1, 1)), None, np.zeros((2, 4)), 0.0, GAMMA, 64, 1e-12, 0, stream_ptr())
    x = np.ones((2, 64), np.complex64) * (1 + 1j)
    xd = to_dev(x)
    nd = to_dev(np.full((2, 64), 0.5, np.complex64))
    f.amplify(xd.data_ptr(), 4.0, nd.data_ptr())
    assert np.allclose(to_host(xd), 2 * x + 0.5)
    with pytest.raises(mmf.MMFError):
        f.amplify(xd.data_ptr(), -1.0)
    f.close()
