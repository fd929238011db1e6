"""The symmetric split-step method with an RK4 nonlinear step (SSFM-RK4, Section 3.1;
MMF_METHOD_SSFM_RK4) on the GPU against the same method in the FP64 oracle, for the
overlap-tensor Kerr term (CUDA cores and tensor cores) and for the kappa form."""
import numpy as np
import pytest

import oracle
import paper_1901_01895_gb300 as mmf
from workloads import make_workload, hg_modes, overlap_tensor, parity_classes, kappa_hg, gamma_from_n2
from workloads.configs import draw_betas

from gpu_util import torch, require_gpu, to_dev, to_host, relerr, rng_fields, stream_ptr

pytestmark = pytest.mark.gpu
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)
SSFM = mmf.MMF_METHOD_SSFM_RK4


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def test_ssfm_rk4_three_modes_vs_oracle():
    wl = make_workload("c0", n_steps=25, L=250.0)
    ref = oracle.propagate(wl.S, wl.n_pol, wl.betas, wl.alpha, wl.gamma, wl.dt, wl.fields, wl.L, wl.n_steps,
                           method="ssfm-rk4")
    f = mmf.Fiber.from_workload(wl, flags=SSFM, stream=stream_ptr())
    xd = to_dev(wl.fields)
    f.propagate(xd.data_ptr(), wl.L, wl.n_steps)
    err = relerr(to_host(xd), ref)
    print(f"ssfm-rk4 c0 25 steps: rel {err:.2e}")
    assert err < 1e-5
    f.close()


@pytest.mark.parametrize("prec,tol", [(mmf.MMF_KERR_FP32, 1e-5), (mmf.MMF_KERR_BF16X3, 1e-5)])
def test_ssfm_rk4_fifteen_modes_two_pol_vs_oracle(prec, tol):
    ms = hg_modes(4)
    S = overlap_tensor(ms, 10e-6)
    b = draw_betas(15, 2, 3)
    N = 512
    x = rng_fields(30, N, 4, 0.02).astype(np.complex64).astype(np.complex128)
    dt = 0.9765625e-12
    ref = oracle.propagate(S, 2, b, 4.6e-5, GAMMA, dt, x, 100.0, 10, method="ssfm-rk4")
    f = mmf.Fiber(15, 2, S, parity_classes(ms), b, 4.6e-5, GAMMA, N, dt, prec | SSFM, stream_ptr())
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), 100.0, 10)
    assert f.device_status() == 0
    err = relerr(to_host(xd), ref)
    print(f"ssfm-rk4 15 x 2 prec {prec}: rel {err:.2e}")
    assert err < tol
    f.close()


def test_ssfm_rk4_kappa_form_vs_oracle():
    k = kappa_hg(hg_modes(4), 10e-6, 2)
    b = draw_betas(15, 2, 6)
    N = 1024
    dt = 0.9765625e-12
    x = rng_fields(30, N, 7, 0.03).astype(np.complex64).astype(np.complex128)
    ref = oracle.propagate_kappa(k, b, 0.0, GAMMA, dt, x, 300.0, 30, method="ssfm-rk4")
    f = mmf.Fiber.from_kappa(k, b, 0.0, GAMMA, N, dt, SSFM, stream_ptr())
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), 300.0, 30)
    err = relerr(to_host(xd), ref)
    print(f"ssfm-rk4 kappa 30 rows: rel {err:.2e}")
    assert err < 1e-5
    f.close()


@pytest.mark.parametrize("order,N,steps", [(4, 1024, 30), (14, 256, 6)])
def test_ssfm_agrawal_kappa_form_vs_oracle(order, N, steps):
    """The iterative split step (kappa form) at 30 and 240 rows with dispersion and loss."""
    ms = hg_modes(order)
    k = kappa_hg(ms, 10e-6, 2)
    P = k.shape[0]
    b = draw_betas(len(ms), 2, 8)
    dt = 0.9765625e-12
    x = rng_fields(P, N, 9, 0.03).astype(np.complex64).astype(np.complex128)
    L = steps * 10.0
    ref = oracle.propagate_kappa(k, b, 2e-5, GAMMA, dt, x, L, steps, method="ssfm-agrawal")
    f = mmf.Fiber.from_kappa(k, b, 2e-5, GAMMA, N, dt, mmf.MMF_METHOD_SSFM_AGRAWAL, stream_ptr())
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), L, steps)
    err = relerr(to_host(xd), ref)
    print(f"ssfm-agrawal kappa P={P} N={N}: rel {err:.2e}")
    assert err < 1e-5
    f.close()


def test_ssfm_agrawal_dispersion_free_is_exact():
    k = kappa_hg(hg_modes(2), 10e-6, 2)
    P, N = k.shape[0], 512
    x = rng_fields(P, N, 10, 0.2)
    L = 800.0
    exact = x * np.exp(1j * GAMMA * (k @ np.abs(x) ** 2) * L)
    f = mmf.Fiber.from_kappa(k, np.zeros((P, 4)), 0.0, GAMMA, N, 1e-12, mmf.MMF_METHOD_SSFM_AGRAWAL, stream_ptr())
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), L, 4)
    err = relerr(to_host(xd), exact)
    print(f"ssfm-agrawal closed form: rel {err:.2e}")
    assert err < 2e-6
    f.close()


def test_unknown_method_is_rejected():
    wl = make_workload("c0", N_t=256)
    with pytest.raises(mmf.MMFError) as e:
        mmf.Fiber.from_workload(wl, flags=3 << 7, stream=stream_ptr())
    assert e.value.code == mmf.MMF_EINVAL
    with pytest.raises(mmf.MMFError) as e:      # the iterative step is defined for the kappa form only
        mmf.Fiber.from_workload(wl, flags=mmf.MMF_METHOD_SSFM_AGRAWAL, stream=stream_ptr())
    assert e.value.code == mmf.MMF_EINVAL
