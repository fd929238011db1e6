"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances follow from FP32 arithmetic: one FFT pair with double-float twiddles
keeps a relative error of a few 1e-7 (log2 N roundings of 6e-8); one Kerr
evaluation in FP32 a few 1e-7 of its magnitude; a propagation of n steps adds
these roundings randomly, so the end-to-end bound is the 1e-5 parity target for the
100-step three-mode case.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1901_01895_gb300 as mmf
from workloads import make_workload, hg_modes, overlap_tensor, parity_classes, gamma_from_n2, alpha_from_db_per_km

from gpu_util import torch, require_gpu, to_dev, to_host, relerr, rng_fields, stream_ptr

pytestmark = pytest.mark.gpu
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)


def fiber(M_order, n_pol, N, dt=1e-12, alpha=0.0, seed=3, modes=None, flags=0):
    ms = hg_modes(M_order) if modes is None else modes
    M = len(ms)
    S = overlap_tensor(ms, 10e-6)
    r = np.random.default_rng(seed)
    b = np.zeros((M * n_pol, 4))
    b0 = r.uniform(-50, 50, M)
    b1 = r.uniform(-0.5e-15, 0.5e-15, M)
    for m in range(M):
        for a in range(n_pol):
            b[m * n_pol + a] = (b0[m], b1[m], -21.7e-27, 0.0)
    f = mmf.Fiber(M, n_pol, S, parity_classes(ms), b, alpha, GAMMA, N, dt, flags, stream_ptr())
    return f, S, b


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("logN", list(range(4, 18)))
def test_linear_operator_vs_oracle(logN):
    N = 1 << logN
    f, S, b = fiber(1, 2, N, dt=0.5e-12, alpha=alpha_from_db_per_km(0.2))
    x = rng_fields(f.P, N, logN, 0.03)
    z = 37.5
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    f.linear(xd.data_ptr(), yd.data_ptr(), z)
    y = to_host(yd)
    ref = oracle.lin(x.astype(np.complex64).astype(np.complex128), b, alpha_from_db_per_km(0.2), 0.5e-12, z)
    err = relerr(y, ref)
    assert err < 2e-6 * max(1.0, logN / 12), err
    # in place gives the same bits
    f.linear(xd.data_ptr(), xd.data_ptr(), z)
    assert np.array_equal(to_host(xd), y)
    f.close()


@pytest.mark.parametrize("algo", [mmf.MMF_KERR_LIST, mmf.MMF_KERR_AUTO])
@pytest.mark.parametrize("order,n_pol", [(1, 1), (1, 2), (2, 1), (2, 2), (4, 2)])
def test_kerr_vs_oracle(order, n_pol, algo):
    N = 1024 + 0   # several sample tiles
    f, S, b = fiber(order, n_pol, N, flags=algo)
    assert f.info()["kerr_path"] == ("list" if algo == mmf.MMF_KERR_LIST else "pairs-simt")
    x = rng_fields(f.P, N, 11 * order + n_pol, 0.05).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    h = 10.0
    f.kerr(xd.data_ptr(), yd.data_ptr(), h)
    y = to_host(yd)
    ref = oracle.KerrList(S, n_pol)(x, GAMMA * h)
    assert relerr(y, ref) < 2e-6
    f.close()


def _kappa_tensor(kappa):
    M = kappa.shape[0]
    S = np.zeros((M,) * 4)
    for p in range(M):
        S[p, p, p, p] = kappa[p, p]
        for q in range(M):
            if q != p:
                S[p, p, q, q] = kappa[p, q] / 2
                S[p, q, p, q] = kappa[p, q] / 2
    return S


@pytest.mark.parametrize("n_pol", [1, 2])
def test_kerr_kappa_form_takes_list_path(n_pol):
    # The paper's own operator (Eq. 1): S is not fully symmetric, so the pair
    # contraction does not apply and the general list path must be chosen.
    kappa = np.array([[1.0, 0.6, 0.3], [0.6, 0.8, 0.45], [0.3, 0.45, 0.7]]) / (np.pi * 1e-10)
    S = _kappa_tensor(kappa)
    N = 512
    b = np.zeros((3 * n_pol, 4))
    f = mmf.Fiber(3, n_pol, S, None, b, 0.0, GAMMA, N, 1e-12, 0, stream_ptr())
    assert f.info()["kerr_path"] == "list"
    x = rng_fields(3 * n_pol, N, 4, 0.2).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 5.0)
    assert relerr(to_host(yd), oracle.KerrList(S, n_pol)(x, GAMMA * 5.0)) < 2e-6
    with pytest.raises(mmf.MMFError):
        mmf.Fiber(3, n_pol, S, None, b, 0.0, GAMMA, N, 1e-12, mmf.MMF_KERR_PAIRS, stream_ptr())
    f.close()


@pytest.mark.parametrize("order,n_samples", [(8, 256), (14, 24)])
def test_kerr_pairs_full_size_sampled(order, n_samples):
    # 45 and 120 HG modes x 2 pol at N_t = 2^17: the Kerr term is pointwise in t, so the
    # oracle evaluated at seeded random samples checks those samples exactly.
    N = 1 << 17
    f, S, b = fiber(order, 2, N)
    x = rng_fields(f.P, N, order, 0.02).astype(np.complex64)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 25.0)
    torch.cuda.synchronize()
    samples = np.sort(np.random.default_rng(order).choice(N, n_samples, replace=False))
    samples[0] = 0
    samples[-1] = N - 1
    y = yd[:, torch.from_numpy(samples).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle.KerrList(S, 2).at(x.astype(np.complex128), GAMMA * 25.0, samples)
    err = relerr(y, ref)
    print(f"order {order}: P={f.P} sampled Kerr rel-L2 {err:.2e}")
    assert err < 3e-6
    f.close()


def test_kerr_small_N_single_partial_tile():
    f, S, b = fiber(1, 2, 16)
    x = rng_fields(f.P, 16, 5, 0.1).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 3.0)
    assert relerr(to_host(yd), oracle.KerrList(S, 2)(x, GAMMA * 3.0)) < 2e-6
    f.close()


def test_energy_fp64_matches_oracle():
    f, S, b = fiber(1, 2, 1 << 15)
    x = rng_fields(f.P, 1 << 15, 2, 0.01).astype(np.complex64)
    e = f.energy(to_dev(x).data_ptr())
    ref = oracle.energy(x.astype(np.complex128), 1e-12)
    assert np.max(np.abs(e / ref - 1)) < 1e-13
    f.close()


@pytest.mark.parametrize("algo", [mmf.MMF_KERR_AUTO, mmf.MMF_KERR_LIST])
def test_c0_three_modes_100_steps_vs_oracle(algo):
    wl = make_workload("c0")
    ref = oracle.propagate_workload(wl)
    f = mmf.Fiber.from_workload(wl, flags=algo, stream=stream_ptr())
    xd = to_dev(wl.fields)
    f.propagate(xd.data_ptr(), wl.L, wl.n_steps)
    y = to_host(xd)
    err = relerr(y, ref)
    print("c0 rel-L2", err)
    assert err < 1e-5
    # per-field energies through the FP64 reduction agree with the oracle's energy of the output
    e = f.energy(xd.data_ptr())
    assert np.max(np.abs(e / oracle.energy(ref, wl.dt) - 1)) < 2e-5
    f.close()


def test_gamma_zero_propagation_is_exact_linear():
    N = 1 << 12
    f0, S, b = fiber(1, 2, N, alpha=alpha_from_db_per_km(0.2))
    f0.close()
    f = mmf.Fiber(3, 2, S, None, b, alpha_from_db_per_km(0.2), 0.0, N, 1e-12, 0, stream_ptr())
    x = rng_fields(6, N, 9, 0.05).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), 2000.0, 20)
    y = to_host(xd)
    ref = oracle.lin(x, b, alpha_from_db_per_km(0.2), 1e-12, 2000.0)
    assert relerr(y, ref) < 1e-5
    f.close()


def test_restart_is_bitwise():
    wl = make_workload("c0", N_t=1024, n_steps=20, L=200.0)
    f = mmf.Fiber.from_workload(wl, stream=stream_ptr())
    a = to_dev(wl.fields)
    b = to_dev(wl.fields)
    f.propagate(a.data_ptr(), 200.0, 20)
    f.propagate(b.data_ptr(), 100.0, 10)
    f.propagate(b.data_ptr(), 100.0, 10)
    assert torch.equal(a, b)
    f.close()


def test_host_buffer_entry_point_matches_device_path():
    wl = make_workload("c0", N_t=2048, n_steps=10, L=100.0)
    f = mmf.Fiber.from_workload(wl, stream=stream_ptr())
    a = to_dev(wl.fields)
    f.propagate(a.data_ptr(), wl.L, wl.n_steps)
    hin = np.ascontiguousarray(wl.fields.astype(np.complex64))
    hout = np.empty_like(hin)
    f.propagate_host(hin, hout, wl.L, wl.n_steps)
    assert np.array_equal(hout, a.cpu().numpy())
    f.close()


@pytest.mark.parametrize("N_t,n_steps", [(1 << 15, 1), (1 << 15, 2), (1 << 17, 3), (1 << 12, 2)])
def test_host_buffer_row_chunks_match_device_path(N_t, n_steps):
    """The host-buffer call cuts its copies into row chunks overlapped with the first and last
    linear step; the kernels and rows are those of the device path, so the bits must agree (two
    polarisations, 15 modes: chunks of whole polarisation pairs; one, two and three steps, the
    last through the captured step graph; the three-pass and the single-CTA linear steps)."""
    wl = make_workload("c1", N_t=N_t, n_steps=n_steps, L=25.0 * n_steps)
    f = mmf.Fiber.from_workload(wl, flags=1, stream=stream_ptr())
    a = to_dev(wl.fields)
    f.propagate(a.data_ptr(), wl.L, wl.n_steps)
    hin = np.ascontiguousarray(wl.fields.astype(np.complex64))
    hout = np.empty_like(hin)
    f.propagate_host(hin, hout, wl.L, wl.n_steps)
    assert np.array_equal(hout, a.cpu().numpy())
    # in place (the same host buffer in and out), twice in a row
    hio = np.ascontiguousarray(wl.fields.astype(np.complex64))
    f.propagate_host(hio, hio, wl.L, wl.n_steps)
    f.propagate_host(hio, hio, wl.L, wl.n_steps)
    f.propagate(a.data_ptr(), wl.L, wl.n_steps)
    assert np.array_equal(hio, a.cpu().numpy())
    f.close()


def test_zero_steps_and_bad_arguments():
    f, S, b = fiber(1, 1, 64)
    x = to_dev(rng_fields(3, 64, 1, 0.1))
    before = x.clone()
    f.propagate(x.data_ptr(), 100.0, 0)
    assert torch.equal(x, before)
    with pytest.raises(mmf.MMFError):
        f.propagate(0, 100.0, 1)
    with pytest.raises(mmf.MMFError):
        f.kerr(x.data_ptr(), x.data_ptr(), 1.0)
    f.close()


def test_c1_first_steps_vs_oracle():
    # 15 modes x 2 pol, N_t = 2^16, 0.2 dB/km: the first 4 steps (h = 10 m) against the oracle.
    wl = make_workload("c1")
    n = 4
    Lp = n * wl.L / wl.n_steps
    ref = oracle.propagate_workload(wl, n_steps=n, L=Lp)
    f = mmf.Fiber.from_workload(wl, stream=stream_ptr())
    xd = to_dev(wl.fields)
    f.propagate(xd.data_ptr(), Lp, n)
    err = relerr(to_host(xd), ref)
    print("c1 first steps rel-L2", err)
    assert err < 3e-6
    f.close()


def test_c2_45_modes_reduced_window_vs_oracle():
    # 45 HG modes x 2 pol (c2 fields and tensor) on a 256-sample window, 3 steps of h = 25 m.
    wl = make_workload("c2", N_t=256)
    n = 3
    Lp = n * wl.L / wl.n_steps
    ref = oracle.propagate_workload(wl, n_steps=n, L=Lp)
    f = mmf.Fiber.from_workload(wl, stream=stream_ptr())
    assert f.info()["kerr_path"] == "pairs-simt"
    xd = to_dev(wl.fields)
    f.propagate(xd.data_ptr(), Lp, n)
    err = relerr(to_host(xd), ref)
    print("c2 (N_t=256) 3 steps rel-L2", err)
    assert err < 3e-6
    f.close()


def test_c3_120_modes_reduced_window_vs_oracle():
    # 120 HG modes x 2 pol (c3 fields and tensor) on a 64-sample window, one step of h = 50 m.
    wl = make_workload("c3", N_t=64)
    Lp = wl.L / wl.n_steps
    ref = oracle.propagate_workload(wl, n_steps=1, L=Lp)
    f = mmf.Fiber.from_workload(wl, stream=stream_ptr())
    xd = to_dev(wl.fields)
    f.propagate(xd.data_ptr(), Lp, 1)
    err = relerr(to_host(xd), ref)
    print("c3 (N_t=64) 1 step rel-L2", err)
    assert err < 3e-6
    f.close()
