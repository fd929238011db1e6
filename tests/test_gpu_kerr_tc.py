"""Tensor-core (tcgen05) Kerr evaluation vs the FP64 oracle through the C ABI.

BF16X3 keeps about 16 significant bits per operand (hi + lo, the lo*lo term dropped), so
one Kerr evaluation carries a relative error of a few 1e-6 (bound 2e-5 here); plain BF16
keeps 8 bits (bound 5e-3).  TF32X3 keeps about 22 bits per operand, but the tensor core's FP32
accumulation over hundreds of pair terms sets its error at the same few 1e-6 (bound 2e-5).  Every call also checks the device status word (no bounded
device-side wait gave up).
"""
import numpy as np
import pytest

import oracle
import paper_1901_01895_gb300 as mmf
from workloads import make_workload, hg_modes, overlap_tensor, parity_classes, gamma_from_n2

from gpu_util import torch, require_gpu, to_dev, to_host, relerr, rng_fields, stream_ptr

pytestmark = pytest.mark.gpu
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)
TOL = {mmf.MMF_KERR_BF16X3: 2e-5, mmf.MMF_KERR_BF16: 5e-3, mmf.MMF_KERR_TF32X3: 2e-5}


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def fiber(order, n_pol, N, prec, width=0):
    ms = hg_modes(order)
    M = len(ms)
    S = overlap_tensor(ms, 10e-6)
    b = np.zeros((M * n_pol, 4))
    b[:, 2] = -21.7e-27
    f = mmf.Fiber(M, n_pol, S, parity_classes(ms), b, 0.0, GAMMA, N, 1e-12, prec | width, stream_ptr())
    return f, S


@pytest.mark.parametrize("bits", [1 << 5, 2 << 5, 3 << 5])
def test_kerr_tc_rejects_reserved_flag_bits(bits):
    with pytest.raises(mmf.MMFError):
        fiber(2, 2, 256, mmf.MMF_KERR_BF16X3, bits)


@pytest.mark.parametrize("prec", [mmf.MMF_KERR_BF16X3, mmf.MMF_KERR_BF16, mmf.MMF_KERR_TF32X3])
@pytest.mark.parametrize("order,n_pol,N", [(1, 1, 256), (1, 1, 16), (3, 1, 1024), (2, 2, 128), (2, 2, 16),
                                           (4, 2, 1024), (8, 2, 512), (11, 2, 64)])
def test_kerr_tc_vs_oracle(order, n_pol, N, prec):
    f, S = fiber(order, n_pol, N, prec)
    assert f.info()["kerr_path"] == "pairs-tcgen05"
    x = rng_fields(f.P, N, 7 * order + n_pol, 0.05).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x)
    yd = torch.zeros_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 10.0)
    assert f.device_status() == 0
    err = relerr(to_host(yd), oracle.KerrList(S, n_pol)(x, GAMMA * 10.0))
    print(f"tc order {order} npol {n_pol} N {N} prec {prec}: rel {err:.2e}")
    assert err < TOL[prec]
    f.close()


@pytest.mark.parametrize("order,n_samples,prec", [(8, 256, mmf.MMF_KERR_BF16X3), (14, 24, mmf.MMF_KERR_BF16X3),
                                                  (8, 256, mmf.MMF_KERR_TF32X3)])
def test_kerr_tc_full_size_sampled(order, n_samples, prec):
    N = 1 << 17
    f, S = fiber(order, 2, N, prec)
    x = rng_fields(f.P, N, order, 0.02).astype(np.complex64)
    xd = to_dev(x)
    yd = torch.zeros_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 25.0)
    assert f.device_status() == 0
    samples = np.sort(np.random.default_rng(order + 1).choice(N, n_samples, replace=False))
    samples[0], samples[-1] = 0, N - 1
    y = yd[:, torch.from_numpy(samples).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle.KerrList(S, 2).at(x.astype(np.complex128), GAMMA * 25.0, samples)
    err = relerr(y, ref)
    print(f"tc order {order} P={f.P} prec {prec} sampled rel {err:.2e}")
    assert err < TOL[prec]
    f.close()


@pytest.mark.parametrize("prec,tol", [(mmf.MMF_KERR_BF16X3, 1e-5), (mmf.MMF_KERR_BF16, 1e-3)])
def test_c0_propagation_tc_vs_oracle(prec, tol):
    wl = make_workload("c0")
    ref = oracle.propagate_workload(wl)
    f = mmf.Fiber.from_workload(wl, flags=prec, stream=stream_ptr())
    xd = to_dev(wl.fields)
    f.propagate(xd.data_ptr(), wl.L, wl.n_steps)
    assert f.device_status() == 0
    err = relerr(to_host(xd), ref)
    print(f"c0 tc prec {prec}: rel-L2 {err:.2e}")
    assert err < tol
    f.close()


def test_c2_reduced_window_tc_vs_oracle():
    wl = make_workload("c2", N_t=256)
    n = 3
    Lp = n * wl.L / wl.n_steps
    ref = oracle.propagate_workload(wl, n_steps=n, L=Lp)
    for prec, tol in [(mmf.MMF_KERR_BF16X3, 1e-5), (mmf.MMF_KERR_BF16, 1e-3), (mmf.MMF_KERR_TF32X3, 1e-5)]:
        f = mmf.Fiber.from_workload(wl, flags=prec, stream=stream_ptr())
        xd = to_dev(wl.fields)
        f.propagate(xd.data_ptr(), Lp, n)
        assert f.device_status() == 0
        err = relerr(to_host(xd), ref)
        print(f"c2 (N_t=256) tc prec {prec}: rel-L2 {err:.2e}")
        assert err < tol
        f.close()
