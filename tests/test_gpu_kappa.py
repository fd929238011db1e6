"""Kappa form of Eq. 1 (self- and cross-phase matrix, mmf_create_kappa) on the GPU vs the
FP64 oracle: single Kerr evaluations, full-size sampled outputs, RK4IP propagations with
dispersion and loss, the dispersion-free closed form, and the edge cases of the kernel
(P not a multiple of 4, N_t below one sample tile, the 256-row limit, non-symmetric kappa).
"""
import numpy as np
import pytest

import oracle
import paper_1901_01895_gb300 as mmf
from workloads import hg_modes, overlap_tensor, kappa_from_overlap, gamma_from_n2
from workloads.configs import draw_betas

from gpu_util import torch, require_gpu, to_dev, to_host, relerr, rng_fields, stream_ptr

pytestmark = pytest.mark.gpu
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)
DT = 0.9765625e-12


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def hg_kappa(order, n_pol=2):
    return kappa_from_overlap(overlap_tensor(hg_modes(order), 10e-6), n_pol)


def random_kappa(P, seed):
    r = np.random.default_rng(seed)
    k = r.uniform(0.1, 1.0, (P, P)) / (np.pi * (10e-6) ** 2)
    return (k + k.T) / 2


# FP32 on the CUDA cores, and BF16x3 on the tensor cores (phi = kappa |x|^2 as a GEMM: both
# operands split hi + lo, hi*hi + hi*lo + lo*hi in FP32; operands kept to ~2^-17, products of
# non-negative terms, so a few 1e-6 per evaluation)
PRECS = [(mmf.MMF_KERR_FP32, "kappa", 1e-6), (mmf.MMF_KERR_BF16X3, "kappa-tcgen05", 2e-5)]


# (HG mode order with two polarisations, or a random kappa of that many rows, N_t); the
# tensor-core tiles are 128 samples and 32 rows deep: N_t = 16 .. 1024 and P = 1 .. 251 cover
# ragged tiles, a single partial row chunk and NP = 256
@pytest.mark.parametrize("prec,path,tol", PRECS)
@pytest.mark.parametrize("kind,N", [("rand1", 64), ("rand3", 16), ("hg2", 256), ("hg4", 1024), ("hg8", 512),
                                    ("hg14", 128), ("rand251", 96)])
def test_kappa_kerr_vs_oracle(kind, N, prec, path, tol):
    k = hg_kappa(int(kind[2:])) if kind.startswith("hg") else random_kappa(int(kind[4:]), len(kind))
    P = k.shape[0]
    b = np.zeros((P, 4))
    f = mmf.Fiber.from_kappa(k, b, 0.0, GAMMA, 1 << int(np.ceil(np.log2(N))), DT, prec, stream_ptr())
    Nt = f.N_t
    assert f.info()["kerr_path"] == path
    x = rng_fields(P, Nt, P + 7, 0.05).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x)
    yd = torch.zeros_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 10.0)
    err = relerr(to_host(yd), oracle.kerr_kappa(k, x, GAMMA * 10.0))
    print(f"kappa {path} P={P} N={Nt}: rel {err:.2e}")
    assert err < tol
    assert f.device_status() == 0          # no bounded wait of the kernel gave up
    f.close()


@pytest.mark.parametrize("prec,path,tol", PRECS)
def test_kappa_stage_input(prec, path, tol):
    """k2 = h N(A_I + k1/2) of Eq. 4c: the stage input formed on the load (90 rows, 2^12)."""
    k = hg_kappa(8)
    P, N = k.shape[0], 1 << 12
    f = mmf.Fiber.from_kappa(k, np.zeros((P, 4)), 0.0, GAMMA, N, DT, prec, stream_ptr())
    x0 = rng_fields(P, N, 21, 0.05).astype(np.complex64)
    x1 = rng_fields(P, N, 22, 0.05).astype(np.complex64)
    d0, d1 = to_dev(x0), to_dev(x1)
    yd = torch.zeros_like(d0)
    f.kerr_stage(d0.data_ptr(), d1.data_ptr(), 0.5, yd.data_ptr(), 25.0)
    x = x0.astype(np.complex128) + 0.5 * x1.astype(np.complex128)
    err = relerr(to_host(yd), oracle.kerr_kappa(k, x, GAMMA * 25.0))
    print(f"kappa {path} stage input: rel {err:.2e}")
    assert err < tol
    f.close()


@pytest.mark.parametrize("prec,path,tol", PRECS)
def test_kappa_full_size_sampled(prec, path, tol):
    """240 rows (120 HG modes x 2 pol) at N_t = 2^17, the launch the bench times; sampled outputs."""
    k = hg_kappa(14)
    P, N = k.shape[0], 1 << 17
    f = mmf.Fiber.from_kappa(k, np.zeros((P, 4)), 0.0, GAMMA, N, DT, prec, stream_ptr())
    x = rng_fields(P, N, 3, 0.02).astype(np.complex64)
    xd = to_dev(x)
    yd = torch.zeros_like(xd)
    f.kerr(xd.data_ptr(), yd.data_ptr(), 50.0)
    samples = np.sort(np.random.default_rng(4).choice(N, 512, replace=False))
    samples[0], samples[-1] = 0, N - 1
    y = yd[:, torch.from_numpy(samples).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle.kerr_kappa(k, x[:, samples].astype(np.complex128), GAMMA * 50.0)
    err = relerr(y, ref)
    print(f"kappa {path} 240 x 2^17 sampled: rel {err:.2e}")
    assert err < tol
    assert f.device_status() == 0
    f.close()


@pytest.mark.parametrize("prec", [mmf.MMF_KERR_FP32, mmf.MMF_KERR_BF16X3])
def test_kappa_propagation_vs_oracle(prec):
    """30 rows (15 HG modes x 2 pol) with dispersion, beta1 offsets and loss, 40 steps."""
    k = hg_kappa(4)
    P, N = k.shape[0], 1024
    b = draw_betas(15, 2, 11)
    x = (rng_fields(P, N, 5, 0.03)).astype(np.complex64).astype(np.complex128)
    L, n = 400.0, 40
    alpha = 4.6e-5
    ref = oracle.propagate_kappa(k, b, alpha, GAMMA, DT, x, L, n)
    f = mmf.Fiber.from_kappa(k, b, alpha, GAMMA, N, DT, prec, stream_ptr())
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), L, n)
    err = relerr(to_host(xd), ref)
    print(f"kappa propagation 30 x 1024, 40 steps, flags {prec}: rel {err:.2e}")
    assert err < 1e-5
    f.close()


@pytest.mark.parametrize("prec", [mmf.MMF_KERR_FP32, mmf.MMF_KERR_BF16X3])
def test_kappa_dispersion_free_closed_form(prec):
    """A_f(z) = A_f(0) exp(i gamma sum_g kappa_fg |A_g(0)|^2 z) with no dispersion or loss."""
    k = random_kappa(11, 2)
    P, N = 11, 256
    x = rng_fields(P, N, 9, 0.5)
    L, n = 500.0, 50
    exact = x * np.exp(1j * GAMMA * (k @ np.abs(x) ** 2) * L)
    f = mmf.Fiber.from_kappa(k, np.zeros((P, 4)), 0.0, GAMMA, N, DT, prec, stream_ptr())
    xd = to_dev(x)
    f.propagate(xd.data_ptr(), L, n)
    err = relerr(to_host(xd), exact)
    print(f"kappa closed form: rel {err:.2e}")
    assert err < 2e-5
    f.close()


def test_kappa_rejects_bad_input():
    b = np.zeros((4, 4))
    k = random_kappa(4, 1)
    k[0, 1] *= 1.5                                   # not symmetric
    with pytest.raises(mmf.MMFError) as e:
        mmf.Fiber.from_kappa(k, b, 0.0, GAMMA, 64, DT)
    assert e.value.code == mmf.MMF_EINVAL
    with pytest.raises(mmf.MMFError) as e:          # beyond 256 rows
        mmf.Fiber.from_kappa(random_kappa(257, 1), np.zeros((257, 4)), 0.0, GAMMA, 64, DT)
    assert e.value.code == mmf.MMF_EINVAL
    for fl in (mmf.MMF_KERR_BF16, mmf.MMF_KERR_TF32X3):   # the kappa form is FP32 or BF16x3
        with pytest.raises(mmf.MMFError) as e:
            mmf.Fiber.from_kappa(random_kappa(4, 1), b, 0.0, GAMMA, 64, DT, fl)
        assert e.value.code == mmf.MMF_EINVAL
    with pytest.raises(mmf.MMFError) as e:          # the iterative split step keeps FP32 phases
        mmf.Fiber.from_kappa(random_kappa(4, 1), b, 0.0, GAMMA, 64, DT,
                             mmf.MMF_KERR_BF16X3 | mmf.MMF_METHOD_SSFM_AGRAWAL)
    assert e.value.code == mmf.MMF_EINVAL
