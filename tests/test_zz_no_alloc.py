"""mmf_energy_noalloc against mmf_energy, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc (device
memory already held by another framework's caching allocator, or loops where the
device-wide synchronisation of cudaMalloc/cudaFree is not allowed).  Its partial sums
live in a buffer compiled into the library and shared by every call, so the test
makes two calls in a row on different inputs and checks both against the handle-based
entry point, which uses its own allocated scratch.  This file is collected last.
"""
import numpy as np
import pytest

import paper_1901_01895_gb300 as mmf
from workloads import hg_modes, overlap_tensor, parity_classes, gamma_from_n2

from gpu_util import torch, require_gpu, rng_fields, stream_ptr

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_energy_on_two_calls_in_a_row():
    require_gpu()
    ms = hg_modes(1)
    P, N, dt = 6, 1 << 17, 0.5e-12
    b = np.zeros((P, 4))
    f = mmf.Fiber(3, 2, overlap_tensor(ms, 10e-6), parity_classes(ms), b, 0.0, gamma_from_n2(2.6e-20, 1550e-9),
                  N, dt, 0, stream_ptr())
    out = torch.zeros(P, dtype=torch.float64, device="cuda")
    for seed in (1, 2):
        x = torch.from_numpy(rng_fields(P, N, seed, 0.03 * seed).astype(np.complex64)).cuda()
        ref = f.energy(x.data_ptr())
        out.fill_(-1.0)
        mmf.mmf_energy_noalloc(x.data_ptr(), P, N, dt, out.data_ptr(), stream_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got / ref - 1)) < 1e-13, (seed, got, ref)
    f.close()


def test_energy_noalloc_rejects_sizes_beyond_its_buffer():
    require_gpu()
    N = 1 << 17                       # 64 partial sums per field
    P = 300                           # 19200 partials > MMF_NOALLOC_ENERGY_MAX = 16384
    x = torch.zeros((P, N), dtype=torch.complex64, device="cuda")
    out = torch.zeros(P, dtype=torch.float64, device="cuda")
    with pytest.raises(mmf.MMFError) as e:
        mmf.mmf_energy_noalloc(x.data_ptr(), P, N, 1e-12, out.data_ptr(), stream_ptr())
    assert e.value.code == mmf.MMF_EINVAL
    assert "exceed" in mmf.mmf_last_error()
