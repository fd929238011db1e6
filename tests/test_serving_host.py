"""Host-side checks of the serving mix and the server boundary (no GPU needed)."""
import numpy as np
import pytest

from workloads.serving import SERVING, SignalBank, serving_requests


def test_serving_mix_is_seeded_and_within_the_stated_ranges():
    a = serving_requests(300)
    b = serving_requests(300)
    assert [(r.n_modes, r.N_t, r.n_steps, r.shift) for r in a] == [(r.n_modes, r.N_t, r.n_steps, r.shift) for r in b]
    assert {r.n_modes for r in a} == set(SERVING["orders"])
    assert {r.N_t for r in a} == set(SERVING["N_t"])
    for r in a:
        assert 1e3 - SERVING["dz"] <= r.L <= 50e3 + SERVING["dz"]
        assert r.n_steps == round(r.L / SERVING["dz"])
        assert -4.0 <= r.power_dbm <= 4.0
        assert r.betas.shape == (r.P, 4)
        # beta per spatial mode, shared by the two polarisations
        assert np.array_equal(r.betas[0::2], r.betas[1::2])
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    # unit-rate Poisson arrivals: mean gap close to 1
    assert 0.8 < np.mean(np.diff(arr)) < 1.2


def test_length_scale_keeps_at_least_one_step():
    r = serving_requests(50, length_scale=1e-6)
    assert all(q.n_steps == 1 for q in r)


def test_signal_bank_scales_power_and_shifts():
    bank = SignalBank()
    rs = serving_requests(40, N_t=[1 << 14], modes=[6])
    x = bank.fields(rs[0])
    assert x.dtype == np.complex64 and x.shape == (12, 1 << 14)
    # mean power per spatial mode (both polarisations) = the launch power
    p_mode = np.mean(np.abs(x.astype(np.complex128)) ** 2, axis=1).reshape(6, 2).sum(axis=1)
    assert np.allclose(p_mode, 1e-3 * 10 ** (rs[0].power_dbm / 10), rtol=1e-5)
    y = bank.fields(rs[1])
    assert not np.allclose(x / np.linalg.norm(x), y / np.linalg.norm(y))


def test_server_without_a_device_fails_cleanly():
    import paper_1901_01895_gb300 as m
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(m.MMFError) as e:
        m.mmf_server_create(0, 0)
    assert e.value.code == m.MMF_ECUDA
    assert m.mmf_server_destroy(0) is None
