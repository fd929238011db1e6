"""Request server (continuous batching) through the C ABI.

Every request is checked against the same propagation run alone through mmf_propagate
(same kernels, one request per handle) and, for small cases, against the FP64 oracle.
A result must not depend on which other requests shared its pool or its graphs: the
kernels compute each (field, slot) row and each time sample independently, so the
served result is expected to be bitwise equal to the lone one; the tests allow 1e-6
relative (rel-L2) for FP32 arithmetic whose summation order could legitimately differ.
"""
import time

import numpy as np
import pytest

import oracle
import paper_1901_01895_gb300 as mmf
from workloads import hg_modes, overlap_tensor, parity_classes, gamma_from_n2
from workloads.configs import draw_betas

from gpu_util import torch, require_gpu, to_dev, to_host, relerr, rng_fields, stream_ptr

pytestmark = pytest.mark.gpu
GAMMA = gamma_from_n2(2.6e-20, 1550e-9)
DT = 1.953125e-12
SAME_TOL = 1e-6


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def fiber_desc(order):
    ms = hg_modes(order)
    return len(ms), overlap_tensor(ms, 10e-6), parity_classes(ms)


def make_req(M, n_pol, N, n_steps, seed, power_w=1e-3, dz=10.0, alpha=0.0):
    betas = draw_betas(M, n_pol, seed)
    x = (rng_fields(M * n_pol, N, seed + 1000, np.sqrt(power_w / 2))).astype(np.complex64)
    return dict(betas=betas, alpha=alpha, N_t=N, dt=DT, L=n_steps * dz, n_steps=n_steps, x=x)


def alone(M, n_pol, S, par, r, flags=0):
    f = mmf.Fiber(M, n_pol, S, par, r["betas"], r["alpha"], GAMMA, r["N_t"], r["dt"], flags, stream_ptr())
    xd = to_dev(r["x"])
    f.propagate(xd.data_ptr(), r["L"], r["n_steps"])
    y = to_host(xd)
    f.close()
    return y


def serve(srv, fid, reqs, gap_s=0.0):
    outs, ids = [], []
    for r in reqs:
        out = np.zeros_like(r["x"])
        ids.append(srv.submit(fid, r["betas"], r["alpha"], r["N_t"], r["dt"], r["L"], r["n_steps"], r["x"], out))
        outs.append(out)
        if gap_s:
            time.sleep(gap_s)
    lat = [srv.wait(i, 120.0) for i in ids]
    return [o.astype(np.complex128) for o in outs], lat


def test_server_matches_alone_and_oracle():
    M, S, par = fiber_desc(2)
    N = 1024
    # different step counts finish at different points inside the pool's K-step graphs
    reqs = [make_req(M, 2, N, n, 10 + i, power_w=10 ** (i - 3)) for i, n in enumerate([3, 7, 12, 20, 33])]
    with mmf.Server() as srv:
        fid = srv.add_fiber(M, 2, S, par, GAMMA)
        outs, lat = serve(srv, fid, reqs)
        st = srv.stats()
    assert st["completed"] == 5 and st["failed"] == 0 and st["pools"] == 1
    assert st["peak_running"] >= 2
    for r, y in zip(reqs, outs):
        ref = alone(M, 2, S, par, r)
        e = relerr(y, ref)
        print(f"steps {r['n_steps']}: served vs alone rel {e:.2e} (bitwise {np.array_equal(y, ref)})")
        assert e <= SAME_TOL
    r = reqs[0]
    ref64 = oracle.propagate(S, 2, r["betas"], 0.0, GAMMA, DT, r["x"].astype(np.complex128), r["L"], r["n_steps"])
    e = relerr(outs[0], ref64)
    print(f"served vs FP64 oracle: {e:.2e}; latencies ms {np.round(lat, 2)}")
    assert e < 1e-5


def test_server_staggered_mixed_shapes_overlap():
    """Requests of two fibers and two N_t arrive while others run; each equals its lone run."""
    fibers = {o: fiber_desc(o) for o in (1, 2)}
    rng = np.random.default_rng(5)
    plan = []
    for i in range(12):
        o = int(rng.choice([1, 2]))
        N = int(rng.choice([512, 2048]))
        n = int(rng.integers(20, 120)) if i < 4 else int(rng.integers(2, 30))
        plan.append((o, make_req(fibers[o][0], 2, N, n, 100 + i, power_w=10 ** rng.uniform(-3.5, -2.5))))
    with mmf.Server() as srv:
        fids = {o: srv.add_fiber(fibers[o][0], 2, fibers[o][1], fibers[o][2], GAMMA) for o in fibers}
        outs, ids = [], []
        for o, r in plan:
            out = np.zeros_like(r["x"])
            ids.append(srv.submit(fids[o], r["betas"], 0.0, r["N_t"], DT, r["L"], r["n_steps"], r["x"], out))
            outs.append(out)
            time.sleep(0.002)
        states_seen = [srv.poll(i)[0] for i in ids]
        for i in ids:
            srv.wait(i, 120.0)
        st = srv.stats()
    print("stats", st, "states right after the last submit", states_seen)
    assert st["completed"] == 12 and st["pools"] >= 3 and st["peak_running"] >= 3
    for (o, r), y in zip(plan, outs):
        M, S, par = fibers[o]
        assert relerr(y.astype(np.complex128), alone(M, 2, S, par, r)) <= SAME_TOL


def test_server_device_buffers():
    M, S, par = fiber_desc(1)
    N = 256
    reqs = [make_req(M, 2, N, n, 30 + n) for n in (4, 9)]
    with mmf.Server() as srv:
        fid = srv.add_fiber(M, 2, S, par, GAMMA)
        ins = [to_dev(r["x"]) for r in reqs]
        outs = [torch.zeros_like(x) for x in ins]
        torch.cuda.synchronize()
        ids = [srv.submit(fid, r["betas"], 0.0, N, DT, r["L"], r["n_steps"], xi.data_ptr(), yo.data_ptr())
               for r, xi, yo in zip(reqs, ins, outs)]
        for i in ids:
            srv.wait(i, 60.0)
        ys = [to_host(y) for y in outs]
    for r, y in zip(reqs, ys):
        assert relerr(y, alone(M, 2, S, par, r)) <= SAME_TOL


def pool_bytes(M, S, par, N):
    with mmf.Server() as srv:
        fid = srv.add_fiber(M, 2, S, par, GAMMA)
        r = make_req(M, 2, N, 2, 1)
        serve(srv, fid, [r])
        return srv.stats()["bytes_in_use"]


def test_server_admission_by_hbm_budget():
    """With room for one pool only, the second shape waits until the first pool is idle and freed."""
    a, b = fiber_desc(1), fiber_desc(2)
    Na, Nb = 1024, 2048
    need = max(pool_bytes(*a, Na), pool_bytes(*b, Nb))
    ra = [make_req(a[0], 2, Na, n, 50 + n) for n in (5, 11)]
    rb = [make_req(b[0], 2, Nb, n, 60 + n) for n in (6, 8)]
    with mmf.Server(hbm_budget_bytes=int(need * 1.2)) as srv:
        fa = srv.add_fiber(a[0], 2, a[1], a[2], GAMMA)
        fb = srv.add_fiber(b[0], 2, b[1], b[2], GAMMA)
        outs, ids = [], []
        for fid, r in [(fa, ra[0]), (fb, rb[0]), (fa, ra[1]), (fb, rb[1])]:
            out = np.zeros_like(r["x"])
            ids.append(srv.submit(fid, r["betas"], 0.0, r["N_t"], DT, r["L"], r["n_steps"], r["x"], out))
            outs.append(out)
        for i in ids:
            srv.wait(i, 120.0)
        st = srv.stats()
    print("budget", need, "stats", st)
    assert st["completed"] == 4 and st["pools"] == 1 and st["bytes_in_use"] <= need * 1.2
    for (desc, r), y in zip([(a, ra[0]), (b, rb[0]), (a, ra[1]), (b, rb[1])], outs):
        M, S, par = desc
        assert relerr(y.astype(np.complex128), alone(M, 2, S, par, r)) <= SAME_TOL


def test_server_rejects_bad_requests():
    M, S, par = fiber_desc(1)
    r = make_req(M, 2, 256, 3, 7)
    out = np.zeros_like(r["x"])
    with mmf.Server(hbm_budget_bytes=1 << 20) as srv:
        fid = srv.add_fiber(M, 2, S, par, GAMMA)
        with pytest.raises(mmf.MMFError) as e:
            srv.submit(fid + 5, r["betas"], 0.0, 256, DT, r["L"], 3, r["x"], out)
        assert e.value.code == mmf.MMF_EINVAL
        with pytest.raises(mmf.MMFError) as e:
            srv.submit(fid, r["betas"], 0.0, 100, DT, r["L"], 3, r["x"], out)
        assert e.value.code == mmf.MMF_EINVAL
        with pytest.raises(mmf.MMFError) as e:
            srv.submit(fid, r["betas"], 0.0, 256, DT, r["L"], 0, r["x"], out)
        assert e.value.code == mmf.MMF_EINVAL
        # a pool of this shape can never fit in 1 MiB: the request fails instead of waiting
        rid = srv.submit(fid, r["betas"], 0.0, 1 << 17, DT, r["L"], 3, np.zeros((6, 1 << 17), np.complex64),
                         np.zeros((6, 1 << 17), np.complex64))
        with pytest.raises(mmf.MMFError) as e:
            srv.wait(rid, 30.0)
        assert e.value.code == mmf.MMF_EBUSY
        with pytest.raises(mmf.MMFError):
            srv.poll(12345)


@pytest.mark.parametrize("prec", [mmf.MMF_KERR_BF16X3, mmf.MMF_KERR_BF16])
def test_server_tensor_core_kerr(prec):
    """Tensor-core Kerr in a pool: sample tiles of finished slots are skipped, results unchanged."""
    M, S, par = fiber_desc(4)
    N = 512
    reqs = [make_req(M, 2, N, n, 70 + n, power_w=3e-3) for n in (2, 5, 9, 17)]
    with mmf.Server() as srv:
        fid = srv.add_fiber(M, 2, S, par, GAMMA, prec)
        outs, _ = serve(srv, fid, reqs)
    for r, y in zip(reqs, outs):
        e = relerr(y, alone(M, 2, S, par, r, prec))
        print(f"prec {prec} steps {r['n_steps']}: served vs alone {e:.2e}")
        assert e <= SAME_TOL
