"""The mode-split exchange of Section 4 (paper_1901_01895_gb300.modesplit) on CPU: two and
three gloo ranks (127.0.0.1) each own whole rows, exchange |A|^2 (kappa form) or the fields
(overlap-tensor form) before every Kerr evaluation, and run RK4IP (Eq. 4) on their rows.  The
rows gathered from the ranks must equal the single-process FP64 oracle propagation; the
per-row arithmetic handed to the ranks is the oracle's (row-local linear operator, Kerr term).
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from workloads import hg_modes, overlap_tensor, kappa_hg, gamma_from_n2
    from workloads.configs import draw_betas
    ms = hg_modes(2)                      # 6 HG modes x 2 pol = 12 rows
    M, n_pol, N = len(ms), 2, 256
    betas = draw_betas(M, n_pol, 7)
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((M * n_pol, N)) + 1j * rng.standard_normal((M * n_pol, N))) * 0.05
    return dict(S=overlap_tensor(ms, 10e-6), kappa=kappa_hg(ms, 10e-6, n_pol), betas=betas, x=x, n_pol=n_pol,
                gamma=gamma_from_n2(2.6e-20, 1550e-9), dt=1e-12, alpha=0.0, L=400.0, n_steps=8)


def _rank(rank, ws, port, form, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_1901_01895_gb300.modesplit import ModeSplit, row_range, kappa_rows
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        c = _case()
        P = c["x"].shape[0]
        r0, r1 = row_range(P, rank, ws)
        b_own = c["betas"][r0:r1]

        def lin(x, z):
            return oracle.lin(x, b_own, c["alpha"], c["dt"], z)

        if form == "kappa":
            ms_ = ModeSplit(rank, ws, P, c["gamma"], lin, kappa_own=kappa_rows(c["kappa"], rank, ws))
        else:
            K = oracle.KerrList(c["S"], c["n_pol"])
            ms_ = ModeSplit(rank, ws, P, c["gamma"], lin, kerr_rows=lambda xa, a, b: K(xa, 1.0)[a:b])
        y = ms_.propagate(c["x"][r0:r1].copy(), c["L"], c["n_steps"])
        q.put((rank, r0, r1, y, ms_.exchanged_values))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,form", [(2, "kappa"), (3, "kappa"), (2, "tensor")])
def test_mode_split_equals_single_process_oracle(ws, form):
    import oracle
    c = _case()
    port = _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, form, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(ws)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    P, N = c["x"].shape
    y = np.empty_like(c["x"])
    exchanged = 0
    for rank, r0, r1, yr, ex in got:
        y[r0:r1] = yr
        exchanged += ex
    if form == "kappa":
        ref = oracle.propagate_kappa(c["kappa"], c["betas"], c["alpha"], c["gamma"], c["dt"], c["x"], c["L"],
                                     c["n_steps"])
    else:
        ref = oracle.propagate(c["S"], c["n_pol"], c["betas"], c["alpha"], c["gamma"], c["dt"], c["x"], c["L"],
                               c["n_steps"])
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err
    # each of the 4 Kerr evaluations per step hands every rank the other ranks' rows:
    # (K - 1) P N values per evaluation in total (|A|^2 real for kappa, complex fields for the tensor)
    assert exchanged == 4 * c["n_steps"] * (ws - 1) * P * N


def test_row_ranges_cover_whole_modes():
    sys.path.insert(0, ROOT)
    from paper_1901_01895_gb300.modesplit import row_range, kappa_rows
    for P in (2, 12, 13, 240):
        for K in (1, 2, 3, 8):
            rr = [row_range(P, k, K) for k in range(K)]
            assert rr[0][0] == 0 and rr[-1][1] == P
            assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
            assert max(b - a for a, b in rr) - min(b - a for a, b in rr) <= 1
    kap = np.arange(36.0).reshape(6, 6)
    assert np.array_equal(kappa_rows(kap, 1, 2), kap[3:6])
