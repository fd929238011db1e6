"""Mode-split RK4IP across processes (Section 4.1-4.3): the paper's multi-GPU scheme, as a study.

The paper distributes whole rows of the signal matrix (spatial x polarisation modes) to K
processes: each process holds 2M/K rows of N samples and applies the linear operator to them
on its own (it is diagonal per row, Section 4.1).  Only the Kerr term couples rows.  For the
kappa form of Eq. 1 it needs the squared moduli |A_g|^2 of every row, so before each of the
four Kerr evaluations of an RK4IP step (Eq. 4) every process shares the |A|^2 of its rows
((2M/K) N real values) and receives the others' ((2M - 2M/K) N).  Its own rows' contribution
to the phase rate phi_f = sum_g kappa_fg |A_g|^2 is computed while the exchange is in flight
(the "own" kernel of Section 4.3), the other processes' contributions when their data has
arrived (the "others" kernels), and then the rotation i gamma h phi_f A_f is applied to the
local rows.  Each process stores only the kappa rows of its own modes (2M/K x 2M, Section
4.4).  For the overlap-tensor form of the Kerr term the coupling is through field products,
so the complex fields themselves are exchanged instead of |A|^2.

Here the exchange runs on torch.distributed (one process per device; gloo on the CPU, NCCL
between GPUs), with an asynchronous all-gather standing in for the paper's MPI_Isend/Irecv
and ncclAllGather.  The per-row arithmetic is passed in by the caller:
  lin(x_own, z)         exp(z Lhat) applied to the local rows (row-local),
  kappa_own             [rows_own, P] float64, the kappa rows of the local modes,
  kerr_rows(x_all)      (tensor form) the Kerr term of the local rows given every row's field,
so the same orchestration drives CPU arithmetic or the CUDA library's kernels.  The library's
single-GPU path does not use this module: on one GB300 all rows fit, and the path runs on one
device with no exchange.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np


def row_range(P: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [r0, r1) of process `rank`: whole modes, as equal as possible, in order."""
    base, extra = divmod(P, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def kappa_rows(kappa: np.ndarray, rank: int, world: int) -> np.ndarray:
    """The kappa rows a process stores: those of its own modes, against all modes."""
    r0, r1 = row_range(kappa.shape[0], rank, world)
    return np.ascontiguousarray(kappa[r0:r1, :])


@dataclass
class ModeSplit:
    """Exchange and RK4IP orchestration of one process.  Exactly one of kappa_own (kappa form)
    and kerr_rows (overlap-tensor form) is given."""
    rank: int
    world: int
    P: int
    gamma: float
    lin: Callable
    kappa_own: Optional[np.ndarray] = None
    kerr_rows: Optional[Callable] = None
    group: object = None

    def __post_init__(self):
        if (self.kappa_own is None) == (self.kerr_rows is None):
            raise ValueError("give either kappa_own (kappa form) or kerr_rows (tensor form)")
        self.r0, self.r1 = row_range(self.P, self.rank, self.world)
        self.ranges = [row_range(self.P, k, self.world) for k in range(self.world)]
        self.exchanged_values = 0          # values received from other processes so far

    # ---- Kerr term of the local rows ---------------------------------------------------
    def _gather(self, local):
        """Asynchronous all-gather of a [rows_own, N] tensor; returns (buffers, work)."""
        import torch
        import torch.distributed as dist
        rows_max = max(b - a for a, b in self.ranges)
        pad = torch.zeros((rows_max, local.shape[1]), dtype=local.dtype)
        pad[: local.shape[0]] = local
        bufs = [torch.empty_like(pad) for _ in range(self.world)]
        work = dist.all_gather(bufs, pad, group=self.group, async_op=True)
        return bufs, work

    def kerr(self, x_own: np.ndarray, scale: float) -> np.ndarray:
        """i * scale * N(x) for the local rows (scale = gamma * h)."""
        import torch
        N = x_own.shape[1]
        if self.kappa_own is not None:
            sq = np.abs(x_own) ** 2                                      # calc_squareabs
            bufs, work = self._gather(torch.from_numpy(sq))
            ko = self.kappa_own
            phi = ko[:, self.r0:self.r1] @ sq                           # own rows, during the exchange
            work.wait()
            for k, (a, b) in enumerate(self.ranges):                    # the others, as they arrive
                if k == self.rank or b == a:
                    continue
                phi += ko[:, a:b] @ bufs[k].numpy()[: b - a]
                self.exchanged_values += (b - a) * N
            return 1j * scale * phi * x_own                             # apply to the local rows
        bufs, work = self._gather(torch.from_numpy(np.ascontiguousarray(x_own)))
        work.wait()
        x_all = np.empty((self.P, N), dtype=x_own.dtype)
        for k, (a, b) in enumerate(self.ranges):
            x_all[a:b] = bufs[k].numpy()[: b - a]
            if k != self.rank:
                self.exchanged_values += (b - a) * N
        return scale * self.kerr_rows(x_all, self.r0, self.r1)

    # ---- one RK4IP step of the local rows (Eq. 4a-4f) ---------------------------------------
    def step(self, A: np.ndarray, h: float) -> np.ndarray:
        """A(z + h) of the local rows; four Kerr evaluations, each with one exchange."""
        s = self.gamma * h
        AI = self.lin(A, h / 2)                                          # (4a)
        k1 = self.lin(self.kerr(A, s), h / 2)                            # (4b)
        k2 = self.kerr(AI + k1 / 2, s)                                   # (4c)
        k3 = self.kerr(AI + k2 / 2, s)                                   # (4d)
        k4 = self.kerr(self.lin(AI + k3, h / 2), s)                      # (4e)
        return self.lin(AI + k1 / 6 + k2 / 3 + k3 / 3, h / 2) + k4 / 6   # (4f)

    def propagate(self, A: np.ndarray, L: float, n_steps: int) -> np.ndarray:
        h = L / n_steps
        for _ in range(n_steps):
            A = self.step(A, h)
        return A
