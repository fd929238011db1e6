"""Serving mix: a seeded stream of independent propagation requests.

Each request is one link simulation of a design sweep: a Hermite-Gaussian fiber with
6, 15, 36 or 45 spatial modes (mode orders <= 2, 4, 7, 8) x 2 polarisations, N_t in
2^14 .. 2^17, a length uniform in 1 .. 50 km stepped at dz = 10 m, and a launch power
uniform in -4 .. +4 dBm per spatial mode, with its own seeded beta0/beta1 offsets.
Arrival times are a Poisson process of unit rate; a caller scales them to the rate it
wants.

Signals: one 16-QAM channel per mode at 32 GBaud, 16 samples/symbol (dt = 1.953125 ps),
RRC roll-off 0.1.  Generating a fresh WDM signal for every request would cost seconds of
host time per request, so one base signal per N_t is drawn for the widest fiber (90
fields, 0 dBm); a request takes its first P rows, scaled to its launch power and shifted
circularly in time by a seeded number of samples (the window is periodic), so requests
differ in content as well as in power.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .configs import COMMON, draw_betas, gamma_from_n2
from .hg import hg_modes, overlap_tensor, parity_classes
from .signals import qam16_wdm_fields

SERVING = dict(orders={6: 2, 15: 4, 36: 7, 45: 8}, n_pol=2, N_t=(1 << 14, 1 << 15, 1 << 16, 1 << 17),
               L_km=(1.0, 50.0), dz=10.0, power_dbm=(-4.0, 4.0), n_requests=2000, seed=4, sps=16)


@dataclass
class Request:
    idx: int
    n_modes: int
    n_pol: int
    N_t: int
    L: float          # m
    n_steps: int
    power_dbm: float
    betas: np.ndarray  # [P, 4]
    shift: int        # circular time shift of the base signal, samples
    arrival: float    # unit-rate Poisson arrival time

    @property
    def P(self) -> int:
        return self.n_modes * self.n_pol

    @property
    def dt(self) -> float:
        return 1.0 / (SERVING["sps"] * COMMON["baud"])

    @property
    def work(self) -> float:
        """Field-sample steps of the request."""
        return float(self.P) * self.N_t * self.n_steps


def serving_requests(n: int | None = None, seed: int | None = None, length_scale: float = 1.0,
                     modes=None, N_t=None) -> list[Request]:
    """The seeded request stream.  length_scale multiplies every length (and so the step
    count at dz = 10 m, at least one step); modes / N_t restrict the choices."""
    cfg = SERVING
    n = cfg["n_requests"] if n is None else n
    rng = np.random.default_rng(cfg["seed"] if seed is None else seed)
    mode_choices = list(cfg["orders"]) if modes is None else list(modes)
    nt_choices = list(cfg["N_t"]) if N_t is None else list(N_t)
    t = 0.0
    out = []
    for i in range(n):
        M = int(rng.choice(mode_choices))
        Nt = int(rng.choice(nt_choices))
        L = rng.uniform(*cfg["L_km"]) * 1e3 * length_scale
        steps = max(1, int(round(L / cfg["dz"])))
        L = steps * cfg["dz"]
        pw = rng.uniform(*cfg["power_dbm"])
        seed_beta = int(rng.integers(1 << 31))
        shift = int(rng.integers(Nt))
        t += rng.exponential(1.0)
        out.append(Request(i, M, cfg["n_pol"], Nt, L, steps, pw, draw_betas(M, cfg["n_pol"], seed_beta), shift, t))
    return out


def fiber_type(n_modes: int) -> dict:
    """Mode list, overlap tensor, parity classes and gamma of the serving fiber with n_modes modes."""
    modes = hg_modes(SERVING["orders"][n_modes])
    return dict(modes=modes, S=overlap_tensor(modes, COMMON["waist"]), parity=parity_classes(modes),
                gamma=gamma_from_n2(COMMON["n2"], COMMON["wavelength"]))


class SignalBank:
    """Base signals per N_t (90 fields, 0 dBm), generated on first use."""

    def __init__(self, seed: int = 40):
        self.seed = seed
        self.base = {}

    def fields(self, req: Request) -> np.ndarray:
        """complex64 [P, N_t] input of a request."""
        if req.N_t not in self.base:
            self.base[req.N_t] = qam16_wdm_fields(45, 2, req.N_t, SERVING["sps"], 1, COMMON["baud"],
                                                  COMMON["spacing"], 0.0, self.seed + req.N_t.bit_length())
        x = self.base[req.N_t][:req.P] * np.sqrt(10.0 ** (req.power_dbm / 10.0))
        return np.ascontiguousarray(np.roll(x, req.shift, axis=1).astype(np.complex64))
