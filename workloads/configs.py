"""The five workloads: three-mode check case, 15/45/120-mode WDM links, serving mix.

Sizes and parameters:
  c0  3 HG modes (order <= 1) x 1 pol, N_t = 4096 (16 samples/symbol, 256 symbols),
      one 16-QAM channel per mode at 0 dBm, lossless, L = 1 km, 100 steps.
  c1  15 HG modes (order <= 4) x 2 pol, N_t = 2^16 (32 samples/symbol), 5 channels,
      -2 dBm/channel, 0.2 dB/km, L = 10 km, 1000 steps.
  c2  45 HG modes (order <= 8) x 2 pol, N_t = 2^17 (64 samples/symbol), 9 channels,
      0 dBm/channel, lossless, L = 5 km, 200 steps.
  c3  120 HG modes (order <= 14) x 2 pol, N_t = 2^17 (32 samples/symbol), 5 channels,
      -3 dBm/channel, lossless, L = 1 km, 20 steps.
  c4  serving mix (see the serving module): modes in {6, 15, 36, 45} x 2 pol,
      N_t in 2^14..2^17, 1-50 km at dz = 10 m, -4..+4 dBm/channel.
All at 32 GBaud, 50 GHz channel grid, lambda = 1550 nm, n2 = 2.6e-20 m^2/W,
mode waist 10 um, beta2 = -21.7 ps^2/km, seeded per-mode beta1 offsets in
+-0.5 ps/km and beta0 offsets in +-50 rad/m, beta3 = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

from .hg import hg_modes, overlap_tensor, parity_classes
from .signals import qam16_wdm_fields

C0 = 299792458.0


def gamma_from_n2(n2: float, wavelength: float) -> float:
    """gamma = n2 omega0 / c0 = 2 pi n2 / lambda  [m/W]; times S [1/m^2] gives 1/(W m)."""
    return 2.0 * math.pi * n2 / wavelength


def alpha_from_db_per_km(db_per_km: float) -> float:
    """Power attenuation coefficient [1/m] from dB/km (power decays as exp(-alpha z))."""
    return db_per_km * math.log(10.0) / 10.0 * 1e-3


CONFIGS = {
    "c0": dict(max_order=1, n_pol=1, N_t=4096, sps=16, n_ch=1, power_dbm=0.0, L=1e3,
               n_steps=100, alpha_db_km=0.0, seed_sym=0, seed_beta=1),
    "c1": dict(max_order=4, n_pol=2, N_t=1 << 16, sps=32, n_ch=5, power_dbm=-2.0, L=10e3,
               n_steps=1000, alpha_db_km=0.2, seed_sym=10, seed_beta=11),
    "c2": dict(max_order=8, n_pol=2, N_t=1 << 17, sps=64, n_ch=9, power_dbm=0.0, L=5e3,
               n_steps=200, alpha_db_km=0.0, seed_sym=20, seed_beta=21),
    "c3": dict(max_order=14, n_pol=2, N_t=1 << 17, sps=32, n_ch=5, power_dbm=-3.0, L=1e3,
               n_steps=20, alpha_db_km=0.0, seed_sym=30, seed_beta=31),
}
COMMON = dict(baud=32e9, spacing=50e9, wavelength=1550e-9, n2=2.6e-20, waist=10e-6,
              beta2=-21.7e-27, beta1_range=0.5e-15, beta0_range=50.0)


@dataclass
class Workload:
    name: str
    modes: list
    n_modes: int
    n_pol: int
    S: np.ndarray            # [n_modes]^4 float64, 1/m^2
    parity: np.ndarray       # [n_modes] int32
    betas: np.ndarray        # [P, 4] float64: beta0 rad/m, beta1 s/m, beta2 s^2/m, beta3 s^3/m
    alpha: float             # 1/m (power)
    gamma: float             # m/W
    N_t: int
    dt: float                # s
    L: float                 # m
    n_steps: int
    fields: np.ndarray = field(repr=False)   # [P, N_t] complex128, sqrt(W)

    @property
    def P(self) -> int:
        return self.n_modes * self.n_pol


def draw_betas(n_modes: int, n_pol: int, seed: int, beta2: float = COMMON["beta2"],
               beta1_range: float = COMMON["beta1_range"],
               beta0_range: float = COMMON["beta0_range"]) -> np.ndarray:
    """Per spatial mode beta0/beta1 offsets (uniform), common beta2, beta3 = 0; shared by pols."""
    rng = np.random.default_rng(seed)
    b0 = rng.uniform(-beta0_range, beta0_range, n_modes)
    b1 = rng.uniform(-beta1_range, beta1_range, n_modes)
    betas = np.zeros((n_modes * n_pol, 4))
    for m in range(n_modes):
        for a in range(n_pol):
            betas[m * n_pol + a] = (b0[m], b1[m], beta2, 0.0)
    return betas


def make_workload(name: str, *, N_t: int | None = None, n_steps: int | None = None,
                  L: float | None = None, max_order: int | None = None,
                  n_pol: int | None = None, power_dbm: float | None = None,
                  with_S: bool = True) -> Workload:
    """Build a seeded workload; keyword overrides shrink it for tests.

    Overriding N_t keeps the sample spacing dt and the samples per symbol of the
    named workload (fewer symbols per channel).
    """
    cfg = dict(CONFIGS[name])
    full_Nt = cfg["N_t"]
    if max_order is not None:
        cfg["max_order"] = max_order
    if n_pol is not None:
        cfg["n_pol"] = n_pol
    if power_dbm is not None:
        cfg["power_dbm"] = power_dbm
    Nt = full_Nt if N_t is None else int(N_t)
    if Nt % cfg["sps"]:
        raise ValueError("N_t must be a multiple of samples/symbol")
    modes = hg_modes(cfg["max_order"])
    M = len(modes)
    S = overlap_tensor(modes, COMMON["waist"]) if with_S else np.zeros((0,))
    betas = draw_betas(M, cfg["n_pol"], cfg["seed_beta"])
    fields = qam16_wdm_fields(M, cfg["n_pol"], Nt, cfg["sps"], cfg["n_ch"], COMMON["baud"],
                              COMMON["spacing"], cfg["power_dbm"], cfg["seed_sym"])
    dt = 1.0 / (cfg["sps"] * COMMON["baud"])
    return Workload(
        name=name, modes=modes, n_modes=M, n_pol=cfg["n_pol"], S=S,
        parity=parity_classes(modes), betas=betas,
        alpha=alpha_from_db_per_km(cfg["alpha_db_km"]),
        gamma=gamma_from_n2(COMMON["n2"], COMMON["wavelength"]),
        N_t=Nt, dt=dt,
        L=cfg["L"] if L is None else float(L),
        n_steps=cfg["n_steps"] if n_steps is None else int(n_steps),
        fields=fields)
