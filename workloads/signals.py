"""Seeded 16-QAM / WDM transmit signals on a periodic time window.

Each field (spatial mode x polarisation) carries n_ch wavelength channels on a
uniform grid, each an independent 16-QAM symbol stream shaped by a root-raised-
cosine filter applied in the frequency domain, so the window is periodic (which
the spectral propagator assumes).  Channel centres sit at (c - (n_ch-1)/2) times
the spacing; the launch power is given per channel per spatial mode and split
equally over the polarisations.
"""
from __future__ import annotations

import numpy as np

_QAM16_LEVELS = np.array([-3.0, -1.0, 1.0, 3.0])


def dbm_to_w(dbm: float) -> float:
    return 1e-3 * 10.0 ** (dbm / 10.0)


def _rrc_response(f: np.ndarray, baud: float, rolloff: float) -> np.ndarray:
    """Root-raised-cosine amplitude response with unit passband gain."""
    a = np.abs(f) / baud
    lo, hi = (1.0 - rolloff) / 2.0, (1.0 + rolloff) / 2.0
    H = np.zeros_like(a)
    H[a <= lo] = 1.0
    band = (a > lo) & (a <= hi)
    H[band] = np.sqrt(0.5 * (1.0 + np.cos(np.pi / rolloff * (a[band] - lo))))
    return H


def qam16_wdm_fields(n_modes: int, n_pol: int, N_t: int, sps: int, n_ch: int, baud: float,
                     ch_spacing: float, power_dbm_per_ch: float, seed: int,
                     rolloff: float = 0.1) -> np.ndarray:
    """Complex128 array [n_modes*n_pol, N_t] in sqrt(W); field index f = mode*n_pol + pol.

    The mean power of every channel in every spatial mode is power_dbm_per_ch
    (summed over polarisations).
    """
    if N_t % sps:
        raise ValueError("N_t must be a multiple of sps")
    n_sym = N_t // sps
    dt = 1.0 / (sps * baud)
    t = np.arange(N_t) * dt
    f = np.fft.fftfreq(N_t, dt)
    H = _rrc_response(f, baud, rolloff)
    rng = np.random.default_rng(seed)
    P = n_modes * n_pol
    out = np.zeros((P, N_t), dtype=np.complex128)
    p_field = dbm_to_w(power_dbm_per_ch) / n_pol
    carriers = [np.exp(2j * np.pi * ((c - (n_ch - 1) / 2.0) * ch_spacing) * t) for c in range(n_ch)]
    for fld in range(P):
        for c in range(n_ch):
            sym = (rng.choice(_QAM16_LEVELS, n_sym) + 1j * rng.choice(_QAM16_LEVELS, n_sym)) / np.sqrt(10.0)
            # the spectrum of the symbols placed every sps samples is their n_sym-point
            # spectrum repeated sps times
            x = np.fft.ifft(np.tile(np.fft.fft(sym), sps) * H)
            x *= np.sqrt(p_field / np.mean(np.abs(x) ** 2))
            out[fld] += x * carriers[c]
    return out


_QPSK_LEVELS = np.array([-1.0, 1.0])


def rrc_response(f: np.ndarray, baud: float, rolloff: float = 0.1) -> np.ndarray:
    """Root-raised-cosine amplitude response (unit passband gain) at frequencies f [Hz]."""
    return _rrc_response(f, baud, rolloff)


def wdm_fields_symbols(n_modes: int, n_pol: int, N_t: int, sps: int, n_ch: int, baud: float, ch_spacing: float,
                       power_dbm_per_ch: float, seed: int, fmt: str = "qpsk", rolloff: float = 0.1):
    """WDM transmit fields and the symbols they carry.

    Returns (fields complex128 [P, N_t] in sqrt(W), symbols complex128 [P, n_ch, N_t // sps]).
    Each field carries n_ch independent channels of unit-mean-power QPSK (or 16-QAM) symbols,
    RRC-shaped in the frequency domain (periodic window), at carriers (c - (n_ch-1)/2) * spacing;
    the power of every channel in every spatial mode is power_dbm_per_ch, split equally over the
    polarisations.  Symbol k of a channel sits at sample k * sps before pulse shaping.
    """
    if N_t % sps:
        raise ValueError("N_t must be a multiple of sps")
    levels, norm = (_QPSK_LEVELS, np.sqrt(2.0)) if fmt == "qpsk" else (_QAM16_LEVELS, np.sqrt(10.0))
    n_sym = N_t // sps
    dt = 1.0 / (sps * baud)
    t = np.arange(N_t) * dt
    H = _rrc_response(np.fft.fftfreq(N_t, dt), baud, rolloff)
    rng = np.random.default_rng(seed)
    P = n_modes * n_pol
    p_field = dbm_to_w(power_dbm_per_ch) / n_pol
    out = np.zeros((P, N_t), dtype=np.complex128)
    syms = np.zeros((P, n_ch, n_sym), dtype=np.complex128)
    for fld in range(P):
        for c in range(n_ch):
            sym = (rng.choice(levels, n_sym) + 1j * rng.choice(levels, n_sym)) / norm
            syms[fld, c] = sym
            x = np.zeros(N_t, dtype=np.complex128)
            x[::sps] = sym
            x = np.fft.ifft(np.fft.fft(x) * H)
            x *= np.sqrt(p_field / np.mean(np.abs(x) ** 2))
            out[fld] += x * np.exp(2j * np.pi * (c - (n_ch - 1) / 2.0) * ch_spacing * t)
    return out, syms
