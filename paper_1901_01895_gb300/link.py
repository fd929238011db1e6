"""Multi-span transmission around the propagator (the paper's application, Section 6).

A link is n_spans spans of the same fiber.  Each span is propagated on the GPU (mmf_propagate,
RK4IP or a split-step method) and followed by a noiseless flat-gain amplifier that restores
the span loss (mmf_amplify).  White noise is added before the receiver so that every channel
sees the requested OSNR, and the linear part of the fiber is undone exactly in the frequency
domain (mmf_linear at z = -L on a lossless copy of the fiber).  That last step is the
"perfect" dispersion compensation of Section 6; it also removes the per-mode group delays,
the part of the delay that clock recovery finds.

The receiver runs on the host (numpy), per field (spatial mode x polarisation) and channel:
down-mixing to baseband, the RRC matched filter, sampling at the symbol instants, data-aided
phase and amplitude recovery over blocks of symbols (the paper's phase recovery, in its
data-aided form), and the squared Q factor from the error vector magnitude,
Q^2 = sum |s|^2 / sum |r - s|^2 (dB).

OSNR convention: signal power of one channel (both polarisations of a spatial mode) over the
noise power of both polarisations in 12.5 GHz.  White noise of variance sigma^2 per complex
field sample has a one-sided density sigma^2 / f_s per polarisation, so
sigma^2 = P_ch f_s / (n_pol * 12.5 GHz * OSNR).

Device memory for the noise comes from PyTorch (plumbing); every operation on the fields
runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import Fiber, MMFError

B_REF = 12.5e9   # OSNR reference bandwidth (0.1 nm at 1550 nm)


def noise_variance(p_ch_w: float, osnr_db: float, fs: float, n_pol: int) -> float:
    """Variance per complex field sample of the white noise that sets a channel's OSNR."""
    return p_ch_w * fs / (n_pol * B_REF * 10.0 ** (osnr_db / 10.0))


def white_noise(shape, sigma2: float, seed: int) -> np.ndarray:
    """Seeded circular complex Gaussian noise, E|n|^2 = sigma2 (complex64)."""
    r = np.random.default_rng(seed)
    n = (r.standard_normal(shape) + 1j * r.standard_normal(shape)) * np.sqrt(sigma2 / 2.0)
    return n.astype(np.complex64)


def _rrc(f: np.ndarray, baud: float, rolloff: float) -> np.ndarray:
    a = np.abs(f) / baud
    lo, hi = (1.0 - rolloff) / 2.0, (1.0 + rolloff) / 2.0
    H = np.zeros_like(a)
    H[a <= lo] = 1.0
    band = (a > lo) & (a <= hi)
    H[band] = np.sqrt(0.5 * (1.0 + np.cos(np.pi / rolloff * (a[band] - lo))))
    return H


def receive(fields: np.ndarray, symbols: np.ndarray, sps: int, baud: float, spacing: float, dt: float,
            rolloff: float = 0.1, block: int = 64) -> dict:
    """Matched filter, sampling, data-aided phase/amplitude recovery and Q^2 per field and channel.

    fields  [P, N_t] received (dispersion-compensated) fields; symbols [P, n_ch, n_sym] sent.
    Returns {"q2_db": [P, n_ch], "evm": [P, n_ch]}.
    """
    P, N = fields.shape
    n_ch, n_sym = symbols.shape[1], symbols.shape[2]
    t = np.arange(N) * dt
    H = _rrc(np.fft.fftfreq(N, dt), baud, rolloff)
    q2 = np.zeros((P, n_ch))
    evm = np.zeros((P, n_ch))
    for c in range(n_ch):
        fc = (c - (n_ch - 1) / 2.0) * spacing
        x = np.asarray(fields, dtype=np.complex128) * np.exp(-2j * np.pi * fc * t)
        y = np.fft.ifft(np.fft.fft(x, axis=1) * H, axis=1)
        r = y[:, ::sps][:, :n_sym]
        s = symbols[:, c]
        err = np.zeros(P)
        for b0 in range(0, n_sym, block):
            rb, sb = r[:, b0:b0 + block], s[:, b0:b0 + block]
            a = np.sum(rb * np.conj(sb), axis=1) / np.sum(np.abs(sb) ** 2, axis=1)   # gain and phase
            err += np.sum(np.abs(rb / a[:, None] - sb) ** 2, axis=1)
        e2 = err / np.sum(np.abs(s) ** 2, axis=1)
        evm[:, c] = np.sqrt(e2)
        q2[:, c] = -10.0 * np.log10(np.maximum(e2, 1e-30))
    return {"q2_db": q2, "evm": evm}


class Link:
    """n_spans spans of one fiber with amplifiers, noise loading and a perfect linear receiver.

    fiber_args: positional arguments of Fiber(...) for the overlap-tensor form
    (n_modes, n_pol, S, parity, betas, alpha, gamma, N_t, dt), or pass kappa= to use the kappa
    form (betas, alpha, gamma, N_t, dt then given as keywords).
    """

    def __init__(self, span_length: float, n_spans: int, steps_per_span: int, *, n_modes=None, n_pol=None,
                 S=None, parity=None, kappa=None, betas, alpha: float, gamma: float, N_t: int, dt: float,
                 flags: int = 0, stream: int = 0):
        self.span_length, self.n_spans, self.steps = float(span_length), int(n_spans), int(steps_per_span)
        self.alpha, self.dt, self.N_t = float(alpha), float(dt), int(N_t)
        b = np.asarray(betas, dtype=np.float64)
        if kappa is not None:
            self.fiber = Fiber.from_kappa(kappa, b, alpha, gamma, N_t, dt, flags, stream)
            self.comp = Fiber.from_kappa(kappa, b, 0.0, 0.0, N_t, dt, 0, stream)
            self.n_pol = 2 if n_pol is None else n_pol
        else:
            self.fiber = Fiber(n_modes, n_pol, S, parity, b, alpha, gamma, N_t, dt, flags, stream)
            self.comp = Fiber(n_modes, n_pol, S, parity, b, 0.0, 0.0, N_t, dt, 0, stream)
            self.n_pol = n_pol
        self.P = self.fiber.P

    def transmit(self, fields_ptr: int, noise_ptr: int = 0, out_ptr: int = 0) -> None:
        """Propagate the device fields (complex64 [P][N_t], in place) over every span with an
        amplifier after each, add the noise (device array or 0) and undo the linear part of the
        whole link into out_ptr (in place when 0)."""
        gain = float(np.exp(self.alpha * self.span_length))
        for k in range(self.n_spans):
            self.fiber.propagate(fields_ptr, self.span_length, self.steps)
            self.fiber.amplify(fields_ptr, gain, noise_ptr if (noise_ptr and k == self.n_spans - 1) else 0)
        self.comp.linear(fields_ptr, out_ptr or fields_ptr, -self.span_length * self.n_spans)

    def close(self):
        for f in (getattr(self, "fiber", None), getattr(self, "comp", None)):
            if f is not None:
                f.close()


def _main():
    """A Section-6-like scenario on Hermite-Gaussian modes: two 80 km spans, noiseless
    amplifiers, OSNR 20 dB, DP-QPSK at 32 GBaud; prints Q^2 per spatial mode."""
    import argparse
    import torch
    from workloads import hg_modes, kappa_hg, gamma_from_n2, alpha_from_db_per_km, wdm_fields_symbols
    from workloads.configs import draw_betas
    ap = argparse.ArgumentParser()
    ap.add_argument("--order", type=int, default=2, help="HG mode order (2: 6 modes)")
    ap.add_argument("--channels", type=int, default=3)
    ap.add_argument("--power-dbm", type=float, default=-1.0)
    ap.add_argument("--osnr-db", type=float, default=20.0)
    ap.add_argument("--spans", type=int, default=2)
    ap.add_argument("--span-km", type=float, default=80.0)
    ap.add_argument("--steps-per-span", type=int, default=800)
    ap.add_argument("--symbols", type=int, default=4096)
    a = ap.parse_args()
    modes = hg_modes(a.order)
    M, npol, baud, spacing = len(modes), 2, 32e9, 50e9
    sps = 8 if a.channels > 1 else 4
    N = a.symbols * sps
    dt = 1.0 / (sps * baud)
    kappa = kappa_hg(modes, 10e-6, npol)
    betas = draw_betas(M, npol, 61)
    x, syms = wdm_fields_symbols(M, npol, N, sps, a.channels, baud, spacing, a.power_dbm, 62)
    link = Link(a.span_km * 1e3, a.spans, a.steps_per_span, kappa=kappa, n_pol=npol, betas=betas,
                alpha=alpha_from_db_per_km(0.23), gamma=gamma_from_n2(2.6e-20, 1550e-9), N_t=N, dt=dt,
                stream=torch.cuda.current_stream().cuda_stream)
    sigma2 = noise_variance(10 ** (a.power_dbm / 10) * 1e-3, a.osnr_db, 1.0 / dt, npol)
    noise = torch.from_numpy(white_noise(x.shape, sigma2, 63)).cuda()
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    link.transmit(xd.data_ptr(), noise.data_ptr())
    torch.cuda.synchronize()
    q = receive(xd.cpu().numpy(), syms, sps, baud, spacing, dt)["q2_db"]
    for m in range(M):
        qm = q[m * npol:(m + 1) * npol]
        print(f"HG{modes[m][0]}{modes[m][1]}: Q^2 min {qm.min():.2f}  mean {qm.mean():.2f}  max {qm.max():.2f} dB")
    link.close()


if __name__ == "__main__":
    _main()
