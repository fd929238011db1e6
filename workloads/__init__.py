"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds no arithmetic of the propagation method itself (no FFT, no
propagator, no Kerr sum, no Runge-Kutta stage): it only builds the *inputs* a
user would hand to the solver -- Hermite-Gaussian mode lists and their overlap
tensor S_plmn, seeded propagation constants, and seeded 16-QAM / WDM signals --
plus the five workload definitions with their sizes.

The paper's mode fields and propagation constants came from a commercial mode
solver (Section 6) and are not available; Hermite-Gaussian modes of a parabolic
index profile stand in for them, with their overlap integrals computed exactly by
Gauss-Hermite quadrature.
"""
from .hg import hg_modes, overlap_tensor, parity_classes, overlap_1d, kappa_from_overlap, kappa_hg, thinned_tensor
from .signals import qam16_wdm_fields, dbm_to_w, wdm_fields_symbols, rrc_response
from .configs import CONFIGS, make_workload, Workload, gamma_from_n2, alpha_from_db_per_km

__all__ = [
    "hg_modes", "overlap_tensor", "parity_classes", "overlap_1d", "kappa_from_overlap", "kappa_hg", "thinned_tensor",
    "qam16_wdm_fields", "dbm_to_w", "wdm_fields_symbols", "rrc_response",
    "CONFIGS", "make_workload", "Workload", "gamma_from_n2", "alpha_from_db_per_km",
]
