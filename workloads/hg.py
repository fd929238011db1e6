"""Hermite-Gaussian (HG) mode sets and their nonlinear overlap tensor.

The paper's nonlinear operator (Section 2, Eq. 1) couples the modes through the
coefficients kappa_ab; the general multimode Kerr form those coefficients come
from (the paper's citation for the multimode NLSE) weights every product
A_l A_m A_n^* by the overlap integral of the four real transverse mode fields,

    S_plmn = Int F_p F_l F_m F_n dA / sqrt(Int F_p^2 Int F_l^2 Int F_m^2 Int F_n^2)   [1/m^2].

For HG modes F_(mx,my)(x, y) = u_mx(x) u_my(y) the integral separates into a
product of two 1-D integrals of four Hermite functions each.  The integrand is a
polynomial times exp(-s^2) after the substitution s = 2x/w, so Gauss-Hermite
quadrature with enough nodes evaluates it exactly (up to rounding).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def hg_modes(max_order: int) -> list[tuple[int, int]]:
    """HG mode indices (mx, my) for all modes with mx + my <= max_order.

    Order g = mx + my ascending; within one order mx descending, so the first
    modes are HG00, HG10, HG01, HG20, HG11, HG02, ...  The count is
    (max_order + 1)(max_order + 2)/2: 3, 15, 45, 120 for orders 1, 4, 8, 14.
    """
    if max_order < 0:
        raise ValueError("max_order must be >= 0")
    return [(mx, g - mx) for g in range(max_order + 1) for mx in range(g, -1, -1)]


def _hermite_phys(n_max: int, s: np.ndarray) -> np.ndarray:
    """Physicists' Hermite polynomials H_0..H_n_max at points s (three-term recurrence)."""
    H = np.zeros((n_max + 1,) + s.shape)
    H[0] = 1.0
    if n_max >= 1:
        H[1] = 2.0 * s
    for n in range(1, n_max):
        H[n + 1] = 2.0 * s * H[n] - 2.0 * n * H[n - 1]
    return H


@lru_cache(maxsize=None)
def _overlap_1d_cached(n_max: int, w: float) -> np.ndarray:
    # u_a(x) = N_a H_a(sqrt(2) x / w) exp(-x^2/w^2), normalised so Int u_a^2 dx = 1:
    # N_a^-2 = (w / sqrt 2) 2^a a! sqrt(pi).
    # Int u_a u_b u_c u_d dx with s = 2x/w:  (w/2) prod(N) Int prod H(s/sqrt2) e^{-s^2} ds.
    n_nodes = 2 * n_max + 8          # exact for polynomial degree <= 4*n_max
    s, wq = np.polynomial.hermite.hermgauss(n_nodes)
    H = _hermite_phys(n_max, s / math.sqrt(2.0))
    lognorm = np.array([-0.5 * (math.log(w / math.sqrt(2.0)) + a * math.log(2.0)
                                + math.lgamma(a + 1) + 0.5 * math.log(math.pi))
                        for a in range(n_max + 1)])
    h = H * np.exp(lognorm)[:, None]          # normalised Hermite functions w/o the Gaussian
    I = np.einsum("q,aq,bq,cq,dq->abcd", wq, h, h, h, h, optimize=True) * (w / 2.0)
    # The integrand is odd when a+b+c+d is odd; the quadrature leaves rounding-level
    # residue there, which is replaced by exact zeros so the parity block-sparsity of
    # S is explicit.
    a = np.arange(n_max + 1)
    odd = (a[:, None, None, None] + a[None, :, None, None] + a[None, None, :, None]
           + a[None, None, None, :]) & 1
    I[odd.astype(bool)] = 0.0
    return I


def overlap_1d(n_max: int, w: float) -> np.ndarray:
    """1-D overlaps I[a,b,c,d] = Int u_a u_b u_c u_d dx of normalised Hermite functions [1/m]."""
    return _overlap_1d_cached(int(n_max), float(w)).copy()


def overlap_tensor(modes: list[tuple[int, int]], w: float) -> np.ndarray:
    """Dense S[p,l,m,n] over the spatial modes (float64, 1/m^2), fully symmetric."""
    mx = np.array([m[0] for m in modes])
    my = np.array([m[1] for m in modes])
    n_max = int(max(mx.max(), my.max()))
    I = _overlap_1d_cached(n_max, float(w))
    Sx = I[np.ix_(mx, mx, mx, mx)]
    Sy = I[np.ix_(my, my, my, my)]
    S = Sx * Sy
    return np.ascontiguousarray(S)


def parity_classes(modes: list[tuple[int, int]]) -> np.ndarray:
    """Parity class of each HG mode: (mx & 1) | (my & 1) << 1 (int32).

    S_plmn is zero unless the four classes XOR to 0.
    """
    return np.array([(m[0] & 1) | ((m[1] & 1) << 1) for m in modes], dtype=np.int32)


def kappa_from_overlap(S: np.ndarray, n_pol: int) -> np.ndarray:
    """Nonlinear coupling matrix of the kappa form (Eq. 1) obtained from the overlap tensor by
    keeping only its self- and cross-phase terms: the coefficient of |A_g|^2 A_f in
    sum_{l,m,n} Sfull_{f l m n} A_l A_m conj(A_n), i.e. kappa_ff = Sfull_ffff and
    kappa_fg = Sfull_ffgg + Sfull_fgfg (g != f), with the isotropic polarisation tensor for
    two polarisations.  For HG modes this gives kappa_(pa)(lb) = 2 S_ppll (1 + 2 d_ab) / 3
    for (p, a) != (l, b): cross-phase between orthogonal polarisations is 2/3 of the
    same-polarisation value.  Returned as [P, P] float64, P = n_modes * n_pol (field index
    f = mode * n_pol + pol).  A synthetic stand-in for kappa values from a mode solver."""
    M = S.shape[0]
    P = M * n_pol
    K = np.zeros((P, P))
    for p in range(M):
        for a in range(n_pol):
            f = p * n_pol + a
            for l in range(M):
                for b in range(n_pol):
                    g = l * n_pol + b
                    if f == g:
                        K[f, g] = S[p, p, p, p]
                    else:
                        t = 1.0 if n_pol == 1 else (1.0 + 2.0 * (a == b)) / 3.0
                        K[f, g] = (S[p, p, l, l] + S[p, l, p, l]) * t
    return K


def kappa_hg(modes: list[tuple[int, int]], w: float, n_pol: int) -> np.ndarray:
    """kappa_from_overlap(overlap_tensor(modes, w), n_pol) without forming the M^4 tensor:
    only S_ppll and S_plpl are needed, each a product of two 1-D overlaps."""
    mx = np.array([m[0] for m in modes])
    my = np.array([m[1] for m in modes])
    I = _overlap_1d_cached(int(max(mx.max(), my.max())), float(w))
    a, b = mx[:, None], mx[None, :]
    c, d = my[:, None], my[None, :]
    s_ppll = I[a, a, b, b] * I[c, c, d, d]
    s_plpl = I[a, b, a, b] * I[c, d, c, d]
    M = len(modes)
    K = np.zeros((M * n_pol, M * n_pol))
    for ap in range(n_pol):
        for bp in range(n_pol):
            t = 1.0 if n_pol == 1 else (1.0 + 2.0 * (ap == bp)) / 3.0
            K[ap::n_pol, bp::n_pol] = (s_ppll + s_plpl) * t
    diag = np.diag(s_ppll)          # S_pppp
    for ap in range(n_pol):
        K[np.arange(M) * n_pol + ap, np.arange(M) * n_pol + ap] = diag
    return K


def thinned_tensor(S: np.ndarray, keep: float, seed: int) -> np.ndarray:
    """A sparser fully symmetric tensor with the structure of S: every symmetry orbit of
    index tuples (all permutations of one sorted (p, l, m, n)) is kept whole with
    probability `keep` (seeded), the self-coupling entries S_pppp always.  Zero entries of S
    stay zero, so the parity block-sparsity is that of S.  A test input: the GPU kernels
    see the same mode count, classes and pass structure as for S, while the FP64 reference
    sum over the nonzero entries gets cheap enough to run on whole 2^17-sample rows."""
    M = S.shape[0]
    idx = np.indices((M,) * 4).reshape(4, -1)
    srt = np.sort(idx, axis=0)
    key = ((srt[0] * M + srt[1]) * M + srt[2]) * M + srt[3]
    u = np.random.default_rng(seed).random(M ** 4)
    diag = (srt[0] == srt[3])
    mask = (u[key] < keep) | diag
    out = np.where(mask.reshape(S.shape), S, 0.0)
    return np.ascontiguousarray(out)
