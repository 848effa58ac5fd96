"""Hierarchical Gibbs sampler: Alg. 1 sweeps alternated with draws of the power spectrum (test
infrastructure only, see ``oracle/__init__``).

The paper (§5, "Power Spectrum Inference" and the Bayesian network of its last figure) describes the
extension in which samples of the signal s and of the power spectrum P(k) are drawn in turn, each with the
other held fixed. This module follows that scheme with the reading stated below (the paper gives no
formulas for the P-step):

* P(k) is piecewise constant over bins: ``bins`` maps each half-spectrum mode (ky, kx) to a bin b, or to
  -1 for modes whose power stays at the given ``Pk`` (for instance k = 0). The map must be symmetric under
  k -> -k, as P(k) is.
* Given s, the unitary Fourier modes of s in bin b are independent Gaussians of variance P_b per real
  degree of freedom pair (<|s_k|^2> = P_b), so with the scale-invariant prior p(P_b) ~ 1/P_b the
  conditional is the inverse gamma P_b | s ~ InvGamma(n_b / 2, S_b / 2) with S_b = sum_{k in b} |s_k|^2 over
  the full spectrum and n_b the number of full-spectrum modes in b. Equivalently P_b = S_b / X_b with
  X_b ~ chi-square(n_b).
* X_b is drawn as sum_{k in b} |zeta'_k|^2 over the full spectrum, where zeta' is Hermitian white noise in
  the same counter layout as the s-draw's zeta (each complex pair contributes Re^2 + Im^2, each
  self-conjugate mode one square) but from Philox stream 6: exactly n_b squared standard normals.

One sweep: t-draw, s-draw with the current band powers (Alg. 1), then the band-power draw from the new s.
"""
from __future__ import annotations

import numpy as np

from . import dft
from .messenger import _fields, default_tau, draw_xi, draw_zeta, pixel_update
from .philox import STREAM_BAND


def full_bins(bins: np.ndarray, W: int) -> np.ndarray:
    """Extend a half-spectrum bin map [H][W/2+1] to the full spectrum [H][W] (kx > W/2 from (-ky, -kx))."""
    H = bins.shape[0]
    full = np.empty((H, W), dtype=np.int64)
    full[:, : W // 2 + 1] = bins
    for kx in range(W // 2 + 1, W):
        for ky in range(H):
            full[ky, kx] = bins[(H - ky) % H, W - kx]
    return full


def radial_bins(H: int, W: int) -> tuple[np.ndarray, int]:
    """Integer-radius bins b = floor(sqrt(ky'^2 + kx^2)) (ky' folded to [-H/2, H/2)) on the half spectrum,
    k = 0 left out (-1); returns (bins [H][W/2+1] int32, n_bins)."""
    ky = np.fft.fftfreq(H) * H
    kx = np.arange(W // 2 + 1)
    r = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    b = np.floor(r).astype(np.int32) - 1          # bin 0 = radius [1, 2)
    b[0, 0] = -1
    return b, int(b.max()) + 1


def band_power_draw(sh_full: np.ndarray, zb_full: np.ndarray, bins_full: np.ndarray, n_bins: int) -> np.ndarray:
    """P_b = S_b / X_b with S_b = sum |s_k|^2 and X_b = sum |zeta'_k|^2 over the full-spectrum modes of bin b."""
    S = np.zeros(n_bins)
    X = np.zeros(n_bins)
    sel = bins_full >= 0
    np.add.at(S, bins_full[sel], np.abs(sh_full[sel]) ** 2)
    np.add.at(X, bins_full[sel], np.abs(zb_full[sel]) ** 2)
    return np.where(X > 0, S / np.where(X > 0, X, 1.0), 0.0)


def sample(d, Ndiag, mask, Pk, bins, P0, n_samples: int, seed: int, *, chain: int = 0, tau: float | None = None,
           burn_in: int = 0, thin: int = 1, init_s=None, A=None):
    """Hierarchical chain -> (samples [n_samples][H][W], band powers [n_samples][n_bins]).

    Sweep i (counter step i): t-draw (with the diagonal response A when given, as in ``messenger``);
    s-draw with P_k = P_b(k) (bins >= 0) or Pk (bins = -1); band-power draw from the new s. Sample m =
    (s, P) after sweep burn_in + (m+1)*thin.
    """
    d, N, miss, Pfix = _fields(d, Ndiag, mask, Pk, A)
    H, W = d.shape
    if tau is None:
        tau = default_tau(N, miss, Pk, A)
    bins = np.asarray(bins)
    bf = full_bins(bins, W)
    n_bins = len(P0)
    Pb = np.asarray(P0, dtype=np.float64).copy()
    s = np.zeros((H, W)) if init_s is None else np.asarray(init_s, dtype=np.float64).copy()
    out_s = np.empty((n_samples, H, W))
    out_P = np.empty((n_samples, n_bins))
    m = 0
    for i in range(burn_in + n_samples * thin):
        Pfull = np.where(bf >= 0, Pb[np.clip(bf, 0, None)], Pfix) if n_bins else Pfix
        t = pixel_update(s, d, N, miss, tau, 1.0, draw_xi(seed, chain, i, H, W), A=A)
        th = dft.dft2(t)
        sh = Pfull / (Pfull + tau) * th + np.sqrt(Pfull * tau / (Pfull + tau)) * draw_zeta(seed, chain, i, H, W)
        s = dft.idft2(sh).real
        Pb = band_power_draw(sh, draw_zeta(seed, chain, i, H, W, STREAM_BAND), bf, n_bins)
        done = i + 1
        if done > burn_in and (done - burn_in) % thin == 0:
            out_s[m] = s
            out_P[m] = Pb
            m += 1
    return out_s, out_P
