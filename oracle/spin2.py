"""Spin-2 (shear) data for a convergence signal: the Kaiser-Squires operator inside the messenger sampler
(test infrastructure only, see ``oracle/__init__``).

The paper's mass-mapping application (§5, "Cosmological Mass Mapping") observes the shear
gamma = gamma1 + i gamma2, a linear image of the convergence kappa (Eq. 1 with A the Kaiser-Squires
operator): in Fourier space gamma_hat = D kappa_hat with D = (k1 + i k2)^2 / |k|^2, |D| = 1. With kappa =
kappa_E + i kappa_B (E and B modes, real fields with power spectra P_E and P_B) and D = c + i s,
c = (k1^2 - k2^2)/|k|^2, s = 2 k1 k2 / |k|^2, the two real shear components are

    gamma1_hat = c kappa_E_hat - s kappa_B_hat,     gamma2_hat = s kappa_E_hat + c kappa_B_hat,

a rotation of (kappa_E, kappa_B) by the angle 2 phi of k. The rotation is real and even in k, so the
shear components stay real fields. The messenger field t = (t1, t2) lives in shear space with T = tau I
(tau = min observed noise variance of either component, Alg. 1 definitions) and the sweep is Alg. 1 for
the pair: per pixel and component the t-draw of Alg. 1 (noise N1, N2, shared mask); in Fourier space the
signal draw rotated into E and B, where each is the scalar update of Alg. 1 with its own power spectrum:

    e = c t1_hat + s t2_hat,  b = -s t1_hat + c t2_hat,
    e' = P_E/(P_E + tau) e + sqrt(P_E tau/(P_E + tau)) zeta_E,  b' likewise with P_B and zeta_B,
    gamma1_hat = c e' - s b',  gamma2_hat = s e' + c b'.

Readings: k1 runs along x (columns), k2 along y (rows). At k = 0 and on the Nyquist row and column, where
the sign of a frequency is ambiguous, (c, s) = (1, 0) (the rotation must be even in k there for real
fields). Draws: xi1 stream 0, xi2 stream 8 (t-draws), zeta_E stream 1, zeta_B stream 9 (the counter
layouts of the scalar sampler).
"""
from __future__ import annotations

import numpy as np

from . import dft
from .messenger import _fields, default_tau, draw_xi, draw_zeta, pixel_update
from .philox import STREAM_S, STREAM_SB, STREAM_T, STREAM_T2


def ks_rotation(H: int, W: int):
    """(c, s) = (cos 2 phi, sin 2 phi) of every full-spectrum mode (FFT order), (1, 0) at k = 0 and on the
    Nyquist row and column."""
    ky = np.fft.fftfreq(H) * H
    kx = np.fft.fftfreq(W) * W
    k1, k2 = kx[None, :], ky[:, None]
    kk = k1 * k1 + k2 * k2
    with np.errstate(invalid="ignore", divide="ignore"):
        c = (k1 * k1 - k2 * k2) / kk
        s = 2.0 * k1 * k2 / kk
    fix = (kk == 0) | (ky == -H / 2)[:, None] | (kx == -W / 2)[None, :]
    c = np.where(fix, 1.0, c)
    s = np.where(fix, 0.0, s)
    return c, s


def shear_from_convergence(kE, kB):
    """(gamma1, gamma2) of real fields kappa_E, kappa_B."""
    H, W = kE.shape
    c, s = ks_rotation(H, W)
    e, b = dft.dft2(kE), dft.dft2(kB)
    return dft.idft2(c * e - s * b).real, dft.idft2(s * e + c * b).real


def convergence_from_shear(g1, g2):
    """(kappa_E, kappa_B) of shear components (the inverse rotation)."""
    H, W = g1.shape
    c, s = ks_rotation(H, W)
    a, b = dft.dft2(g1), dft.dft2(g2)
    return dft.idft2(c * a + s * b).real, dft.idft2(-s * a + c * b).real


def _spectra(PE, PB, W):
    return dft.half_to_full(np.asarray(PE, np.float64), W), dft.half_to_full(np.asarray(PB, np.float64), W)


def sweep(g1, g2, d1, d2, N1, N2, miss, PEf, PBf, c, s, tau, xi=None, zeta=None, A=None):
    """One Alg. 1 sweep of the pair; xi = (xi1, xi2), zeta = (zeta_E, zeta_B) or None (G -> 0); A: one
    diagonal pixel response for both components, or None."""
    t1 = pixel_update(g1, d1, N1, miss, tau, 1.0, None if xi is None else xi[0], A=A)
    t2 = pixel_update(g2, d2, N2, miss, tau, 1.0, None if xi is None else xi[1], A=A)
    a, b = dft.dft2(t1), dft.dft2(t2)
    e, bb = c * a + s * b, -s * a + c * b
    e = PEf / (PEf + tau) * e
    bb = PBf / (PBf + tau) * bb
    if zeta is not None:
        e = e + np.sqrt(PEf * tau / (PEf + tau)) * zeta[0]
        bb = bb + np.sqrt(PBf * tau / (PBf + tau)) * zeta[1]
    return dft.idft2(c * e - s * bb).real, dft.idft2(s * e + c * bb).real


def _setup(d1, d2, N1, N2, mask, PE, PB, tau, A=None):
    d1, N1v, miss, _ = _fields(d1, N1, mask, PE, A)
    d2 = np.asarray(d2, np.float64)
    N2v = np.asarray(N2, np.float64)
    H, W = d1.shape
    if tau is None:
        tau = min(default_tau(N1v, miss, PE, A), default_tau(N2v, miss, PE, A))
    PEf, PBf = _spectra(PE, PB, W)
    c, s = ks_rotation(H, W)
    return d1, d2, N1v, N2v, miss, PEf, PBf, c, s, tau


def sample(d1, d2, N1, N2, mask, PE, PB, n_samples: int, seed: int, *, chain: int = 0, tau: float | None = None,
           init=None, A=None):
    """Spin-2 chain from gamma = 0 (or init = (g1, g2)) -> [n_samples][2][H][W] shear samples; sweep i uses
    counter step i; A: one diagonal pixel response for both components (None: A = I)."""
    d1, d2, N1v, N2v, miss, PEf, PBf, c, s, tau = _setup(d1, d2, N1, N2, mask, PE, PB, tau, A)
    H, W = d1.shape
    g1, g2 = (np.zeros((H, W)), np.zeros((H, W))) if init is None else (np.array(init[0], float), np.array(init[1], float))
    out = np.empty((n_samples, 2, H, W))
    for i in range(n_samples):
        xi = (draw_xi(seed, chain, i, H, W, STREAM_T), draw_xi(seed, chain, i, H, W, STREAM_T2))
        ze = (draw_zeta(seed, chain, i, H, W, STREAM_S), draw_zeta(seed, chain, i, H, W, STREAM_SB))
        g1, g2 = sweep(g1, g2, d1, d2, N1v, N2v, miss, PEf, PBf, c, s, tau, xi, ze, A)
        out[i, 0], out[i, 1] = g1, g2
    return out


def wiener_messenger(d1, d2, N1, N2, mask, PE, PB, n_iter: int, tau: float | None = None):
    """G -> 0 iteration of the pair at lambda = 1 (no cooling) for n_iter sweeps -> (g1, g2)."""
    d1, d2, N1v, N2v, miss, PEf, PBf, c, s, tau = _setup(d1, d2, N1, N2, mask, PE, PB, tau)
    g1, g2 = np.zeros_like(d1), np.zeros_like(d1)
    for _ in range(n_iter):
        g1, g2 = sweep(g1, g2, d1, d2, N1v, N2v, miss, PEf, PBf, c, s, tau)
    return g1, g2


def apply_covariance(v1, v2, PE, PB):
    """S v for a shear pair v: rotation of (v1_hat, v2_hat) into E and B, multiplication by P_E and P_B
    (unitary DFT), rotation back."""
    H, W = np.asarray(v1).shape
    PEf, PBf = _spectra(PE, PB, W)
    c, s = ks_rotation(H, W)
    a, b = dft.dft2(np.asarray(v1, np.float64)), dft.dft2(np.asarray(v2, np.float64))
    e, q = PEf * (c * a + s * b), PBf * (-s * a + c * b)
    return dft.idft2(c * e - s * q).real, dft.idft2(s * e + c * q).real


def residual(g1, g2, d1, d2, N1, N2, mask, PE, PB) -> float:
    """Relative residual of a shear map g in the Wiener-filter system multiplied through by S (Eq. 2-3):
    ||g + S N^-1 (g - d)|| / ||S N^-1 d||, N^-1 = 0 on masked pixels, norms over both components."""
    obs = np.asarray(mask) == 0
    inv1 = np.where(obs, 1.0 / np.where(obs, np.asarray(N1, np.float64), 1.0), 0.0)
    inv2 = np.where(obs, 1.0 / np.where(obs, np.asarray(N2, np.float64), 1.0), 0.0)
    g1, g2 = np.asarray(g1, np.float64), np.asarray(g2, np.float64)
    d1, d2 = np.asarray(d1, np.float64), np.asarray(d2, np.float64)
    r1, r2 = apply_covariance(inv1 * (g1 - d1), inv2 * (g2 - d2), PE, PB)
    b1, b2 = apply_covariance(inv1 * d1, inv2 * d2, PE, PB)
    num = np.sqrt(np.sum((g1 + r1) ** 2) + np.sum((g2 + r2) ** 2))
    return float(num / np.sqrt(np.sum(b1 ** 2) + np.sum(b2 ** 2)))


def dense_covariance(PE, PB, H: int, W: int) -> np.ndarray:
    """Shear covariance [2n][2n] (component-major) of the E/B model, by dense algebra."""
    U = np.kron(dft.dft_matrix(H), dft.dft_matrix(W))
    PEf, PBf = _spectra(PE, PB, W)
    c, s = ks_rotation(H, W)
    c, s, PEf, PBf = c.ravel(), s.ravel(), PEf.ravel(), PBf.ravel()
    blocks = [[c * c * PEf + s * s * PBf, c * s * (PEf - PBf)], [c * s * (PEf - PBf), s * s * PEf + c * c * PBf]]
    n = H * W
    S = np.zeros((2 * n, 2 * n))
    for i in range(2):
        for j in range(2):
            M = (U.conj().T * blocks[i][j]) @ U
            assert np.max(np.abs(M.imag)) < 1e-10
            S[i * n:(i + 1) * n, j * n:(j + 1) * n] = M.real
    return 0.5 * (S + S.T)


def wiener_dense(d1, d2, N1, N2, mask, PE, PB):
    """Wiener filter of the shear (Eq. 2-3 with the shear covariance) -> (g1, g2)."""
    H, W = np.asarray(d1).shape
    S = dense_covariance(PE, PB, H, W)
    m = (np.asarray(mask).ravel() == 0)
    o = np.flatnonzero(np.concatenate([m, m]))
    N = np.concatenate([np.asarray(N1, np.float64).ravel(), np.asarray(N2, np.float64).ravel()])
    d = np.concatenate([np.asarray(d1, np.float64).ravel(), np.asarray(d2, np.float64).ravel()])
    C = S[np.ix_(o, o)] + np.diag(N[o])
    g = S[:, o] @ np.linalg.solve(C, d[o])
    n = H * W
    return g[:n].reshape(H, W), g[n:].reshape(H, W)


def posterior_cov_dense(N1, N2, mask, PE, PB) -> np.ndarray:
    H, W = np.asarray(N1).shape
    S = dense_covariance(PE, PB, H, W)
    m = (np.asarray(mask).ravel() == 0)
    o = np.flatnonzero(np.concatenate([m, m]))
    N = np.concatenate([np.asarray(N1, np.float64).ravel(), np.asarray(N2, np.float64).ravel()])
    C = S[np.ix_(o, o)] + np.diag(N[o])
    return S - S[:, o] @ np.linalg.solve(C, S[o, :])
