"""Gaussian log-likelihood of the data and its gradient, by dense algebra (test infrastructure only).

The data model of Eq. 1 (A = I) with the Gaussian likelihood and prior of §2.1 gives the evidence
d_o ~ N(0, C), C = S_oo + N_oo, over the observed pixels o (missing pixels have infinite noise, §1.1).
The power spectrum is the parametric P(k) = A (k/k0)^n (P = 0 at k = 0) and the noise is
N = alpha * sigma2 for a known base map sigma2. Then

    lnL = -1/2 d_o^T C^-1 d_o - 1/2 ln det C - (n_o/2) ln 2 pi
    d lnL / d theta = 1/2 x^T (dC/dtheta) x - 1/2 tr(C^-1 dC/dtheta),   x = C^-1 d_o,

with dC/dA = dS_oo/dA (dP/dA = P/A), dC/dn = dS_oo/dn (dP/dn = P ln(k/k0)), dC/dalpha = sigma2_oo.
The quadratic part Q = -1/2 d_o^T C^-1 d_o has gradient 1/2 x^T (dC/dtheta) x.

The Wiener map itself, s_W(theta) = S[:, o] C^-1 d_o (Eq. 2-3), has the derivative

    d s_W / d theta = dS[:, o] x - S[:, o] C^-1 (dC/dtheta) x,

so a cotangent g (all pixels) pulls back to g^T dS[:, o] x - y^T (dC/dtheta) x with y = C^-1 S[o, :] g.
"""
from __future__ import annotations

import numpy as np

from . import dft


def _kgrid_half(H: int, W: int) -> np.ndarray:
    ky = np.fft.fftfreq(H)[:, None]
    kx = (np.arange(W // 2 + 1) / W)[None, :]
    return np.sqrt(ky * ky + kx * kx)


def psd_tables(H: int, W: int, A: float, n: float, k0: float):
    """P, dP/dA, dP/dn on the half-spectrum grid [H][W/2+1] (cycles/pixel, P = 0 at k = 0)."""
    k = _kgrid_half(H, W)
    P = np.zeros_like(k)
    dn = np.zeros_like(k)
    nz = k > 0
    P[nz] = A * (k[nz] / k0) ** n
    dn[nz] = P[nz] * np.log(k[nz] / k0)
    dA = P / A
    return P, dA, dn


def _dense_S(Ph: np.ndarray, H: int, W: int) -> np.ndarray:
    U = np.kron(dft.dft_matrix(H), dft.dft_matrix(W))
    Pf = dft.half_to_full(Ph, W).ravel()
    S = ((U.conj().T * Pf) @ U).real
    return 0.5 * (S + S.T)


def loglike_dense(d, sigma2, mask, A: float, n: float, k0: float, alpha: float):
    """Returns (lnL, Q) with Q = -1/2 d_o^T C^-1 d_o."""
    H, W = np.asarray(d).shape
    P, _, _ = psd_tables(H, W, A, n, k0)
    S = _dense_S(P, H, W)
    o = np.flatnonzero(np.asarray(mask).ravel() == 0)
    C = S[np.ix_(o, o)] + np.diag(alpha * np.asarray(sigma2, dtype=np.float64).ravel()[o])
    do = np.asarray(d, dtype=np.float64).ravel()[o]
    x = np.linalg.solve(C, do)
    sign, logdet = np.linalg.slogdet(C)
    assert sign > 0
    Q = -0.5 * float(do @ x)
    return Q - 0.5 * logdet - 0.5 * o.size * np.log(2 * np.pi), Q


def loglike_grad_dense(d, sigma2, mask, A: float, n: float, k0: float, alpha: float):
    """Exact gradient of lnL w.r.t. (A, n, alpha) and of its quadratic part Q; returns (grad, grad_Q)."""
    H, W = np.asarray(d).shape
    P, dA, dn = psd_tables(H, W, A, n, k0)
    S = _dense_S(P, H, W)
    o = np.flatnonzero(np.asarray(mask).ravel() == 0)
    s2 = np.asarray(sigma2, dtype=np.float64).ravel()[o]
    C = S[np.ix_(o, o)] + np.diag(alpha * s2)
    Ci = np.linalg.inv(C)
    x = Ci @ np.asarray(d, dtype=np.float64).ravel()[o]
    dCs = [_dense_S(dA, H, W)[np.ix_(o, o)], _dense_S(dn, H, W)[np.ix_(o, o)], np.diag(s2)]
    gq = np.array([0.5 * x @ dC @ x for dC in dCs])
    tr = np.array([np.sum(Ci * dC) for dC in dCs])      # tr(C^-1 dC), both symmetric
    return gq - 0.5 * tr, gq


def wiener_param_dense(d, sigma2, mask, A: float, n: float, k0: float, alpha: float) -> np.ndarray:
    """Wiener filter (Eq. 2-3) for P = A (k/k0)^n and N = alpha * sigma2, by the dense solve -> [H][W]."""
    H, W = np.asarray(d).shape
    P, _, _ = psd_tables(H, W, A, n, k0)
    S = _dense_S(P, H, W)
    o = np.flatnonzero(np.asarray(mask).ravel() == 0)
    C = S[np.ix_(o, o)] + np.diag(alpha * np.asarray(sigma2, dtype=np.float64).ravel()[o])
    x = np.linalg.solve(C, np.asarray(d, dtype=np.float64).ravel()[o])
    return (S[:, o] @ x).reshape(H, W)


def wiener_vjp_dense(d, sigma2, mask, A: float, n: float, k0: float, alpha: float, g) -> np.ndarray:
    """g^T d s_W / d(A, n, alpha) for the Wiener map of :func:`wiener_param_dense` (dense algebra)."""
    H, W = np.asarray(d).shape
    P, dA, dn = psd_tables(H, W, A, n, k0)
    S = _dense_S(P, H, W)
    o = np.flatnonzero(np.asarray(mask).ravel() == 0)
    s2 = np.asarray(sigma2, dtype=np.float64).ravel()[o]
    C = S[np.ix_(o, o)] + np.diag(alpha * s2)
    x = np.linalg.solve(C, np.asarray(d, dtype=np.float64).ravel()[o])
    gv = np.asarray(g, dtype=np.float64).ravel()
    dSs = [_dense_S(dA, H, W), _dense_S(dn, H, W), np.zeros_like(S)]
    dCs = [dSs[0][np.ix_(o, o)], dSs[1][np.ix_(o, o)], np.diag(s2)]
    out = []
    for dS, dC in zip(dSs, dCs):
        ds = dS[:, o] @ x - S[:, o] @ np.linalg.solve(C, dC @ x)
        out.append(gv @ ds)
    return np.array(out)
