"""Dense-matrix Wiener filter and Wiener posterior (Eq. 2-4), for images of at most a few thousand pixels.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``). With A = I and missing pixels at infinite noise
(§1.1), the Wiener filter of Eq. 2-3 restricted to the observed set o is

    s_W = S[:, o] (S[o, o] + N[o, o])^-1 d[o]

and the posterior of Eq. 4 is Gaussian with mean s_W and covariance

    C = S - S[:, o] (S[o, o] + N[o, o])^-1 S[o, :]   ( = (S^-1 + N^-1)^-1 when both inverses exist ).

Both stay well defined when S is singular (P = 0 at k = 0). S is built from the power spectrum
(Eq. 7) as U^dagger diag(P) U with U the unitary 2D DFT (Kronecker product of 1D DFT matrices).
"""
from __future__ import annotations

import numpy as np

from . import dft


def signal_covariance(Pk, H: int, W: int) -> np.ndarray:
    """Real n x n signal covariance S = U^dagger diag(P) U, pixels flattened row-major (n = H*W)."""
    U = np.kron(dft.dft_matrix(H), dft.dft_matrix(W))
    P = dft.half_to_full(np.asarray(Pk, dtype=np.float64), W).ravel()
    S = (U.conj().T * P) @ U
    assert np.max(np.abs(S.imag)) < 1e-10 * max(1.0, np.max(np.abs(S.real)))
    S = S.real
    return 0.5 * (S + S.T)


def _observed_system(Ndiag, mask, Pk, extra_noise):
    H, W = np.asarray(Ndiag).shape
    S = signal_covariance(Pk, H, W)
    o = np.flatnonzero(np.asarray(mask).ravel() == 0)
    N = np.asarray(Ndiag, dtype=np.float64).ravel()[o] + extra_noise
    C = S[np.ix_(o, o)] + np.diag(N)
    return S, o, C


def wiener_dense(d, Ndiag, mask, Pk, extra_noise: float = 0.0) -> np.ndarray:
    """s_W = S[:, o] (S_oo + N_oo + extra I)^-1 d_o -> float64 [H][W]."""
    H, W = np.asarray(d).shape
    S, o, C = _observed_system(Ndiag, mask, Pk, extra_noise)
    if o.size == 0:
        return np.zeros((H, W))
    x = np.linalg.solve(C, np.asarray(d, dtype=np.float64).ravel()[o])
    return (S[:, o] @ x).reshape(H, W)


def posterior_cov_dense(Ndiag, mask, Pk) -> np.ndarray:
    """Posterior covariance S - S[:, o] C^-1 S[o, :] (n x n)."""
    S, o, C = _observed_system(Ndiag, mask, Pk, 0.0)
    if o.size == 0:
        return S
    return S - S[:, o] @ np.linalg.solve(C, S[o, :])
