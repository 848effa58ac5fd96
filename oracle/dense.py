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


def _observed_system(Ndiag, mask, Pk, extra_noise, A=None):
    """S, the data pixels o, the response A_o on them and C = A_o S_oo A_o + N_oo + extra I."""
    H, W = np.asarray(Ndiag).shape
    S = signal_covariance(Pk, H, W)
    keep = np.asarray(mask).ravel() == 0
    Av = np.ones(H * W) if A is None else np.asarray(A, dtype=np.float64).ravel()
    o = np.flatnonzero(keep & (Av != 0))
    N = np.asarray(Ndiag, dtype=np.float64).ravel()[o] + extra_noise
    Ao = Av[o]
    C = Ao[:, None] * S[np.ix_(o, o)] * Ao[None, :] + np.diag(N)
    return S, o, Ao, C


def wiener_dense(d, Ndiag, mask, Pk, extra_noise: float = 0.0, A=None) -> np.ndarray:
    """s_W = S[:, o] A_o (A_o S_oo A_o + N_oo + extra I)^-1 d_o -> float64 [H][W] (A = I by default: the
    data model d = A s + n of Eq. 1 with a diagonal response)."""
    H, W = np.asarray(d).shape
    S, o, Ao, C = _observed_system(Ndiag, mask, Pk, extra_noise, A)
    if o.size == 0:
        return np.zeros((H, W))
    x = np.linalg.solve(C, np.asarray(d, dtype=np.float64).ravel()[o])
    return (S[:, o] @ (Ao * x)).reshape(H, W)


def posterior_cov_dense(Ndiag, mask, Pk, A=None) -> np.ndarray:
    """Posterior covariance S - S[:, o] A_o C^-1 A_o S[o, :] (n x n)."""
    S, o, Ao, C = _observed_system(Ndiag, mask, Pk, 0.0, A)
    if o.size == 0:
        return S
    SA = S[:, o] * Ao[None, :]
    return S - SA @ np.linalg.solve(C, SA.T)
