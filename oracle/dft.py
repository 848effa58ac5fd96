"""Unitary 2D DFT written out as explicit DFT-matrix products (test infrastructure only).

The paper's transform (Eq. 6, §2.1) is the unnormalised sum s~_k = sum_x s_x exp(-i k.x). Its power
spectrum (Eq. 7) is quoted per unitary mode in this code base: ``P_k = <|(U s)_k|^2>`` with U the
unitary DFT, so U = F / sqrt(n). Only numpy matrix products are used (no FFT), so a reader can check
each line against the definition.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def dft_matrix(N: int) -> np.ndarray:
    """U_N[k, x] = exp(-2 pi i k x / N) / sqrt(N): the 1D unitary DFT (Eq. 6 scaled by 1/sqrt(N))."""
    j = np.arange(N)
    M = np.exp(-2j * np.pi * np.outer(j, j) / N) / np.sqrt(N)
    M.setflags(write=False)
    return M


def dft2(x: np.ndarray) -> np.ndarray:
    """Unitary 2D DFT of a real or complex [H][W] array -> full complex spectrum [H][W] (ky, kx FFT order)."""
    H, W = x.shape
    return dft_matrix(H) @ x @ dft_matrix(W).T


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse of :func:`dft2` (U^dagger = conj(U), as U_N is symmetric)."""
    H, W = X.shape
    return np.conj(dft_matrix(H)) @ X @ np.conj(dft_matrix(W)).T


def half_to_full(Ph: np.ndarray, W: int) -> np.ndarray:
    """Extend a symmetric half-spectrum table ``[H][W//2+1]`` (P depends on |k| only, Eq. 7) to ``[H][W]``.

    Entry (ky, kx) with kx > W/2 is the entry at (-ky, -kx) = ((H-ky) % H, W-kx).
    """
    H = Ph.shape[0]
    full = np.empty((H, W), dtype=np.float64)
    full[:, : W // 2 + 1] = Ph
    for kx in range(W // 2 + 1, W):
        for ky in range(H):
            full[ky, kx] = Ph[(H - ky) % H, W - kx]
    return full
