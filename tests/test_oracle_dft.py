"""Pins for oracle.dft: explicit DFT sums, numpy.fft, unitarity and the half-spectrum extension."""
import cmath

import numpy as np

from oracle import dft
from paper_1810_02821_gb300 import synth


def _explicit_dft2(x):
    """The unnormalised sum of Eq. 6 written out term by term, then scaled to the unitary convention."""
    H, W = x.shape
    out = np.zeros((H, W), dtype=complex)
    for ky in range(H):
        for kx in range(W):
            acc = 0j
            for y in range(H):
                for xx in range(W):
                    acc += x[y, xx] * cmath.exp(-2j * cmath.pi * (ky * y / H + kx * xx / W))
            out[ky, kx] = acc
    return out / np.sqrt(H * W)


def test_dft2_matches_explicit_sum():
    rng = np.random.default_rng(1)
    for H, W in [(4, 8), (8, 8), (8, 4)]:
        x = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
        assert np.max(np.abs(dft.dft2(x) - _explicit_dft2(x))) < 1e-12


def test_dft2_matches_numpy_fft():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((16, 32))
    np.testing.assert_allclose(dft.dft2(x), np.fft.fft2(x, norm="ortho"), atol=1e-12)
    X = rng.standard_normal((16, 32)) + 1j * rng.standard_normal((16, 32))
    np.testing.assert_allclose(dft.idft2(X), np.fft.ifft2(X, norm="ortho"), atol=1e-12)


def test_unitary_and_hermitian():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((16, 16))
    X = dft.dft2(x)
    assert abs(np.linalg.norm(X) - np.linalg.norm(x)) < 1e-12
    np.testing.assert_allclose(dft.idft2(X).real, x, atol=1e-12)
    # real input -> Hermitian spectrum X[-k] = conj X[k]
    Xm = X[(-np.arange(16)) % 16][:, (-np.arange(16)) % 16]
    np.testing.assert_allclose(Xm, np.conj(X), atol=1e-12)


def test_half_to_full_matches_direct_power_law():
    H, W = 16, 8
    Ph = synth.power_law_pk(H, W, 2.0, -1.5, 1.0 / 16)
    full = dft.half_to_full(Ph, W)
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    k = np.sqrt(ky ** 2 + kx ** 2)
    direct = np.where(k > 0, 2.0 * (np.where(k > 0, k, 1.0) * 16) ** -1.5, 0.0)
    np.testing.assert_allclose(full, direct.astype(np.float32), rtol=1e-6)
