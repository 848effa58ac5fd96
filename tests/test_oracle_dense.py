"""Pins for oracle.dense: circulant structure of S, and the textbook forms of Eq. 2-4 when S, N invert."""
import numpy as np

from oracle import dense
from paper_1810_02821_gb300 import synth


def test_signal_covariance_is_the_power_spectrum_circulant():
    H, W = 8, 16
    Pk = synth.power_law_pk(H, W, 1.0, -2.0, 1.0 / 16).astype(np.float64)
    S = dense.signal_covariance(Pk, H, W)
    # autocovariance c(dy, dx) from numpy's inverse real FFT of the power spectrum
    c = np.fft.irfft2(Pk, s=(H, W)) * 1.0  # = (1/n) sum_k P_k e^{+ik.x}
    ys, xs = np.divmod(np.arange(H * W), W)
    C = c[(ys[:, None] - ys[None, :]) % H, (xs[:, None] - xs[None, :]) % W]
    np.testing.assert_allclose(S, C, atol=1e-12)
    # trace = sum of all mode powers (pixel variance times n)
    assert abs(np.trace(S) - (Pk[:, 0].sum() + Pk[:, -1].sum() + 2 * Pk[:, 1:-1].sum()) / 1.0 / (H * W) * (H * W)) < 1e-9


def _invertible_problem(H=8, seed=0):
    p = synth.make_problem(H, seed=seed, mask_frac=0.0, sigma2=(0.1, 0.6))
    Pk = p.Pk.astype(np.float64).copy()
    Pk[0, 0] = 0.7   # make S invertible
    return p, Pk


def test_wiener_dense_matches_textbook_form():
    p, Pk = _invertible_problem()
    H, W = p.shape
    S = dense.signal_covariance(Pk, H, W)
    N = np.diag(p.Ndiag.astype(np.float64).ravel())
    d = p.d.astype(np.float64).ravel()
    # Eq. 4 precision form: (S^-1 + N^-1)^-1 N^-1 d
    ref = np.linalg.solve(np.linalg.inv(S) + np.linalg.inv(N), np.linalg.solve(N, d))
    np.testing.assert_allclose(dense.wiener_dense(p.d, p.Ndiag, p.mask, Pk).ravel(), ref, rtol=1e-10, atol=1e-12)
    Cref = np.linalg.inv(np.linalg.inv(S) + np.linalg.inv(N))
    np.testing.assert_allclose(dense.posterior_cov_dense(p.Ndiag, p.mask, Pk), Cref, rtol=1e-9, atol=1e-12)


def test_missing_pixels_are_the_infinite_noise_limit():
    p = synth.make_problem(8, seed=3, mask_frac=0.2)
    Pk = p.Pk.astype(np.float64).copy()
    Pk[0, 0] = 0.5
    big = np.where(p.mask == 1, 1e12, p.Ndiag.astype(np.float64))
    ref = dense.wiener_dense(p.d, big, np.zeros_like(p.mask), Pk)
    got = dense.wiener_dense(p.d, p.Ndiag, p.mask, Pk)
    np.testing.assert_allclose(got, ref, atol=1e-9)
    # values of d at missing pixels are ignored
    d2 = p.d.copy()
    d2[p.mask == 1] = 123.0
    np.testing.assert_allclose(dense.wiener_dense(d2, p.Ndiag, p.mask, Pk), got, atol=1e-12)


def test_minimum_variance_property():
    """§2.1: W minimises <(Wd - s)^T (Wd - s)>; its value is tr(C_post). Monte-Carlo over (s, n)."""
    rng = np.random.default_rng(11)
    p = synth.make_problem(8, seed=5, mask_frac=0.1)
    H, W = p.shape
    S = dense.signal_covariance(p.Pk, H, W)
    C = dense.posterior_cov_dense(p.Ndiag, p.mask, p.Pk)
    L = np.linalg.cholesky(S + 1e-12 * np.eye(H * W))
    o = p.mask.ravel() == 0
    M = 4000
    s = (L @ rng.standard_normal((H * W, M))).T
    n = rng.standard_normal((M, H * W)) * np.sqrt(p.Ndiag.astype(np.float64).ravel())
    d = np.where(o, s + n, 0.0)
    est = np.stack([dense.wiener_dense(di.reshape(H, W), p.Ndiag, p.mask, p.Pk).ravel() for di in d[:400]])
    mse = np.mean(np.sum((est - s[:400]) ** 2, axis=1))
    assert abs(mse - np.trace(C)) < 0.1 * np.trace(C)
    # a perturbed linear filter does worse
    est2 = 1.05 * est
    assert np.mean(np.sum((est2 - s[:400]) ** 2, axis=1)) > mse
