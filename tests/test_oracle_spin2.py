"""Pins for the spin-2 (shear) oracle: the Kaiser-Squires rotation against the complex form D = (k1 + i k2)^2
/ |k|^2, its unitarity, the messenger Wiener filter against the dense solve, the sampler against the dense
posterior, and E-only spectra giving no B mode."""
import numpy as np

from oracle import dft
from oracle import spin2 as S2
from paper_1810_02821_gb300 import synth


def _pair(H, seed):
    p = synth.make_problem(H, seed=seed, mask_frac=0.1, slope=-2.0, k0=1.0 / H, sigma2=(0.2, 1.0))
    rng = np.random.default_rng(seed + 50)
    N2 = rng.uniform(0.2, 1.0, (H, H)).astype(np.float32)
    d2 = np.where(p.mask == 1, 0.0, rng.standard_normal((H, H))).astype(np.float32)
    return p, d2, N2


def test_rotation_is_the_complex_kaiser_squires_operator():
    H = W = 16
    rng = np.random.default_rng(1)
    kappa = rng.standard_normal((H, W))
    K = np.fft.fft2(kappa)
    ky = np.fft.fftfreq(H) * H
    kx = np.fft.fftfreq(W) * W
    K[H // 2, :] = 0.0          # a field without power on the Nyquist lines, where D's sign is ambiguous
    K[:, W // 2] = 0.0
    kappa = np.fft.ifft2(K).real
    k1, k2 = kx[None, :], ky[:, None]
    kk = k1 ** 2 + k2 ** 2
    D = np.where(kk > 0, (k1 + 1j * k2) ** 2 / np.where(kk > 0, kk, 1), 1.0)
    gamma = np.fft.ifft2(D * np.fft.fft2(kappa))
    g1, g2 = S2.shear_from_convergence(kappa, np.zeros_like(kappa))
    np.testing.assert_allclose(g1, gamma.real, atol=1e-12)
    np.testing.assert_allclose(g2, gamma.imag, atol=1e-12)


def test_rotation_round_trip():
    rng = np.random.default_rng(2)
    kE, kB = rng.standard_normal((2, 8, 8))
    e, b = S2.convergence_from_shear(*S2.shear_from_convergence(kE, kB))
    np.testing.assert_allclose(e, kE, atol=1e-13)
    np.testing.assert_allclose(b, kB, atol=1e-13)


def test_messenger_wiener_filter_matches_dense():
    for H, seed in ((8, 3), (16, 4)):
        p, d2, N2 = _pair(H, seed)
        PB = 0.3 * p.Pk
        ref = S2.wiener_dense(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)
        it = S2.wiener_messenger(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, 4000)
        for a, b in zip(it, ref):
            assert np.linalg.norm(a - b) < 1e-10 * np.linalg.norm(b)


def test_sampler_matches_dense_posterior_and_e_only_has_no_b_mode():
    H = 8
    p, d2, N2 = _pair(H, 5)
    PB = 0.4 * p.Pk
    mean = np.concatenate([g.ravel() for g in S2.wiener_dense(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)])
    C = S2.posterior_cov_dense(p.Ndiag, N2, p.mask, p.Pk, PB)
    R, burn = 700, 30
    xs = np.stack([S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, burn, seed=7, chain=c)[-1].ravel()
                   for c in range(R)])
    sd = np.sqrt(np.diag(C) / R)
    assert np.max(np.abs(xs.mean(0) - mean) / sd) < 4.5
    se = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / R)
    assert np.max(np.abs(np.cov(xs.T) - C) / se) < 5.5
    g = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, np.zeros_like(p.Pk), 3, seed=1)
    for m in range(3):
        _, kB = S2.convergence_from_shear(g[m, 0], g[m, 1])
        assert np.abs(kB).max() < 1e-12 * max(1.0, np.abs(g[m]).max())


def test_covariance_application_and_residual():
    """S v by FFTs equals the dense shear covariance times v; the residual is 0 at the dense Wiener filter,
    1 at g = 0, and positive for a wrong map (the dense solve with a B-spectrum error)."""
    H = 8
    p, d2, N2 = _pair(H, 6)
    PB = 0.3 * p.Pk
    rng = np.random.default_rng(7)
    v1, v2 = rng.standard_normal((2, H, H))
    S = S2.dense_covariance(p.Pk, PB, H, H)
    Sv = S @ np.concatenate([v1.ravel(), v2.ravel()])
    a1, a2 = S2.apply_covariance(v1, v2, p.Pk, PB)
    np.testing.assert_allclose(np.concatenate([a1.ravel(), a2.ravel()]), Sv, atol=1e-12 * np.abs(Sv).max())
    g = S2.wiener_dense(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)
    assert S2.residual(*g, p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB) < 1e-12
    z = np.zeros((H, H))
    assert abs(S2.residual(z, z, p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB) - 1.0) < 1e-14
    gw = S2.wiener_dense(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, 1.5 * PB)
    assert S2.residual(*gw, p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB) > 1e-3


def test_spin2_pixel_response_reductions():
    """A = 1 gives the spin-2 chain without A; A = 0 at a pixel equals masking it in both components."""
    H = 8
    p, d2, N2 = _pair(H, 9)
    PB = 0.3 * p.Pk
    ref = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, 2, seed=4)
    one = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, 2, seed=4, A=np.ones((H, H)))
    np.testing.assert_allclose(ref, one, rtol=0, atol=1e-12)
    A = np.ones((H, H))
    A[2, 6] = 0.0
    m2 = p.mask.copy()
    m2[2, 6] = 1
    zero = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, 2, seed=4, A=A)
    masked = S2.sample(p.d, d2, p.Ndiag, N2, m2, p.Pk, PB, 2, seed=4)
    np.testing.assert_allclose(zero, masked, rtol=0, atol=1e-12)
