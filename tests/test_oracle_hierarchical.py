"""Pins for the hierarchical Gibbs oracle (band-power draws alternated with Alg. 1 sweeps): the chi-square
counting of the band draw, the inverse-gamma moments, the noise-free limit and the reduction to Alg. 1."""
import numpy as np

from oracle import dft
from oracle import hierarchical as HG
from oracle import messenger as M
from oracle.philox import STREAM_BAND
from paper_1810_02821_gb300 import synth


def test_band_draw_counts_one_square_per_full_spectrum_mode():
    H = W = 16
    bins, nb = HG.radial_bins(H, W)
    bf = HG.full_bins(bins, W)
    n_b = np.bincount(bf[bf >= 0], minlength=nb)
    X = np.zeros(nb)
    X2 = np.zeros(nb)
    R = 400
    for i in range(R):
        z = M.draw_zeta(3, 0, i, H, W, STREAM_BAND)
        x = np.zeros(nb)
        np.add.at(x, bf[bf >= 0], np.abs(z[bf >= 0]) ** 2)
        X += x
        X2 += x * x
    mean, var = X / R, X2 / R - (X / R) ** 2
    # chi-square(n_b): mean n_b, variance 2 n_b
    assert np.all(np.abs(mean - n_b) < 5 * np.sqrt(2 * n_b / R)), (mean, n_b)
    assert np.all(np.abs(var / (2 * n_b) - 1) < 0.35)


def test_band_draw_inverse_gamma_moments():
    H = W = 16
    bins, nb = HG.radial_bins(H, W)
    bf = HG.full_bins(bins, W)
    n_b = np.bincount(bf[bf >= 0], minlength=nb)
    rng = np.random.default_rng(0)
    sh = dft.dft2(rng.standard_normal((H, W)))
    S = np.zeros(nb)
    np.add.at(S, bf[bf >= 0], np.abs(sh[bf >= 0]) ** 2)
    R = 1500
    P = np.array([HG.band_power_draw(sh, M.draw_zeta(9, 1, i, H, W, STREAM_BAND), bf, nb) for i in range(R)])
    ok = n_b > 8
    inv_mean = (1.0 / P[:, ok]).mean(0)                       # E[1/P_b] = n_b / S_b
    assert np.all(np.abs(inv_mean / (n_b[ok] / S[ok]) - 1) < 5 * np.sqrt(2.0 / (n_b[ok] * R)))
    mean = P[:, ok].mean(0)                                   # E[P_b] = S_b / (n_b - 2)
    ref = S[ok] / (n_b[ok] - 2)
    sd = ref * np.sqrt(2.0 / (n_b[ok] - 4))
    assert np.all(np.abs(mean - ref) < 5 * sd / np.sqrt(R))


def test_noise_free_limit_draws_band_powers_of_the_data():
    H = W = 16
    p = synth.make_problem(H, seed=4, mask_frac=0.0, slope=-2.0, k0=1.0 / H, sigma2=(1e-8, 1e-8))
    Nd = np.full((H, W), 1e-8, np.float32)
    bins, nb = HG.radial_bins(H, W)
    bf = HG.full_bins(bins, W)
    n_b = np.bincount(bf[bf >= 0], minlength=nb)
    S = np.zeros(nb)
    dh = dft.dft2(p.d.astype(np.float64))
    np.add.at(S, bf[bf >= 0], np.abs(dh[bf >= 0]) ** 2)
    _, Ps = HG.sample(p.d, Nd, p.mask, p.Pk, bins, np.ones(nb), 1200, seed=5)
    Ps = Ps[1:]
    ok = n_b > 8
    ref = S[ok] / (n_b[ok] - 2)
    sd = ref * np.sqrt(2.0 / (n_b[ok] - 4))
    assert np.all(np.abs(Ps[:, ok].mean(0) - ref) < 5 * sd / np.sqrt(len(Ps)))


def test_without_sampled_bins_it_is_alg1():
    p = synth.make_problem(16, seed=6, mask_frac=0.1)
    bins = np.full((16, 9), -1, np.int32)
    xs, Ps = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, np.zeros(0), 3, seed=2, chain=1)
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 3, seed=2, chain=1)
    np.testing.assert_allclose(xs, ref, rtol=1e-12, atol=1e-13)
    assert Ps.shape == (3, 0)


def test_full_spectrum_bins_follow_k_to_minus_k():
    # angular bins (direction modulo pi) are symmetric under k -> -k but not under ky -> -ky alone
    H = W = 16
    def ang(ky, kx):  # bin edges offset by 0.1 rad so that no lattice direction sits on an edge
        return (np.floor(((np.arctan2(ky, kx) + 0.1) % np.pi) / (np.pi / 4))).astype(np.int64) % 4
    kyf = np.fft.fftfreq(H) * H
    kxh = np.arange(W // 2 + 1)
    half = ang(kyf[:, None], kxh[None, :])
    kxf = np.fft.fftfreq(W) * W
    # the Nyquist row and column are their own negatives (a direction there is ambiguous): left out
    direct = ang(kyf[:, None], kxf[None, :])
    full = HG.full_bins(half, W)
    rows = [r for r in range(H) if r != H // 2]
    cols = [c for c in range(W) if c != W // 2]
    np.testing.assert_array_equal(full[np.ix_(rows, cols)], direct[np.ix_(rows, cols)])


def test_band_draw_noise_is_independent_of_the_signal_draw():
    H = W = 16
    bins, nb = HG.radial_bins(H, W)
    bf = HG.full_bins(bins, W)
    a, b = [], []
    for i in range(300):
        zs = M.draw_zeta(2, 0, i, H, W)
        zb = M.draw_zeta(2, 0, i, H, W, STREAM_BAND)
        a.append(np.sum(np.abs(zs[bf >= 0]) ** 2))
        b.append(np.sum(np.abs(zb[bf >= 0]) ** 2))
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.25


def test_pixel_response_reductions():
    """With a pixel response A the hierarchical chain follows the general t-update: A = 1 gives the chain
    without A, and A = 0 at a pixel gives the chain with that pixel masked; a constant A = c equals the
    A = 1 chain for data d / c and noise N / c^2 (the response's exact rescaling)."""
    H = 16
    p = synth.make_problem(H, seed=8, mask_frac=0.1, slope=-2.0, k0=1.0 / H, sigma2=(0.05, 0.5))
    bins, nb = HG.radial_bins(H, H)
    P0 = np.full(nb, 0.5)
    ref = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, 3, seed=2)
    one = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, 3, seed=2, A=np.ones((H, H)))
    for a, b in zip(ref, one):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    A = np.ones((H, H))
    A[3, 5] = 0.0
    m2 = p.mask.copy()
    m2[3, 5] = 1
    zero = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, 3, seed=2, A=A)
    masked = HG.sample(p.d, p.Ndiag, m2, p.Pk, bins, P0, 3, seed=2)
    for a, b in zip(zero, masked):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    c = 1.7
    scaled = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, 3, seed=2, A=np.full((H, H), c))
    plain = HG.sample(p.d.astype(np.float64) / c, p.Ndiag.astype(np.float64) / c ** 2, p.mask, p.Pk, bins, P0, 3,
                      seed=2)
    # (at the pixel that sets tau, N_bar = N - A^2 tau is a rounding residue instead of an exact 0, and its
    # square root scales a noise draw: agreement to about 1e-8 of the field, where a wrong scaling is O(1))
    for a, b in zip(scaled, plain):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-7 * np.abs(b).max())
