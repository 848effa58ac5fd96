"""Planted mistakes in the oracle: each plausible error in Alg. 1 as written out in ``oracle/`` (a wrong
variance, scale, sign, conjugation, level, response power or generator constant) is planted on the CPU
with monkeypatch, and at least one of the oracle's pins must then fail. This shows that the pins can see
the mistakes they are meant to catch; no GPU code is involved."""
import numpy as np
import pytest

import test_oracle_dft as TD
import test_oracle_messenger as TM
import test_oracle_philox as TP
import test_oracle_response as TR
from oracle import dense, dft, philox
from oracle import messenger as M


def _fails(pin, *args):
    """True if the pin raises (an assertion, or the oracle's own Hermitian-symmetry check)."""
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def test_pins_pass_unplanted():
    assert not _fails(TM.test_messenger_wf_matches_dense, 16, 1, 0.15)
    assert not _fails(TM.test_fixed_lambda_fixed_point_is_wf_with_extra_noise)
    assert not _fails(TM.test_masked_data_values_are_ignored_and_all_masked_gives_zero)
    assert not _fails(TM.test_zeta_is_unitary_dft_of_white_noise)


def test_wrong_t_draw_variance(monkeypatch):
    """Alg. 1 t-update with its standard deviation scaled by 1.5: the stationary law of the chain is no
    longer the posterior, so the dense posterior covariance pin fails."""
    orig = M.pixel_update

    def bad(s, d, N, miss, tau, lam, xi=None, A=None):
        return orig(s, d, N, miss, tau, lam, None if xi is None else 1.5 * xi, A)

    monkeypatch.setattr(M, "pixel_update", bad)
    assert _fails(TM.test_sampler_matches_dense_posterior)


def test_wrong_s_draw_variance(monkeypatch):
    """Alg. 1 s-update noise scaled by 1.5: the exact per-mode posterior of the homogeneous case fails."""
    orig = M.fourier_update

    def bad(t, Pfull, tau, lam, zeta=None):
        return orig(t, Pfull, tau, lam, None if zeta is None else 1.5 * zeta)

    monkeypatch.setattr(M, "fourier_update", bad)
    assert _fails(TM.test_homogeneous_sampler_draws_exact_posterior_per_mode)


def test_sign_error_in_messenger_mean(monkeypatch):
    """mu_t = (T d - N_bar s)/(T + N_bar) instead of + N_bar s: the converged map is not the dense WF."""
    def bad(s, d, N, miss, tau, lam, xi=None, A=None):
        T = lam * tau
        Nbar = np.where(miss, 0.0, N - tau)
        denom = np.where(miss, 1.0, T + Nbar)
        mu = np.where(miss, s, (T * d - Nbar * s) / denom)
        return mu if xi is None else mu + np.sqrt(np.where(miss, T, T * Nbar / denom)) * xi

    monkeypatch.setattr(M, "pixel_update", bad)
    assert _fails(TM.test_fixed_lambda_fixed_point_is_wf_with_extra_noise)


def test_filter_ignores_the_messenger_level(monkeypatch):
    """s-update filter P/(P + tau) instead of P/(P + lambda tau): the level-lambda fixed point is no longer
    the Wiener filter with noise N + (lambda - 1) tau."""
    def bad(t, Pfull, tau, lam, zeta=None):
        sh = Pfull / (Pfull + tau) * dft.dft2(t)
        return dft.idft2(sh).real

    monkeypatch.setattr(M, "fourier_update", bad)
    assert _fails(TM.test_fixed_lambda_fixed_point_is_wf_with_extra_noise)


def test_missing_pixels_pull_towards_the_data(monkeypatch):
    """A missing pixel's messenger mean pulled halfway towards its (meaningless) data value: the fixed point
    is no longer the dense filter, which never reads d at a missing pixel."""
    orig = M.pixel_update

    def bad(s, d, N, miss, tau, lam, xi=None, A=None):
        out = orig(s, d, N, miss, tau, lam, xi, A)
        return np.where(miss, 0.5 * (out + d), out)

    monkeypatch.setattr(M, "pixel_update", bad)
    assert _fails(TM.test_fixed_lambda_fixed_point_is_wf_with_extra_noise)


def test_edge_column_mirror_not_conjugated(monkeypatch):
    """The kx = 0 column's modes ky > H/2 copied from ky without the complex conjugate: the noise field is
    no longer the transform of a real field."""
    orig = M.draw_zeta

    def bad(seed, chain, step, H, W, stream=1):
        z = orig(seed, chain, step, H, W, stream)
        ky = np.arange(H // 2 + 1, H)
        z[ky, 0] = z[H - ky, 0]
        return z

    monkeypatch.setattr(M, "draw_zeta", bad)
    assert _fails(TM.test_zeta_is_unitary_dft_of_white_noise)


def test_self_conjugate_modes_drawn_complex(monkeypatch):
    """The four self-conjugate modes given half the variance (a complex draw's real part only)."""
    orig = M.draw_zeta

    def bad(seed, chain, step, H, W, stream=1):
        z = orig(seed, chain, step, H, W, stream)
        for ky in (0, H // 2):
            for kx in (0, W // 2):
                z[ky, kx] = z[ky, kx] / np.sqrt(2.0)
        return z

    monkeypatch.setattr(M, "draw_zeta", bad)
    assert _fails(TM.test_zeta_is_unitary_dft_of_white_noise)


def test_unnormalised_dft(monkeypatch):
    """The paper's unnormalised sum (Eq. 6) in place of the unitary transform the P_k convention needs."""
    orig = dft.dft2

    def bad(x):
        H, W = x.shape
        return orig(x) * np.sqrt(H * W)

    monkeypatch.setattr(dft, "dft2", bad)
    assert _fails(TD.test_unitary_and_hermitian)


def test_dft_exponent_sign_flipped(monkeypatch):
    """exp(+2 pi i k x / N) in the forward transform (the inverse's kernel): the explicit sum of Eq. 6
    disagrees on complex input."""
    def bad(x):
        H, W = x.shape
        return np.conj(dft.dft_matrix(H)) @ x @ np.conj(dft.dft_matrix(W)).T

    monkeypatch.setattr(dft, "dft2", bad)
    assert _fails(TD.test_dft2_matches_explicit_sum)


def test_response_power_one_instead_of_two(monkeypatch):
    """The general t-update with N_bar = N - A tau (A where Alg. 1 has A^2): the messenger filter no longer
    matches the dense filter with a response."""
    orig = M.pixel_update

    def bad(s, d, N, miss, tau, lam, xi=None, A=None):
        if A is None:
            return orig(s, d, N, miss, tau, lam, xi, A)
        A = np.asarray(A, dtype=np.float64)
        T = lam * tau
        Nbar = np.where(miss, 0.0, np.maximum(N - np.abs(A) * tau, 0.0))
        denom = np.where(miss, 1.0, T * A * A + Nbar)
        mu = np.where(miss, s, T * A * d / denom + Nbar * s / denom)
        return mu if xi is None else mu + np.sqrt(np.where(miss, T, T * Nbar / denom)) * xi

    monkeypatch.setattr(M, "pixel_update", bad)
    assert _fails(TR.test_messenger_wiener_filter_with_response_matches_dense)


def test_dense_posterior_missing_a_term(monkeypatch):
    """C_post = S - S_{:,o} (S_oo + N_oo)^-1 S_{o,:} with the subtracted term halved: the Monte-Carlo covariance
    of the (correct) sampler disagrees with it."""
    orig = dense.posterior_cov_dense

    def bad(Ndiag, mask, Pk, A=None):
        H, W = np.asarray(Ndiag).shape
        S = dense.signal_covariance(Pk, H, W)
        return 0.5 * (S + orig(Ndiag, mask, Pk, A))

    monkeypatch.setattr(dense, "posterior_cov_dense", bad)
    assert _fails(TM.test_sampler_matches_dense_posterior)


def test_wrong_philox_multiplier(monkeypatch, curand_philox):
    """One Philox round multiplier off by one bit: curand's own generator disagrees."""
    monkeypatch.setattr(philox, "M1", philox.M1 ^ 0x10)
    assert _fails(TP.test_philox_matches_curand, curand_philox)


curand_philox = TP.curand_philox
