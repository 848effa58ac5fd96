"""Pins for the diagonal pixel response A of the data model d = A s + n (Eq. 1; Alg. 1 definitions with
A_i^2 > 0): the dense Wiener filter and posterior against the information form, the messenger iteration
and sampler against the dense results, and the reductions A = 1, A = c and A_i = 0."""
import numpy as np

from oracle import dense
from oracle import messenger as M
from paper_1810_02821_gb300 import synth


def _problem(H, seed, zeros=3):
    p = synth.make_problem(H, seed=seed, mask_frac=0.1, slope=-2.0, k0=1.0 / H, sigma2=(0.2, 1.0))
    rng = np.random.default_rng(seed + 100)
    A = rng.uniform(0.3, 1.7, size=(H, H))
    A[rng.integers(0, H, zeros), rng.integers(0, H, zeros)] = 0.0
    return p, A


def test_dense_wiener_filter_with_response_is_the_information_form():
    H = 8
    p, A = _problem(H, 1)
    Pk = p.Pk.astype(np.float64).copy()
    Pk[0, 0] = 0.7                                    # S invertible for the information form
    S = dense.signal_covariance(Pk, H, H)
    obs = ((p.mask == 0) & (A != 0)).ravel()
    Ninv = np.where(obs, 1.0 / p.Ndiag.astype(np.float64).ravel(), 0.0)
    a = A.ravel()
    Q = np.linalg.inv(S) + np.diag(a * Ninv * a)       # posterior precision S^-1 + A N^-1 A
    mean = np.linalg.solve(Q, a * Ninv * p.d.astype(np.float64).ravel())
    np.testing.assert_allclose(dense.wiener_dense(p.d, p.Ndiag, p.mask, Pk, A=A).ravel(), mean, rtol=1e-9,
                               atol=1e-12)
    np.testing.assert_allclose(dense.posterior_cov_dense(p.Ndiag, p.mask, Pk, A=A), np.linalg.inv(Q), rtol=1e-8,
                               atol=1e-12)


def test_messenger_wiener_filter_with_response_matches_dense():
    for H, seed in ((8, 2), (16, 3)):
        p, A = _problem(H, seed)
        ref = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk, A=A)
        s, it, rho = M.wf_solve(p.d, p.Ndiag, p.mask, p.Pk, tol=1e-12, A=A)
        assert rho < 1e-12
        assert np.linalg.norm(s - ref) < 1e-10 * np.linalg.norm(ref)


def test_response_reductions():
    H = 8
    p, A = _problem(H, 4)
    ones = np.ones((H, H))
    np.testing.assert_allclose(dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk, A=ones),
                               dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk), rtol=1e-12, atol=1e-14)
    s1, _, _ = M.wf_solve(p.d, p.Ndiag, p.mask, p.Pk, tol=1e-12, A=ones)
    s0, _, _ = M.wf_solve(p.d, p.Ndiag, p.mask, p.Pk, tol=1e-12)
    np.testing.assert_allclose(s1, s0, rtol=1e-10, atol=1e-13)
    # constant response c: the same as data d / c with noise N / c^2
    c = 0.6
    d64, N64 = p.d.astype(np.float64), p.Ndiag.astype(np.float64)
    np.testing.assert_allclose(dense.wiener_dense(d64, N64, p.mask, p.Pk, A=np.full((H, H), c)),
                               dense.wiener_dense(d64 / c, N64 / c ** 2, p.mask, p.Pk), rtol=1e-10, atol=1e-13)
    # A_i = 0 is a missing pixel
    zero = A == 0
    m2 = np.where(zero, 1, p.mask).astype(np.uint8)
    A2 = np.where(zero, 1.0, A)
    np.testing.assert_allclose(dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk, A=A),
                               dense.wiener_dense(p.d, p.Ndiag, m2, p.Pk, A=A2), rtol=1e-12, atol=1e-14)
    assert M.default_tau(p.Ndiag, p.mask, p.Pk, A) == M.default_tau(p.Ndiag, m2, p.Pk, A2)
    xa = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 2, seed=3, A=A)
    xb = M.sample(p.d, p.Ndiag, m2, p.Pk, 2, seed=3, A=A2)
    np.testing.assert_allclose(xa, xb, rtol=1e-12, atol=1e-14)


def test_sampler_with_response_matches_dense_posterior():
    H = 8
    p, A = _problem(H, 5, zeros=2)
    sW = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk, A=A).ravel()
    C = dense.posterior_cov_dense(p.Ndiag, p.mask, p.Pk, A=A)
    n_chains, burn = 1500, 40
    xs = np.stack([M.sample(p.d, p.Ndiag, p.mask, p.Pk, 1, seed=6, chain=c, burn_in=burn - 1, A=A)[0].ravel()
                   for c in range(n_chains)])
    sd = np.sqrt(np.diag(C) / n_chains)
    assert np.max(np.abs(xs.mean(0) - sW) / sd) < 4.5
    se = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / n_chains)
    assert np.max(np.abs(np.cov(xs.T) - C) / se) < 5.5
