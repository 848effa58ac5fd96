"""Pins for oracle.likelihood: scipy's multivariate normal log-pdf, finite differences, power-law tables."""
import numpy as np
import pytest

from oracle import likelihood as LL
from paper_1810_02821_gb300 import synth

scipy_stats = pytest.importorskip("scipy.stats")


def _problem(H=8, seed=0):
    p = synth.make_problem(H, seed=seed, mask_frac=0.15, slope=-2.0, k0=1.0 / H, sigma2=(0.05, 0.3))
    return p.d.astype(np.float64), p.Ndiag.astype(np.float64), p.mask


def test_psd_tables_match_synth_power_law():
    P, dA, dn = LL.psd_tables(16, 16, 1.7, -1.8, 1.0 / 16)
    np.testing.assert_allclose(P, synth.power_law_pk(16, 16, 1.7, -1.8, 1.0 / 16), rtol=1e-6)
    h = 1e-6
    Pp, _, _ = LL.psd_tables(16, 16, 1.7, -1.8 + h, 1.0 / 16)
    Pm, _, _ = LL.psd_tables(16, 16, 1.7, -1.8 - h, 1.0 / 16)
    np.testing.assert_allclose(dn, (Pp - Pm) / (2 * h), rtol=1e-6, atol=1e-12)


def test_loglike_matches_multivariate_normal_logpdf():
    d, s2, mask = _problem()
    A, n, k0, alpha = 1.3, -1.7, 1.0 / 8, 0.9
    lnL, Q = LL.loglike_dense(d, s2, mask, A, n, k0, alpha)
    P, _, _ = LL.psd_tables(8, 8, A, n, k0)
    # covariance of the observed pixels rebuilt from numpy.fft autocovariance (independent of oracle.dft)
    c = np.fft.irfft2(P, s=(8, 8))
    ys, xs = np.divmod(np.arange(64), 8)
    S = c[(ys[:, None] - ys[None, :]) % 8, (xs[:, None] - xs[None, :]) % 8]
    o = np.flatnonzero(mask.ravel() == 0)
    C = S[np.ix_(o, o)] + np.diag(alpha * s2.ravel()[o])
    ref = scipy_stats.multivariate_normal(mean=np.zeros(o.size), cov=C).logpdf(d.ravel()[o])
    assert abs(lnL - ref) < 1e-9 * max(1.0, abs(ref))
    assert abs(Q + 0.5 * d.ravel()[o] @ np.linalg.solve(C, d.ravel()[o])) < 1e-10


def test_gradient_matches_finite_differences():
    d, s2, mask = _problem(seed=3)
    th = np.array([1.3, -1.7, 0.9])
    k0 = 1.0 / 8
    g, gq = LL.loglike_grad_dense(d, s2, mask, th[0], th[1], k0, th[2])
    for i in range(3):
        h = 1e-5 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        Lp, Qp = LL.loglike_dense(d, s2, mask, tp[0], tp[1], k0, tp[2])
        Lm, Qm = LL.loglike_dense(d, s2, mask, tm[0], tm[1], k0, tm[2])
        assert abs(g[i] - (Lp - Lm) / (2 * h)) < 1e-6 * max(1.0, abs(g[i]))
        assert abs(gq[i] - (Qp - Qm) / (2 * h)) < 1e-6 * max(1.0, abs(gq[i]))


def test_wiener_param_dense_is_the_dense_wiener_filter():
    from oracle import dense
    d, s2, mask = _problem(seed=5)
    P, _, _ = LL.psd_tables(8, 8, 1.3, -1.7, 1.0 / 8)
    np.testing.assert_allclose(LL.wiener_param_dense(d, s2, mask, 1.3, -1.7, 1.0 / 8, 0.9),
                               dense.wiener_dense(d, 0.9 * s2, mask, P), rtol=1e-10, atol=1e-12)


def test_wiener_vjp_matches_finite_differences_of_the_dense_filter():
    d, s2, mask = _problem(seed=7)
    g = np.random.default_rng(1).standard_normal(d.shape)
    th = np.array([1.3, -1.7, 0.9])
    k0 = 1.0 / 8
    v = LL.wiener_vjp_dense(d, s2, mask, th[0], th[1], k0, th[2], g)
    for i in range(3):
        h = 1e-5 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = g.ravel() @ (LL.wiener_param_dense(d, s2, mask, tp[0], tp[1], k0, tp[2]) -
                          LL.wiener_param_dense(d, s2, mask, tm[0], tm[1], k0, tm[2])).ravel() / (2 * h)
        assert abs(v[i] - fd) < 1e-6 * max(1.0, abs(fd)), (i, v[i], fd)
