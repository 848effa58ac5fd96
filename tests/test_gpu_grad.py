"""GPU checks of the differentiation form: spectral powers vs numpy.fft, gradients vs the dense oracle
(exact trace, 16x16) and vs central finite differences of the data term (256x256, h = 1e-3, to 1e-4)."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import likelihood as LL
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


@pytest.mark.parametrize("H", [32, 128, 256])
def test_spectral_power_matches_numpy(H):
    rng = np.random.default_rng(H)
    a = rng.standard_normal((3, H, H)).astype(np.float32)
    b = rng.standard_normal((3, H, H)).astype(np.float32)
    w = np.stack([synth.power_law_pk(H, H, 1.0, -2.0), synth.power_law_pk(H, H, 0.5, -1.0)]).astype(np.float32)
    got = wf.wf_spectral_power(torch.from_numpy(a).cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda(), -1.0)
    for f in range(3):
        V = np.fft.fft2((a[f] - b[f]).astype(np.float64), norm="ortho")
        for j in range(2):
            wfull = np.empty((H, H))
            wfull[:, : H // 2 + 1] = w[j]
            wfull[:, H // 2 + 1:] = w[j][(-np.arange(H)) % H][:, (H - np.arange(H // 2 + 1, H))]
            ref = float(np.sum(wfull * np.abs(V) ** 2))
            assert abs(got[f, j] - ref) < 1e-5 * ref


def _prob16(seed):
    p = synth.make_problem(16, seed=seed, mask_frac=0.1, slope=-2.0, k0=1.0 / 16, sigma2=(0.05, 0.3))
    return p


def test_gradient_matches_dense_oracle_16():
    p = _prob16(5)
    amp, slope, k0, alpha = 1.3, -1.8, 1.0 / 16, 0.9
    dev = to_dev(p)
    r = wf.wf_loglike_grad(dev[0], dev[1], dev[2], amp, slope, k0, alpha, n_probes=400, seed=3, tol=1e-7)
    g_ref, gq_ref = LL.loglike_grad_dense(p.d, p.Ndiag, p.mask, amp, slope, k0, alpha)
    _, q_ref = LL.loglike_dense(p.d, p.Ndiag, p.mask, amp, slope, k0, alpha)
    assert abs(r.quad - q_ref) < 1e-4 * abs(q_ref)
    np.testing.assert_allclose(r.grad_quad, gq_ref, rtol=1e-4)
    sd = np.sqrt(r.grad_var)
    assert np.all(np.abs(r.grad - g_ref) < 5 * sd + 1e-4 * np.abs(g_ref)), (r.grad, g_ref, sd)


def test_gradient_quad_term_matches_finite_differences_256():
    rng = np.random.default_rng(0)
    H = 256
    amp, slope, alpha = float(rng.uniform(0.5, 2)), float(rng.uniform(-2.5, -1.5)), 1.0
    k0 = 1.0 / H
    p = synth.make_problem(H, seed=1, mask_frac=0.1, slope=slope, amp=amp, k0=k0, sigma2=(0.01, 0.2))
    dev = to_dev(p)
    r = wf.wf_loglike_grad(dev[0], dev[1], dev[2], amp, slope, k0, alpha, tol=1e-7, with_trace=False)
    th = np.array([amp, slope, alpha])
    for i in range(3):
        h = 1e-3 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        qp = wf.wf_loglike_grad(dev[0], dev[1], dev[2], tp[0], tp[1], k0, tp[2], tol=1e-7, with_trace=False).quad
        qm = wf.wf_loglike_grad(dev[0], dev[1], dev[2], tm[0], tm[1], k0, tm[2], tol=1e-7, with_trace=False).quad
        fd = (qp - qm) / (2 * h)
        # the solves' FP64 residual is below 1e-7, so the data term is accurate to far below what h = 1e-3
        # differences need for 1e-4; the central difference's own truncation error is O(h^2)
        assert abs(r.grad_quad[i] - fd) < 1e-4 * abs(fd) + 1e-6, (i, r.grad_quad[i], fd)


def test_autograd_function_returns_the_gradient():
    p = _prob16(7)
    dev = to_dev(p)
    theta = torch.tensor([1.1, -2.0, 1.2], dtype=torch.float64, requires_grad=True)
    q = wf.wiener_loglik(theta, dev[0], dev[1], dev[2], 1.0 / 16, 64, 9, 1e-6)
    q.backward()
    r = wf.wf_loglike_grad(dev[0], dev[1], dev[2], 1.1, -2.0, 1.0 / 16, 1.2, n_probes=64, seed=9, tol=1e-6)
    np.testing.assert_allclose(theta.grad.numpy(), r.grad, rtol=1e-12)
    assert abs(q.item() - r.quad) < 1e-12 * abs(r.quad)


# ---------------------------------------------------------------------------------------------------
# Wiener-map vector-Jacobian product (one adjoint solve; C is symmetric)
# ---------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("H", [16, 32])
def test_wiener_vjp_matches_dense_oracle(H):
    p = synth.make_problem(H, seed=H + 1, mask_frac=0.1, slope=-2.0, k0=1.0 / H, sigma2=(0.05, 0.3))
    amp, slope, k0, alpha = 1.3, -1.8, 1.0 / H, 0.9
    g = np.random.default_rng(H).standard_normal((H, H)).astype(np.float32)
    dev = to_dev(p)
    s, v = wf.wf_wiener_vjp(dev[0], dev[1], dev[2], amp, slope, k0, alpha, torch.from_numpy(g).cuda(), tol=3e-8)
    s_ref = LL.wiener_param_dense(p.d, p.Ndiag, p.mask, amp, slope, k0, alpha)
    v_ref = LL.wiener_vjp_dense(p.d, p.Ndiag, p.mask, amp, slope, k0, alpha, g)
    assert rel(s.cpu().numpy(), s_ref) < 1e-6
    np.testing.assert_allclose(v, v_ref, rtol=1e-4, atol=1e-6 * np.abs(v_ref).max())


def test_wiener_vjp_matches_finite_differences_256():
    rng = np.random.default_rng(5)
    H = 256
    amp, slope, alpha = float(rng.uniform(0.5, 2)), float(rng.uniform(-2.5, -1.5)), 1.0
    k0 = 1.0 / H
    p = synth.make_problem(H, seed=2, mask_frac=0.1, slope=slope, amp=amp, k0=k0, sigma2=(0.01, 0.2))
    dev = to_dev(p)
    g = torch.from_numpy(rng.standard_normal((H, H)).astype(np.float32)).cuda()
    _, v = wf.wf_wiener_vjp(dev[0], dev[1], dev[2], amp, slope, k0, alpha, g, tol=3e-8)
    th = np.array([amp, slope, alpha])
    gd = g.double()
    for i in range(3):
        h = 1e-3 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        sp, _ = wf.wf_wiener_vjp(dev[0], dev[1], dev[2], tp[0], tp[1], k0, tp[2], tol=3e-8)
        sm, _ = wf.wf_wiener_vjp(dev[0], dev[1], dev[2], tm[0], tm[1], k0, tm[2], tol=3e-8)
        fd = float((gd * (sp.double() - sm.double())).sum()) / (2 * h)
        assert abs(v[i] - fd) < 1e-3 * abs(fd) + 1e-6, (i, v[i], fd)


def test_wiener_map_autograd_uses_the_checkpointed_forward():
    p = _prob16(11)
    dev = to_dev(p)
    g = torch.from_numpy(np.random.default_rng(2).standard_normal((16, 16)).astype(np.float32)).cuda()
    theta = torch.tensor([0.9, -1.6, 1.1], dtype=torch.float64, requires_grad=True)
    s = wf.wiener_map(theta, dev[0], dev[1], dev[2], 1.0 / 16, 3e-8)
    (s.double() * g.double()).sum().backward()
    s2, v = wf.wf_wiener_vjp(dev[0], dev[1], dev[2], 0.9, -1.6, 1.0 / 16, 1.1, g, tol=3e-8)
    assert rel(s.detach().cpu().numpy(), s2.cpu().numpy()) < 1e-7
    np.testing.assert_allclose(theta.grad.numpy(), v, rtol=1e-6)


def test_batched_loglike_gradient_equals_single_calls():
    rng = np.random.default_rng(9)
    imgs, probs = [], []
    for i, H in enumerate([16, 64, 256, 256, 128]):
        amp, slope = float(rng.uniform(0.5, 2)), float(rng.uniform(-2.5, -1.5))
        p = synth.make_problem(H, seed=40 + i, mask_frac=0.1, slope=slope, amp=amp, k0=1.0 / H, sigma2=(0.01, 0.2))
        dev = to_dev(p)
        imgs.append((dev[0], dev[1], dev[2], amp, slope, 1.0 / H, 1.0, 7 + i))
        probs.append(p)
    got = wf.wf_loglike_grad_batch(imgs, n_probes=4, tol=1e-6)
    for (d, s2, m, amp, slope, k0, alpha, seed), g in zip(imgs, got):
        r = wf.wf_loglike_grad(d, s2, m, amp, slope, k0, alpha, n_probes=4, seed=seed, tol=1e-6)
        assert abs(g.quad - r.quad) < 1e-4 * abs(r.quad)
        np.testing.assert_allclose(g.grad_quad, r.grad_quad, rtol=1e-3)
        sd = np.sqrt(r.grad_var) + 1e-12
        # same probes, solves to the same tolerance: the stochastic gradients agree far inside their error
        assert np.all(np.abs(g.grad - r.grad) < 0.05 * sd + 1e-3 * np.abs(r.grad)), (g.grad, r.grad, sd)
