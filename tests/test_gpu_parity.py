"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the same seeded inputs.

Tolerances (stated in the task and derived from FP32 arithmetic): samples draw-for-draw within 1e-4
relative L2 per sample; Wiener filter within 1e-5 relative L2 of the exact (dense / oracle) solution.
"""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import dense, messenger as M
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu

SAMPLE_TOL = 1e-4
WF_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


def test_plain32_wiener_filter_matches_dense():
    """The plain 32x32 case: a solve to relative residual 1e-6 delivers it. The residual the call reports is
    the FP64 residual of the map it returns, so the oracle's own FP64 residual of that map agrees with it."""
    p = synth.config_plain32(0)
    r = wf.wf_solve(*to_dev(p), tol=1e-6)
    ref = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk)
    s = r.s.cpu().numpy()
    assert r.status == 0 and 0 < r.resid < 1e-6
    assert rel(s, ref) < WF_TOL
    rho = M.residual(s.astype(np.float64), p.d, p.Ndiag, p.mask, p.Pk)
    assert rho < 1e-6
    assert abs(rho - r.resid) <= 1e-3 * rho + 1e-14, (rho, r.resid)


@pytest.mark.parametrize("H", [16, 32, 64, 128, 256, 512, 1024])
def test_reported_residual_is_the_true_residual(H):
    """At every size the default solve's reported residual is the FP64 residual of the returned map (the
    oracle's, to 1e-3 of itself) and is below the requested tolerance."""
    if H == 128:
        p = synth.config_paper128(0)
    elif H <= 64:
        p = synth.make_problem(H, seed=H + 5, mask_frac=0.1, block=(1, H // 4, 2, H // 3))
    else:
        p = synth.make_problem(H, seed=H + 5, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    r = wf.wf_solve(*to_dev(p), tol=1e-6)
    assert r.status == 0 and 0 <= r.resid < 1e-6, (r.status, r.resid)
    rho = M.residual(r.s.double().cpu().numpy(), p.d, p.Ndiag, p.mask, p.Pk)
    assert rho < 1e-6 and abs(rho - r.resid) <= 1e-3 * rho + 1e-14, (H, rho, r.resid)


def test_plain32_1000_samples_draw_for_draw():
    p = synth.config_plain32(0)
    got = wf.wf_sample(*to_dev(p), 1000, seed=2024).cpu().numpy()
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 1000, seed=2024)
    errs = np.array([rel(got[i], ref[i]) for i in range(1000)])
    assert errs.max() < SAMPLE_TOL, errs.max()


@pytest.mark.parametrize("H", [16, 32, 64, 128])
def test_sample_chains_burn_thin(H):
    p = synth.make_problem(H, seed=H, mask_frac=0.1, block=(1, H // 4, 2, H // 3))
    chains = [0, 3, 5]
    got = wf.wf_sample_ex(*to_dev(p), seed=11, n_samples=4, n_chains=6, chain_offset=100, burn_in=3,
                          thin=2).cpu().numpy()
    for c in chains:
        ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 4, seed=11, chain=100 + c, burn_in=3, thin=2)
        for m in range(4):
            assert rel(got[c, m], ref[m]) < SAMPLE_TOL, (H, c, m)


@pytest.mark.parametrize("H", [16, 64, 128])
def test_wiener_filter_sizes(H):
    p = synth.config_paper128(0) if H == 128 else synth.make_problem(H, seed=H + 1, mask_frac=0.12,
                                                                      block=(2, H // 3, H // 4, H // 2))
    # the FP32 iteration's fixed point sits ~3e-6 from the exact filter at 128^2 (FP32 transform
    # round-off), so the residual target is set below the default to keep the error under WF_TOL
    r = wf.wf_solve(*to_dev(p), tol=1e-7)
    assert r.status == 0
    s = r.s.cpu().numpy()
    if H <= 16:
        ref = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk)
    else:
        ref, _, rho = M.wf_solve(p.d, p.Ndiag, p.mask, p.Pk, tol=1e-9)
        assert rho < 1e-9
    assert rel(s, ref) < WF_TOL, rel(s, ref)


def test_full_size_128_1024_chains_sampled():
    """The benchmark configuration (128^2, 1024 chains x 100 samples, one launch): sampled chains vs oracle."""
    p = synth.config_paper128(0)
    got = wf.wf_sample_ex(*to_dev(p), seed=7, n_samples=100, n_chains=1024)
    assert got.shape == (1024, 100, 128, 128)
    assert bool(torch.isfinite(got).all())
    for c in (0, 511, 1023):
        ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 100, seed=7, chain=c)
        g = got[c].cpu().numpy()
        errs = [rel(g[m], ref[m]) for m in range(100)]
        assert max(errs) < SAMPLE_TOL, (c, max(errs))


def test_full_size_128_one_long_chain_thin_10_sampled():
    """The long-chain configuration (one chain, 10^4 kept samples of 10^5 sweeps, thin 10): the first kept
    samples and a later one vs the oracle (each sample needs only the sweeps before it)."""
    p = synth.config_paper128(0)
    got = wf.wf_sample_ex(*to_dev(p), seed=11, n_samples=10000, n_chains=1, thin=10)
    assert got.shape == (1, 10000, 128, 128) and bool(torch.isfinite(got).all())
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 30, seed=11, thin=10)
    g = got[0, :30].cpu().numpy()
    assert max(rel(g[m], ref[m]) for m in range(30)) < SAMPLE_TOL


def test_resume_is_exact_and_runs_are_deterministic():
    p = synth.make_problem(64, seed=2, mask_frac=0.1)
    dev = to_dev(p)
    a = wf.wf_sample_ex(*dev, seed=5, n_samples=10, n_chains=2)
    b = wf.wf_sample_ex(*dev, seed=5, n_samples=10, n_chains=2)
    assert torch.equal(a, b)
    r = wf.wf_sample_ex(*dev, seed=5, n_samples=4, n_chains=2, start_step=6, init_s=a[:, 5].contiguous())
    assert torch.equal(r, a[:, 6:10])


def test_missing_pixel_values_are_ignored():
    p = synth.make_problem(32, seed=4, mask_frac=0.2)
    d2 = p.d.copy()
    d2[p.mask == 1] = 1e30
    dev = to_dev(p)
    dev2 = (torch.from_numpy(d2).cuda(),) + dev[1:]
    assert torch.equal(wf.wf_sample(*dev, 5, seed=1), wf.wf_sample(*dev2, 5, seed=1))
    assert torch.equal(wf.wf_solve(*dev).s, wf.wf_solve(*dev2).s)


def test_all_masked_and_zero_power():
    q = synth.flat_problem(32, seed=1, all_masked=True)
    r = wf.wf_solve(*to_dev(q))
    assert float(r.s.abs().max()) == 0.0
    x = wf.wf_sample(*to_dev(q), 200, seed=3).cpu().numpy()
    ref = M.sample(q.d, q.Ndiag, q.mask, q.Pk, 200, seed=3)
    assert max(rel(x[i], ref[i]) for i in range(200)) < SAMPLE_TOL
    p = synth.make_problem(32, seed=2)
    dev = list(to_dev(p))
    dev[3] = torch.zeros_like(dev[3])
    assert float(wf.wf_sample(*dev, 4, seed=1).abs().max()) == 0.0
    assert float(wf.wf_solve(*dev).s.abs().max()) == 0.0


def test_homogeneous_noise_gives_diagonal_wiener_filter():
    p = synth.flat_problem(64, seed=3, sigma2=0.3)
    p.Pk[:] = synth.power_law_pk(64, 64, 1.0, -2.0)
    r = wf.wf_solve(*to_dev(p), tol=1e-6)
    Ph = p.Pk.astype(np.float64)
    ref = np.fft.irfft2(Ph / (Ph + float(p.Ndiag[0, 0])) * np.fft.rfft2(p.d.astype(np.float64)), s=(64, 64))
    assert rel(r.s.cpu().numpy(), ref) < WF_TOL


def test_error_statuses():
    p = synth.make_problem(32, seed=6, mask_frac=0.1)
    dev = to_dev(p)
    tau_bad = float(p.Ndiag[p.mask == 0].min()) * 1.5
    with pytest.raises(wf.WFError) as e:
        wf.wf_solve(*dev, tau=tau_bad)
    assert e.value.status == 2
    with pytest.raises(wf.WFError) as e:
        wf.wf_sample_ex(*dev, seed=1, n_samples=2, tau=tau_bad)
    assert e.value.status == 2
    d_nan = dev[0].clone()
    idx = np.argwhere(p.mask == 0)[0]
    d_nan[idx[0], idx[1]] = float("nan")
    with pytest.raises(wf.WFError) as e:
        wf.wf_sample(d_nan, *dev[1:], 2, seed=1)
    assert e.value.status == 6
    r = wf.wf_solve_ex(*dev, tol=1e-12, max_iter=3, refine=0, allow_not_converged=True)
    assert r.status == 5 and r.iters == 3
    out = torch.full((0, 32, 32), 0.0, device="cuda")
    assert wf.wf_sample(*dev, 0, seed=1, out=out).shape == (0, 32, 32)
    # a caller-chosen tau below the minimum is valid and gives the same Wiener filter
    t = float(p.Ndiag[p.mask == 0].min()) * 0.5
    a = wf.wf_solve(*dev, tol=1e-7).s.cpu().numpy()
    b = wf.wf_solve(*dev, tau=t, tol=1e-7).s.cpu().numpy()
    assert rel(b, a) < WF_TOL


def test_posterior_moments_16():
    """Many independent chains after burn-in: mean vs s_W and covariance vs C_post (Eq. 4)."""
    p = synth.make_problem(16, seed=8, mask_frac=0.15, slope=-2.0, k0=1.0 / 16, sigma2=(0.2, 1.0))
    n_chains = 20000
    x = wf.wf_sample_ex(*to_dev(p), seed=99, n_samples=1, n_chains=n_chains, burn_in=60)
    x = x[:, 0].reshape(n_chains, -1).double().cpu().numpy()
    sW = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk).ravel()
    C = dense.posterior_cov_dense(p.Ndiag, p.mask, p.Pk)
    z = (x.mean(0) - sW) / np.sqrt(np.diag(C) / n_chains)
    assert np.max(np.abs(z)) < 5.0
    Cs = np.cov(x.T)
    se = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / n_chains)
    assert np.max(np.abs(Cs - C) / se) < 6.0
