"""GPU parity of the large-image paths: N = 256 and 512 sample with one thread-block cluster per chain
(the field in distributed shared memory) or with the fields in global memory (one cooperative kernel, also
the Wiener filter and N = 1024); both run the oracle's chain draw for draw."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import messenger as M
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu

SAMPLE_TOL = 1e-4
WF_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


@pytest.fixture(params=["cluster", "global"])
def sampler(request):
    prev = wf.wf_set_large_image_sampler(request.param)
    yield request.param
    wf.wf_set_large_image_sampler(prev)


@pytest.mark.parametrize("H", [256, 512])
def test_sample_large_draw_for_draw(H, sampler):
    p = synth.make_problem(H, seed=H, mask_frac=0.1, block=(10, 60, 20, 90), slope=-2.0, k0=1.0 / 32,
                           sigma2=(0.05, 0.5))
    n_samples = 3 if H == 256 else 2
    got = wf.wf_sample_ex(*to_dev(p), seed=13, n_samples=n_samples, n_chains=3, chain_offset=7, burn_in=1)
    got = got.cpu().numpy()
    for c in ([0, 2] if H == 256 else [1]):
        ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, n_samples, seed=13, chain=7 + c, burn_in=1)
        for m in range(n_samples):
            assert rel(got[c, m], ref[m]) < SAMPLE_TOL, (H, c, m, rel(got[c, m], ref[m]))


@pytest.mark.parametrize("H", [256, 512])
def test_cluster_and_global_samplers_agree(H):
    """Many chains with thinning, per-chain initial states and BF16 storage: the cluster sampler and the
    global-memory sampler draw the same chain (FP32 results agree to rounding, ragged chain count)."""
    p = synth.make_problem(H, seed=H + 1, mask_frac=0.15, slope=-1.5, k0=1.0 / 16, sigma2=(0.02, 0.8))
    dev = to_dev(p)
    chains = 7 if H == 256 else 3
    g = torch.Generator().manual_seed(H)
    init = torch.randn((chains, H, H), generator=g).cuda() * 0.1
    kw = dict(seed=77, n_samples=3, n_chains=chains, chain_offset=5, start_step=11, burn_in=2, thin=2, init_s=init)
    out = {}
    for mode in ("cluster", "global"):
        prev = wf.wf_set_large_image_sampler(mode)
        try:
            out[mode] = wf.wf_sample_ex(*dev, **kw).cpu().numpy()
            out[mode + "_bf16"] = wf.wf_sample_ex(*dev, out_dtype="bf16", **kw).float().cpu().numpy()
        finally:
            wf.wf_set_large_image_sampler(prev)
    for c in range(chains):
        for m in range(3):
            assert rel(out["cluster"][c, m], out["global"][c, m]) < 1e-5, (c, m)
            assert rel(out["cluster_bf16"][c, m], out["cluster"][c, m]) < 2.0 ** -8
    # and the first chain is the oracle's (chain word 5, step words from 11)
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 2 + 3 * 2, seed=77, chain=5, start_step=11,
                   init_s=init[0].cpu().numpy())
    for m in range(3):
        assert rel(out["cluster"][0, m], ref[2 + 2 * m + 1]) < SAMPLE_TOL


@pytest.mark.parametrize("H,below", [(256, 31), (512, 7)])
def test_automatic_path_switch_keeps_the_chain(H, below):
    """In the default (automatic) mode 31 chains of 256^2 (7 of 512^2) run on the global-memory kernels and
    one more on clusters; the chains they share (same chain words) agree to FP32 rounding."""
    p = synth.make_problem(H, seed=31, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    prev = wf.wf_set_large_image_sampler("auto")
    try:
        few = wf.wf_sample_ex(*dev, seed=5, n_samples=2, n_chains=below, chain_offset=3).cpu().numpy()
        many = wf.wf_sample_ex(*dev, seed=5, n_samples=2, n_chains=below + 1, chain_offset=3).cpu().numpy()
    finally:
        wf.wf_set_large_image_sampler(prev)
    for c in (0, below // 2, below - 1):
        for m in range(2):
            assert rel(few[c, m], many[c, m]) < 1e-5, (c, m)


@pytest.mark.parametrize("H", [256, 512])
def test_large_degenerate_cases(H, sampler):
    """Zero power: every sample and the filter are exactly 0. Every pixel missing: the filter is 0 and the
    samples are draws from the prior, the oracle's draw for draw."""
    p = synth.make_problem(H, seed=H + 17, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = list(to_dev(p))
    dev[3] = torch.zeros_like(dev[3])
    assert float(wf.wf_sample_ex(*dev, seed=1, n_samples=2, n_chains=16).abs().max()) == 0.0
    assert float(wf.wf_solve(*dev).s.abs().max()) == 0.0
    q = synth.flat_problem(H, seed=2, all_masked=True)
    assert float(wf.wf_solve(*to_dev(q)).s.abs().max()) == 0.0
    got = wf.wf_sample_ex(*to_dev(q), seed=4, n_samples=2, n_chains=16, chain_offset=1).cpu().numpy()
    ref = M.sample(q.d, q.Ndiag, q.mask, q.Pk, 2, seed=4, chain=1)
    for m in range(2):
        assert rel(got[0, m], ref[m]) < SAMPLE_TOL, m


def test_sample_1024_one_sweep():
    p = synth.make_problem(1024, seed=4, mask_frac=0.05, slope=-1.5, sigma2=(0.001, 0.1))
    got = wf.wf_sample_ex(*to_dev(p), seed=3, n_samples=1, n_chains=1).cpu().numpy()
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 1, seed=3)
    assert rel(got[0, 0], ref[0]) < SAMPLE_TOL


def _easy(H):
    # small signal-to-noise range so that the iteration converges in tens of sweeps
    return synth.make_problem(H, seed=H + 3, mask_frac=0.05, slope=-1.0, k0=1.0 / 4, sigma2=(0.5, 1.0))


@pytest.mark.parametrize("H", [256, 512])
def test_wiener_filter_large(H, sampler):
    p = _easy(H)
    r = wf.wf_solve(*to_dev(p), tol=1e-7)
    assert r.status == 0
    ref, it, rho = M.wf_solve(p.d, p.Ndiag, p.mask, p.Pk, tol=1e-10)
    assert rho < 1e-10
    assert rel(r.s.cpu().numpy(), ref) < WF_TOL


@pytest.mark.parametrize("H", [256, 512])
def test_wiener_filter_cluster_and_global_agree(H):
    """A harder problem (slope -2, k0 = 1/32, 15% masked, noise U[0.02, 0.8]: many cooling levels): the
    cluster and global-memory solves take the same schedule and reach the same filter."""
    p = synth.make_problem(H, seed=H + 9, mask_frac=0.15, slope=-2.0, k0=1.0 / 32, sigma2=(0.02, 0.8))
    dev = to_dev(p)
    res = {}
    for mode in ("cluster", "global"):
        prev = wf.wf_set_large_image_sampler(mode)
        try:
            res[mode] = wf.wf_solve_ex(*dev, tol=1e-6, max_iter=20000, refine=0)
        finally:
            wf.wf_set_large_image_sampler(prev)
    c, g = res["cluster"], res["global"]
    assert c.status == 0 and g.status == 0
    assert abs(c.iters - g.iters) <= 8, (c.iters, g.iters)
    assert rel(c.s.cpu().numpy(), g.s.cpu().numpy()) < 1e-5
    s = c.s.double().cpu().numpy()
    assert _residual_fft(s, p) < 2e-6


def _residual_fft(s, p):
    """||s + S N^-1 (s - d)|| / ||S N^-1 d|| with numpy.fft (unitary; N^-1 = 0 on missing pixels)."""
    obs = p.mask == 0
    Ninv = np.where(obs, 1.0 / p.Ndiag.astype(np.float64), 0.0)
    P = p.Pk.astype(np.float64)
    H, W = p.d.shape
    S = lambda v: np.fft.irfft2(P * np.fft.rfft2(v, norm="ortho"), s=(H, W), norm="ortho")
    d = p.d.astype(np.float64)
    b = S(Ninv * d)
    r = s + S(Ninv * (s - d))
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_wiener_filter_1024_converges():
    p = synth.make_problem(1024, seed=9, mask_frac=0.1, slope=-1.5, sigma2=(0.01, 0.1))
    r = wf.wf_solve_ex(*to_dev(p), tol=1e-6, max_iter=20000)
    assert r.status == 0
    s = r.s.double().cpu().numpy()
    assert _residual_fft(s, p) < 2e-5
