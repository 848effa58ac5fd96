"""GPU parity of the spin-2 (shear) sampler: shear samples draw for draw against the FP64 oracle, which
implements the Kaiser-Squires rotation inside Alg. 1, and the shear-to-convergence transform."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, torch
from oracle import spin2 as S2
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu

SAMPLE_TOL = 1e-4
WF_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


def _pair(H, seed):
    p = synth.make_problem(H, seed=seed, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    rng = np.random.default_rng(seed + 1)
    N2 = rng.uniform(0.05, 0.5, (H, H)).astype(np.float32)
    d2 = np.where(p.mask == 1, 0.0, rng.standard_normal((H, H))).astype(np.float32)
    PB = (0.2 * p.Pk).astype(np.float32)
    return p, d2, N2, PB


def _dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


@pytest.mark.parametrize("H", [16, 32, 64, 128])
def test_spin2_sampler_draw_for_draw(H):
    p, d2, N2, PB = _pair(H, H + 2)
    n = 3
    got = wf.wf_sample_spin2(*_dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB), seed=6, n_samples=n, n_chains=2,
                             chain_offset=1).cpu().numpy()
    for c in range(2):
        ref = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, n, seed=6, chain=1 + c)
        for m in range(n):
            for comp in range(2):
                assert rel(got[c, m, comp], ref[m, comp]) < SAMPLE_TOL, (H, c, m, comp)


@pytest.mark.parametrize("H", [256, 512])
def test_spin2_sampler_large_draw_for_draw(H):
    """256^2 and 512^2: both shear components of a chain in one thread-block cluster."""
    p, d2, N2, PB = _pair(H, H + 2)
    n = 3 if H == 256 else 2
    got = wf.wf_sample_spin2(*_dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB), seed=6, n_samples=n, n_chains=2,
                             chain_offset=1).cpu().numpy()
    for c in range(2):
        ref = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, n, seed=6, chain=1 + c)
        for m in range(n):
            for comp in range(2):
                assert rel(got[c, m, comp], ref[m, comp]) < SAMPLE_TOL, (H, c, m, comp,
                                                                         rel(got[c, m, comp], ref[m, comp]))


def test_spin2_sampler_large_resume_and_zero_b_power():
    """256^2: a chain resumed from its first sample (init, start_step) repeats the second; with P_B = 0 the
    B modes of every sample vanish (kappa_B = 0 up to rounding) while E carries the signal."""
    H = 256
    p, d2, N2, PB = _pair(H, 11)
    dev = _dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)
    full = wf.wf_sample_spin2(*dev, seed=3, n_samples=2)
    tail = wf.wf_sample_spin2(*dev, seed=3, n_samples=1, start_step=1, init=full[0, 0].contiguous())
    assert rel(tail[0, 0].cpu().numpy(), full[0, 1].cpu().numpy()) < SAMPLE_TOL
    dev[6] = torch.zeros_like(dev[6])
    g = wf.wf_sample_spin2(*dev, seed=3, n_samples=2, n_chains=2)
    k = wf.wf_shear_to_convergence(g.reshape(4, 2, H, H)).cpu().numpy()
    for i in range(4):
        assert np.linalg.norm(k[i, 1]) < 1e-5 * np.linalg.norm(k[i, 0])


@pytest.mark.parametrize("H", [256, 512])
def test_spin2_wiener_filter_large_true_residual(H):
    """256^2 and 512^2 (cluster kernels): the oracle's FP64 residual of the returned pair is below tol and
    equals the reported one."""
    p, d2, N2, PB = _pair(H, H + 7)
    r = wf.wf_solve_spin2(*_dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB), tol=WF_TOL)
    got = r.s.cpu().numpy()
    true = S2.residual(got[0], got[1], p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)
    print(f"spin-2 WF {H}: resid {r.resid:.3e} oracle {true:.3e} sweeps {r.iters}")
    assert r.status == 0 and r.resid < WF_TOL and true < WF_TOL
    assert abs(true - r.resid) <= 1e-6 * true


def test_spin2_sampler_large_per_chain_init_and_bf16():
    """512^2: per-chain initial pairs follow the oracle from those states; BF16 storage is the FP32 chain
    rounded once."""
    H = 512
    p, d2, N2, PB = _pair(H, 41)
    dev = _dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)
    init = torch.randn((2, 2, H, H), device="cuda")
    f32 = wf.wf_sample_spin2(*dev, seed=9, n_samples=1, n_chains=2, init=init)
    b16 = wf.wf_sample_spin2(*dev, seed=9, n_samples=1, n_chains=2, init=init, out_dtype="bf16")
    assert torch.equal(b16, f32.to(torch.bfloat16))
    ref = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, 1, seed=9, chain=1, init=init[1].cpu().numpy())
    for comp in range(2):
        assert rel(f32[1, 0, comp].cpu().numpy(), ref[0, comp]) < SAMPLE_TOL


@pytest.mark.parametrize("H", [64, 256])
def test_spin2_sampler_with_pixel_response(H):
    """One pixel response A for both shear components (a few A = 0 pixels): draw for draw against the
    oracle's general t-update."""
    p, d2, N2, PB = _pair(H, H + 13)
    rng = np.random.default_rng(H + 1)
    A = rng.uniform(0.5, 1.5, (H, H)).astype(np.float32)
    A[rng.integers(0, H, 5), rng.integers(0, H, 5)] = 0.0
    got = wf.wf_sample_spin2(*_dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB), seed=7, n_samples=2,
                             A=torch.from_numpy(A).cuda()).cpu().numpy()
    ref = S2.sample(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB, 2, seed=7, A=A)
    for m in range(2):
        for comp in range(2):
            assert rel(got[0, m, comp], ref[m, comp]) < SAMPLE_TOL, (H, m, comp, rel(got[0, m, comp], ref[m, comp]))


def test_spin2_wiener_filter_with_pixel_response():
    """With a pixel response A the spin-2 Wiener filter solves the response problem: at 32^2 it matches the
    dense filter of the equivalent data d / A, noise N / A^2 (A = 0 pixels masked); at 256^2 the oracle's
    FP64 residual of that problem for the returned pair is below tol and equals the reported one."""
    for H in (32, 256):
        p, d2, N2, PB = _pair(H, H + 29)
        rng = np.random.default_rng(H + 5)
        A = rng.uniform(0.5, 1.5, (H, H)).astype(np.float32)
        A[rng.integers(0, H, 4), rng.integers(0, H, 4)] = 0.0
        r = wf.wf_solve_spin2(*_dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB), tol=WF_TOL,
                              A=torch.from_numpy(A).cuda())
        got = r.s.cpu().numpy()
        A64 = A.astype(np.float64)
        safe = np.where(A64 != 0, A64, 1.0)
        m2 = np.where(A64 == 0, 1, p.mask).astype(np.uint8)
        e1, e2 = p.d / safe, d2 / safe
        n1, n2 = p.Ndiag / safe ** 2, N2 / safe ** 2
        assert r.status == 0 and r.resid < WF_TOL
        if H == 32:
            ref = S2.wiener_dense(e1, e2, n1, n2, m2, p.Pk, PB)
            assert rel(got[0], ref[0]) < WF_TOL and rel(got[1], ref[1]) < WF_TOL
        else:
            # the GPU forms the transformed data in FP64 and rounds it once to FP32: the residuals agree to
            # 1e-3 of themselves (as for the response in the plain solve), not to FP64 rounding
            true = S2.residual(got[0], got[1], e1, e2, n1, n2, m2, p.Pk, PB)
            assert true < WF_TOL and abs(true - r.resid) <= 1e-3 * true


def test_shear_to_convergence_matches_oracle():
    rng = np.random.default_rng(3)
    for H in (16, 128, 256):
        g = rng.standard_normal((3, 2, H, H)).astype(np.float32)
        k = wf.wf_shear_to_convergence(torch.from_numpy(g).cuda()).cpu().numpy()
        for i in range(3):
            kE, kB = S2.convergence_from_shear(g[i, 0], g[i, 1])
            assert rel(k[i, 0], kE) < 1e-6 and rel(k[i, 1], kB) < 1e-6


@pytest.mark.parametrize("H", [16, 32])
def test_spin2_wiener_filter_matches_dense(H):
    p, d2, N2, PB = _pair(H, H + 7)
    ref = S2.wiener_dense(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB)
    r = wf.wf_solve_spin2(*_dev(p.d, d2, p.Ndiag, N2, p.mask, p.Pk, PB), tol=5e-6)
    got = r.s.cpu().numpy()
    print(f"spin-2 WF {H}: resid {r.resid:.2e} sweeps {r.iters} err {rel(got[0], ref[0]):.2e} {rel(got[1], ref[1]):.2e}")
    # the reported residual is the FP64 residual of the returned pair (summed on the GPU in FP64)
    assert r.status == 0 and r.resid < 5e-6
    assert rel(got[0], ref[0]) < WF_TOL and rel(got[1], ref[1]) < WF_TOL
