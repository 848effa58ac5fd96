"""GPU parity with a diagonal pixel response A (d = A s + n, Eq. 1; the Alg. 1 t-update with A_i^2 > 0):
samples draw for draw and Wiener filters against the oracle, which implements the general update."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import dense
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


def _problem(H, seed, zeros=5):
    p = synth.make_problem(H, seed=seed, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    rng = np.random.default_rng(seed + 7)
    A = rng.uniform(0.4, 1.6, size=(H, H)).astype(np.float32)
    A[rng.integers(0, H, zeros), rng.integers(0, H, zeros)] = 0.0
    return p, A


@pytest.mark.parametrize("H", [32, 128, 256])
def test_sampler_with_response_draw_for_draw(H):
    p, A = _problem(H, H)
    n = 3 if H < 256 else 2
    got = wf.wf_sample_ex(*to_dev(p), seed=11, n_samples=n, n_chains=2, chain_offset=4,
                          A=torch.from_numpy(A).cuda()).cpu().numpy()
    for c in range(2):
        ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, n, seed=11, chain=4 + c, A=A)
        for m in range(n):
            assert rel(got[c, m], ref[m]) < SAMPLE_TOL, (H, c, m)


@pytest.mark.parametrize("H", [16, 32])
def test_wiener_filter_with_response_matches_dense(H):
    p, A = _problem(H, H + 1)
    ref = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk, A=A)
    r = wf.wf_solve_ex(*to_dev(p), tol=1e-7, A=torch.from_numpy(A).cuda())
    assert r.status == 0 and rel(r.s.cpu().numpy(), ref) < WF_TOL
    rr = wf.wf_solve_ex(*to_dev(p), tol=1e-7, refine=8, A=torch.from_numpy(A).cuda())
    assert rr.status == 0 and rel(rr.s.cpu().numpy(), ref) < 1e-6
    rho = M.residual(rr.s.double().cpu().numpy(), p.d, p.Ndiag, p.mask, p.Pk, A=A)
    assert abs(rho - rr.resid) <= 1e-3 * rho + 1e-13, (rho, rr.resid)


def test_unit_response_is_the_identity_and_large_solve():
    p, _ = _problem(64, 3)
    ones = torch.ones((64, 64), dtype=torch.float32, device="cuda")
    a = wf.wf_sample_ex(*to_dev(p), seed=2, n_samples=2, A=ones)
    b = wf.wf_sample_ex(*to_dev(p), seed=2, n_samples=2)
    assert torch.equal(a, b)
    q, A = _problem(256, 5)
    q = synth.make_problem(256, seed=5, mask_frac=0.05, slope=-1.0, k0=1.0 / 4, sigma2=(0.5, 1.0))
    r = wf.wf_solve_ex(*to_dev(q), tol=1e-7, refine=4, A=torch.from_numpy(A).cuda())
    ref, _, rho = M.wf_solve(q.d, q.Ndiag, q.mask, q.Pk, tol=1e-10, A=A)
    assert r.status == 0 and rho < 1e-10
    assert rel(r.s.cpu().numpy(), ref) < WF_TOL
