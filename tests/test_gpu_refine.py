"""Mixed-precision iterative refinement of the Wiener filter (FP32 messenger solves, FP64 residuals).

The FP32 messenger iteration stalls at a relative residual of a few 1e-6 (its FFT round-off); with
``refine`` > 0 the library evaluates r = N^-1 (d - s) - S^-1 s and ||S r|| / ||S N^-1 d|| in FP64 on the
GPU and adds FP32 messenger solutions of (S^-1 + N^-1) e = r. These tests check the returned map against
the dense FP64 Wiener filter (Eq. 2-3), check the reported residual against the oracle's FP64 residual
of the same map, and run the 1024x1024 precision case (P ~ k^-1.5, noise range 100, 25% circular holes)
to relative residual 1e-7. The returned map is FP32, so its own residual floors near 1e-8.
"""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev
from oracle import dense
from oracle import messenger as M
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


def kbin_errors(got, ref, nbins=6):
    """Relative error per |k| bin (unitary spectra, half plane): ||F(got - ref)||_bin / ||F ref||_bin."""
    H, W = ref.shape
    ky = np.fft.fftfreq(H)[:, None]
    kx = (np.arange(W // 2 + 1) / W)[None, :]
    k = np.sqrt(ky * ky + kx * kx)
    E = np.fft.rfft2(np.asarray(got, np.float64) - ref)
    R = np.fft.rfft2(ref)
    edges = np.linspace(0.0, k.max() + 1e-12, nbins + 1)
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        sel = (k >= a) & (k < b)
        den = np.linalg.norm(R[sel])
        out.append(np.linalg.norm(E[sel]) / den if den > 0 else 0.0)
    return np.array(out)


SMALL = {32: dict(n_holes=8, r_range=(1.5, 5.0)), 64: dict(n_holes=16, r_range=(2.0, 8.0))}


@pytest.mark.parametrize("H", [32, 64])
def test_refined_matches_dense(H):
    p = synth.config_precision(H, seed=H, **SMALL[H])
    ref = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk)
    plain = wf.wf_solve_ex(*to_dev(p), tol=1e-5, max_iter=400000, refine=0)
    r = wf.wf_solve_ex(*to_dev(p), tol=1e-7, refine=8, refine_tol=1e-3, max_iter=400000)
    assert r.status == 0 and r.resid < 1e-7, (r.status, r.resid)
    s = r.s.double().cpu().numpy()
    rho = M.residual(s, p.d, p.Ndiag, p.mask, p.Pk)
    assert abs(rho - r.resid) <= 1e-3 * rho + 1e-14, (rho, r.resid)
    e_ref, e_plain = rel(s, ref), rel(plain.s.cpu().numpy(), ref)
    kb = kbin_errors(s, ref)
    print(f"H={H} plain err {e_plain:.2e}  refined err {e_ref:.2e} (resid {r.resid:.2e}, {r.iters} sweeps)  "
          f"per-k-bin {np.array2string(kb, precision=1)}")
    assert e_ref < 1e-6
    assert kb.max() < 1e-5


def test_refined_paper128_vs_plain_floor():
    p = synth.config_paper128()
    r = wf.wf_solve_ex(*to_dev(p), tol=2e-8, refine=8, refine_tol=1e-3)
    assert r.status == 0 and r.resid < 2e-8
    s = r.s.double().cpu().numpy()
    assert abs(M.residual(s, p.d, p.Ndiag, p.mask, p.Pk) - r.resid) <= 1e-3 * r.resid + 1e-14


def test_refine_reports_not_converged_when_steps_run_out():
    p = synth.config_paper128()
    r = wf.wf_solve_ex(*to_dev(p), tol=1e-14, refine=1, refine_tol=1e-2, allow_not_converged=True)
    assert r.status == 5 and r.resid > 1e-14
    s = r.s.double().cpu().numpy()
    assert abs(M.residual(s, p.d, p.Ndiag, p.mask, p.Pk) - r.resid) <= 1e-3 * r.resid + 1e-14


def test_precision_1024_to_1e7():
    p = synth.config_precision(1024, seed=0)
    r = wf.wf_solve_ex(*to_dev(p), tol=1e-7, refine=8, refine_tol=1e-3, max_iter=400000)
    assert r.status == 0 and r.resid < 1e-7, (r.status, r.resid)
    s = r.s.double().cpu().numpy()
    rho = M.residual(s, p.d, p.Ndiag, p.mask, p.Pk)
    print(f"1024x1024 precision case: resid {r.resid:.3e} (oracle FP64 {rho:.3e}), {r.iters} sweeps")
    assert rho < 1.01e-7
    assert abs(rho - r.resid) <= 1e-3 * rho + 1e-14
