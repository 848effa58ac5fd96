"""GPU parity of the hierarchical Gibbs sampler (Alg. 1 sweeps alternated with band-power draws, the power
spectrum inference of §5): samples and band powers draw for draw against the FP64 oracle."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import hierarchical as HG
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu

SAMPLE_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


@pytest.mark.parametrize("H", [16, 32, 64, 128])
def test_band_sampler_draw_for_draw(H):
    p = synth.make_problem(H, seed=H + 9, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    bins, nb = HG.radial_bins(H, H)
    P0 = np.full(nb, 0.5, np.float32)
    n = 4
    xs, Ps = wf.wf_sample_band(*to_dev(p), torch.from_numpy(bins).cuda(), torch.from_numpy(P0).cuda(), seed=8,
                               n_samples=n, n_chains=2, chain_offset=3)
    xs, Ps = xs.cpu().numpy(), Ps.cpu().numpy()
    for c in range(2):
        rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, n, seed=8, chain=3 + c)
        for m in range(n):
            assert rel(xs[c, m], rs[m]) < SAMPLE_TOL, (H, c, m, rel(xs[c, m], rs[m]))
            assert rel(Ps[c, m], rP[m]) < SAMPLE_TOL, (H, c, m, rel(Ps[c, m], rP[m]))


def test_band_sampler_checks_and_fixed_bins():
    p = synth.make_problem(32, seed=3, mask_frac=0.1)
    dev = to_dev(p)
    bins, nb = HG.radial_bins(32, 32)
    P0 = torch.full((nb,), 0.5, device="cuda")
    bad = torch.from_numpy(bins).cuda().clone()
    bad[3, 4] = nb
    with pytest.raises(wf.WFError) as e:
        wf.wf_sample_band(*dev, bad, P0, seed=1, n_samples=1)
    assert e.value.status == 1
    with pytest.raises(wf.WFError):
        wf.wf_sample_band(*dev, torch.from_numpy(bins).cuda(), -P0, seed=1, n_samples=1)
    # every mode fixed (bins = -1, no bands): the plain sampler's draws
    none = torch.full((32, 17), -1, dtype=torch.int32, device="cuda")
    xs, Ps = wf.wf_sample_band(*dev, none, torch.zeros(0, device="cuda"), seed=5, n_samples=3, chain_offset=2)
    ref = wf.wf_sample_ex(*dev, seed=5, n_samples=3, chain_offset=2)
    assert torch.equal(xs, ref) and Ps.shape == (1, 3, 0)
