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


@pytest.mark.parametrize("H", [256, 512])
def test_band_sampler_large_draw_for_draw(H):
    """256^2 and 512^2: one thread-block cluster per chain, band statistics summed across the cluster."""
    p = synth.make_problem(H, seed=H + 9, mask_frac=0.1, block=(10, 60, 20, 90), slope=-2.0, k0=1.0 / 32,
                           sigma2=(0.05, 0.5))
    bins, nb = HG.radial_bins(H, H)
    P0 = np.full(nb, 0.5, np.float32)
    n = 4 if H == 256 else 3
    xs, Ps = wf.wf_sample_band(*to_dev(p), torch.from_numpy(bins).cuda(), torch.from_numpy(P0).cuda(), seed=8,
                               n_samples=n, n_chains=2, chain_offset=3, burn_in=1)
    xs, Ps = xs.cpu().numpy(), Ps.cpu().numpy()
    for c in range(2):
        rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, n, seed=8, chain=3 + c, burn_in=1)
        for m in range(n):
            assert rel(xs[c, m], rs[m]) < SAMPLE_TOL, (H, c, m, rel(xs[c, m], rs[m]))
            assert rel(Ps[c, m], rP[m]) < SAMPLE_TOL, (H, c, m, rel(Ps[c, m], rP[m]))


def test_band_sampler_large_thin_resume_and_fixed_bins():
    """256^2: thinning and a resumed chain (start_step, init_s, the band powers carried over) repeat the
    uninterrupted chain; with every mode fixed (bins = -1) the band sampler is the plain cluster sampler."""
    H = 256
    p = synth.make_problem(H, seed=5, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    bins, nb = HG.radial_bins(H, H)
    bd = torch.from_numpy(bins).cuda()
    P0 = torch.full((nb,), 0.5, device="cuda")
    full, fP = wf.wf_sample_band(*dev, bd, P0, seed=4, n_samples=2, thin=2)
    rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0.cpu().numpy(), 2, seed=4, thin=2)
    for m in range(2):
        assert rel(full[0, m].cpu().numpy(), rs[m]) < SAMPLE_TOL
        assert rel(fP[0, m].cpu().numpy(), rP[m]) < SAMPLE_TOL
    # resume after sweep 2 from (s, P) of the first kept sample
    tail, tP = wf.wf_sample_band(*dev, bd, fP[0, 0].contiguous(), seed=4, n_samples=1, thin=2, start_step=2,
                                 init_s=full[0, 0].contiguous())
    assert rel(tail[0, 0].cpu().numpy(), full[0, 1].cpu().numpy()) < SAMPLE_TOL
    assert rel(tP[0, 0].cpu().numpy(), fP[0, 1].cpu().numpy()) < SAMPLE_TOL
    none = torch.full((H, H // 2 + 1), -1, dtype=torch.int32, device="cuda")
    xs, Ps = wf.wf_sample_band(*dev, none, torch.zeros(0, device="cuda"), seed=5, n_samples=2, n_chains=2)
    prev = wf.wf_set_large_image_sampler("cluster")
    try:
        ref = wf.wf_sample_ex(*dev, seed=5, n_samples=2, n_chains=2)
    finally:
        wf.wf_set_large_image_sampler(prev)
    assert torch.equal(xs, ref) and Ps.shape == (2, 2, 0)
    with pytest.raises(wf.WFError) as e:  # more bins than the 256^2 kernel holds
        wf.wf_sample_band(*dev, bd, torch.full((257,), 0.5, device="cuda"), seed=1, n_samples=1)
    assert e.value.status == 1


def test_band_sampler_large_chains_loop_and_repeat_exactly():
    """256^2 with more chains than clusters can be resident (each cluster runs several chains in turn):
    chains early and late in the loop follow the oracle, and the band sums, taken in a fixed order, make a
    repeated call bit-identical."""
    H, chains = 256, 300
    p = synth.make_problem(H, seed=21, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    bins, nb = HG.radial_bins(H, H)
    bd, P0 = torch.from_numpy(bins).cuda(), torch.full((nb,), 0.5, device="cuda")
    xs, Ps = wf.wf_sample_band(*dev, bd, P0, seed=12, n_samples=1, n_chains=chains, burn_in=1)
    xs2, Ps2 = wf.wf_sample_band(*dev, bd, P0, seed=12, n_samples=1, n_chains=chains, burn_in=1)
    assert torch.equal(xs, xs2) and torch.equal(Ps, Ps2)
    for c in (0, 151, chains - 1):
        rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0.cpu().numpy(), 1, seed=12, chain=c, burn_in=1)
        assert rel(xs[c, 0].cpu().numpy(), rs[0]) < SAMPLE_TOL, (c, rel(xs[c, 0].cpu().numpy(), rs[0]))
        assert rel(Ps[c, 0].cpu().numpy(), rP[0]) < SAMPLE_TOL, c


def test_band_sampler_large_storage_options():
    """512^2: BF16 sample storage is the FP32 chain rounded once (torch's round-to-nearest-even), band powers
    not kept, per-chain initial states; a bin outside [-1, n_bins) is refused before any sweep."""
    H = 512
    p = synth.make_problem(H, seed=31, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    bins, nb = HG.radial_bins(H, H)
    bd, P0 = torch.from_numpy(bins).cuda(), torch.full((nb,), 0.5, device="cuda")
    init = torch.randn((2, H, H), device="cuda")
    f32, Pf = wf.wf_sample_band(*dev, bd, P0, seed=2, n_samples=2, n_chains=2, init_s=init)
    b16, Pn = wf.wf_sample_band(*dev, bd, P0, seed=2, n_samples=2, n_chains=2, init_s=init, out_dtype="bf16",
                                keep_P=False)
    assert Pn is None and torch.equal(b16, f32.to(torch.bfloat16))
    rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0.cpu().numpy(), 2, seed=2, chain=1,
                       init_s=init[1].cpu().numpy())
    assert rel(f32[1, 1].cpu().numpy(), rs[1]) < SAMPLE_TOL and rel(Pf[1, 1].cpu().numpy(), rP[1]) < SAMPLE_TOL
    bad = bd.clone()
    bad[5, 7] = nb
    with pytest.raises(wf.WFError) as e:
        wf.wf_sample_band(*dev, bad, P0, seed=1, n_samples=1)
    assert e.value.status == 1


@pytest.mark.parametrize("H", [32, 128])
def test_band_sampler_repeats_exactly(H):
    """The band sums run in a fixed order at every size: a repeated call is bit-identical (3 chains at 32^2
    leave one field of the last CTA inactive)."""
    p = synth.make_problem(H, seed=H + 3, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    bins, nb = HG.radial_bins(H, H)
    bd, P0 = torch.from_numpy(bins).cuda(), torch.full((nb,), 0.5, device="cuda")
    a = wf.wf_sample_band(*dev, bd, P0, seed=5, n_samples=3, n_chains=3)
    b = wf.wf_sample_band(*dev, bd, P0, seed=5, n_samples=3, n_chains=3)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("H", [64, 256])
def test_band_sampler_empty_band(H):
    """A band with no modes (an extra bin id the map never uses) keeps P_b = 0, and the other bands and the
    samples still follow the oracle."""
    p = synth.make_problem(H, seed=H + 17, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    bins, nb = HG.radial_bins(H, H)
    P0 = np.full(nb + 1, 0.5, np.float32)
    xs, Ps = wf.wf_sample_band(*to_dev(p), torch.from_numpy(bins).cuda(), torch.from_numpy(P0).cuda(), seed=3,
                               n_samples=2)
    rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, 2, seed=3)
    Ps = Ps.cpu().numpy()
    assert np.all(Ps[0, :, nb] == 0.0) and np.all(rP[:, nb] == 0.0)
    for m in range(2):
        assert rel(xs[0, m].cpu().numpy(), rs[m]) < SAMPLE_TOL and rel(Ps[0, m], rP[m]) < SAMPLE_TOL


@pytest.mark.parametrize("H", [64, 256])
def test_band_sampler_with_pixel_response(H):
    """A diagonal pixel response A (with a few A = 0 pixels): samples and band powers follow the oracle's
    general t-update draw for draw."""
    p = synth.make_problem(H, seed=H + 23, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    rng = np.random.default_rng(H)
    A = rng.uniform(0.5, 1.5, (H, H)).astype(np.float32)
    A[rng.integers(0, H, 5), rng.integers(0, H, 5)] = 0.0
    bins, nb = HG.radial_bins(H, H)
    P0 = np.full(nb, 0.5, np.float32)
    xs, Ps = wf.wf_sample_band(*to_dev(p), torch.from_numpy(bins).cuda(), torch.from_numpy(P0).cuda(), seed=6,
                               n_samples=2, A=torch.from_numpy(A).cuda())
    rs, rP = HG.sample(p.d, p.Ndiag, p.mask, p.Pk, bins, P0, 2, seed=6, A=A)
    for m in range(2):
        assert rel(xs[0, m].cpu().numpy(), rs[m]) < SAMPLE_TOL, (H, m, rel(xs[0, m].cpu().numpy(), rs[m]))
        assert rel(Ps[0, m].cpu().numpy(), rP[m]) < SAMPLE_TOL
