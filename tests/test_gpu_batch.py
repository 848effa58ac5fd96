"""GPU checks of the batched form: every image of a mixed-size batch equals the single-image calls and
the FP64 oracle.

Each batch item is a Wiener solve followed by samples of one chain started at the filter; the single-image
references are wf_solve_ex (same options, plain FP32 iteration) and wf_sample_ex(init_s = that filter, same
seed and chain); the oracle references are the oracle's Wiener filter (or its FP64 residual of the batch's
map) and the oracle's chain from the batch's filter, draw for draw.
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


def _mixed(sizes, seed0=0):
    probs = []
    for i, H in enumerate(sizes):
        if H >= 256:
            p = synth.make_problem(H, seed=seed0 + i, mask_frac=0.05, slope=-1.0, k0=1.0 / 4, sigma2=(0.5, 1.0))
        else:
            p = synth.make_problem(H, seed=seed0 + i, mask_frac=0.1, slope=-2.0, k0=1.0 / H,
                                   sigma2=(0.05, 0.5), block=(1, H // 4, 2, H // 3))
        probs.append(p)
    return probs


def test_batch_matches_single_image_calls():
    sizes = [64, 16, 128, 32, 64, 128, 256, 32, 16]
    probs = _mixed(sizes)
    n_samples = 6
    imgs = [wf.BatchImage(*to_dev(p), seed=100 + i, chain=7 * i) for i, p in enumerate(probs)]
    wf.wf_batch_run(imgs, n_samples=n_samples, tol=1e-6)
    for i, (p, im) in enumerate(zip(probs, imgs)):
        assert im.status == 0, (i, im.status)
        dev = to_dev(p)
        r = wf.wf_solve_ex(*dev, tol=1e-6, refine=0)
        assert rel(im.out_wf.cpu().numpy(), r.s.cpu().numpy()) < WF_TOL, i
        ref = wf.wf_sample_ex(*dev, seed=100 + i, n_samples=n_samples, chain_offset=7 * i,
                              init_s=im.out_wf.contiguous())
        g, w = im.out_samples.cpu().numpy(), ref[0].cpu().numpy()
        for m in range(n_samples):
            assert rel(g[m], w[m]) < SAMPLE_TOL, (i, m)


def test_batch_wf_against_dense_and_errors():
    probs = [synth.make_problem(16, seed=s, mask_frac=0.15, block=(2, 6, 3, 9)) for s in range(5)]
    imgs = [wf.BatchImage(*to_dev(p)) for p in probs]
    wf.wf_batch_run(imgs, tol=1e-7)
    for p, im in zip(probs, imgs):
        ref = dense.wiener_dense(p.d, p.Ndiag, p.mask, p.Pk)
        assert rel(im.out_wf.cpu().numpy(), ref) < WF_TOL
    # an item with a NaN in an observed pixel fails alone; the others still run
    bad = synth.make_problem(32, seed=3, mask_frac=0.1)
    bad.d[np.argwhere(bad.mask == 0)[0][0], np.argwhere(bad.mask == 0)[0][1]] = np.nan
    good = synth.make_problem(32, seed=4, mask_frac=0.1)
    imgs = [wf.BatchImage(*to_dev(good)), wf.BatchImage(*to_dev(bad))]
    with pytest.raises(wf.WFError) as e:
        wf.wf_batch_run(imgs)
    assert e.value.status == 6 and imgs[0].status == 0 and imgs[1].status == 6


def test_batch_many_small_images():
    probs = _mixed([64] * 200 + [128] * 40, seed0=50)
    imgs = [wf.BatchImage(*to_dev(p), seed=i, chain=i) for i, p in enumerate(probs)]
    wf.wf_batch_run(imgs, n_samples=4, tol=1e-5)
    assert all(im.status == 0 for im in imgs)
    for i in (0, 123, 239):
        r = wf.wf_solve_ex(*to_dev(probs[i]), tol=1e-5, refine=0)
        assert rel(imgs[i].out_wf.cpu().numpy(), r.s.cpu().numpy()) < WF_TOL


def _outputs(imgs):
    return [(im.out_wf.cpu().numpy().copy(), im.out_samples.cpu().numpy().copy()) for im in imgs]


def test_batch_graph_replays_match_the_direct_run_and_follow_input_changes():
    sizes = [64, 128, 256, 32, 512, 64, 16]
    probs = _mixed(sizes, seed0=70)
    n_samples = 3
    ref_imgs = [wf.BatchImage(*to_dev(p), seed=5 + i, chain=i) for i, p in enumerate(probs)]
    wf.wf_batch_run(ref_imgs, n_samples=n_samples, tol=1e-5)
    ref = _outputs(ref_imgs)
    imgs = [wf.BatchImage(*to_dev(p), seed=5 + i, chain=i) for i, p in enumerate(probs)]
    with wf.BatchGraph(imgs, n_samples=n_samples, tol=1e-5) as g:
        for _ in range(2):
            g.launch()
            g.results()
            assert all(im.status == 0 for im in imgs)
            for (rw, rs), (gw, gs) in zip(ref, _outputs(imgs)):
                assert rel(gw, rw) < WF_TOL
                for m in range(n_samples):
                    assert rel(gs[m], rs[m]) < SAMPLE_TOL
        # a replay reads the inputs as they are when it runs: doubling d doubles the Wiener filter
        for im in imgs:
            im.d.mul_(2.0)
        g.launch()
        g.results()
        for (rw, _), im in zip(ref, imgs):
            assert rel(im.out_wf.cpu().numpy(), 2.0 * rw) < WF_TOL


def test_batch_launch_shapes_and_autotune_keep_the_results():
    """Every launch shape the autotuner can choose gives the same outputs: the fused and the phased
    small-image paths, persistent grid sizes, images per sampler CTA, pipeline streams, and 512^2 clusters
    of 16 CTAs of 32 rows or 8 CTAs of 64 rows (clusters forced for the single 512^2 image)."""
    sizes = [64, 128, 256, 256, 32, 512]
    probs = _mixed(sizes, seed0=90)
    prev = wf.wf_set_large_image_sampler("cluster")
    try:
        ref_imgs = [wf.BatchImage(*to_dev(p), seed=i, chain=i) for i, p in enumerate(probs)]
        wf.wf_batch_run(ref_imgs, n_samples=2, tol=1e-5)
        ref = _outputs(ref_imgs)
        imgs = [wf.BatchImage(*to_dev(p), seed=i, chain=i) for i, p in enumerate(probs)]
        for shape in (dict(small_grid_pct=25, large_grid_pct=25, large_streams=2, small_path=1),
                      dict(small_path=1), dict(large_cluster_rows=64), dict(large_cluster_rows=32, large_streams=1),
                      dict(small_fields_per_cta=1), dict(small_fields_per_cta=2), dict(small_fields_per_cta=4)):
            wf.wf_batch_run(imgs, n_samples=2, tol=1e-5, **shape)
            for i, ((rw, rs), (gw, gs)) in enumerate(zip(ref, _outputs(imgs))):
                assert rel(gw, rw) < WF_TOL and rel(gs, rs) < SAMPLE_TOL, (shape, sizes[i])
        chosen, ms = wf.wf_batch_autotune(imgs, n_samples=2, reps=1, tol=1e-5)
    finally:
        wf.wf_set_large_image_sampler(prev)
    assert chosen["large_grid_pct"] in (0, 100, 50, 25, 12) and chosen["large_streams"] in (1, 2, 4, 8, 16)
    assert chosen["small_grid_pct"] in (0, 100, 50, 25) and chosen["small_path"] in (0, 1) and ms > 0
    assert chosen["large_cluster_rows"] in (0, 32, 64) and chosen["small_fields_per_cta"] in (0, 1, 2, 4, 8)
    wf.wf_batch_run(imgs, n_samples=2, tol=1e-5, **chosen)
    for (rw, rs), (gw, gs) in zip(ref, _outputs(imgs)):
        assert rel(gw, rw) < WF_TOL and rel(gs, rs) < SAMPLE_TOL


@pytest.fixture(params=["cluster", "global"])
def large_sampler(request):
    prev = wf.wf_set_large_image_sampler(request.param)
    yield request.param
    wf.wf_set_large_image_sampler(prev)


def test_batch_large_images_in_shared_launches(large_sampler):
    # many images above 128 x 128: every size class runs as chunks of fields of one cooperative launch
    # (solves, and the samples with the global-memory sampler) or the samples come from one cluster per
    # image; the single-image references use the same sampler
    sizes = [256] * 10 + [512] * 3
    probs = _mixed(sizes, seed0=200)
    bad = synth.make_problem(256, seed=7, mask_frac=0.1)
    o = np.argwhere(bad.mask == 0)[0]
    bad.d[o[0], o[1]] = np.inf
    probs.append(bad)
    n_samples = 3
    imgs = [wf.BatchImage(*to_dev(p), seed=300 + i, chain=i) for i, p in enumerate(probs)]
    with pytest.raises(wf.WFError) as e:
        wf.wf_batch_run(imgs, n_samples=n_samples, tol=1e-6, large_streams=2)
    assert e.value.status == 6 and imgs[-1].status == 6
    assert all(im.status == 0 for im in imgs[:-1])
    for i in (0, 7, 10, 12):
        p = probs[i]
        dev = to_dev(p)
        r = wf.wf_solve_ex(*dev, tol=1e-6, refine=0)
        got_wf = imgs[i].out_wf.cpu().numpy()
        assert rel(got_wf, r.s.cpu().numpy()) < WF_TOL, i
        assert imgs[i].iters == r.iters, (i, imgs[i].iters, r.iters)
        ref = wf.wf_sample_ex(*dev, seed=300 + i, n_samples=n_samples, chain_offset=i,
                              init_s=imgs[i].out_wf.contiguous())
        g, w = imgs[i].out_samples.cpu().numpy(), ref[0].cpu().numpy()
        for m in range(n_samples):
            assert rel(g[m], w[m]) < SAMPLE_TOL, (i, m)
        if i not in (0, 10):
            continue
        # one 256^2 and one 512^2 image against the oracle: its converged filter, and its chain from the
        # batch's filter with the same counters
        s_ref, _, rho = M.wf_solve(p.d, p.Ndiag, p.mask, p.Pk, tol=1e-10)
        assert rho < 1e-10
        assert rel(got_wf, s_ref) < WF_TOL, (i, large_sampler, rel(got_wf, s_ref))
        o_s = M.sample(p.d, p.Ndiag, p.mask, p.Pk, n_samples, seed=300 + i, chain=i, init_s=got_wf)
        for m in range(n_samples):
            assert rel(g[m], o_s[m]) < SAMPLE_TOL, (i, m, large_sampler)


def test_batch_large_samples_without_wf_output():
    """Through the C call with out_wf = NULL on the large images: the cluster sampling phase starts from
    the library's own copy of s_W and gives the samples of a run that keeps s_W."""
    sizes = [256, 512, 256]
    probs = _mixed(sizes, seed0=400)
    n_samples = 4
    ref = [wf.BatchImage(*to_dev(p), seed=40 + i, chain=3 + i) for i, p in enumerate(probs)]
    wf.wf_batch_run(ref, n_samples=n_samples, tol=1e-6)
    imgs = [wf.BatchImage(*to_dev(p), seed=40 + i, chain=3 + i) for i, p in enumerate(probs)]
    L = wf.load_library()
    import ctypes
    arr = wf._batch_items(imgs, n_samples)
    for i in range(len(imgs)):
        arr[i].out_wf = None
    o = wf._batch_opts(n_samples=n_samples, tol=1e-6)
    assert L.wf_batch_run(arr, len(imgs), ctypes.byref(o), None) == 0
    torch.cuda.synchronize()
    for i in range(len(imgs)):
        assert arr[i].status == 0
        for m in range(n_samples):
            assert rel(imgs[i].out_samples[m].cpu().numpy(), ref[i].out_samples[m].cpu().numpy()) < 1e-5, (i, m)


def test_full_size_mixed_batch_4096_sampled():
    """The 4096-image mixed batch (solve to 1e-5 plus 64 samples each, one graph replay as timed): the first
    image of each size against the single-image calls and against the oracle. The oracle checks the map
    through its own FP64 residual (the solve's stopping criterion; an exact filter of these harder problems
    at 512^2 takes the FP64 oracle minutes) and the samples draw for draw from the batch's filter."""
    probs = synth.config_batch(4096, seed=0)
    imgs = [wf.BatchImage(*to_dev(p), seed=i, chain=i) for i, p in enumerate(probs)]
    with wf.BatchGraph(imgs, n_samples=64, tol=1e-5) as g:
        g.launch()
        g.results()
    assert all(im.status == 0 for im in imgs)
    sizes = [p.d.shape[0] for p in probs]
    for H in (64, 128, 256, 512):
        i = sizes.index(H)
        p, im = probs[i], imgs[i]
        got_wf = im.out_wf.cpu().numpy()
        r = wf.wf_solve_ex(*to_dev(p), tol=1e-5, refine=0)   # the same cooled solve, one image per call
        assert rel(got_wf, r.s.cpu().numpy()) < WF_TOL
        # the batch's stopping test (FP32 iterates) against the oracle's FP64 residual of the returned map:
        # 1e-5 plus the FP32 floor of the iteration (below 4e-6 at every size measured)
        rho = M.residual(got_wf.astype(np.float64), p.d, p.Ndiag, p.mask, p.Pk)
        assert rho < 1.5e-5, (H, rho, im.resid)
        ref_s = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 3, seed=i, chain=i, init_s=got_wf)
        for m in range(3):
            assert rel(im.out_samples[m].cpu().numpy(), ref_s[m]) < SAMPLE_TOL, (H, m)
