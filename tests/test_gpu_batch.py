"""GPU checks of the batched form: every image of a mixed-size batch equals the single-image calls.

Each batch item is a Wiener solve followed by samples of one chain started at the filter; the single-image
references are wf_solve_ex (same options) and wf_sample_ex(init_s = that filter, same seed and chain).
"""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import dense
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
        r = wf.wf_solve_ex(*dev, tol=1e-6)
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
        r = wf.wf_solve_ex(*to_dev(probs[i]), tol=1e-5)
        assert rel(imgs[i].out_wf.cpu().numpy(), r.s.cpu().numpy()) < WF_TOL
