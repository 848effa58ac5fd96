"""Sample outputs in page-locked host memory: the kernels store each sample straight into a pinned CPU
buffer mapped into the device address space. The host buffer must hold exactly what the same call writes
to device memory (the draws and arithmetic do not depend on where the samples go), for every element type
and for both the on-chip (<= 128) and the global-memory (>= 256) sampler; pageable CPU tensors are
refused by the binding."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import messenger as M
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


@pytest.mark.parametrize("H", [32, 128, 256])
@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_host_output_equals_device_output(H, dt):
    p = synth.make_problem(H, seed=H + 11, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    chains, n = 3, 4
    kw = dict(seed=9, n_samples=n, n_chains=chains, chain_offset=2, burn_in=2, thin=2, out_dtype=dt)
    on_dev = wf.wf_sample_ex(*dev, **kw)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dt]
    host = torch.full((chains, n, H, H), float("nan"), dtype=tdt).pin_memory()
    got = wf.wf_sample_ex(*dev, out=host, **kw)
    assert got is host and not got.is_cuda
    assert torch.equal(host, on_dev.cpu())
    if dt == "f32":  # and the samples are the oracle's (chain word 2 + 1, sweep 2 + 2 (m + 1))
        ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 2 + n * 2, seed=9, chain=3)
        for m in range(n):
            assert rel(host[1, m].numpy(), ref[2 + 2 * m + 1]) < 1e-4


@pytest.mark.parametrize("mode", ["cluster", "global"])
def test_host_output_large_paths(mode):
    """256^2 with the sample stores of the cluster kernel and of the global-memory kernel going to host
    memory."""
    p = synth.make_problem(256, seed=5, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    prev = wf.wf_set_large_image_sampler(mode)
    try:
        kw = dict(seed=3, n_samples=2, n_chains=4, out_dtype="bf16")
        on_dev = wf.wf_sample_ex(*dev, **kw)
        host = torch.zeros((4, 2, 256, 256), dtype=torch.bfloat16).pin_memory()
        wf.wf_sample_ex(*dev, out=host, **kw)
    finally:
        wf.wf_set_large_image_sampler(prev)
    assert torch.equal(host, on_dev.cpu())


def test_host_output_single_chain_call():
    p = synth.make_problem(64, seed=3, mask_frac=0.2, slope=-2.0, k0=1.0 / 16, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    host = torch.zeros((5, 64, 64)).pin_memory()
    wf.wf_sample(*dev, n_samples=5, seed=21, out=host)
    assert torch.equal(host, wf.wf_sample(*dev, n_samples=5, seed=21).cpu())


def test_pageable_host_output_refused():
    p = synth.make_problem(32, seed=4, mask_frac=0.1, slope=-2.0, k0=1.0 / 8, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    with pytest.raises(TypeError):
        wf.wf_sample_ex(*dev, seed=1, n_samples=2, out=torch.zeros((1, 2, 32, 32)))
