"""Reduced-precision sample storage: the chain runs in FP32 and each kept sample is rounded once to BF16 or
FP16 on the way out. The stored values must equal the FP32 samples rounded to nearest even (checked
bit for bit against torch's conversion) and stay within the format's rounding of the FP64 oracle."""
import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from oracle import messenger as M
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu

# unit roundoff 2^-8 (BF16) and 2^-11 (FP16), relative L2 over a sample, plus the FP32 path's own error
BOUND = {"bf16": 2.0 ** -8 + 1e-4, "f16": 2.0 ** -11 + 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    build.build()
    wf.load_library()


@pytest.mark.parametrize("H", [32, 128, 256])
def test_reduced_precision_samples(H):
    p = synth.make_problem(H, seed=H + 5, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
    dev = to_dev(p)
    n, chains = 3, 2
    f32 = wf.wf_sample_ex(*dev, seed=4, n_samples=n, n_chains=chains, chain_offset=1)
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, n, seed=4, chain=2)
    for name, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        got = wf.wf_sample_ex(*dev, seed=4, n_samples=n, n_chains=chains, chain_offset=1, out_dtype=name)
        assert got.dtype == tdt
        assert torch.equal(got, f32.to(tdt)), name
        for m in range(n):
            e = rel(got[1, m].float().cpu().numpy(), ref[m])
            assert e < BOUND[name], (H, name, m, e)
