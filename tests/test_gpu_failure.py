"""Failure detection without a GPU fault: a device-side wait that nothing releases gives up after its
poll limit and returns WF_ERR_TIMEOUT, and the context stays usable for the next call."""
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


def test_unreleased_grid_barrier_times_out_and_the_context_survives():
    status, ms = wf.wf_selftest_wait_timeout(64)
    assert status == 7, status          # WF_ERR_TIMEOUT
    assert 0 < ms < 60000, ms
    p = synth.make_problem(32, seed=2, mask_frac=0.1)
    got = wf.wf_sample_ex(*to_dev(p), seed=3, n_samples=2).cpu().numpy()
    ref = M.sample(p.d, p.Ndiag, p.mask, p.Pk, 2, seed=3)
    assert rel(got[0, 1], ref[1]) < 1e-4
    assert torch.cuda.is_available()
