"""wf_sample_noalloc: the sampler for callers that cannot allocate device memory at call time.

Such callers (real-time loops that cannot wait on the allocator, host applications whose device memory
is all owned by their own pool or fixed in advance) get the same samples as wf_sample_ex, with the
scratch tables kept in a static device array inside the library. The test calls the entry point through
the C ABI twice in a row (different image sizes, so the second call runs on the first call's leftover
scratch contents) and compares each result with wf_sample_ex within the sampler tolerance of the other
GPU tests.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import need_gpu, rel, to_dev, torch
from paper_1810_02821_gb300 import build, synth, wf

pytestmark = pytest.mark.gpu

SAMPLE_TOL = 1e-4


def _entry():
    L = wf.load_library()
    fn = L.wf_sample_noalloc
    fn.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.POINTER(wf.SampleOpts), ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return L, fn


def _noalloc(p, seed, n_samples, n_chains, out):
    L, fn = _entry()
    d, Nd, mk, Pk = to_dev(p)
    o = wf.SampleOpts()
    L.wf_sample_opts_default(ctypes.byref(o))
    o.n_samples, o.n_chains = n_samples, n_chains
    H, W = p.d.shape
    st = fn(d.data_ptr(), Nd.data_ptr(), mk.data_ptr(), Pk.data_ptr(), H, W, seed, ctypes.byref(o),
            out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, (d, Nd, mk, Pk)


def test_noalloc_matches_allocating_sampler_twice():
    need_gpu()
    build.build()
    cases = [(synth.config_paper128(0), 31, 3, 5), (synth.config_plain32(0), 32, 4, 6)]
    for p, seed, n_samples, n_chains in cases:
        H, W = p.d.shape
        out = torch.full((n_chains, n_samples, H, W), float("nan"), device="cuda")
        st, dev = _noalloc(p, seed, n_samples, n_chains, out)
        assert st == 0, wf.load_library().wf_status_string(st)
        ref = wf.wf_sample_ex(*dev, seed=seed, n_samples=n_samples, n_chains=n_chains)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        for c in range(n_chains):
            for m in range(n_samples):
                assert rel(got[c, m], want[c, m]) < SAMPLE_TOL, (H, c, m)


def test_noalloc_rejects_oversized_and_bad_arguments():
    """Every rejected call is refused before a launch; real device buffers are passed anyway, so a
    reordering of the checks could not send a kernel to a bogus address."""
    need_gpu()
    build.build()
    L, fn = _entry()
    o = wf.SampleOpts()
    L.wf_sample_opts_default(ctypes.byref(o))
    o.n_samples = 1
    big = torch.zeros(256 * 256, device="cuda")
    bm = torch.zeros(256 * 256, dtype=torch.uint8, device="cuda")
    ptr = big.data_ptr()
    # beyond the static scratch
    assert fn(ptr, ptr, bm.data_ptr(), ptr, 256, 256, 0, ctypes.byref(o), ptr, None) == 3
    # a null input
    assert fn(None, ptr, bm.data_ptr(), ptr, 32, 32, 0, ctypes.byref(o), ptr, None) == 1


def test_noalloc_output_in_mapped_host_memory():
    """The output pointer passes the same check as wf_sample_ex's: page-locked host memory that the
    device can address is accepted, and the kernel's stores there equal a device-buffer call."""
    need_gpu()
    build.build()
    p = synth.config_plain32(0)
    host = torch.full((2, 3, 32, 32), float("nan")).pin_memory()
    st, dev = _noalloc(p, 5, 3, 2, host)
    torch.cuda.synchronize()
    assert st == 0, wf.load_library().wf_status_string(st)
    ref = wf.wf_sample_ex(*dev, seed=5, n_samples=3, n_chains=2)
    assert torch.equal(host, ref.cpu())
