"""CPU checks of the boundary: the library builds, loads and exports every function of include/wf.h."""
import ctypes
import os

import pytest

from paper_1810_02821_gb300 import build, wf


@pytest.fixture(scope="module")
def lib():
    build.build()
    return wf.load_library()


def test_header_declares_the_documented_calls():
    names = wf.header_functions()
    for n in ["wf_solve", "wf_solve_ex", "wf_sample", "wf_sample_ex", "wf_status_string", "wf_last_cuda_error",
              "wf_supported_size", "wf_solve_opts_default", "wf_sample_opts_default", "wf_abi_version"]:
        assert n in names


def test_library_exports_every_header_symbol(lib):
    for name in wf.header_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    assert lib.wf_abi_version() >> 16 == 1
    for n in (16, 32, 64, 128):
        assert lib.wf_supported_size(n, n) == 1
    assert lib.wf_supported_size(128, 64) == 0 and lib.wf_supported_size(48, 48) == 0
    for s in range(8):
        assert lib.wf_status_string(s)
    o = wf.SolveOpts()
    lib.wf_solve_opts_default(ctypes.byref(o))
    assert o.tol == 1e-6 and o.eta == 0.5 and o.check == 4 and o.max_iter > 0
    so = wf.SampleOpts()
    lib.wf_sample_opts_default(ctypes.byref(so))
    assert so.n_chains == 1 and so.thin == 1 and so.burn_in == 0


def test_argument_errors_need_no_gpu(lib):
    # null pointers and bad shapes are rejected before any CUDA call
    assert lib.wf_sample(None, None, None, None, 32, 32, 1, 0, None, None) == 1
    assert lib.wf_solve(None, None, None, None, 32, 32, 0.0, 1e-6, None, None, None, None) == 1
    p = ctypes.c_void_p(16)
    assert lib.wf_sample(p, p, p, p, 48, 48, 1, 0, p, None) == 3
    assert lib.wf_solve(p, p, p, p, 64, 32, 0.0, 1e-6, p, None, None, None) == 3
    o = wf.SampleOpts()
    lib.wf_sample_opts_default(ctypes.byref(o))
    o.n_samples, o.thin = 1, 0
    assert lib.wf_sample_ex(p, p, p, p, 32, 32, 0, ctypes.byref(o), p, None) == 1


def test_product_path_has_no_oracle_import():
    import paper_1810_02821_gb300 as pkg
    root = os.path.dirname(pkg.__file__)
    for dirpath, _, files in os.walk(root):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
