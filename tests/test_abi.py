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
    # large-image path selector (per thread): automatic by default, global or cluster on request
    assert wf.wf_set_large_image_sampler("global") == "auto"
    assert wf.wf_set_large_image_sampler("cluster") == "global"
    assert wf.wf_set_large_image_sampler("auto") == "cluster"
    with pytest.raises(ValueError):
        wf.wf_set_large_image_sampler("smem")


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


def test_refine_options_validated_without_gpu(lib):
    o = wf.SolveOpts()
    lib.wf_solve_opts_default(ctypes.byref(o))
    assert o.refine == 3 and o.refine_tol == 1e-3 and not o.init_s
    p = ctypes.c_void_p(16)
    it, rs = ctypes.c_int32(0), ctypes.c_double(0.0)
    for field, value in (("refine", -1), ("refine_tol", 0.0)):
        bad = wf.SolveOpts()
        lib.wf_solve_opts_default(ctypes.byref(bad))
        bad.refine = 2
        setattr(bad, field, value)
        assert lib.wf_solve_ex(p, p, p, p, 32, 32, ctypes.byref(bad), p, ctypes.byref(it), ctypes.byref(rs), None) == 1


def test_option_structs_match_the_header(tmp_path):
    """sizeof/offsetof of the option structs as a C compiler lays them out from include/wf.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"wf_solve_opts": wf.SolveOpts, "wf_sample_opts": wf.SampleOpts,
               "wf_batch_item": wf.BatchItem, "wf_batch_opts": wf.BatchOpts, "wf_lik_item": wf.LikItem}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "wf.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", build.INCLUDE, str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                          text=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_batch_graph_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p(None)
    assert lib.wf_batch_graph_create(None, 0, None, ctypes.byref(h)) == 1 and not h.value
    items = (wf.BatchItem * 1)()
    o = wf.BatchOpts()
    lib.wf_batch_opts_default(ctypes.byref(o))
    assert o.small_grid_pct == 0 and o.large_grid_pct == 0 and o.large_streams >= 1
    o.small_grid_pct = 101
    assert lib.wf_batch_graph_create(items, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    assert lib.wf_batch_run(items, 1, ctypes.byref(o), None) == 1
    assert lib.wf_batch_autotune(items, 1, ctypes.byref(o), 1, None, None) == 1
    assert lib.wf_batch_graph_launch(None, None) == 1
    assert lib.wf_batch_graph_results(None, items, 1, None) == 1
    lib.wf_batch_graph_destroy(None)


def test_noalloc_rejects_a_response_without_gpu(lib):
    p = ctypes.c_void_p(16)
    o = wf.SampleOpts()
    lib.wf_sample_opts_default(ctypes.byref(o))
    assert not o.A
    o.n_samples, o.A = 1, 16
    fn = lib.wf_sample_noalloc
    fn.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.POINTER(wf.SampleOpts), ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    assert fn(p, p, p, p, 32, 32, 0, ctypes.byref(o), p, None) == 1


def test_sample_output_type_validated_without_gpu(lib):
    p = ctypes.c_void_p(16)
    o = wf.SampleOpts()
    lib.wf_sample_opts_default(ctypes.byref(o))
    assert o.out_dtype == 0
    o.n_samples, o.out_dtype = 1, 3
    assert lib.wf_sample_ex(p, p, p, p, 32, 32, 0, ctypes.byref(o), p, None) == 1


def test_selftest_argument_check_without_gpu(lib):
    assert lib.wf_selftest_wait_timeout(0, None) == 1


def test_band_and_spin2_size_and_bin_checks_without_gpu(lib):
    """The hierarchical and spin-2 calls take sizes up to 512 x 512 and at most 256 bands up to 256 x 256
    (512 at 512 x 512); larger requests are refused before any CUDA call."""
    p = ctypes.c_void_p(16)
    o = wf.SampleOpts()
    lib.wf_sample_opts_default(ctypes.byref(o))
    o.n_samples = 1
    band = lib.wf_sample_band
    assert band(p, p, p, p, p, 4, p, 1024, 1024, 0, ctypes.byref(o), p, None, None) == 3
    assert band(p, p, p, p, p, 257, p, 256, 256, 0, ctypes.byref(o), p, None, None) == 1
    assert band(p, p, p, p, p, 513, p, 512, 512, 0, ctypes.byref(o), p, None, None) == 1
    assert band(p, p, p, p, p, 257, p, 128, 128, 0, ctypes.byref(o), p, None, None) == 1
    assert lib.wf_sample_spin2(p, p, p, p, p, p, p, 1024, 1024, 0, ctypes.byref(o), p, None) == 3
    assert lib.wf_solve_spin2(p, p, p, p, p, p, p, 1024, 1024, None, p, None, None, None) == 3
