"""Python binding of the C ABI in ``include/wf.h`` (argument marshalling only).

Every function takes CUDA tensors from PyTorch (which owns device memory and streams), checks dtype,
device and shape, and passes raw pointers to ``libwfgpu.so``. All arithmetic runs in the CUDA kernels;
there is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libwfgpu.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "wf.h")

WF_OK = 0
STATUS_NAMES = {0: "WF_OK", 1: "WF_ERR_ARG", 2: "WF_ERR_TAU", 3: "WF_ERR_SHAPE", 4: "WF_ERR_CUDA",
                5: "WF_ERR_NOT_CONVERGED", 6: "WF_ERR_NONFINITE", 7: "WF_ERR_TIMEOUT"}


class WFError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({detail})")


class SolveOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tol", ctypes.c_double), ("eta", ctypes.c_double),
                ("level_tol", ctypes.c_double), ("level_max", ctypes.c_int32), ("check", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("refine", ctypes.c_int32), ("init_s", ctypes.c_void_p),
                ("refine_tol", ctypes.c_double), ("A", ctypes.c_void_p)]


class SampleOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("n_samples", ctypes.c_int64), ("n_chains", ctypes.c_int32),
                ("chain_offset", ctypes.c_uint32), ("start_step", ctypes.c_uint32), ("burn_in", ctypes.c_int32),
                ("thin", ctypes.c_int32), ("init_per_chain", ctypes.c_int32), ("init_s", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("out_dtype", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_void_p), ("Ndiag", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("Pk", ctypes.c_void_p),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("out_wf", ctypes.c_void_p),
                ("out_samples", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("chain", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("resid", ctypes.c_double)]


class LikItem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_void_p), ("sigma2", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("params", ctypes.c_double * 4),
                ("seed", ctypes.c_uint64), ("quad", ctypes.c_double), ("grad_quad", ctypes.c_double * 3),
                ("grad", ctypes.c_double * 3), ("grad_var", ctypes.c_double * 3), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tol", ctypes.c_double), ("eta", ctypes.c_double),
                ("level_tol", ctypes.c_double), ("level_max", ctypes.c_int32), ("check", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("n_samples", ctypes.c_int32), ("large_streams", ctypes.c_int32),
                ("small_grid_pct", ctypes.c_int32), ("large_grid_pct", ctypes.c_int32), ("small_path", ctypes.c_int32),
                ("large_cluster_rows", ctypes.c_int32), ("small_fields_per_cta", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``libwfgpu.so`` (built by ``paper_1810_02821_gb300.build``) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libwfgpu.so not found at {path}: run `python -m paper_1810_02821_gb300.build` "
                           "(the CUDA library is required; there is no CPU fallback)")
    L = ctypes.CDLL(path)
    P, I32, I64, U32, U64, D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_double)
    L.wf_solve.argtypes = [P, P, P, P, I32, I32, D, D, P, ctypes.POINTER(I32), ctypes.POINTER(D), P]
    L.wf_solve_ex.argtypes = [P, P, P, P, I32, I32, ctypes.POINTER(SolveOpts), P, ctypes.POINTER(I32),
                              ctypes.POINTER(D), P]
    L.wf_sample.argtypes = [P, P, P, P, I32, I32, I64, U64, P, P]
    L.wf_sample_ex.argtypes = [P, P, P, P, I32, I32, U64, ctypes.POINTER(SampleOpts), P, P]
    L.wf_sample_band.argtypes = [P, P, P, P, P, I32, P, I32, I32, U64, ctypes.POINTER(SampleOpts), P, P, P]
    L.wf_sample_band.restype = ctypes.c_int
    L.wf_sample_spin2.argtypes = [P, P, P, P, P, P, P, I32, I32, U64, ctypes.POINTER(SampleOpts), P, P]
    L.wf_sample_spin2.restype = ctypes.c_int
    L.wf_solve_spin2.argtypes = [P, P, P, P, P, P, P, I32, I32, ctypes.POINTER(SolveOpts), P,
                                 ctypes.POINTER(I32), ctypes.POINTER(D), P]
    L.wf_solve_spin2.restype = ctypes.c_int
    L.wf_shear_to_convergence.argtypes = [P, I64, I32, I32, P, P]
    L.wf_shear_to_convergence.restype = ctypes.c_int
    for name in ("wf_solve", "wf_solve_ex", "wf_sample", "wf_sample_ex"):
        getattr(L, name).restype = ctypes.c_int
    L.wf_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
    L.wf_solve_opts_default.restype = None
    L.wf_sample_opts_default.argtypes = [ctypes.POINTER(SampleOpts)]
    L.wf_sample_opts_default.restype = None
    L.wf_supported_size.argtypes = [I32, I32]
    L.wf_supported_size.restype = I32
    L.wf_status_string.argtypes = [ctypes.c_int]
    L.wf_status_string.restype = ctypes.c_char_p
    L.wf_last_cuda_error.argtypes = []
    L.wf_last_cuda_error.restype = I32
    L.wf_abi_version.argtypes = []
    L.wf_abi_version.restype = I32
    L.wf_batch_opts_default.argtypes = [ctypes.POINTER(BatchOpts)]
    L.wf_batch_opts_default.restype = None
    L.wf_batch_run.argtypes = [ctypes.POINTER(BatchItem), I32, ctypes.POINTER(BatchOpts), P]
    L.wf_batch_run.restype = ctypes.c_int
    L.wf_batch_graph_create.argtypes = [ctypes.POINTER(BatchItem), I32, ctypes.POINTER(BatchOpts),
                                        ctypes.POINTER(ctypes.c_void_p)]
    L.wf_batch_graph_create.restype = ctypes.c_int
    L.wf_batch_graph_launch.argtypes = [P, P]
    L.wf_batch_graph_launch.restype = ctypes.c_int
    L.wf_batch_graph_results.argtypes = [P, ctypes.POINTER(BatchItem), I32, P]
    L.wf_batch_graph_results.restype = ctypes.c_int
    L.wf_batch_graph_destroy.argtypes = [P]
    L.wf_batch_graph_destroy.restype = None
    L.wf_batch_autotune.argtypes = [ctypes.POINTER(BatchItem), I32, ctypes.POINTER(BatchOpts), I32,
                                    ctypes.POINTER(D), P]
    L.wf_batch_autotune.restype = ctypes.c_int
    L.wf_spectral_power.argtypes = [P, P, ctypes.c_float, I32, P, I32, I32, I32, ctypes.POINTER(D), P]
    L.wf_spectral_power.restype = ctypes.c_int
    L.wf_loglike_grad.argtypes = [P, P, P, I32, I32, ctypes.POINTER(D), I32, U64, D, ctypes.POINTER(D),
                                  ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), P, P]
    L.wf_loglike_grad.restype = ctypes.c_int
    L.wf_loglike_grad_batch.argtypes = [ctypes.POINTER(LikItem), I32, I32, D, P]
    L.wf_loglike_grad_batch.restype = ctypes.c_int
    L.wf_selftest_wait_timeout.argtypes = [I32, ctypes.POINTER(D)]
    L.wf_selftest_wait_timeout.restype = ctypes.c_int
    L.wf_measure_fp32_peak.argtypes = [I32, ctypes.c_int64, ctypes.POINTER(D), ctypes.POINTER(D), P]
    L.wf_measure_fp32_peak.restype = ctypes.c_int
    L.wf_wiener_vjp.argtypes = [P, P, P, I32, I32, ctypes.POINTER(D), P, P, D, ctypes.POINTER(D), P, P]
    L.wf_wiener_vjp.restype = ctypes.c_int
    L.wf_set_large_image_sampler.argtypes = [I32]
    L.wf_set_large_image_sampler.restype = I32
    L.wf_set_kernel_timing.argtypes = [I32]
    L.wf_set_kernel_timing.restype = None
    L.wf_last_kernel_ms.argtypes = []
    L.wf_last_kernel_ms.restype = D
    _lib = L
    return L


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions declared in ``include/wf.h``."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(wf_[a-z0-9_]+)\s*\(", txt)))


def _check(status: int, where: str, ok=(WF_OK,)):
    if status not in ok:
        L = load_library()
        detail = L.wf_status_string(status).decode()
        if status == 4:
            detail += f", cudaError {L.wf_last_cuda_error()}"
        raise WFError(status, where, detail)


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, shape, name, host_ok=False):
    import torch
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or host_ok):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _out(t, dtype, shape, name):
    """A sample output: a CUDA tensor, or a page-locked CPU tensor (pin_memory) that the kernel writes
    directly over the CPU-GPU link (the library refuses page-locked memory it cannot map)."""
    import torch
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned():
            raise TypeError(f"{name} must be a CUDA tensor or a pinned (page-locked) CPU tensor")
        return _dev(t, dtype, shape, name, host_ok=True)
    return _dev(t, dtype, shape, name)


def _inputs(d, Ndiag, mask, Pk):
    import torch
    H, W = d.shape
    return (H, W, _dev(d, torch.float32, (H, W), "d"), _dev(Ndiag, torch.float32, (H, W), "Ndiag"),
            _dev(mask, torch.uint8, (H, W), "mask"), _dev(Pk, torch.float32, (H, W // 2 + 1), "Pk"))


@dataclass
class SolveResult:
    s: object      # torch tensor [H][W]
    iters: int
    resid: float
    status: int


def wf_solve(d, Ndiag, mask, Pk, tau: float = 0.0, tol: float = 1e-6, out=None, stream=None,
             allow_not_converged: bool = False) -> SolveResult:
    """Wiener filter s_W = S (S + N)^-1 d by the cooled messenger iteration (C call ``wf_solve``)."""
    return wf_solve_ex(d, Ndiag, mask, Pk, tau=tau, tol=tol, out=out, stream=stream,
                       allow_not_converged=allow_not_converged)


def wf_solve_ex(d, Ndiag, mask, Pk, *, tau: float = 0.0, tol: float = 1e-6, eta: float = 0.5,
                level_tol: float = 1e-2, level_max: int = 64, check: int = 4, max_iter: int = 20000,
                refine: int = 3, refine_tol: float = 1e-3, init_s=None, A=None, out=None, stream=None,
                allow_not_converged: bool = False) -> SolveResult:
    """All options of the cooled Wiener-filter solve (C call ``wf_solve_ex``).

    ``refine`` > 0 (default 3) is mixed-precision iterative refinement: after the FP32 messenger solve (to
    max(tol, 1e-5)), up to ``refine`` corrections, each an FP32 messenger solve of (S^-1 + N^-1) e = r (to
    relative residual ``refine_tol``) for the residual r = N^-1 (d - s) - S^-1 s evaluated in FP64. The
    returned residual is then the FP64 relative residual ||S r|| / ||S N^-1 d|| of the returned map, and
    ``iters`` counts the sweeps of all solves. ``refine=0``: the plain FP32 iteration to ``tol``, whose
    reported residual is its own estimate from consecutive FP32 iterates.
    ``A``: optional CUDA float32 [H][W] diagonal pixel response of d = A s + n.
    """
    import torch
    L = load_library()
    H, W, pd, pn, pm, pp = _inputs(d, Ndiag, mask, Pk)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=d.device)
    po = _dev(out, torch.float32, (H, W), "out")
    o = SolveOpts()
    L.wf_solve_opts_default(ctypes.byref(o))
    o.tau, o.tol, o.eta, o.level_tol = float(tau), float(tol), float(eta), float(level_tol)
    o.level_max, o.check, o.max_iter = int(level_max), int(check), int(max_iter)
    o.refine, o.refine_tol = int(refine), float(refine_tol)
    o.init_s = _dev(init_s, torch.float32, (H, W), "init_s").value if init_s is not None else None
    o.A = _dev(A, torch.float32, (H, W), "A").value if A is not None else None
    it = ctypes.c_int32(0)
    rs = ctypes.c_double(0.0)
    st = L.wf_solve_ex(pd, pn, pm, pp, H, W, ctypes.byref(o), po, ctypes.byref(it), ctypes.byref(rs),
                       _stream_ptr(stream))
    _check(st, "wf_solve_ex", ok=(WF_OK, 5) if allow_not_converged else (WF_OK,))
    return SolveResult(out, it.value, rs.value, st)


def wf_sample(d, Ndiag, mask, Pk, n_samples: int, seed: int, out=None, stream=None):
    """``n_samples`` posterior draws of one chain from s0 = 0 (C call ``wf_sample``) -> [n][H][W]."""
    import torch
    L = load_library()
    H, W, pd, pn, pm, pp = _inputs(d, Ndiag, mask, Pk)
    if out is None:
        out = torch.empty((n_samples, H, W), dtype=torch.float32, device=d.device)
    po = _out(out, torch.float32, (n_samples, H, W), "out")
    st = L.wf_sample(pd, pn, pm, pp, H, W, int(n_samples), int(seed) & 0xFFFFFFFFFFFFFFFF, po, _stream_ptr(stream))
    _check(st, "wf_sample")
    return out


def wf_sample_ex(d, Ndiag, mask, Pk, seed: int, n_samples: int, *, n_chains: int = 1, chain_offset: int = 0,
                 start_step: int = 0, burn_in: int = 0, thin: int = 1, tau: float = 0.0, init_s=None,
                 A=None, out_dtype: str = "f32", out=None, stream=None):
    """Several chains with burn-in, thinning and resume (C call ``wf_sample_ex``) -> [chains][n][H][W].
    ``A``: optional CUDA float32 [H][W] diagonal pixel response of d = A s + n. ``out_dtype``: "f32", or
    "bf16" / "f16" for samples rounded once from the FP32 chain state. ``out``: a CUDA tensor, or a pinned
    CPU tensor that the kernel fills directly over the CPU-GPU link."""
    import torch
    L = load_library()
    H, W, pd, pn, pm, pp = _inputs(d, Ndiag, mask, Pk)
    codes = {"f32": (0, torch.float32), "bf16": (1, torch.bfloat16), "f16": (2, torch.float16)}
    if out_dtype not in codes:
        raise ValueError(f"out_dtype must be one of {sorted(codes)}")
    code, tdt = codes[out_dtype]
    if out is None:
        out = torch.empty((n_chains, n_samples, H, W), dtype=tdt, device=d.device)
    po = _out(out, tdt, (n_chains, n_samples, H, W), "out")
    o = SampleOpts()
    L.wf_sample_opts_default(ctypes.byref(o))
    o.tau, o.n_samples, o.n_chains = float(tau), int(n_samples), int(n_chains)
    o.chain_offset, o.start_step, o.burn_in, o.thin = int(chain_offset), int(start_step), int(burn_in), int(thin)
    if init_s is not None:
        per_chain = init_s.dim() == 3
        shape = (n_chains, H, W) if per_chain else (H, W)
        o.init_s = _dev(init_s, torch.float32, shape, "init_s").value
        o.init_per_chain = 1 if per_chain else 0
    o.A = _dev(A, torch.float32, (H, W), "A").value if A is not None else None
    o.out_dtype = code
    st = L.wf_sample_ex(pd, pn, pm, pp, H, W, int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o), po,
                        _stream_ptr(stream))
    _check(st, "wf_sample_ex")
    return out


def wf_sample_band(d, Ndiag, mask, Pk, bins, P0, seed: int, n_samples: int, *, n_chains: int = 1,
                   chain_offset: int = 0, start_step: int = 0, burn_in: int = 0, thin: int = 1, tau: float = 0.0,
                   init_s=None, A=None, out_dtype: str = "f32", keep_P: bool = True, stream=None):
    """Hierarchical Gibbs sampler (C call ``wf_sample_band``): samples [chains][n][H][W] and band powers
    [chains][n][n_bins] (None unless ``keep_P``). ``bins``: CUDA int32 [H][W/2+1] (-1: power from Pk);
    ``P0``: CUDA float32 [n_bins] initial band powers; ``A``: optional pixel response [H][W]."""
    import torch
    L = load_library()
    H, W, pd, pn, pm, pp = _inputs(d, Ndiag, mask, Pk)
    n_bins = int(P0.numel())
    pb = _dev(bins, torch.int32, (H, W // 2 + 1), "bins")
    p0 = _dev(P0, torch.float32, (n_bins,), "P0")
    codes = {"f32": (0, torch.float32), "bf16": (1, torch.bfloat16), "f16": (2, torch.float16)}
    code, tdt = codes[out_dtype]
    out = torch.empty((n_chains, n_samples, H, W), dtype=tdt, device=d.device)
    outP = torch.empty((n_chains, n_samples, n_bins), dtype=torch.float32, device=d.device) if keep_P else None
    o = SampleOpts()
    L.wf_sample_opts_default(ctypes.byref(o))
    o.tau, o.n_samples, o.n_chains = float(tau), int(n_samples), int(n_chains)
    o.chain_offset, o.start_step, o.burn_in, o.thin = int(chain_offset), int(start_step), int(burn_in), int(thin)
    if init_s is not None:
        per_chain = init_s.dim() == 3
        o.init_s = _dev(init_s, torch.float32, (n_chains, H, W) if per_chain else (H, W), "init_s").value
        o.init_per_chain = 1 if per_chain else 0
    o.out_dtype = code
    o.A = _dev(A, torch.float32, (H, W), "A").value if A is not None else None
    st = L.wf_sample_band(pd, pn, pm, pp, pb, n_bins, p0, H, W, int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o),
                          ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(outP.data_ptr()) if outP is not None else None, _stream_ptr(stream))
    _check(st, "wf_sample_band")
    return out, outP


def wf_sample_spin2(d1, d2, N1, N2, mask, PE, PB, seed: int, n_samples: int, *, n_chains: int = 1,
                    chain_offset: int = 0, start_step: int = 0, burn_in: int = 0, thin: int = 1, tau: float = 0.0,
                    init=None, A=None, out_dtype: str = "f32", stream=None):
    """Spin-2 (shear) sampler (C call ``wf_sample_spin2``) -> shear samples [chains][n][2][H][W]; ``A``:
    optional pixel response [H][W] of both components."""
    import torch
    L = load_library()
    H, W, pd1, pn1, pm, pe = _inputs(d1, N1, mask, PE)
    pd2 = _dev(d2, torch.float32, (H, W), "d2")
    pn2 = _dev(N2, torch.float32, (H, W), "N2")
    pb = _dev(PB, torch.float32, (H, W // 2 + 1), "PB")
    codes = {"f32": (0, torch.float32), "bf16": (1, torch.bfloat16), "f16": (2, torch.float16)}
    code, tdt = codes[out_dtype]
    out = torch.empty((n_chains, n_samples, 2, H, W), dtype=tdt, device=d1.device)
    o = SampleOpts()
    L.wf_sample_opts_default(ctypes.byref(o))
    o.tau, o.n_samples, o.n_chains = float(tau), int(n_samples), int(n_chains)
    o.chain_offset, o.start_step, o.burn_in, o.thin = int(chain_offset), int(start_step), int(burn_in), int(thin)
    if init is not None:
        per_chain = init.dim() == 4
        o.init_s = _dev(init, torch.float32, (n_chains, 2, H, W) if per_chain else (2, H, W), "init").value
        o.init_per_chain = 1 if per_chain else 0
    o.out_dtype = code
    o.A = _dev(A, torch.float32, (H, W), "A").value if A is not None else None
    st = L.wf_sample_spin2(pd1, pd2, pn1, pn2, pm, pe, pb, H, W, int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o),
                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(st, "wf_sample_spin2")
    return out


def wf_solve_spin2(d1, d2, N1, N2, mask, PE, PB, *, tol: float = 1e-5, tau: float = 0.0, eta: float = 0.5,
                   level_sweeps: int = 64, check: int = 16, max_iter: int = 50000, allow_not_converged: bool = False,
                   A=None, stream=None) -> SolveResult:
    """Wiener filter of a shear pair (C call ``wf_solve_spin2``) -> SolveResult with s = [2][H][W]; ``A``:
    optional pixel response [H][W] of both components."""
    import torch
    L = load_library()
    H, W, pd1, pn1, pm, pe = _inputs(d1, N1, mask, PE)
    pd2 = _dev(d2, torch.float32, (H, W), "d2")
    pn2 = _dev(N2, torch.float32, (H, W), "N2")
    pb = _dev(PB, torch.float32, (H, W // 2 + 1), "PB")
    out = torch.empty((2, H, W), dtype=torch.float32, device=d1.device)
    o = SolveOpts()
    L.wf_solve_opts_default(ctypes.byref(o))
    o.tau, o.tol, o.eta = float(tau), float(tol), float(eta)
    o.level_max, o.check, o.max_iter = int(level_sweeps), int(check), int(max_iter)
    o.A = _dev(A, torch.float32, (H, W), "A").value if A is not None else None
    it = ctypes.c_int32(0)
    rs = ctypes.c_double(0.0)
    st = L.wf_solve_spin2(pd1, pd2, pn1, pn2, pm, pe, pb, H, W, ctypes.byref(o), ctypes.c_void_p(out.data_ptr()),
                          ctypes.byref(it), ctypes.byref(rs), _stream_ptr(stream))
    _check(st, "wf_solve_spin2", ok=(WF_OK, 5) if allow_not_converged else (WF_OK,))
    return SolveResult(out, it.value, rs.value, st)


def wf_shear_to_convergence(gamma, stream=None):
    """(kappa_E, kappa_B) of shear fields [..., 2, H, W] (C call ``wf_shear_to_convergence``)."""
    import torch
    L = load_library()
    H, W = gamma.shape[-2:]
    g = gamma.reshape(-1, 2, H, W)
    _dev(g, torch.float32, tuple(g.shape), "gamma")
    out = torch.empty_like(g)
    st = L.wf_shear_to_convergence(ctypes.c_void_p(g.data_ptr()), int(g.shape[0]), H, W,
                                   ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(st, "wf_shear_to_convergence")
    return out.reshape(gamma.shape)


@dataclass
class BatchImage:
    """One image of a batch: CUDA tensors d, Ndiag [H][W] f32, mask [H][W] u8, Pk [H][W/2+1] f32."""
    d: object
    Ndiag: object
    mask: object
    Pk: object
    seed: int = 0
    chain: int = 0
    out_wf: object = None       # [H][W] f32, allocated if None
    out_samples: object = None  # [n_samples][H][W] f32, allocated if None and n_samples > 0
    status: int = -1
    iters: int = 0
    resid: float = -1.0


def _batch_items(images, n_samples: int):
    import torch
    arr = (BatchItem * len(images))()
    for i, im in enumerate(images):
        H, W, pd, pn, pm, pp = _inputs(im.d, im.Ndiag, im.mask, im.Pk)
        if im.out_wf is None:
            im.out_wf = torch.empty((H, W), dtype=torch.float32, device=im.d.device)
        if n_samples > 0 and im.out_samples is None:
            im.out_samples = torch.empty((n_samples, H, W), dtype=torch.float32, device=im.d.device)
        arr[i].d, arr[i].Ndiag, arr[i].mask, arr[i].Pk = pd.value, pn.value, pm.value, pp.value
        arr[i].H, arr[i].W = H, W
        arr[i].out_wf = _dev(im.out_wf, torch.float32, (H, W), "out_wf").value
        arr[i].out_samples = (_dev(im.out_samples, torch.float32, (n_samples, H, W), "out_samples").value
                              if n_samples > 0 else None)
        arr[i].seed = int(im.seed) & 0xFFFFFFFFFFFFFFFF
        arr[i].chain = int(im.chain)
    return arr


def _batch_opts(n_samples=0, tau=0.0, tol=1e-5, eta=0.5, level_tol=1e-2, level_max=64, check=4, max_iter=20000,
                large_streams=8, small_grid_pct=0, large_grid_pct=0, small_path=0, large_cluster_rows=0,
                small_fields_per_cta=0) -> BatchOpts:
    L = load_library()
    o = BatchOpts()
    L.wf_batch_opts_default(ctypes.byref(o))
    o.tau, o.tol, o.eta, o.level_tol = float(tau), float(tol), float(eta), float(level_tol)
    o.level_max, o.check, o.max_iter, o.n_samples = int(level_max), int(check), int(max_iter), int(n_samples)
    o.large_streams, o.small_grid_pct, o.large_grid_pct = int(large_streams), int(small_grid_pct), int(large_grid_pct)
    o.small_path, o.large_cluster_rows = int(small_path), int(large_cluster_rows)
    o.small_fields_per_cta = int(small_fields_per_cta)
    return o


def _batch_copy_results(images, arr):
    for i, im in enumerate(images):
        im.status, im.iters, im.resid = arr[i].status, arr[i].iters, arr[i].resid


def wf_batch_run(images, *, n_samples: int = 0, stream=None, allow_not_converged: bool = False, **opts):
    """Wiener filter + ``n_samples`` posterior samples for every image (C call ``wf_batch_run``).

    ``opts``: tau, tol, eta, level_tol, level_max, check, max_iter, large_streams, small_grid_pct,
    large_grid_pct, small_path, large_cluster_rows, small_fields_per_cta (as ``wf_batch_opts``). Fills ``out_wf``, ``out_samples``, ``status``, ``iters`` and
    ``resid`` of each ``BatchImage``.
    """
    L = load_library()
    arr = _batch_items(images, n_samples)
    o = _batch_opts(n_samples=n_samples, **opts)
    st = L.wf_batch_run(arr, len(images), ctypes.byref(o), _stream_ptr(stream))
    _batch_copy_results(images, arr)
    _check(st, "wf_batch_run", ok=(WF_OK, 5) if allow_not_converged else (WF_OK,))
    return images


class BatchGraph:
    """The batch recorded once as a CUDA graph (C calls ``wf_batch_graph_*``): ``launch()`` replays it
    asynchronously on a stream, ``results()`` waits and fills each image's status / iters / resid."""

    def __init__(self, images, *, n_samples: int = 0, **opts):
        L = load_library()
        self.images = images
        self._arr = _batch_items(images, n_samples)
        o = _batch_opts(n_samples=n_samples, **opts)
        h = ctypes.c_void_p(None)
        _check(L.wf_batch_graph_create(self._arr, len(images), ctypes.byref(o), ctypes.byref(h)),
               "wf_batch_graph_create")
        self._h = h

    def launch(self, stream=None):
        _check(load_library().wf_batch_graph_launch(self._h, _stream_ptr(stream)), "wf_batch_graph_launch")

    def results(self, stream=None, allow_not_converged: bool = False):
        st = load_library().wf_batch_graph_results(self._h, self._arr, len(self.images), _stream_ptr(stream))
        _batch_copy_results(self.images, self._arr)
        _check(st, "wf_batch_graph_results", ok=(WF_OK, 5) if allow_not_converged else (WF_OK,))
        return self.images

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().wf_batch_graph_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def wf_batch_autotune(images, *, n_samples: int = 0, reps: int = 1, stream=None, **opts):
    """Launch-shape autotuner of the batched form (C call ``wf_batch_autotune``) -> (chosen options dict,
    best replay ms). The images' outputs are overwritten by the trial runs."""
    L = load_library()
    arr = _batch_items(images, n_samples)
    o = _batch_opts(n_samples=n_samples, **opts)
    best = ctypes.c_double(0.0)
    _check(L.wf_batch_autotune(arr, len(images), ctypes.byref(o), int(reps), ctypes.byref(best), _stream_ptr(stream)),
           "wf_batch_autotune")
    return dict(large_streams=o.large_streams, small_grid_pct=o.small_grid_pct,
                large_grid_pct=o.large_grid_pct, small_path=o.small_path,
                large_cluster_rows=o.large_cluster_rows, small_fields_per_cta=o.small_fields_per_cta), best.value


def wf_spectral_power(a, w, b=None, sgn: float = 1.0, stream=None):
    """sum_k w_j(k) |(U v_f)_k|^2 with v = a + sgn*b (C call ``wf_spectral_power``) -> numpy [F][nw].

    a, b: CUDA float32 [F][H][W] (or [H][W]); w: CUDA float32 [nw][H][W/2+1] (or [H][W/2+1]).
    """
    import numpy as np
    import torch
    L = load_library()
    a3 = a if a.dim() == 3 else a.unsqueeze(0)
    w3 = w if w.dim() == 3 else w.unsqueeze(0)
    F, H, W = a3.shape
    nw = w3.shape[0]
    pa = _dev(a3, torch.float32, (F, H, W), "a")
    pb = _dev(b if b.dim() == 3 else b.unsqueeze(0), torch.float32, (F, H, W), "b") if b is not None else None
    pw = _dev(w3, torch.float32, (nw, H, W // 2 + 1), "w")
    out = (ctypes.c_double * (F * nw))()
    st = L.wf_spectral_power(pa, pb, float(sgn), F, pw, nw, H, W, out, _stream_ptr(stream))
    _check(st, "wf_spectral_power")
    return np.array(out[:]).reshape(F, nw)


@dataclass
class LogLikGrad:
    quad: float          # Q = -1/2 d^T C^-1 d
    grad_quad: object    # numpy [3]: dQ/d(amp, slope, alpha)
    grad: object         # numpy [3]: d lnL/d(amp, slope, alpha) (stochastic trace) or None
    grad_var: object     # numpy [3]: variance of the trace estimate or None
    wf: object           # torch [H][W]: Wiener filter of d


def wf_loglike_grad(d, sigma2, mask, amp: float, slope: float, k0: float, alpha: float, *, n_probes: int = 16,
                    seed: int = 0, tol: float = 1e-7, with_trace: bool = True, stream=None) -> LogLikGrad:
    """Log-likelihood quadratic term and gradients w.r.t. (amp, slope, alpha) (C call ``wf_loglike_grad``)."""
    import numpy as np
    import torch
    L = load_library()
    H, W = d.shape
    pd = _dev(d, torch.float32, (H, W), "d")
    ps = _dev(sigma2, torch.float32, (H, W), "sigma2")
    pm = _dev(mask, torch.uint8, (H, W), "mask")
    prm = (ctypes.c_double * 4)(float(amp), float(slope), float(k0), float(alpha))
    q = ctypes.c_double(0.0)
    gq, g, gv = (ctypes.c_double * 3)(), (ctypes.c_double * 3)(), (ctypes.c_double * 3)()
    out = torch.empty((H, W), dtype=torch.float32, device=d.device)
    st = L.wf_loglike_grad(pd, ps, pm, H, W, prm, int(n_probes), int(seed) & 0xFFFFFFFFFFFFFFFF, float(tol),
                           ctypes.byref(q), gq, g if with_trace else None, gv if with_trace else None,
                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(st, "wf_loglike_grad")
    return LogLikGrad(q.value, np.array(gq[:]), np.array(g[:]) if with_trace else None,
                      np.array(gv[:]) if with_trace else None, out)


def wf_loglike_grad_batch(images, *, n_probes: int = 16, tol: float = 1e-7, stream=None):
    """Log-likelihood data terms and gradients of many images (C call ``wf_loglike_grad_batch``).

    ``images``: sequence of (d, sigma2, mask, amp, slope, k0, alpha, seed) with CUDA tensors; returns a
    list of LogLikGrad (``wf`` is None)."""
    import numpy as np
    import torch
    L = load_library()
    arr = (LikItem * len(images))()
    for i, (d, s2, m, amp, slope, k0, alpha, seed) in enumerate(images):
        H, W = d.shape
        arr[i].d = _dev(d, torch.float32, (H, W), "d").value
        arr[i].sigma2 = _dev(s2, torch.float32, (H, W), "sigma2").value
        arr[i].mask = _dev(m, torch.uint8, (H, W), "mask").value
        arr[i].H, arr[i].W = H, W
        arr[i].params[:] = [float(amp), float(slope), float(k0), float(alpha)]
        arr[i].seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    st = L.wf_loglike_grad_batch(arr, len(images), int(n_probes), float(tol), _stream_ptr(stream))
    _check(st, "wf_loglike_grad_batch", ok=(WF_OK, 5))
    return [LogLikGrad(a.quad, np.array(a.grad_quad[:]), np.array(a.grad[:]) if n_probes else None,
                       np.array(a.grad_var[:]) if n_probes else None, None) for a in arr]


def _make_loglik_function():
    import torch

    class WienerLogLik(torch.autograd.Function):
        """theta = (amp, slope, alpha) -> Q = -1/2 d^T C^-1 d (the data term of lnL).

        The backward pass returns the gradient of the full log-likelihood, including the log-determinant
        term through its stochastic trace (Hutchinson probes), so gradient-based inference sees d lnL /
        d theta; the forward value omits the constant and the log-determinant. The forward call computes
        and keeps (checkpoints) the Wiener solution and the gradient, so backward runs no new solve.
        """

        @staticmethod
        def forward(ctx, theta, d, sigma2, mask, k0, n_probes, seed, tol):
            t = theta.detach().double().cpu().numpy()
            r = wf_loglike_grad(d, sigma2, mask, t[0], t[1], k0, t[2], n_probes=n_probes, seed=seed, tol=tol)
            ctx.save_for_backward(torch.as_tensor(r.grad, dtype=theta.dtype, device=theta.device))
            ctx.wf = r.wf
            return torch.as_tensor(r.quad, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad, None, None, None, None, None, None, None

    return WienerLogLik


_WienerLogLik = None


def wiener_loglik(theta, d, sigma2, mask, k0: float, n_probes: int = 16, seed: int = 0, tol: float = 1e-7):
    """Differentiable data term of the Gaussian log-likelihood (see WienerLogLik)."""
    global _WienerLogLik
    if _WienerLogLik is None:
        _WienerLogLik = _make_loglik_function()
    return _WienerLogLik.apply(theta, d, sigma2, mask, k0, n_probes, seed, tol)


def wf_set_kernel_timing(enable: bool) -> None:
    load_library().wf_set_kernel_timing(1 if enable else 0)


def wf_set_large_image_sampler(mode: str) -> str:
    """Path for 256 x 256 and 512 x 512 images on this thread (samplers, Wiener filters, batches): "auto"
    (default: thread-block clusters from 32 chains or batch images at 256^2 and from 8 at 512^2, else the
    global-memory kernels),
    "cluster" (one cluster per chain or image wherever the device can host it) or "global" (fields in
    global memory, cooperative launches). Returns the previous mode."""
    modes = {"auto": 0, "global": 1, "cluster": 2}
    if mode not in modes:
        raise ValueError(f"mode must be one of {sorted(modes)}")
    prev = load_library().wf_set_large_image_sampler(modes[mode])
    return {0: "auto", 1: "global", 2: "cluster"}[prev]


def wf_last_kernel_ms() -> float:
    return float(load_library().wf_last_kernel_ms())


def wf_supported_size(H: int, W: int) -> bool:
    return bool(load_library().wf_supported_size(H, W))


def wf_wiener_vjp(d, sigma2, mask, amp: float, slope: float, k0: float, alpha: float, g=None, *, s_w=None,
                  tol: float = 1e-7, out=None, stream=None):
    """Wiener map s_W(amp, slope, alpha) and, for a cotangent ``g``, g^T ds_W/d(amp, slope, alpha)
    (C call ``wf_wiener_vjp``). ``s_w``: the forward Wiener filter kept from an earlier call (skips that
    solve). Returns (s_W tensor, vjp numpy[3] or None)."""
    import numpy as np
    import torch
    L = load_library()
    H, W = d.shape
    pd = _dev(d, torch.float32, (H, W), "d")
    ps = _dev(sigma2, torch.float32, (H, W), "sigma2")
    pm = _dev(mask, torch.uint8, (H, W), "mask")
    pg = _dev(g, torch.float32, (H, W), "g") if g is not None else None
    pw = _dev(s_w, torch.float32, (H, W), "s_w") if s_w is not None else None
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=d.device)
    po = _dev(out, torch.float32, (H, W), "out")
    prm = (ctypes.c_double * 4)(float(amp), float(slope), float(k0), float(alpha))
    v = (ctypes.c_double * 3)()
    st = L.wf_wiener_vjp(pd, ps, pm, H, W, prm, pg, pw, float(tol), v if g is not None else None, po,
                         _stream_ptr(stream))
    _check(st, "wf_wiener_vjp")
    return out, (np.array(v[:]) if g is not None else None)


def _make_wiener_map_function():
    import torch

    class WienerMap(torch.autograd.Function):
        """theta = (amp, slope, alpha) -> the Wiener filter s_W [H][W] of d (Eq. 2-3) for P = amp (k/k0)^slope
        and N = alpha * sigma2. The forward solve is kept (checkpointed) for the backward pass, which runs
        one adjoint Wiener solve per cotangent (``wf_wiener_vjp``)."""

        @staticmethod
        def forward(ctx, theta, d, sigma2, mask, k0, tol):
            t = theta.detach().double().cpu().numpy()
            s, _ = wf_wiener_vjp(d, sigma2, mask, t[0], t[1], k0, t[2], tol=tol)
            ctx.args = (d, sigma2, mask, k0, tol, t, theta.dtype, theta.device)
            ctx.save_for_backward(s)
            return s

        @staticmethod
        def backward(ctx, g):
            (s,) = ctx.saved_tensors
            d, sigma2, mask, k0, tol, t, dtype, device = ctx.args
            _, v = wf_wiener_vjp(d, sigma2, mask, t[0], t[1], k0, t[2], g.contiguous().float(), s_w=s, tol=tol)
            return torch.as_tensor(v, dtype=dtype, device=device), None, None, None, None, None

    return WienerMap


_WienerMap = None


def wiener_map(theta, d, sigma2, mask, k0: float, tol: float = 1e-7):
    """Differentiable Wiener filter as a function of theta = (amp, slope, alpha) (see WienerMap)."""
    global _WienerMap
    if _WienerMap is None:
        _WienerMap = _make_wiener_map_function()
    return _WienerMap.apply(theta, d, sigma2, mask, k0, tol)


def wf_selftest_wait_timeout(n_blocks: int = 64):
    """Run the bounded-wait self-test (C call ``wf_selftest_wait_timeout``) -> (status, elapsed ms); the
    expected status is 7 (WF_ERR_TIMEOUT)."""
    L = load_library()
    ms = ctypes.c_double(0.0)
    st = L.wf_selftest_wait_timeout(int(n_blocks), ctypes.byref(ms))
    return st, ms.value


def wf_measure_fp32_peak(paired: bool = False, iters: int = 65536, stream=None):
    """Measured FP32 FMA throughput of the current device (C call ``wf_measure_fp32_peak``) ->
    (TFLOP/s, ms) of one launch that fills every SM with independent FMA chains."""
    L = load_library()
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = L.wf_measure_fp32_peak(1 if paired else 0, int(iters), ctypes.byref(tf), ctypes.byref(ms),
                                _stream_ptr(stream))
    _check(st, "wf_measure_fp32_peak")
    return tf.value, ms.value
