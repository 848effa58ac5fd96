"""GB300-native messenger-field Wiener filter and Wiener-posterior sampler (Jeffrey, Heavens & Fortio).

``wf``     — the C-ABI binding (``wf_solve``, ``wf_solve_ex``, ``wf_sample``, ``wf_sample_ex``);
``synth``  — seeded synthetic inputs shaped like the paper's workloads;
``build``  — in-tree nvcc build of ``libwfgpu.so`` for sm_103a.
"""
from . import synth  # noqa: F401
