"""GB300-native volumetric restricted power diagram with fractional Euler
characteristics and connected components (MATTopo, arXiv 2403.18761).

The computation lives in ``librpd.so`` (CUDA, sm_103a; C-ABI in
``include/rpd.h``).  ``rpd`` is the Python binding.
"""
from .rpd import (rpd_build, rpd_build_batch, rpd_autotune, build_workload, Ctx, Mlp, RpdError, load, header_symbols, rpd_launch_count, rpd_peak_fma, RPD_CELL,
                  RPD_FACE, RPD_EDGE, RPD_VERTEX, RPD_FP64, RPD_FP32_FILTERED)

__all__ = ["rpd_build", "rpd_build_batch", "rpd_autotune", "build_workload", "Ctx", "Mlp", "RpdError", "load", "header_symbols", "rpd_launch_count", "rpd_peak_fma", "RPD_CELL", "RPD_FACE",
           "RPD_EDGE", "RPD_VERTEX", "RPD_FP64", "RPD_FP32_FILTERED"]
