"""GB300-native canonical density matrix perturbation theory (sm_103a CUDA + C ABI).

The compute path lives in libcdmpt.so (csrc/); this package holds its build
script and a thin ctypes binding. Importing the package does not load the
library; the first binding call does, and it raises if the library is missing.
"""
from .cdmpt import (  # noqa: F401
    Handle, CdmptError, solve, gemm_f32, gemm_f64, lib, version, default_opts, create,
    set_opts, set_H, solve_raw, polarizability, get_stats, last_error, destroy, EXPORTS,
    LIB_PATH, spectral_bounds, spectral_bounds_noalloc, DensityMatrix, Polarizability, FreeEnergy,
    Batch, split_tf32, gemm_f32_split, gemm_pair, check_bounded_wait, FP64, FP32, MIXED_TF32, MIXED_BF16, GEMM_AUTO, GEMM_SIMT,
    GEMM_TC_TF32,
    GEMM_TC_3XTF32, GEMM_TC_BF16,
)
