"""GB300 smoothed-aggregation AMG with classical and material-aware
strength of connection (arXiv 2602.05686): CUDA kernels for sm_103a behind
the C ABI in include/sa.h, with a thin ctypes binding."""
from .api import (EXPORTED, Hierarchy, Options, Problem, SAError, SolveInfo, default_options, lib, lib_path, solve_group,
                  launch_count, profile_enable, profile_read, strength)
from .build import build

__all__ = ["Hierarchy", "SAError", "build", "lib", "lib_path", "default_options", "strength", "solve_group", "Options", "Problem",
           "SolveInfo", "EXPORTED", "profile_enable", "profile_read", "launch_count"]
