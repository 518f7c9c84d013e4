"""GB300-native multilayer Gaussian-graph fast summation and Lanczos eigensolver.

The compute path is the CUDA library libmlfastsum.so (C ABI in
include/ml_fastsum.h); this package holds its sources (csrc/), the build
script (build.py), the thin ctypes binding (_lib.py) and the seeded
synthetic workloads (workloads.py).
"""
from ._lib import (MLError, Plan, ml_fastsum_apply, ml_fastsum_plan, ml_lanczos_eigs, load,  # noqa: F401
                   version)
