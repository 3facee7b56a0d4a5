"""GB300-native fast time-domain boundary element method (marching on in time)
for transient electromagnetic scattering off perfect electric conductors.

All computation runs in ``libtdbem.so`` (hand-written CUDA for sm_103a behind
the C ABI of ``include/tdbem.h``); this package only marshals arguments.
Importing it loads the library and fails loudly when it has not been built.
"""
from ._binding import (TDBEM_DIRECT, TDBEM_FAST, TDBEM_P_BF16, TDBEM_P_BF16X3, TDBEM_P_FP32, TDBEM_P_TF32,
                       TDBEM_P_TF32X3,
                       Info, Params, Solver, TdbemError, lib, library_path, march_many)

__all__ = ["Solver", "march_many", "Params", "Info", "TdbemError", "lib", "library_path", "TDBEM_DIRECT", "TDBEM_FAST",
           "TDBEM_P_FP32", "TDBEM_P_TF32", "TDBEM_P_BF16", "TDBEM_P_BF16X3", "TDBEM_P_TF32X3"]
