"""B300-native JGS2: per-vertex Jacobi sweep with the precomputed, co-rotated,
cubature-sampled overshoot correction (Lan et al., ACM TOG), behind the C ABI of
include/jgs2.h. The compute runs in libjgs2.so (CUDA, sm_103a); this package only
marshals arguments."""
from .jgs2 import (CORR_ASM, CORR_ELEM, CORR_OFF, FP32, FP64, Cloth, JGS2Error, Mesh, StepReport,  # noqa: F401
                   adjoint_opts, alu_peak, lib, precompute_opts, step_opts)
