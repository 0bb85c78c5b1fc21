"""GB300 (sm_103a) library for the cascaded central-moment thermal lattice Boltzmann
method of Hajabdollahi & Premnath (arXiv:1710.04751): the fused stream-and-collide
step of a differentially heated cavity, with a C ABI (include/lbm.h) and this thin
Python binding."""
from .lbm import (  # noqa: F401
    ADIABATIC_BOUNCE_BACK, ADIABATIC_SPECULAR, BC_ADIABATIC_BOX, BC_CAVITY, BC_PERIODIC,
    BC_XWALLS, BF16_DEV, D3Q7, D3Q15, EXPORTS, FP16_DEV, FP32, FP64, LBM, LBMError, arena_bytes, default_options,
    derive_params, library_path, load, nusselt_noalloc,
)
from .batch import Batch  # noqa: F401
