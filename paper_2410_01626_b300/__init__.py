"""B300-native fast multipole Coulomb solver for lambda-dynamics constant pH.

Energy E, forces F and per-site derivatives dV/dlambda of the Coulomb energy
of lambda-interpolated charges (arXiv 2410.01626, Sec. 2.1 Eq. 1 and Sec. 2.6)
in an open or periodic cube, computed by hand-written sm_103a CUDA kernels
behind a C ABI (``include/fmmcph.h``).  PyTorch supplies device memory and
streams only.
"""
from .binding import (FMM, Batch, FmmError, KE_DEFAULT, STAGES, host_operator, host_regular, lambda_bias, lambda_pfc,
                      lambda_step, library_path, load, pinned_empty)
from .autograd import FMMEnergy, FMMEnergy4, fmm_energy, fmm_energy4

load()  # fail loudly at import when the native library is missing

__all__ = ["FMM", "Batch", "lambda_step", "FmmError", "FMMEnergy", "FMMEnergy4", "fmm_energy", "fmm_energy4", "KE_DEFAULT", "STAGES", "host_operator",
           "host_regular", "library_path", "load", "pinned_empty", "lambda_pfc", "lambda_bias"]
