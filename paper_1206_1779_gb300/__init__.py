"""GB300 (sm_103a) solver for the Landau-gauge ghost-gluon Dyson-Schwinger system
of arXiv:1206.1779: Newton-matrix and residual assembly, device Newton steps and
the gluon Schwinger function, behind the C ABI of include/dse.h."""
from ._binding import (DSE_ERR_ARG, DSE_ERR_CUDA, DSE_ERR_NONFINITE, DSE_ERR_NOT_CONVERGED, DSE_ERR_SINGULAR,
                       DSE_ERR_UNSUPPORTED, DSE_OK, DSE_PEAK_FP32_FMA, DSE_PEAK_FP32X2_FMA, DSE_PEAK_FP64_DMMA,
                       DSE_PEAK_FP64_FMA, DSE_PEAK_MUFU_EX2, DSE_PEAK_MUFU_LG2, EXPORTS, Batch, DseError, Plan, Problem, alu_peak, library_path, load,
                       status_string)
from . import inputs

__all__ = ["Plan", "Batch", "Problem", "DseError", "load", "library_path", "status_string", "inputs", "EXPORTS",
           "DSE_OK", "DSE_ERR_ARG", "DSE_ERR_NONFINITE", "DSE_ERR_SINGULAR", "DSE_ERR_CUDA",
           "DSE_ERR_UNSUPPORTED", "DSE_ERR_NOT_CONVERGED", "alu_peak", "DSE_PEAK_FP64_FMA", "DSE_PEAK_FP32_FMA",
           "DSE_PEAK_MUFU_EX2", "DSE_PEAK_MUFU_LG2", "DSE_PEAK_FP64_DMMA",
           "DSE_PEAK_FP32X2_FMA"]
