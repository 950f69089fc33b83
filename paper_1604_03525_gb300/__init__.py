"""GB300 (sm_103a) library for the Wannier-interpolated electron linewidth of EPW.

The compute path is hand-written CUDA behind the C ABI of include/epw.h;
this package only marshals arguments.  Importing it does not load the CUDA
library; the first call does (and fails loudly when it cannot).
"""
from .api import (BF16X3, FP32, FP64, PRECISIONS, TF32X3, Batch, EPWError, Model, eliashberg,  # noqa: F401
                  launch_count, plan_linewidth)
