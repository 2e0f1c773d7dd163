"""GB300-native GridSPT hot path (arXiv:1807.04215): CUDA kernels for sm_103a behind
the C ABI of include/gridspt.h, with a thin ctypes binding (``gridspt``)."""
from . import gridspt  # noqa: F401
from .gridspt import (Plan, bispectrum, c2r, linear_amplitude, make_linear_field, power,  # noqa: F401
                      r2c, run_orders)
