"""GB300-native solver for the linearised non-isothermal single-phase flow
system with the block preconditioner of Roy, Jonsthovel, Lemon and Wathen
(arXiv 1902.00095).

The compute path is the CUDA library libthermo.so (C-ABI in
include/thermo.h); `thermo` is its ctypes binding.
"""
from .thermo import Solver, AMG, default_opts, load, ThermoError  # noqa: F401
