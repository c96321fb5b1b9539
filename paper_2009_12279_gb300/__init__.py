"""GB300-native coupled lattice Boltzmann + Oldroyd-B solver (Kuron et al., arXiv:2009.12279).

The compute path is the CUDA library liblbve.so (C ABI in include/lbve.h); the Python
modules here marshal arguments (lbve), build the library (build), generate seeded
synthetic workloads (workloads) and schedule many solves (serve).
"""
from .lbve import LbveError, Pool, Solver, Solver2D, device_bytes, load, make_params  # noqa: F401
