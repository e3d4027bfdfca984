"""GB300-native complex-Jacobian gain calibration (Smirnov & Tasse, arXiv:1502.06974).

The compute path is the CUDA library ``libgaincal.so`` (C ABI in include/gaincal.h, sources in
``csrc/``); ``api`` marshals torch tensors into it.  ``synth`` generates seeded synthetic
observations.  There is no CPU fallback: calls fail if the library is missing.
"""
from .api import (Layout, calibrate_dd_alljones, calibrate_dd_cohjones, calibrate_di_jones2x2, calibrate_di_scalar, jhj_jhr_di_jones2x2,
                  jhj_jhr_di_scalar, launch_count, release)

__all__ = ['Layout', 'calibrate_di_scalar', 'calibrate_di_jones2x2', 'calibrate_dd_cohjones', 'calibrate_dd_alljones', 'jhj_jhr_di_scalar',
           'jhj_jhr_di_jones2x2', 'launch_count', 'release']
