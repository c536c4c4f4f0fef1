"""GB300-native (sm_103a) isothermal lattice Boltzmann: the CS D2Q9 and FD
WENO-5/SSP-RK3 time-step updates of arXiv:1904.02471 behind a C ABI.

``paper_1904_02471_gb300.lbm`` is the ctypes binding of the library;
``paper_1904_02471_gb300.build`` compiles it in-tree with nvcc.
"""
from .lbm import (Batch, Lattice, LbmError, lbm_fd_max_dt, lbm_fit_decay, lbm_nu,  # noqa: F401
                  lbm_tau_fd_from_lu, lbm_tau_lu_from_fd, lbm_tau_star, lbm_velocity_set, make_spec,
                  spec_from_nu)
