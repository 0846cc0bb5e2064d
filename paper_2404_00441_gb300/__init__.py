"""GB300 (sm_103a) CCWSIM best-match search: thin Python binding of libccw.so.

Every step of the search runs in the library's CUDA kernels; this package only
marshals arguments (PyTorch provides device memory and streams).
"""
from .ccw import (CCWError, TI, Net, ccf_map, ccf_search, idwt_paste, launch_count,  # noqa: F401
                  lattice, library_path, load, philox_dev, philox_host, profile_enable,
                  profile_read, profile_read_phases, profile_read_proposal, set_nn_path, simulate, simulate_groups, LOG_FLAG_DONE,
                  LOG_FLAG_PROPOSAL, LOG_FLAG_UNIFORM)
from . import proposal  # noqa: F401
