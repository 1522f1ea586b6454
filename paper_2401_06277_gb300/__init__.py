"""GB300-native Q2-Q1 Stokes solver: FGMRES + monolithic geometric multigrid with additive Vanka.

The compute path is the CUDA library ``_lib/libstokes_vanka.so`` (C ABI in
include/stokes_vanka.h); this package only marshals arguments.
"""
from .stokes import *  # noqa: F401,F403
from .stokes import Batch, Hierarchy, StokesError, library_path, vec_len  # noqa: F401
from .autograd import StokesSolve, stokes_solve  # noqa: F401
