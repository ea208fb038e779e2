"""GB300-native monolithic ph-multigrid preconditioner for high-order
Taylor-Hood / Scott-Vogelius Stokes (arXiv 2407.07253), used inside FGMRES.

The computation lives in ``_lib/libstokes_mg.so`` (CUDA for sm_103a plus the
host-side finite-element setup in C++), reached through the C ABI of
``include/stokes_mg.h``; this package only marshals arguments.
"""
from ._binding import (BATCH_3XTF32, BATCH_MAX, BATCH_TF32, FP64, HIER_DIRECT, HIER_EXPLICIT,  # noqa: F401
                       HIER_GRADUAL, HIER_HMG, MIXED, SV, TH, StokesError, StokesMG, default_opts, lib, library_path)
