"""GB300 walker propagation for phaseless finite-temperature AFQMC of the 3D
uniform electron gas (arXiv:2012.12228).

The compute path is the CUDA library ``libftq.so`` (C ABI in
``include/ftq.h``); this package only marshals arguments to it.  There is no
CPU fallback: importing works without a GPU, but creating a ``Propagator``
needs the built library and a CUDA device and raises otherwise.
"""
from .binding import (Batch, FTQ_FP64, FTQ_MIXED, FTQ_MIXED_SIMT, FTQ_MIXED_F64UDT, FTQ_PHASELESS, FTQ_FREE, FTQ_OVERLAP_PAPER,
                      FTQ_OVERLAP_MODIFIED, FTQError, Propagator, load_library, library_path, mu_estimates, tune_mu)

__all__ = ["Batch", "FTQ_FP64", "FTQ_MIXED", "FTQ_MIXED_SIMT", "FTQ_MIXED_F64UDT", "FTQ_PHASELESS", "FTQ_FREE", "FTQ_OVERLAP_PAPER",
           "FTQ_OVERLAP_MODIFIED", "FTQError",
           "Propagator", "load_library", "library_path", "mu_estimates", "tune_mu"]
