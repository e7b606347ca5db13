"""GB300 (sm_103a) implementation of the CVF water model's parallel Metropolis
hot path (arXiv:2505.05919): packed 2D lattice, Philox-driven checkerboard
sweep, N_HB / N_sigma reductions and the FP64 isobaric volume move, and the
paper's own cubic lattice with its layered six-arm passes, behind the C ABI
of ``include/cvf.h``."""
from . import _capi
from ._capi import CvfError, cvf_params, cvf_obs
from .lattice import Lattice, params, params_from_dict
from .batch import Batch, tile_configs
from .lattice3 import Lattice3, params3

__all__ = ["Lattice", "Lattice3", "params3", "Batch", "tile_configs", "params", "params_from_dict", "CvfError",
           "cvf_params", "cvf_obs", "_capi"]
