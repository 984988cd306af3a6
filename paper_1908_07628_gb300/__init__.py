"""GB300 (sm_103a) STEM-EELS maps with the linear-scaling scattering-matrix method.

Brown, Ciston & Ophus, arXiv 1908.07628.  The computation lives in the CUDA
library libstemeels.so (C ABI in include/stem_eels.h); this package only builds
it and marshals arguments to it.
"""
from ._lib import (Context, EelsError, SMatrix, build_smatrix_for, build_smatrix_static,  # noqa: F401
                   inelastic_map_tiles_for, resumable_map,
                   checked_build, count_beams, fp32_fma_rate,
                   footprint_bytes, inelastic_map_for, load, memory_model,
                   quadratic_reference_map_for, EXPORTS, LIB_PATH, Server, make_request,
                   request_footprint)
