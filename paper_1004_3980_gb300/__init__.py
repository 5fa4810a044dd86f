"""GB300 (sm_103a) implementation of the per-patch inference of "Hashing Image
Patches for Zooming" (Das Gupta): LSH hashing, exact nearest-neighbour
selection among the hashed candidates, LLE weights, HR blend and overlap
average, cross-bilateral error back-projection.

The compute path is libzoom.so (hand-written CUDA behind the C ABI of
include/zoom.h); this package only marshals arguments.
"""
from .zoom import (Context, DegradeFunction, Dictionary, Index, ReconstructFunction,  # noqa: F401
                   UpscaleParams, backproject, degrade, degrade_adjoint, dictionary_hr,
                   map_energy_grads, query, reconstruct, reconstruct_adjoint, reconstruct_with,
                   sample_crops, upscale, upscale_batch, batch_release, lsh_draws, sample_positions)
