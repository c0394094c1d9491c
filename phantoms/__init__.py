"""Seeded synthetic diffusion-MRI inputs shared by the FP64 oracle and the GPU path.

This module only *generates data*: acquisition schemes, ground-truth tissue
maps, noiseless ground-truth signals and Rician noise. It holds none of the
fitting method's arithmetic (no transforms of fit parameters, no loss, no
priors, no gradients, no optimiser). The ground-truth simulator below uses
per-voxel diffusivities and its own code; the fit model's fixed diffusivities
are deliberately different (the paper fits a mismatched model, Sec. 4
"Crossing-Fiber Benchmark").

Every generator is deterministic for a given seed. Random draws come from
numpy's PCG64 so that the same seed gives the same arrays on any machine; only
the deterministic signal evaluation may run on a torch device.

Layouts (the library's input format):
  mask   uint8  [nx, ny, nz]                      (C order)
  signal float32 [V, N]   masked voxels in C order of (x, y, z), N fastest
  bvals  float32 [N]      s/mm^2
  bvecs  float32 [N, 3]   unit vectors (zero rows for b = 0)
"""
from .schemes import (electrostatic_directions, make_scheme, scheme_96, scheme_193, scheme_288,
                      scheme_360)
from .volumes import (BENCH_ANGLES, Volume, crossing_benchmark, crossing_patch, crossing_sweep, bundle_phantom,
                      brain_phantom, multi_volume_batch, random_volume, default_init,
                      n_params)

__all__ = [
    "electrostatic_directions", "make_scheme", "scheme_96", "scheme_193", "scheme_288", "scheme_360",
    "BENCH_ANGLES", "crossing_benchmark", "Volume", "crossing_patch", "crossing_sweep", "bundle_phantom", "brain_phantom",
    "multi_volume_batch", "random_volume", "default_init", "n_params",
]
