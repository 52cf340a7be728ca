"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only draws numbers (phantoms, noise, detector counts, shift sets, PSF taps).
It contains none of the super-resolution arithmetic: no image-formation operator, no
objective, no solver.
"""
from .inputs import (  # noqa: F401
    phantom,
    gaussian_psf,
    half_pixel_shifts,
    third_pixel_shifts,
    phase_shifts,
    gaussian_noise,
    impulse_noise,
    poisson_counts,
    random_field,
    smooth_field,
    batch_rois,
    CONFIG_SEEDS,
)
