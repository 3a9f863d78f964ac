"""Seeded synthetic inputs for the wildfire-temperature retrieval.

This package is shared by the tests, the benchmark and the CPU oracle's
callers. It produces *inputs only*: band tables (wavelengths, solar
irradiance, transmittance per water-vapour bin, endmember reflectances),
per-pixel truth states and standard-normal noise variates from a
counter-based generator. It holds none of the retrieval's arithmetic: it
never evaluates the forward model, a Jacobian, a moment or a solver step.
Turning a truth state into radiance is done by the caller with either the
oracle's forward model (tests) or the library's own forward kernel (bench).
"""
from .scenes import (  # noqa: F401
    N_BANDS_DEFAULT, TGRID_LO, TGRID_HI, band_centres, make_tables, Tables,
    make_config1_truth, make_config2_truth, make_config3_scenes,
    make_config5_fine_truth, make_injection_experiment, Truth, noise_normals,
    splitmix64, counter_u64, counter_uniform, STREAM_NOISE, STREAM_MLP,
    wv_quantise, state_bounds, block_mean_shape,
)
