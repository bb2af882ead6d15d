"""Seeded synthetic inputs shaped like the imaging problems of arXiv:2406.08703.

This package generates *inputs* only: aperture transmissions, Zernike basis
images, binary phase gratings, flat fields, source positions and fluxes,
wavelength grids, and Poisson counts drawn from a given expectation image.
It holds none of the method's arithmetic (no phasor, no propagation, no
likelihood); both the FP64 oracle and the CUDA path consume what it returns.
"""

from .generators import (  # noqa: F401
    ARCSEC,
    Problem,
    aperture,
    binary_grating,
    flat_field,
    make_problem,
    noll_to_nm,
    perturbed_start,
    pixel_coords,
    poisson_counts,
    serving_request_shapes,
    smooth_gaussian_noise,
    synthetic_counts,
    zernike_basis,
)
