"""Small optical models of the Laplace-approximation tests (oracle pins and GPU
parity): a full-period case whose information matrix has a closed form, and an
aberrated several-source case with dithers, two wavelengths and a flat field."""

import numpy as np

import workloads as W

LAM = 600e-9


def laplace_problem(ni=24, D=0.1, noll=(2, 3, 4, 7, 8), n_src=1, flux=(1e6,), pos=((0.0, 0.0),), lambdas=(LAM,),
                    os=1, n_det=None, pixscale=None, dither=((0.0, 0.0),), coeff=None, obsc=0.1):
    """Hard-edged annular pupil (radius 0.48 D, obstruction obsc D) on a centred grid, so it is
    exactly centrosymmetric; by default the full-period case (one wavelength, oversample 1,
    Nd = Ni, pixel = lambda / D) with no aberration."""
    c = W.pixel_coords(ni, D)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(xx, yy)
    T = ((r <= 0.48 * D) & (r >= obsc * D)).astype(np.float64)
    basis = W.zernike_basis(list(noll), ni, D)
    n_det = ni if n_det is None else n_det
    return W.Problem(name="laplace", n_pupil=ni, diameter=D, n_det=n_det,
                     pixscale=(LAM / D if pixscale is None else pixscale), oversample=os,
                     lambdas=np.array(lambdas, dtype=np.float64), weights=np.ones(len(lambdas)),
                     flux=np.array(flux, dtype=np.float64), pos=np.array(pos, dtype=np.float64).reshape(n_src, 2),
                     dither=np.array(dither, dtype=np.float64), noll=list(noll), basis=basis,
                     coeff=np.zeros(len(noll)) if coeff is None else np.array(coeff, dtype=np.float64),
                     transmission=T, opd_fixed=np.zeros((ni, ni)), opd_pix=None, flat=np.ones((n_det, n_det)))


def aberrated_problem(n_src=3, seed=5):
    rng = np.random.default_rng(seed)
    """n_src stars within 2 lambda/D of the axis, Noll 2, 3, 5, 6 at 30 nm RMS, two wavelengths,
    two exposures (one dithered by a fraction of a pixel), oversample 2, flat N(1, 0.05)."""
    p = laplace_problem(ni=20, D=0.1, noll=(2, 3, 5, 6), n_src=n_src, flux=rng.uniform(2e5, 1e6, n_src),
                        pos=rng.uniform(-2, 2, (n_src, 2)) * LAM / 0.1, lambdas=(560e-9, 640e-9), os=2, n_det=14,
                        pixscale=0.6 * LAM / 0.1, dither=((0.0, 0.0), (0.3 * LAM / 0.1, -0.2 * LAM / 0.1)),
                        coeff=30e-9 * rng.standard_normal(4), obsc=0.15)
    p.flat = 1 + 0.05 * rng.standard_normal((p.n_det, p.n_det))
    return p
