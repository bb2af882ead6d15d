"""Pins of the oracle's Fresnel regime (Sec. 1: a detector slightly out of
focus adds quadratic phase factors before and after the transform):

- in focus (focal shift 0) it is the Fraunhofer model, to rounding;
- the chirp-transform-chirp form equals the Fresnel diffraction integral
  written directly in its convolution form, sum_x P(x) exp(-i pi |x|^2 /
  (lambda f)) exp(i pi |r - x|^2 / (lambda z)) (lens, then free propagation
  over z), on a tiny grid by brute force;
- far from focus the image of a point source tends to the geometric shadow
  of the pupil, an annulus of outer radius (D/2) |dz| / f in the detector
  plane, with the obstruction's shadow dark;
- the analytic gradient agrees with central differences of the loss.
"""

import numpy as np
import pytest

import workloads as W


def _fresnel_problem(n_pupil=12, n_det=10, os=1, pos=(0.0, 0.0), f=0.5, dz=2e-3, lam=600e-9, D=0.02, obsc=0.3,
                     pixscale=None):
    c = W.pixel_coords(n_pupil, D)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(xx, yy)
    # an asymmetric pupil (annulus with one quadrant half-transmitting), so the sign of the
    # defocus matters
    T = ((r <= 0.5 * D) & (r >= obsc * 0.5 * D)).astype(np.float64)
    T[(xx > 0) & (yy > 0)] *= 0.5
    ps = 0.5 * lam / D if pixscale is None else pixscale
    return W.Problem(name="fresnel", n_pupil=n_pupil, diameter=D, n_det=n_det, pixscale=ps, oversample=os,
                     lambdas=np.array([lam]), weights=np.ones(1), flux=np.ones(1), pos=np.array([pos]),
                     dither=np.zeros((1, 2)), noll=[], basis=np.zeros((0, n_pupil, n_pupil)), coeff=np.zeros(0),
                     transmission=T, opd_fixed=np.zeros((n_pupil, n_pupil)), opd_pix=None,
                     flat=np.ones((n_det, n_det)), focal_length=f, focal_shift=dz)


def test_in_focus_is_fraunhofer(oracle_lib):
    p = _fresnel_problem(dz=0.0, pos=(3e-6, -2e-6))
    q = p.copy()
    q.focal_length = 0.0
    _, a = oracle_lib.forward(p, with_psf=True)
    _, b = oracle_lib.forward(q, with_psf=True)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(b)


@pytest.mark.parametrize("dz", [2e-3, -1.5e-3])
def test_matches_fresnel_integral_by_brute_force(oracle_lib, dz):
    p = _fresnel_problem(dz=dz, pos=(4e-6, 1e-6), os=2, n_det=7)
    lam, f, z = p.lambdas[0], p.focal_length, p.focal_length + dz
    n, D, no = p.n_pupil, p.diameter, p.n_det * p.oversample
    dx = D / n
    x = W.pixel_coords(n, D)
    pitch = p.pixscale * f / p.oversample  # detector spacing of the output samples
    r = (np.arange(no) - 0.5 * (no - 1)) * pitch
    # the pupil field: normalised transmission with the source tilt
    T = p.transmission / np.sqrt(np.sum(p.transmission**2))
    X, Y = np.meshgrid(x, x, indexing="xy")
    P = T * np.exp(2j * np.pi * (X * p.pos[0, 0] + Y * p.pos[0, 1]) / lam)
    lens = np.exp(-1j * np.pi * (X**2 + Y**2) / (lam * f))
    du = pitch / z  # the model's transform normalisation sqrt(dx du / lambda) per axis
    U = np.zeros((no, no), complex)
    for ky in range(no):
        for kx in range(no):
            kern = np.exp(1j * np.pi * ((r[kx] - X) ** 2 + (r[ky] - Y) ** 2) / (lam * z))
            U[ky, kx] = (dx * du / lam) * np.sum(P * lens * kern)
    _, psf = oracle_lib.forward(p, with_psf=True)
    assert np.max(np.abs(psf[0] - np.abs(U) ** 2)) <= 1e-11 * np.max(np.abs(U) ** 2)


def _shadow(oracle_lib, n_pupil, n_det, dz, pix_per_lod):
    """Energy fraction in the geometric annulus (5% margin) and the obstruction shadow's mean
    (0.2-0.6 of its radius, clear of the central Arago spot) over the annulus' mean."""
    D, f, lam = 0.05, 1.0, 600e-9
    p = _fresnel_problem(n_pupil=n_pupil, n_det=n_det, D=D, f=f, dz=dz, lam=lam, obsc=0.4,
                         pixscale=pix_per_lod * lam / D)
    p.transmission = (p.transmission > 0).astype(np.float64)  # plain annulus here
    _, psf = oracle_lib.forward(p, with_psf=True)
    I = psf[0]
    c = (np.arange(n_det) - 0.5 * (n_det - 1)) * p.pixscale * f
    R = np.hypot(*np.meshgrid(c, c, indexing="xy"))
    r_out = 0.5 * D * dz / f
    r_in = 0.4 * r_out
    ring = (R >= r_in - 0.05 * r_out) & (R <= 1.05 * r_out)
    shadow = (R >= 0.2 * r_in) & (R <= 0.6 * r_in)
    return I[ring].sum() / I.sum(), I[shadow].mean() / I[(R >= r_in) & (R <= r_out)].mean()


def test_far_from_focus_is_the_geometric_shadow(oracle_lib):
    """The shadow sharpens toward geometric optics as the defocus grows (Fresnel number ~20 -> ~50)."""
    ring1, dark1 = _shadow(oracle_lib, 256, 200, 0.02, 0.5)
    ring2, dark2 = _shadow(oracle_lib, 384, 240, 0.05, 1.0)
    assert ring2 >= 0.97 and dark2 <= 0.06
    assert ring2 > ring1 and dark2 < dark1


def test_gradient_central_differences_in_the_fresnel_regime(oracle_lib):
    p = W.make_problem("custom", seed=4, n_pupil=16, n_det=8, oversample=2, n_lambda=2, n_src=2, n_exp=2,
                       dither_px=0.5, flux_total=2e5, obscuration=0.2, grating=True)
    p.noll = [2, 4, 7]
    p.basis = W.zernike_basis(p.noll, p.n_pupil, p.diameter)
    p.coeff = 20e-9 * np.random.default_rng(4).standard_normal(3)
    p.transmission = W.aperture(p.n_pupil, p.diameter, 0.2, oversample=1)
    p.opd_pix = W.smooth_gaussian_noise(p.n_pupil, 5e-9, 1.0, 5)
    p.focal_length, p.focal_shift = 1.5, 3e-4
    d = W.poisson_counts(oracle_lib.forward(p), 6)
    q0 = W.perturbed_start(p, 7)
    g = oracle_lib.loss_grad(q0, d)

    def fd(setter, h):
        a, b = q0.copy(), q0.copy()
        setter(a, h)
        setter(b, -h)
        return (oracle_lib.loss(a, d) - oracle_lib.loss(b, d)) / (2 * h)

    checks = []
    for j in range(3):
        def s(q, h, j=j):
            q.coeff = q.coeff.copy()
            q.coeff[j] += h
        checks.append((g["coeff"][j], fd(s, 5e-12)))
    for iy, ix in ((5, 7), (9, 3), (8, 8)):
        def s(q, h, iy=iy, ix=ix):
            q.opd_pix = q.opd_pix.copy()
            q.opd_pix[iy, ix] += h
        checks.append((g["opd_pix"][iy, ix], fd(s, 2e-11)))
    for si in range(2):
        for ax in range(2):
            def s(q, h, si=si, ax=ax):
                q.pos = q.pos.copy()
                q.pos[si, ax] += h
            checks.append((g["pos"][si, ax], fd(s, 1e-4 * q0.pixscale / q0.oversample)))
        def s(q, h, si=si):
            q.flux = q.flux.copy()
            q.flux[si] += h
        checks.append((g["flux"][si], fd(s, 1e-6 * q0.flux[si])))
    for ana, num in checks:
        assert ana == pytest.approx(num, rel=2e-6, abs=1e-9 * max(1.0, abs(num)))
