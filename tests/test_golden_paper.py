"""Checks of the paper's printed worked-example numbers (tests/golden/paper_setup.txt).

They pin the unit conventions of the inputs (arcsec -> rad, lambda/D, Nyquist
sampling) and the parameter grouping of the gradient (positions, fluxes,
Zernike coefficients, one flat-field value per detector pixel).
"""

import math
import os

import numpy as np

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_setup.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("=", 1))
            vals = [float(x) for x in v.split()]
            out[k] = vals if len(vals) > 1 else vals[0]
    return out


def test_paper_problem_matches_listing():
    g = _golden()
    p = W.make_problem("paper")
    assert np.allclose(p.lambdas * 1e9, g["wavelengths_nm"])
    assert p.diameter == g["diameter_m"] and p.n_det == g["det_npix"]
    assert math.isclose(p.pixscale / W.ARCSEC, g["det_pixsize_arcsec"])
    assert p.noll[0] == g["noll_first"] and len(p.noll) == g["noll_count"]
    # 60 PSFs per image (stars x wavelengths), in each of the 5 images
    assert p.n_src == g["n_stars"] and p.n_src * p.n_lambda == g["n_psf"]
    assert p.n_exp == g["n_images"] and p.n_psf == g["n_psf"] * g["n_images"]
    assert p.n_pupil == g["wavefront_npix_text"]


def test_paper_parameter_count():
    g = _golden()
    p = W.make_problem("paper")
    groups = dict(pos=p.pos.size, flux=p.flux.size, zern=p.coeff.size, flat=p.flat.size)
    assert groups["pos"] == g["n_position_params"]
    assert groups["flux"] == g["n_flux_params"]
    assert groups["zern"] == g["n_aberration_params"]
    assert groups["flat"] == g["n_detector_params"]
    assert p.opd_pix is None  # the paper's run fits no pixel OPD map
    assert sum(groups.values()) == g["n_params_total"]


def test_paper_dither_and_sampling():
    g = _golden()
    p = W.make_problem("paper")
    lam_over_d = p.lambdas[1] / p.diameter
    assert abs(g["dither_px"] * p.pixscale / lam_over_d - g["dither_lambda_over_d"]) < 0.03
    # the dithers are whole pixels of g["dither_px"] along each axis (the first image is undithered)
    steps = p.dither / p.pixscale
    assert np.allclose(steps[0], 0) and np.allclose(np.abs(steps[1:]), g["dither_px"])
    nyq = lam_over_d / 2
    assert abs(nyq / p.pixscale / g["nyquist_factor"] - 1) < 0.03
