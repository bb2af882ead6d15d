"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element
by element, on seeded inputs -- tiny, ragged (tile edges), a reduced and the
full binary-star workload, and sampled outputs plus exact identities at the
million-parameter calibration size."""

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, compare, fit_problem, gpu_eval, oracle_eval, rel_l2

pytestmark = pytest.mark.gpu

FORMS = ["fp32", "f16x3", "bf16x4", "bf16x3", "bf16x3sa", "tf32x3", "bf16"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2406_08703_gb300 as P

    P.load()


@pytest.fixture(scope="module")
def tiny():
    truth, data, start = fit_problem("tiny")
    return start, data, oracle_eval(start, data)


@pytest.mark.parametrize("form", FORMS)
def test_tiny_workload(tiny, form):
    """64^2 pupil -> 256^2 oversampled grid, one wavelength, one star (the tiny workload)."""
    start, data, ref = tiny
    out = gpu_eval(start, data, form)
    err = compare(out, ref, form)
    print(form, err)


RAGGED = [
    dict(n_pupil=17, n_det=9, oversample=3, n_lambda=2, n_src=2, n_exp=2, dither_px=0.5, obscuration=0.2,
         grating=True, n_zern_max=6, opd_pix_rms=3e-9),
    dict(n_pupil=40, n_det=50, oversample=2, n_lambda=3, n_src=1, n_exp=1, n_zern_max=4),
    dict(n_pupil=136, n_det=35, oversample=4, n_lambda=2, n_src=3, n_exp=1, obscuration=0.2, grating=True,
         n_zern_max=10, opd_pix_rms=5e-9),
]


@pytest.mark.parametrize("case", range(len(RAGGED)))
@pytest.mark.parametrize("form", FORMS)
def test_ragged_shapes(case, form):
    """Sizes that are not multiples of any tile: partial tiles in every dimension."""
    _, data, start = fit_problem("custom", seed=10 + case, **RAGGED[case])
    out = gpu_eval(start, data, form)
    compare(out, oracle_eval(start, data), form)


@pytest.mark.parametrize("form", ["fp32", "bf16x3"])
def test_many_zernike_terms(form):
    """80 Zernike terms (more than the 64 a block of the gradient reduction sums at a time) over a
    37^2 pupil (1369 pixels: a partial last block of 64): every Zernike gradient element."""
    _, data, start = fit_problem("custom", seed=90, n_pupil=37, n_det=20, oversample=2, n_lambda=2, n_src=1,
                                 n_exp=2, dither_px=0.5, n_zern_max=80, obscuration=0.1)
    assert start.n_zern == 80
    compare(gpu_eval(start, data, form), oracle_eval(start, data), form)


def _long_problem(case):
    """512-long contractions (the two-sided MFT of Sec. 3 over a 512^2 pupil) onto a small
    detector, so the oracle checks every output."""
    if case == 0:
        # evaluated at an unaberrated hard-edged pupil and an on-axis star: every phasor sample is the
        # same, so the rounding of the operands and of the accumulation adds up coherently at the PSF
        # peak.  The data come from an aberrated, shifted star of another flux, so that every gradient
        # carries signal (at the data's own truth they are Poisson noise, sums that nearly cancel)
        p = W.make_problem("custom", seed=70, n_pupil=512, n_det=24, oversample=2, zern_rms=0.0)
        p.transmission = W.aperture(512, p.diameter, 0.0, oversample=1)
        truth = p.copy()
        truth.coeff = 20e-9 * np.random.default_rng(71).standard_normal(p.n_zern)
        truth.pos = truth.pos + 0.3 * p.pixscale
        truth.flux = 1.2 * p.flux
        truth.flat = W.flat_field(p.n_det, 0.05, 72)
        return p, W.poisson_counts(oracle.forward(truth), 73)
    truth, data, start = fit_problem("custom", seed=72, n_pupil=512, n_det=32, oversample=2, n_lambda=2, n_src=2,
                                     obscuration=0.2, grating=True, n_zern_max=8, opd_pix_rms=5e-9)
    return start, data


@pytest.mark.parametrize("case", range(2))
@pytest.mark.parametrize("form", FORMS)
def test_long_contractions(case, form):
    """K = 512 in both forward contractions and the adjoint 1^T: model, PSF, loss and every
    gradient element against the oracle."""
    p, data = _long_problem(case)
    err = compare(gpu_eval(p, data, form), oracle_eval(p, data), form)
    print(form, case, err)


@pytest.fixture(scope="module")
def binary_reduced():
    truth, data, start = fit_problem("binary", n_lambda=4)
    return start, data, oracle_eval(start, data)


@pytest.mark.parametrize("form", FORMS)
def test_binary_reduced(binary_reduced, form):
    """Binary-star workload (256^2 pupil, 1024^2 grid, 2 stars) with 4 of its 32 wavelengths."""
    start, data, ref = binary_reduced
    compare(gpu_eval(start, data, form), ref, form)


@pytest.fixture(scope="module")
def binary_full():
    truth, data, start = fit_problem("binary")
    return start, data, oracle_eval(start, data)


@pytest.mark.parametrize("form", ["fp32", "f16x3", "bf16x4", "bf16x3", "bf16x3sa", "tf32x3"])
def test_binary_full_size(binary_full, form):
    """The full binary-star workload: 32 wavelengths x 2 stars = 64 PSFs of 1024^2."""
    start, data, ref = binary_full
    err = compare(gpu_eval(start, data, form, want_psf=False), ref, form)
    print(form, err)


def test_adjoint_chunking_is_bitwise_identical():
    """Per-wavelength recomputation in chunks of 1, 3 or 5 of the 8 PSFs gives identical bits (a
    chunk of all PSFs keeps the field instead: test_kept_field_matches_recomputed_field)."""
    _, data, start = fit_problem("custom", seed=5, **RAGGED[0])
    outs = [gpu_eval(start, data, "fp32", psf_chunk=c, want_psf=False) for c in (1, 3, 5)]
    for o in outs[1:]:
        assert o["loss"] == outs[0]["loss"]
        for k in o["grads"]:
            assert np.array_equal(o["grads"][k], outs[0]["grads"][k]), k


@pytest.mark.parametrize("form", ["bf16x3", "f16x3", "tf32x3", "fp32"])
def test_kept_field_matches_recomputed_field(form):
    """The adjoint from the field stage 2 keeps (the default when the adjoint takes every PSF at
    once; in the FP16 form also the mirror-paired adjoint contractions) against the adjoint that
    recomputes each PSF's field (a PSF chunk of 1; unpaired adjoint contractions): the same loss
    and model, and gradients that differ only by the rounding of the two routes."""
    _, data, start = fit_problem("custom", seed=16, **RAGGED[2])
    kept = gpu_eval(start, data, form, want_psf=False)
    recomputed = gpu_eval(start, data, form, psf_chunk=1, want_psf=False)
    assert kept["loss"] == recomputed["loss"]
    assert np.array_equal(kept["model"], recomputed["model"])
    bound = {"bf16x3": 2e-4, "f16x3": 1e-4, "tf32x3": 1e-4, "fp32": 1e-5}[form]
    for k, v in kept["grads"].items():
        if v is not None and np.any(v):
            assert rel_l2(v, recomputed["grads"][k]) < bound, k


@pytest.mark.parametrize("form", ["bf16x3", "f16x3"])
def test_repeat_is_deterministic(form):
    _, data, start = fit_problem("custom", seed=6, **RAGGED[2])
    a = gpu_eval(start, data, form, want_psf=False)
    b = gpu_eval(start, data, form, want_psf=False)
    assert a["loss"] == b["loss"]
    for k in a["grads"]:
        assert np.array_equal(a["grads"][k], b["grads"][k])


@pytest.fixture(scope="module")
def calib_full():
    """The million-parameter calibration workload at full size, hard-edged pupil so
    the Z2/Z3 identities hold exactly; data from an analytic image."""
    p = W.make_problem("calib")
    p = W.perturbed_start(p, 41)
    p.transmission = W.aperture(p.n_pupil, p.diameter, 0.0, oversample=1)
    p.coeff = 10e-9 * np.random.default_rng(3).standard_normal(p.n_zern)
    data = W.synthetic_counts((p.n_exp, p.n_det, p.n_det), 1e9, np.zeros((1, 2)), 12.0, 44)
    return p, data


@pytest.mark.parametrize("form", ["fp32", "f16x3", "bf16x4", "bf16x3", "bf16x3sa", "tf32x3"])
def test_calib_full_size_sampled(calib_full, form):
    """512^2 pupil, 16 wavelengths x 8 exposures, 2048^2 grid: sampled model pixels
    against direct sums, and identities that hold at any size."""
    p, data = calib_full
    out = gpu_eval(p, data, form, want_psf=False)
    m = out["model"]
    rng = np.random.default_rng(0)
    e_idx = list(rng.integers(0, p.n_exp, 16))
    q_idx = list(rng.integers(0, p.n_det**2, 16))
    e0, q0 = np.unravel_index(np.argmax(m.reshape(p.n_exp, -1)), (p.n_exp, p.n_det**2))
    e_idx.append(int(e0))
    q_idx.append(int(q0))
    ref = oracle.model_at(p, e_idx, q_idx)
    got = m.reshape(p.n_exp, -1)[e_idx, q_idx]
    print(form, "calib sampled model error / peak", float(np.max(np.abs(got - ref)) / ref[-1]))
    assert np.max(np.abs(got - ref)) <= TOL[form]["psf"] * ref[-1]
    g = out["grads"]
    s_m = float(np.sum(m - data))
    assert np.dot(p.flux, g["d_flux"]) == pytest.approx(s_m, rel=1e-4)
    assert np.sum(p.flat * g["d_flat"]) == pytest.approx(s_m, rel=1e-4)
    assert np.all(g["d_opd_pix"][p.transmission == 0] == 0)
    assert p.noll[:2] == [2, 3]
    for ax in (0, 1):
        lhs, rhs = np.sum(g["d_pos"][:, ax]), p.diameter / 4 * g["d_zern"][ax]
        assert abs(lhs - rhs) <= 2e-3 * max(abs(rhs), 1e-30)
    assert out["diag"]["device_error"] == 0


def test_autograd_function_matches_loss_grad():
    import torch

    import paper_2406_08703_gb300 as P

    _, data, start = fit_problem("custom", seed=8, **RAGGED[1])
    plan = P.dlx_make_mft(P.desc_from_problem(start, P.DLX_FP32_SIMT))
    prm = P.params_from_problem(start)
    fixed = {k: prm[k] for k in ("transmission", "opd_fixed", "zern_basis", "weights", "dither")}
    leaves = {k: prm[k].clone().requires_grad_(True) for k in ("zern_coeff", "flat", "flux", "pos")}
    dt = torch.as_tensor(data, device="cuda")
    L = P.psf_loss(plan, dt, fixed, leaves["zern_coeff"], None, leaves["flat"], leaves["flux"], leaves["pos"])
    (2.0 * L).backward()
    loss, grads, _ = P.dlx_loss_grad(plan, prm, dt)
    torch.cuda.synchronize()
    assert L.item() == loss.item()
    for k, gk in (("zern_coeff", "d_zern"), ("flat", "d_flat"), ("flux", "d_flux"), ("pos", "d_pos")):
        assert torch.allclose(leaves[k].grad, 2.0 * grads[gk], rtol=1e-6, atol=0)


def test_adam_matches_numpy():
    import torch

    import paper_2406_08703_gb300 as P

    rng = np.random.default_rng(1)
    n = 10007
    th, m, v = rng.standard_normal(n), np.zeros(n), np.zeros(n)
    T = {k: torch.tensor(a, dtype=torch.float32, device="cuda") for k, a in (("th", th), ("m", m), ("v", v))}
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    for t in range(1, 6):
        g = rng.standard_normal(n)
        P.dlx_adam(T["th"], torch.tensor(g, dtype=torch.float32, device="cuda"), T["m"], T["v"], lr, t)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        th = th - lr * (m / (1 - b1**t)) / (np.sqrt(v / (1 - b2**t)) + eps)
    torch.cuda.synchronize()
    assert rel_l2(T["th"].cpu().numpy(), th) < 1e-6


@pytest.mark.parametrize("os_", [1, 2, 3, 4])
@pytest.mark.parametrize("form", ["fp32", "bf16x3", "bf16x4", "f16x3"])
def test_many_sources_with_prf_prior(form, os_):
    """12 sources (the two-pass binning beyond 8 sources) at every oversample path, 2 dithered
    exposures, and the chi^2 prior on the pixel response (Sec. 4), element by element against the
    oracle."""
    _, data, start = fit_problem("custom", seed=14, n_pupil=48, n_det=24 if os_ < 3 else 14, oversample=os_,
                                 n_lambda=2, n_src=12, n_exp=2, dither_px=0.5, obscuration=0.2, grating=True,
                                 n_zern_max=6)
    start.prf_sigma = 0.1
    start.flat = W.flat_field(start.n_det, 0.1, 15)
    err = compare(gpu_eval(start, data, form, want_psf=False), oracle_eval(start, data), form)
    print(form, err)


@pytest.fixture(scope="module")
def paper_full():
    """The paper's example at full size (Sec. 3-4): 20 stars x 3 wavelengths x 5 dithered images,
    512^2 pupil -> 1024^2 detector, chi^2 prior on the pixel response; data from an analytic image."""
    p = W.perturbed_start(W.make_problem("paper"), 61)
    data = W.synthetic_counts((p.n_exp, p.n_det, p.n_det), 1e8, p.pos / p.pixscale, 3.0, 62)
    return p, data


@pytest.mark.parametrize("form,crop", [("fp32", False), ("bf16x3", False), ("bf16x3", True)])
def test_paper_full_size_sampled(paper_full, form, crop):
    """300 PSFs at 512^2 -> 1024^2 (or, with crop, 60 on a 1064^2 detector and five windows of
    each, as Sec. 3 does): sampled model pixels against direct sums, and the Euler identities of
    the flux and flat-field gradients (the prior's own part taken out)."""
    p, data = paper_full
    out = gpu_eval(p, data, form, want_psf=False, crop=crop)
    if crop:
        assert out["info"].n_psf == 60 and out["info"].n_mft_out == 1064
    m = out["model"]
    rng = np.random.default_rng(1)
    e_idx = list(rng.integers(0, p.n_exp, 12))
    q_idx = list(rng.integers(0, p.n_det**2, 12))
    e0, q0 = np.unravel_index(np.argmax(m.reshape(p.n_exp, -1)), (p.n_exp, p.n_det**2))
    e_idx.append(int(e0))
    q_idx.append(int(q0))
    ref = oracle.model_at(p, e_idx, q_idx)
    got = m.reshape(p.n_exp, -1)[e_idx, q_idx]
    print(form, "paper sampled model error / peak", float(np.max(np.abs(got - ref)) / ref[-1]))
    assert np.max(np.abs(got - ref)) <= TOL[form]["psf"] * ref[-1]
    g = out["grads"]
    s_m = float(np.sum(m - data))
    prior_part = (p.flat - 1.0) / p.prf_sigma**2
    assert np.dot(p.flux, g["d_flux"]) == pytest.approx(s_m, rel=1e-4)
    assert np.sum(p.flat * (g["d_flat"] - prior_part)) == pytest.approx(s_m, rel=1e-4)
    assert out["diag"]["device_error"] == 0


CROP = [
    # the paper's pattern (centre and four diagonal steps), small: 3 stars, 2 wavelengths, os 2
    dict(n_pupil=40, n_det=24, oversample=2, n_lambda=2, n_src=3, n_exp=5, obscuration=0.2, grating=True,
         n_zern_max=6, dither=[(0, 0), (3, 3), (3, -3), (-3, 3), (-3, -3)]),
    # asymmetric steps, odd detector, os 4 (the float4 window loads), one image at the edge of the window
    dict(n_pupil=33, n_det=15, oversample=4, n_lambda=1, n_src=2, n_exp=3, n_zern_max=4,
         dither=[(0, 0), (5, -1), (-2, 4)]),
    # os 3 (the generic binning path), a single undithered image
    dict(n_pupil=24, n_det=10, oversample=3, n_lambda=2, n_src=1, n_exp=1, n_zern_max=3, dither=[(0, 0)]),
    # ten sources (the two-pass binning) with windows, os 4
    dict(n_pupil=32, n_det=12, oversample=4, n_lambda=2, n_src=10, n_exp=3, n_zern_max=4,
         dither=[(0, 0), (2, -1), (-1, 2)]),
]


def _crop_problem(case, seed):
    kw = dict(CROP[case])
    dpx = np.array(kw.pop("dither"), dtype=np.float64)
    truth, data, start = fit_problem("custom", seed=seed, **kw)
    start.dither = dpx * start.pixscale
    truth.dither = start.dither.copy()
    data = W.poisson_counts(oracle.forward(truth), seed)
    return start, data


@pytest.mark.parametrize("case", range(len(CROP)))
@pytest.mark.parametrize("form", ["fp32", "bf16x3", "bf16x4", "f16x3"])
def test_integer_dither_windows(case, form):
    """Integer-pixel dithers as windows of one larger detector (Sec. 3): model, PSF, loss and every
    gradient against the oracle's plain per-exposure model with the same dithers as angles."""
    start, data = _crop_problem(case, 20 + case)
    out = gpu_eval(start, data, form, crop=True)
    assert out["info"].n_mft_out == (start.n_det + 2 * int(round(np.max(np.abs(start.dither)) / start.pixscale))) \
        * start.oversample
    err = compare(out, oracle_eval(start, data), form)
    print(form, case, err)


def test_integer_dither_windows_match_angles_on_the_gpu():
    """The window model and the per-exposure model agree on the GPU itself (FP32 form)."""
    start, data = _crop_problem(0, 30)
    a = gpu_eval(start, data, "fp32", crop=True)
    b = gpu_eval(start, data, "fp32", crop=False)
    peak = np.max(np.abs(b["model"]))
    assert np.max(np.abs(a["model"] - b["model"])) <= 2e-6 * peak
    assert a["loss"] == pytest.approx(b["loss"], rel=1e-6)
    for k in a["grads"]:
        if b["grads"][k] is not None:
            assert rel_l2(a["grads"][k], b["grads"][k]) < 1e-5, k


def _defocused(problem, data_seed, edge_rad, f=1.2):
    """Fresnel regime (Sec. 1) with the detector moved from focus so that the quadratic phase reaches
    about edge_rad at the pupil edge at the shortest wavelength; data from the oracle."""
    R = 0.5 * problem.diameter
    dz = edge_rad * float(np.min(problem.lambdas)) * f * f / (np.pi * R * R)
    problem.focal_length, problem.focal_shift = f, dz
    return W.poisson_counts(oracle.forward(problem), data_seed)


@pytest.mark.parametrize("case", range(2))
@pytest.mark.parametrize("form", FORMS)
def test_fresnel_regime(case, form):
    """The detector out of focus (quadratic phase factors around the transform, Sec. 1): model, PSF,
    loss and every gradient against the oracle's chirp-transform-chirp definition."""
    truth, _, start = fit_problem("custom", seed=40 + case, **RAGGED[case])
    data = _defocused(truth, 41 + case, 3.0)
    start.focal_length, start.focal_shift = truth.focal_length, truth.focal_shift
    err = compare(gpu_eval(start, data, form), oracle_eval(start, data), form)
    print(form, case, err)


@pytest.mark.parametrize("form", ["fp32", "bf16x3"])
def test_fresnel_binary_reduced(form):
    """Binary-star shapes (256^2 pupil, 1024^2 grid, 4 wavelengths) with a strong defocus: about 30
    rad of quadratic phase at the pupil edge, the chirp carried in FP64-reduced tilt tables."""
    truth, _, start = fit_problem("binary", n_lambda=4)
    data = _defocused(truth, 45, 30.0)
    start.focal_length, start.focal_shift = truth.focal_length, truth.focal_shift
    err = compare(gpu_eval(start, data, form, want_psf=False), oracle_eval(start, data), form)
    print(form, err)


def test_fresnel_with_integer_dither_windows():
    """Fresnel regime and integer-dither windows together, against the oracle.  Out of focus a
    pointing offset theta moves the image by theta z / f, so the dithers that move it by whole
    pixels are k pixscale f / z."""
    start, _ = _crop_problem(0, 50)
    k = np.rint(start.dither / start.pixscale)
    _defocused(start, 51, 4.0)
    start.dither = k * start.pixscale * start.focal_length / (start.focal_length + start.focal_shift)
    data = W.poisson_counts(oracle.forward(start), 52)
    err = compare(gpu_eval(start, data, "bf16x3", crop=True), oracle_eval(start, data), "bf16x3")
    print(err)
