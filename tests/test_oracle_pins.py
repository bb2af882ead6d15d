"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form (Airy pattern), a library routine (numpy's FFT, scipy's Bessel
functions), brute force, an exact invariance of the Fraunhofer transform
(shift theorem, centrosymmetry, twin image, Parseval), or central finite
differences of the oracle's own loss for its analytic gradient.  The cases
are chosen so that a dropped term, a flipped sign, a transposed operand or a
wrong normalisation in the oracle fails at least one of them.
"""

import math

import numpy as np
import pytest

import workloads as W

LAM = 595e-9


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- MFT pins

def test_separable_mft_equals_fourfold_sum(oracle_lib):
    """The separable two-product MFT equals the direct 4-fold DFT sum (Sec. 3)."""
    rng = np.random.default_rng(0)
    for ni, no in ((7, 9), (6, 11), (5, 4)):
        P = _rand_c(rng, (ni, ni))
        dx, du = 0.125 / ni, 1.3e-6
        E1 = oracle_lib.mft(P, dx, no, du, LAM)
        E2 = oracle_lib.mft_direct(P, dx, no, du, LAM)
        assert np.max(np.abs(E1 - E2)) <= 1e-13 * np.max(np.abs(E2))


def test_mft_equals_zero_padded_fft(oracle_lib):
    """With odd sizes and du = lambda/(No dx) the MFT is the centred, zero-padded DFT."""
    rng = np.random.default_rng(1)
    for ni, no in ((15, 33), (9, 9), (21, 45)):
        dx = 0.125 / ni
        du = LAM / (no * dx)
        P = _rand_c(rng, (ni, ni))
        pad = np.zeros((no, no), complex)
        o = (no - ni) // 2
        pad[o:o + ni, o:o + ni] = P
        ref = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(pad))) / no
        E = oracle_lib.mft(P, dx, no, du, LAM)
        assert np.max(np.abs(E - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_mft_matrix_is_isometry_at_fft_sampling(oracle_lib):
    """A^H A = I when No dx du / lambda = 1 (energy conservation of the normalisation)."""
    for ni, no in ((8, 16), (13, 13), (10, 37)):
        dx = 0.125 / ni
        A = oracle_lib.mft_matrix(no, ni, dx, LAM / (no * dx), LAM)
        assert np.allclose(A.conj().T @ A, np.eye(ni), atol=1e-12)


def test_mft_matrix_mirror_symmetry_and_half_axis_contraction(oracle_lib):
    """On the centred grids (x_{Ni-1-n} = -x_n, u_{No-1-k} = -u_k) the oracle's matrix satisfies
    A[k][Ni-1-n] = conj(A[k][n]) and A[No-1-k][n] = conj(A[k][n]); hence a contraction over the
    pupil axis equals one over half of it, sum_j Re(A) (v_j + v_m) + i Im(A) (v_j - v_m), m = Ni-1-j,
    the middle sample of an odd axis counted once -- the identity the mirror-paired contractions of
    the FP16 form rely on.  A grid centred one sample off fails the first two checks."""
    rng = np.random.default_rng(11)
    for ni, no in ((8, 12), (9, 7), (17, 33)):
        A = oracle_lib.mft_matrix(no, ni, 0.125 / ni, 1.3e-6, LAM)
        assert np.allclose(A[:, ::-1], A.conj(), rtol=0, atol=1e-14 * np.abs(A).max())
        assert np.allclose(A[::-1, :], A.conj(), rtol=0, atol=1e-14 * np.abs(A).max())
        v = _rand_c(rng, ni)
        hn = (ni + 1) // 2
        j = np.arange(hn)
        vm = np.where(ni - 1 - j != j, v[ni - 1 - j], 0.0)
        S, D = v[j] + vm, v[j] - vm
        half = A[:, :hn].real @ S + 1j * (A[:, :hn].imag @ D)
        assert np.max(np.abs(half - A @ v)) <= 1e-13 * np.max(np.abs(A @ v))


def test_parseval(oracle_lib):
    """Unit-power pupil -> unit total intensity at FFT sampling; less on a smaller field."""
    ni = 32
    D = 0.125
    T = W.aperture(ni, D, 0.2)
    rng = np.random.default_rng(2)
    P = T * np.exp(1j * rng.standard_normal((ni, ni)))
    P /= np.sqrt(np.sum(np.abs(P) ** 2))
    dx = D / ni
    for no in (32, 48, 64):
        E = oracle_lib.mft(P, dx, no, LAM / (no * dx), LAM)
        assert abs(np.sum(np.abs(E) ** 2) - 1.0) < 1e-12
    E = oracle_lib.mft(P, dx, 16, LAM / (64 * dx), LAM)
    assert np.sum(np.abs(E) ** 2) < 1.0


def test_adjoint_dot_product(oracle_lib):
    """<M P, G> = <P, M^H G> for the MFT M and its adjoint (complex inner product)."""
    rng = np.random.default_rng(3)
    for ni, no in ((8, 12), (16, 7)):
        P, G = _rand_c(rng, (ni, ni)), _rand_c(rng, (no, no))
        dx, du = 0.1 / ni, 2.1e-6
        lhs = np.vdot(oracle_lib.mft(P, dx, no, du, LAM), G)
        rhs = np.vdot(P, oracle_lib.mft_adjoint(G, ni, dx, du, LAM))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- physics pins

@pytest.fixture(scope="module")
def airy_cut(oracle_lib):
    ni, D = 256, 0.125
    T = W.aperture(ni, D, 0.0)
    P = T / np.sqrt(np.sum(T**2))
    no = 401
    du = 1.4 * LAM / D / 200
    E = oracle_lib.mft(P, D / ni, no, du, LAM)
    return dict(I=np.abs(E) ** 2, du=du, D=D, no=no, T=T, dx=D / ni)


def test_airy_profile(airy_cut):
    """Unobstructed circular pupil: I(theta)/I(0) = [2 J1(v)/v]^2, v = pi D theta / lambda."""
    from scipy.special import j1

    I, du, D, no = airy_cut["I"], airy_cut["du"], airy_cut["D"], airy_cut["no"]
    c = no // 2
    row = I[c, c:]
    theta = np.arange(row.size) * du
    v = np.pi * D * theta / LAM
    with np.errstate(invalid="ignore", divide="ignore"):
        airy = np.where(v > 0, (2 * j1(v) / v) ** 2, 1.0)
    assert np.max(np.abs(row / row[0] - airy)) < 2e-3
    # peak: I(0) = (du/lambda)^2 pi D^2/4 up to pupil pixelisation
    peak = (du / LAM) ** 2 * math.pi * D**2 / 4
    assert abs(row[0] / peak - 1) < 5e-3


def test_airy_first_zero_and_encircled_energy(airy_cut):
    """First dark ring at 1.21967 lambda/D; energy inside it 1 - J0(3.8317)^2 = 0.8378."""
    from scipy.special import j0, jn_zeros

    I, du, D, no = airy_cut["I"], airy_cut["du"], airy_cut["D"], airy_cut["no"]
    c = no // 2
    z1 = jn_zeros(1, 1)[0] / math.pi  # 1.21967 lambda/D
    theta = np.arange(no - c) * du / (LAM / D)
    row = I[c, c:]
    win = (theta > 1.1) & (theta < 1.35)
    tmin = theta[win][np.argmin(row[win])]
    assert abs(tmin - z1) < 0.01
    k = (np.arange(no) - c) * du
    rr = np.hypot(*np.meshgrid(k, k)) / (LAM / D)
    ee = I[rr < z1].sum()
    assert abs(ee - (1 - j0(jn_zeros(1, 1)[0]) ** 2)) < 3e-3


def test_shift_theorem(oracle_lib):
    """A source moved by m oversampled pixels moves the PSF array by m exactly."""
    p = W.make_problem("custom", n_pupil=24, n_det=12, oversample=3)
    du = p.pixscale / p.oversample
    E0 = oracle_lib.psf_field(p, 0, 0, 0)
    for mx, my in ((3, 0), (0, -2), (2, 5)):
        q = p.copy()
        q.pos = np.array([[mx * du, my * du]])
        E1 = oracle_lib.psf_field(q, 0, 0, 0)
        no = p.n_out
        ys, xs = slice(max(my, 0), no + min(my, 0)), slice(max(mx, 0), no + min(mx, 0))
        ys0, xs0 = slice(max(-my, 0), no + min(-my, 0)), slice(max(-mx, 0), no + min(-mx, 0))
        assert np.max(np.abs(E1[ys, xs] - E0[ys0, xs0])) <= 1e-12 * np.max(np.abs(E0))


def test_z2_z3_equal_tilt(oracle_lib):
    """Noll Z2 = 4x/D (Z3 = 4y/D): coefficient c gives the field of a source at 4c/D."""
    base = W.make_problem("custom", n_pupil=32, n_det=16, oversample=2)
    # hard-edged support so every transmitting pixel lies inside the Zernike unit disk
    base.transmission = W.aperture(32, base.diameter, 0.0, oversample=1)
    for j, axis in ((2, 0), (3, 1)):
        c = 37e-9
        p = base.copy()
        p.noll = [j]
        p.basis = W.zernike_basis([j], p.n_pupil, p.diameter)
        p.coeff = np.array([c])
        q = base.copy()
        q.noll, q.basis, q.coeff = [], np.zeros((0, 32, 32)), np.zeros(0)
        q.pos = np.zeros((1, 2))
        q.pos[0, axis] = 4 * c / p.diameter
        Ep, Eq = oracle_lib.psf_field(p, 0, 0, 0), oracle_lib.psf_field(q, 0, 0, 0)
        assert np.max(np.abs(Ep - Eq)) <= 1e-10 * np.max(np.abs(Eq))


def test_centrosymmetry_of_zero_phase_psf(oracle_lib):
    """Any real pupil field (even an asymmetric one) gives I[k] = I[-k] (Hermitian symmetry)."""
    rng = np.random.default_rng(4)
    ni = 20
    T = W.aperture(ni, 0.1) * (1 + 0.5 * rng.random((ni, ni)))
    T[:, : ni // 3] *= 0.2  # asymmetric support
    for no in (17, 24):
        E = oracle_lib.mft(T, 0.1 / ni, no, 1.7e-6, LAM)
        I = np.abs(E) ** 2
        assert np.max(np.abs(I - I[::-1, ::-1])) <= 1e-12 * I.max()
        assert np.max(np.abs(I - I[::-1, :])) > 1e-6 * I.max()  # not mirror-symmetric


def test_twin_image_ambiguity(oracle_lib):
    """P(x) -> conj(P(-x)) leaves the intensity unchanged (sign ambiguity, Sec. 3)."""
    rng = np.random.default_rng(5)
    ni, no = 18, 21
    P = W.aperture(ni, 0.1) * np.exp(1j * rng.standard_normal((ni, ni)))
    P2 = np.conj(P[::-1, ::-1])
    I1 = np.abs(oracle_lib.mft(P, 0.1 / ni, no, 1.5e-6, LAM)) ** 2
    I2 = np.abs(oracle_lib.mft(P2, 0.1 / ni, no, 1.5e-6, LAM)) ** 2
    assert np.max(np.abs(I1 - I2)) <= 1e-12 * I1.max()
    I3 = np.abs(oracle_lib.mft(np.conj(P), 0.1 / ni, no, 1.5e-6, LAM)) ** 2
    assert np.max(np.abs(I1 - I3)) > 1e-6 * I1.max()  # conjugation alone does change it


def test_phasor_definition(oracle_lib):
    """Phasor = T_hat exp(i 2pi/lambda OPD) at zero tilt, unit power (normalise=True)."""
    p = W.make_problem("custom", n_pupil=16, n_det=8, oversample=2, obscuration=0.3)
    P = oracle_lib.phasor(p, 0, 0, 0)
    assert abs(np.sum(np.abs(P) ** 2) - 1) < 1e-13
    opd = oracle_lib.opd(p)
    assert np.allclose(opd, p.opd_fixed + np.tensordot(p.coeff, p.basis, 1), atol=1e-20)
    T = p.transmission / np.sqrt(np.sum(p.transmission**2))
    assert np.allclose(P, T * np.exp(2j * np.pi * opd / p.lambdas[0]), atol=1e-14)


# ---------------------------------------------------------------- model + gradient pins

def _small_model(seed=11, with_pix=True):
    p = W.make_problem("custom", seed=seed, n_pupil=16, n_det=8, oversample=2, n_lambda=2, n_src=2, n_exp=2,
                       dither_px=0.5, flux_total=2e5, obscuration=0.2, grating=True)
    p.noll = [2, 3, 4, 5, 7]
    p.basis = W.zernike_basis(p.noll, p.n_pupil, p.diameter)
    p.coeff = 20e-9 * np.random.default_rng(seed).standard_normal(5)
    p.weights = np.array([0.7, 1.3])
    # hard-edged support: every transmitting pixel lies inside the Zernike unit disk
    p.transmission = W.aperture(p.n_pupil, p.diameter, 0.2, oversample=1)
    if with_pix:
        p.opd_pix = W.smooth_gaussian_noise(p.n_pupil, 5e-9, 1.0, seed + 1)
    return p


@pytest.fixture(scope="module")
def fit_case(oracle_lib):
    truth = _small_model()
    data = W.poisson_counts(oracle_lib.forward(truth), 21)
    start = W.perturbed_start(truth, 22)
    start.coeff = 0.5 * truth.coeff
    start.opd_pix = 0.5 * truth.opd_pix
    start.flat = W.flat_field(truth.n_det, 0.05, 23)
    return start, data


def test_model_is_binned_flux_weighted_psf(oracle_lib, fit_case):
    p, _ = fit_case
    model, psf = oracle_lib.forward(p, with_psf=True)
    os_ = p.oversample
    binned = psf.reshape(p.n_exp, p.n_det, os_, p.n_det, os_).sum(axis=(2, 4))
    assert np.allclose(model, p.flat * binned, rtol=1e-13)
    # per-PSF intensities weighted by normalised spectrum and flux
    ref = np.zeros_like(psf[0])
    w = p.weights / p.weights.sum()
    for s in range(p.n_src):
        for l in range(p.n_lambda):
            ref += p.flux[s] * w[l] * np.abs(oracle_lib.psf_field(p, l, s, 0)) ** 2
    assert np.allclose(psf[0], ref, rtol=1e-12)


def test_loss_is_poisson_nll(oracle_lib, fit_case):
    p, d = fit_case
    m = oracle_lib.forward(p)
    L = oracle_lib.loss(p, d)
    assert L == pytest.approx(np.sum(m - d * np.log(m)), rel=1e-13)


def test_weight_scale_invariance(oracle_lib, fit_case):
    p, d = fit_case
    q = p.copy()
    q.weights = 3.7 * p.weights
    assert oracle_lib.loss(q, d) == pytest.approx(oracle_lib.loss(p, d), rel=1e-13)


def _fd(oracle_lib, p, d, setter, h):
    a, b = p.copy(), p.copy()
    setter(a, +h)
    setter(b, -h)
    return (oracle_lib.loss(a, d) - oracle_lib.loss(b, d)) / (2 * h)


def test_gradient_central_differences(oracle_lib, fit_case):
    """Analytic adjoint vs central finite differences for every parameter group."""
    p, d = fit_case
    g = oracle_lib.loss_grad(p, d)
    rng = np.random.default_rng(7)
    checks = []

    for j in range(p.n_zern):
        def s(q, h, j=j):
            q.coeff = q.coeff.copy()
            q.coeff[j] += h
        checks.append((g["coeff"][j], _fd(oracle_lib, p, d, s, 2e-11)))
    for _ in range(6):
        iy, ix = rng.integers(3, 13, 2)

        def s(q, h, iy=iy, ix=ix):
            q.opd_pix = q.opd_pix.copy()
            q.opd_pix[iy, ix] += h
        checks.append((g["opd_pix"][iy, ix], _fd(oracle_lib, p, d, s, 2e-11)))
    for _ in range(6):
        iy, ix = rng.integers(0, 8, 2)

        def s(q, h, iy=iy, ix=ix):
            q.flat = q.flat.copy()
            q.flat[iy, ix] += h
        checks.append((g["flat"][iy, ix], _fd(oracle_lib, p, d, s, 1e-6)))
    for si in range(p.n_src):
        def s(q, h, si=si):
            q.flux = q.flux.copy()
            q.flux[si] += h
        checks.append((g["flux"][si], _fd(oracle_lib, p, d, s, 1e-6 * p.flux[si])))
        for ax in range(2):
            def s(q, h, si=si, ax=ax):
                q.pos = q.pos.copy()
                q.pos[si, ax] += h
            checks.append((g["pos"][si, ax], _fd(oracle_lib, p, d, s, 1e-4 * p.pixscale / p.oversample)))
    for ana, num in checks:
        assert ana == pytest.approx(num, rel=2e-6, abs=1e-9 * max(1.0, abs(num)))


def test_euler_identities(oracle_lib, fit_case):
    """m is homogeneous of degree 1 in the fluxes and in the flat field, so
    sum_s F_s dL/dF_s = sum_p m g_m = sum_p FF_p dL/dFF_p."""
    p, d = fit_case
    g = oracle_lib.loss_grad(p, d)
    m = g["model"]
    s_m = np.sum(m - d)
    assert np.dot(p.flux, g["flux"]) == pytest.approx(s_m, rel=1e-11)
    assert np.sum(p.flat * g["flat"]) == pytest.approx(s_m, rel=1e-11)


def test_tilt_zernike_consistency(oracle_lib, fit_case):
    """A common tilt of every source equals the Noll Z2/Z3 slope 4/D."""
    p, d = fit_case
    g = oracle_lib.loss_grad(p, d)
    assert p.noll[0] == 2 and p.noll[1] == 3
    assert np.sum(g["pos"][:, 0]) == pytest.approx(p.diameter / 4 * g["coeff"][0], rel=1e-9)
    assert np.sum(g["pos"][:, 1]) == pytest.approx(p.diameter / 4 * g["coeff"][1], rel=1e-9)


def test_pixel_opd_gradient_zero_outside_aperture(oracle_lib, fit_case):
    p, d = fit_case
    g = oracle_lib.loss_grad(p, d)
    out = p.transmission == 0
    assert out.any()
    assert np.all(g["opd_pix"][out] == 0.0)
    assert np.any(g["opd_pix"][~out] != 0.0)


def test_zernike_gradient_is_basis_projection(oracle_lib, fit_case):
    p, d = fit_case
    g = oracle_lib.loss_grad(p, d)
    assert np.allclose(g["coeff"], np.tensordot(p.basis, g["opd_pix"], 2), rtol=1e-12)


# ---------------------------------------------------------------- input generators

NOLL_TABLE = {1: (0, 0), 2: (1, 1), 3: (1, -1), 4: (2, 0), 5: (2, -2), 6: (2, 2), 7: (3, -1), 8: (3, 1),
              9: (3, -3), 10: (3, 3), 11: (4, 0), 12: (4, 2), 13: (4, -2), 14: (4, 4), 15: (4, -4),
              16: (5, 1), 17: (5, -1), 18: (5, 3), 19: (5, -3), 20: (5, 5), 21: (5, -5), 22: (6, 0)}


def test_noll_index_table():
    for j, nm in NOLL_TABLE.items():
        assert W.noll_to_nm(j) == nm


def test_zernike_basis_orthonormal():
    npix, D = 400, 1.0
    Z = W.zernike_basis(list(range(1, 16)), npix, D)
    c = W.pixel_coords(npix, D)
    inside = np.hypot(*np.meshgrid(c, c)) <= 0.5 * D
    G = np.einsum("iyx,jyx->ij", Z * inside, Z * inside) / inside.sum()
    assert np.max(np.abs(G - np.eye(15))) < 2e-2
    Z2 = W.zernike_basis([2], npix, D)[0]
    xx = np.meshgrid(c, c)[0]
    assert np.allclose(Z2[inside], 4 * xx[inside] / D)


def test_sampled_model_equals_full_forward(oracle_lib, fit_case):
    """The per-pixel direct-sum model equals the full forward at the sampled pixels."""
    p, _ = fit_case
    m = oracle_lib.forward(p)
    rng = np.random.default_rng(9)
    e = rng.integers(0, p.n_exp, 12)
    q = rng.integers(0, p.n_det * p.n_det, 12)
    got = oracle_lib.model_at(p, e, q)
    assert np.allclose(got, m.reshape(p.n_exp, -1)[e, q], rtol=1e-12, atol=0)


# ---------------------------------------------------------------- chi^2 prior on the pixel response

def test_prf_prior_posterior_mode(oracle_lib, fit_case):
    """With the chi^2 prior (Sec. 4: pixel response about 1, s.d. sigma) and one exposure, the
    flat-field gradient of one pixel is b - d/FF + (FF - 1)/sigma^2 with b the unflattened model,
    so it vanishes at the positive root of FF^2/sigma^2 + (b - 1/sigma^2) FF - d = 0: the
    per-pixel posterior mode, found here by the quadratic formula, not by the oracle."""
    p, _ = fit_case
    q = p.copy()
    q.dither = q.dither[:1]
    q.flat = np.ones_like(q.flat)
    b = oracle_lib.forward(q)[0]  # FF = 1: the model is the binned flux-weighted intensity
    d = W.poisson_counts(b[None], 31)
    sigma = 0.1
    a2 = 1.0 / sigma**2
    c1 = b - a2
    ff = (-c1 + np.sqrt(c1 * c1 + 4 * a2 * d[0])) / (2 * a2)
    q.flat = ff
    q.prf_sigma = sigma
    g = oracle_lib.loss_grad(q, d)["flat"]
    scale = b + d[0] / ff + np.abs(ff - 1) * a2  # size of the three terms
    assert np.max(np.abs(g) / scale) < 1e-12
    # without the prior the same point is not stationary
    q.prf_sigma = 0.0
    assert np.max(np.abs(oracle_lib.loss_grad(q, d)["flat"]) / scale) > 1e-3


def test_prf_prior_gradient_central_differences(oracle_lib, fit_case):
    p, d = fit_case
    q = p.copy()
    q.prf_sigma = 0.1
    g = oracle_lib.loss_grad(q, d)
    rng = np.random.default_rng(9)
    for _ in range(6):
        iy, ix = rng.integers(0, 8, 2)

        def s(r, h, iy=iy, ix=ix):
            r.flat = r.flat.copy()
            r.flat[iy, ix] += h
        assert g["flat"][iy, ix] == pytest.approx(_fd(oracle_lib, q, d, s, 1e-6), rel=2e-6)
    # the prior changes no other group
    g0 = oracle_lib.loss_grad(p, d)
    for k in ("coeff", "opd_pix", "flux", "pos"):
        assert np.array_equal(g[k], g0[k])
