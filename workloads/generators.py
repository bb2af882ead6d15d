"""Seeded input generators for the differentiable-optics workloads.

Every array here is an *input* to the forward model of arXiv:2406.08703
(Sec. 3): the grey aperture transmission (Listing 1, `dlu.circle` /
`dlu.combine` on a 3x supersampled grid), Noll-indexed Zernike basis images
(Listing 1, `dlu.zernike_basis`), a smoothed binary phase grating standing in
for the Toliman pupil mask (Sec. 3; the paper's `mask.npy` is not public), the
pixel response map (Listing 2, `1 + 0.1 N(0,1)`), source positions/fluxes,
wavelength grids, and Poisson counts drawn from a caller-supplied expectation.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.  Angles are
in radians (1 arcsec = pi/648000 rad); lengths in metres.  Arrays are
row-major ``[y][x]`` with pixel-centred symmetric grids.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

ARCSEC = math.pi / 648000.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def pixel_coords(npix: int, diameter: float) -> np.ndarray:
    """Centred 1-D pixel coordinates spanning ``diameter`` (Listing 1, `dlu.pixel_coords`).

    Pixel i sits at (i - (npix-1)/2) * diameter/npix, so the array spans the
    diameter exactly and an even-sized grid has no pixel at the origin.
    """
    return (np.arange(npix, dtype=np.float64) - 0.5 * (npix - 1)) * (diameter / npix)


def aperture(npix: int, diameter: float, obscuration: float = 0.0, oversample: int = 3) -> np.ndarray:
    """Grey circular aperture with optional central obscuration (Listing 1).

    The outer circle has radius D/2, the inverted inner circle has radius
    ``obscuration*D/2``.  Both are evaluated on an ``oversample``-times finer
    grid and the hard masks are averaged over each oversample x oversample
    block, giving the area-fraction anti-aliasing of `dlu.combine`.
    """
    fine = pixel_coords(npix * oversample, diameter)
    yy, xx = np.meshgrid(fine, fine, indexing="ij")
    r = np.hypot(xx, yy)
    mask = (r <= 0.5 * diameter).astype(np.float64)
    if obscuration > 0.0:
        mask *= (r > 0.5 * obscuration * diameter).astype(np.float64)
    return mask.reshape(npix, oversample, npix, oversample).mean(axis=(1, 3))


def noll_to_nm(j: int) -> tuple[int, int]:
    """Noll (1976) single index j >= 1 -> (radial order n, azimuthal m).

    Within radial order n the |m| values run upward from n mod 2; each
    non-zero |m| occupies two consecutive indices, the even index carrying the
    cosine term (m > 0) and the odd index the sine term (m < 0).
    """
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    first = n * (n + 1) // 2 + 1  # first Noll index of order n
    pos = j - first  # position inside the order
    if n % 2 == 0:
        if pos == 0:
            return n, 0
        mabs = 2 * ((pos + 1) // 2)
    else:
        mabs = 2 * (pos // 2) + 1
    return n, (mabs if j % 2 == 0 else -mabs)


def _radial(n: int, mabs: int, rho: np.ndarray) -> np.ndarray:
    out = np.zeros_like(rho)
    for k in range((n - mabs) // 2 + 1):
        c = ((-1) ** k) * math.factorial(n - k) / (
            math.factorial(k) * math.factorial((n + mabs) // 2 - k) * math.factorial((n - mabs) // 2 - k)
        )
        out += c * rho ** (n - 2 * k)
    return out


def zernike_basis(noll: list[int], npix: int, diameter: float) -> np.ndarray:
    """Noll-normalised Zernike images on the pupil grid (Listing 1, `dlu.zernike_basis`).

    Unit RMS over the unit disk of radius D/2; zero outside it.  Coefficients
    multiplying these images are metres of RMS OPD.  x is the column axis and
    phi is measured from +x toward +y, so Z2 = 2 rho cos(phi) = 4 x / D.
    """
    c = pixel_coords(npix, diameter)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    rho = np.hypot(xx, yy) / (0.5 * diameter)
    phi = np.arctan2(yy, xx)
    inside = rho <= 1.0
    out = np.zeros((len(noll), npix, npix), dtype=np.float64)
    for i, j in enumerate(noll):
        n, m = noll_to_nm(j)
        r = _radial(n, abs(m), rho)
        if m == 0:
            z = math.sqrt(n + 1) * r
        elif m > 0:
            z = math.sqrt(2 * (n + 1)) * r * np.cos(m * phi)
        else:
            z = math.sqrt(2 * (n + 1)) * r * np.sin(-m * phi)
        out[i] = np.where(inside, z, 0.0)
    return out


def _gauss_smooth(img: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur (reflecting edges), radius 4 sigma."""
    rad = int(math.ceil(4 * sigma))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    out = img
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        for i, w in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(i, i + out.shape[axis])
            acc += w * p[tuple(sl)]
        out = acc
    return out


def binary_grating(npix: int, cell: int, sigma: float, seed: int) -> np.ndarray:
    """Seeded 0/1 pattern on ``cell`` x ``cell`` pixel blocks, Gaussian-smoothed.

    A synthetic stand-in for the binary diffractive pupil (Sec. 3); values lie
    in [0, 1].  Multiply by half the band-centre wavelength to get an OPD with
    a half-wave step between the two regions.
    """
    nc = -(-npix // cell)
    cells = _rng(seed).integers(0, 2, size=(nc, nc)).astype(np.float64)
    img = np.kron(cells, np.ones((cell, cell)))[:npix, :npix]
    return _gauss_smooth(img, sigma)


def smooth_gaussian_noise(npix: int, rms: float, sigma: float, seed: int) -> np.ndarray:
    """Gaussian white noise smoothed by a Gaussian of ``sigma`` pixels, rescaled to ``rms``."""
    w = _rng(seed).standard_normal((npix, npix))
    s = _gauss_smooth(w, sigma)
    return s * (rms / s.std())


def flat_field(npix: int, sd: float, seed: int, dead_frac: float = 0.0, dead_value: float = 0.1) -> np.ndarray:
    """Pixel response map 1 + sd N(0,1) (Listing 2), with an optional seeded set of dead pixels."""
    rng = _rng(seed)
    ff = 1.0 + sd * rng.standard_normal((npix, npix))
    if dead_frac > 0.0:
        nd = int(round(dead_frac * npix * npix))
        idx = rng.choice(npix * npix, size=nd, replace=False)
        ff.reshape(-1)[idx] = dead_value
    return ff


def poisson_counts(expectation: np.ndarray, seed: int) -> np.ndarray:
    """Photon-noise data: independent Poisson draws of the expectation image (Sec. 3), int32."""
    lam = np.clip(np.asarray(expectation, dtype=np.float64), 0.0, None)
    d = _rng(seed).poisson(lam)
    if d.max(initial=0) >= 2**31:
        raise OverflowError("counts exceed int32")
    return d.astype(np.int32)


def synthetic_counts(shape: tuple[int, ...], total: float, centres_px: np.ndarray, width_px: float, seed: int) -> np.ndarray:
    """Poisson counts of an analytic expectation (a sum of Gaussian spots plus a floor).

    Used where the data must be generated at sizes the oracle cannot afford:
    the expectation is *not* the optical model, only an image with the same
    total flux and a concentrated-light-on-a-floor structure.  ``shape`` is
    (n_exp, nd, nd); ``centres_px`` is (n_spots, 2) pixel offsets (x, y) from
    the detector centre.
    """
    ne, ny, nx = shape
    yy, xx = np.meshgrid(np.arange(ny) - 0.5 * (ny - 1), np.arange(nx) - 0.5 * (nx - 1), indexing="ij")
    img = np.zeros((ny, nx))
    for cx, cy in np.atleast_2d(centres_px):
        img += np.exp(-0.5 * ((xx - cx) ** 2 + (yy - cy) ** 2) / width_px**2)
    img = img / img.sum() * 0.98 + 0.02 / img.size
    exp_img = np.broadcast_to(img * (total / ne), shape)
    return poisson_counts(exp_img, seed)


@dataclasses.dataclass
class Problem:
    """All inputs of one forward-model evaluation (truth or a starting point)."""

    name: str
    n_pupil: int
    diameter: float
    n_det: int
    pixscale: float  # rad per detector pixel
    oversample: int
    lambdas: np.ndarray  # (n_lambda,) m
    weights: np.ndarray  # (n_lambda,) unnormalised spectral weights
    flux: np.ndarray  # (n_src,) photons per source per exposure
    pos: np.ndarray  # (n_src, 2) (theta_x, theta_y) rad
    dither: np.ndarray  # (n_exp, 2) rad, known offsets
    noll: list
    basis: np.ndarray  # (n_zern, n, n)
    coeff: np.ndarray  # (n_zern,) m RMS
    transmission: np.ndarray  # (n, n)
    opd_fixed: np.ndarray  # (n, n) m
    opd_pix: Optional[np.ndarray]  # (n, n) m, or None when the pixel OPD map is not a parameter
    flat: np.ndarray  # (n_det, n_det)
    prf_sigma: float = 0.0  # s.d. of the chi^2 prior on the flat field about 1 (0: no prior)
    focal_length: float = 0.0  # m; > 0: Fresnel regime with the detector at focal_length + focal_shift
    focal_shift: float = 0.0  # m

    @property
    def n_lambda(self) -> int:
        return len(self.lambdas)

    @property
    def n_src(self) -> int:
        return len(self.flux)

    @property
    def n_exp(self) -> int:
        return len(self.dither)

    @property
    def n_zern(self) -> int:
        return len(self.coeff)

    @property
    def n_out(self) -> int:
        return self.n_det * self.oversample

    @property
    def n_psf(self) -> int:
        return self.n_lambda * self.n_src * self.n_exp

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def copy(self) -> "Problem":
        out = dataclasses.replace(self)
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, np.ndarray):
                setattr(out, f.name, v.copy())
        return out


def _band(n: int, lo: float = 530e-9, hi: float = 640e-9) -> np.ndarray:
    return np.linspace(lo, hi, n) if n > 1 else np.array([0.5 * (lo + hi)])


def make_problem(name: str, seed: Optional[int] = None, **over) -> Problem:
    """The workloads, with the truth parameters.

    ``tiny``      64^2 unobstructed pupil, Noll 4-11, 595 nm, one on-axis star (1e6),
                  64^2 detector at 0.375 arcsec, oversample 4, flat N(1, 0.05).
    ``binary``    256^2 pupil with 0.2 D obstruction and a smoothed 0/1 grating at
                  half-wave of 585 nm; two stars 8 arcsec apart, flux 1e8 total,
                  ratio 0.3; 32 wavelengths in 530-640 nm; 256^2 detector, oversample
                  4; Noll 2-21; pixel OPD truth N(0, 5 nm) smoothed 3 px; flat N(1, 0.03).
    ``calib``     512^2 pupil, Noll 2-36 + pixel OPD; 16 wavelengths; 8 dithered
                  exposures (U(-0.5, 0.5) px) of one star with 1e9 photons in total;
                  1024^2 detector, oversample 2; flat N(1, 0.02) with 1% dead at 0.1.
    ``paper``     the configuration of Sec. 3 (20 stars, 545/595/645 nm, 512^2 pupil,
                  D = 0.5 m, 1024^2 detector at 12 mas, Noll 4-10, flat 1 + 0.1 N(0,1)).
    ``custom``    keyword overrides of the tiny case (n_pupil, n_det, oversample,
                  n_lambda, n_src, n_exp, n_zern_max, obscuration, grating, ...).

    Keyword overrides apply to the shape parameters listed under ``custom``.
    """
    seeds = {"tiny": 1, "binary": 2, "calib": 4, "paper": 6, "custom": 7}
    seed = seeds.get(name, 7) if seed is None else seed
    rng = _rng(seed)
    if name == "tiny":
        cfg = dict(n_pupil=64, diameter=0.125, n_det=64, pix_arcsec=0.375, oversample=4, n_lambda=1,
                   lam_single=595e-9, noll=list(range(4, 12)), zern_rms=20e-9, obscuration=0.0,
                   grating=False, n_src=1, flux_total=1e6, sep_arcsec=0.0, ratio=1.0, n_exp=1,
                   dither_px=0.0, flat_sd=0.05, dead_frac=0.0, opd_pix_rms=None)
    elif name == "binary":
        cfg = dict(n_pupil=256, diameter=0.125, n_det=256, pix_arcsec=0.375, oversample=4, n_lambda=32,
                   lam_single=None, noll=list(range(2, 22)), zern_rms=20e-9, obscuration=0.2,
                   grating=True, n_src=2, flux_total=1e8, sep_arcsec=8.0, ratio=0.3, n_exp=1,
                   dither_px=0.0, flat_sd=0.03, dead_frac=0.0, opd_pix_rms=5e-9)
    elif name == "calib":
        cfg = dict(n_pupil=512, diameter=0.125, n_det=1024, pix_arcsec=0.375, oversample=2, n_lambda=16,
                   lam_single=None, noll=list(range(2, 37)), zern_rms=20e-9, obscuration=0.0,
                   grating=False, n_src=1, flux_total=1e9, sep_arcsec=0.0, ratio=1.0, n_exp=8,
                   dither_px=0.5, flat_sd=0.02, dead_frac=0.01, opd_pix_rms=5e-9)
    elif name == "paper":
        # Sec. 3's example: 20 stars x 3 wavelengths, 512^2 wavefront -> 1024^2 detector, the
        # undithered image and four integer-pixel dithers of +-20 pixels (5 images)
        cfg = dict(n_pupil=512, diameter=0.5, n_det=1024, pix_arcsec=0.012, oversample=1, n_lambda=3,
                   lam_single=None, noll=list(range(4, 11)), zern_rms=20e-9, obscuration=0.2,
                   grating=True, n_src=20, flux_total=1e8, sep_arcsec=None, ratio=1.0, n_exp=5,
                   dither_px=20.0, flat_sd=0.1, dead_frac=0.0, opd_pix_rms=None)
    elif name == "custom":
        cfg = dict(n_pupil=64, diameter=0.125, n_det=64, pix_arcsec=0.375, oversample=4, n_lambda=1,
                   lam_single=595e-9, noll=list(range(4, 12)), zern_rms=20e-9, obscuration=0.0,
                   grating=False, n_src=1, flux_total=1e6, sep_arcsec=0.0, ratio=1.0, n_exp=1,
                   dither_px=0.0, flat_sd=0.05, dead_frac=0.0, opd_pix_rms=None)
    else:
        raise ValueError(f"unknown workload {name!r}")
    for k, v in over.items():
        if k not in cfg and k != "n_zern_max":
            raise KeyError(k)
        cfg[k] = v
    if "n_zern_max" in over:
        cfg["noll"] = list(range(2, 2 + over["n_zern_max"]))

    ni, D, nd, osf = cfg["n_pupil"], cfg["diameter"], cfg["n_det"], cfg["oversample"]
    pix = cfg["pix_arcsec"] * ARCSEC
    if name == "paper":
        lambdas = 1e-9 * np.linspace(545.0, 645.0, 3)
    elif cfg["n_lambda"] == 1 and cfg["lam_single"] is not None:
        lambdas = np.array([cfg["lam_single"]])
    else:
        lambdas = _band(cfg["n_lambda"])
    weights = np.ones_like(lambdas)
    trans = aperture(ni, D, cfg["obscuration"])
    if cfg["grating"]:
        lam_c = 585e-9 if name != "paper" else 595e-9
        opd_fixed = 0.5 * lam_c * binary_grating(ni, max(ni // 16, 1), 3.0, seed + 100)
    else:
        opd_fixed = np.zeros((ni, ni))
    noll = list(cfg["noll"])
    basis = zernike_basis(noll, ni, D)
    coeff = cfg["zern_rms"] * rng.standard_normal(len(noll))
    ns = cfg["n_src"]
    if name == "paper":
        fov = 0.4 * nd * pix
        pos = rng.uniform(-fov, fov, size=(ns, 2))
        flux = np.full(ns, cfg["flux_total"] / ns)
    elif ns == 2 and cfg["sep_arcsec"]:
        half = 0.5 * cfg["sep_arcsec"] * ARCSEC
        pos = np.array([[-half, 0.0], [half, 0.0]])
        f1 = cfg["flux_total"] / (1.0 + cfg["ratio"])
        flux = np.array([f1, cfg["ratio"] * f1])
    else:
        spread = 0.15 * nd * pix
        pos = np.zeros((ns, 2)) if ns == 1 else rng.uniform(-spread, spread, size=(ns, 2))
        flux = np.full(ns, cfg["flux_total"] / ns)
    ne = cfg["n_exp"]
    flux = flux / ne  # total flux spread evenly over the exposures (Sec. 3)
    if name == "paper":
        # (0, 0) and the four (+-20, +-20) pixel offsets, cut to n_exp
        steps = np.array([[0, 0], [1, 1], [1, -1], [-1, 1], [-1, -1]], np.float64)
        dither = cfg["dither_px"] * pix * steps[:ne] if ne <= 5 else np.zeros((ne, 2))
    elif ne > 1 and cfg["dither_px"]:
        dither = rng.uniform(-cfg["dither_px"], cfg["dither_px"], size=(ne, 2)) * pix
    else:
        dither = np.zeros((ne, 2))
    opd_pix = None
    if cfg["opd_pix_rms"] is not None:
        opd_pix = smooth_gaussian_noise(ni, cfg["opd_pix_rms"], 3.0, seed + 200)
    flat = flat_field(nd, cfg["flat_sd"], seed + 300, cfg["dead_frac"])
    # Sec. 4 fits the paper's example with a chi^2 prior matching the pixel-response spread
    prf_sigma = cfg["flat_sd"] if name == "paper" else 0.0
    return Problem(name=name, n_pupil=ni, diameter=D, n_det=nd, pixscale=pix, oversample=osf,
                   lambdas=lambdas, weights=weights, flux=flux, pos=pos, dither=dither, noll=noll,
                   basis=basis, coeff=coeff, transmission=trans, opd_fixed=opd_fixed, opd_pix=opd_pix,
                   flat=flat, prf_sigma=prf_sigma)


def perturbed_start(truth: Problem, seed: int) -> Problem:
    """Starting point of a fit (Sec. 4): unaberrated, uniform flat field, positions
    perturbed by N(0, 1 px), fluxes multiplied by N(1, 0.1)."""
    rng = _rng(seed)
    p = truth.copy()
    p.coeff = np.zeros_like(truth.coeff)
    if p.opd_pix is not None:
        p.opd_pix = np.zeros_like(truth.opd_pix)
    p.flat = np.ones_like(truth.flat)
    p.pos = truth.pos + truth.pixscale * rng.standard_normal(truth.pos.shape)
    p.flux = truth.flux * rng.normal(1.0, 0.1, size=truth.flux.shape)
    return p


def serving_request_shapes(n: int, seed: int) -> list[dict]:
    """Shapes of mixed-size fit requests: pupil {128, 256, 512}, detector
    {64, 128, 256, 512}, oversample {2, 4}, wavelengths {1, 8, 32, 64}, 1-3 sources."""
    rng = _rng(seed)
    out = []
    for _ in range(n):
        out.append(dict(n_pupil=int(rng.choice([128, 256, 512])), n_det=int(rng.choice([64, 128, 256, 512])),
                        oversample=int(rng.choice([2, 4])), n_lambda=int(rng.choice([1, 8, 32, 64])),
                        n_src=int(rng.integers(1, 4))))
    return out
