"""FP64 CPU oracle for the forward model, Poisson likelihood and gradient of
arXiv:2406.08703 (Sec. 3-4), written as plain C in ``dlx_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Importable by the tests, the package smoke check
and the benchmark's CPU baseline leg; the product library never calls it.
Every routine is pinned by the CPU tests (closed forms, library FFTs, brute
force, finite differences); none is marked "parity unpinned".
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_d = C.POINTER(C.c_double)
_i = C.POINTER(C.c_int)


class _Problem(C.Structure):
    _fields_ = [
        ("n_pupil", C.c_int), ("diameter", C.c_double), ("n_det", C.c_int), ("pixscale", C.c_double),
        ("oversample", C.c_int), ("n_lambda", C.c_int), ("lambdas", _d), ("weights", _d), ("n_src", C.c_int),
        ("flux", _d), ("pos", _d), ("n_exp", C.c_int), ("dither", _d), ("n_zern", C.c_int), ("basis", _d),
        ("coeff", _d), ("transmission", _d), ("opd_fixed", _d), ("opd_pix", _d), ("flat", _d),
        ("prf_sigma", C.c_double), ("focal_length", C.c_double), ("focal_shift", C.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        cp = C.c_void_p
        _lib.orc_mft.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, cp, cp]
        _lib.orc_mft_direct.argtypes = _lib.orc_mft.argtypes
        _lib.orc_mft_adjoint.argtypes = _lib.orc_mft.argtypes
        _lib.orc_mft_matrix.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, cp]
        _lib.orc_coords.argtypes = [C.c_int, C.c_double, cp]
        _lib.orc_opd.argtypes = [C.POINTER(_Problem), cp]
        _lib.orc_phasor.argtypes = [C.POINTER(_Problem), cp, C.c_int, C.c_int, C.c_int, cp]
        _lib.orc_psf_field.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_int, cp]
        _lib.orc_forward.argtypes = [C.POINTER(_Problem), cp, cp]
        _lib.orc_loss.argtypes = [C.POINTER(_Problem), cp]
        _lib.orc_loss.restype = C.c_double
        _lib.orc_loss_grad.argtypes = [C.POINTER(_Problem), cp, cp, cp, cp, cp, cp, cp, cp]
        _lib.orc_loss_grad.restype = C.c_long
        _lib.orc_model_at.argtypes = [C.POINTER(_Problem), C.c_int, cp, cp, cp]
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_set_threads.restype = C.c_int
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Marshalled:
    """Keeps the float64 copies alive while the C struct points into them."""

    def __init__(self, p):
        self.arrs = {k: _f64(getattr(p, k)) for k in
                     ("lambdas", "weights", "flux", "pos", "dither", "basis", "coeff", "transmission",
                      "opd_fixed", "flat")}
        self.arrs["opd_pix"] = None if p.opd_pix is None else _f64(p.opd_pix)
        if self.arrs["basis"].size == 0:
            self.arrs["basis"] = np.zeros((0,), np.float64)
        s = _Problem()
        s.n_pupil, s.diameter, s.n_det = p.n_pupil, p.diameter, p.n_det
        s.pixscale, s.oversample = p.pixscale, p.oversample
        s.n_lambda, s.n_src, s.n_exp, s.n_zern = len(p.lambdas), len(p.flux), len(p.dither), len(p.coeff)
        s.prf_sigma = float(getattr(p, "prf_sigma", 0.0) or 0.0)
        s.focal_length = float(getattr(p, "focal_length", 0.0) or 0.0)
        s.focal_shift = float(getattr(p, "focal_shift", 0.0) or 0.0)
        for k, a in self.arrs.items():
            setattr(s, k, C.cast(a.ctypes.data, _d) if a is not None else None)
        self.s = s

    def ref(self):
        return C.byref(self.s)


def coords(n: int, spacing: float) -> np.ndarray:
    out = np.zeros(n)
    lib().orc_coords(n, spacing, _ptr(out))
    return out


def mft_matrix(n_out, n_in, dx, du, lam):
    A = np.zeros((n_out, n_in), np.complex128)
    lib().orc_mft_matrix(n_out, n_in, dx, du, lam, _ptr(A))
    return A


def mft(P, dx, n_out, du, lam):
    P = _c128(P)
    E = np.zeros((n_out, n_out), np.complex128)
    lib().orc_mft(P.shape[0], dx, n_out, du, lam, _ptr(P), _ptr(E))
    return E


def mft_direct(P, dx, n_out, du, lam):
    P = _c128(P)
    E = np.zeros((n_out, n_out), np.complex128)
    lib().orc_mft_direct(P.shape[0], dx, n_out, du, lam, _ptr(P), _ptr(E))
    return E


def mft_adjoint(G, n_in, dx, du, lam):
    G = _c128(G)
    out = np.zeros((n_in, n_in), np.complex128)
    lib().orc_mft_adjoint(n_in, dx, G.shape[0], du, lam, _ptr(G), _ptr(out))
    return out


def opd(p):
    m = _Marshalled(p)
    out = np.zeros((p.n_pupil, p.n_pupil))
    lib().orc_opd(m.ref(), _ptr(out))
    return out


def phasor(p, l, s, e):
    m = _Marshalled(p)
    o = opd(p)
    P = np.zeros((p.n_pupil, p.n_pupil), np.complex128)
    lib().orc_phasor(m.ref(), _ptr(o), l, s, e, _ptr(P))
    return P


def psf_field(p, l, s, e):
    m = _Marshalled(p)
    E = np.zeros((p.n_out, p.n_out), np.complex128)
    lib().orc_psf_field(m.ref(), l, s, e, _ptr(E))
    return E


def forward(p, with_psf: bool = False):
    """Model image [n_exp][n_det][n_det]; with_psf also returns the oversampled
    flux-weighted intensity [n_exp][n_out][n_out] before binning."""
    m = _Marshalled(p)
    model = np.zeros((p.n_exp, p.n_det, p.n_det))
    psf = np.zeros((p.n_exp, p.n_out, p.n_out)) if with_psf else None
    lib().orc_forward(m.ref(), _ptr(model), _ptr(psf))
    return (model, psf) if with_psf else model


def loss(p, data):
    m = _Marshalled(p)
    d = np.ascontiguousarray(data, dtype=np.int32)
    return float(lib().orc_loss(m.ref(), _ptr(d)))


def loss_grad(p, data):
    """Returns dict(loss, model, coeff, opd_pix, flat, flux, pos, clamped)."""
    m = _Marshalled(p)
    d = np.ascontiguousarray(data, dtype=np.int32)
    L = np.zeros(1)
    out = dict(model=np.zeros((p.n_exp, p.n_det, p.n_det)), coeff=np.zeros(p.n_zern),
               opd_pix=np.zeros((p.n_pupil, p.n_pupil)), flat=np.zeros((p.n_det, p.n_det)),
               flux=np.zeros(p.n_src), pos=np.zeros((p.n_src, 2)))
    clamped = lib().orc_loss_grad(m.ref(), _ptr(d), _ptr(L), _ptr(out["model"]), _ptr(out["coeff"]),
                                  _ptr(out["opd_pix"]), _ptr(out["flat"]), _ptr(out["flux"]), _ptr(out["pos"]))
    out["loss"] = float(L[0])
    out["clamped"] = int(clamped)
    return out


def model_at(p, e_idx, p_idx):
    """Model values at (exposure, flat pixel index) pairs, each by direct sums."""
    m = _Marshalled(p)
    e = np.ascontiguousarray(e_idx, dtype=np.int32)
    q = np.ascontiguousarray(p_idx, dtype=np.int32)
    out = np.zeros(len(e))
    lib().orc_model_at(m.ref(), len(e), _ptr(e), _ptr(q), _ptr(out))
    return out


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (n < 1: one per processor); returns the count in use."""
    os.environ["OMP_NUM_THREADS"] = str(n) if n > 0 else str(os.cpu_count() or 1)
    return int(lib().orc_set_threads(int(n)))
