"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/dlx.h declares; the Python binding covers them; argument validation
rejects bad shapes before touching a device."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dlx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dlx_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def native():
    from paper_2406_08703_gb300 import _native

    _native.load()
    return _native


def test_header_declares_the_path(native):
    names = _declared()
    for required in ("dlx_make_mft", "dlx_forward", "dlx_loss_grad", "dlx_submit", "dlx_poll"):
        assert required in names


def test_library_exports_every_declared_symbol(native):
    lib = C.CDLL(native.lib_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(native):
    assert set(_declared()) <= set(native.SIGNATURES)


def test_invalid_shapes_rejected_without_a_device(native):
    lib = native.load()
    lam = (C.c_double * 1)(595e-9)
    h = C.c_void_p()
    bad = [
        dict(n_pupil=1), dict(n_det=0), dict(oversample=0), dict(n_src=0), dict(n_exp=0), dict(precision=9),
        dict(diameter_m=0.0), dict(pixscale_rad=-1.0), dict(prf_prior_sigma=-0.1),
        dict(focal_length_m=-1.0), dict(focal_shift_m=1e-3), dict(focal_length_m=1.0, focal_shift_m=-1.0),
        dict(n_lambda=0), dict(n_zern=-1), dict(lambda_m=None),
        dict(lambda_m=C.cast((C.c_double * 1)(-595e-9), C.POINTER(C.c_double))),
        dict(lambda_m=C.cast((C.c_double * 1)(float("inf")), C.POINTER(C.c_double))),
        dict(focal_length_m=float("nan")),
    ]
    for over in bad:
        kw = dict(n_pupil=16, diameter_m=0.1, n_det=8, pixscale_rad=1e-6, oversample=2, n_lambda=1,
                  lambda_m=C.cast(lam, C.POINTER(C.c_double)), n_src=1, n_exp=1, n_zern=0, precision=0,
                  psf_chunk=0, workspace_limit_bytes=0)
        kw.update(over)
        d = native.MftDesc(**kw)
        rc = lib.dlx_make_mft(C.byref(d), 0, C.byref(h))
        assert rc == -1, (over, rc)
        assert lib.dlx_last_error()
    kw["n_src"] = 33
    kw["precision"] = 0
    kw["prf_prior_sigma"] = 0.0
    kw["diameter_m"] = 0.1
    kw["pixscale_rad"] = 1e-6
    kw["focal_length_m"] = 0.0
    kw["focal_shift_m"] = 0.0
    d = native.MftDesc(**kw)
    assert lib.dlx_make_mft(C.byref(d), 0, C.byref(h)) == -6  # RANGE
    assert lib.dlx_make_mft(None, 0, C.byref(h)) == -1
    kw["n_src"] = 1
    kw["n_exp"] = 2
    for bad_px, code in (((0, 0, 4097, 0), -6), ((0, 0, 0, -5000), -6)):
        dpx = (C.c_int32 * 4)(*bad_px)
        d = native.MftDesc(**kw, dither_px=C.cast(dpx, C.POINTER(C.c_int32)))
        assert lib.dlx_make_mft(C.byref(d), 0, C.byref(h)) == code
    kw["n_det"] = 4000
    dpx = (C.c_int32 * 4)(0, 0, 4096, 0)  # (4000 + 8192) * 2 > 16384
    d = native.MftDesc(**kw, dither_px=C.cast(dpx, C.POINTER(C.c_int32)))
    assert lib.dlx_make_mft(C.byref(d), 0, C.byref(h)) == -6
    assert lib.dlx_adam(None, None, None, None, 5, 1e-3, 0.9, 0.999, 1e-8, 1, None) == -1


def test_laplace_entries_validate_without_a_device(native):
    lib = native.load()
    fake = C.c_void_p(16)  # never dereferenced: every call below fails its argument checks first
    assert lib.dlx_model_jvp(None, None, fake, 1, 1.0, fake, fake, None) == -1
    assert lib.dlx_model_vjp(None, None, fake, None, None) == -1
    assert lib.dlx_model_vjp_jvp(None, None, fake, fake, 1, 1.0, None, None, None) == -1
    assert lib.dlx_nll_cotangent(None, fake, 4, fake, None) == -1
    for n_par in (0, 129):
        assert lib.dlx_fisher_gram(fake, n_par, 10, fake, None, fake, fake, None) == -6  # RANGE
    assert lib.dlx_fisher_gram(fake, 4, 0, fake, None, fake, fake, None) == -1
    assert lib.dlx_fisher_gram(None, 4, 10, fake, None, fake, fake, None) == -1


def test_version_string(native):
    assert b"sm_103a" in native.load().dlx_version()
