"""GPU: the hand-written adjoint is the transpose of the forward linearisation (the dot-product
test of an adjoint).  For a random optical-path direction t and a random pixel weight c,

    < c, J t >  =  < t, J^T c >_OPD,

with J t from dlx_model_jvp (the model's derivative along OPD -> OPD + e t, exact as a central
difference because the model is quadratic in the phasor) and J^T c from dlx_model_vjp (the pixel
OPD gradient of sum c m).  The same holds per source for the positions (t = the pupil x or y
coordinate, one source's bit) and for the Zernike terms (t = Z_j).  Both sides come from the GPU
path alone, so this checks the adjoint chain (stage 2^T, stage 1^T, phase gradient, binning and
window folds) against the forward chain independently of the oracle, for the plan variants whose
adjoints differ: sub-pixel dithers, integer-dither windows, more than eight sources (two-pass
binning and the split-plane fold) and the Fresnel regime."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "dithered": dict(n_pupil=40, n_det=20, oversample=2, n_lambda=3, n_src=2, n_exp=2, n_zern_max=6),
    "windows": dict(n_pupil=36, n_det=16, oversample=2, n_lambda=2, n_src=3, n_exp=3, n_zern_max=5),
    "ten_sources": dict(n_pupil=32, n_det=12, oversample=3, n_lambda=2, n_src=10, n_exp=1, n_zern_max=4),
    "fresnel": dict(n_pupil=40, n_det=20, oversample=2, n_lambda=2, n_src=2, n_exp=1, n_zern_max=5),
}
TOL = {"fp32": 2e-5, "bf16x3": 2e-4, "f16x3": 2e-4}


def _problem(name):
    kw = dict(CASES[name])
    p = W.make_problem("custom", seed=90 + len(name), opd_pix_rms=5e-9, **kw)
    if name == "dithered":
        p.dither = np.array([[0.0, 0.0], [0.37, -0.21]]) * p.pixscale
    if name == "windows":
        p.dither = np.array([[0, 0], [2, -1], [-1, 3]], dtype=np.float64) * p.pixscale
    if name == "fresnel":
        f, R = 1.2, 0.5 * p.diameter
        p.focal_length = f
        p.focal_shift = 3.0 * float(np.min(p.lambdas)) * f * f / (np.pi * R * R)  # ~3 rad of edge phase
    return p


def _dot_check(lhs, rhs, scale, tol, what):
    assert abs(lhs - rhs) <= tol * scale, (what, lhs, rhs, scale)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("form", ["fp32", "bf16x3", "f16x3"])
def test_adjoint_is_the_transpose_of_the_linearisation(name, form):
    import torch

    import paper_2406_08703_gb300 as P

    p = _problem(name)
    crop = name == "windows"
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.PRECISIONS[form], crop=crop))
    prm = P.params_from_problem(p)
    i = plan.info
    rng = np.random.default_rng(7)
    ni = p.n_pupil
    lam_min = float(np.min(p.lambdas))
    c = torch.as_tensor(rng.uniform(-1.0, 1.0, (i.n_exp, i.n_det, i.n_det)).astype(np.float32), device="cuda")
    g = P.dlx_model_vjp(plan, prm, c)  # J^T c for every parameter group
    model = P.dlx_forward(plan, prm)
    torch.cuda.synchronize()
    tol = TOL[form]

    def jvp(t, mask):
        t = np.ascontiguousarray(t, dtype=np.float32)
        alpha = 1.0 / (2 * np.pi / lam_min * max(float(np.max(np.abs(t))), 1e-30))  # alpha max|a| = 1
        out = P.dlx_model_jvp(plan, prm, torch.as_tensor(t, device="cuda"), mask, alpha)
        torch.cuda.synchronize()
        return out.double().cpu().numpy()

    cn = c.double().cpu().numpy()
    all_src = (1 << p.n_src) - 1
    # a random optical-path direction (about 10 nm) against the pixel-OPD gradient
    t = 1e-8 * rng.standard_normal((ni, ni))
    jt = jvp(t, all_src)
    lhs = float(np.sum(cn * jt))
    rhs = float(np.sum(t.astype(np.float32).astype(np.float64) * g["d_opd_pix"].double().cpu().numpy()))
    _dot_check(lhs, rhs, float(np.sum(np.abs(cn * jt))), tol, "opd")
    # Zernike terms: t = Z_j
    dz = g["d_zern"].double().cpu().numpy()
    for j in range(len(p.coeff)):
        jt = jvp(p.basis[j], all_src)
        _dot_check(float(np.sum(cn * jt)), dz[j], float(np.sum(np.abs(cn * jt))), tol, f"zern {j}")
    # positions: t = the pupil x or y coordinate, one source at a time (Fresnel: the tilt is the
    # same phase ramp, so the identity holds there too)
    xs = W.pixel_coords(ni, p.diameter)
    yy, xx = np.meshgrid(xs, xs, indexing="ij")
    dp = g["d_pos"].double().cpu().numpy()
    for s in range(min(p.n_src, 3)):
        for a, tmap in ((0, xx), (1, yy)):
            jt = jvp(tmap, 1 << s)
            _dot_check(float(np.sum(cn * jt)), dp[s, a], float(np.sum(np.abs(cn * jt))), tol, f"pos {s} {a}")
    # flux: the model is linear in F_s with flat field included, so sum c m_s / F_s = dL/dF_s; with every
    # source at once, sum_s F_s d/dF_s (sum c m) = sum c m
    fl = prm["flux"].double().cpu().numpy()
    tot = float(np.sum(cn * model.double().cpu().numpy()))
    _dot_check(float(np.sum(fl * g["d_flux"].double().cpu().numpy())), tot,
               float(np.sum(np.abs(cn * model.double().cpu().numpy()))), tol, "flux")
    # flat field: m = FF B, so d/dFF (sum c m) = c B = c m / FF, summed over exposures
    ff = prm["flat"].double().cpu().numpy()
    want = np.sum(cn * model.double().cpu().numpy(), axis=0) / ff
    got = g["d_flat"].double().cpu().numpy()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want)), "flat"
    plan.close()
