"""GPU parity of the Laplace-approximation errors (Sec. 4): the Jacobian
columns from dlx_model_jvp, the Gram products of dlx_fisher_gram and the
second-order term from dlx_model_vjp_jvp, against the FP64 oracle's
differences, and the closed forms of the full-period case on the GPU's own
result.

Tolerances.  A Jacobian column is (m(+a) - m(-a)) / (2 alpha) with the largest
phase change a near 1 rad, so its error is the forward model's (1e-5 of the
peak for the forms below) times a factor of order 1: bounded at 1e-4 of the
column's largest entry.  The Fisher and Gauss-Newton matrices are sums of
products of those columns: 1e-4 of sqrt(H_ii H_jj).  The Hessian adds
differences of two likelihood gradients, each within the form's gradient bound
(1e-4 FP32, 1e-3 BF16x3 relative L2), so it is held to those bounds of
sqrt(H_ii H_jj) (measured: 1.6e-7 FP32, 5e-6 BF16x3, as small as the Fisher
matrix's error, because near the data the second-order term is small).  The
errors themselves are compared after the inversion, relative, at 10x those
bounds: the aberrated case's condition number after scaling to unit diagonal is
below 10^2."""

import numpy as np
import pytest

from laplace_cases import LAM, aberrated_problem, laplace_problem

pytestmark = pytest.mark.gpu

TOL = {"fp32": dict(J=1e-4, info=1e-4, hess=1e-4), "bf16x3": dict(J=1e-4, info=1e-4, hess=1e-3),
       "f16x3": dict(J=1e-4, info=1e-4, hess=1e-3)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2406_08703_gb300 as P

    P.load()


def _gpu(problem, form, data=None, kinds=("fisher",), crop=False):
    import torch

    import paper_2406_08703_gb300 as P
    from paper_2406_08703_gb300.laplace import Laplace

    plan = P.dlx_make_mft(P.desc_from_problem(problem, P.PRECISIONS[form], crop=crop))
    prm = P.params_from_problem(problem)
    lp = Laplace(plan)
    J = lp.jacobian(prm).double().cpu().numpy()
    dt = None if data is None else torch.as_tensor(np.ascontiguousarray(data, dtype=np.int32), device="cuda")
    out = {k: lp.information(prm, dt, k).cpu().numpy() for k in kinds}
    torch.cuda.synchronize()
    assert P.dlx_plan_diagnostics(plan)["device_error"] == 0
    return J, out, lp.labels


def _rel(H, ref):
    s = np.sqrt(np.outer(np.abs(np.diag(ref)), np.abs(np.diag(ref))))
    s[s == 0] = np.max(np.abs(np.diag(ref)))
    return float(np.max(np.abs(H - ref) / s))


@pytest.mark.parametrize("form", ["fp32", "bf16x3", "f16x3"])
def test_full_period_closed_form(form):
    """Fisher entries of the full-period case: 4 k^2 N <t_i t_j>_A between odd tangents, zero
    with the even defocus term, N / F^2 for the flux and zero between flux and phase."""
    import oracle

    p = laplace_problem()
    _, out, labs = _gpu(p, form)
    H = out["fisher"]
    N = float(np.sum(oracle.forward(p)))
    k = 2 * np.pi / LAM
    A2 = p.transmission**2
    c = np.asarray([(i - 0.5 * (p.n_pupil - 1)) * p.diameter / p.n_pupil for i in range(p.n_pupil)])
    tan = {("pos", 0, 0): np.broadcast_to(c[None, :], A2.shape), ("pos", 0, 1): np.broadcast_to(c[:, None], A2.shape)}
    for j in range(p.n_zern):
        tan[("zern", j)] = p.basis[j]
    odd = lambda t: np.allclose(t, -t[::-1, ::-1], atol=1e-12 * np.max(np.abs(t)))  # noqa: E731
    want = np.zeros_like(H)
    for a, la in enumerate(labs):
        for b, lb in enumerate(labs):
            if la[0] == "flux" and lb[0] == "flux":
                want[a, b] = N / p.flux[0] ** 2
            elif la[0] != "flux" and lb[0] != "flux" and odd(tan[la]) and odd(tan[lb]):
                want[a, b] = 4 * k * k * N * np.sum(A2 * tan[la] * tan[lb]) / np.sum(A2)
    err = _rel(H, want)
    print(form, "full-period Fisher error", err)
    assert err < TOL[form]["info"]


@pytest.fixture(scope="module")
def aberrated():
    import oracle
    from oracle import laplace as OL

    p = aberrated_problem()
    data = np.random.default_rng(9).poisson(oracle.forward(p)).astype(np.int32)
    J, labs = OL.jacobian(p)
    ref = {k: OL.information(p, data if k != "fisher" else None, k)[0] for k in ("fisher", "gauss_newton", "hessian")}
    return p, data, J, ref, labs


@pytest.mark.parametrize("form", ["fp32", "bf16x3", "f16x3"])
def test_aberrated_against_oracle(aberrated, form):
    """Three stars, two wavelengths, two exposures (one dithered), a flat field and four Zernike
    terms including the tilts: J, the three curvature matrices and the marginal errors."""
    from oracle import laplace as OL

    p, data, Jref, ref, labs_ref = aberrated
    J, out, labs = _gpu(p, form, data, kinds=("fisher", "gauss_newton", "hessian"))
    assert labs == labs_ref
    ej = float(np.max(np.abs(J - Jref).max(axis=1) / np.abs(Jref).max(axis=1)))
    errs = {k: _rel(out[k], ref[k]) for k in out}
    # the tilts Z2, Z3 are degenerate with the mean position: marginal errors without them
    keep = [i for i, lab in enumerate(labs) if lab not in (("zern", 0), ("zern", 1))]
    es = {}
    for k in out:
        s_gpu = OL.sigma(out[k][np.ix_(keep, keep)])
        s_ref = OL.sigma(ref[k][np.ix_(keep, keep)])
        es[k] = float(np.max(np.abs(s_gpu / s_ref - 1)))
    print(form, "J", ej, "info", errs, "sigma", es)
    assert ej < TOL[form]["J"]
    assert errs["fisher"] < TOL[form]["info"] and errs["gauss_newton"] < TOL[form]["info"]
    assert errs["hessian"] < TOL[form]["hess"]
    assert es["fisher"] < 10 * TOL[form]["info"] and es["gauss_newton"] < 10 * TOL[form]["info"]
    assert es["hessian"] < 10 * TOL[form]["hess"]


def test_gram_kernel_against_numpy():
    """dlx_fisher_gram alone: ragged pixel count, both weightings, 128 parameters (the maximum)."""
    import torch

    import paper_2406_08703_gb300 as P

    rng = np.random.default_rng(2)
    for n, npix in ((1, 5), (7, 1000), (67, 33333), (128, 4099)):
        J = rng.standard_normal((n, npix)).astype(np.float32)
        m = rng.uniform(0.5, 50, npix).astype(np.float32)
        d = rng.poisson(m).astype(np.int32)
        Jt, mt, dt = (torch.as_tensor(a, device="cuda") for a in (J, m, d))
        for data, w in ((None, 1 / m.astype(np.float64)), (dt, d / m.astype(np.float64) ** 2)):
            F = P.dlx_fisher_gram(Jt, mt, data).cpu().numpy()
            ref = (J.astype(np.float64) * w) @ J.astype(np.float64).T
            assert np.array_equal(F, F.T)
            assert _rel(F, ref) < 1e-5, (n, npix)
        F1 = P.dlx_fisher_gram(Jt, mt).cpu().numpy()
        F2 = P.dlx_fisher_gram(Jt, mt).cpu().numpy()
        assert np.array_equal(F1, F2)


def test_vjp_matches_loss_gradient():
    """dlx_model_vjp with cot = 1 - d/m (dlx_nll_cotangent) is dlx_loss_grad's gradient without the
    prior (here none), bit for bit: the same kernels run on the same weights."""
    import torch

    import paper_2406_08703_gb300 as P

    p = aberrated_problem()
    data = np.random.default_rng(1).poisson(np.full((p.n_exp, p.n_det, p.n_det), 50.0)).astype(np.int32)
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.DLX_FP32_SIMT))
    prm = P.params_from_problem(p)
    dt = torch.as_tensor(data, device="cuda")
    _, g, _ = P.dlx_loss_grad(plan, prm, dt)
    m = P.dlx_forward(plan, prm)
    cot = P.dlx_nll_cotangent(m, dt)
    v = P.dlx_model_vjp(plan, prm, cot)
    torch.cuda.synchronize()
    for k in g:
        assert torch.equal(g[k], v[k]), k


def test_jvp_rejects_bad_alpha():
    import torch

    import paper_2406_08703_gb300 as P

    p = laplace_problem()
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.DLX_FP32_SIMT))
    prm = P.params_from_problem(p)
    t = torch.zeros((p.n_pupil, p.n_pupil), dtype=torch.float32, device="cuda")
    for a in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(P.DlxError):
            P.dlx_model_jvp(plan, prm, t, 1, a)


@pytest.mark.parametrize("form", ["bf16x3", "f16x3"])
def test_paper_full_size_sampled(form):
    """The paper's example (20 stars x 3 wavelengths x 5 images, 512^2 -> 1024^2, Noll 4-10): Jacobian
    entries at sampled pixels against the oracle's differences of direct sums, and properties of the
    Hessian that hold at any size (symmetric, positive definite at the truth, marginal errors no
    smaller than the conditional ones 1/sqrt(H_ii))."""
    import torch

    import oracle
    import paper_2406_08703_gb300 as P
    import workloads as W
    from oracle import laplace as OL
    from paper_2406_08703_gb300.laplace import Laplace

    p = W.make_problem("paper")
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.PRECISIONS[form]))
    prm = P.params_from_problem(p)
    lp = Laplace(plan)
    J = lp.jacobian(prm)
    rows = [lp.labels.index(lab) for lab in (("pos", 0, 0), ("pos", 7, 1), ("flux", 3), ("zern", 2))]
    rng = np.random.default_rng(5)
    for k in rows:
        lab = lp.labels[k]
        row = J[k].double().cpu().numpy()
        top = np.argsort(np.abs(row))[-4:]
        idx = np.concatenate([top, rng.integers(0, row.size, 4)])
        e_idx, q_idx = np.unravel_index(idx, (p.n_exp, p.n_det**2))
        ref = OL._richardson(lambda q: oracle.model_at(q, list(e_idx), list(q_idx)), p, lab)
        err = float(np.max(np.abs(row[idx] - ref)) / np.max(np.abs(ref)))
        print(form, lab, "sampled J error / row max", err)
        assert err < TOL[form]["J"]
    del J
    m = P.dlx_forward(plan, prm).cpu().numpy()
    dt = torch.as_tensor(W.poisson_counts(m, 17), device="cuda")
    H = lp.information(prm, dt, "hessian").cpu().numpy()
    assert np.max(np.abs(H - H.T)) <= 1e-12 * np.max(np.abs(H))
    res = OL.sigma(H)  # raises if H is singular
    assert np.all(np.linalg.eigvalsh(H / np.sqrt(np.outer(np.diag(H), np.diag(H)))) > 0)
    assert np.all(res >= (1 - 1e-9) / np.sqrt(np.diag(H)))


@pytest.mark.parametrize("form", ["fp32", "bf16x3", "f16x3"])
def test_integer_dither_windows_against_oracle(form):
    """The Laplace passes on a window plan (integer dithers, Sec. 3): the tangent forwards, the
    cotangent pass of the window NLL and the one-source plans of the same windows, against the
    oracle's per-exposure model with the same dithers as angles."""
    import oracle
    from oracle import laplace as OL

    p = aberrated_problem()
    k = np.array([(0, 0), (2, -1), (-1, 2)], dtype=np.float64)
    p.dither = k * p.pixscale
    data = np.random.default_rng(19).poisson(oracle.forward(p)).astype(np.int32)
    Jref, labs_ref = OL.jacobian(p)
    ref = {kd: OL.information(p, data if kd != "fisher" else None, kd)[0] for kd in ("fisher", "hessian")}
    J, out, labs = _gpu(p, form, data, kinds=("fisher", "hessian"), crop=True)
    assert labs == labs_ref
    ej = float(np.max(np.abs(J - Jref).max(axis=1) / np.abs(Jref).max(axis=1)))
    errs = {kd: _rel(out[kd], ref[kd]) for kd in out}
    print(form, "windows: J", ej, "info", errs)
    assert ej < TOL[form]["J"]
    assert errs["fisher"] < TOL[form]["info"]
    assert errs["hessian"] < TOL[form]["hess"]


def test_fresnel_regime_against_oracle():
    """The Laplace passes in the Fresnel regime (Sec. 1): the tangent phasors carry the pupil chirp
    through the same tilt tables; J and the Fisher matrix against the oracle's differences."""
    import oracle
    from oracle import laplace as OL

    p = aberrated_problem()
    # detector moved so the pupil chirp reaches about 3 rad at the edge: pi R^2 dz / (f^2 lambda)
    f = 1.0
    p.focal_length, p.focal_shift = f, 3.0 * LAM * f * f / (np.pi * (0.5 * p.diameter) ** 2)
    Jref, labs_ref = OL.jacobian(p)
    ref = OL.information(p, None, "fisher")[0]
    J, out, labs = _gpu(p, "fp32")
    ej = float(np.max(np.abs(J - Jref).max(axis=1) / np.abs(Jref).max(axis=1)))
    err = _rel(out["fisher"], ref)
    print("fresnel: J", ej, "fisher", err, "focal shift", p.focal_shift)
    assert labs == labs_ref
    assert ej < TOL["fp32"]["J"] and err < TOL["fp32"]["info"]
