"""The million-parameter calibration workload at full size on the GPU:
512^2 pupil, Noll 2-36 plus a 512^2 pixel OPD map, 16 wavelengths, 8 dithered
exposures, 1024^2 detector with oversample 2 (2048^2 fields), flat field with
1% dead pixels -- about 1.31 M parameters.

- the gradient against central finite differences of the GPU loss on 64 random
  parameters drawn from every group;
- 100 Adam steps through dlx_loss_grad + dlx_adam lower the loss.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def calib():
    import torch

    import paper_2406_08703_gb300 as P

    P.load()
    truth = W.make_problem("calib")
    plan = P.dlx_make_mft(P.desc_from_problem(truth, P.DLX_BF16X4))
    # data: Poisson counts of the GPU model at the truth (a GPU-only property test)
    m_true = P.dlx_forward(plan, P.params_from_problem(truth))
    torch.cuda.synchronize()
    data = W.poisson_counts(m_true.double().cpu().numpy(), 77)
    start = W.perturbed_start(truth, 78)
    start.coeff = 0.5 * truth.coeff
    start.opd_pix = 0.5 * truth.opd_pix
    start.flat = W.flat_field(truth.n_det, 0.01, 79)
    return P, plan, truth, start, torch.as_tensor(data, device="cuda")


def _loss(P, plan, prm, dt):
    import torch

    loss, _, _ = P.dlx_loss_grad(plan, prm, dt, grads={k: None for k in P.GRAD_KEYS})
    torch.cuda.synchronize()
    return float(loss.item())


def test_parameter_count(calib):
    P, plan, truth, start, dt = calib
    n = truth.n_zern + truth.n_pupil**2 + truth.n_det**2 + 3 * truth.n_src
    assert n == 35 + 262144 + 1048576 + 3  # about 1.31 M


def test_gradient_matches_central_differences_on_64_parameters(calib):
    """12 Zernike coefficients, 20 flat-field pixels, the flux, both position
    coordinates, and 29 random smooth directions in the pixel-OPD map.  A single
    pupil pixel moves the model by less than one FP32 ulp, so the pixel-OPD group
    is checked along directions (a 0.1 nm RMS map over the aperture) instead of
    one pixel at a time.  Steps keep the loss change far above the FP32 rounding
    of its per-pixel terms and the phase change below 1e-2 rad."""
    import torch

    P, plan, truth, start, dt = calib
    prm = P.params_from_problem(start)
    _, grads, _ = P.dlx_loss_grad(plan, prm, dt)
    torch.cuda.synchronize()
    g = {k: v.double().cpu().numpy() for k, v in grads.items()}
    rng = np.random.default_rng(5)
    counts = dt.sum(0).cpu().numpy().ravel()
    bright = np.argsort(counts)[-4096:]  # bright pixels carry the flat-field information
    picks = ([("zern_coeff", (int(j),), 2e-10) for j in rng.choice(start.n_zern, 12, replace=False)] +
             [("flat", tuple(int(x) for x in np.unravel_index(i, start.flat.shape)), 1e-2)
              for i in rng.choice(bright, 20, replace=False)] +
             [("flux", (0,), 1e-3 * float(start.flux[0])), ("pos", (0, 0), 2e-3 * start.pixscale),
              ("pos", (0, 1), 2e-3 * start.pixscale)])
    support = (start.transmission > 0).astype(np.float64)
    for i in range(29):
        v = W.smooth_gaussian_noise(start.n_pupil, 1.0, 8.0, 500 + i) * support
        v /= np.sqrt(np.mean(v[support > 0] ** 2))
        picks.append(("opd_pix", v, 1e-10))
    assert len(picks) == 64
    gkey = dict(zern_coeff="d_zern", opd_pix="d_opd_pix", flat="d_flat", flux="d_flux", pos="d_pos")
    bad = []
    for name, idx, h in picks:
        vals = []
        for sgn in (+1, -1):
            q = {k: (v.clone() if k == name else v) for k, v in prm.items()}
            if name == "opd_pix":
                q[name] += torch.as_tensor(sgn * h * idx, dtype=torch.float32, device="cuda")
            else:
                q[name][idx] += sgn * h
            vals.append(_loss(P, plan, q, dt))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(np.sum(g[gkey[name]] * idx)) if name == "opd_pix" else float(g[gkey[name]][idx])
        tol = 2e-2 if name == "flat" else 1e-2
        if not abs(fd - an) <= tol * max(abs(an), abs(fd)):
            bad.append((name, idx if name != "opd_pix" else "direction", an, fd))
    assert not bad, bad


def test_hundred_adam_steps_lower_the_loss(calib):
    import torch

    P, plan, truth, start, dt = calib
    prm = P.params_from_problem(start)
    lr = dict(zern_coeff=1e-9, opd_pix=2e-10, flat=5e-4, flux=1e5, pos=2e-8)
    gk = dict(zern_coeff="d_zern", opd_pix="d_opd_pix", flat="d_flat", flux="d_flux", pos="d_pos")
    state = {k: (torch.zeros_like(prm[k]), torch.zeros_like(prm[k])) for k in lr}
    losses = []
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grads = P.empty_grads(plan)
    for t in range(1, 101):
        P.dlx_loss_grad(plan, prm, dt, loss=loss, grads=grads)
        losses.append(loss.clone())
        for k, a in lr.items():
            P.dlx_adam(prm[k], grads[gk[k]], state[k][0], state[k][1], a, t)
    torch.cuda.synchronize()
    L = np.array([x.item() for x in losses])
    assert np.all(np.isfinite(L))
    assert P.dlx_plan_diagnostics(plan)["device_error"] == 0
    assert L[-1] < L[0]
    assert np.mean(L[-10:]) < np.mean(L[:10])
