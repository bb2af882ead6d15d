"""GPU: the staged fit of Sec. 4 on a small problem whose data the oracle made at the truth."""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def test_staged_fit_freezes_groups_and_descends():
    import torch

    import paper_2406_08703_gb300 as P
    from paper_2406_08703_gb300.fit import paper_schedule, staged_fit

    truth = W.make_problem("custom", seed=71, n_pupil=48, n_det=32, oversample=2, n_lambda=2, n_src=4, n_exp=2,
                           dither_px=0.5, obscuration=0.2, grating=True, n_zern_max=6, flux_total=4e7)
    truth.prf_sigma = 0.05
    data = W.poisson_counts(oracle.forward(truth), 72)
    start = W.perturbed_start(truth, 73)
    plan = P.dlx_make_mft(P.desc_from_problem(start, P.DLX_BF16X3))
    prm = P.params_from_problem(start)
    dt = torch.as_tensor(data, device="cuda")
    lr = dict(zern=1e-9, flux=2e-3 * float(np.mean(truth.flux)), pos=0.05 * truth.pixscale, flat=2e-3)
    stages = paper_schedule(lr, epochs_psf=60, epochs_prf=20)
    flat0 = prm["flat"].clone()
    losses = staged_fit(plan, prm, dt, stages[:1])
    torch.cuda.synchronize()
    assert torch.equal(prm["flat"], flat0)  # frozen in the first stage
    pos1, flux1, coeff1 = prm["pos"].clone(), prm["flux"].clone(), prm["zern_coeff"].clone()
    losses2 = staged_fit(plan, prm, dt, stages[1:])
    torch.cuda.synchronize()
    assert torch.equal(prm["pos"], pos1) and torch.equal(prm["flux"], flux1)  # frozen in the second
    assert torch.equal(prm["zern_coeff"], coeff1)
    L = np.concatenate([losses.cpu().numpy(), losses2.cpu().numpy()])
    # the loss falls in each stage, and the oracle agrees on the final parameters
    assert L[59] < L[0] and L[-1] < L[60]
    fitted = start.copy()
    fitted.coeff = prm["zern_coeff"].double().cpu().numpy()
    fitted.flux = prm["flux"].double().cpu().numpy()
    fitted.pos = prm["pos"].double().cpu().numpy()
    fitted.flat = prm["flat"].double().cpu().numpy()
    assert oracle.loss(fitted, data) < oracle.loss(start, data)
    # positions move toward the truth
    e0 = np.abs(start.pos - truth.pos).mean()
    e1 = np.abs(fitted.pos - truth.pos).mean()
    print("loss", L[0], L[59], L[-1], "position error (px)", e0 / truth.pixscale, e1 / truth.pixscale)
    assert e1 < 0.5 * e0
    plan.close()
