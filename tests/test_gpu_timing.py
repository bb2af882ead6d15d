"""GPU: the per-kernel-class timing of a plan (dlx_plan_set_timing / dlx_plan_get_timing), which
the benchmark's roofline reads: every launch is counted whether timing is on or not, only the
selected classes get events, and reading resets the accumulators."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_class_timing_counts_and_masks():
    import torch

    import paper_2406_08703_gb300 as P

    P.load()
    p = W.perturbed_start(W.make_problem("custom", seed=9, n_pupil=48, n_det=24, oversample=2, n_lambda=3, n_src=2,
                                         n_exp=1, n_zern_max=5), 10)
    data = torch.as_tensor(W.poisson_counts(np.full((1, 24, 24), 40.0), 11), device="cuda")
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.DLX_BF16X3))
    prm = P.params_from_problem(p)
    P.dlx_loss_grad(plan, prm, data)
    P.dlx_plan_get_timing(plan)  # the plan's set-up launches and the first evaluation

    # timing off: launches are counted, nothing is timed
    P.dlx_plan_set_timing(plan, False)
    for _ in range(2):
        P.dlx_loss_grad(plan, prm, data)
    off = P.dlx_plan_get_timing(plan)
    per_eval = off["total_launches"] / 2
    assert per_eval == int(per_eval) and per_eval >= 8
    assert all(v["events"] == 0 and v["ms"] == 0 for k, v in off.items() if isinstance(v, dict))
    assert off["stage1"]["launches"] == 2 and off["stage2_intensity"]["launches"] == 2

    # every class timed: each class that launched has one event pair per evaluation and time
    P.dlx_plan_set_timing(plan, True)
    for _ in range(3):
        P.dlx_loss_grad(plan, prm, data)
    on = P.dlx_plan_get_timing(plan)
    assert on["total_launches"] == 3 * per_eval
    for k, v in on.items():
        if isinstance(v, dict) and v["launches"] > 0:
            assert v["events"] >= 3 and v["ms"] > 0, k

    # one class: only it carries events
    P.dlx_plan_set_timing(plan, True, classes=["adjoint_stage2T"])
    P.dlx_loss_grad(plan, prm, data)
    one = P.dlx_plan_get_timing(plan)
    assert one["adjoint_stage2T"]["events"] == 1 and one["adjoint_stage2T"]["ms"] > 0
    assert all(v["events"] == 0 for k, v in one.items() if isinstance(v, dict) and k != "adjoint_stage2T")

    # reading reset everything
    again = P.dlx_plan_get_timing(plan)
    assert again["total_launches"] == 0
    torch.cuda.synchronize()
    plan.close()
