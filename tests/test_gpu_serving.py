"""GPU tests of the continuous-batching fit server: a request's result is the
same alone and in a mix of concurrent requests, it agrees with the direct
loss/gradient call and with a manual Adam loop, admission respects the HBM
budget, and host-side faults (admission refusal, a NaN input, a poll
deadline) come back as error statuses."""

import time

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

LR = dict(zern=2e-9, opd_pix=1e-9, flat=1e-3, flux=1e3, pos=1e-8)


@pytest.fixture(scope="module")
def P():
    import paper_2406_08703_gb300 as P

    P.load()
    return P


def _request(seed, **over):
    truth = W.make_problem("custom", seed=seed, **over)
    data = W.poisson_counts(oracle.forward(truth), seed + 1)
    start = W.perturbed_start(truth, seed + 2)
    return start, data


SHAPE_A = dict(n_pupil=64, n_det=32, oversample=2, n_lambda=3, n_src=2, n_zern_max=6, opd_pix_rms=3e-9)
SHAPE_B = dict(n_pupil=48, n_det=24, oversample=4, n_lambda=2, n_src=1, n_zern_max=4)


def _serve(P, reqs, n_steps=3, max_slots=8, budget=0, form="bf16x4", crop=False):
    from paper_2406_08703_gb300.server import result_shapes

    srv = P.dlx_server_create(0, budget, max_slots)
    tickets = [srv.submit(p, d, n_steps=n_steps, lr=LR, precision=P.PRECISIONS[form], crop=crop) for p, d in reqs]
    out = [srv.poll(t, timeout_s=120.0, shapes=result_shapes(p)) for t, (p, _) in zip(tickets, reqs)]
    stats = srv.stats()
    srv.close()
    return out, stats


@pytest.mark.parametrize("form", ["bf16x4", "f16x3"])
def test_same_result_alone_and_in_the_mix(P, form):
    a = _request(31, **SHAPE_A)
    alone, _ = _serve(P, [a], form=form)
    mix = [_request(40 + i, **SHAPE_A) for i in range(3)] + [_request(50, **SHAPE_B), _request(51, **SHAPE_B)]
    mixed, stats = _serve(P, mix[:2] + [a] + mix[2:], form=form)
    x, y = alone[0], mixed[2]
    assert stats["grouped_launches"] > 0  # same-shape requests shared launches
    assert x["loss"] == pytest.approx(y["loss"], rel=1e-9)
    for k in ("zern_coeff", "opd_pix", "flux", "pos", "flat", "g_zern", "g_flat", "g_pos"):
        assert rel_l2(y[k], x[k]) < 1e-6, k


@pytest.mark.parametrize("form_name", ["bf16x3", "f16x3"])
def test_mid_flight_admission_gives_the_solo_result(P, form_name):
    """Continuous batching: six same-shape requests with uneven step counts on a server with two
    slots, in the BF16x3 and FP16x3 forms.  As a request finishes, a queued one is admitted into the
    freed slot while the other slot's request is still stepping, and when the finished request sat
    below the last active slot, that slot's request (inputs, parameters, Adam state) is moved down
    into the freed one mid-fit.  Every request's loss, parameters and gradients equal its run alone
    (one slot, same K): the split's random bits follow the PSF's index inside its slot, and the
    reductions have a fixed order per slot, so only the stage-2 work split, which depends on the
    active-slot count, may reorder sums (within 1e-6)."""
    from paper_2406_08703_gb300.server import result_shapes

    ks = [2, 40, 9, 3, 7, 4]
    reqs = [_request(140 + i, **SHAPE_A) for i in range(len(ks))]
    form = P.PRECISIONS[form_name]
    keys = ("zern_coeff", "opd_pix", "flux", "pos", "flat", "g_zern", "g_opd_pix", "g_flat", "g_flux", "g_pos")

    def run(batch):
        srv = P.dlx_server_create(0, 0, 2)
        tickets = [srv.submit(p, d, n_steps=k, lr=LR, precision=form) for (p, d), k in batch]
        out = [srv.poll(t, timeout_s=120.0, shapes=result_shapes(p)) for t, ((p, _), _) in zip(tickets, batch)]
        stats = srv.stats()
        srv.close()
        return out, stats

    mixed, stats = run(list(zip(reqs, ks)))
    assert stats["completed"] == len(ks) and stats["grouped_launches"] > 0
    assert stats["midflight_admits"] >= 1, stats  # a slot was refilled next to a running fit
    assert stats["slot_moves"] >= 1, stats  # a running fit was moved down into a freed slot
    for i, (rq, k) in enumerate(zip(reqs, ks)):
        (alone,), _ = run([(rq, k)])
        y = mixed[i]
        assert y["steps_done"] == k and alone["steps_done"] == k
        assert y["loss"] == pytest.approx(alone["loss"], rel=1e-9), i
        for key in keys:
            assert rel_l2(y[key], alone[key]) < 1e-6, (i, key)


@pytest.mark.parametrize("form", ["bf16x4", "f16x3"])
def test_single_evaluation_matches_direct_call(P, form):
    import torch

    p, d = _request(60, **SHAPE_A)
    res, _ = _serve(P, [(p, d)], n_steps=0, form=form)
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.PRECISIONS[form]))
    loss, grads, _ = P.dlx_loss_grad(plan, P.params_from_problem(p), torch.as_tensor(d, device="cuda"))
    torch.cuda.synchronize()
    assert res[0]["loss"] == pytest.approx(loss.item(), rel=1e-9)
    assert rel_l2(res[0]["g_zern"], grads["d_zern"].cpu().numpy()) < 1e-6
    assert rel_l2(res[0]["g_flat"], grads["d_flat"].cpu().numpy()) < 1e-6
    assert res[0]["steps_done"] == 1


def _window_request(seed, n_src=3):
    """Whole-pixel dithers (the paper's windows, Sec. 3), small: three exposures."""
    truth = W.make_problem("custom", seed=seed, n_pupil=40, n_det=20, oversample=2, n_lambda=2, n_src=n_src, n_exp=3,
                           n_zern_max=5)
    truth.dither = np.array([(0, 0), (2, -1), (-1, 3)], dtype=np.float64) * truth.pixscale
    data = W.poisson_counts(oracle.forward(truth), seed + 1)
    return W.perturbed_start(truth, seed + 2), data


def test_windows_served_alone_in_the_mix_and_as_a_plan(P):
    """Integer-dither window requests: one evaluation equals the window plan's loss and gradient,
    and K Adam steps give the same result alone and among other window requests of its shape
    (slots of one bucket)."""
    import torch

    a = _window_request(110)
    one, _ = _serve(P, [a], n_steps=0, crop=True)
    plan = P.dlx_make_mft(P.desc_from_problem(a[0], P.DLX_BF16X4, crop=True))
    loss, grads, _ = P.dlx_loss_grad(plan, P.params_from_problem(a[0]), torch.as_tensor(a[1], device="cuda"))
    torch.cuda.synchronize()
    assert one[0]["loss"] == pytest.approx(loss.item(), rel=1e-9)
    for k, gk in (("g_zern", "d_zern"), ("g_flat", "d_flat"), ("g_flux", "d_flux"), ("g_pos", "d_pos")):
        assert rel_l2(one[0][k], grads[gk].cpu().numpy()) < 1e-6, k
    alone, _ = _serve(P, [a], n_steps=3, crop=True)
    others = [_window_request(120 + i) for i in range(2)]
    mixed, stats = _serve(P, [others[0], a, others[1]], n_steps=3, crop=True)
    assert stats["grouped_launches"] > 0
    x, y = alone[0], mixed[1]
    assert x["loss"] == pytest.approx(y["loss"], rel=1e-9)
    for k in ("zern_coeff", "flux", "pos", "flat", "g_zern", "g_flat", "g_pos"):
        assert rel_l2(y[k], x[k]) < 1e-6, k


def test_fresnel_request_matches_direct_call(P):
    """A request in the Fresnel regime (Sec. 1): focal length and focus offset key its bucket and
    reach its plan; one evaluation equals the direct call."""
    import torch

    p, d = _request(130, **SHAPE_B)
    p.focal_length, p.focal_shift = 1.2, 2e-4
    res, _ = _serve(P, [(p, d)], n_steps=0)
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.DLX_BF16X4))
    loss, grads, _ = P.dlx_loss_grad(plan, P.params_from_problem(p), torch.as_tensor(d, device="cuda"))
    torch.cuda.synchronize()
    assert res[0]["loss"] == pytest.approx(loss.item(), rel=1e-9)
    assert rel_l2(res[0]["g_zern"], grads["d_zern"].cpu().numpy()) < 1e-6
    q = p.copy()
    q.focal_length, q.focal_shift = 0.0, 0.0
    res0, _ = _serve(P, [(q, d)], n_steps=0)
    assert abs(res0[0]["loss"] - res[0]["loss"]) > 1e-6 * abs(res[0]["loss"])  # the defocus is not dropped


def test_adam_steps_match_manual_loop(P):
    import torch

    p, d = _request(70, **SHAPE_A)
    res, _ = _serve(P, [(p, d)], n_steps=4)
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.DLX_BF16X4))
    prm = P.params_from_problem(p)
    dt = torch.as_tensor(d, device="cuda")
    groups = [("zern_coeff", "d_zern", LR["zern"]), ("opd_pix", "d_opd_pix", LR["opd_pix"]),
              ("flat", "d_flat", LR["flat"]), ("flux", "d_flux", LR["flux"]), ("pos", "d_pos", LR["pos"])]
    state = {k: (torch.zeros_like(prm[k]), torch.zeros_like(prm[k])) for k, _, _ in groups}
    for t in range(1, 5):
        _, grads, _ = P.dlx_loss_grad(plan, prm, dt)
        for k, gk, lr in groups:
            P.dlx_adam(prm[k], grads[gk], state[k][0], state[k][1], lr, t)
    torch.cuda.synchronize()
    for k, _, _ in groups:
        assert rel_l2(res[0][k], prm[k].cpu().numpy()) < 1e-5, k


def test_resumed_request_continues_bitwise(P):
    """K1 steps, then K2 more from the returned parameters and Adam state, equal K1 + K2 in one request."""
    import dataclasses

    from paper_2406_08703_gb300.server import result_shapes, state_size

    p, d = _request(75, **SHAPE_A)
    sh = result_shapes(p, state=True)
    form = P.PRECISIONS["bf16x3"]

    def run(prob, k, state=None):
        srv = P.dlx_server_create(0, 0, 2)
        t = srv.submit(prob, d, n_steps=k, lr=LR, precision=form, state=state)
        r = srv.poll(t, timeout_s=120.0, shapes=sh)
        srv.close()
        return r

    whole = run(p, 6)
    first = run(p, 2)
    assert first["adam_step"] == 2 and whole["adam_step"] == 6
    n = state_size(p)
    assert first["adam_m"].shape == (n,) and np.count_nonzero(first["adam_v"]) > n // 4
    mid = dataclasses.replace(p, coeff=first["zern_coeff"][:len(p.coeff)].copy(), opd_pix=first["opd_pix"].copy(),
                              flux=first["flux"].copy(), pos=first["pos"].copy(), flat=first["flat"].copy())
    st = {k: first[k] for k in ("adam_m", "adam_v", "adam_step")}
    second = run(mid, 4, st)
    assert second["adam_step"] == 6 and second["steps_done"] == 4
    assert second["loss"] == whole["loss"]
    for k in ("zern_coeff", "opd_pix", "flux", "pos", "flat", "g_zern", "g_opd_pix", "g_flat", "g_pos", "adam_m",
              "adam_v"):
        assert np.array_equal(second[k], whole[k]), k
    # an evaluation (K = 0) takes no Adam step and hands the state back unchanged
    ev = run(mid, 0, st)
    assert ev["adam_step"] == 2
    assert np.array_equal(ev["adam_m"], first["adam_m"]) and np.array_equal(ev["adam_v"], first["adam_v"])
    srv = P.dlx_server_create(0, 0, 1)
    with pytest.raises(Exception):
        srv.submit(mid, d, n_steps=1, lr=LR, precision=form, state=dict(st, adam_step=-1))
    with pytest.raises(ValueError):
        srv.submit(mid, d, n_steps=1, lr=LR, precision=form, state=dict(st, adam_m=st["adam_m"][:-1]))
    srv.close()


def test_admission_respects_budget_and_all_complete(P):
    reqs = [_request(80 + i, **(SHAPE_A if i % 2 else SHAPE_B)) for i in range(6)]
    from paper_2406_08703_gb300.server import result_shapes

    budget = 1 << 30
    srv = P.dlx_server_create(0, budget, 2)
    tickets = [srv.submit(p, d, n_steps=5, lr=LR) for p, d in reqs]
    peak = 0
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < 120:
        s = srv.stats()
        peak = max(peak, s["hbm_in_use"])
        for t, (p, _) in zip(tickets, reqs):
            if t not in done:
                r = srv.poll(t, 0.0, result_shapes(p))
                if r is not None:
                    done[t] = r
        time.sleep(0.005)
    stats = srv.stats()
    srv.close()
    assert len(done) == len(tickets)
    assert peak <= budget
    assert stats["completed"] == len(tickets) and stats["rejected"] == 0
    assert all(np.isfinite(r["loss"]) for r in done.values())


def test_host_side_faults_return_status(P):
    from paper_2406_08703_gb300._native import DlxError

    p, d = _request(90, **SHAPE_B)
    srv = P.dlx_server_create(0, 0, 4)
    srv.inject_fault(1)  # next admission refused
    t = srv.submit(p, d, n_steps=1, lr=LR)
    with pytest.raises(DlxError) as e:
        srv.poll(t, 60.0)
    assert e.value.code == -2  # NOMEM
    srv.inject_fault(2)  # next admitted request gets a NaN input
    t = srv.submit(p, d, n_steps=1, lr=LR)
    with pytest.raises(DlxError) as e:
        srv.poll(t, 60.0)
    assert e.value.code == -4  # NONFINITE
    t = srv.submit(p, d, n_steps=200, lr=LR)
    with pytest.raises(DlxError) as e:
        srv.poll(t, 1e-3)
    assert e.value.code == -5  # TIMEOUT
    assert srv.poll(t, 120.0) is not None
    srv.close()


def test_request_larger_than_budget_is_rejected(P):
    from paper_2406_08703_gb300._native import DlxError

    p, d = _request(95, **SHAPE_A)
    srv = P.dlx_server_create(0, 1 << 20, 2)
    with pytest.raises(DlxError) as e:
        srv.submit(p, d, n_steps=1, lr=LR)
    assert e.value.code == -2
    srv.close()
