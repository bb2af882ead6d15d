"""GPU: the library's checked mode and its bounded device waits.

- Level 1 rejects, before any launch, arrays that are host memory, misaligned, or too small
  for the plan's shapes (dlx_check_loss_grad_args and dlx_check_buffer launch nothing; the
  checked dlx_forward is given pinned host memory only, which the device could read anyway).
- A contraction whose operand copy is withheld (dlx_plan_inject_fault) ends after its bounded
  wait with the device error flag raised, nothing faults, and the next evaluation is bitwise
  the one before.
- Level 2 turns that expiry into the call's TIMEOUT status, naming the kernel class.
"""

import ctypes as C
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2406_08703_gb300 as P

    P.load()
    p = W.make_problem("custom", seed=21, n_pupil=48, n_det=24, oversample=2, n_lambda=2, n_src=2, n_exp=1,
                       n_zern_max=5)
    data = torch.as_tensor(W.poisson_counts(np.full((1, 24, 24), 40.0), 3), device="cuda")
    plan = P.dlx_make_mft(P.desc_from_problem(p, P.DLX_BF16X3))
    prm = P.params_from_problem(p)
    yield P, plan, prm, data
    P.dlx_set_checks(0)
    torch.cuda.synchronize()
    plan.close()


def _c_args(P, plan, prm, grads, over=None):
    from paper_2406_08703_gb300 import _native as N

    c = N.Params(*[P._ptr(prm.get(k)) for k in P.PARAM_KEYS])
    for k, v in (over or {}).items():
        setattr(c, k, v)
    g = N.Grads(*[P._ptr(grads.get(k)) for k in P.GRAD_KEYS])
    return c, g


def test_level1_rejects_bad_arrays_without_launching(env):
    import torch

    from paper_2406_08703_gb300 import _native as N

    P, plan, prm, data = env
    lib = N.load()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grads = P.empty_grads(plan)
    nd = plan.info.n_det

    def check(over=None, data_ptr=None, loss_ptr=None):
        c, g = _c_args(P, plan, prm, grads, over)
        rc = lib.dlx_check_loss_grad_args(plan.handle, C.byref(c), data_ptr or data.data_ptr(),
                                          loss_ptr or loss.data_ptr(), C.byref(g), None)
        return rc, lib.dlx_last_error().decode()

    assert check()[0] == 0
    # a flat field at the end of an allocation of its own (16 MiB, above the caching allocator's
    # shared-segment sizes): exactly Nd^2 floats pass, one fewer is reported
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    big = torch.empty(4 * 1024 * 1024, dtype=torch.float32, device="cuda")
    exact, short = big[-nd * nd:], big[-(nd * nd - 1):]
    assert check({"flat": exact.data_ptr()})[0] == 0
    rc, msg = check({"flat": short.data_ptr()})
    assert rc == -1 and "params.flat" in msg and "bytes needed" in msg, msg
    assert P.dlx_check_buffer(big.data_ptr(), big.numel() * 4) == 0
    assert P.dlx_check_buffer(big.data_ptr() + 4, big.numel() * 4) == -1
    # misaligned double, host memory (pinned and pageable), another device's memory is not faked
    rc, msg = check(loss_ptr=loss.data_ptr() + 4)
    assert rc == -1 and "loss" in msg and "aligned" in msg, msg
    pinned = torch.zeros(nd * nd, dtype=torch.float32).pin_memory()
    rc, msg = check({"flat": pinned.data_ptr()})
    assert rc == -1 and "params.flat" in msg and "host" in msg, msg
    pageable = np.zeros(nd * nd, dtype=np.int32)
    rc, msg = check(data_ptr=pageable.ctypes.data)
    assert rc == -1 and "data" in msg, msg
    # a missing required array
    rc, msg = check({"weights": None})
    assert rc == -1 and "weights" in msg, msg

    # the checked entry points refuse before launching (pinned host memory only: readable anyway)
    model = torch.empty((1, nd, nd), dtype=torch.float32, device="cuda")
    P.dlx_set_checks(1)
    try:
        assert P.dlx_get_checks() == 1
        c, g = _c_args(P, plan, prm, grads, {"flat": pinned.data_ptr()})
        rc = lib.dlx_forward(plan.handle, C.byref(c), P._ptr(model), None)
        assert rc == -1 and "params.flat" in lib.dlx_last_error().decode()
        rc = lib.dlx_loss_grad(plan.handle, C.byref(c), data.data_ptr(), loss.data_ptr(), C.byref(g), None, None)
        assert rc == -1
        # correct arrays pass the checks and give the unchecked result
        P.dlx_forward(plan, prm, model)
        torch.cuda.synchronize()
        m1 = model.clone()
    finally:
        P.dlx_set_checks(0)
    P.dlx_forward(plan, prm, model)
    torch.cuda.synchronize()
    assert torch.equal(model, m1)
    with pytest.raises(Exception):
        P.dlx_set_checks(3)


def test_withheld_copy_ends_in_the_bounded_wait(env):
    import torch

    P, plan, prm, data = env
    loss0, _, _ = P.dlx_loss_grad(plan, prm, data)
    torch.cuda.synchronize()
    L0 = loss0.item()
    assert P.dlx_plan_diagnostics(plan)["device_error"] == 0

    P.dlx_plan_inject_fault(plan, 1)
    t0 = time.perf_counter()
    P.dlx_loss_grad(plan, prm, data)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    err = P.dlx_plan_diagnostics(plan)["device_error"]
    assert err != 0 and 0.9 < dt < 30, (err, dt)

    # the plan and the context are intact: the next evaluation is bitwise the first
    loss1, _, _ = P.dlx_loss_grad(plan, prm, data)
    torch.cuda.synchronize()
    assert loss1.item() == L0
    assert P.dlx_plan_diagnostics(plan)["device_error"] == 0


def test_level2_reports_the_expired_wait_and_its_class(env):
    import torch

    P, plan, prm, data = env
    P.dlx_set_checks(2)
    try:
        loss0, _, _ = P.dlx_loss_grad(plan, prm, data)  # every class synchronised and checked
        torch.cuda.synchronize()
        L0 = loss0.item()
        P.dlx_plan_inject_fault(plan, 1)
        with pytest.raises(Exception, match=r"TIMEOUT.*stage1"):
            P.dlx_loss_grad(plan, prm, data)
        torch.cuda.synchronize()
        assert P.dlx_plan_diagnostics(plan)["device_error"] == 0  # reported by the status
        loss1, _, _ = P.dlx_loss_grad(plan, prm, data)
        torch.cuda.synchronize()
        assert loss1.item() == L0
    finally:
        P.dlx_set_checks(0)
    # the FP32 form has no such waits
    plan32 = P.dlx_make_mft(P.desc_from_problem(W.make_problem("custom", seed=21, n_pupil=48, n_det=24, oversample=2,
                                                                n_lambda=2, n_src=2, n_exp=1, n_zern_max=5),
                                                P.DLX_FP32_SIMT))
    with pytest.raises(Exception):
        P.dlx_plan_inject_fault(plan32, 1)
    plan32.close()
