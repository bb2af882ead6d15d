"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
compare with the FP64 oracle."""

import numpy as np

import oracle
import workloads as W

# Tolerances per arithmetic form: PSF max error relative to the peak, loss relative
# error, gradient relative L2 error per parameter group (`grad`) and the largest
# error of any gradient element relative to the group's largest element
# (`grad_max`).  Every split form and the FP32 form meet 1e-5 of the peak on the PSF.
# The hi part of every split keeps 8 significant bits, so its hi*hi products fit the
# tensor core's accumulator alignment window; TF32x3 and FP16x3 carry the next 11
# bits in lo (measured up to 7.1e-6 and 7.3e-6 of the peak, 1.6e-6 / 1.1e-6 on a
# coherent 512-long contraction, where full-width hi parts measured 1.9e-5 / 1.5e-5).
# Gradients (worst over the GPU parity cases, relative L2 / element of group max):
# FP32 2.3e-6 / 2.1e-6; FP16x3, TF32x3 and BF16x4 (round-to-nearest splits) up to
# 4.5e-5; BF16x3 up to 6.5e-4 / 7.0e-4: its stochastic split removes the coherent
# bias at the PSF peak but leaves a noise floor about four times the
# round-to-nearest split's, and gradients that weigh the faint PSF wings (flux and
# flat through 1 - d/m) see it.  BF16x3sa shares BF16x3's forward; its adjoint
# contracts the stochastically rounded hi parts alone, so its gradients carry
# zero-mean noise of about 2^-8 / sqrt(K) per contraction: up to 2.2e-3 / 4.1e-3.
# Plain BF16 is reported as measured and only bounded loosely here.
TOL = {
    "fp32": dict(psf=1e-5, loss=1e-6, grad=1e-5, grad_max=1e-5),
    "f16x3": dict(psf=1e-5, loss=1e-6, grad=1e-4, grad_max=1e-4),
    "tf32x3": dict(psf=1e-5, loss=1e-6, grad=1e-4, grad_max=1e-4),
    "bf16x4": dict(psf=1e-5, loss=1e-6, grad=1e-4, grad_max=1e-4),
    "bf16x3": dict(psf=1e-5, loss=1e-6, grad=1e-3, grad_max=1e-3),
    "bf16x3sa": dict(psf=1e-5, loss=1e-6, grad=3e-3, grad_max=6e-3),
    "bf16": dict(psf=1e-2, loss=1e-3, grad=5e-2, grad_max=5e-2),
}


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def fit_problem(name, seed=3, **over):
    """Truth, Poisson data from the oracle at the truth, and a perturbed start."""
    truth = W.make_problem(name, **over)
    data = W.poisson_counts(oracle.forward(truth), seed)
    start = W.perturbed_start(truth, seed + 1)
    if start.opd_pix is not None:
        start.opd_pix = 0.5 * truth.opd_pix
    start.coeff = 0.5 * truth.coeff
    start.flat = W.flat_field(truth.n_det, 0.02, seed + 2)
    return truth, data, start


def gpu_eval(problem, data, precision, psf_chunk=0, want_psf=True, crop=False):
    import torch

    import paper_2406_08703_gb300 as P

    plan = P.dlx_make_mft(P.desc_from_problem(problem, P.PRECISIONS[precision], psf_chunk=psf_chunk, crop=crop))
    prm = P.params_from_problem(problem)
    psf = P.dlx_psf(plan, prm) if want_psf else None
    model = P.dlx_forward(plan, prm)
    dt = torch.as_tensor(np.ascontiguousarray(data, dtype=np.int32), device="cuda")
    model_lg = torch.empty_like(model)
    loss, grads, _ = P.dlx_loss_grad(plan, prm, dt, model=model_lg)
    torch.cuda.synchronize()
    diag = P.dlx_plan_diagnostics(plan)
    f = lambda t: None if t is None else t.double().cpu().numpy()  # noqa: E731
    out = dict(psf=f(psf), model=f(model), model_lg=f(model_lg), loss=float(loss.item()),
               grads={k: f(v) for k, v in grads.items()}, diag=diag, info=plan.info)
    plan.close()
    return out


def oracle_eval(problem, data):
    ref = oracle.loss_grad(problem, data)
    _, psf = oracle.forward(problem, with_psf=True)
    ref["psf"] = psf
    return ref


def compare(out, ref, precision, groups=("coeff", "opd_pix", "flat", "flux", "pos")):
    """Returns a dict of the measured errors and asserts the tolerances."""
    tol = TOL[precision]
    err = {}
    if out["psf"] is not None:
        err["psf"] = float(np.max(np.abs(out["psf"] - ref["psf"])) / ref["psf"].max())
    err["model"] = float(np.max(np.abs(out["model"] - ref["model"])) / ref["model"].max())
    err["model_lg"] = float(np.max(np.abs(out["model_lg"] - out["model"])) / ref["model"].max())
    err["loss"] = abs(out["loss"] - ref["loss"]) / abs(ref["loss"])
    gmap = dict(coeff="d_zern", opd_pix="d_opd_pix", flat="d_flat", flux="d_flux", pos="d_pos")
    for g in groups:
        if ref[g].size:
            err[g] = rel_l2(out["grads"][gmap[g]], ref[g])
            top = float(np.max(np.abs(ref[g])))
            if top > 0:  # element by element: the largest error against the group's largest element
                err[g + "_max"] = float(np.max(np.abs(out["grads"][gmap[g]] - ref[g]))) / top
    print("compare", precision, err)
    assert out["diag"]["device_error"] == 0
    assert err.get("psf", 0) <= tol["psf"], err
    assert err["model"] <= tol["psf"], err
    assert err["model_lg"] == 0.0, err
    assert err["loss"] <= tol["loss"], err
    for g in groups:
        if g in err:
            assert err[g] <= tol["grad"], (g, err)
        if g + "_max" in err:
            assert err[g + "_max"] <= tol["grad_max"], (g, err)
    return err
