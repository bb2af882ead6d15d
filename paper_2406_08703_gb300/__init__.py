"""GB300 (sm_103a) differentiable-optics hot path of arXiv:2406.08703.

Thin Python binding of the C ABI in include/dlx.h.  Every step of the path
(MFT matrices, OPD, phasor, the four MFT contractions, intensity, binning,
flat field, Poisson NLL, gradient reductions, Adam) runs in the library's
CUDA kernels; this module only marshals torch tensors (device memory and
streams) into the ABI structs.  The functions carry the ABI's names.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

import numpy as np

from . import _native as N
from ._native import (DLX_BF16, DLX_BF16X3, DLX_BF16X3SA, DLX_BF16X4, DLX_F16X3, DLX_FP32_SIMT, DLX_TF32X3,  # noqa: F401
                      PRECISIONS, DlxError)

PARAM_KEYS = ("transmission", "opd_fixed", "zern_basis", "zern_coeff", "opd_pix", "weights", "flux", "pos", "dither",
              "flat")
GRAD_KEYS = ("d_zern", "d_opd_pix", "d_flat", "d_flux", "d_pos")


def _torch():
    import torch

    return torch


def load():
    """Load (building if needed) the CUDA library; raises if it is unavailable."""
    return N.load()


@dataclasses.dataclass
class MftDesc:
    n_pupil: int
    diameter_m: float
    n_det: int
    pixscale_rad: float
    oversample: int
    lambdas: Sequence[float]
    n_src: int
    n_exp: int = 1
    n_zern: int = 0
    precision: int = DLX_F16X3
    psf_chunk: int = 0
    workspace_limit_bytes: int = 0
    prf_prior_sigma: float = 0.0
    # integer-pixel dithers [n_exp][2] (x, y): one MFT per source on a larger detector, images
    # as windows of it (Sec. 3); None = dithers are the params' angles
    dither_px: Optional[Sequence] = None
    # Fresnel regime: lens focal length and detector offset from focus (metres); 0, 0 = Fraunhofer
    focal_length_m: float = 0.0
    focal_shift_m: float = 0.0

    def to_c(self):
        lam = (C.c_double * len(self.lambdas))(*[float(x) for x in self.lambdas])
        dpx = None
        if self.dither_px is not None:
            flat = [int(v) for row in self.dither_px for v in row]
            if len(flat) != 2 * self.n_exp:
                raise ValueError("dither_px needs n_exp (x, y) pairs")
            dpx = (C.c_int32 * len(flat))(*flat)
        d = N.MftDesc(self.n_pupil, self.diameter_m, self.n_det, self.pixscale_rad, self.oversample,
                      len(self.lambdas), C.cast(lam, C.POINTER(C.c_double)), self.n_src, self.n_exp, self.n_zern,
                      int(self.precision), self.psf_chunk, self.workspace_limit_bytes, float(self.prf_prior_sigma),
                      C.cast(dpx, C.POINTER(C.c_int32)) if dpx is not None else None, float(self.focal_length_m),
                      float(self.focal_shift_m))
        return d, (lam, dpx)


class Plan:
    """Owns a dlx_plan (MFT matrices + workspaces on one device)."""

    def __init__(self, handle: int, desc: MftDesc, device: int):
        self.handle = C.c_void_p(handle)
        self.desc = desc
        self.device = device
        self.info = dlx_plan_get_info(self)

    def close(self):
        if self.handle:
            N.check(load().dlx_destroy_plan(self.handle), "dlx_destroy_plan")
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def integer_dithers(p) -> Optional[list]:
    """The problem's dithers in whole pixels [(x, y), ...] when every one moves the image by an
    integer number of pixels (to 1e-6 of a pixel), else None.  A pointing offset theta moves the
    image by theta / pixscale pixels at focus and by theta z / (f pixscale) in the Fresnel regime."""
    step = p.pixscale
    f = float(getattr(p, "focal_length", 0.0) or 0.0)
    if f > 0:
        step *= f / (f + float(getattr(p, "focal_shift", 0.0) or 0.0))
    k = np.asarray(p.dither, dtype=np.float64) / step
    r = np.rint(k)
    return r.astype(int).tolist() if np.all(np.abs(k - r) <= 1e-6) else None


def desc_from_problem(p, precision=DLX_F16X3, crop: bool = False, **kw) -> MftDesc:
    """MftDesc of a workloads.Problem-like object (duck-typed).  crop=True computes integer-pixel
    dithers as windows of one larger detector (raises if a dither is not a whole pixel)."""
    kw.setdefault("prf_prior_sigma", float(getattr(p, "prf_sigma", 0.0) or 0.0))
    kw.setdefault("focal_length_m", float(getattr(p, "focal_length", 0.0) or 0.0))
    kw.setdefault("focal_shift_m", float(getattr(p, "focal_shift", 0.0) or 0.0))
    if crop:
        dpx = integer_dithers(p)
        if dpx is None:
            raise ValueError("crop=True needs dithers of whole pixels")
        kw.setdefault("dither_px", dpx)
    return MftDesc(n_pupil=p.n_pupil, diameter_m=p.diameter, n_det=p.n_det, pixscale_rad=p.pixscale,
                   oversample=p.oversample, lambdas=list(p.lambdas), n_src=len(p.flux), n_exp=len(p.dither),
                   n_zern=len(p.coeff), precision=precision, **kw)


def params_from_problem(p, device="cuda") -> dict:
    """float32 device tensors of a workloads.Problem-like object's arrays."""
    torch = _torch()

    def t(a):
        return None if a is None else torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)

    out = {k: t(getattr(p, k)) for k in ("transmission", "opd_fixed", "opd_pix", "weights", "flux", "pos", "dither",
                                         "flat")}
    out["zern_basis"] = t(p.basis) if len(p.coeff) else None
    out["zern_coeff"] = t(p.coeff) if len(p.coeff) else None
    return out


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_tensor(name, t, shape, dtype, device):
    torch = _torch()
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous {dtype} CUDA tensor")
    if t.device.index != device:
        raise ValueError(f"{name}: tensor on cuda:{t.device.index}, plan on cuda:{device}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")


def _param_shapes(plan: Plan):
    i = plan.info
    ni, nd = i.n_pupil, i.n_det
    return dict(transmission=(ni, ni), opd_fixed=(ni, ni), zern_basis=(i.n_zern, ni, ni), zern_coeff=(i.n_zern,),
                opd_pix=(ni, ni), weights=(i.n_lambda,), flux=(i.n_src,), pos=(i.n_src, 2), dither=(i.n_exp, 2),
                flat=(nd, nd))


def _params_c(plan: Plan, params: dict):
    torch = _torch()
    shapes = _param_shapes(plan)
    for k in PARAM_KEYS:
        _check_tensor(k, params.get(k), shapes[k], torch.float32, plan.device)
    return N.Params(*[_ptr(params.get(k)) for k in PARAM_KEYS])


def _stream(plan: Plan, stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(plan.device)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ------------------------------------------------------------------ ABI-named calls

def dlx_make_mft(desc: MftDesc, device: int = 0) -> Plan:
    d, keep = desc.to_c()
    h = C.c_void_p()
    N.check(load().dlx_make_mft(C.byref(d), device, C.byref(h)), "dlx_make_mft")
    del keep
    return Plan(h.value, desc, device)


def dlx_destroy_plan(plan: Plan) -> None:
    plan.close()


def dlx_plan_get_info(plan: Plan):
    info = N.PlanInfo()
    N.check(load().dlx_plan_get_info(plan.handle, C.byref(info)), "dlx_plan_get_info")
    return info


def dlx_forward(plan: Plan, params: dict, model=None, stream=None):
    torch = _torch()
    i = plan.info
    if model is None:
        model = torch.empty((i.n_exp, i.n_det, i.n_det), dtype=torch.float32, device=f"cuda:{plan.device}")
    _check_tensor("model", model, (i.n_exp, i.n_det, i.n_det), torch.float32, plan.device)
    prm = _params_c(plan, params)
    N.check(load().dlx_forward(plan.handle, C.byref(prm), _ptr(model), _stream(plan, stream)), "dlx_forward")
    return model


def dlx_model_jvp(plan: Plan, params: dict, t_map, src_mask: int, alpha: float, jvp=None, work=None,
                  stream=None):
    """dm/dalpha of the model along the optical-path change t_map (metres,
    [Ni][Ni] float32 device tensor) of the sources in src_mask (bit s = source s)."""
    torch = _torch()
    i = plan.info
    shp = (i.n_exp, i.n_det, i.n_det)
    dev = f"cuda:{plan.device}"
    if jvp is None:
        jvp = torch.empty(shp, dtype=torch.float32, device=dev)
    if work is None:
        work = torch.empty(shp, dtype=torch.float32, device=dev)
    _check_tensor("t_map", t_map, (i.n_pupil, i.n_pupil), torch.float32, plan.device)
    _check_tensor("jvp", jvp, shp, torch.float32, plan.device)
    _check_tensor("work", work, shp, torch.float32, plan.device)
    prm = _params_c(plan, params)
    N.check(load().dlx_model_jvp(plan.handle, C.byref(prm), _ptr(t_map), C.c_uint32(src_mask & 0xffffffff),
                                 float(alpha), _ptr(jvp), _ptr(work), _stream(plan, stream)), "dlx_model_jvp")
    return jvp


def dlx_forward_noalloc(desc: MftDesc, params: dict, model, device: int = 0, stream=None):
    """dlx_forward in the FP32 form without a plan and without any device
    allocation (working memory from the library's fixed 16 MiB device array);
    for callers that cannot allocate.  `model` is the caller's output buffer."""
    torch = _torch()
    i = dict(n_pupil=desc.n_pupil, n_det=desc.n_det, n_zern=desc.n_zern, n_lambda=len(desc.lambdas),
             n_src=desc.n_src, n_exp=desc.n_exp)
    shapes = dict(transmission=(i["n_pupil"],) * 2, opd_fixed=(i["n_pupil"],) * 2,
                  zern_basis=(i["n_zern"], i["n_pupil"], i["n_pupil"]), zern_coeff=(i["n_zern"],),
                  opd_pix=(i["n_pupil"],) * 2, weights=(i["n_lambda"],), flux=(i["n_src"],), pos=(i["n_src"], 2),
                  dither=(i["n_exp"], 2), flat=(i["n_det"],) * 2)
    for k in PARAM_KEYS:
        _check_tensor(k, params.get(k), shapes[k], torch.float32, device)
    _check_tensor("model", model, (i["n_exp"], i["n_det"], i["n_det"]), torch.float32, device)
    prm = N.Params(*[_ptr(params.get(k)) for k in PARAM_KEYS])
    d, keep = desc.to_c()
    st = torch.cuda.current_stream(device) if stream is None else stream
    with torch.cuda.device(device):
        N.check(load().dlx_forward_noalloc(C.byref(d), C.byref(prm), _ptr(model), C.c_void_p(st.cuda_stream)),
                "dlx_forward_noalloc")
    del keep
    return model


def dlx_psf(plan: Plan, params: dict, out=None, stream=None):
    torch = _torch()
    i = plan.info
    if out is None:
        out = torch.empty((i.n_exp, i.n_out, i.n_out), dtype=torch.float32, device=f"cuda:{plan.device}")
    _check_tensor("psf_os", out, (i.n_exp, i.n_out, i.n_out), torch.float32, plan.device)
    prm = _params_c(plan, params)
    N.check(load().dlx_psf(plan.handle, C.byref(prm), _ptr(out), _stream(plan, stream)), "dlx_psf")
    return out


def empty_grads(plan: Plan, which=GRAD_KEYS) -> dict:
    torch = _torch()
    i = plan.info
    shapes = dict(d_zern=(i.n_zern,), d_opd_pix=(i.n_pupil, i.n_pupil), d_flat=(i.n_det, i.n_det),
                  d_flux=(i.n_src,), d_pos=(i.n_src, 2))
    dev = f"cuda:{plan.device}"
    return {k: (torch.empty(shapes[k], dtype=torch.float32, device=dev) if k in which else None) for k in GRAD_KEYS}


def dlx_loss_grad(plan: Plan, params: dict, data, loss=None, grads: Optional[dict] = None, model=None, stream=None):
    """Returns (loss[1] float64 tensor, grads dict, model or None); asynchronous on the stream."""
    torch = _torch()
    i = plan.info
    _check_tensor("data", data, (i.n_exp, i.n_det, i.n_det), torch.int32, plan.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=f"cuda:{plan.device}")
    _check_tensor("loss", loss, (1,), torch.float64, plan.device)
    if grads is None:
        grads = empty_grads(plan)
    gshapes = dict(d_zern=(i.n_zern,), d_opd_pix=(i.n_pupil, i.n_pupil), d_flat=(i.n_det, i.n_det),
                   d_flux=(i.n_src,), d_pos=(i.n_src, 2))
    for k in GRAD_KEYS:
        _check_tensor(k, grads.get(k), gshapes[k], torch.float32, plan.device)
    if model is not None:
        _check_tensor("model", model, (i.n_exp, i.n_det, i.n_det), torch.float32, plan.device)
    prm = _params_c(plan, params)
    g = N.Grads(*[_ptr(grads.get(k)) for k in GRAD_KEYS])
    N.check(load().dlx_loss_grad(plan.handle, C.byref(prm), _ptr(data), _ptr(loss), C.byref(g), _ptr(model),
                                 _stream(plan, stream)), "dlx_loss_grad")
    return loss, grads, model


def _grads_c(plan: Plan, grads: dict):
    torch = _torch()
    i = plan.info
    gshapes = dict(d_zern=(i.n_zern,), d_opd_pix=(i.n_pupil, i.n_pupil), d_flat=(i.n_det, i.n_det),
                   d_flux=(i.n_src,), d_pos=(i.n_src, 2))
    for k in GRAD_KEYS:
        _check_tensor(k, grads.get(k), gshapes[k], torch.float32, plan.device)
    return N.Grads(*[_ptr(grads.get(k)) for k in GRAD_KEYS])


def dlx_model_vjp(plan: Plan, params: dict, cot, grads: Optional[dict] = None, stream=None) -> dict:
    """grads = J^T cot: the gradient of sum_p cot[p] m[p] (cot float32 [n_exp][Nd][Nd])."""
    torch = _torch()
    i = plan.info
    _check_tensor("cot", cot, (i.n_exp, i.n_det, i.n_det), torch.float32, plan.device)
    if grads is None:
        grads = empty_grads(plan)
    g = _grads_c(plan, grads)
    prm = _params_c(plan, params)
    N.check(load().dlx_model_vjp(plan.handle, C.byref(prm), _ptr(cot), C.byref(g), _stream(plan, stream)),
            "dlx_model_vjp")
    return grads


def dlx_model_vjp_jvp(plan: Plan, params: dict, cot, t_map, src_mask: int, alpha: float,
                      grads: Optional[dict] = None, work: Optional[dict] = None, stream=None) -> dict:
    """d/dalpha of J^T cot along the phasor tangent t_map of the sources in src_mask, cot fixed."""
    torch = _torch()
    i = plan.info
    _check_tensor("cot", cot, (i.n_exp, i.n_det, i.n_det), torch.float32, plan.device)
    _check_tensor("t_map", t_map, (i.n_pupil, i.n_pupil), torch.float32, plan.device)
    if grads is None:
        grads = empty_grads(plan)
    if work is None:
        work = empty_grads(plan, [k for k in GRAD_KEYS if grads.get(k) is not None])
    g, w = _grads_c(plan, grads), _grads_c(plan, work)
    prm = _params_c(plan, params)
    N.check(load().dlx_model_vjp_jvp(plan.handle, C.byref(prm), _ptr(cot), _ptr(t_map),
                                     C.c_uint32(src_mask & 0xffffffff), float(alpha), C.byref(g), C.byref(w),
                                     _stream(plan, stream)), "dlx_model_vjp_jvp")
    return grads


def dlx_nll_cotangent(model, data, cot=None, stream=None):
    """cot = 1 - d / max(m, 1e-30): the Poisson NLL's dL/dm (model float32, data int32, same size)."""
    torch = _torch()
    if model.numel() != data.numel():
        raise ValueError("model and data differ in size")
    dev = model.device.index
    _check_tensor("model", model, tuple(model.shape), torch.float32, dev)
    _check_tensor("data", data, tuple(model.shape), torch.int32, dev)
    if cot is None:
        cot = torch.empty_like(model)
    _check_tensor("cot", cot, tuple(model.shape), torch.float32, dev)
    st = torch.cuda.current_stream(dev) if stream is None else stream
    N.check(load().dlx_nll_cotangent(_ptr(model), _ptr(data), int(model.numel()), _ptr(cot),
                                     C.c_void_p(st.cuda_stream if hasattr(st, "cuda_stream") else int(st))),
            "dlx_nll_cotangent")
    return cot


GRAM_MAX_PAR = 128
GRAM_BLOCKS = 256


def dlx_fisher_gram(J, model, data=None, F=None, work=None, stream=None):
    """F = J diag(w) J^T with w = 1/m (data None) or d/m^2; J float32 [n_par][n_pix] on the device,
    model float32 and data int32 of n_pix elements.  Returns F (float64 [n_par][n_par])."""
    torch = _torch()
    if J.dim() != 2 or not J.is_cuda or J.dtype != torch.float32 or not J.is_contiguous():
        raise TypeError("J: expected a contiguous 2-D float32 CUDA tensor")
    n, npix = J.shape
    dev = J.device.index
    if model.numel() != npix:
        raise ValueError(f"model has {model.numel()} elements, J rows have {npix}")
    _check_tensor("model", model, tuple(model.shape), torch.float32, dev)
    if data is not None:
        if data.numel() != npix:
            raise ValueError(f"data has {data.numel()} elements, J rows have {npix}")
        _check_tensor("data", data, tuple(data.shape), torch.int32, dev)
    if F is None:
        F = torch.empty((n, n), dtype=torch.float64, device=J.device)
    if work is None:
        work = torch.empty(GRAM_BLOCKS * n * (n + 1) // 2, dtype=torch.float64, device=J.device)
    _check_tensor("F", F, (n, n), torch.float64, dev)
    if work.dtype != torch.float64 or work.numel() < GRAM_BLOCKS * n * (n + 1) // 2:
        raise ValueError("work: float64 tensor of at least GRAM_BLOCKS * n (n + 1) / 2 elements")
    st = torch.cuda.current_stream(dev) if stream is None else stream
    N.check(load().dlx_fisher_gram(_ptr(J), int(n), int(npix), _ptr(model), _ptr(data), _ptr(F), _ptr(work),
                                   C.c_void_p(st.cuda_stream if hasattr(st, "cuda_stream") else int(st))),
            "dlx_fisher_gram")
    return F


def dlx_plan_diagnostics(plan: Plan):
    c = C.c_int64()
    e = C.c_int32()
    N.check(load().dlx_plan_diagnostics(plan.handle, C.byref(c), C.byref(e)), "dlx_plan_diagnostics")
    return dict(clamped=c.value, device_error=e.value)


def dlx_set_checks(level: int) -> None:
    """Checked mode of the library (process-wide): 0 off, 1 argument checks before every launch,
    2 also a synchronising check after every kernel class."""
    N.check(load().dlx_set_checks(int(level)), "dlx_set_checks")


def dlx_get_checks() -> int:
    return int(load().dlx_get_checks())


def dlx_check_buffer(ptr: int, nbytes: int, device: int = 0) -> int:
    """Status of the checked mode's test of one device array (0 = OK); launches nothing."""
    return int(load().dlx_check_buffer(C.c_void_p(ptr), nbytes, device))


def dlx_plan_inject_fault(plan: Plan, kind: int = 1) -> None:
    """Test hook: the next tensor-core contraction's bounded wait expires (device error flag)."""
    N.check(load().dlx_plan_inject_fault(plan.handle, kind), "dlx_plan_inject_fault")


def dlx_plan_set_timing(plan: Plan, enable: bool = True, classes=None) -> None:
    """Times every kernel class (enable=True), none (False), or only the named ones."""
    if not enable:
        mask = 0
    elif classes is None:
        mask = -1
    else:
        names = list(dlx_plan_get_timing_names())
        mask = 0
        for c in classes:
            mask |= 1 << names.index(c)
    N.check(load().dlx_plan_set_timing(plan.handle, mask), "dlx_plan_set_timing")


KERNEL_CLASSES = ("mft_matrices", "prologue", "stage1", "stage2_intensity", "bin_nll", "loss", "adjoint_field",
                  "adjoint_stage2T", "adjoint_stage1T", "grad_reduce", "adam", "adjoint_field_scale")


def dlx_plan_get_timing_names():
    return KERNEL_CLASSES


def dlx_plan_get_timing(plan: Plan) -> dict:
    """{class: dict(ms, events, launches)} plus 'total_launches'; synchronous, resets."""
    t = N.KernelTimes()
    N.check(load().dlx_plan_get_timing(plan.handle, C.byref(t)), "dlx_plan_get_timing")
    out = {t.name[i].decode(): dict(ms=t.ms[i], events=t.events[i], launches=t.launches[i])
           for i in range(t.n_classes)}
    out["total_launches"] = t.total_launches
    return out


def dlx_adam(theta, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    torch = _torch()
    for name, x in (("theta", theta), ("grad", grad), ("m", m), ("v", v)):
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.numel() != theta.numel():
            raise TypeError(f"{name}: contiguous float32 CUDA tensor of theta's size expected")
    st = torch.cuda.current_stream(theta.device) if stream is None else stream
    N.check(load().dlx_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(), lr, beta1, beta2, eps, t,
                            C.c_void_p(st.cuda_stream)), "dlx_adam")


# ------------------------------------------------------------------ autograd

def _autograd_fn():
    torch = _torch()

    class DlxPSFLoss(torch.autograd.Function):
        """Poisson NLL of the optical model with the library's hand-written adjoint.

        forward(plan, data, fixed, zern_coeff, opd_pix, flat, flux, pos) -> loss (float64 scalar);
        `fixed` holds transmission, opd_fixed, zern_basis, weights and dither.  The gradient
        of every differentiable input is computed in the same dlx_loss_grad call.
        """

        @staticmethod
        def forward(ctx, plan, data, fixed, zern_coeff, opd_pix, flat, flux, pos):
            params = dict(fixed, zern_coeff=zern_coeff, opd_pix=opd_pix, flat=flat, flux=flux, pos=pos)
            which = ["d_flat", "d_flux", "d_pos"] + (["d_zern"] if zern_coeff is not None else []) + (
                ["d_opd_pix"] if opd_pix is not None else [])
            grads = empty_grads(plan, which)
            loss, grads, _ = dlx_loss_grad(plan, params, data, grads=grads)
            ctx.save_for_backward(*[grads[k] if grads[k] is not None else torch.empty(0) for k in
                                    ("d_zern", "d_opd_pix", "d_flat", "d_flux", "d_pos")])
            ctx.has = (zern_coeff is not None, opd_pix is not None)
            return loss[0]

        @staticmethod
        def backward(ctx, gout):
            dz, dpix, dflat, dflux, dpos = ctx.saved_tensors
            s = gout.to(torch.float32)
            return (None, None, None, s * dz if ctx.has[0] else None, s * dpix if ctx.has[1] else None, s * dflat,
                    s * dflux, s * dpos)

    return DlxPSFLoss


_DlxPSFLoss = None


def psf_loss(plan: Plan, data, fixed: dict, zern_coeff, opd_pix, flat, flux, pos):
    """Differentiable loss: torch.autograd.Function over dlx_loss_grad."""
    global _DlxPSFLoss
    if _DlxPSFLoss is None:
        _DlxPSFLoss = _autograd_fn()
    return _DlxPSFLoss.apply(plan, data, fixed, zern_coeff, opd_pix, flat, flux, pos)


from .server import Server, dlx_poll, dlx_server_create, dlx_submit  # noqa: E402,F401
