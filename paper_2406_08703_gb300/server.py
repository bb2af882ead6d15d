"""Binding of the continuous-batching fit server (dlx_server_create / dlx_submit / dlx_poll).

Marshalling only: the scheduler, admission, grouped launches and CUDA graphs
live in the C library (csrc/server.cu).
"""

from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _native as N

_GROUPS = ("zern", "opd_pix", "flat", "flux", "pos")


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


class Server:
    """A fit server on one device.  Requests are workloads.Problem-like objects plus data."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, max_slots: int = 16):
        h = C.c_void_p()
        N.check(N.load().dlx_server_create(device, hbm_budget, max_slots, C.byref(h)), "dlx_server_create")
        self.handle = h
        self._keep = {}

    def close(self):
        if self.handle:
            N.check(N.load().dlx_server_destroy(self.handle), "dlx_server_destroy")
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, problem, data, n_steps: int = 10, lr: Optional[dict] = None, precision: int = N.DLX_F16X3,
               crop: bool = False, state: Optional[dict] = None) -> int:
        """crop=True serves whole-pixel dithers as windows of one larger detector per source.
        state = a poll result's {"adam_m", "adam_v", "adam_step"} (with the problem's parameters set to
        that result's) continues that fit exactly; None starts a fresh one."""
        p = problem
        lam = (C.c_double * len(p.lambdas))(*[float(x) for x in p.lambdas])
        dpx = None
        if crop:
            from . import integer_dithers

            k = integer_dithers(p)
            if k is None:
                raise ValueError("crop=True needs dithers of whole pixels")
            dpx = (C.c_int32 * (2 * len(k)))(*[int(v) for row in k for v in row])
        desc = N.MftDesc(p.n_pupil, p.diameter, p.n_det, p.pixscale, p.oversample, len(p.lambdas),
                         C.cast(lam, C.POINTER(C.c_double)), len(p.flux), len(p.dither), len(p.coeff), precision, 0, 0,
                         float(getattr(p, "prf_sigma", 0.0) or 0.0),
                         C.cast(dpx, C.POINTER(C.c_int32)) if dpx is not None else None,
                         float(getattr(p, "focal_length", 0.0) or 0.0), float(getattr(p, "focal_shift", 0.0) or 0.0))
        arrs = dict(transmission=_f32(p.transmission), opd_fixed=_f32(p.opd_fixed),
                    zern_basis=_f32(p.basis) if len(p.coeff) else None, weights=_f32(p.weights),
                    dither=_f32(p.dither), zern_coeff=_f32(p.coeff) if len(p.coeff) else None,
                    opd_pix=_f32(p.opd_pix), flux=_f32(p.flux), pos=_f32(p.pos), flat=_f32(p.flat),
                    data=np.ascontiguousarray(data, dtype=np.int32))
        req = N.Request()
        req.desc = desc
        for k, a in arrs.items():
            setattr(req, k, None if a is None else a.ctypes.data)
        req.n_steps = n_steps
        if state is not None:
            n = state_size(p)
            for k in ("adam_m", "adam_v"):
                a = _f32(state.get(k))
                if a is not None:
                    if a.size != n:
                        raise ValueError(f"{k} has {a.size} values, the packed parameters {n}")
                    arrs[k] = a
                    setattr(req, k, a.ctypes.data)
            req.adam_step = int(state.get("adam_step", 0))
        lr = lr or {}
        for i, g in enumerate(_GROUPS):
            req.lr[i] = float(lr.get(g, 0.0))
        t = C.c_uint64()
        N.check(N.load().dlx_submit(self.handle, C.byref(req), C.byref(t)), "dlx_submit")
        return t.value

    def poll(self, ticket: int, timeout_s: float = 0.0, shapes: Optional[dict] = None):
        """Returns None while pending, else a dict with the final parameters, gradient and timings
        (and the Adam state when `shapes` holds "adam_m" / "adam_v", see result_shapes(state=True))."""
        sh = shapes or {}
        out = {k: np.zeros(v, np.float32) for k, v in sh.items()}
        res = N.Result()
        for k in ("zern_coeff", "opd_pix", "flux", "pos", "flat", "g_zern", "g_opd_pix", "g_flux", "g_pos", "g_flat",
                  "adam_m", "adam_v"):
            setattr(res, k, out[k].ctypes.data if k in out else None)
        rc = N.load().dlx_poll(self.handle, ticket, timeout_s, C.byref(res))
        if rc == N.DLX_PENDING:
            return None
        N.check(rc, "dlx_poll")
        out.update(loss=res.loss, queued_s=res.queued_s, latency_s=res.latency_s, steps_done=res.steps_done,
                   adam_step=res.adam_step)
        return out

    def stats(self) -> dict:
        s = N.ServerStats()
        N.check(N.load().dlx_server_get_stats(self.handle, C.byref(s)), "dlx_server_get_stats")
        return {k: getattr(s, k) for k, _ in N.ServerStats._fields_}

    def inject_fault(self, kind: int):
        N.check(N.load().dlx_server_inject_fault(self.handle, kind), "dlx_server_inject_fault")


def state_size(problem) -> int:
    """Length of the packed Adam moments [zern_coeff | opd_pix (when fitted) | flat | flux | pos]."""
    p = problem
    ni = p.n_pupil * p.n_pupil if p.opd_pix is not None else 0
    return len(p.coeff) + ni + p.n_det * p.n_det + 3 * len(p.flux)


def result_shapes(problem, state: bool = False) -> dict:
    p = problem
    nz, ni, nd, ns = len(p.coeff), p.n_pupil, p.n_det, len(p.flux)
    sh = dict(zern_coeff=(max(nz, 1),), opd_pix=(ni, ni), flux=(ns,), pos=(ns, 2), flat=(nd, nd),
              g_zern=(max(nz, 1),), g_opd_pix=(ni, ni), g_flux=(ns,), g_pos=(ns, 2), g_flat=(nd, nd))
    if state:
        sh.update(adam_m=(state_size(p),), adam_v=(state_size(p),))
    return sh


def dlx_server_create(device: int = 0, hbm_budget: int = 0, max_slots: int = 16) -> Server:
    return Server(device, hbm_budget, max_slots)


def dlx_submit(server: Server, problem, data, n_steps: int = 10, lr: Optional[dict] = None,
               precision: int = N.DLX_F16X3) -> int:
    return server.submit(problem, data, n_steps, lr, precision)


def dlx_poll(server: Server, ticket: int, timeout_s: float = 0.0, shapes: Optional[dict] = None):
    return server.poll(ticket, timeout_s, shapes)
