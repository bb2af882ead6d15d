"""Benchmark: fwd+grad evaluations per second of the differentiable-optics model.

One step = one dlx_loss_grad over the whole model (every wavelength x source x
exposure PSF: phasor, two-sided MFT, intensity, binning, flat field, Poisson
NLL, and the full adjoint to the Zernike, pixel-OPD, flat-field, flux and
position gradients).  The default workload is the million-parameter
calibration: 512^2 pupil with Zernikes 2-36 and a 512^2 pixel OPD map, 16
wavelengths x 8 dithered exposures of one star = 128 PSFs onto a 2048^2
oversampled grid (1024^2 detector, oversample 2), synthetic seeded inputs.  The
binary-star fit (256^2 pupil, 32 wavelengths x 2 stars onto 1024^2) is timed
beside it under the key "binary".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form f16x3] [--impl reference]

Prints one JSON line (rank 0).  `value` is device-timed (CUDA events on the
launching stream, inputs resident); `e2e` times the same call with host inputs
copied in from pinned memory and the loss and gradients copied back.  The
reference arm (--impl reference) times the FP64 CPU oracle on this host's cores,
each step one bounded sample of the same workload (the whole evaluation where
it takes seconds, else one wavelength x exposure slice of it).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+grad PSF evals/s & tensor-pipe % at ≤1e-5 rel err; p50/p99 latency"
WORKLOADS = {
    "binary": "binary-star polychromatic fit: 256^2 pupil (0.2 D obstruction, 0/pi grating), 32 wavelengths "
              "530-640 nm x 2 stars, 256^2 detector oversample 4 (1024^2 MFT per PSF), fwd + full gradient",
    "tiny": "tiny: 64^2 unobstructed pupil, Noll 4-11, one wavelength (595 nm), one star, 64^2 detector "
            "oversample 4 (256^2 MFT), fwd + full gradient",
    "calib": "million-parameter calibration: 512^2 pupil, Noll 2-36 + 512^2 pixel OPD, 16 wavelengths x 8 "
             "dithered exposures, 1024^2 detector oversample 2 (2048^2 MFT per PSF), fwd + full gradient",
    "paper": "the paper's example (Sec. 3-4): 20 stars x 3 wavelengths x 5 integer-dithered images, 512^2 pupil "
             "(0.2 D obstruction, 0/pi grating), 1024^2 detector at 12 mas, Noll 4-10, chi^2 prior on the pixel "
             "response, fwd + full gradient",
}


def workload_name(w):
    return WORKLOADS.get(w, w)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--form", default="f16x3", choices=["f16x3", "bf16x3", "bf16x3sa", "bf16x4", "tf32x3", "bf16", "fp32"])
    ap.add_argument("--impl", default="dlx", choices=["dlx", "reference"])
    ap.add_argument("--workload", default=None,
                    help="workload of the main line (default calib) or of --fit / --laplace (default paper)")
    ap.add_argument("--lambdas", type=int, default=0,
                    help="use only this many of the workload's wavelengths (same per-PSF shapes; profiling captures)")
    ap.add_argument("--no-forms", action="store_true", help="skip the side-by-side FP32 / other-form lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-binary", action="store_true",
                    help="skip the binary-star workload timed beside the main one")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the short serving measurement added to the main line")
    ap.add_argument("--no-kernel-timing", action="store_true",
                    help="time the steps without the per-kernel-class events (no roofline line)")
    ap.add_argument("--serving", action="store_true",
                    help="the serving workload instead: mixed-size fit requests through dlx_submit/dlx_poll")
    ap.add_argument("--fit", action="store_true",
                    help="time the paper's staged fit instead (Sec. 4: 100 epochs with the pixel response frozen, "
                         "then 50 of the pixel response alone) on --workload (default paper)")
    ap.add_argument("--laplace", action="store_true",
                    help="time the Laplace-approximation errors instead (Sec. 4: the likelihood Hessian over "
                         "positions, fluxes and Zernikes, inverted) on --workload (default paper)")
    ap.add_argument("--crop", action="store_true",
                    help="main line: compute whole-pixel dithers as windows of one larger detector per source "
                         "(Sec. 3), as --fit and --laplace do by default")
    ap.add_argument("--no-crop", action="store_true",
                    help="--fit / --laplace: compute every image's PSFs, not windows of one larger detector per "
                         "source, even where the dithers are whole pixels")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--serving-shapes", type=int, default=6)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, local):
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist

    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


N_LAMBDAS = 0  # set from --lambdas
CROP = False  # set from --crop


def dither_windows(problem):
    """The whole-pixel dither steps of an in-focus problem, or None (the crop shapes of --crop)."""
    k = np.asarray(problem.dither, dtype=np.float64) / problem.pixscale
    r = np.rint(k)
    return r.astype(int) if problem.focal_length == 0 and np.all(np.abs(k - r) <= 1e-6) else None


def shapes(problem, crop):
    """PSFs per evaluation and MFT output samples per side (crop: one PSF per source and
    wavelength on a detector wide enough for every window)."""
    k = dither_windows(problem) if crop and problem.n_exp > 1 else None
    if k is None:
        return problem.n_psf, problem.n_det * problem.oversample
    return problem.n_lambda * problem.n_src, (problem.n_det + 2 * int(np.max(np.abs(k)))) * problem.oversample


def streams_past_l2(problem, crop):
    """True when a step streams more than 256 MB (twice the 129 MB L2): the phasors and the
    first-stage products of every PSF in the four-plane 16-bit split, 64-padded rows."""
    B, no = shapes(problem, crop)
    ldi = -(-problem.n_pupil // 64) * 64
    return B * 8 * (problem.n_pupil + no) * ldi > (256 << 20)


def workload_config(workload, problem, crop, world):
    """The `config` of both arms' JSON lines: the workload and its sizes, and the L2 policy."""
    B, no = shapes(problem, crop)
    big = streams_past_l2(problem, crop)
    return dict(workload=workload_name(workload), psfs_per_eval=B, pupil=problem.n_pupil, mft_out=no,
                parallelism=f"replicas x{world}" if world > 1 else "single",
                l2=("no flush: per-step working set > 129 MB L2" if big
                    else "256 MB write before every step (working set below the 129 MB L2)"))


def make_inputs(workload, seed_offset=0):
    """Seeded synthetic inputs: the workload's truth, a perturbed starting point and
    Poisson data of an analytic image with the workload's total flux."""
    import workloads as W

    truth = W.make_problem(workload, **({"n_lambda": N_LAMBDAS} if N_LAMBDAS else {}))
    start = W.perturbed_start(truth, 100 + seed_offset)
    total = float(np.sum(truth.flux)) * truth.n_exp
    pix = truth.pixscale
    centres = truth.pos / pix
    data = W.synthetic_counts((truth.n_exp, truth.n_det, truth.n_det), total, centres, 6.0, 200 + seed_offset)
    return truth, start, data


class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


CONTRACTIONS = ("stage1", "stage2_intensity", "adjoint_field", "adjoint_stage2T", "adjoint_stage1T")


def run_form(P, torch, workload, form, steps, warmup, device, timing=True):
    """Device-timed fwd+grad steps of one arithmetic form; returns a dict.

    With `timing`, a short pass with events around every kernel class first gives
    the per-class breakdown (`kt_all`, per step) and the dominant contraction; the
    timed steps then carry events around that class only (two event records per
    step), so the roofline's kernel time is measured inside the timed region
    without slowing the rest of it."""
    truth, start, data = make_inputs(workload)
    crop = CROP and start.n_exp > 1 and P.integer_dithers(start) is not None
    plan = P.dlx_make_mft(P.desc_from_problem(start, P.PRECISIONS[form], crop=crop), device=device)
    prm = P.params_from_problem(start, device=f"cuda:{device}")
    dt = torch.as_tensor(data, device=f"cuda:{device}")
    grads = P.empty_grads(plan)
    loss = torch.empty(1, dtype=torch.float64, device=f"cuda:{device}")
    model = torch.empty((start.n_exp, start.n_det, start.n_det), device=f"cuda:{device}")
    stream = torch.cuda.current_stream(device)
    for _ in range(warmup):
        P.dlx_loss_grad(plan, prm, dt, loss=loss, grads=grads, model=model, stream=stream)
    torch.cuda.synchronize(device)
    P.dlx_plan_get_timing(plan)  # reset counters
    kt_all, dom = None, None
    if timing:
        nb = max(3, steps // 4)
        P.dlx_plan_set_timing(plan, True)
        for _ in range(nb):
            P.dlx_loss_grad(plan, prm, dt, loss=loss, grads=grads, model=model, stream=stream)
        kt = P.dlx_plan_get_timing(plan)
        kt_all = {k: v["ms"] / nb for k, v in kt.items() if isinstance(v, dict) and v["ms"] > 0}
        dom = max((k for k in kt_all if k in CONTRACTIONS), key=lambda k: kt_all[k], default=None)
        P.dlx_plan_set_timing(plan, dom is not None, classes=[dom] if dom else None)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    # a step that streams less than twice the 129 MB L2 is preceded by a 256 MB write (outside its events)
    flush = (torch.empty(64 << 20, dtype=torch.float32, device=f"cuda:{device}")
             if not streams_past_l2(start, crop) else None)
    torch.cuda.synchronize(device)
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(stream)
        P.dlx_loss_grad(plan, prm, dt, loss=loss, grads=grads, model=model, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(device)
    times = np.array([a.elapsed_time(b) for a, b in ev])
    kt = P.dlx_plan_get_timing(plan)
    P.dlx_plan_set_timing(plan, False)
    diag = P.dlx_plan_diagnostics(plan)
    info = plan.info
    out = dict(form=form, ms=times, kt=kt, kt_all=kt_all, dom=dom, info=info, diag=diag, loss=float(loss.item()),
               l2_flush=flush is not None,
               plan=plan, prm=prm, start=start, data=data)
    return out


def e2e_run(P, torch, r, steps, device):
    """Same call through the public API with host inputs: every step copies its inputs from
    pinned host memory, evaluates, and reads its loss and gradients back to the host.  Steps
    are pipelined two deep on three streams, as a caller evaluating a stream of problems would
    run them: step i+1's upload and step i-1's read-back overlap step i's evaluation, and the
    host waits for each step's own read-back before it counts the step as done."""
    plan, data = r["plan"], r["data"]
    host = {k: (None if v is None else v.cpu().pin_memory()) for k, v in r["prm"].items()}
    hdata = torch.as_tensor(data).pin_memory()
    dev_name = f"cuda:{device}"
    up, comp, down = (torch.cuda.Stream(device) for _ in range(3))
    bufs = []
    for _ in range(2):
        grads = P.empty_grads(plan)
        bufs.append(dict(
            dev={k: (None if v is None else torch.empty_like(v)) for k, v in r["prm"].items()},
            ddata=torch.empty_like(hdata, device=dev_name), grads=grads,
            loss=torch.empty(1, dtype=torch.float64, device=dev_name),
            hgrads={k: (None if v is None else torch.empty(v.shape, dtype=v.dtype).pin_memory())
                    for k, v in grads.items()},
            hloss=torch.empty(1, dtype=torch.float64).pin_memory(),
            uploaded=torch.cuda.Event(), evaluated=torch.cuda.Event(), read=torch.cuda.Event(), used=False))
    h2d = sum(v.numel() * v.element_size() for v in host.values() if v is not None) + hdata.numel() * 4
    d2h = 8 + sum(v.numel() * v.element_size() for v in bufs[0]["hgrads"].values() if v is not None)

    def enqueue(i):
        b = bufs[i % 2]
        if b["used"]:  # the buffers of step i - 2: its evaluation read them, its read-back emptied them
            up.wait_event(b["evaluated"])
            comp.wait_event(b["read"])
        with torch.cuda.stream(up):
            for k, v in host.items():
                if v is not None:
                    b["dev"][k].copy_(v, non_blocking=True)
            b["ddata"].copy_(hdata, non_blocking=True)
            b["uploaded"].record(up)
        comp.wait_event(b["uploaded"])
        P.dlx_loss_grad(plan, b["dev"], b["ddata"], loss=b["loss"], grads=b["grads"], stream=comp)
        b["evaluated"].record(comp)
        down.wait_event(b["evaluated"])
        with torch.cuda.stream(down):
            b["hloss"].copy_(b["loss"], non_blocking=True)
            for k, v in b["grads"].items():
                if v is not None:
                    b["hgrads"][k].copy_(v, non_blocking=True)
            b["read"].record(down)
        b["used"] = True

    def run(n):
        enqueue(0)
        for i in range(n):
            if i + 1 < n:
                enqueue(i + 1)
            bufs[i % 2]["read"].synchronize()  # step i's loss and gradients are on the host

    run(3)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize(device)
    dt = (time.perf_counter() - t0) / steps
    return dict(s_per_step=dt, h2d=h2d, d2h=d2h)


GMAP = dict(coeff="d_zern", opd_pix="d_opd_pix", flat="d_flat", flux="d_flux", pos="d_pos")


def sample_parity(P, torch, sub, data, form, ref):
    """The GPU path against the oracle's result on the timed sample (the same inputs on both
    sides), element by element: model max error of the peak, loss relative error, and per
    gradient group the relative L2 error and the largest element error of the group's largest
    element."""
    plan = P.dlx_make_mft(P.desc_from_problem(sub, P.PRECISIONS[form]))
    prm = P.params_from_problem(sub)
    dt = torch.as_tensor(np.ascontiguousarray(data, dtype=np.int32), device="cuda")
    model = torch.empty((sub.n_exp, sub.n_det, sub.n_det), device="cuda")
    loss, g, _ = P.dlx_loss_grad(plan, prm, dt, model=model)
    torch.cuda.synchronize()
    m = model.double().cpu().numpy()
    worst, which, groups = 0.0, None, {}
    for k, gk in GMAP.items():
        if g.get(gk) is None or ref[k].size == 0 or not np.any(ref[k]):
            continue
        a, b = g[gk].double().cpu().numpy(), ref[k]
        e = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        groups[k] = dict(rel_l2=e, max_err_of_max=float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
        if e > worst:
            worst, which = e, k
    out = dict(form=form, model_max_err_of_peak=float(np.max(np.abs(m - ref["model"])) / np.max(ref["model"])),
               loss_rel_err=abs(loss.item() - ref["loss"]) / abs(ref["loss"]), grad_rel_l2_worst=worst,
               grad_worst_group=which, grads=groups, effective_precision=int(plan.info.precision))
    plan.close()
    return out


# a whole evaluation whose MFT work (forward and adjoint) is below this many complex multiply-adds
# takes seconds on the host's cores, and is the oracle's sample as it stands
ORACLE_WHOLE_CMAC = 5e10


def oracle_sample(workload):
    """The oracle's bounded sample of a workload and the share of the evaluation's PSFs it holds.
    The whole evaluation where its MFT work is below ORACLE_WHOLE_CMAC (tiny, binary: seconds on
    the host), else one (wavelength, exposure) slice -- the first wavelength and the first exposure
    with every source -- whose cost is that share of the evaluation's (every PSF costs the same;
    the binning and likelihood are a small part)."""
    truth, start, data = make_inputs(workload)
    ni, no = start.n_pupil, start.n_det * start.oversample
    cmac = 2.0 * start.n_psf * (no * ni * ni + no * no * ni)
    if cmac <= ORACLE_WHOLE_CMAC:
        return start, data, 1.0, f"the whole evaluation ({start.n_psf} PSFs)", start
    sub = start.copy()
    sub.lambdas, sub.weights = start.lambdas[:1], start.weights[:1]
    sub.dither = start.dither[:1]
    frac = 1.0 / (start.n_lambda * start.n_exp)
    desc = (f"one (wavelength, exposure) slice: the first of {start.n_lambda} wavelengths and the first of "
            f"{start.n_exp} exposures with all {start.n_src} source(s), {sub.n_psf} of {start.n_psf} PSFs at full "
            f"size; evals/s = {frac:.6f} / seconds per slice (extrapolated by the PSF count)")
    return sub, data[:1], frac, desc, start


def cpu_baseline(workload, budget_s=12.0, form=None):
    """The FP64 oracle as it stands, on this host's cores, on the bounded sample of the workload
    (oracle_sample), timed for about budget_s; the same sample once on one core.  With `form`, the
    GPU path is also compared with the oracle's result on that sample."""
    import oracle

    sub, data, frac, desc, _ = oracle_sample(workload)
    oracle.lib()
    cores = oracle.set_threads(0)  # one thread per host core
    ref = oracle.loss_grad(sub, data)  # warm (thread pool, page-in); kept for the parity check
    t0, n = time.perf_counter(), 0
    while True:
        oracle.loss_grad(sub, data)
        n += 1
        if (time.perf_counter() - t0 > budget_s and n >= 2) or n >= 20:
            break
    dt = (time.perf_counter() - t0) / n
    # the same sample once on one core
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.loss_grad(sub, data)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(0)
    parity = None
    if form is not None:
        import torch

        import paper_2406_08703_gb300 as P

        parity = sample_parity(P, torch, sub, data, form, ref)
    return dict(value=frac / dt, unit="evals/s", cores=cores, kind="oracle", parity_on_sample=parity,
                seconds_per_sample=dt, sample=f"{desc}; {n} timed runs of {dt:.2f} s",
                single_core=dict(value=frac / dt1, unit="evals/s", cores=1,
                                 sample=f"the same sample, 1 run, {dt1:.2f} s"))


SERVING_METRIC = "serving: fit requests (K Adam fwd+grad steps each) evals/s and p50/p99 request latency"


def serving_requests(n_req, n_shapes, seed=55):
    """Seeded fit requests of mixed sizes: pupil {128, 256, 512}, detector {64..512}, oversample {2, 4},
    wavelengths {1, 8, 32, 64}, 1-3 stars, drawn from a pool of `n_shapes` shapes; truths as in the tiny
    workload (Noll Zernikes, smoothed pixel OPD, flat field); data are Poisson counts of an analytic image."""
    import workloads as W

    shapes = W.serving_request_shapes(n_shapes, seed)
    base = {}
    rng = np.random.default_rng(seed + 1)
    out = []
    for i in range(n_req):
        k = int(rng.integers(len(shapes)))
        if k not in base:
            sh = shapes[k]
            base[k] = W.make_problem("custom", seed=seed + 10 + k, n_pupil=sh["n_pupil"], n_det=sh["n_det"],
                                     oversample=sh["oversample"], n_lambda=sh["n_lambda"], n_src=sh["n_src"],
                                     n_zern_max=8, opd_pix_rms=5e-9)
        truth = base[k]
        start = W.perturbed_start(truth, seed + 1000 + i)
        start.opd_pix = np.zeros_like(truth.opd_pix)
        data = W.synthetic_counts((truth.n_exp, truth.n_det, truth.n_det), float(np.sum(truth.flux)) * truth.n_exp,
                                  truth.pos / truth.pixscale, 4.0, seed + 2000 + i)
        out.append((k, start, data))
    return out


def serving_run(P, reqs, form, n_steps, rate=None, seed=0):
    """Submit every request (all at once, or at Poisson arrival times of `rate` per
    second) to a fresh server; returns per-request latencies and the evals/s."""
    import threading

    from paper_2406_08703_gb300.server import result_shapes

    lr = dict(zern=1e-9, opd_pix=1e-10, flat=1e-3, flux=1e3, pos=1e-8)
    srv = P.dlx_server_create(0, 0, 16)
    prec = P.PRECISIONS[form]
    # warm-up: one request per shape builds each bucket's plan and captures its graphs
    warm = {}
    for k, p, d in reqs:
        if k not in warm:
            warm[k] = srv.submit(p, d, n_steps=n_steps, lr=lr, precision=prec)
    for k, t in warm.items():
        srv.poll(t, 600.0)
    tickets = [None] * len(reqs)
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()

    def submitter():
        t_next = time.perf_counter()
        for i, (k, p, d) in enumerate(reqs):
            if rate:
                t_next += rng.exponential(1.0 / rate)
                dt = t_next - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            tickets[i] = srv.submit(p, d, n_steps=n_steps, lr=lr, precision=prec)

    th = threading.Thread(target=submitter)
    th.start()
    lat, done = [], set()
    while len(done) < len(reqs):
        for i, (k, p, d) in enumerate(reqs):
            if i in done or tickets[i] is None:
                continue
            r = srv.poll(tickets[i], 0.0)
            if r is not None:
                lat.append(r["latency_s"])
                done.add(i)
        time.sleep(0.0005)
    th.join()
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    evals = len(reqs) * max(1, n_steps)
    # algorithmic MFT work of the served evaluations (8 FLOP per complex MAC): forward stage 1 and
    # stage 2 and the adjoint's two stages per PSF, and the recomputed field in the forms whose
    # buckets do not keep stage 2's fields (all but the BF16 split forms)
    kept = form in ("bf16x3", "bf16x4", "f16x3")
    flop = 0.0
    for k, p, d in reqs:
        ni, no = p.n_pupil, p.n_det * p.oversample
        s1, s2 = 8.0 * no * ni * ni, 8.0 * no * no * ni
        flop += max(1, n_steps) * p.n_lambda * p.n_src * p.n_exp * (2 * s1 + (2 if kept else 3) * s2)
    return dict(evals_per_s=evals / wall, requests_per_s=len(reqs) / wall, wall_s=wall,
                tflops_algorithmic=flop / wall / 1e12,
                p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                grouped_launches=int(stats["grouped_launches"]), graph_launches=int(stats["graph_launches"]))


def serving_bench(args):
    import torch

    import paper_2406_08703_gb300 as P

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    P.load()
    n_steps = 10
    reqs = serving_requests(args.serving_requests, args.serving_shapes)
    sat = serving_run(P, reqs, args.form, n_steps)
    rates = {}
    for frac in (0.25, 0.5, 0.75, 0.9, 1.1):  # Poisson arrivals at fractions of the saturated capacity
        rates[str(frac)] = serving_run(P, reqs, args.form, n_steps, rate=frac * sat["requests_per_s"], seed=7)
    small = reqs[: max(4, len(reqs) // 4)]
    fp32 = serving_run(P, small, "fp32", n_steps)
    split_small = serving_run(P, small, args.form, n_steps)
    line = dict(metric=SERVING_METRIC, value=sat["evals_per_s"], unit="evals/s", n_gpus=1, steps=n_steps,
                warmup=1, ms_per_step=1e3 / sat["evals_per_s"], higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype=f"{args.form} split (fp32 accumulate)", data="synthetic",
                config=dict(workload=f"{len(reqs)} fit requests of {args.serving_shapes} mixed shapes (pupil 128-512, "
                                     "detector 64-512, oversample 2-4, 1-64 wavelengths, 1-3 stars), K=10 Adam "
                                     "steps each", form=args.form),
                saturated=sat, poisson_rates=rates,
                forms={"fp32": dict(fp32, requests=len(small)), args.form: dict(split_small, requests=len(small))})
    print(json.dumps(line), flush=True)


def use_crop(P, problem, args) -> bool:
    """Integer-pixel dithers become windows of one larger detector per source (Sec. 3) unless
    --no-crop is given."""
    return (not args.no_crop) and problem.n_exp > 1 and P.integer_dithers(problem) is not None


def dither_mode(crop, problem) -> str:
    if crop:
        return (f"{problem.n_exp} integer dithers as windows of one PSF per source and wavelength on a larger "
                "detector (Sec. 3)")
    return f"{problem.n_exp} exposures, each with its own PSFs"


FIT_METRIC = "staged fit (Sec. 4): wall-clock seconds for 150 epochs of loss + gradient + Adam"


def fit_bench(args):
    """The paper's optimisation at the paper's scale: 100 epochs of positions, fluxes and
    aberrations with the pixel response frozen, then 50 epochs of the pixel response
    alone, every epoch a full loss + gradient and an Adam update, all on the device.
    Data: Poisson counts of an analytic image (the oracle cannot make data at this
    size and no input comes from the CUDA path), so the time, not the recovery, is
    the result."""
    import torch

    import paper_2406_08703_gb300 as P
    from paper_2406_08703_gb300.fit import paper_schedule, staged_fit

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    P.load()
    import workloads as W

    wl = args.workload or "paper"
    truth = W.make_problem(wl)
    start = W.perturbed_start(truth, 81)
    data = W.synthetic_counts((start.n_exp, start.n_det, start.n_det), float(np.sum(truth.flux)) * start.n_exp,
                              truth.pos / truth.pixscale, 3.0, 82)
    crop = use_crop(P, start, args)
    plan = P.dlx_make_mft(P.desc_from_problem(start, P.PRECISIONS[args.form], crop=crop))
    prm = P.params_from_problem(start)
    dt = torch.as_tensor(data, device="cuda")
    lr = dict(zern=1e-9, flux=2e-3 * float(np.mean(truth.flux)), pos=0.05 * truth.pixscale, flat=2e-3)
    stages = paper_schedule(lr)
    warm = P.params_from_problem(start)
    staged_fit(plan, warm, dt, [(max(args.warmup, 3), lr)])  # warm-up on a copy
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    losses = staged_fit(plan, prm, dt, stages)
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    secs = a.elapsed_time(b) / 1e3
    L = losses.cpu().numpy()
    n = len(L)
    i = plan.info
    line = dict(metric=FIT_METRIC, value=secs, unit="s", n_gpus=1, steps=n, warmup=max(args.warmup, 3),
                ms_per_step=1e3 * secs / n, higher_is_better=False, scaling="weak", vs_baseline=None,
                dtype=DTYPES.get(args.form, args.form), data="synthetic",
                config=dict(workload=workload_name(wl), form=args.form, psfs_per_eval=i.n_psf, pupil=i.n_pupil,
                            mft_out=i.n_mft_out, dithers=dither_mode(crop, start), epochs=[s[0] for s in stages],
                            lr=lr,
                            l2="no flush: per-step working set > 129 MB L2"),
                evals_per_s=n / secs, loss_first=float(L[0]), loss_last_stage1=float(L[stages[0][0] - 1]),
                loss_last=float(L[-1]), clocks=clk,
                context="the paper reports ~6.5 min for its 150-epoch fit (~2.75 s per loss + gradient) on an "
                        "Apple M1 Max CPU")
    plan.close()
    print(json.dumps(line), flush=True)


LAPLACE_METRIC = ("Laplace errors (Sec. 4): wall-clock seconds for the likelihood Hessian over positions, fluxes "
                  "and Zernikes and its inverse")


def laplace_bench(args):
    """The paper's error estimate at the paper's scale: the Hessian of the Poisson likelihood over
    the 20 stars' positions and fluxes and the Zernike coefficients (pixel response fixed), and
    the marginal errors from its inverse; also the Fisher and Gauss-Newton matrices.  Each timed
    step is one full Laplace.errors() call, host inversion included.  Data: Poisson counts of the
    model at the truth (made on the device by the forward model, then drawn on the host), so the
    fit point is the truth."""
    import torch

    import paper_2406_08703_gb300 as P
    from paper_2406_08703_gb300.laplace import Laplace

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    P.load()
    import workloads as W

    wl = args.workload or "paper"
    truth = W.make_problem(wl)
    crop = use_crop(P, truth, args)
    plan = P.dlx_make_mft(P.desc_from_problem(truth, P.PRECISIONS[args.form], crop=crop))
    prm = P.params_from_problem(truth)
    m = P.dlx_forward(plan, prm).cpu().numpy()
    data = W.poisson_counts(m, 91)
    dt = torch.as_tensor(data, device="cuda")
    lp = Laplace(plan)
    out = {}
    for kind in ("fisher", "gauss_newton", "hessian"):
        for _ in range(max(args.warmup, 3) if kind == "hessian" else 1):
            lp.errors(prm, dt, kind)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = max(1, args.steps if kind == "hessian" else 1)
        for _ in range(n):
            res = lp.errors(prm, dt, kind)
        torch.cuda.synchronize()
        out[kind] = ((time.perf_counter() - t0) / n, res)
    clocks = Clocks(0)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    J = lp.jacobian(prm)
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_jac = a.elapsed_time(b) / 1e3
    secs, res = out["hessian"]
    i = plan.info
    ns = i.n_src
    # each star's expected counts over all images: F_s times the sum of its unit-flux model
    n_s = np.array([float(J[lp.labels.index(("flux", s))].double().sum()) for s in range(ns)]) * truth.flux
    del J
    # Sec. 5's photon-noise relations and its mean ratio of recovered to expected error:
    # sigma_F / F = 1 / sqrt(N), sigma_theta = (1/pi) sqrt(2 / N) lambda / D, sigma_zern = 1 / sqrt(N) rad RMS
    lam_c = float(np.sum(truth.weights * truth.lambdas) / np.sum(truth.weights))
    rel_flux = (res["sigma_flux"] / truth.flux) * np.sqrt(n_s)
    rel_pos = res["sigma_pos"] / ((1 / np.pi) * np.sqrt(2 / n_s)[:, None] * lam_c / truth.diameter)
    rel_zern = res["sigma_zern"] * (2 * np.pi / lam_c) * np.sqrt(n_s.sum())
    line = dict(metric=LAPLACE_METRIC, value=secs, unit="s", n_gpus=1, steps=max(1, args.steps),
                warmup=max(args.warmup, 3), ms_per_step=1e3 * secs, higher_is_better=False, scaling="weak",
                vs_baseline=None, dtype=DTYPES.get(args.form, args.form),
                data="synthetic", gpu_launches=None,
                config=dict(workload=workload_name(wl), form=args.form, psfs_per_eval=i.n_psf, pupil=i.n_pupil,
                            mft_out=i.n_mft_out, dithers=dither_mode(crop, truth), n_par=len(lp.labels),
                            n_src=ns, n_zern=i.n_zern),
                seconds=dict(hessian=secs, gauss_newton=out["gauss_newton"][0], fisher=out["fisher"][0],
                             jacobian_only=t_jac),
                sigma=dict(pos_mas_median=float(np.median(res["sigma_pos"]) * 206264.806e3),
                           flux_rel_median=float(np.median(res["sigma_flux"] / truth.flux)),
                           zern_nm=[float(x) * 1e9 for x in res["sigma_zern"]],
                           total_counts=float(n_s.sum())),
                sigma_relative=dict(flux=float(np.mean(rel_flux)), position=float(np.mean(rel_pos)),
                                    zernike=float(np.mean(rel_zern))),
                clocks=clk,
                context="the paper computes these errors (Hessian marginalised over positions, fluxes and "
                        "aberrations) without reporting a time")
    plan.close()
    print(json.dumps(line), flush=True)


def reference_arm(args, rank, world):
    """--impl reference: the FP64 CPU oracle timed on this host, rank 0 only.  Each step is one
    oracle run of the workload's bounded sample (oracle_sample); `ms_per_step` is that run's
    measured time, and `value` the evaluations per second it implies (the sample's share of the
    PSFs over the seconds per step)."""
    if rank != 0:
        return
    import oracle

    sub, data, frac, desc, start = oracle_sample(args.workload)
    oracle.lib()
    cores = oracle.set_threads(0)  # one thread per host core
    for _ in range(args.warmup):
        oracle.loss_grad(sub, data)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.loss_grad(sub, data)
    dt = (time.perf_counter() - t0) / args.steps
    value = frac / dt
    line = dict(impl="reference", metric=METRIC, value=value, unit="evals/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * dt, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=workload_config(args.workload, start, CROP, world),
                step=f"one oracle run of {desc}",
                cpu_baseline=dict(value=value, unit="evals/s", cores=cores, kind="oracle", sample=desc),
                e2e=dict(value=value, unit="evals/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# algorithmic FLOP per launch of each contraction class (8 per complex MAC), one launch per class per eval
def contraction_flop(B, ni, no):
    return {"stage1": 8.0 * B * no * ni * ni, "stage2_intensity": 8.0 * B * no * no * ni,
            "adjoint_field": 8.0 * B * no * no * ni, "adjoint_stage2T": 8.0 * B * ni * no * no,
            "adjoint_stage1T": 8.0 * B * ni * ni * no}


# DRAM bytes (read + written) per launch of a form's contractions, from ncu captures of this
# build on reduced cases of 16 PSFs (the calibration shapes with 2 of 16 wavelengths), scaled to a
# full launch by the PSF count, in which their traffic grows (every PSF's operands are distinct
# and the A(lambda) blocks are per wavelength); none for a kernel, form or workload without a
# capture of the current code
TRAFFIC_16 = {
    "f16x3": {"calib": {"stage1": 124.86e6, "stage2_intensity": 896.64e6, "adjoint_stage2T": 851.07e6,
                        "adjoint_stage1T": 183.38e6}},
    "bf16x3": {"calib": {"stage1": 131.90e6, "adjoint_stage2T": 892.43e6, "adjoint_stage1T": 198.76e6}},
}


def roofline(r, form, workload, clk, peaks):
    """Roofline of the dominant contraction of a run_form result: algorithmic FLOP per launch over
    its mean event-timed launch in the timed region, against the measured tensor peak that
    matches the clocks sampled during the run."""
    kt, dom, info = r["kt"], r["dom"], r["info"]
    classes = {k: v for k, v in kt.items() if isinstance(v, dict)}
    ni, no, B = info.n_pupil, info.n_mft_out, info.n_psf
    alg = contraction_flop(B, ni, no)
    if dom not in alg or classes[dom]["events"] <= 0:
        return None
    # tensor instructions per algorithmic product: forward contractions of BF16x4 take 4, its adjoint 3;
    # the FP16 form's mirror-paired contractions 1.5 (six real products per 16-wide step over the
    # paired axis, against eight FLOP per complex MAC over the full one, for axes whose halves are
    # multiples of 16 as at these workloads)
    adj = dom.startswith("adjoint")
    split = {"bf16x4": 3.0 if adj else 4.0, "bf16x3sa": 1.0 if adj else 3.0, "f16x3": 1.5, "bf16x3": 3.0,
             "tf32x3": 3.0, "bf16": 1.0, "fp32": 1.0}[form]
    nom_ratio = {"f16x3": 1.0, "bf16x4": 1.0, "bf16x3": 1.0, "bf16x3sa": 1.0, "bf16": 1.0, "tf32x3": 1.1 / 2.25}
    t16 = TRAFFIC_16.get(form, {}).get(workload, {}).get(dom) if not N_LAMBDAS else None
    traffic = t16 / 16 * B if t16 else None
    per_launch_ms = classes[dom]["ms"] / max(classes[dom]["events"], 1)
    achieved = alg[dom] / (per_launch_ms / 1e3) / 1e12
    if form == "fp32":
        peak = 152 * 128 * 2 * (clk["sm_mhz"] or 1920.0) * 1e6 / 1e12
        return dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                    traffic=None, kernel=dom, peak_source="152 SMs x 128 FP32 lanes x 2 x median SM clock")
    # the burst peak while the sampled clocks stayed at their maximum with no power cap (the
    # kernel ran as cuBLAS did for the burst figure), else the sustained one
    capped = ("sw_power_cap" in (clk.get("reasons") or []) or
              (clk.get("sm_mhz") or 0) < 0.97 * (clk.get("sm_max_mhz") or 0))
    key = "bf16_tflops_sustained" if capped else "bf16_tflops"
    if key in peaks:
        base, src, tag = peaks[key], f"MEASURED_PEAKS.json {key}", " (of measured)"
    else:
        base, src = (1700.0, "recipe fallback 1.7 PFLOP/s sustained") if capped else \
            (1900.0, "recipe fallback 1.9 PFLOP/s burst")
        tag = " (of fallback)"
    peak = base * nom_ratio[form]
    return dict(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                traffic=traffic, traffic_unit="bytes per launch", kernel=dom,
                executed_tflops=achieved * split, executed_frac=achieved * split / peak,
                peak_source=src + (" x nominal tf32/bf16 ratio 1.1/2.25" if form == "tf32x3" else "") + tag)


DTYPES = {"f16x3": "f16x3 split (fp32 accumulate)", "bf16x4": "bf16x4 split (fp32 accumulate)",
          "bf16x3sa": "bf16x3 stochastic split, bf16 stochastic adjoint (fp32 accumulate)",
          "bf16x3": "bf16x3 split (fp32 accumulate)", "tf32x3": "tf32x3 split (fp32 accumulate)",
          "bf16": "bf16 (fp32 accumulate)", "fp32": "f32"}


def main():
    global N_LAMBDAS, CROP
    args = parse()
    fit_like = args.fit or args.laplace
    if args.workload is None and not fit_like:
        args.workload = "calib"
    N_LAMBDAS = args.lambdas
    CROP = args.crop
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.serving:
        if rank == 0:
            serving_bench(args)
        return
    if args.fit:
        if rank == 0:
            fit_bench(args)
        return
    if args.laplace:
        if rank == 0:
            laplace_bench(args)
        return
    import torch

    import paper_2406_08703_gb300 as P

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    dist = init_dist(world, local)
    device = local if world > 1 else 0
    torch.cuda.set_device(device)
    P.load()
    peaks = measured_peaks()

    clocks = Clocks(device)
    barrier(dist)
    torch.cuda.synchronize(device)
    clocks.start()
    t_wall = time.perf_counter()
    r = run_form(P, torch, args.workload, args.form, args.steps, args.warmup, device,
                 timing=not args.no_kernel_timing)
    torch.cuda.synchronize(device)
    barrier(dist)
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = r["ms"]
    total_ms = max_over_ranks(dist, float(ms.sum()))
    info = r["info"]
    evals_per_s = world * args.steps / (total_ms / 1e3)
    ms_step = total_ms / args.steps
    B = info.n_psf
    crop = CROP and r["start"].n_exp > 1 and P.integer_dithers(r["start"]) is not None
    line = dict(metric=METRIC, value=evals_per_s, unit="evals/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype=DTYPES[args.form], data="synthetic",
                config=workload_config(args.workload, r["start"], crop, world),
                form=args.form, working_set_mb=round(info.workspace_bytes / 2**20),
                psf_evals_per_s=evals_per_s * B,
                latency_ms=dict(p50=float(np.percentile(ms, 50)), p99=float(np.percentile(ms, 99))),
                tflops_algorithmic=evals_per_s / world * info.flop_loss_grad / 1e12,
                gpu_launches=int(r["kt"]["total_launches"]), clocks=clk,
                roofline=roofline(r, args.form, args.workload, clk, peaks),
                kernels=({k: round(v, 4) for k, v in r["kt_all"].items()} if r["kt_all"] else {}),
                wall_s=wall, device_error=r["diag"]["device_error"])

    # e2e through the public API with host buffers
    e = e2e_run(P, torch, r, max(3, args.steps // 3), device)
    line["e2e"] = dict(value=world / max_over_ranks(dist, e["s_per_step"]), unit="evals/s",
                       h2d_bytes_per_step=e["h2d"], d2h_bytes_per_step=e["d2h"],
                       pipeline="two steps deep: upload, evaluation and read-back on their own streams")
    r["plan"].close()
    del r

    if not args.no_forms and rank == 0:
        forms = {}
        for f in ("fp32", "f16x3", "bf16x4", "bf16x3", "bf16x3sa", "tf32x3", "bf16"):
            if f == args.form:
                continue
            try:
                rf = run_form(P, torch, args.workload, f, max(5, args.steps // 3), 2, device, timing=False)
                forms[f] = dict(value=1e3 / float(rf["ms"].mean()), p50_ms=float(np.percentile(rf["ms"], 50)),
                                p99_ms=float(np.percentile(rf["ms"], 99)))
                rf["plan"].close()
                del rf
            except Exception as ex:  # report, do not hide
                forms[f] = dict(error=str(ex))
        line["forms"] = forms

    if not args.no_binary and args.workload != "binary" and rank == 0:
        # the binary-star fit (256^2 pupil, 32 wavelengths x 2 stars onto 1024^2), timed the same way
        clk_b = Clocks(device)
        clk_b.start()
        rb = run_form(P, torch, "binary", args.form, args.steps, args.warmup, device,
                      timing=not args.no_kernel_timing)
        cb = clk_b.stop()
        msb = rb["ms"]
        line["binary"] = dict(
            workload=workload_name("binary"), value=1e3 * len(msb) / float(msb.sum()), unit="evals/s",
            ms_per_step=float(msb.mean()), steps=len(msb),
            latency_ms=dict(p50=float(np.percentile(msb, 50)), p99=float(np.percentile(msb, 99))),
            roofline=roofline(rb, args.form, "binary", cb, peaks),
            kernels=({k: round(v, 4) for k, v in rb["kt_all"].items()} if rb["kt_all"] else {}), clocks=cb)
        rb["plan"].close()
        del rb

    if not args.no_serving and rank == 0:
        # the fit server on a short mixed-size request stream (the full sweep: --serving)
        reqs = serving_requests(60, args.serving_shapes)
        sat = serving_run(P, reqs, args.form, 10)
        poi = serving_run(P, reqs, args.form, 10, rate=0.75 * sat["requests_per_s"], seed=7)
        keep = ("evals_per_s", "requests_per_s", "p50_ms", "p99_ms", "tflops_algorithmic", "grouped_launches",
                "graph_launches")
        line["serving"] = dict(
            workload=f"60 fit requests of {args.serving_shapes} mixed shapes (pupil 128-512, detector 64-512, "
                     "oversample 2-4, 1-64 wavelengths, 1-3 stars), K=10 Adam steps each",
            saturated={k: sat[k] for k in keep}, poisson_075={k: poi[k] for k in keep})

    if not args.no_cpu and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, form=args.form)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
