"""dlx_forward_noalloc against dlx_forward.

dlx_forward_noalloc serves callers that cannot allocate device memory, such
as a host application that reserves all of the GPU's memory through its own
allocator at start-up and forbids further allocation while it runs.  It
computes the same model as dlx_forward (FP32 CUDA-core form) from the
library's fixed device scratch array.  This test calls it through the C ABI
twice in a row -- with different parameters, so the second call must not
depend on what the first left in the shared array -- and compares each output
with dlx_forward on a plan, within the FP32 form's tolerance (1e-5 of the
peak).  The file sorts last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5  # max |difference| / peak, as for the FP32 form's parity tests


def _problems():
    a = W.make_problem("custom", seed=21, n_pupil=64, n_det=48, oversample=3, n_lambda=3, n_src=2, n_exp=2,
                       dither_px=0.5, n_zern_max=6, opd_pix_rms=4e-9, obscuration=0.2, grating=True)
    a = W.perturbed_start(a, 22)
    a.coeff = 15e-9 * np.random.default_rng(23).standard_normal(a.n_zern)
    b = a.copy()
    b.pos = a.pos + 0.7 * a.pixscale
    b.flux = 1.3 * a.flux
    b.coeff = -a.coeff
    return a, b


def test_noalloc_forward_matches_planned_forward_twice():
    import torch

    import paper_2406_08703_gb300 as P

    assert torch.cuda.is_available()
    P.load()
    for p in _problems():
        prm = P.params_from_problem(p)
        desc = P.desc_from_problem(p, P.DLX_FP32_SIMT)
        out = torch.full((p.n_exp, p.n_det, p.n_det), float("nan"), device="cuda")
        P.dlx_forward_noalloc(desc, prm, out)
        plan = P.dlx_make_mft(desc)
        ref = P.dlx_forward(plan, prm)
        torch.cuda.synchronize()
        got, want = out.double().cpu().numpy(), ref.double().cpu().numpy()
        plan.close()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= TOL * want.max()


def test_noalloc_many_sources_matches_planned_forward():
    """Twelve sources, past the eight that the one-pass binning holds in registers."""
    import torch

    import paper_2406_08703_gb300 as P

    P.load()
    p = W.perturbed_start(W.make_problem("custom", seed=31, n_pupil=32, n_det=24, oversample=2, n_lambda=2,
                                         n_src=12, n_exp=2, dither_px=0.5, n_zern_max=4), 32)
    prm = P.params_from_problem(p)
    desc = P.desc_from_problem(p, P.DLX_FP32_SIMT)
    out = torch.full((p.n_exp, p.n_det, p.n_det), float("nan"), device="cuda")
    for _ in range(2):
        P.dlx_forward_noalloc(desc, prm, out)
        plan = P.dlx_make_mft(desc)
        ref = P.dlx_forward(plan, prm)
        torch.cuda.synchronize()
        got, want = out.double().cpu().numpy(), ref.double().cpu().numpy()
        plan.close()
        assert np.max(np.abs(got - want)) <= TOL * want.max()


def test_noalloc_rejects_shapes_beyond_the_scratch():
    import paper_2406_08703_gb300 as P
    from paper_2406_08703_gb300._native import DlxError

    P.load()
    big = W.make_problem("binary", n_lambda=4)
    prm = P.params_from_problem(big)
    desc = P.desc_from_problem(big, P.DLX_FP32_SIMT)
    import torch

    out = torch.empty((1, big.n_det, big.n_det), device="cuda")
    with pytest.raises(DlxError) as e:
        P.dlx_forward_noalloc(desc, prm, out)
    assert e.value.code == -6  # RANGE
    assert "16 MiB" in str(e.value)
