"""dlx_forward_noalloc against dlx_forward and the FP64 oracle.

dlx_forward_noalloc serves callers that cannot allocate device memory, such
as a host application that reserves all of the GPU's memory through its own
allocator at start-up and forbids further allocation while it runs.  It
computes the same model as dlx_forward (FP32 CUDA-core form) from the
library's fixed 16 MiB device scratch array.  These tests call it through the
C ABI twice in a row -- with different parameters, so the second call must not
depend on what the first left in the shared array -- and compare each output
with dlx_forward on a plan and with the oracle's model, element by element,
within the FP32 form's tolerance (1e-5 of the peak); they check that a call
after the first leaves the device's free memory unchanged, run a shape whose
working memory sits just under the 16 MiB limit, and see the next larger shape
refused.  The file sorts last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5  # max |difference| / peak, as for the FP32 form's parity tests
SCRATCH = 16 << 20
NORM_PARTS = 1024  # blocks of the pupil-power pass, one partial each
MAX_SRC = 32  # flux partials per reduction block


def _need_bytes(ni, nd, os_, nl, ns, ne, sm_count):
    """Working memory of one call, region by region as the entry point lays it out (each region
    starts on a 256-byte boundary; rows padded to 8 elements)."""
    no = nd * os_
    ldi, ldo = -(-ni // 8) * 8, -(-no // 8) * 8
    B, nse = nl * ns * ne, ns * ne
    red_blocks = max(1, min(-(-nd * nd // 256), 2 * sm_count))
    regions = [8 * nl, 4 * nl, 4 * nl, 8, 4 * NORM_PARTS, 16 * B * ni, 4 * ni * ni, 8 * nl * no * ldi,
               8 * nl * ni * ldo, 8 * B * ni * ldi, 8 * B * no * ldi, 4 * nse * no * no, 8 * red_blocks * (1 + MAX_SRC),
               8, 8 * NORM_PARTS, 4]
    off = 0
    for r in regions:
        off = -(-off // 256) * 256 + r
    return off


@pytest.fixture(scope="module")
def P():
    import torch

    import paper_2406_08703_gb300 as P

    assert torch.cuda.is_available()
    P.load()
    return P


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


def _noalloc(P, p):
    import torch

    prm = P.params_from_problem(p)
    desc = P.desc_from_problem(p, P.DLX_FP32_SIMT)
    out = torch.full((p.n_exp, p.n_det, p.n_det), float("nan"), device="cuda")
    P.dlx_forward_noalloc(desc, prm, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), prm, desc


def _err_of_peak(got, want):
    return float(np.max(np.abs(got - want)) / np.max(want))


def test_noalloc_forward_matches_planned_forward_and_oracle_twice(P):
    import torch

    for p in _problems():
        got, prm, desc = _noalloc(P, p)
        plan = P.dlx_make_mft(desc)
        ref = P.dlx_forward(plan, prm)
        torch.cuda.synchronize()
        want = ref.double().cpu().numpy()
        plan.close()
        assert np.all(np.isfinite(got))
        assert _err_of_peak(got, want) <= TOL
        assert _err_of_peak(got, oracle.forward(p)) <= TOL


def test_noalloc_many_sources_matches_planned_forward_and_oracle(P):
    """Twelve sources, past the eight that the one-pass binning holds in registers."""
    import torch

    p = W.perturbed_start(W.make_problem("custom", seed=31, n_pupil=32, n_det=24, oversample=2, n_lambda=2,
                                         n_src=12, n_exp=2, dither_px=0.5, n_zern_max=4), 32)
    want_oracle = oracle.forward(p)
    for _ in range(2):
        got, prm, desc = _noalloc(P, p)
        plan = P.dlx_make_mft(desc)
        ref = P.dlx_forward(plan, prm)
        torch.cuda.synchronize()
        want = ref.double().cpu().numpy()
        plan.close()
        assert _err_of_peak(got, want) <= TOL
        assert _err_of_peak(got, want_oracle) <= TOL


def test_noalloc_call_leaves_free_device_memory_unchanged(P):
    """After a first call (which loads the scratch array and the kernels it runs), a call of
    the same shape takes no device memory: the device's free memory is the same before and
    after it."""
    import torch

    p = _problems()[0]
    prm = P.params_from_problem(p)
    desc = P.desc_from_problem(p, P.DLX_FP32_SIMT)
    out = torch.empty((p.n_exp, p.n_det, p.n_det), device="cuda")
    P.dlx_forward_noalloc(desc, prm, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        P.dlx_forward_noalloc(desc, prm, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert _err_of_peak(out.double().cpu().numpy(), oracle.forward(p)) <= TOL


def test_noalloc_shape_just_under_the_scratch_limit(P):
    """A 64^2 pupil onto 128^2 samples with as many wavelengths as fit: working memory just under
    16 MiB runs and matches the oracle; one wavelength more is refused with DLX_ERR_RANGE."""
    import torch

    from paper_2406_08703_gb300._native import DlxError

    sm = torch.cuda.get_device_properties(0).multi_processor_count
    ni, nd, os_ = 64, 64, 2
    nl = max(L for L in range(1, 257) if _need_bytes(ni, nd, os_, L, 1, 1, sm) <= SCRATCH)
    assert nl < 256 and _need_bytes(ni, nd, os_, nl, 1, 1, sm) > SCRATCH - (256 << 10)
    p = W.make_problem("custom", seed=35, n_pupil=ni, n_det=nd, oversample=os_, n_lambda=nl, n_src=1,
                       n_zern_max=5, obscuration=0.2)
    p = W.perturbed_start(p, 36)
    got, _, _ = _noalloc(P, p)
    assert _err_of_peak(got, oracle.forward(p)) <= TOL
    q = W.make_problem("custom", seed=35, n_pupil=ni, n_det=nd, oversample=os_, n_lambda=nl + 1, n_src=1,
                       n_zern_max=5, obscuration=0.2)
    out = torch.empty((1, nd, nd), device="cuda")
    with pytest.raises(DlxError) as e:
        P.dlx_forward_noalloc(P.desc_from_problem(q, P.DLX_FP32_SIMT), P.params_from_problem(q), out)
    assert e.value.code == -6  # RANGE
    assert str(_need_bytes(ni, nd, os_, nl + 1, 1, 1, sm)) in str(e.value)


def test_noalloc_rejects_shapes_beyond_the_scratch(P):
    import torch

    from paper_2406_08703_gb300._native import DlxError

    big = W.make_problem("binary", n_lambda=4)
    prm = P.params_from_problem(big)
    desc = P.desc_from_problem(big, P.DLX_FP32_SIMT)
    out = torch.empty((1, big.n_det, big.n_det), device="cuda")
    with pytest.raises(DlxError) as e:
        P.dlx_forward_noalloc(desc, prm, out)
    assert e.value.code == -6  # RANGE
    assert "16 MiB" in str(e.value)
