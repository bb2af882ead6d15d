"""GPU parity at the edges of the input space, against the FP64 oracle: the smallest shapes
(a 5^2 pupil, a one-pixel detector, odd grids far below one tile), no Zernike terms and no
pixel-OPD map, the largest source count a plan takes (32: two-pass binning and the split-plane
fold), data of zero counts, and a source of zero flux.  Below 32 pupil samples the BF16 split
forms run the FP16 split (their 17-bit operands missed 1e-5 of the PSF peak there: 1.0-3.2e-5)."""

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import compare, fit_problem, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu

FORMS = ["fp32", "f16x3", "bf16x4", "bf16x3", "bf16x3sa", "tf32x3"]

EDGES = {
    # one detector pixel (3 x 3 MFT samples), a 5^2 pupil, no Zernike terms, no pixel map
    "one_pixel": dict(n_pupil=5, n_det=1, oversample=3, n_lambda=1, n_src=1, n_exp=1, n_zern_max=0),
    # the unit sizes of the test plan: 5^2 -> 7^2 (no oversampling) and 17^2 -> 33^2
    "five_to_seven": dict(n_pupil=5, n_det=7, oversample=1, n_lambda=2, n_src=2, n_exp=1, n_zern_max=3),
    "seventeen_to_33": dict(n_pupil=17, n_det=11, oversample=3, n_lambda=1, n_src=1, n_exp=2, dither_px=0.5,
                            n_zern_max=5, opd_pix_rms=3e-9),
    # 32 sources, the most a plan takes
    "max_sources": dict(n_pupil=24, n_det=12, oversample=2, n_lambda=2, n_src=32, n_exp=1, n_zern_max=3),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import paper_2406_08703_gb300 as P

    P.load()


@pytest.mark.parametrize("name", list(EDGES))
@pytest.mark.parametrize("form", FORMS)
def test_edge_shapes(name, form):
    import paper_2406_08703_gb300 as P

    _, data, start = fit_problem("custom", seed=60 + len(name), **EDGES[name])
    out = gpu_eval(start, data, form)
    assert out["info"].n_zern == len(start.coeff)
    if form in ("bf16x3", "bf16x4", "bf16x3sa") and start.n_pupil < 32:
        # a 16-bit split does not average its representation error down over so few pupil
        # samples: such plans run the 22-bit FP16 split, and say so
        assert out["info"].precision == P.DLX_F16X3
    else:
        assert out["info"].precision == P.PRECISIONS[form]
    err = compare(out, oracle_eval(start, data), form)
    print(name, form, err)


@pytest.mark.parametrize("form", ["fp32", "bf16x3"])
def test_zero_counts_and_a_dark_source(form):
    """Data of zero counts everywhere (the loss is the model's sum, dL/dm = 1) and one of three
    sources at zero flux (its position gradient is zero, its flux gradient is not)."""
    _, _, start = fit_problem("custom", seed=70, n_pupil=32, n_det=16, oversample=2, n_lambda=2, n_src=3, n_exp=1,
                              n_zern_max=4)
    start.flux = start.flux.copy()
    start.flux[1] = 0.0
    data = np.zeros((start.n_exp, start.n_det, start.n_det), dtype=np.int32)
    out = gpu_eval(start, data, form)
    ref = oracle_eval(start, data)
    compare(out, ref, form, groups=("coeff", "flat", "flux"))
    assert out["loss"] == pytest.approx(float(np.sum(ref["model"])), rel=1e-6)
    assert np.all(out["grads"]["d_pos"][1] == 0.0)
    assert abs(out["grads"]["d_flux"][1]) > 0
    # the live sources' position gradients against the oracle
    live = [0, 2]
    got, want = out["grads"]["d_pos"][live], ref["pos"][live]
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want)
