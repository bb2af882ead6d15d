"""Pins of the oracle's Laplace-approximation curvature (Sec. 4) against what
the mathematics fixes:

- full-period case (one wavelength, oversample 1, Nd = Ni, pixel = lambda/D, a
  centrosymmetric pupil, no aberration): the MFT is a unitary DFT up to scale,
  the field is real, and Parseval's theorem gives every Fisher entry in closed
  form -- 4 k^2 N <t_i t_j>_A for two odd phase tangents t (tilts, comas), zero
  for any even one (defocus), N / F^2 for the flux and zero between flux and
  phase; the likelihood Hessian then has H_FF = sum(d) / F^2 and H_F,phase = 0
  for any data;
- flux block of any model: the model is linear in each flux, so
  F_st = sum m_s m_t / (F_s F_t m) and H_st = sum d m_s m_t / (F_s F_t m^2)
  with m_s the one-source models, and sigma_F = F / sqrt(N) for one star;
- tilt identity: Z2 = 4 x / D on the pupil, so dm/dc_2 = (4 / D) sum_s dm/dtheta_{s,x};
- the Hessian from differences of the analytic gradient equals the one from
  second differences of the loss itself.
"""

import math

import numpy as np
import pytest

import workloads as W
from laplace_cases import LAM, aberrated_problem as _aberrated, laplace_problem as _problem

def _odd(t):
    return np.allclose(t, -t[::-1, ::-1], atol=1e-12 * np.max(np.abs(t)))


def test_fisher_full_period_closed_form(oracle_lib):
    from oracle import laplace as OL

    p = _problem()
    H, labs = OL.information(p, kind="fisher")
    N = float(np.sum(oracle_lib.forward(p)))
    F = float(p.flux[0])
    k = 2 * math.pi / LAM
    A2 = p.transmission**2
    c = W.pixel_coords(p.n_pupil, p.diameter)
    tan = {("pos", 0, 0): np.broadcast_to(c[None, :], A2.shape), ("pos", 0, 1): np.broadcast_to(c[:, None], A2.shape)}
    for j in range(p.n_zern):
        tan[("zern", j)] = p.basis[j]
    want = np.zeros_like(H)
    for a, la in enumerate(labs):
        for b, lb in enumerate(labs):
            if la[0] == "flux" and lb[0] == "flux":
                want[a, b] = N / F**2
            elif la[0] != "flux" and lb[0] != "flux" and _odd(tan[la]) and _odd(tan[lb]):
                want[a, b] = 4 * k * k * N * np.sum(A2 * tan[la] * tan[lb]) / np.sum(A2)
    scale = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    scale[scale == 0] = np.max(np.diag(want))
    assert labs[-3] == ("zern", 2) and not _odd(p.basis[2])  # Z4, defocus: even, no first-order signal
    assert np.max(np.abs(H - want) / scale) < 1e-7


def test_hessian_full_period_flux_entries(oracle_lib):
    """Any data: H_FF = sum(d) / F^2 and H_F,phase = 0 (the total model does not depend on the phase)."""
    from oracle import laplace as OL

    p = _problem(noll=(4, 7))
    m = oracle_lib.forward(p)
    data = np.random.default_rng(3).poisson(m * 1.1).astype(np.int32)
    H, labs = OL.information(p, data, kind="hessian")
    f = labs.index(("flux", 0))
    F = float(p.flux[0])
    assert H[f, f] == pytest.approx(float(data.sum()) / F**2, rel=1e-9)
    others = [i for i in range(len(labs)) if i != f]
    assert np.max(np.abs(H[f, others]) / np.sqrt(H[f, f] * np.abs(np.diag(H)[others]))) < 1e-7


def _one_source_models(oracle_lib, p):
    out = []
    for s in range(p.n_src):
        q = p.copy()
        q.flux, q.pos = p.flux[s:s + 1].copy(), p.pos[s:s + 1].copy()
        out.append(oracle_lib.forward(q).reshape(-1))
    return out


def test_flux_block_matches_one_source_models(oracle_lib):
    from oracle import laplace as OL

    p = _aberrated()
    m = oracle_lib.forward(p).reshape(-1)
    ms = _one_source_models(oracle_lib, p)
    data = np.random.default_rng(9).poisson(m).astype(np.int32)
    Fi, labs = OL.information(p, kind="fisher", groups=("flux",))
    Hh, _ = OL.information(p, data, kind="hessian", groups=("flux",))
    Gn, _ = OL.information(p, data, kind="gauss_newton", groups=("flux",))
    F = p.flux
    d = data.reshape(-1).astype(np.float64)
    for s in range(p.n_src):
        for t in range(p.n_src):
            fst = np.sum(ms[s] * ms[t] / m) / (F[s] * F[t])
            hst = np.sum(d * ms[s] * ms[t] / m**2) / (F[s] * F[t])
            assert Fi[s, t] == pytest.approx(fst, rel=1e-9)
            assert Hh[s, t] == pytest.approx(hst, rel=1e-8)
            assert Gn[s, t] == pytest.approx(hst, rel=1e-9)  # the flux block has no second-order term


def test_single_star_flux_sigma(oracle_lib):
    """Flux alone, one star: sigma_F = F / sqrt(N), N the expected total count."""
    from oracle import laplace as OL

    p = _aberrated(n_src=1)
    H, _ = OL.information(p, kind="fisher", groups=("flux",))
    N = float(np.sum(oracle_lib.forward(p)))
    assert OL.sigma(H)[0] == pytest.approx(p.flux[0] / math.sqrt(N), rel=1e-10)


def test_tilt_identity_in_jacobian_and_hessian(oracle_lib):
    """Z2 = 4x/D and Z3 = 4y/D on the pupil: the c_2 (c_3) column is 4/D times the sum of the
    theta_x (theta_y) columns of all sources, in J and in the Hessian."""
    from oracle import laplace as OL

    p = _aberrated()
    assert p.noll[:2] == [2, 3]
    J, labs = OL.jacobian(p)
    m = oracle_lib.forward(p)
    data = np.random.default_rng(4).poisson(m).astype(np.int32)
    H, _ = OL.information(p, data, kind="hessian")
    for ax in (0, 1):
        z = labs.index(("zern", ax))
        ps = [labs.index(("pos", s, ax)) for s in range(p.n_src)]
        lhs = J[z]
        rhs = 4 / p.diameter * J[ps].sum(axis=0)
        assert np.max(np.abs(lhs - rhs)) <= 1e-8 * np.max(np.abs(lhs))
        hz = H[z]
        hp = 4 / p.diameter * H[ps].sum(axis=0)
        assert np.max(np.abs(hz - hp)) <= 1e-7 * np.max(np.abs(hz))


def test_hessian_equals_second_differences_of_the_loss(oracle_lib):
    """Two routes to the same matrix: differences of the analytic gradient, and second differences
    of the loss with one Richardson step."""
    from oracle import laplace as OL

    p = _aberrated(n_src=2)
    p.basis, p.coeff, p.noll = p.basis[2:], p.coeff[2:], p.noll[2:]
    m = oracle_lib.forward(p)
    data = np.random.default_rng(6).poisson(m).astype(np.int32)
    H, labs = OL.information(p, data, kind="hessian")
    n = len(labs)
    h = np.array([OL._step(p, lab) for lab in labs])

    def L(shifts):
        q = p
        for k, v in shifts:
            q = OL._shifted(q, labs[k], v)
        return oracle_lib.loss(q, data)

    def d2(i, j, s):
        if i == j:
            return (L([(i, s * h[i])]) - 2 * L([]) + L([(i, -s * h[i])])) / (s * h[i]) ** 2
        return (L([(i, s * h[i]), (j, s * h[j])]) - L([(i, s * h[i]), (j, -s * h[j])])
                - L([(i, -s * h[i]), (j, s * h[j])]) + L([(i, -s * h[i]), (j, -s * h[j])])) / (4 * s * s * h[i] * h[j])

    B = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            B[i, j] = B[j, i] = (4 * d2(i, j, 0.5) - d2(i, j, 1.0)) / 3
    scale = np.sqrt(np.outer(np.abs(np.diag(H)), np.abs(np.diag(H))))
    assert np.max(np.abs(H - B) / scale) < 1e-5
