"""FP64 oracle of the Laplace-approximation curvature of arXiv:2406.08703
(Sec. 4): the Hessian of the Poisson negative log-likelihood over the source
positions, fluxes and Zernike coefficients with the pixel response held fixed,
its Gauss-Newton term and the expected (Fisher) information, and the errors
sqrt(diag(H^-1)).

TEST INFRASTRUCTURE ONLY, like the rest of this package.  Everything here
follows the definitions with nothing but the FP64 forward model and the FP64
analytic gradient of ``dlx_oracle.c``:
  J[i][p] = dm_p / dtheta_i   by central differences of the model,
  H[i][j] = dg_i / dtheta_j   by central differences of the gradient g of
                              sum (m - d ln m),
each with one Richardson step, D = (4 D(h/2) - D(h)) / 3 with
D(h) = (f(theta + h) - f(theta - h)) / (2 h), so the truncation error is O(h^4).
Fisher = J diag(1/m) J^T, Gauss-Newton = J diag(d/m^2) J^T.
Pinned in tests/test_oracle_laplace.py by closed forms (flux-only and
full-period DFT cases, where Parseval's theorem fixes every entry) and by the
tilt identity between positions and the Z2/Z3 coefficients.
"""

from __future__ import annotations

import copy
import math

import numpy as np

from . import forward, loss_grad

GROUPS = ("pos", "flux", "zern")


def labels(n_src, n_zern, groups=GROUPS):
    """Parameter order: ("pos", s, axis), ("flux", s), ("zern", j)."""
    out = []
    for g in groups:
        if g == "pos":
            out += [("pos", s, a) for s in range(n_src) for a in (0, 1)]
        elif g == "flux":
            out += [("flux", s) for s in range(n_src)]
        elif g == "zern":
            out += [("zern", j) for j in range(n_zern)]
    return out


def _step(p, lab):
    """Difference step: 0.01 rad of phase at the pupil edge (positions), 0.01 rad per unit of
    the basis (Zernikes), 1% of the flux (the model is linear in it)."""
    lam = float(np.min(p.lambdas))
    if lab[0] == "pos":
        return 1e-2 * lam / (math.pi * p.diameter)
    if lab[0] == "zern":
        return 1e-2 * lam / (2 * math.pi)
    return 1e-2 * max(abs(float(p.flux[lab[1]])), 1.0)


def _shifted(p, lab, delta):
    q = copy.deepcopy(p)
    if lab[0] == "pos":
        q.pos = np.array(q.pos, dtype=np.float64)
        q.pos[lab[1], lab[2]] += delta
    elif lab[0] == "flux":
        q.flux = np.array(q.flux, dtype=np.float64)
        q.flux[lab[1]] += delta
    else:
        q.coeff = np.array(q.coeff, dtype=np.float64)
        q.coeff[lab[1]] += delta
    return q


def _richardson(f, p, lab):
    h = _step(p, lab)

    def d(hh):
        return (f(_shifted(p, lab, hh)) - f(_shifted(p, lab, -hh))) / (2 * hh)

    return (4 * d(h / 2) - d(h)) / 3


def jacobian(p, groups=GROUPS):
    """J [n_par][n_exp Nd Nd] (float64)."""
    labs = labels(len(p.flux), len(p.coeff), groups)
    return np.stack([_richardson(lambda q: forward(q).reshape(-1), p, lab) for lab in labs]), labs


def _grad_vector(p, data, labs):
    g = loss_grad(p, data)
    out = np.empty(len(labs))
    for k, lab in enumerate(labs):
        if lab[0] == "pos":
            out[k] = g["pos"][lab[1], lab[2]]
        elif lab[0] == "flux":
            out[k] = g["flux"][lab[1]]
        else:
            out[k] = g["coeff"][lab[1]]
    return out


def information(p, data=None, kind="hessian", groups=GROUPS):
    """(matrix, labels) of the kind "hessian", "gauss_newton" or "fisher"."""
    labs = labels(len(p.flux), len(p.coeff), groups)
    if kind == "hessian":
        H = np.stack([_richardson(lambda q: _grad_vector(q, data, labs), p, lab) for lab in labs], axis=1)
        return 0.5 * (H + H.T), labs
    J, _ = jacobian(p, groups)
    m = np.maximum(forward(p).reshape(-1), 1e-30)
    w = 1.0 / m if kind == "fisher" else np.asarray(data, dtype=np.float64).reshape(-1) / (m * m)
    return (J * w) @ J.T, labs


def sigma(H):
    """Marginal 1-sigma errors sqrt(diag(H^-1))."""
    return np.sqrt(np.diag(np.linalg.inv(H)))
