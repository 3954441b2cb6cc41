"""Pins of the oracle's isotropic ground cost (reading Q19, the ||u||_{1,2} formulation
the paper builds on) against things other than its own formulas: the prox against a
numerical minimisation of its subproblem, the reduction to the anisotropic norm in 1D,
the sqrt(2) bracket between the two norms, and the converged value against the maximum of
the smooth eps-regularised dual problem found by an independent optimiser (L-BFGS).
No GPU needed.
"""

import math

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import emd_oracle as O
import synth


def test_vector_shrink_is_the_prox_of_the_euclidean_norm():
    """u = shrink_vec(v, a) / (1 + eps a) minimises ||u|| + eps/2 ||u||^2 + ||u - v||^2 / (2a)
    over the plane (Nelder-Mead from a distant start)."""
    rng = np.random.default_rng(4)
    for _ in range(40):
        v = rng.standard_normal(2) * rng.choice([0.1, 1.0, 5.0])
        a = float(rng.uniform(0.05, 2.0))
        eps = float(rng.choice([0.0, 1e-2, 0.5]))
        sx, st = O.shrink_vec(np.array([v[0]]), np.array([v[1]]), a)
        u = np.array([sx[0], st[0]]) / (1.0 + eps * a)

        def f(w):
            return math.hypot(w[0], w[1]) + 0.5 * eps * (w @ w) + ((w - v) @ (w - v)) / (2 * a)

        best = minimize(f, v + 3.0, method="Nelder-Mead",
                        options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000))
        assert f(u) <= best.fun + 1e-10
        np.testing.assert_allclose(u, best.x, atol=1e-5)


def test_vector_shrink_zeroes_short_vectors_and_keeps_direction():
    vx, vt = np.array([0.3, 3.0, 0.0]), np.array([0.4, 4.0, 0.0])
    sx, st = O.shrink_vec(vx, vt, 0.5)  # lengths 0.5 (= threshold), 5, 0
    assert sx[0] == 0.0 and st[0] == 0.0 and sx[2] == 0.0 and st[2] == 0.0
    np.testing.assert_allclose([sx[1], st[1]], [3.0 * 0.9, 4.0 * 0.9], rtol=1e-15)


def test_isotropic_equals_anisotropic_in_1d():
    """nr = 1 has no x flux, so the two norms are the same problem."""
    dt, obs, preds = synth.shift_sweep_1d(nt=96, shifts=[0.07])
    a = O.pdhg(obs, preds[0][1], dt, 1.0, max_iter=400)
    b = O.pdhg(obs, preds[0][1], dt, 1.0, max_iter=400, norm=O.NORM_ISO)
    assert b["trials"] == a["trials"]
    np.testing.assert_allclose(b["ut"], a["ut"], rtol=1e-12, atol=1e-15)
    assert b["dist"] == pytest.approx(a["dist"], rel=1e-12)


def _tiny(seed, nr, nt):
    rng = np.random.default_rng(seed)
    return np.maximum(rng.standard_normal((nr, nt)), 0), np.maximum(rng.standard_normal((nr, nt)), 0)


def _dual_max(f, dt, dx, eps, norm):
    """max over phi of <phi, f> - sum h*(grad phi), the dual of the eps-regularised problem,
    written out here from the definitions: grad is the backward difference with a zero first
    row / column, h*(w) = (|w| - 1)_+^2 / (2 eps) per component (anisotropic) or of the cell
    vector (isotropic).  Returns the maximum (times dx dt)."""
    nr, nt = f.shape

    def neg(x):
        phi = x.reshape(nr, nt)
        gx = np.zeros_like(phi)
        gt = np.zeros_like(phi)
        gx[1:] = (phi[1:] - phi[:-1]) / dx
        gt[:, 1:] = (phi[:, 1:] - phi[:, :-1]) / dt
        if norm == O.NORM_ISO:
            n = np.sqrt(gx * gx + gt * gt)
            e = np.maximum(n - 1.0, 0.0)
            hs = (e * e).sum() / (2 * eps)
            with np.errstate(invalid="ignore", divide="ignore"):
                s = np.where(n > 0, e / (eps * n), 0.0)
            wx, wt = s * gx, s * gt
        else:
            ex, et = np.maximum(np.abs(gx) - 1, 0), np.maximum(np.abs(gt) - 1, 0)
            hs = ((ex * ex).sum() + (et * et).sum()) / (2 * eps)
            wx, wt = np.sign(gx) * ex / eps, np.sign(gt) * et / eps
        val = (phi * f).sum() - hs
        # d/dphi of sum h*(grad phi) = grad^T (w): adjoint of the backward differences
        gr = np.zeros_like(phi)
        gr[1:] += wx[1:] / dx
        gr[:-1] -= wx[1:] / dx
        gr[:, 1:] += wt[:, 1:] / dt
        gr[:, :-1] -= wt[:, 1:] / dt
        return -val, -(f - gr).ravel()

    r = minimize(neg, np.zeros(nr * nt), jac=True, method="L-BFGS-B",
                 options=dict(maxiter=20000, ftol=1e-15, gtol=1e-11))
    return -r.fun * dx * dt


@pytest.mark.parametrize("norm", [O.NORM_ISO, O.NORM_ANISO])
@pytest.mark.parametrize("seed,nr,nt,dt,dx", [(21, 4, 5, 0.2, 0.3), (22, 3, 6, 0.25, 0.25)])
def test_converged_value_equals_the_dual_maximum(norm, seed, nr, nt, dt, dx):
    """Strong duality: Algorithm 1's primal value at convergence equals the maximum of the
    smooth dual, found here by L-BFGS on the dual written from the definitions."""
    obs, pred = _tiny(seed, nr, nt)
    eps = 0.05
    r = O.pdhg(obs, pred, dt, dx, max_iter=60000, tol=1e-11, eps=eps, norm=norm)
    d = _dual_max(O.source_term(obs, pred), dt, dx, eps, norm)
    assert r["dist"] == pytest.approx(d, rel=1e-6)


@pytest.mark.parametrize("seed,nr,nt", [(23, 4, 6), (24, 5, 5)])
def test_isotropic_between_anisotropic_over_sqrt2_and_anisotropic(seed, nr, nt):
    """||v||_1 / sqrt(2) <= ||v||_2 <= ||v||_1 for every cell vector, so the optima obey the
    same bracket (and the isotropic one is strictly cheaper when flux moves diagonally)."""
    obs, pred = _tiny(seed, nr, nt)
    a = O.pdhg(obs, pred, 0.2, 0.2, max_iter=60000, tol=1e-10)
    b = O.pdhg(obs, pred, 0.2, 0.2, max_iter=60000, tol=1e-10, norm=O.NORM_ISO)
    assert a["dist_l1"] / math.sqrt(2) * (1 - 1e-6) <= b["dist_l1"] <= a["dist_l1"] * (1 + 1e-6)
    assert b["dist_l1"] < a["dist_l1"] * (1 - 1e-3)
    assert abs(b["gap"]) <= 1e-4 * b["dist"]
