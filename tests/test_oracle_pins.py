"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test checks one part of the oracle against a hand-worked fixture, a closed form,
a library routine, an exact LP or an invariant of the mathematics, chosen so that a
plausible mistake (dropped term, wrong sign or index, transposed operand, wrong step
order) fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import emd_oracle as O
from oracle import exact as X
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fixture(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# ----------------------------------------------------------------------------- operators

def test_operators_hand_worked():
    g = _fixture("operators_2x3.json")
    phi = np.array(g["phi"], float)
    gx, gt = O.gradient(phi, g["dt"], g["dx"])
    np.testing.assert_array_equal(gx, g["grad_x"])
    np.testing.assert_array_equal(gt, g["grad_t"])
    d = O.divergence(np.array(g["ux"], float), np.array(g["ut"], float), g["dt"], g["dx"])
    np.testing.assert_array_equal(d, g["div"])
    # the fixture's inner products satisfy the Sec. 2.2 identity by hand as well
    assert (np.array(g["ux"])[1] * gx[1]).sum() + (np.array(g["ut"])[:, 1:] * gt[:, 1:]).sum() == g["inner_u_grad_phi"]
    assert (d * phi).sum() == -g["inner_u_grad_phi"]


@pytest.mark.parametrize("shape", [(1, 2), (1, 17), (2, 2), (3, 5), (16, 9), (7, 64)])
def test_adjoint_identity(shape):
    rng = np.random.default_rng(sum(shape))
    dt, dx = 0.37, 1.9
    phi = rng.standard_normal(shape)
    ux, ut = rng.standard_normal(shape), rng.standard_normal(shape)
    ux[0, :] = 0.0  # outer faces are not unknowns
    ut[:, 0] = 0.0
    gx, gt = O.gradient(phi, dt, dx)
    lhs = (ux * gx).sum() + (ut * gt).sum()
    rhs = -(O.divergence(ux, ut, dt, dx) * phi).sum()
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("shape", [(1, 8), (5, 7), (12, 30)])
def test_divergence_conserves_mass(shape):
    """Zero flux through the boundary: the divergence of any flux sums to zero."""
    rng = np.random.default_rng(3)
    d = O.divergence(rng.standard_normal(shape), rng.standard_normal(shape), 0.01, 3.0)
    assert abs(d.sum()) <= 1e-9 * np.abs(d).sum()


@pytest.mark.parametrize("nr,nt,dt,dx", [(1, 12, 0.1, 1.0), (4, 6, 0.5, 2.0), (9, 13, 1e-3, 12.5), (6, 3, 1.0, 0.1)])
def test_laplacian_spectrum_matches_textbook(nr, nt, dt, dx):
    """-div grad is the Neumann 5-point Laplacian: its top eigenvalue is the textbook
    4/dx^2 sin^2(pi (nr-1)/(2 nr)) + 4/dt^2 sin^2(pi (nt-1)/(2 nt)), below the Sec. 2.2 bound."""
    n = nr * nt
    L = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        gx, gt = O.gradient(e.reshape(nr, nt), dt, dx)
        L[:, c] = -O.divergence(gx, gt, dt, dx).ravel()
    assert np.allclose(L, L.T, atol=1e-9 * np.abs(L).max())
    lam = np.linalg.eigvalsh(L).max()
    exact = 4 / dt ** 2 * math.sin(math.pi * (nt - 1) / (2 * nt)) ** 2
    if nr > 1:
        exact += 4 / dx ** 2 * math.sin(math.pi * (nr - 1) / (2 * nr)) ** 2
    assert lam == pytest.approx(exact, rel=1e-10)
    assert lam <= O.lambda_bound(nr, dt, dx)


def test_shrink_hand_worked():
    for x, y, want in _fixture("operators_2x3.json")["shrink_cases"]:
        assert O.shrink(np.array([x]), y)[0] == pytest.approx(want, abs=0)


def test_prox_minimises_primal_subproblem():
    """The primal update equals the minimiser of the Sec. 2.2 subproblem
    |u| + eps/2 u^2 - g u + (u - v)^2 / (2 alpha), found by a bounded scalar search."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(7)
    for _ in range(40):
        v, g = rng.standard_normal() * 2, rng.standard_normal() * 3
        alpha, eps = 10 ** rng.uniform(-2, 0.5), 10 ** rng.uniform(-4, 0)
        obj = lambda u: abs(u) + 0.5 * eps * u * u - g * u + (u - v) ** 2 / (2 * alpha)  # noqa: E731
        best = minimize_scalar(obj, bounds=(-50, 50), method="bounded", options={"xatol": 1e-12}).x
        # primal_step on a 1x2 grid: phi = [0, g dt] gives grad_t = g at j = 1
        phi = np.array([[0.0, g]])
        _, ut = O.primal_step(np.zeros((1, 2)), np.array([[0.0, v]]), phi, alpha, eps, 1.0, 1.0)
        assert ut[0, 1] == pytest.approx(best, abs=1e-6 * (1 + abs(best)))
        assert obj(ut[0, 1]) <= obj(best) + 1e-12  # at least as good as the search


def test_mainini_hand_worked_and_invariants():
    g = _fixture("operators_2x3.json")
    mu, nu = O.mainini(g["p_obs"], g["p_pred"])
    np.testing.assert_array_equal(mu, g["mu"])
    np.testing.assert_array_equal(nu, g["nu"])
    obs, pred = synth.gather_pair_hyperbolic(nt=64, nr=8)
    mu, nu = O.mainini(obs, pred)
    assert (mu >= 0).all() and (nu >= 0).all()
    np.testing.assert_array_equal(mu - nu, pred.astype(float) - obs.astype(float))
    # at most one of the two parts of each gather is non-zero per cell
    assert (np.minimum(np.maximum(pred, 0), np.maximum(-pred, 0)) == 0).all()


# ----------------------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("axis", ["t", "x"])
def test_pdhg_three_iterations_hand_worked(axis):
    """1x3 grid, dt = 1, f = [-1, 0, 1], eps = 0, delta = 1, no balancing; worked by hand.

    The same numbers hold on the transposed 3x1 grid (transport along receivers, dx = 1)
    once alpha_0 = 1/2 is passed explicitly (there lambda's bound also counts 4/dt^2).

    lambda = 4, alpha_0 = 1/2.  Iter 0: u^1 = 0, a = sqrt(2)/2 passes (the test ratio
    ||grad dphi|| / ||dphi|| = 1 here, so a trial passes iff a <= zeta).  Iter 1: u^2 = 0
    because alpha_1 |grad phi^1| = 1/2 < alpha_1; a = alpha_1 sqrt(1 + theta_1) = 1.0987
    fails, a / 2 passes (2 trials).  Iter 2: u^3_t = a2 (a1 + a2 - 1) at j = 1, 2 and the
    first trial a = a2 sqrt(1 + theta_2) = 0.7323 passes.
    """
    obs = np.array([[1.0, 0.0, 0.0]])
    pred = np.array([[0.0, 0.0, 1.0]])
    f = np.array([-1.0, 0.0, 1.0])
    a1 = 0.5 * math.sqrt(2.0)
    th1 = a1 / 0.5
    a2 = 0.5 * a1 * math.sqrt(1.0 + th1)
    th2 = a2 / a1
    c = a2 * (a1 + a2 - 1.0)
    a3 = a2 * math.sqrt(1.0 + th2)
    th3 = a3 / a2
    phi3 = (a1 + a2) * f + a3 * (1.0 - (1.0 + th3) * c) * f
    if axis == "t":
        r = O.pdhg(obs, pred, 1.0, 1.0, max_iter=3, eps=0.0, delta=1.0, balance=O.BAL_NONE, record=True)
        along, across, phi = r["ut"][0], r["ux"], r["phi"][0]
    else:
        r = O.pdhg(obs.T, pred.T, 1.0, 1.0, max_iter=3, eps=0.0, delta=1.0, balance=O.BAL_NONE,
                   alpha0=0.5, record=True)
        along, across, phi = r["ux"][:, 0], r["ut"], r["phi"][:, 0]
    tr = r["trace"]
    np.testing.assert_allclose(tr[:, 0], [a1, a2, a3], rtol=1e-14)
    np.testing.assert_allclose(tr[:, 1], [th1, th2, th3], rtol=1e-14)
    np.testing.assert_array_equal(tr[:, 2], [1, 2, 1])
    assert r["trials"] == 4
    np.testing.assert_allclose(along, [0.0, c, c], rtol=1e-14)
    np.testing.assert_allclose(phi, phi3, rtol=1e-14)
    np.testing.assert_array_equal(across, 0.0)


def test_linesearch_trace_properties():
    """Every iteration: theta_{k+1} = alpha_{k+1} / alpha_k and
    alpha_{k+1} = alpha_k sqrt(1 + theta_k) xi^(trials - 1) (Algorithm 1)."""
    obs, pred = synth.gather_pair_hyperbolic(nt=48, nr=6, dt=4e-3)
    r = O.pdhg(obs, pred, 4e-3, 10.0, max_iter=300, record=True)
    tr = r["trace"]
    alpha = np.concatenate([[1.0 / math.sqrt(1e5 * O.lambda_bound(6, 4e-3, 10.0))], tr[:, 0]])
    theta = np.concatenate([[1.0], tr[:, 1]])
    np.testing.assert_allclose(theta[1:], alpha[1:] / alpha[:-1], rtol=1e-13)
    np.testing.assert_allclose(alpha[1:], alpha[:-1] * np.sqrt(1 + theta[:-1]) * 0.5 ** (tr[:, 2] - 1), rtol=1e-13)
    assert tr[:, 2].max() > 1  # the backtracking branch is exercised


def test_swap_negates_phi_exactly():
    """The iteration is odd in f: swapping the gathers negates u and phi bit for bit."""
    obs, pred = synth.gather_pair_hyperbolic(nt=40, nr=5)
    a = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150)
    b = O.pdhg(pred, obs, 2e-3, 10.0, max_iter=150)
    np.testing.assert_array_equal(a["phi"], -b["phi"])
    np.testing.assert_array_equal(a["ut"], -b["ut"])
    assert a["dist"] == b["dist"] and a["trials"] == b["trials"]


# ----------------------------------------------------------------------------- converged results

@pytest.mark.parametrize("shift", [-0.05, 0.02, 0.1])
def test_1d_closed_form_w1(shift):
    """nr = 1: the converged distance equals the textbook W1 = integral |F_mu - F_nu|
    (also via scipy.stats.wasserstein_distance), and u is the forced cumulative flux."""
    from scipy.stats import wasserstein_distance
    dt, obs, preds = synth.shift_sweep_1d(nt=64, shifts=[shift])
    pred = preds[0][1]
    f = O.source_term(obs, pred)
    mu, nu = np.maximum(f, 0)[0], np.maximum(-f, 0)[0]
    t = np.arange(64) * dt
    w_text = O.w1_1d(mu, nu, dt)
    w_scipy = wasserstein_distance(t, t, mu, nu) * mu.sum() * dt
    assert w_text == pytest.approx(w_scipy, rel=1e-12)
    # dx is ignored when nr = 1 (reading Q11): pass an odd value to show it
    r = O.pdhg(obs, pred, dt, 7.0, max_iter=30000, tol=1e-9)
    assert r["dist_l1"] == pytest.approx(w_text, rel=2e-5)
    ut = O.forced_flux_1d(f, dt)
    np.testing.assert_allclose(r["ut"][0], ut, atol=2e-5 * np.abs(ut).max())
    assert r["dist"] == pytest.approx(w_text + dt * 0.5e-4 * (ut ** 2).sum(), rel=2e-5)


def _tiny_case(seed, nr, nt):
    rng = np.random.default_rng(seed)
    obs = np.maximum(rng.standard_normal((nr, nt)), 0)
    pred = np.maximum(rng.standard_normal((nr, nt)), 0)
    return obs, pred


@pytest.mark.parametrize("seed,nr,nt,dt,dx", [(1, 5, 7, 0.1, 0.2), (2, 4, 4, 1.0, 1.0), (3, 3, 8, 0.05, 0.3)])
def test_converged_distance_equals_exact_lps(seed, nr, nt, dt, dx):
    """Tiny grids: PDHG converges to the min-cost flow on the grid graph, which equals the
    Kantorovich LP with the Manhattan cost; dist lies in [W, W + dx dt eps/2 ||u_W||^2]."""
    obs, pred = _tiny_case(seed, nr, nt)
    f = O.source_term(obs, pred)
    W, lux, lut = X.w1_flux_lp(f, dt, dx)
    Wt = X.w1_transport_lp(np.maximum(f, 0), np.maximum(-f, 0), dt, dx)
    assert W == pytest.approx(Wt, rel=1e-9)
    # the LP flux is feasible for the oracle's divergence: an independent check of div's signs
    np.testing.assert_allclose(O.divergence(lux, lut, dt, dx) + f, 0.0, atol=1e-9)
    r = O.pdhg(obs, pred, dt, dx, max_iter=20000, tol=1e-10)
    assert r["dist_l1"] == pytest.approx(W, rel=1e-6)
    bound = W + dx * dt * 0.5e-4 * ((lux ** 2).sum() + (lut ** 2).sum())
    assert r["dist"] <= bound * (1 + 1e-6)
    assert r["dist"] >= W * (1 - 1e-6)
    assert abs(r["gap"]) <= 1e-4 * r["dist"]


def test_fixed_step_and_linesearch_reach_same_point():
    obs, pred = _tiny_case(4, 4, 6)
    a = O.pdhg(obs, pred, 0.2, 0.5, max_iter=20000, tol=1e-10)
    b = O.pdhg(obs, pred, 0.2, 0.5, max_iter=60000, tol=1e-10, linesearch=0)
    assert a["dist"] == pytest.approx(b["dist"], rel=1e-6)


def test_single_trace_reduces_to_1d():
    """Only one non-zero trace: x-transport cannot help, so the 2D distance is dx times the
    1D closed form of that trace."""
    dt, obs1, preds = synth.shift_sweep_1d(nt=48, shifts=[0.06])
    nr, row = 4, 2
    obs = np.zeros((nr, 48))
    pred = np.zeros((nr, 48))
    obs[row], pred[row] = obs1[0], preds[0][1][0]
    f = O.source_term(obs1, preds[0][1])[0]
    w = O.w1_1d(np.maximum(f, 0), np.maximum(-f, 0), dt)
    r = O.pdhg(obs, pred, dt, 0.3, max_iter=30000, tol=1e-9, balance=O.BAL_NONE)
    assert r["dist_l1"] == pytest.approx(0.3 * w, rel=1e-4)


def test_translation_invariance_in_time():
    """Moving both gathers along t, away from the boundary, leaves the converged distance unchanged."""
    rng = np.random.default_rng(9)
    nr, nt, s = 3, 24, 5
    obs = np.zeros((nr, nt))
    pred = np.zeros((nr, nt))
    obs[:, 4:10] = np.maximum(rng.standard_normal((nr, 6)), 0)
    pred[:, 6:12] = np.maximum(rng.standard_normal((nr, 6)), 0)
    pred *= obs.sum() / pred.sum()
    a = O.pdhg(obs, pred, 0.1, 0.4, max_iter=20000, tol=1e-10, balance=O.BAL_NONE)
    b = O.pdhg(np.roll(obs, s, 1), np.roll(pred, s, 1), 0.1, 0.4, max_iter=20000, tol=1e-10, balance=O.BAL_NONE)
    assert a["dist"] == pytest.approx(b["dist"], rel=1e-6)


def test_adjoint_source_matches_finite_differences():
    """Central differences (FP64) of the converged distance w.r.t. Pcal cells against
    dx dt (phi - mean phi) (Sec. 2.3 adjoint source, reading Q8)."""
    obs, pred = _tiny_case(5, 3, 5)
    dt, dx = 0.25, 0.5
    kw = dict(max_iter=20000, tol=1e-11)
    base = O.pdhg(obs, pred, dt, dx, **kw)
    g, gobs = O.adjoint_source(base["phi"], dt, dx)
    np.testing.assert_array_equal(gobs, -g)
    h = 1e-3
    checked = 0
    for (i, j) in [(0, 1), (1, 2), (2, 3)]:
        p1, p2 = pred.copy(), pred.copy()
        p1[i, j] += h
        p2[i, j] -= h
        fd = (O.pdhg(obs, p1, dt, dx, **kw)["dist"] - O.pdhg(obs, p2, dt, dx, **kw)["dist"]) / (2 * h)
        assert fd == pytest.approx(g[i, j], abs=2e-3 * np.abs(g).max())
        checked += 1
    assert checked == 3


def test_lsd_misfit_and_adjoint():
    obs, pred = synth.gather_pair_hyperbolic(nt=32, nr=4)
    v, g = O.lsd_misfit(obs, pred, 2e-3, 10.0)
    d = pred.astype(float) - obs
    assert v == pytest.approx(0.5 * 2e-3 * 10.0 * (d ** 2).sum(), rel=1e-14)
    h = 1e-4
    p1 = pred.astype(float).copy()
    p2 = pred.astype(float).copy()
    p1[1, 7] += h
    p2[1, 7] -= h
    fd = (O.lsd_misfit(obs, p1, 2e-3, 10.0)[0] - O.lsd_misfit(obs, p2, 2e-3, 10.0)[0]) / (2 * h)
    assert fd == pytest.approx(g[1, 7], rel=1e-6, abs=1e-12)


def test_stopping_residual_hand_worked():
    """Reading Q6's residual on the 1x3 fixture above, run with mean balancing: the raw
    difference Pcal - Pobs = [0, 1, 2] has mean 1, so the balanced f is [-1, 0, 1] and
    the iterates are the hand-worked ones.  By hand: u^1 = u^2 = 0, so r_feas = ||f|| /
    ||f|| = 1 and r_step = 0 / tiny = 0; u^3_t = c at j = 1, 2 gives div u^3 + f =
    (1 - c) [-1, 0, 1], so r_feas = |1 - c|, and r_step = ||u^3|| / ||u^3|| = 1.  A norm
    of the unbalanced f (sqrt 5) or a dropped square root fails this."""
    obs = np.array([[1.0, 0.0, 0.0]])
    pred = np.array([[1.0, 1.0, 2.0]])
    a1 = 0.5 * math.sqrt(2.0)
    a2 = 0.5 * a1 * math.sqrt(1.0 + a1 / 0.5)
    c = a2 * (a1 + a2 - 1.0)
    r = O.pdhg(obs, pred, 1.0, 1.0, max_iter=3, eps=0.0, delta=1.0, balance=O.BAL_MEAN, record=True)
    tr = r["trace"]
    np.testing.assert_array_equal(tr[:, 2], [1, 2, 1])
    np.testing.assert_allclose(tr[:, 3], [1.0, 1.0, 1.0 - c], rtol=1e-14)
    np.testing.assert_array_equal(tr[:, 4], [0.0, 0.0, 1.0])
    assert r["r_feas"] == pytest.approx(1.0 - c, rel=1e-14)
    assert r["r_step"] == 1.0 and r["residual"] == 1.0
    # the stopping test reads the same values: tol between them stops at the third check
    s = O.pdhg(obs, pred, 1.0, 1.0, max_iter=50, eps=0.0, delta=1.0, tol=1.0, check_every=3)
    assert s["iters"] == 3


def test_linesearch_l1_norm_hand_worked():
    """The printed l1 form of the linesearch test (reading Q3, ls_norm = 1) on a 1x3 grid,
    dt = 1, f = [-1, 1, 0], eps = 0, delta = 1, xi = 0.9, no balancing; one iteration by
    hand.  u^1 = 0 (phi^0 = 0), so the trial potential is a f and its time gradient
    a [0, 2, -1]: the l1 test reads a * 3a <= 0.99 * 2a (a <= 0.66), the Euclidean one
    a sqrt(5) a <= 0.99 sqrt(2) a (a <= 0.6261).  Trials a = 0.7071, 0.6364, 0.5728: l1
    accepts the second, l2 the third."""
    obs = np.array([[1.0, 0.0, 0.0]])
    pred = np.array([[0.0, 1.0, 0.0]])
    f = np.array([-1.0, 1.0, 0.0])
    kw = dict(max_iter=1, eps=0.0, delta=1.0, xi=0.9, balance=O.BAL_NONE, record=True)
    a0 = 0.5 * math.sqrt(2.0)
    for ls_norm, trials in ((1, 2), (2, 3)):
        r = O.pdhg(obs, pred, 1.0, 1.0, ls_norm=ls_norm, **kw)
        a = a0 * 0.9 ** (trials - 1)
        assert r["trials"] == trials
        assert r["alpha"] == pytest.approx(a, rel=1e-14)
        assert r["theta"] == pytest.approx(a / 0.5, rel=1e-14)
        np.testing.assert_allclose(r["phi"][0], a * f, rtol=1e-14)
        np.testing.assert_array_equal(r["ut"], 0.0)


def test_forced_trials_replay_is_bit_identical():
    """Replaying the oracle's own trial counts reproduces its run bit for bit, with no
    recorded disagreement; forcing one more trial at an iteration whose first trial
    passed records that trial's gap and takes one more backtracking step there."""
    obs, pred = synth.gather_pair_hyperbolic(nt=48, nr=6, dt=4e-3)
    kw = dict(max_iter=200, record=True)
    r = O.pdhg(obs, pred, 4e-3, 10.0, **kw)
    tr = r["trace"]
    assert tr[:, 2].max() > 1
    q = O.pdhg(obs, pred, 4e-3, 10.0, force_trials=tr[:, 2].astype(int), **kw)
    for key in ("phi", "ux", "ut"):
        np.testing.assert_array_equal(q[key], r[key])
    np.testing.assert_array_equal(q["trace"][:, :6], tr[:, :6])
    np.testing.assert_array_equal(q["trace"][:, 6], 0.0)
    assert q["dist"] == r["dist"] and q["trials"] == r["trials"]
    k = int(np.nonzero(tr[:, 2] == 1)[0][5])
    forced = tr[:, 2].astype(int).copy()
    forced[k] = 2
    s = O.pdhg(obs, pred, 4e-3, 10.0, force_trials=forced, **kw)
    st = s["trace"]
    np.testing.assert_array_equal(st[:k], tr[:k])
    assert st[k, 2] == 2 and st[k, 6] == pytest.approx(tr[k, 5], rel=1e-12)
    a_prev = tr[k - 1, 0] if k > 0 else 1.0 / math.sqrt(1e5 * O.lambda_bound(6, 4e-3, 10.0))
    th_prev = tr[k - 1, 1] if k > 0 else 1.0
    assert st[k, 0] == pytest.approx(a_prev * math.sqrt(1.0 + th_prev) * 0.5, rel=1e-14)
    assert not np.array_equal(s["phi"], r["phi"])


def test_binary32_storage_model():
    """store_f32 only rounds the kept iterates: every returned entry is a binary32 value,
    the default run is untouched, and on a gather of a few thousand cells the distance
    moves by rounding's size (well under 1e-6), while on a 2 x 2 grid with the lateral flux
    shut it moves by more than 1e-5 (phi of O(1) against time differences near 1e-3)."""
    obs, pred = synth.gather_pair_hyperbolic(nt=96, nr=24, dt=2e-3)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150)
    q = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150, store_f32=True)
    for key in ("phi", "ux", "ut"):
        np.testing.assert_array_equal(q[key], q[key].astype(np.float32).astype(np.float64))
    assert not np.array_equal(r["phi"], r["phi"].astype(np.float32).astype(np.float64))
    assert q["trials"] == r["trials"]
    assert abs(q["dist"] - r["dist"]) <= 1e-6 * r["dist"]
    rng = np.random.default_rng(2002)
    obs, pred = synth.gather_pair_hyperbolic(nt=8, nr=2, dt=2e-3, seed=4)
    obs, pred = obs[:, :2].copy(), pred[:, :2].copy()
    pred += 0.05 * rng.standard_normal(pred.shape).astype(np.float32)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150)
    q = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150, store_f32=True)
    assert np.all(r["ux"] == 0.0) and abs(q["dist"] - r["dist"]) > 1e-5 * r["dist"]


def test_identical_gathers_keep_the_step_and_stay_finite():
    """Reading Q20: identical gathers (f = 0) make p and q identically zero, so the dual move is
    zero for every step size.  The step stays at alpha_0 with theta = 1 and one trial per
    iteration.  phi and u stay exactly zero and finite past the 1,500 iterations after which a
    step growing by the upper end sqrt(1 + theta) would overflow.  Gathers one ulp apart take
    the usual upper-end trial (backtracked by xi) from the first iteration."""
    for obs, dt, dx in [(synth.shift_sweep_1d(nt=256)[1], 1 / 255, 1.0),
                        (synth.gather_pair_hyperbolic(nt=64, nr=8)[0], 2e-3, 10.0)]:
        r = O.pdhg(obs, obs.copy(), dt, dx, max_iter=2500, record=True)
        tr = r["trace"]
        a0 = 1.0 / math.sqrt(1e5 * O.lambda_bound(obs.shape[0], dt, dx))
        assert r["status"] == O.STATUS_OK and r["iters"] == 2500 and r["trials"] == 2500
        np.testing.assert_array_equal(tr[:, 0], a0)
        np.testing.assert_array_equal(tr[:, 1], 1.0)
        for key in ("phi", "ux", "ut"):
            assert np.all(r[key] == 0.0)
        assert r["dist"] == 0.0
        near = obs.copy()
        near.flat[near.size // 2] = np.nextafter(near.flat[near.size // 2], np.float32(np.inf))
        q = O.pdhg(obs, near, dt, dx, max_iter=3, record=True)
        t = int(q["trace"][0, 2]) - 1  # backtracking steps of the first iteration
        assert q["trace"][0, 0] == pytest.approx(a0 * math.sqrt(2.0) * 0.5 ** t, rel=1e-15)
        assert q["trace"][0, 1] != 1.0


def test_exact_fixed_point_keeps_the_upper_end():
    """Reading Q20's scope: the lower-end step is for identical gathers only.  A 1 x 2 gather
    pair passes through exact fixed points of the iteration (r_feas = r_step = 0 at iteration
    112, p and q identically zero with f != 0); it still takes the upper-end trial there, so
    no iteration has theta = 1."""
    rng = np.random.default_rng(1002)
    obs, pred = synth.gather_pair_hyperbolic(nt=8, nr=1, dt=2e-3, seed=3)
    obs, pred = obs[:, :2].copy(), pred[:, :2].copy()
    pred += 0.05 * rng.standard_normal(pred.shape).astype(np.float32)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150, record=True)
    tr = r["trace"]
    assert ((tr[:, 3] == 0.0) & (tr[:, 4] == 0.0)).any()
    assert not (tr[:, 1] == 1.0).any()
