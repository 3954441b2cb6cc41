"""Pins of the oracle's multigrid warm start (Sec. 2.2 closing paragraph, Sec. 3.3).

Each check is against something other than the oracle's own formulas: hand-worked
restrictions, conservation of mass, the analytic values of a band-limited signal at
positions taken from the cell geometry, and exact LPs / the 1D closed form for the
converged two-grid solve.  No GPU needed.
"""

import numpy as np
import pytest

from oracle import emd_oracle as O
from oracle import exact as X
from oracle import multigrid as MG
import synth


# ----------------------------------------------------------------------------- restriction

def test_restrict_hand_worked_with_ragged_tail():
    a = np.array([[1.0, 1.0, 2.0, 2.0, 3.0],
                  [0.0, 4.0, -2.0, 6.0, 8.0]])
    # blocks of 2; the fifth sample shares its block with a padded zero
    np.testing.assert_array_equal(MG.restrict_time(a, 2), [[1.0, 2.0, 1.5], [2.0, 2.0, 4.0]])
    np.testing.assert_array_equal(MG.restrict_time(a, 5), [[9.0 / 5], [16.0 / 5]])
    assert MG.coarse_length(5, 2) == 3 and MG.coarse_length(6, 3) == 2 and MG.coarse_length(7, 3) == 3


@pytest.mark.parametrize("nt,r", [(23, 4), (24, 4), (64, 7), (9, 9), (5, 8)])
def test_restrict_conserves_mass(nt, r):
    """r dt sum_J f_c = dt sum_j f: the coarse gather carries the fine gather's mass."""
    a = np.random.default_rng(nt * r).standard_normal((3, nt))
    c = MG.restrict_time(a, r)
    assert c.shape == (3, -(-nt // r))
    np.testing.assert_allclose(r * c.sum(axis=1), a.sum(axis=1), rtol=1e-13, atol=1e-13)


def test_restrict_block_constant_and_identity():
    vals = np.array([[0.5, -1.0, 3.0, 2.0]])
    np.testing.assert_array_equal(MG.restrict_time(np.repeat(vals, 3, axis=1), 3), vals)
    a = np.random.default_rng(0).standard_normal((2, 11))
    np.testing.assert_array_equal(MG.restrict_time(a, 1), a)


# ----------------------------------------------------------------------------- sinc interpolation

def _gauss(t, t0, s):
    return np.exp(-0.5 * ((t - t0) / s) ** 2)


@pytest.mark.parametrize("r", [2, 3, 5, 10])
def test_sinc_reproduces_band_limited_signal_cell_centres(r):
    """Cell-centred data: fine cell j has its centre at time j dt, coarse cell J (fine
    cells rJ .. rJ + r - 1) at (rJ + (r - 1)/2) dt.  A Gaussian 3 coarse samples wide has
    no spectrum above the coarse Nyquist frequency worth speaking of, so interpolating its
    coarse samples gives its fine samples up to the truncation of the record."""
    nc = 40
    nt = nc * r
    dt = 1.0
    sigma = 3.0 * r * dt
    assert MG.sinc_bandlimit_error_bound(3.0) < 1e-15
    t0 = 0.5 * nt * dt
    tc = (r * np.arange(nc) + (r - 1) / 2.0) * dt
    tf = np.arange(nt) * dt
    got = MG.sinc_interpolate(_gauss(tc, t0, sigma)[None, :], r, nt, staggered=False)[0]
    np.testing.assert_allclose(got, _gauss(tf, t0, sigma), atol=1e-9)


@pytest.mark.parametrize("r", [2, 3, 5, 10])
def test_sinc_reproduces_band_limited_signal_time_faces(r):
    """Time-face data: fine face j lies between cells j - 1 and j, at (j - 1/2) dt; coarse
    face J at (rJ - 1/2) dt."""
    nc = 40
    nt = nc * r
    dt = 0.004
    sigma = 3.0 * r * dt
    t0 = 0.5 * nt * dt
    tc = (r * np.arange(nc) - 0.5) * dt
    tf = (np.arange(nt) - 0.5) * dt
    got = MG.sinc_interpolate(_gauss(tc, t0, sigma)[None, :], r, nt, staggered=True)[0]
    np.testing.assert_allclose(got, _gauss(tf, t0, sigma), atol=1e-9)


def test_sinc_interpolates_through_coarse_samples():
    """Where a fine position coincides with a coarse one the coarse value comes back
    exactly (sinc vanishes at every other integer): r odd for cell centres (fine cell
    rJ + (r-1)/2), any r for time faces (fine face rJ)."""
    rng = np.random.default_rng(5)
    v = rng.standard_normal((3, 9))
    r = 3
    c = MG.sinc_interpolate(v, r, 27, staggered=False)
    np.testing.assert_allclose(c[:, 1::3], v, atol=1e-14)
    for r in (2, 4):
        s = MG.sinc_interpolate(v, r, 9 * r, staggered=True)
        np.testing.assert_allclose(s[:, ::r], v, atol=1e-14)
    np.testing.assert_allclose(MG.sinc_interpolate(v, 1, 9, False), v, atol=1e-14)
    np.testing.assert_allclose(MG.sinc_interpolate(v, 1, 9, True), v, atol=1e-14)


def test_warm_start_zeroes_outer_faces_and_optional_phi():
    rng = np.random.default_rng(6)
    phi_c, ux_c, ut_c = (rng.standard_normal((4, 5)) for _ in range(3))
    phi, m = MG.warm_start(phi_c, ux_c, ut_c, 2, 10)
    assert m.shape == (2, 4, 10) and phi.shape == (4, 10)
    assert not m[0, 0].any() and not m[1, :, 0].any()
    assert m[0, 1:].any() and m[1, :, 1:].any() and phi.any()
    phi0, _ = MG.warm_start(phi_c, ux_c, ut_c, 2, 10, interpolate_phi=False)
    assert not phi0.any()


# ----------------------------------------------------------------------------- two-grid solve

def _tiny(seed, nr, nt):
    rng = np.random.default_rng(seed)
    return np.maximum(rng.standard_normal((nr, nt)), 0), np.maximum(rng.standard_normal((nr, nt)), 0)


@pytest.mark.parametrize("seed,nr,nt,r,dt,dx", [(11, 4, 12, 2, 0.1, 0.3), (12, 3, 10, 3, 0.05, 0.2)])
def test_two_grid_solves_match_exact_lps(seed, nr, nt, r, dt, dx):
    """The coarse solve is the EMD of the block-averaged gathers at spacing r dt (its LP
    built here from a restriction written out by hand); the fine solve, started from the
    interpolated coarse solution, still converges to the fine grid's min-cost flow."""
    obs, pred = _tiny(seed, nr, nt)
    nc = -(-nt // r)
    pad = lambda a: np.concatenate([a, np.zeros((nr, nc * r - nt))], axis=1)
    fc = np.mean(pad(pred).reshape(nr, nc, r), 2) - np.mean(pad(obs).reshape(nr, nc, r), 2)
    fc -= fc.mean()
    Wc, _, _ = X.w1_flux_lp(fc, r * dt, dx)
    W, _, _ = X.w1_flux_lp(O.source_term(obs, pred), dt, dx)
    c, f = MG.pdhg_multigrid(obs, pred, dt, dx, r,
                             coarse=O.Params(max_iter=20000, tol=1e-10),
                             fine=O.Params(max_iter=20000, tol=1e-10))
    assert c["dist_l1"] == pytest.approx(Wc, rel=1e-6)
    assert f["dist_l1"] == pytest.approx(W, rel=1e-6)
    assert f["status"] == O.STATUS_OK and abs(f["gap"]) <= 1e-4 * f["dist"]


def test_two_grid_1d_matches_closed_form():
    """nr = 1 (Q11): the two-grid solve ends at the textbook W1 of the fine trace."""
    dt, obs, preds = synth.shift_sweep_1d(nt=96, shifts=[0.08])
    pred = preds[0][1]
    f = O.source_term(obs, pred)[0]
    w = O.w1_1d(np.maximum(f, 0), np.maximum(-f, 0), dt)
    c, fr = MG.pdhg_multigrid(obs, pred, dt, 1.0, 4,
                              coarse=O.Params(max_iter=3000, tol=1e-6),
                              fine=O.Params(max_iter=30000, tol=1e-9))
    assert fr["dist_l1"] == pytest.approx(w, rel=2e-5)
    # the coarse solve is the closed form of the block-averaged trace at spacing 4 dt
    fc = (pred - obs)[0].reshape(24, 4).mean(axis=1)
    fc -= fc.mean()
    wc = O.w1_1d(np.maximum(fc, 0), np.maximum(-fc, 0), 4 * dt)
    assert c["dist_l1"] == pytest.approx(wc, rel=1e-4)


def test_two_grid_needs_fewer_fine_iterations():
    """The point of the strategy: from the interpolated coarse solution the fine solve
    reaches the tolerance in fewer iterations than from zero."""
    dt, obs, preds = synth.shift_sweep_1d(nt=512, shifts=[0.1])
    pred = preds[0][1]
    tol = 1e-4
    cold = O.pdhg(obs, pred, dt, 1.0, max_iter=40000, tol=tol)
    _, warm = MG.pdhg_multigrid(obs, pred, dt, 1.0, 8,
                                coarse=O.Params(max_iter=40000, tol=tol),
                                fine=O.Params(max_iter=40000, tol=tol))
    assert warm["residual"] <= tol and cold["residual"] <= tol
    assert warm["iters"] < 0.5 * cold["iters"]
    assert warm["dist"] == pytest.approx(cold["dist"], rel=1e-3)
