"""Two-grid solve on the GPU (Sec. 2.2 closing paragraph, Sec. 3.3) against the oracle.

Each stage through the C ABI against the oracle's stage on the same seeded input: the
time restriction, the sinc interpolation (also its exact cases), and the whole two-grid
solve at fixed iteration counts on a case whose linesearch decisions have no near ties in
either stage (so FP32 and FP64 take the same steps).  Then the properties the strategy
exists for -- the same converged distance as a single solve, fewer fine iterations --
and the batched two-grid solve against per-gather ones.
"""

import numpy as np
import pytest
import torch

from oracle import emd_oracle as O
from oracle import multigrid as MG
import synth

pytestmark = pytest.mark.gpu

DIST_RTOL = 1e-4
PHI_RTOL = 1e-3


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07284_gb300 import build
    build.build()
    import paper_1808_07284_gb300 as P
    return P


DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def _rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ----------------------------------------------------------------------------- restriction

@pytest.mark.parametrize("nr,nt,r", [(5, 23, 4), (64, 256, 1), (64, 256, 3), (7, 1001, 10), (400, 3000, 10),
                                     (1, 1024, 8), (3, 9, 9)])
def test_restriction_matches_oracle(P, nr, nt, r):
    a = np.random.default_rng(nr * nt + r).standard_normal((nr, nt)).astype(np.float32)
    out = torch.full((nr, -(-nt // r)), float("nan"), device=DEV)
    P.emd_restrict_time(_t(a), r, out)
    torch.cuda.synchronize()
    want = MG.restrict_time(a, r)
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-6 * np.abs(a).max() * max(1.0, np.sqrt(r)))
    if r == 1:
        np.testing.assert_array_equal(got, a)


# ----------------------------------------------------------------------------- interpolation

@pytest.mark.parametrize("staggered", [False, True])
@pytest.mark.parametrize("nr,nc,r", [(3, 9, 2), (70, 40, 3), (130, 37, 5), (64, 300, 10), (1, 128, 8), (9, 2, 7)])
def test_sinc_interpolation_matches_oracle(P, nr, nc, r, staggered):
    """Ragged row tiles (70, 130 receivers on 64-row tiles) and fine-sample tiles."""
    nt = nc * r - (r // 2)  # a fine record that ends inside the last coarse cell
    v = np.random.default_rng(nc + 100 * r).standard_normal((nr, nc)).astype(np.float32)
    out = torch.full((nr, nt), float("nan"), device=DEV)
    P.emd_prolong_time(_t(v), r, out, staggered)
    torch.cuda.synchronize()
    want = MG.sinc_interpolate(v, r, nt, staggered)
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert _rel_l2(got, want) <= 2e-6
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6 * np.abs(v).max() * np.log(nc + 2))


def test_sinc_interpolation_exact_cases(P):
    """factor 1 is the identity and coincident positions return the coarse value, bit for
    bit (every other kernel entry of such a column is zero); outer faces are zeroed."""
    rng = np.random.default_rng(3)
    v = rng.standard_normal((33, 50)).astype(np.float32)
    for staggered in (False, True):
        out = torch.empty((33, 50), device=DEV)
        P.emd_prolong_time(_t(v), 1, out, staggered)
        np.testing.assert_array_equal(out.cpu().numpy(), v)
    out = torch.empty((33, 150), device=DEV)
    P.emd_prolong_time(_t(v), 3, out, False)  # centre of coarse cell J = fine cell 3J + 1
    np.testing.assert_array_equal(out.cpu().numpy()[:, 1::3], v)
    out = torch.empty((33, 200), device=DEV)
    P.emd_prolong_time(_t(v), 4, out, True, zero_row0=True, zero_col0=True)  # face J = fine face 4J
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got[1:, 4::4], v[1:, 1:])
    assert not got[0].any() and not got[:, 0].any()


# ----------------------------------------------------------------------------- whole two-grid solve

def _oracle_two_grid(obs, pred, dt, dx, r, kc, kf):
    c = O.pdhg(MG.restrict_time(obs, r), MG.restrict_time(pred, r), dt * r, dx, max_iter=kc, record=True)
    phi0, m0 = MG.warm_start(c["phi"], c["ux"], c["ut"], r, obs.shape[1])
    f = O.pdhg(obs, pred, dt, dx, max_iter=kf, record=True, phi_init=phi0, m_init=m0)
    return c, f


@pytest.mark.parametrize("r,kc,kf", [(4, 200, 150), (5, 150, 100)])
def test_two_grid_solve_matches_oracle(P, r, kc, kf):
    """256 x 64 hyperbolic gathers (dt = 2 ms, dx = 10 m), fixed iteration counts in both
    stages.  The oracle's linesearch test never comes within 1e-3 of its threshold here,
    so both sides take every decision alike and the results compare element by element."""
    obs, pred = synth.gather_pair_hyperbolic()
    nr, nt = obs.shape
    c, f = _oracle_two_grid(obs.astype(np.float64), pred.astype(np.float64), 2e-3, 10.0, r, kc, kf)
    assert c["trace"][:, 5].min() > 1e-3 and f["trace"][:, 5].min() > 1e-3
    dist, phi, m, info = P.emd(_t(obs), _t(pred), 2e-3, 10.0, max_iter=kf,
                               multigrid=dict(factor=r, coarse_max_iter=kc, coarse_tol=0.0))
    ci = info["coarse"]
    assert (ci["iters"], ci["ls_trials"]) == (c["iters"], c["trials"])
    assert ci["dist"] == pytest.approx(c["dist"], rel=DIST_RTOL)
    assert (info["iters"], info["ls_trials"]) == (f["iters"], f["trials"])
    assert dist == pytest.approx(f["dist"], rel=DIST_RTOL)
    assert _rel_l2(phi.cpu().numpy(), f["phi"]) <= PHI_RTOL
    assert _rel_l2(m[0].cpu().numpy(), f["ux"]) <= PHI_RTOL
    assert _rel_l2(m[1].cpu().numpy(), f["ut"]) <= PHI_RTOL
    assert info["launches"] >= ci["launches"] + 2


def test_two_grid_without_phi_matches_oracle(P):
    """interpolate_phi = 0: the fine solve starts from phi = 0 (the paper's sentence read
    literally)."""
    obs, pred = synth.gather_pair_hyperbolic()
    r, kc, kf = 4, 200, 150
    c = O.pdhg(MG.restrict_time(obs, r), MG.restrict_time(pred, r), 2e-3 * r, 10.0, max_iter=kc)
    phi0, m0 = MG.warm_start(c["phi"], c["ux"], c["ut"], r, obs.shape[1], interpolate_phi=False)
    f = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=kf, record=True, phi_init=phi0, m_init=m0)
    if f["trace"][:, 5].min() <= 1e-3:
        pytest.skip("near tie in the oracle's linesearch for this case")
    dist, phi, m, info = P.emd(_t(obs), _t(pred), 2e-3, 10.0, max_iter=kf,
                               multigrid=dict(factor=r, coarse_max_iter=kc, interpolate_phi=0))
    assert (info["iters"], info["ls_trials"]) == (f["iters"], f["trials"])
    assert dist == pytest.approx(f["dist"], rel=DIST_RTOL)
    assert _rel_l2(phi.cpu().numpy(), f["phi"]) <= PHI_RTOL


def test_two_grid_converges_to_single_solve(P):
    """Normalised domain (the paper's Omega = [0, 1]^2, Sec. 3.4): both strategies run to
    the same residual and agree on the distance; the two-grid fine solve needs fewer
    iterations than the single solve."""
    obs, pred = synth.gather_pair_hyperbolic()
    nr, nt = obs.shape
    dt, dx, tol = 1.0 / (nt - 1), 1.0 / (nr - 1), 1e-3
    d1, _, _, i1 = P.emd(_t(obs), _t(pred), dt, dx, max_iter=100000, tol=tol)
    d2, _, _, i2 = P.emd(_t(obs), _t(pred), dt, dx, max_iter=100000, tol=tol,
                         multigrid=dict(factor=4, coarse_max_iter=100000, coarse_tol=tol))
    assert i1["status"] == i2["status"] == P.EMD_OK
    assert i1["residual"] <= tol and i2["residual"] <= tol
    assert d2 == pytest.approx(d1, rel=2e-2)
    assert i2["iters"] < i1["iters"]
    o = O.pdhg(obs, pred, dt, dx, max_iter=100000, tol=tol)
    assert d2 == pytest.approx(o["dist"], rel=2e-2)


def test_two_grid_on_a_fresh_configuration_keeps_its_warm_start(P):
    """The first solve of a new gather size autotunes the tile shape with trial solves;
    those must not overwrite phi and m, which hold the interpolated warm start.  The first
    and the second call (shape cached) must agree."""
    obs, pred = synth.gather_pair_hyperbolic(nt=1004, nr=97, seed=77)
    runs = []
    for _ in range(2):
        d, phi, m, info = P.emd(_t(obs), _t(pred), 2e-3, 10.0, max_iter=120,
                                multigrid=dict(factor=4, coarse_max_iter=200))
        runs.append((d, phi.cpu().numpy(), info))
    (d1, p1, i1), (d2, p2, i2) = runs
    assert i1["iters"] == i2["iters"] == 120
    assert d1 == pytest.approx(d2, rel=1e-4)
    assert _rel_l2(p1, p2) <= 1e-3


def test_in_place_warm_start_on_a_fresh_configuration(P):
    """phi_init aliasing the phi output (and m_init the m output) on a first-use size: the
    autotuner's trial solves leave the outputs alone, so in-place and out-of-place warm
    starts give the same solve."""
    obs, pred = synth.gather_pair_hyperbolic(nt=1012, nr=99, seed=78)
    o, p = _t(obs), _t(pred)
    _, phi0, m0, _ = P.emd(o, p, 2e-3, 10.0, max_iter=50, tile=7)  # a warm start, fixed tile: no tuning
    ref_phi, ref_m = phi0.clone(), m0.clone()
    d_out, phi_out, _, i_out = P.emd(o, p, 2e-3, 10.0, max_iter=60, phi_init=ref_phi, m_init=ref_m, tile=7)
    nr, nt = obs.shape
    phi = phi0.clone()
    m = m0.clone()
    ws = P.new_workspace(P.emd_workspace_size(nt, nr), o.device)
    res = P.emd_dyn_solve(o, p, 2e-3, 10.0, P.emd_default_params(max_iter=60, phi_init=phi, m_init=m),
                          phi, m, ws)  # tile 0: first use of this size runs the autotuner
    assert res.iters == i_out["iters"] == 60
    assert res.dist == pytest.approx(d_out, rel=1e-4)
    assert _rel_l2(phi.cpu().numpy(), phi_out.cpu().numpy()) <= 1e-3


def test_batched_two_grid_equals_single(P):
    """Uneven gathers through one batched two-grid call against one call per gather."""
    gathers = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=s)
               for nt, nr, s in [(600, 40, 1), (1003, 70, 2), (257, 9, 3), (800, 130, 4)]]
    obs = [_t(a) for a, _ in gathers]
    pred = [_t(b) for _, b in gathers]
    mg = dict(factor=5, coarse_max_iter=300, coarse_tol=0.0)
    dists, phis, ms, infos = P.emd_batched(obs, pred, 2e-3, 10.0, max_iter=100, multigrid=mg)
    for b in range(len(gathers)):
        d, phi, m, info = P.emd(obs[b], pred[b], 2e-3, 10.0, max_iter=100, multigrid=mg)
        assert infos[b]["status"] == info["status"] == P.EMD_OK
        assert infos[b]["iters"] == info["iters"] == 100
        assert infos[b]["coarse"]["iters"] == info["coarse"]["iters"] == 300
        assert dists[b] == pytest.approx(d, rel=2e-3)
        assert _rel_l2(phis[b].cpu().numpy(), phi.cpu().numpy()) <= 2e-2
