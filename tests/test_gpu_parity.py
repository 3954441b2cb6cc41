"""CUDA path vs the FP64 oracle, element by element, through the C ABI (needs a GPU).

Tolerances: dist within 1e-4 relative and phi within 1e-3 relative L2 after the same
number of accepted iterations; u within 1e-3 relative L2; trial counts equal.  The GPU
iterates are FP32 (rounding 6e-8 per step) and its inner products FP32 within a warp,
FP64 above; the oracle is FP64 throughout.  On few-cell grids, whose answer moves by
more than 1e-4 under binary32 storage alone, the dist and u tolerances come from that
measured change (storage_rtol).
"""

import math
import multiprocessing as mp

import numpy as np
import pytest
import torch

import synth
from oracle import emd_oracle as O

pytestmark = pytest.mark.gpu

DIST_RTOL = 1e-4
PHI_RTOL = 1e-3


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07284_gb300 import build
    build.build()
    import paper_1808_07284_gb300 as P
    return P


def gpu_solve(P, obs, pred, dt, dx, trace=False, **kw):
    dev = torch.device("cuda:0")
    o = torch.from_numpy(np.ascontiguousarray(obs, np.float32)).to(dev)
    p = torch.from_numpy(np.ascontiguousarray(pred, np.float32)).to(dev)
    check = kw.pop("check", True)
    tr = None
    if trace:
        tr = torch.full((kw.get("max_iter", 2000), 4), float("nan"), dtype=torch.float64, device=dev)
        kw["trace"] = tr
    dist, phi, m, info = P.emd(o, p, dt, dx, check=check, **kw)
    torch.cuda.synchronize()
    m = m.double().cpu().numpy()
    out = dict(dist=dist, phi=phi.double().cpu().numpy(), ux=m[0], ut=m[1], info=info)
    if trace:
        out["trace"] = tr.cpu().numpy()
    return out


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_parity(g, r, trials=True, exact_trials=False, dist_rtol=DIST_RTOL, u_rtol=PHI_RTOL):
    """Same accepted iterations; the same linesearch trials (up to a rare near-tie decision
    unless exact_trials: the GPU tests the ratio of two FP64 sums of FP32 products, the
    oracle of FP64 norms); then dist, phi and u within the stated tolerances."""
    assert g["info"]["status"] == 0
    assert g["info"]["iters"] == r["iters"]
    if exact_trials:
        assert g["info"]["ls_trials"] == r["trials"]
    elif trials:
        assert abs(g["info"]["ls_trials"] - r["trials"]) <= max(2, r["trials"] // 1000)
    assert g["dist"] == pytest.approx(r["dist"], rel=dist_rtol)
    assert g["info"]["dist_l1"] == pytest.approx(r["dist_l1"], rel=dist_rtol)
    assert rel_l2(g["phi"], r["phi"]) <= PHI_RTOL
    u_g = np.concatenate([g["ux"].ravel(), g["ut"].ravel()])
    u_r = np.concatenate([r["ux"].ravel(), r["ut"].ravel()])
    assert rel_l2(u_g, u_r) <= u_rtol


def storage_rtol(r, obs, pred, dt, dx, **kw):
    """Distance and flux tolerances of an instance from its own conditioning: the oracle is
    rerun with its iterates rounded to binary32 after every iteration (the GPU's storage
    precision) and the relative changes of dist and u measured.  On a few-cell gather with the lateral flux still
    shut (dx = 10 m against dt = 2 ms), phi climbs as the dual ascent on the imbalance
    between receivers to O(1) while its time differences, which set u, stay near 1e-3, so
    that rounding alone moves dist by 2e-4 - 3e-4 and u by 4e-4 - 9e-4; on gathers of more
    than a few dozen cells both by about 1e-8 - 1e-6.  The GPU rounds at more points of a
    pass than the model (w, div w and the dual update besides the stored iterates), each a
    perturbation of the same size: it is allowed four times the model's change, and never
    less than DIST_RTOL and PHI_RTOL."""
    q = O.pdhg(obs, pred, dt, dx, store_f32=True, **kw)
    assert q["iters"] == r["iters"] and q["trials"] == r["trials"]
    u_q = np.concatenate([q["ux"].ravel(), q["ut"].ravel()])
    u_r = np.concatenate([r["ux"].ravel(), r["ut"].ravel()])
    return dict(dist_rtol=max(DIST_RTOL, 4.0 * abs(q["dist"] - r["dist"]) / r["dist"]),
                u_rtol=max(PHI_RTOL, 4.0 * rel_l2(u_q, u_r)))


NEAR_TIE = 1e-3  # relative gap |lhs - rhs| / rhs of a linesearch test that counts as a tie
# Runs that approach convergence over thousands of iterations (normalised domain, residual
# 1e-2): the linesearch quantities there are small differences of FP32 iterates, so the two
# sides of a replayed decision can sit 1e-3 - 1e-2 apart (largest measured: 2.3e-3 on a
# 4,810-iteration gather) while both branches remain valid steps of the method.
NEAR_TIE_CONVERGING = 1e-2


def feasibility_bound(g, r, dt, dx):
    """Largest |r_feas(GPU) - r_feas(oracle)| the two final iterates allow: both are
    ||div u + f|| / ||f|| of their own u, so by the triangle inequality they differ by at
    most ||div(u_gpu - u_oracle)|| / ||f||.  The residual is a small difference of O(|f|)
    terms, so the iterates' relative drift shows up in it magnified about 1 / r_feas
    times."""
    d = O.divergence(g["ux"] - r["ux"], g["ut"] - r["ut"], dt, dx)
    return float(np.linalg.norm(d) / np.linalg.norm(r["f"]))


def assert_feasibility_close(g, r, dt, dx):
    """The GPU's reported r_feas (an FP64 sum of FP32 terms, FP32 f) within the bound above,
    plus 1e-6 for the FP32 rounding of f and the sum."""
    bound = feasibility_bound(g, r, dt, dx)
    assert abs(g["info"]["r_feas"] - r["r_feas"]) <= 1.05 * bound + 1e-6 * (1 + r["r_feas"]), (
        g["info"]["r_feas"], r["r_feas"], bound)


def replay_parity(P, obs, pred, dt, dx, K, gpu_kw=None, **kw):
    """Fixed-count parity over the whole run, with the GPU's decisions replayed.

    The GPU runs K iterations and records each iteration's linesearch trial count; the
    FP64 oracle then runs the same K iterations taking exactly those counts
    (force_trials) while still evaluating its own test.  Where the two sides of
    Algorithm 1's test nearly tie, FP32 iterates may take the other branch, and both
    branches are valid iterations of the method: every trial on which the oracle's own
    test disagrees with the GPU's choice must be such a tie (relative gap < NEAR_TIE).
    Then the step sizes agree to 1e-9 at every iteration, the feasibility residual to 1e-2
    at every iteration (it magnifies the iterates' drift about 1 / r_feas times; the final
    one is held to the exact bound of assert_feasibility_close), and the final distance,
    phi and u within the stated tolerances.
    Returns (gpu run, oracle replay, first iteration the oracle would have decided
    otherwise or K).  gpu_kw: launch options of the GPU side only (tile, launch_mode)."""
    gk = dict(gpu_kw or {})
    g = gpu_solve(P, obs, pred, dt, dx, max_iter=K, trace=True, **kw, **gk)
    assert g["info"]["status"] == 0 and g["info"]["iters"] == K
    forced = g["trace"][:K, 2].astype(int)
    r = O.pdhg(obs, pred, dt, dx, max_iter=K, record=True, force_trials=forced, **kw)
    ot, gt = r["trace"], g["trace"][:K]
    dis = ot[:, 6]
    assert dis.max() < NEAR_TIE, f"iteration {int(np.argmax(dis))}: decided otherwise away from a tie"
    np.testing.assert_allclose(gt[:, 0], ot[:, 0], rtol=1e-9)
    np.testing.assert_allclose(gt[:, 1], ot[:, 1], rtol=1e-9)
    np.testing.assert_allclose(gt[:, 3], ot[:, 3], rtol=1e-2, atol=1e-7)
    assert_parity(g, r, exact_trials=True)
    assert_feasibility_close(g, r, dt, dx)
    first = int(np.argmax(dis > 0)) if (dis > 0).any() else K
    return g, r, first


def test_small_gather_2000_iterations(pkg, capsys):
    """Hyperbolic 256 x 64 gather, dt = 2 ms, dx = 10 m, mean balance, Algorithm 1, 2000
    fixed iterations: every decision replayed, dist within 1e-4, phi and u within 1e-3 at
    iteration 2000; the FP64 mass sums, the residual and the duality gap."""
    obs, pred = synth.gather_pair_hyperbolic()
    g, r, first = replay_parity(pkg, obs, pred, 2e-3, 10.0, 2000)
    with capsys.disabled():
        print(f"\n256x64, 2000 iterations: first decision the oracle would take otherwise: {first}; "
              f"contradicted iterations {int((r['trace'][:, 6] > 0).sum())}, largest gap "
              f"{r['trace'][:, 6].max():.2e}; dist rel {abs(g['dist'] - r['dist']) / r['dist']:.2e}, "
              f"phi rel {rel_l2(g['phi'], r['phi']):.2e}")
    info = g["info"]
    assert info["mass_mu"] == pytest.approx(2e-3 * 10.0 * O.mainini(obs, pred)[0].sum(), rel=1e-12)
    assert info["mass_nu"] == pytest.approx(2e-3 * 10.0 * O.mainini(obs, pred)[1].sum(), rel=1e-12)
    assert info["imbalance"] == pytest.approx(r["imbalance"], rel=1e-9, abs=1e-12)
    # r_step = ||u^K - u^{K-1}|| / ||u^K|| magnifies the drift by ||u|| / ||du|| the same way
    assert info["r_step"] == pytest.approx(r["r_step"], rel=5e-2)
    assert info["residual"] == pytest.approx(r["residual"], rel=5e-2)
    assert info["duality_gap"] == pytest.approx(r["gap"], rel=1e-3)


def test_small_gather_normalised_domain(pkg):
    """Same gather on Omega = [0,1]^2 (dt = 1/(nt-1), dx = 1/(nr-1)) as in the paper's runs."""
    obs, pred = synth.gather_pair_hyperbolic()
    dt, dx = 1 / 255, 1 / 63
    r = O.pdhg(obs, pred, dt, dx, max_iter=500)
    g = gpu_solve(pkg, obs, pred, dt, dx, max_iter=500)
    assert_parity(g, r)


SHAPES = [(1, 2), (1, 37), (2, 2), (3, 5), (17, 130), (33, 251), (9, 1000), (40, 121)]


@pytest.mark.parametrize("tile", [0, 10])
@pytest.mark.parametrize("nr,nt", SHAPES)
def test_ragged_shapes(pkg, nr, nt, tile):
    """Ragged and degenerate grids (one receiver, two samples, a partial last strip) with
    the automatic choice and with the marching solve forced."""
    rng = np.random.default_rng(nr * 1000 + nt)
    obs, pred = synth.gather_pair_hyperbolic(nt=max(nt, 8), nr=nr, dt=2e-3, seed=nr + nt)
    obs, pred = obs[:, :nt].copy(), pred[:, :nt].copy()
    pred += 0.05 * rng.standard_normal(pred.shape).astype(np.float32)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=150)
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=150, tile=tile)
    assert_parity(g, r, **storage_rtol(r, obs, pred, 2e-3, 10.0, max_iter=150))
    if tile:
        assert g["info"]["tile"] == tile


MARCH = 10  # tile id of the first marching-solve shape (11 marching warps, 6 rows in flight)


@pytest.mark.parametrize("tile", range(1, 12))
def test_every_tile_shape(pkg, tile):
    """Each compiled tile shape gives the oracle's iterates on a gather spanning several
    tiles (shapes 10 and 11: the marching solve, several strips and segments)."""
    assert tile <= pkg.emd_tile_count()
    obs, pred = synth.gather_pair_hyperbolic(nt=300, nr=37, seed=5)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=120)
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=120, tile=tile)
    assert_parity(g, r)


def test_fixed_step_mode(pkg):
    obs, pred = synth.gather_pair_hyperbolic(nt=128, nr=24, seed=3)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=400, linesearch=0)
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=400, linesearch=0)
    assert_parity(g, r)


def test_no_balancing(pkg):
    obs, pred = synth.gather_pair_hyperbolic(nt=128, nr=16, seed=4)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=300, balance=O.BAL_NONE)
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=300, balance=0)
    assert_parity(g, r)


@pytest.mark.parametrize("nt,nr", [(200, 20), (600, 40)])
@pytest.mark.parametrize("tol", [0.0, 1e-2])
def test_launch_modes_agree(pkg, tol, nt, nr):
    """Automatic (0: the shared-memory solve for 200 x 20, one persistent launch for
    600 x 40), plain per-pass launches (1) and graph replays (2) run the same iteration,
    with a fixed count and with a tolerance stop."""
    obs, pred = synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=6)
    dt, dx = (2e-3, 10.0) if tol == 0 else (1 / (nt - 1), 1 / (nr - 1))
    runs = [gpu_solve(pkg, obs, pred, dt, dx, max_iter=130 if tol == 0 else 20000, tol=tol,
                      launch_mode=m) for m in (0, 1, 2)]
    for r in runs:
        assert r["info"]["status"] == 0
        assert r["info"]["iters"] == runs[0]["info"]["iters"]
        assert r["info"]["ls_trials"] == runs[0]["info"]["ls_trials"]
        assert r["dist"] == pytest.approx(runs[0]["dist"], rel=1e-9)
        assert rel_l2(r["phi"], runs[0]["phi"]) <= 1e-6
    if tol == 0:
        assert runs[0]["info"]["iters"] == 130
    else:
        assert runs[0]["info"]["residual"] <= tol and runs[0]["info"]["iters"] < 20000


def test_tolerance_stopping(pkg):
    """tol > 0 stops at the first multiple of check_every whose residual is <= tol
    (normalised domain, where FP32 iterates resolve the steps; see the precision notes).
    The oracle replays the GPU's decisions up to its stop: the iterates agree there, the
    oracle's own residual is <= tol at the stop and above it at every earlier check,
    unless within 1e-2 of tol (the per-iteration residual tolerance of replay_parity)."""
    obs, pred = synth.gather_pair_hyperbolic(nt=96, nr=12, seed=3)
    dt, dx = 1 / 95, 1 / 11
    g = gpu_solve(pkg, obs, pred, dt, dx, max_iter=8000, tol=1e-2, check_every=10, trace=True)
    K = g["info"]["iters"]
    assert K % 10 == 0 and K < 8000 and g["info"]["residual"] <= 1e-2
    r = O.pdhg(obs, pred, dt, dx, max_iter=K, record=True, force_trials=g["trace"][:K, 2].astype(int))
    assert r["trace"][:, 6].max() < NEAR_TIE
    assert_parity(g, r, exact_trials=True)
    res = np.maximum(r["trace"][:, 3], r["trace"][:, 4])
    checks = res[9::10]
    assert checks[-1] <= 1e-2 * (1 + 1e-2)
    assert (checks[:-1] > 1e-2 * (1 - 1e-2)).all()
    assert_feasibility_close(g, r, dt, dx)


def test_warm_start(pkg):
    obs, pred = synth.gather_pair_hyperbolic(nt=96, nr=10, seed=8)
    rng = np.random.default_rng(1)
    phi0 = (0.01 * rng.standard_normal(obs.shape)).astype(np.float32)
    m0 = (0.001 * rng.standard_normal((2,) + obs.shape)).astype(np.float32)
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=100, phi_init=phi0.astype(float),
               m_init=np.stack([np.where(np.arange(10)[:, None] > 0, m0[0], 0),
                                np.where(np.arange(96)[None, :] > 0, m0[1], 0)]))
    dev = torch.device("cuda:0")
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=100,
                  phi_init=torch.from_numpy(phi0).to(dev), m_init=torch.from_numpy(m0).to(dev))
    assert_parity(g, r)


def test_1d_shift_sweep_matches_closed_form(pkg):
    """nt = 1024 on [0, 1] (dt = 1/(nt-1)), 8 Hz Ricker shifted: the same iterates as the
    oracle after 800 iterations (decisions replayed), and, run on, the distance of the
    closed-form W1."""
    dt, obs, preds = synth.shift_sweep_1d(nt=1024, shifts=[-0.06, 0.03, 0.2])
    for s, pred in preds:
        replay_parity(pkg, obs, pred, dt, 1.0, 800)
        f = O.source_term(obs, pred)[0]
        w = O.w1_1d(np.maximum(f, 0), np.maximum(-f, 0), dt)
        c = gpu_solve(pkg, obs, pred, dt, 1.0, max_iter=200000, tol=1e-7)
        assert c["info"]["dist_l1"] == pytest.approx(w, rel=1e-3), (s, c["info"])


@pytest.mark.parametrize("case,tile", [("1d", 0), ("2d", 0), ("2d", 7), ("2d", MARCH)])
def test_identical_gathers(pkg, case, tile):
    """Reading Q20 on every solver path: identical gathers make p and q identically zero, so the
    step stays at alpha_0 (theta = 1, one trial per iteration) as in the oracle.  After 2500
    iterations, past the point where a growing step overflows, phi and m are exactly zero and
    finite, the distance is 0, and the adjoint source is zero."""
    if case == "1d":
        dt, obs, _ = synth.shift_sweep_1d(nt=1024, shifts=[0.1])
        dx = 1.0
    else:
        obs, _ = synth.gather_pair_hyperbolic()
        dt, dx = 2e-3, 10.0
    K = 2500
    g = gpu_solve(pkg, obs, obs.copy(), dt, dx, max_iter=K, trace=True, tile=tile)
    r = O.pdhg(obs, obs.copy(), dt, dx, max_iter=K, record=True)
    info = g["info"]
    assert info["status"] == 0 and info["iters"] == K and info["ls_trials"] == K == r["trials"]
    np.testing.assert_allclose(g["trace"][:, 0], r["trace"][:, 0], rtol=1e-15)
    np.testing.assert_array_equal(g["trace"][:, 1], 1.0)
    for key in ("phi", "ux", "ut"):
        assert np.all(g[key] == 0.0), key
    assert g["dist"] == 0.0 and info["dist_l1"] == 0.0
    if tile:
        assert info["tile"] == tile
    dev = torch.device("cuda:0")
    o = torch.from_numpy(obs).to(dev)
    pr = o.clone().requires_grad_(True)
    pkg.emd_loss(pr, o, dt, dx, max_iter=300).backward()
    assert torch.all(pr.grad == 0.0)


def test_decompose(pkg):
    obs, pred = synth.gather_pair_transmissive(nt=500, nr=40, seed=9)
    dev = torch.device("cuda:0")
    o = torch.from_numpy(obs).to(dev)
    p = torch.from_numpy(pred).to(dev)
    mu = torch.empty_like(o)
    nu = torch.empty_like(o)
    mm, mn = pkg.emd_decompose(o, p, 1e-3, 12.5, mu, nu)
    # elementwise in FP32: max and one add, the same operations the oracle does in FP64
    mu_ref = np.maximum(pred, 0) + np.maximum(-obs, 0)
    nu_ref = np.maximum(obs, 0) + np.maximum(-pred, 0)
    np.testing.assert_array_equal(mu.cpu().numpy(), mu_ref.astype(np.float32))
    np.testing.assert_array_equal(nu.cpu().numpy(), nu_ref.astype(np.float32))
    m64, n64 = O.mainini(obs, pred)
    assert mm == pytest.approx(1e-3 * 12.5 * m64.sum(), rel=1e-12)
    assert mn == pytest.approx(1e-3 * 12.5 * n64.sum(), rel=1e-12)


def test_adjoint_and_autograd(pkg):
    obs, pred = synth.gather_pair_hyperbolic(nt=128, nr=16, seed=10)
    dt, dx = 2e-3, 10.0
    dev = torch.device("cuda:0")
    o = torch.from_numpy(obs).to(dev).requires_grad_(True)
    p = torch.from_numpy(pred).to(dev).requires_grad_(True)
    loss = pkg.emd_loss(p, o, dt, dx, max_iter=300)
    (3.0 * loss).backward()
    r = O.pdhg(obs, pred, dt, dx, max_iter=300)
    g_ref, go_ref = O.adjoint_source(r["phi"], dt, dx, grad_out=3.0)
    assert loss.item() == pytest.approx(r["dist"], rel=DIST_RTOL)
    assert rel_l2(p.grad.double().cpu().numpy(), g_ref) <= PHI_RTOL
    assert rel_l2(o.grad.double().cpu().numpy(), go_ref) <= PHI_RTOL
    gp = p.grad.double().cpu().numpy()
    assert abs(gp.mean()) <= 1e-6 * np.abs(gp).max()


def test_batched_equals_single(pkg):
    """Uneven gathers solved together give each gather's own single-solve result."""
    pairs = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=s)
             for s, (nt, nr) in enumerate([(200, 17), (96, 40), (333, 9), (64, 1)])]
    dev = torch.device("cuda:0")
    O_ = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    P_ = [torch.from_numpy(p).to(dev) for _, p in pairs]
    d, phis, ms, infos = pkg.emd_batched(O_, P_, 2e-3, 10.0, max_iter=200)
    for b, (o, p) in enumerate(pairs):
        r = O.pdhg(o, p, 2e-3, 10.0, max_iter=200)
        g = dict(dist=d[b], phi=phis[b].double().cpu().numpy(), ux=ms[b][0].double().cpu().numpy(),
                 ut=ms[b][1].double().cpu().numpy(), info=infos[b])
        assert_parity(g, r)


def test_batched_with_tolerance_stops_each_gather(pkg):
    """Gathers in one batch stop independently at their own tolerance crossing: each one
    gives the same iterations and distance as its own single solve, and the oracle's
    stopping iteration is close to it."""
    shapes = [(96, 12, 3), (72, 12, 6), (100, 10, 8)]
    pairs = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=s) for nt, nr, s in shapes]
    dts = [1 / (nt - 1) for nt, _, _ in shapes]
    dxs = [1 / (nr - 1) for _, nr, _ in shapes]
    dev = torch.device("cuda:0")
    O_ = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    P_ = [torch.from_numpy(p).to(dev) for _, p in pairs]
    d, phis, ms, infos = pkg.emd_batched(O_, P_, dts, dxs, max_iter=8000, tol=1e-2)
    its = [i["iters"] for i in infos]
    assert len(set(its)) > 1  # the gathers stop at different iterations
    for b, (o, p) in enumerate(pairs):
        assert infos[b]["residual"] <= 1e-2 and its[b] < 8000 and its[b] % 10 == 0
        single = gpu_solve(pkg, o, p, dts[b], dxs[b], max_iter=8000, tol=1e-2)
        assert single["info"]["iters"] == its[b]
        assert single["dist"] == pytest.approx(d[b], rel=1e-9)
        assert rel_l2(phis[b].double().cpu().numpy(), single["phi"]) <= 1e-6
        r = O.pdhg(o, p, dts[b], dxs[b], max_iter=8000, tol=1e-2)
        assert abs(its[b] - r["iters"]) <= 0.2 * r["iters"]


@pytest.mark.parametrize("tile", [7, MARCH])
def test_batched_tolerance_rebalanced(pkg, tile):
    """Four gathers above the shared-memory size, solved as one batch to residual 1e-2 on
    the normalised domain: they stop after about 1200, 1500, 2400 and 4800 iterations, so
    the persistent solve, run in chunks, deals the running gathers' tiles over the CTAs
    again three times.  Each gather equals the oracle replaying its own decisions, and
    stops at the first check where the oracle's own residual is <= tol."""
    cases = [(240, 40, 3), (300, 36, 6), (180, 50, 8), (200, 44, 12)]
    pairs = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=s) for nt, nr, s in cases]
    dts = [1 / (nt - 1) for nt, _, _ in cases]
    dxs = [1 / (nr - 1) for _, nr, _ in cases]
    dev = torch.device("cuda:0")
    O_ = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    P_ = [torch.from_numpy(p).to(dev) for _, p in pairs]
    kmax = 20000
    tr = torch.full((len(cases), kmax, 4), float("nan"), dtype=torch.float64, device=dev)
    d, phis, ms, infos = pkg.emd_batched(O_, P_, dts, dxs, max_iter=kmax, tol=1e-2, trace=tr, tile=tile)
    trb = tr.cpu().numpy()
    its = [i["iters"] for i in infos]
    assert len(set(its)) == len(its) and max(its) > 2 * 160  # several chunks, stops apart
    assert infos[0]["launches"] > 3  # prepare, more than one chunk, finalize
    for b, (o, p) in enumerate(pairs):
        K = its[b]
        assert infos[b]["status"] == 0 and infos[b]["residual"] <= 1e-2 and K % 10 == 0
        gb = dict(dist=d[b], phi=phis[b].double().cpu().numpy(), ux=ms[b][0].double().cpu().numpy(),
                  ut=ms[b][1].double().cpu().numpy(), info=infos[b])
        r = O.pdhg(o, p, dts[b], dxs[b], max_iter=K, record=True, force_trials=trb[b, :K, 2].astype(int))
        assert r["trace"][:, 6].max() < NEAR_TIE_CONVERGING
        assert_parity(gb, r, exact_trials=True)
        res = np.maximum(r["trace"][:, 3], r["trace"][:, 4])[9::10]
        assert res[-1] <= 1e-2 * (1 + 1e-2) and (res[:-1] > 1e-2 * (1 - 1e-2)).all()


@pytest.mark.parametrize("nt,nr,gpu_kw", [
    (300, 24, dict(tile=7)),         # persistent TMA solve (decider warp)
    (300, 24, dict(tile=MARCH)),     # marching solve
    (300, 24, dict(launch_mode=1)),  # per-pass launches (last CTA decides)
    (256, 16, {}),                   # whole solve in one CTA's shared memory
])
def test_backtracking_past_32_trials(pkg, nt, nr, gpu_kw):
    """An initial step 1000 / sqrt(delta lambda) with xi = 0.9: the first decision takes 45
    trials in the oracle's sequential backtracking, so the deciding warp's first round of
    32 lane-parallel trials (whose step sizes are prepared per lane) all fail and the
    second round, evaluated from the scaled coefficients, must pick the same trial.  The
    later decisions take 1-25 trials.  Element parity after 60 iterations, decisions replayed."""
    obs, pred = synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=9)
    dt, dx = 2e-3, 10.0
    lam = 4.0 / dx ** 2 + 4.0 / dt ** 2
    kw = dict(alpha0=1000.0 / math.sqrt(1e5 * lam), xi=0.9, ls_max_trials=120)
    first = O.pdhg(obs, pred, dt, dx, max_iter=1, record=True, **kw)
    assert int(first["trace"][0, 2]) > 32
    replay_parity(pkg, obs, pred, dt, dx, 60, gpu_kw=gpu_kw, **kw)


@pytest.mark.parametrize("tile", [MARCH, MARCH + 1])
def test_march_large_gather_replay(pkg, tile):
    """The marching solve on the 8000 x 648 marine gather (several segments per strip, one
    unit per warp) and on a 4-shot batch of uneven gathers (many units per warp, warps
    crossing gathers): 40 iterations, decisions replayed, element parity per gather."""
    o, p = synth.gather_pair_marine(shot=3)
    replay_parity(pkg, o, p, 2e-3, 25.0, 40, gpu_kw=dict(tile=tile))
    pairs = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=s) for nt, nr, s in
             [(1500, 333, 1), (2007, 200, 2), (977, 517, 3), (3001, 64, 4)]]
    dev = torch.device("cuda:0")
    O_ = [torch.from_numpy(a).to(dev) for a, _ in pairs]
    P_ = [torch.from_numpy(b).to(dev) for _, b in pairs]
    K = 60
    tr = torch.full((len(pairs), K, 4), float("nan"), dtype=torch.float64, device=dev)
    d, phis, ms, infos = pkg.emd_batched(O_, P_, 1e-3, 12.5, max_iter=K, trace=tr, tile=tile)
    trb = tr.cpu().numpy()
    for b, (a, q) in enumerate(pairs):
        gb = dict(dist=d[b], phi=phis[b].double().cpu().numpy(), ux=ms[b][0].double().cpu().numpy(),
                  ut=ms[b][1].double().cpu().numpy(), info=infos[b])
        r = O.pdhg(a, q, 1e-3, 12.5, max_iter=K, record=True, force_trials=trb[b, :, 2].astype(int))
        assert r["trace"][:, 6].max() < NEAR_TIE
        assert_parity(gb, r, exact_trials=True)


def test_nan_input_reports_nonfinite(pkg):
    obs, pred = synth.gather_pair_hyperbolic(nt=64, nr=8)
    pred[3, 10] = np.nan
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=50, check=False)
    assert g["info"]["status"] == pkg.EMD_ERR_NONFINITE


def test_linesearch_failure_is_reported(pkg):
    obs, pred = synth.gather_pair_hyperbolic(nt=64, nr=8)
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=50, debug_fault=1, check=False)
    assert g["info"]["status"] == pkg.EMD_ERR_LINESEARCH
    assert g["info"]["iters"] == 0 and g["info"]["ls_trials"] == 40


@pytest.mark.parametrize("tile", [7, MARCH])
def test_device_wait_timeout_is_reported_and_the_context_survives(pkg, tile):
    """debug_fault = 2: the persistent solve's decisions are never published, so the
    compute warps' bounded wait on the decision counter (4 s of %globaltimer) runs out.
    The solve returns EMD_ERR_TIMEOUT instead of hanging, and the next solve on the same
    CUDA context is correct."""
    obs, pred = synth.gather_pair_hyperbolic(nt=600, nr=40, seed=6)
    g = gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=50, tile=tile, debug_fault=2, check=False)
    assert g["info"]["status"] == pkg.EMD_ERR_TIMEOUT
    r = O.pdhg(obs, pred, 2e-3, 10.0, max_iter=50)
    assert_parity(gpu_solve(pkg, obs, pred, 2e-3, 10.0, max_iter=50, tile=tile), r)


def test_transmissive_full_size_sampled(pkg):
    """The 3000 x 400 gather at full size: same iterates as the oracle after 25 iterations."""
    obs, pred = synth.gather_pair_transmissive()
    r = O.pdhg(obs, pred, 1e-3, 12.5, max_iter=25)
    g = gpu_solve(pkg, obs, pred, 1e-3, 12.5, max_iter=25)
    assert_parity(g, r)


def test_transmissive_converged_properties(pkg):
    """The 3000 x 400 gather on Omega = [0,1]^2 run to residual 1e-3; then feasibility, the
    distance and the duality gap recomputed on the host in FP64 from the returned u, phi."""
    obs, pred = synth.gather_pair_transmissive()
    dt, dx = 1 / 2999, 1 / 399
    g = gpu_solve(pkg, obs, pred, dt, dx, max_iter=100000, tol=1e-3)
    info = g["info"]
    assert info["status"] == 0 and info["residual"] <= 1e-3 and info["iters"] < 100000
    f = O.source_term(obs, pred)
    res = O.divergence(g["ux"], g["ut"], dt, dx) + f
    assert np.linalg.norm(res) / np.linalg.norm(f) == pytest.approx(info["r_feas"], rel=0.05, abs=2e-6)
    val, l1 = O.objective(g["ux"], g["ut"], 1e-4)
    assert info["dist"] == pytest.approx(dx * dt * val, rel=1e-5)
    assert info["dist_l1"] == pytest.approx(dx * dt * l1, rel=1e-5)
    gap = O.duality_gap(g["ux"], g["ut"], g["phi"], f, 1e-4, dt, dx)
    assert info["duality_gap"] == pytest.approx(gap, rel=2e-2, abs=1e-3 * info["dist"])


def test_converged_crop_against_oracle(pkg, capsys):
    """Converged parity on a 128 x 400 crop of the transmissive gather on the paper's
    normalised domain (Omega = [0,1]^2): the GPU and the FP64 oracle each run Algorithm 1
    on their own decisions to residual 1e-4 (about 41,000 iterations).  Both stop within
    one percent of the same iteration and below 1e-4, and the converged distance, phi and u
    agree within 1e-4 / 1e-3.  (Replaying the GPU's decisions does not reach this far: near
    convergence the steps shrink below the FP32 iterates' drift, so the two sides' test
    values stop tracking each other, while both runs still converge to the same point.)"""
    obs, pred = synth.gather_pair_transmissive()
    o, p = obs[100:228, 600:1000].copy(), pred[100:228, 600:1000].copy()
    nr, nt = o.shape
    dt, dx = 1 / (nt - 1), 1 / (nr - 1)
    g = gpu_solve(pkg, o, p, dt, dx, max_iter=100000, tol=1e-4)
    r = O.pdhg(o, p, dt, dx, max_iter=100000, tol=1e-4)
    info = g["info"]
    assert info["status"] == 0 and info["residual"] <= 1e-4 and r["residual"] <= 1e-4
    assert abs(info["iters"] - r["iters"]) <= 0.01 * r["iters"]
    assert g["dist"] == pytest.approx(r["dist"], rel=DIST_RTOL)
    assert rel_l2(g["phi"], r["phi"]) <= PHI_RTOL
    u_g = np.concatenate([g["ux"].ravel(), g["ut"].ravel()])
    u_r = np.concatenate([r["ux"].ravel(), r["ut"].ravel()])
    assert rel_l2(u_g, u_r) <= PHI_RTOL
    with capsys.disabled():
        print(f"\n128x400 normalised, tol 1e-4: iterations gpu {info['iters']} oracle {r['iters']}; residual gpu "
              f"{info['residual']:.3e} oracle {r['residual']:.3e}; dist rel {abs(g['dist'] - r['dist']) / r['dist']:.2e}; "
              f"phi rel {rel_l2(g['phi'], r['phi']):.2e}; u rel {rel_l2(u_g, u_r):.2e}")


# ----------------------------------------------------------------------------- differentiable misfit

def test_gradient_matches_oracle_finite_differences(pkg):
    """A 64 x 32 crop of the reflective gather on Omega = [0,1]^2, solved to a tight
    residual: the GPU adjoint source (EMDFunction backward) against central finite
    differences (eps = 1e-3, FP64) of the converged oracle distance, and against the
    oracle's own adjoint source.  (With the physical 1 ms / 12.5 m spacings PDHG does not
    converge in any affordable iteration count, FP64 included; see the design notes.)"""
    obs, pred = synth.gather_pair_reflective(shot=0)
    o = obs[0:32, 180:244].astype(np.float64)
    p = pred[0:32, 180:244].astype(np.float64)
    dt, dx = 1 / 63, 1 / 31
    kw = dict(max_iter=60000, tol=1e-9)
    base = O.pdhg(o, p, dt, dx, **kw)
    assert base["residual"] <= 1e-8
    g_orc, _ = O.adjoint_source(base["phi"], dt, dx)
    dev = torch.device("cuda:0")
    to = torch.from_numpy(o.astype(np.float32)).to(dev)
    tp = torch.from_numpy(p.astype(np.float32)).to(dev).requires_grad_(True)
    loss = pkg.emd_loss(tp, to, dt, dx, max_iter=200000, tol=1e-7)
    loss.backward()
    g = tp.grad.double().cpu().numpy()
    assert loss.item() == pytest.approx(base["dist"], rel=1e-4)
    assert rel_l2(g, g_orc) <= 2e-2
    h = 1e-3
    scale = np.abs(g_orc).max()
    for (i, j) in [(5, 20), (12, 30), (20, 40), (27, 10)]:
        p1, p2 = p.copy(), p.copy()
        p1[i, j] += h
        p2[i, j] -= h
        fd = (O.pdhg(o, p1, dt, dx, **kw)["dist"] - O.pdhg(o, p2, dt, dx, **kw)["dist"]) / (2 * h)
        assert g[i, j] == pytest.approx(fd, abs=2e-2 * scale), (i, j)


def _replay_reflective(shot, trials, w, K):
    """The oracle on reflective shot `shot` with the GPU's trial counts (a spawn-pool worker):
    distance, adjoint source for upstream weight w, and the replay trace."""
    obs, pred = synth.gather_pair_reflective(shot=shot)
    r = O.pdhg(obs, pred, 1e-3, 12.5, max_iter=K, record=True, force_trials=np.asarray(trials, np.int64))
    g, _ = O.adjoint_source(r["phi"], 1e-3, 12.5, grad_out=w)
    return r["dist"], g.astype(np.float32), r["trace"]


def test_batched_autograd_reflective_16x4000x480(pkg):
    """Sixteen reflective gathers of 4000 x 480 (dt = 1 ms, dx = 12.5 m) through the batched
    autograd function at 200 iterations (the paper runs 100-200 per EMD), each distance
    weighted differently in the loss.  Three sampled gathers against the FP64 oracle replaying
    the GPU's decisions: every contradicted decision a near tie, step sizes to 1e-9, distance
    within 1e-4 and the weighted adjoint source within 1e-3.  Batched and single solves of a
    gather agree to 1e-5 where they took the same decisions."""
    K = 200
    dev = torch.device("cuda:0")
    pairs = [synth.gather_pair_reflective(shot=s) for s in range(16)]
    obs = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    preds = [torch.from_numpy(p).to(dev).requires_grad_(True) for _, p in pairs]
    trace = torch.full((16, K, 4), float("nan"), dtype=torch.float64, device=dev)
    d = pkg.emd_loss_batched(preds, obs, 1e-3, 12.5, max_iter=K, trace=trace)
    assert d.shape == (16,) and torch.isfinite(d).all()
    w = torch.linspace(0.5, 2.0, 16, device=dev)
    (w * d).sum().backward()
    tr = trace.cpu().numpy()
    sampled = (0, 7, 15)
    with mp.get_context("spawn").Pool(len(sampled)) as pool:
        jobs = {b: pool.apply_async(_replay_reflective, (b, tr[b, :, 2].astype(int).tolist(), float(w[b]), K))
                for b in sampled}
        for b in sampled:
            single_tr = torch.full((K, 4), float("nan"), dtype=torch.float64, device=dev)
            single = pkg.emd_loss(preds[b].detach().clone().requires_grad_(True), obs[b], 1e-3, 12.5,
                                  max_iter=K, trace=single_tr)
            if np.array_equal(single_tr.cpu().numpy()[:, 2], tr[b, :, 2]):
                assert d[b].item() == pytest.approx(single.item(), rel=1e-5)
        for b, job in jobs.items():
            dist, g_ref, otr = job.get()
            assert otr[:, 6].max() < NEAR_TIE, (b, int(np.argmax(otr[:, 6])))
            np.testing.assert_allclose(tr[b, :, 0], otr[:, 0], rtol=1e-9)
            assert d[b].item() == pytest.approx(dist, rel=DIST_RTOL)
            assert rel_l2(preds[b].grad.double().cpu().numpy(), g_ref.astype(np.float64)) <= PHI_RTOL


def test_host_misfit_matches_device_path_and_oracle(pkg):
    """emd_misfit_batched_host (host gathers in, distances and adjoint sources out) on five
    gathers of mixed, ragged sizes, four page-locked and one pageable: the same distances,
    trial counts and adjoint sources as the device-pointer batched solve plus batched
    adjoint on the same data, and two sampled gathers equal to the oracle (distance, and
    adjoint source dx dt (phi - mean phi)) after the same 150 iterations."""
    dev = torch.device("cuda:0")
    sizes = [(300, 37, 5), (128, 24, 6), (141, 5, 7), (64, 1, 8), (1000, 9, 9)]
    pairs = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=sd) for nt, nr, sd in sizes]
    dts, dxs = [2e-3] * 5, [10.0] * 5
    h_obs = [torch.from_numpy(o).pin_memory() for o, _ in pairs]
    h_pred = [torch.from_numpy(p).pin_memory() if b != 2 else torch.from_numpy(p.copy())
              for b, (_, p) in enumerate(pairs)]
    assert not h_pred[2].is_pinned()
    dists, grads, infos = pkg.emd_misfit_host(h_obs, h_pred, dts, dxs, max_iter=150)
    assert all(i["status"] == 0 and i["iters"] == 150 for i in infos)
    d_obs = [t.to(dev) for t in h_obs]
    d_pred = [t.to(dev) for t in h_pred]
    dd, phis, _ms, dinfos = pkg.emd_batched(d_obs, d_pred, dts, dxs, max_iter=150)
    gps = [torch.empty_like(t) for t in phis]
    ws = pkg.new_workspace(pkg.emd_batched_adjoint_workspace_size(5), dev)
    pkg.emd_adjoint_batched(phis, dts, dxs, pkg.EMD_BAL_MEAN, None, gps, None, ws)
    torch.cuda.synchronize()
    for b in range(5):
        assert infos[b]["ls_trials"] == dinfos[b]["ls_trials"] and infos[b]["tile"] == dinfos[b]["tile"]
        assert dists[b] == pytest.approx(dd[b], rel=1e-6)
        assert rel_l2(grads[b].double().numpy(), gps[b].double().cpu().numpy()) <= 1e-5
    for b in (0, 2):
        o, p = pairs[b]
        r = O.pdhg(o, p, dts[b], dxs[b], max_iter=150)
        g_ref, _ = O.adjoint_source(r["phi"], dts[b], dxs[b])
        assert dists[b] == pytest.approx(r["dist"], rel=DIST_RTOL)
        assert rel_l2(grads[b].double().numpy(), g_ref) <= PHI_RTOL
    only, none, _ = pkg.emd_misfit_host(h_obs, h_pred, dts, dxs, adjoint=False, max_iter=150)
    assert none is None
    assert only == pytest.approx(dists, rel=1e-6)


def test_marine_shots_sampled(pkg):
    """Two 8000 x 648 streamer gathers (dt = 2 ms, dx = 25 m) solved as one batch: each
    matches the FP64 oracle element-wise after the same 12 iterations."""
    dev = torch.device("cuda:0")
    pairs = [synth.gather_pair_marine(shot=s) for s in (0, 77)]
    O_ = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    P_ = [torch.from_numpy(p).to(dev) for _, p in pairs]
    d, phis, ms, infos = pkg.emd_batched(O_, P_, 2e-3, 25.0, max_iter=12)
    for b, (o, p) in enumerate(pairs):
        r = O.pdhg(o, p, 2e-3, 25.0, max_iter=12)
        g = dict(dist=d[b], phi=phis[b].double().cpu().numpy(), ux=ms[b][0].double().cpu().numpy(),
                 ut=ms[b][1].double().cpu().numpy(), info=infos[b])
        assert_parity(g, r, exact_trials=True)


def test_1d_shift_sweep_61_shifts_batched(pkg):
    """The 1D study in full: Ricker 8 Hz on [0, 1] (nt = 1024) against 61 shifted copies
    (-0.3 .. 0.3 s), all 61 solved in one batch (one resident CTA per shift).  Every
    distance matches the closed-form W1, and the misfit against the shift has a single
    minimum at zero shift and grows with |shift| until the two signals stop overlapping,
    where it flattens (the plateau of the discussion section)."""
    dt, obs, preds = synth.shift_sweep_1d(nt=1024)
    dev = torch.device("cuda:0")
    O_ = [torch.from_numpy(obs).to(dev)] * len(preds)
    P_ = [torch.from_numpy(p).to(dev) for _, p in preds]
    d, phis, ms, infos = pkg.emd_batched(O_, P_, dt, 1.0, max_iter=100000)
    assert all(bool(torch.isfinite(ph).all()) for ph in phis)  # zero shift included (Q20)
    shifts = np.array([s for s, _ in preds])
    w = []
    for (s, p), info in zip(preds, infos):
        assert info["status"] == 0 and info["launches"] == 3
        f = O.source_term(obs, p)[0]
        w.append(O.w1_1d(np.maximum(f, 0), np.maximum(-f, 0), dt))
    w = np.array(w)
    l1 = np.array([i["dist_l1"] for i in infos])
    nz = w > 0
    assert np.max(np.abs(l1[nz] - w[nz]) / w[nz]) <= 2e-3
    assert l1[np.argmin(np.abs(shifts))] <= 1e-6 * l1.max()
    order = np.argsort(np.abs(shifts))
    for side in (shifts > 0, shifts < 0):
        idx = [i for i in order if side[i]]
        vals = l1[idx]
        assert np.all(np.diff(vals) >= -2e-3 * vals.max())  # non-decreasing in |shift|
    far = np.abs(shifts) >= 0.2
    assert np.ptp(l1[far]) <= 2e-3 * l1.max()  # plateau once the signals no longer overlap


# ----------------------------------------------------------------------------- isotropic ground cost

@pytest.mark.parametrize("nt,nr,kw", [
    (256, 64, dict()),                 # persistent TMA solve
    (64, 64, dict()),                  # shared-memory resident solve (4096 cells)
    (256, 64, dict(tile=1)),           # plain per-pass kernel, 16 x 120 tiles
    (256, 64, dict(tile=MARCH)),       # marching solve
    (200, 40, dict(launch_mode=1)),    # per-pass TMA launches
])
def test_isotropic_parity(pkg, nt, nr, kw):
    """norm = EMD_NORM_ISO (reading Q19) on every solver path against the oracle's
    isotropic Algorithm 1, element by element after 600 iterations, decisions replayed."""
    obs, pred = synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=11)
    replay_parity(pkg, obs, pred, 2e-3, 10.0, 600, gpu_kw=kw, norm=O.NORM_ISO)


def test_isotropic_batched_equals_single(pkg):
    """Two gathers solved as one batch and one by one (isotropic cost): each run equals the
    oracle replaying its own decisions, and where both runs took the same decisions they
    agree to 1e-5."""
    gathers = [synth.gather_pair_hyperbolic(nt=nt, nr=nr, seed=s) for nt, nr, s in [(300, 50, 1), (180, 30, 2)]]
    dev = torch.device("cuda:0")
    O_ = [torch.from_numpy(a).to(dev) for a, _ in gathers]
    P_ = [torch.from_numpy(b).to(dev) for _, b in gathers]
    K = 300
    tr = torch.full((2, K, 4), float("nan"), dtype=torch.float64, device=dev)
    d, phis, ms, infos = pkg.emd_batched(O_, P_, 2e-3, 10.0, max_iter=K, norm=pkg.EMD_NORM_ISO, trace=tr)
    trb = tr.cpu().numpy()
    for b, (o, p) in enumerate(gathers):
        assert infos[b]["iters"] == K
        gb = dict(dist=d[b], phi=phis[b].double().cpu().numpy(), ux=ms[b][0].double().cpu().numpy(),
                  ut=ms[b][1].double().cpu().numpy(), info=infos[b])
        r = O.pdhg(o, p, 2e-3, 10.0, max_iter=K, norm=O.NORM_ISO, record=True,
                   force_trials=trb[b, :, 2].astype(int))
        assert r["trace"][:, 6].max() < NEAR_TIE
        assert_parity(gb, r, exact_trials=True)
        gs = gpu_solve(pkg, o, p, 2e-3, 10.0, max_iter=K, norm=O.NORM_ISO, trace=True)
        if np.array_equal(gs["trace"][:, 2], trb[b, :, 2]):
            assert gs["dist"] == pytest.approx(d[b], rel=1e-5)
            assert rel_l2(gb["phi"], gs["phi"]) <= 1e-5


def test_isotropic_converged_against_oracle_and_bracket(pkg):
    """Normalised domain, run to residual 1e-3: the isotropic distance matches the oracle's
    converged one and lies between the anisotropic distance over sqrt(2) and it."""
    obs, pred = synth.gather_pair_hyperbolic(nt=96, nr=12, seed=3)
    dt, dx = 1 / 95, 1 / 11
    gi = gpu_solve(pkg, obs, pred, dt, dx, max_iter=40000, tol=1e-3, norm=O.NORM_ISO)
    ga = gpu_solve(pkg, obs, pred, dt, dx, max_iter=40000, tol=1e-3)
    ri = O.pdhg(obs, pred, dt, dx, max_iter=40000, tol=1e-3, norm=O.NORM_ISO)
    assert gi["info"]["residual"] <= 1e-3 and ri["residual"] <= 1e-3
    assert gi["info"]["dist_l1"] == pytest.approx(ri["dist_l1"], rel=2e-2)
    assert ga["info"]["dist_l1"] / np.sqrt(2) <= gi["info"]["dist_l1"] <= ga["info"]["dist_l1"]
