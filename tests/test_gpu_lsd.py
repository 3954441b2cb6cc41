"""The least-squares misfit kernel (Sec. 2.1, adjoint source Sec. 2.3) against the oracle,
and the 1D time-shift study of Sec. 3.1 with both misfits from the GPU: the LSD curve has
two local minima beside the global one (cycle skipping), the EMD curve a single minimum.
"""

import numpy as np
import pytest
import torch

from oracle import emd_oracle as O
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07284_gb300 import build
    build.build()
    import paper_1808_07284_gb300 as P
    return P


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


@pytest.mark.parametrize("nr,nt,dt,dx", [(1, 1024, 1 / 1023, 1.0), (64, 256, 2e-3, 10.0), (400, 3000, 1e-3, 12.5),
                                         (7, 333, 4e-3, 25.0)])
def test_lsd_matches_oracle(P, nr, nt, dt, dx):
    obs, pred = synth.gather_pair_hyperbolic(nt=nt, nr=max(nr, 1), seed=nr + nt)
    obs, pred = obs[:nr], pred[:nr]
    gp = torch.full((nr, nt), float("nan"), device=DEV)
    go = torch.full((nr, nt), float("nan"), device=DEV)
    v = P.emd_lsd(_t(obs), _t(pred), dt, dx, grad_pred=gp, grad_obs=go)
    want, g = O.lsd_misfit(obs, pred, dt, dx)
    assert v == pytest.approx(want, rel=1e-6)
    tol = 1e-6 * np.abs(g).max()
    np.testing.assert_allclose(gp.cpu().numpy(), g, rtol=0, atol=tol)
    np.testing.assert_array_equal(go.cpu().numpy(), -gp.cpu().numpy())


def test_lsd_loss_backward_is_the_adjoint_source(P):
    obs, pred = synth.gather_pair_hyperbolic()
    p = _t(pred).requires_grad_(True)
    o = _t(obs).requires_grad_(True)
    loss = P.lsd_loss(p, o, 2e-3, 10.0)
    (2.0 * loss).backward()
    want, g = O.lsd_misfit(obs, pred, 2e-3, 10.0)
    assert float(loss.detach()) == pytest.approx(want, rel=1e-6)
    np.testing.assert_allclose(p.grad.cpu().numpy(), 2.0 * g, rtol=0, atol=2e-6 * np.abs(g).max())
    np.testing.assert_allclose(o.grad.cpu().numpy(), -2.0 * g, rtol=0, atol=2e-6 * np.abs(g).max())


def _local_minima(v):
    return [i for i in range(1, len(v) - 1) if v[i] < v[i - 1] and v[i] < v[i + 1]]


def test_shift_study_lsd_cycle_skips_emd_does_not(P):
    """Sec. 3.1: Ricker 8 Hz on [0, 1] (nt = 1024, T = 1) against 61 shifted copies.  The
    LSD misfit against the shift has a global minimum at zero shift and two local minima
    (at about +-0.11 s, one period away); the EMD has only the minimum at zero."""
    dt, obs, preds = synth.shift_sweep_1d(nt=1024)
    shifts = np.array([s for s, _ in preds])
    o = _t(obs)
    lsd = np.array([P.emd_lsd(o, _t(p), dt, 1.0) for _, p in preds])
    want = np.array([O.lsd_misfit(obs, p, dt, 1.0)[0] for _, p in preds])
    np.testing.assert_allclose(lsd, want, rtol=1e-6)
    loc = _local_minima(lsd)
    assert len(loc) == 3 and shifts[np.argmin(lsd)] == 0.0
    assert sorted(np.round(np.abs(shifts[loc]), 2)) == [0.0, 0.11, 0.11]
    # the side minima are real dips: the curve rises by more than a tenth of its range
    # between each of them and the global minimum
    i0 = int(np.argmin(np.abs(shifts)))
    for i in loc:
        if i != i0:
            lo, hi = sorted((i, i0))
            assert lsd[lo:hi + 1].max() - lsd[i] > 0.1 * lsd.max()
    d, _, _, infos = P.emd_batched([o] * len(preds), [_t(p) for _, p in preds], dt, 1.0, max_iter=100000)
    emd = np.array([i["dist_l1"] for i in infos])
    # unimodal up to the flatness of the plateau (far shifts, no overlap): running
    # minimum from each end towards zero shift never rises by more than 2e-3 of the range
    tol = 2e-3 * emd.max()
    left, right = emd[:i0 + 1], emd[i0:][::-1]
    for side in (left, right):
        assert np.all(side[1:] <= np.minimum.accumulate(side)[:-1] + tol)
    assert np.argmin(emd) == i0


def _spectral_centroid(x):
    """Power-weighted mean frequency bin of a real signal."""
    X = np.abs(np.fft.rfft(x)) ** 2
    return float((np.arange(X.size) * X).sum() / X.sum())


def test_emd_adjoint_source_is_an_envelope_of_the_lsd_one(P):
    """Sec. 3.1: the EMD adjoint source of a shifted Ricker pair looks like an envelope of the
    LSD one (the difference of the two signals).  Measured by its power spectrum: for shifts
    of 30 - 150 ms, the EMD adjoint source (from emd_loss's backward) has its spectral
    centroid at most 0.7 times the LSD adjoint source's (from lsd_loss's backward); the
    oracle, run to the same iteration count, gives 0.18 - 0.60.  The EMD solves run as one
    batch, each to 20,000 iterations."""
    dt, obs, preds = synth.shift_sweep_1d(nt=1024, shifts=[0.03, 0.06, 0.1, 0.15])
    o = _t(obs)
    ps = [_t(p).requires_grad_(True) for _, p in preds]
    P.emd_loss_batched(ps, [o] * len(ps), dt, 1.0, max_iter=20000).sum().backward()
    for (s, p), pe in zip(preds, ps):
        pl = _t(p).requires_grad_(True)
        P.lsd_loss(pl, o, dt, 1.0).backward()
        g_emd = pe.grad.double().cpu().numpy()[0]
        g_lsd = pl.grad.double().cpu().numpy()[0]
        assert np.isfinite(g_emd).all() and np.abs(g_emd).max() > 0
        ratio = _spectral_centroid(g_emd) / _spectral_centroid(g_lsd)
        assert ratio <= 0.7, (s, ratio)
