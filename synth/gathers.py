"""Seeded synthetic shot-gather pairs (observed, predicted) on an ``[nr][nt]`` grid.

Every array is float32, C-contiguous, shape ``(nr, nt)``: row ``i`` is receiver ``i``
(offset ``x_i = (i + 1) * dx`` from the source) and column ``j`` is time ``t_j = j * dt``.
The recipes follow the shapes and event types of the paper's experiments (a 1D shifted
Ricker study, a crosshole gather of 1000 x 128, Marmousi gathers of 3000 x 227, the
Chevron 2014 streamer data); the paper's own data sets are not available, so these
seeded stand-ins take their place.

Draw order inside each generator is fixed, so a seed fully determines the output.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "ricker",
    "gather_pair_hyperbolic",
    "shift_sweep_1d",
    "gather_pair_transmissive",
    "batch_uneven_hyperbolic",
    "gather_pair_reflective",
    "gather_pair_marine",
    "workload",
]


def ricker(t: np.ndarray, f0: float) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f0^2 t^2) exp(-pi^2 f0^2 t^2), peak at t = 0."""
    a = (np.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _add_events(out: np.ndarray, dt: float, tau: np.ndarray, amp: np.ndarray, f0: float) -> None:
    """Add amp[e, i] * ricker(t - tau[e, i]) to row i of ``out`` for every event e.

    The wavelet is evaluated only within +-2.5 / f0 of its peak (its value there is
    below 1e-25 of the peak), so large gathers stay cheap to build.
    """
    nr, nt = out.shape
    half = int(np.ceil(2.5 / f0 / dt)) + 1
    offs = np.arange(-half, half + 1)
    rows = np.repeat(np.arange(nr)[:, None], offs.size, axis=1)
    for e in range(tau.shape[0]):
        centre = np.floor(tau[e] / dt).astype(np.int64)
        idx = centre[:, None] + offs[None, :]
        val = amp[e][:, None] * ricker(idx * dt - tau[e][:, None], f0)
        ok = (idx >= 0) & (idx < nt)
        out[rows[ok], idx[ok]] += val[ok]


def _offsets(nr: int, dx: float) -> np.ndarray:
    return (np.arange(nr) + 1.0) * dx


def gather_pair_hyperbolic(nt=256, nr=64, dt=2e-3, dx=10.0, n_events=3, f0=10.0,
                           shift_ms=40.0, seed=0):
    """Three hyperbolic events t(x) = sqrt(t0^2 + x^2 / v^2) (the small single-gather case).

    t0 ~ U[0.1, 0.4] s, v ~ U[1500, 3000] m/s, unit amplitude, Ricker ``f0``.  The
    predicted gather moves every t0 by U[-shift_ms, shift_ms] ms.
    Draw order: t0 (n_events), v (n_events), shifts (n_events).
    """
    rng = np.random.default_rng(seed)
    t0 = rng.uniform(0.1, 0.4, n_events)
    v = rng.uniform(1500.0, 3000.0, n_events)
    sh = rng.uniform(-shift_ms, shift_ms, n_events) * 1e-3
    x = _offsets(nr, dx)
    amp = np.ones((n_events, nr))
    obs = np.zeros((nr, nt))
    pred = np.zeros((nr, nt))
    _add_events(obs, dt, np.sqrt(t0[:, None] ** 2 + (x[None, :] / v[:, None]) ** 2), amp, f0)
    _add_events(pred, dt, np.sqrt((t0 + sh)[:, None] ** 2 + (x[None, :] / v[:, None]) ** 2), amp, f0)
    return obs.astype(np.float32), pred.astype(np.float32)


def shift_sweep_1d(nt=1024, f0=8.0, t_obs=0.5, shifts=None):
    """The 1D time-shift study: Ricker 8 Hz at t = 0.5 on [0, 1] (dt = 1/(nt-1)).

    Returns ``(dt, obs[1, nt], [(shift, pred[1, nt]), ...])`` with shifts in seconds,
    by default 61 values from -0.3 to 0.3.
    """
    if shifts is None:
        shifts = np.linspace(-0.3, 0.3, 61)
    dt = 1.0 / (nt - 1)
    t = np.arange(nt) * dt
    obs = ricker(t - t_obs, f0)[None, :].astype(np.float32)
    preds = [(float(s), ricker(t - t_obs - s, f0)[None, :].astype(np.float32)) for s in shifts]
    return dt, obs, preds


def _noise_like(rng, sig: np.ndarray, snr_db: float) -> np.ndarray:
    rms = np.sqrt(np.mean(sig.astype(np.float64) ** 2))
    return rng.standard_normal(sig.shape) * rms * 10.0 ** (-snr_db / 20.0)


def gather_pair_transmissive(nt=3000, nr=400, dt=1e-3, dx=12.5, f0=8.0, snr_db=30.0, seed=2):
    """Eight transmitted events: 1 direct, 3 refracted, 4 diffractions (the mid-size gather).

    direct: tau = x / v, v ~ U[1500, 2000]; refracted: tau = x / v_r + t_i,
    v_r ~ U[2500, 4500], t_i ~ U[0.1, 0.8]; diffractions: tau = sqrt(t_d^2 + (x - x_d)^2 / v^2),
    t_d ~ U[0.3, 2.5], x_d ~ U[0, nr dx], v ~ U[1800, 3000].  Amplitudes U[0.2, 1] times
    (dx / x)^(1/2).  Predicted: every event's traveltime moved by U[-1.5, 1.5] / f0 s
    (up to 1.5 periods, cycle-skipped) plus Gaussian noise at ``snr_db``.
    Draw order: v_direct, (v_r, t_i) x3, (t_d, x_d, v) x4, amplitudes (8), shifts (8), noise.
    """
    rng = np.random.default_rng(seed)
    x = _offsets(nr, dx)
    v_d = rng.uniform(1500.0, 2000.0)
    refr = [(rng.uniform(2500.0, 4500.0), rng.uniform(0.1, 0.8)) for _ in range(3)]
    diff = [(rng.uniform(0.3, 2.5), rng.uniform(0.0, nr * dx), rng.uniform(1800.0, 3000.0))
            for _ in range(4)]
    a0 = rng.uniform(0.2, 1.0, 8)
    sh = rng.uniform(-1.5, 1.5, 8) / f0
    tau = [x / v_d] + [x / vr + ti for vr, ti in refr] + \
          [np.sqrt(td ** 2 + (x - xd) ** 2 / v ** 2) for td, xd, v in diff]
    tau = np.array(tau)
    amp = a0[:, None] * np.sqrt(dx / x)[None, :]
    obs = np.zeros((nr, nt))
    pred = np.zeros((nr, nt))
    _add_events(obs, dt, tau, amp, f0)
    _add_events(pred, dt, tau + sh[:, None], amp, f0)
    pred += _noise_like(rng, pred, snr_db)
    return obs.astype(np.float32), pred.astype(np.float32)


def batch_uneven_hyperbolic(n_shots=48, dt=1e-3, dx=12.5, seed=3, shots=None):
    """Uneven batch: nr ~ U{200..640}, nt ~ U{1500..5000}, hyperbolic events per shot.

    Sizes come from ``seed``; shot s uses seed 1000 + s for its events (three hyperbolas
    as in the small case, Ricker 10 Hz, shifts up to 40 ms).  ``shots`` selects a subset
    of shot indices (the sizes are still drawn for all ``n_shots``).
    Returns a list of ``(obs, pred)``.
    """
    rng = np.random.default_rng(seed)
    nrs = rng.integers(200, 641, n_shots)
    nts = rng.integers(1500, 5001, n_shots)
    out = []
    for s in (range(n_shots) if shots is None else shots):
        out.append(gather_pair_hyperbolic(nt=int(nts[s]), nr=int(nrs[s]), dt=dt, dx=dx,
                                          seed=1000 + s))
    return out


def gather_pair_reflective(nt=4000, nr=480, dt=1e-3, dx=12.5, f0=6.0, n_refl=20, shot=0, seed=4):
    """Twenty hyperbolic reflections (the differentiable-misfit batch, one shot of 16).

    t0 ~ sorted U[0.2, 3.8], v_rms(t0) = 1500 + 400 t0, reflectivity N(0, 1), Ricker 6 Hz.
    Predicted: v_rms scaled by (1 + 0.08 sin(2 pi t0 / 4 + phase_s)), phase_s ~ U[0, 2 pi).
    Shot s draws from seed * 1000 + s: t0, reflectivity, phase.
    """
    rng = np.random.default_rng(seed * 1000 + shot)
    t0 = np.sort(rng.uniform(0.2, 3.8, n_refl))
    r = rng.standard_normal(n_refl)
    ph = rng.uniform(0.0, 2.0 * np.pi)
    x = _offsets(nr, dx)
    v = 1500.0 + 400.0 * t0
    vp = v * (1.0 + 0.08 * np.sin(2.0 * np.pi * t0 / 4.0 + ph))
    amp = np.repeat(r[:, None], nr, axis=1)
    obs = np.zeros((nr, nt))
    pred = np.zeros((nr, nt))
    _add_events(obs, dt, np.sqrt(t0[:, None] ** 2 + (x[None, :] / v[:, None]) ** 2), amp, f0)
    _add_events(pred, dt, np.sqrt(t0[:, None] ** 2 + (x[None, :] / vp[:, None]) ** 2), amp, f0)
    return obs.astype(np.float32), pred.astype(np.float32)


def _band(sig: np.ndarray, dt: float, lo: float, hi: float | None, taper: float = 1.0) -> np.ndarray:
    """Zero-phase FFT band mask along time with cosine tapers of width ``taper`` Hz."""
    nt = sig.shape[-1]
    fr = np.fft.rfftfreq(nt, dt)
    m = np.ones_like(fr)
    if lo > 0:
        m = np.where(fr < lo - taper, 0.0, m)
        ramp = (fr >= lo - taper) & (fr < lo)
        m = np.where(ramp, 0.5 - 0.5 * np.cos(np.pi * (fr - lo + taper) / taper), m)
    if hi is not None:
        m = np.where(fr > hi + taper, 0.0, m)
        ramp = (fr > hi) & (fr <= hi + taper)
        m = np.where(ramp, 0.5 + 0.5 * np.cos(np.pi * (fr - hi) / taper), m)
    return np.fft.irfft(np.fft.rfft(sig, axis=-1) * m, n=nt, axis=-1)


def gather_pair_marine(nt=8000, nr=648, dt=2e-3, dx=25.0, f0=5.0, n_refl=40, shot=0, seed=5,
                       snr_db=20.0):
    """Marine-streamer gather: 40 reflections + a water-bottom multiple (the large batch).

    Observed from v(z) = 1500 + 0.5 z, predicted from the same law with v scaled by
    (1 + e_s), e_s ~ U[-0.15, 0.15].  Reflector depths ~ sorted U[200, 6000] m, the
    first one is the water bottom; its first multiple arrives at twice the zero-offset
    time, polarity reversed, half amplitude.  Ricker 5 Hz with energy below 3 Hz removed,
    3-15 Hz band-limited Gaussian noise at ``snr_db``.  Shot s draws from seed * 1000 + s:
    depths, reflectivity, velocity error, noise.
    """
    rng = np.random.default_rng(seed * 1000 + shot)
    z = np.sort(rng.uniform(200.0, 6000.0, n_refl))
    r = rng.standard_normal(n_refl)
    err = rng.uniform(-0.15, 0.15)
    x = _offsets(nr, dx)

    def traveltimes(scale):
        # v(z) = v0 + k z: vertical two-way time and an RMS-velocity hyperbola.
        v0, k = 1500.0 * scale, 0.5 * scale
        t0 = 2.0 * np.log1p(k * z / v0) / k
        # RMS velocity of a linear law: integral of v dz over integral of dz / v.
        vrms = np.sqrt(k * (v0 * z + 0.5 * k * z ** 2) / np.log1p(k * z / v0))
        tau = np.sqrt(t0[:, None] ** 2 + (x[None, :] / vrms[:, None]) ** 2)
        tm = np.sqrt((2.0 * t0[0]) ** 2 + (x / vrms[0]) ** 2)
        return np.vstack([tau, tm[None, :]])

    amp = np.vstack([np.repeat(r[:, None], nr, axis=1), np.full((1, nr), -0.5 * r[0])])
    obs = np.zeros((nr, nt))
    pred = np.zeros((nr, nt))
    _add_events(obs, dt, traveltimes(1.0), amp, f0)
    _add_events(pred, dt, traveltimes(1.0 + err), amp, f0)
    obs = _band(obs, dt, 3.0, None)
    pred = _band(pred, dt, 3.0, None)
    noise = _band(rng.standard_normal(obs.shape), dt, 3.0, 15.0)
    noise *= np.sqrt(np.mean(obs ** 2)) * 10 ** (-snr_db / 20.0) / max(np.sqrt(np.mean(noise ** 2)), 1e-30)
    obs = obs + noise
    return obs.astype(np.float32), pred.astype(np.float32)


def marine_shot(shot: int):
    """gather_pair_marine of one shot with the default geometry (a picklable one-argument
    form, for generating the 128-shot batch in a process pool)."""
    return gather_pair_marine(shot=shot)


def workload(name: str):
    """Named workloads: returns ``(obs, pred, dt, dx)`` for the single-gather cases."""
    if name == "hyperbolic_256x64":
        o, p = gather_pair_hyperbolic()
        return o, p, 2e-3, 10.0
    if name == "transmissive_3000x400":
        o, p = gather_pair_transmissive()
        return o, p, 1e-3, 12.5
    raise KeyError(name)
