"""Plain float64 statement of the dynamic-formulation EMD misfit and its PDHG solver.

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU baseline use
this module.  It is deliberately slow and literal: every step is a whole-array numpy
expression in the order and notation of the paper, with no fusion and no reordering.

Grid convention (Sec. 2.2): arrays are ``[nr][nt]``, row i = receiver, column j = time,
spacings ``dx`` (receivers) and ``dt`` (time).  The flux is ``u = (ux, ut)``.

Readings taken where the paper is silent, ambiguous or inconsistent (each one is
listed with its reason in the design notes of the repository):

* Q1  divergence := -gradient^T (the adjoint identity of Sec. 2.2 wins over the
       printed boundary row); the outer faces carry zero flux.
* Q2  fixed-step PDHG uses alpha = beta = 1/sqrt(lambda); the linesearch starts from
       alpha_0 = 1/sqrt(delta lambda), lambda = 4/dx^2 + 4/dt^2.
* Q3  the linesearch test uses Euclidean norms by default (ls_norm=2); ls_norm=1 gives
       the printed l1 norms.
* Q4  alpha_{k+1} starts at the upper end alpha_k sqrt(1 + theta_k).
* Q5  dist = Phi * dx * dt with Phi = ||u||_{1,1} + eps/2 ||u||_2^2; dist_l1 drops eps.
* Q6  stopping residual r = max(||div u + f|| / ||f||, ||u^{k+1} - u^k|| / ||u^{k+1}||),
       tested every ``check_every`` iterations; tol = 0 runs exactly ``max_iter``.
* Q7  balance=MEAN subtracts the mean of f = Pcal - Pobs; balance=NONE solves as printed.
* Q8  gradient of the returned distance w.r.t. Pcal is dx dt (phi - mean phi) (MEAN) or
       dx dt phi (NONE); w.r.t. Pobs it is the negative.
* Q10 u^0 = 0 and phi^0 = 0 unless a warm start is given; a warm start's outer faces
       (x flux of receiver 0, time flux of sample 0) are set to zero (Q1).
* Q11 nr = 1 means a 1D problem: no x component, lambda = 4/dt^2, cell area dt.
* Q12 the backtracking gives up after ``ls_max_trials`` trials (status LINESEARCH).
* Q13 ``iters`` counts accepted outer iterations; trials are counted separately.
* Q19 norm=2 selects the isotropic ground cost of the formulation the paper builds on,
       ||u||_{1,2} = sum_ij sqrt((u^x_ij)^2 + (u^t_ij)^2), pairing the two flux components
       of one grid index as the paper's ||u||_{1,1} sums them; the prox becomes the vector
       shrink max(1 - alpha/||v||, 0) v and the conjugate in the gap (||w|| - 1)_+^2 / 2 eps.
       norm=1 (default) is the paper's anisotropic ||u||_{1,1}.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

BAL_NONE = 0
BAL_MEAN = 1

NORM_ANISO = 1  # ||u||_{1,1}: |u^x| + |u^t| per cell (Sec. 2.2)
NORM_ISO = 2    # ||u||_{1,2}: sqrt((u^x)^2 + (u^t)^2) per cell (Q19)

STATUS_OK = 0
STATUS_NONFINITE = 3
STATUS_LINESEARCH = 4


@dataclass
class Params:
    """Solver parameters; defaults are the paper's constants (Sec. 2.2)."""

    eps: float = 1e-4          # regularisation epsilon of Phi
    xi: float = 0.5            # backtracking factor
    zeta: float = 0.99         # linesearch test constant
    delta: float = 1e5         # beta = delta * alpha
    alpha0: float = 0.0        # <= 0: 1/sqrt(delta lambda) (linesearch) or 1/sqrt(lambda)
    max_iter: int = 2000
    tol: float = 0.0
    check_every: int = 10
    ls_max_trials: int = 40
    linesearch: int = 1
    ls_norm: int = 2
    balance: int = BAL_MEAN
    norm: int = NORM_ANISO
    phi_init: np.ndarray | None = field(default=None, repr=False)
    m_init: np.ndarray | None = field(default=None, repr=False)
    # Replay input (test infrastructure, not part of the method): when given, iteration k
    # runs exactly force_trials[k] linesearch trials and accepts the last one, whatever
    # its own test says; the test is still evaluated and every trial on which it disagrees
    # with the forced outcome is recorded (trace column 6).  Used to follow the decisions
    # another implementation took at near ties and compare the iterates afterwards.
    force_trials: np.ndarray | None = field(default=None, repr=False)
    # Storage model (test infrastructure, not part of the method): when True, u and phi are
    # rounded to binary32 after every accepted iteration, as a solver that keeps its iterates
    # in single precision does.  Used only to measure how far an instance's answer moves
    # under that rounding (its conditioning), never as the reference answer.
    store_f32: bool = False


# --------------------------------------------------------------------------- decomposition

def mainini(p_obs, p_pred):
    """Mainini decomposition and recombination (Sec. 2.1).

    P = P^+ - P^- for each gather; the compared measures are
    mu = Pcal^+ + Pobs^-  and  nu = Pobs^+ + Pcal^-, both nonnegative.
    """
    p_obs = np.asarray(p_obs, np.float64)
    p_pred = np.asarray(p_pred, np.float64)
    pcal_pos, pcal_neg = np.maximum(p_pred, 0.0), np.maximum(-p_pred, 0.0)
    pobs_pos, pobs_neg = np.maximum(p_obs, 0.0), np.maximum(-p_obs, 0.0)
    mu = pcal_pos + pobs_neg
    nu = pobs_pos + pcal_neg
    return mu, nu


def cell_area(nr: int, dt: float, dx: float) -> float:
    """dx dt for a 2D gather; dt alone when nr = 1 (Q11)."""
    return dt if nr == 1 else dx * dt


def source_term(p_obs, p_pred, balance=BAL_MEAN):
    """f = Pcal - Pobs, the source of the constraint div u + f = 0 (Eq. for f_OT).

    The paper notes that the decomposition need not be formed to solve the problem:
    only the difference mu - nu = Pcal - Pobs enters.  With balance=MEAN the mean of f
    is removed so that the zero-flux problem is feasible (Q7).
    """
    f = np.asarray(p_pred, np.float64) - np.asarray(p_obs, np.float64)
    if balance == BAL_MEAN:
        f = f - f.mean()
    return f


# --------------------------------------------------------------------------- operators

def gradient(phi, dt, dx):
    """Backward differences with zero on the first row / column (Sec. 2.2).

    (d_x phi)_{i,j} = (phi_{i,j} - phi_{i-1,j}) / dx for i > 1, else 0;
    (d_t phi)_{i,j} = (phi_{i,j} - phi_{i,j-1}) / dt for j > 1, else 0.
    """
    phi = np.asarray(phi, np.float64)
    gx = np.zeros_like(phi)
    gt = np.zeros_like(phi)
    gx[1:, :] = (phi[1:, :] - phi[:-1, :]) / dx
    gt[:, 1:] = (phi[:, 1:] - phi[:, :-1]) / dt
    return gx, gt


def divergence(ux, ut, dt, dx):
    """Divergence as the negative adjoint of ``gradient`` (Sec. 2.2 identity; reading Q1).

    ux_{i,j} is the flux through the face between cells i-1 and i; the faces outside
    the grid (ux_{1,j} and beyond row nr, ut_{i,1} and beyond column nt) carry zero:
    (div u)_{i,j} = (ux_{i+1,j} - ux_{i,j}) / dx + (ut_{i,j+1} - ut_{i,j}) / dt.
    For i < nr this is the printed forward difference (ux_{1,j} stays 0); at i = nr it
    is -ux_{nr,j} / dx, which keeps <u, grad phi> = -<div u, phi> exact.
    """
    fx = np.array(ux, np.float64)
    ft = np.array(ut, np.float64)
    fx[0, :] = 0.0
    ft[:, 0] = 0.0
    nr, nt = fx.shape
    div_x = np.zeros((nr, nt))
    div_x[:-1, :] += fx[1:, :]
    div_x -= fx
    div_t = np.zeros((nr, nt))
    div_t[:, :-1] += ft[:, 1:]
    div_t -= ft
    return div_x / dx + div_t / dt


def lambda_bound(nr: int, dt: float, dx: float) -> float:
    """Gershgorin bound on the largest eigenvalue of -div grad (Sec. 2.2): 4/dx^2 + 4/dt^2."""
    return 4.0 / dt ** 2 + (4.0 / dx ** 2 if nr > 1 else 0.0)


def shrink(x, y):
    """shrink(x, y) = (1 - y/|x|) x if |x| >= y, else 0 (Sec. 2.2), componentwise."""
    x = np.asarray(x, np.float64)
    ax = np.abs(x)
    out = np.zeros_like(x)
    big = ax >= y
    if y == 0:
        return x.copy()
    out[big] = (1.0 - y / ax[big]) * x[big]
    return out


def shrink_vec(vx, vt, y):
    """Vector shrink of the isotropic norm (Q19): max(1 - y/||v||, 0) v per cell, v = (vx, vt);
    the prox of y ||.||_2, as shrink is the prox of y |.|."""
    vx = np.asarray(vx, np.float64)
    vt = np.asarray(vt, np.float64)
    n = np.sqrt(vx * vx + vt * vt)
    scale = np.zeros_like(n)
    big = n > y
    scale[big] = 1.0 - y / n[big]
    return scale * vx, scale * vt


def primal_step(ux, ut, phi, alpha, eps, dt, dx, norm=NORM_ANISO):
    """Eq. (primal-update): u^{k+1} = shrink(u^k + alpha grad phi^k, alpha) / (1 + eps alpha);
    with norm=NORM_ISO the shrink acts on the vector (u^x, u^t) of each cell (Q19)."""
    gx, gt = gradient(phi, dt, dx)
    c = 1.0 / (1.0 + eps * alpha)
    if norm == NORM_ISO:
        nx, nt_ = shrink_vec(ux + alpha * gx, ut + alpha * gt, alpha)
        return nx * c, nt_ * c
    return shrink(ux + alpha * gx, alpha) * c, shrink(ut + alpha * gt, alpha) * c


def dual_step(phi, bx, bt, f, beta, dt, dx):
    """Eq. (dual-update): phi^{k+1} = phi^k + beta (div ubar^{k+1} + Pcal - Pobs)."""
    return phi + beta * (divergence(bx, bt, dt, dx) + f)


def _norm_vec(gx, gt, ls_norm):
    if ls_norm == 1:
        return float(np.abs(gx).sum() + np.abs(gt).sum())
    return math.sqrt(float((gx * gx).sum() + (gt * gt).sum()))


def _norm_scalar(d, ls_norm):
    if ls_norm == 1:
        return float(np.abs(d).sum())
    return math.sqrt(float((d * d).sum()))


# --------------------------------------------------------------------------- objective

def objective(ux, ut, eps, norm=NORM_ANISO):
    """Phi = ||u||_{1,1} + eps/2 ||u||_2^2 (Sec. 2.2) and its norm part (||u||_{1,2} with
    norm=NORM_ISO, Q19)."""
    if norm == NORM_ISO:
        l1 = float(np.sqrt(ux * ux + ut * ut).sum())
    else:
        l1 = float(np.abs(ux).sum() + np.abs(ut).sum())
    l2 = float((ux * ux).sum() + (ut * ut).sum())
    return l1 + 0.5 * eps * l2, l1


def duality_gap(ux, ut, phi, f, eps, dt, dx, norm=NORM_ANISO):
    """dx dt [ Phi(u) - D(phi) ] with D(phi) = <phi, f> - sum h*(grad phi) (from the Lagrangian).

    h(v) = |v| + eps/2 v^2 has the conjugate h*(w) = max(|w| - 1, 0)^2 / (2 eps), per
    component; for the isotropic norm h(v) = ||v|| + eps/2 ||v||^2 of the cell vector and
    h*(w) = max(||w|| - 1, 0)^2 / (2 eps).
    """
    nr = phi.shape[0]
    gx, gt = gradient(phi, dt, dx)
    prim, _ = objective(ux, ut, eps, norm)
    if norm == NORM_ISO:
        hs = np.maximum(np.sqrt(gx * gx + gt * gt) - 1.0, 0.0) ** 2 / (2.0 * eps)
    else:
        hs = (np.maximum(np.abs(gx) - 1.0, 0.0) ** 2 + np.maximum(np.abs(gt) - 1.0, 0.0) ** 2) / (2.0 * eps)
    dual = float((phi * f).sum()) - float(hs.sum())
    return cell_area(nr, dt, dx) * (prim - dual)


# --------------------------------------------------------------------------- Algorithm 1

def pdhg(p_obs, p_pred, dt, dx, params: Params | None = None, record: bool = False, **kw):
    """PDHG with linesearch for the EMD (Algorithm 1), float64.

    Per outer iteration k:
      1. u^{k+1} = prox step (Eq. primal-update) with alpha_k;
      2. a = alpha_k sqrt(1 + theta_k);
      3. repeat: theta = a / alpha_k, beta = delta a,
                 ubar = u^{k+1} + theta (u^{k+1} - u^k),
                 phi+ = phi^k + beta (div ubar + f)       (Eq. dual-update)
         until sqrt(delta) a ||grad phi+ - grad phi^k|| <= zeta ||phi+ - phi^k||,
         shrinking a by xi after each failed test;
      4. alpha_{k+1} = a, theta_{k+1} = theta, phi^{k+1} = phi+.
    With linesearch=0 it is the fixed-step PDHG of Sec. 2.2 (ubar = 2u^{k+1} - u^k).

    Returns a dict with dist, dist_l1, phi, ux, ut, iters, trials, status, residual,
    r_feas, r_step, alpha, theta, imbalance, gap (and a per-iteration ``trace`` when
    ``record`` is set: alpha, theta, trials, r_feas, r_step, the smallest relative gap
    |lhs - rhs| / rhs between the two sides of the linesearch test over the iteration's
    trials -- a near tie there is where a computation in other precision may decide
    differently -- and, with ``force_trials``, the largest relative gap among the trials
    whose own test outcome contradicts the forced one, 0 when the forced count is the
    test's own choice).
    """
    p = params if params is not None else Params()
    if kw:
        p = Params(**{**asdict(p), **kw})
    p_obs = np.asarray(p_obs, np.float64)
    p_pred = np.asarray(p_pred, np.float64)
    nr, nt = p_obs.shape
    area = cell_area(nr, dt, dx)
    imbalance = area * float((p_pred - p_obs).sum())
    f = source_term(p_obs, p_pred, p.balance)
    lam = lambda_bound(nr, dt, dx)

    if p.linesearch:
        alpha = p.alpha0 if p.alpha0 > 0 else 1.0 / math.sqrt(p.delta * lam)
        beta = p.delta * alpha
    else:
        alpha = p.alpha0 if p.alpha0 > 0 else 1.0 / math.sqrt(lam)
        beta = 1.0 / (lam * alpha)
    theta = 1.0

    if p.m_init is not None:
        ux = np.array(p.m_init[0], np.float64)
        ut = np.array(p.m_init[1], np.float64)
        ux[0, :] = 0.0  # Q1: the outer faces carry no flux, whatever the warm start holds
        ut[:, 0] = 0.0
    else:
        ux = np.zeros((nr, nt))
        ut = np.zeros((nr, nt))
    phi = np.zeros((nr, nt)) if p.phi_init is None else np.array(p.phi_init, np.float64)

    fnorm = math.sqrt(float((f * f).sum()))
    status = STATUS_OK
    trials_total = 0
    iters = 0
    r_feas = r_step = math.inf
    trace = []
    forced = None if p.force_trials is None else np.asarray(p.force_trials, np.int64)
    if forced is not None and p.linesearch:
        if forced.size < p.max_iter or (forced[:p.max_iter] < 1).any():
            raise ValueError("force_trials needs a count >= 1 for each of the max_iter iterations")
    for k in range(p.max_iter):
        nux, nut = primal_step(ux, ut, phi, alpha, p.eps, dt, dx, p.norm)
        disagree = 0.0
        if p.linesearch:
            # Reading Q20: identical gathers (the balanced f identically zero) with p = div u^{k+1}
            # + f and q = div(u^{k+1} - u^k) both identically zero make the dual move beta (p +
            # theta q) zero for every step size, so every trial passes on every iteration.  The
            # step then takes the lower end alpha_k of [alpha_k, alpha_k sqrt(1 + theta_k)]
            # (theta = 1) rather than growing by about 1.6 per iteration until it overflows and
            # inf * 0 turns phi into NaN.
            still = False
            if fnorm == 0.0:
                pk = divergence(nux, nut, dt, dx) + f
                qk = divergence(nux - ux, nut - ut, dt, dx)
                still = not pk.any() and not qk.any()
            a = alpha if still else alpha * math.sqrt(1.0 + theta)
            accepted = False
            margin = math.inf  # closest any trial of this iteration came to the test's threshold
            want = None if forced is None else int(forced[k])
            for trial in range(1, p.ls_max_trials + 1):
                th = a / alpha
                beta = p.delta * a
                bx = nux + th * (nux - ux)
                bt = nut + th * (nut - ut)
                nphi = dual_step(phi, bx, bt, f, beta, dt, dx)
                dphi = nphi - phi
                gdx, gdt = gradient(dphi, dt, dx)
                trials_total += 1
                lhs = math.sqrt(p.delta) * a * _norm_vec(gdx, gdt, p.ls_norm)
                rhs = p.zeta * _norm_scalar(dphi, p.ls_norm)
                gap = abs(lhs - rhs) / rhs if rhs > 0 else math.inf
                margin = min(margin, gap)
                passed = lhs <= rhs
                if want is not None:  # replay: the forced count decides, the test is recorded
                    if passed != (trial == want):
                        disagree = max(disagree, gap)
                    passed = trial == want
                if passed:
                    accepted = True
                    break
                a = p.xi * a
            if not accepted:
                status = STATUS_LINESEARCH
                break
            alpha, theta = a, th
        else:
            trial = 1
            margin = math.inf
            nphi = dual_step(phi, 2.0 * nux - ux, 2.0 * nut - ut, f, beta, dt, dx)
            trials_total += 1
        res = divergence(nux, nut, dt, dx) + f
        rf = math.sqrt(float((res * res).sum()))
        r_feas = rf / fnorm if fnorm > 0 else rf
        du = math.sqrt(float(((nux - ux) ** 2).sum() + ((nut - ut) ** 2).sum()))
        un = math.sqrt(float((nux * nux).sum() + (nut * nut).sum()))
        r_step = du / max(un, 1e-30)
        ux, ut, phi = nux, nut, nphi
        if p.store_f32:
            ux, ut, phi = (a.astype(np.float32).astype(np.float64) for a in (ux, ut, phi))
        iters = k + 1
        if record:
            trace.append((alpha, theta, trial, r_feas, r_step, margin, disagree))
        if not (np.isfinite(phi).all() and np.isfinite(ux).all() and np.isfinite(ut).all()):
            status = STATUS_NONFINITE
            break
        if p.tol > 0 and iters % p.check_every == 0 and max(r_feas, r_step) <= p.tol:
            break

    phi_val, l1 = objective(ux, ut, p.eps, p.norm)
    out = dict(
        dist=area * phi_val, dist_l1=area * l1, phi=phi, ux=ux, ut=ut, f=f,
        iters=iters, trials=trials_total, status=status,
        residual=max(r_feas, r_step), r_feas=r_feas, r_step=r_step,
        alpha=alpha, theta=theta, imbalance=imbalance,
        gap=duality_gap(ux, ut, phi, f, p.eps, dt, dx, p.norm) if p.eps > 0 else float("nan"),
    )
    if record:
        out["trace"] = np.array(trace)
    return out


# --------------------------------------------------------------------------- closed forms

def w1_1d(mu, nu, dt):
    """Textbook 1D W1 between densities of equal mass on t_j = j dt: sum_j dt |F_mu - F_nu|.

    F is the cumulative mass dt * cumsum(.); the difference is constant between grid
    points, and vanishes after the last one when the masses are equal.
    """
    Fm = dt * np.cumsum(np.asarray(mu, np.float64))
    Fn = dt * np.cumsum(np.asarray(nu, np.float64))
    return dt * float(np.abs(Fm - Fn)[:-1].sum())


def forced_flux_1d(f, dt):
    """For nr = 1 the constraint fixes u completely: ut_{j+1} = -dt sum_{k<=j} f_k (ut_1 = 0)."""
    f = np.asarray(f, np.float64).ravel()
    ut = np.zeros_like(f)
    ut[1:] = -dt * np.cumsum(f)[:-1]
    return ut


def adjoint_source(phi, dt, dx, balance=BAL_MEAN, grad_out=1.0):
    """Adjoint source (Sec. 2.3): d f_OT / d Pcal = phi; scaled to the returned distance (Q8).

    Returns (d dist / d Pcal, d dist / d Pobs).
    """
    phi = np.asarray(phi, np.float64)
    area = cell_area(phi.shape[0], dt, dx)
    g = phi - phi.mean() if balance == BAL_MEAN else phi
    g = grad_out * area * g
    return g, -g


def lsd_misfit(p_obs, p_pred, dt, dx):
    """Least-squares misfit 1/2 integral (Pcal - Pobs)^2 (Sec. 2.1) and its adjoint source."""
    d = np.asarray(p_pred, np.float64) - np.asarray(p_obs, np.float64)
    area = cell_area(d.shape[0], dt, dx)
    return 0.5 * area * float((d * d).sum()), area * d
