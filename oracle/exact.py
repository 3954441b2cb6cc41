"""Exact linear programs for the discrete EMD on tiny grids (TEST INFRASTRUCTURE).

Both LPs are solved with ``scipy.optimize.linprog`` (HiGHS).  They pin the PDHG oracle
from outside: at eps = 0 the dynamic problem of Sec. 2.1 with the l1 ground norm on the
grid graph is a min-cost flow, and by the equivalence of the formulations stated in
Sec. 2.1 it equals the Kantorovich transport LP with the Manhattan ground cost
dx |i_a - i_b| + dt |j_a - j_b|.
"""

from __future__ import annotations

import numpy as np


def _linprog():
    from scipy.optimize import linprog  # imported lazily: only the pin tests need scipy
    from scipy.sparse import coo_matrix
    return linprog, coo_matrix


def w1_flux_lp(f, dt, dx):
    """Min-cost flow on the grid graph with supplies dx dt f (sum f = 0).

    x-edges join (i-1, j) and (i, j) at cost dx per unit mass, t-edges join (i, j-1) and
    (i, j) at cost dt.  A unit of mass on an x-edge is dx dt |ux| / dt of flux, so the
    cost dx |F| equals dx dt |ux|: the optimum is min dx dt ||u||_{1,1} subject to
    div u + f = 0 with zero flux through the boundary.
    Returns (W, ux, ut) with the optimal flux in the units of u.
    """
    linprog, coo_matrix = _linprog()
    f = np.asarray(f, np.float64)
    nr, nt = f.shape
    area = dt if nr == 1 else dx * dt
    node = lambda i, j: i * nt + j  # noqa: E731
    tails, heads, costs, kinds = [], [], [], []
    for i in range(nr):
        for j in range(nt):
            if i >= 1:
                tails.append(node(i - 1, j)); heads.append(node(i, j)); costs.append(dx); kinds.append((0, i, j))
            if j >= 1:
                tails.append(node(i, j - 1)); heads.append(node(i, j)); costs.append(dt); kinds.append((1, i, j))
    ne = len(tails)
    # variables: forward flow F+_e (tail -> head) then backward flow F-_e, both >= 0
    rows, cols, vals = [], [], []
    for e in range(ne):
        rows += [tails[e], heads[e], tails[e], heads[e]]
        cols += [e, e, ne + e, ne + e]
        vals += [1.0, -1.0, -1.0, 1.0]
    A = coo_matrix((vals, (rows, cols)), shape=(nr * nt, 2 * ne)).tocsr()
    b = area * f.ravel()  # net outflow of each cell
    c = np.concatenate([costs, costs])
    res = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    flow = res.x[:ne] - res.x[ne:]
    ux = np.zeros((nr, nt))
    ut = np.zeros((nr, nt))
    for e, (kind, i, j) in enumerate(kinds):
        # flow from cell i-1 to cell i carries mass; the flux that moves it is
        # ux = -flow / dt (div u = -f makes u point against the mass leaving a source).
        if kind == 0:
            ux[i, j] = -flow[e] / dt
        else:
            ut[i, j] = -flow[e] / (dx if nr > 1 else 1.0)
    return float(res.fun), ux, ut


def w1_transport_lp(mu, nu, dt, dx):
    """Kantorovich LP between point masses dx dt mu_a and dx dt nu_b at the cell centres.

    Ground cost c(a, b) = dx |i_a - i_b| + dt |j_a - j_b| (the anisotropic l1 norm);
    requires sum mu = sum nu.  Returns the optimal cost.
    """
    linprog, coo_matrix = _linprog()
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    nr, nt = mu.shape
    area = dt if nr == 1 else dx * dt
    src = np.argwhere(mu > 0)
    snk = np.argwhere(nu > 0)
    ns, nk = len(src), len(snk)
    if ns == 0 or nk == 0:
        return 0.0
    cost = (dx * np.abs(src[:, None, 0] - snk[None, :, 0]) +
            dt * np.abs(src[:, None, 1] - snk[None, :, 1])).ravel()
    rows, cols = [], []
    for a in range(ns):
        for b in range(nk):
            v = a * nk + b
            rows += [a, ns + b]
            cols += [v, v]
    A = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(ns + nk, ns * nk)).tocsr()
    beq = area * np.concatenate([mu[tuple(src.T)], nu[tuple(snk.T)]])
    res = linprog(cost, A_eq=A, b_eq=beq, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return float(res.fun)
