"""Multigrid warm start of the EMD solve, float64 -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU baseline use this module (see the
package header).  The paper speeds up large gathers by a two-grid strategy (Sec. 2.2,
closing paragraph; Sec. 3.3): it solves the EMD on a resampled, coarser gather first,
builds the primal variable u on the original grid by sinc interpolation, and then runs
the primal-dual method on the fine grid from there.  In Sec. 3.3 only the time axis is
resampled (3000 x 227 samples become 301 x 227) and the coarse solve runs 150
iterations.

Readings taken where the paper is silent (listed with their reasons in the repository's
design notes):

* Q14 the coarse grid coarsens the time axis by an integer factor r and keeps every
       receiver.  Coarse sample J is the mean of fine samples rJ .. rJ + r - 1, the record
       being padded with zeros to a multiple of r, so the coarse gather carries the same
       mass (r dt sum_J f_c = dt sum_j f) and the coarse spacing is r dt.
* Q15 the coarse solve is Algorithm 1 unchanged, with the coarse spacings, run to a
       coarse tolerance or for a fixed number of iterations (Sec. 3.3 uses 150).
* Q16 "sinc interpolation" is the Whittaker-Shannon sum over every coarse sample of the
       record, v(x) = sum_J v_J sinc(x - J) with sinc(y) = sin(pi y) / (pi y), evaluated
       at the fine positions in coarse sample units.  Cell-centred quantities (phi and
       the x flux) sit at the cell centres: fine cell j is at x = (j - (r - 1)/2) / r.
       The time flux u^t[j] sits on the face between cells j - 1 and j: fine face j is
       at x = j / r.  The faces on the outer boundary (x flux of receiver 0, time flux
       of sample 0) carry no flux and are set to zero.
* Q17 phi is interpolated the same way as u and handed to the fine solve with it
       (``interpolate_phi``, default on); with it off the fine solve starts from
       phi = 0, as the paper's sentence reads literally.
"""

from __future__ import annotations

import math
from dataclasses import asdict, replace

import numpy as np

from .emd_oracle import Params, pdhg


def coarse_length(nt: int, r: int) -> int:
    """Number of coarse samples for nt fine samples and factor r (Q14)."""
    return -(-nt // r)


def restrict_time(a, r: int):
    """Coarse gather (Q14): mean of each block of r time samples, zero-padded tail.

    ``a`` is [nr][nt]; the result is [nr][ceil(nt / r)] in float64.
    """
    a = np.asarray(a, np.float64)
    nr, nt = a.shape
    nc = coarse_length(nt, r)
    padded = np.zeros((nr, nc * r))
    padded[:, :nt] = a
    return padded.reshape(nr, nc, r).sum(axis=2) / r


def fine_positions(nt: int, r: int, staggered: bool):
    """Fine sample positions in coarse sample units (Q16).

    Cell-centred: the centre of fine cell j lies at fine time j; coarse cell J covers fine
    cells rJ .. rJ + r - 1, so its centre lies at rJ + (r - 1)/2.  Staggered (time faces):
    fine face j lies at j - 1/2 and coarse face J at rJ - 1/2.
    """
    j = np.arange(nt, dtype=np.float64)
    return j / r if staggered else (j - (r - 1) / 2.0) / r


def sinc_interpolate(v, r: int, nt: int, staggered: bool):
    """Whittaker-Shannon interpolation of coarse rows ``v`` [nr][nc] onto nt fine
    positions (Q16): out[i, j] = sum_J v[i, J] sinc(x_j - J)."""
    v = np.asarray(v, np.float64)
    nc = v.shape[1]
    x = fine_positions(nt, r, staggered)
    kernel = np.sinc(x[None, :] - np.arange(nc, dtype=np.float64)[:, None])  # [nc][nt]
    return v @ kernel


def warm_start(phi_c, ux_c, ut_c, r: int, nt: int, interpolate_phi: bool = True):
    """Fine-grid starting point from a coarse solution (Q16, Q17): (phi0, m0[2][nr][nt])."""
    ux = sinc_interpolate(ux_c, r, nt, staggered=False)
    ut = sinc_interpolate(ut_c, r, nt, staggered=True)
    ux[0, :] = 0.0
    ut[:, 0] = 0.0
    phi = sinc_interpolate(phi_c, r, nt, staggered=False) if interpolate_phi \
        else np.zeros_like(ux)
    return phi, np.stack([ux, ut])


def pdhg_multigrid(p_obs, p_pred, dt, dx, factor: int, coarse: Params | None = None,
                   fine: Params | None = None, interpolate_phi: bool = True):
    """Two-grid solve (Sec. 2.2 closing paragraph, Sec. 3.3): restrict both gathers in
    time by ``factor``, run Algorithm 1 on the coarse grid (spacing factor * dt), sinc-
    interpolate its solution to the fine grid and run Algorithm 1 from there.

    Returns ``(coarse_result, fine_result)``, the two ``pdhg`` result dicts; the fine one
    carries the distance, phi and the flux of the fine grid.
    """
    coarse = coarse if coarse is not None else Params()
    fine = fine if fine is not None else Params()
    p_obs = np.asarray(p_obs, np.float64)
    p_pred = np.asarray(p_pred, np.float64)
    nt = p_obs.shape[1]
    c = pdhg(restrict_time(p_obs, factor), restrict_time(p_pred, factor),
             factor * dt, dx, replace(coarse, phi_init=None, m_init=None))
    phi0, m0 = warm_start(c["phi"], c["ux"], c["ut"], factor, nt, interpolate_phi)
    f = pdhg(p_obs, p_pred, dt, dx, Params(**{**asdict(fine), "phi_init": phi0, "m_init": m0}))
    return c, f


def sinc_bandlimit_error_bound(sigma: float) -> float:
    """Aliasing bound for a Gaussian of width ``sigma`` samples under Whittaker-Shannon
    interpolation: its spectrum beyond the Nyquist frequency is below exp(-2 pi^2
    sigma^2 / 4); the tests use this to size a tolerance, not to compute anything."""
    return math.exp(-2.0 * math.pi ** 2 * sigma ** 2 / 4.0)
