"""GB300-native dynamic-formulation EMD misfit (arXiv 1808.07284).

The earth mover's distance between an observed and a predicted seismic gather
(receivers x time), compared through the Mainini recombination of Sec. 2.1 and solved
as the dynamic L1 transport problem of Sec. 2.2 by PDHG with linesearch (Algorithm 1),
in hand-written sm_103a CUDA behind the C ABI of ``include/emd_gb300.h``.  PyTorch
provides device memory, streams and autograd; every step of the method runs in the
library's kernels.

    dist, phi, m, info = emd(f_obs, f_pred, dt, dx, max_iter=2000)
    loss = emd_loss(f_pred, f_obs, dt, dx)      # differentiable w.r.t. both gathers
"""

from __future__ import annotations

from ._binding import (  # noqa: F401
    EMD_BAL_MEAN, EMD_BAL_NONE, EMD_ERR_ARG, EMD_NORM_ANISO, EMD_NORM_ISO, EMD_ERR_CUDA, EMD_ERR_LINESEARCH,
    EMD_ERR_NONFINITE, EMD_ERR_TIMEOUT, EMD_ERR_WORKSPACE, EMD_OK, EXPORTS,
    EmdError, EmdMgParams, EmdParams, EmdResult, emd_adjoint, emd_adjoint_batched,
    emd_batched_adjoint_workspace_size, emd_batched_mg_workspace_size,
    emd_batched_workspace_size, emd_decompose, emd_default_mg_params, emd_default_params,
    emd_dyn_solve, emd_dyn_solve_batched, emd_dyn_solve_batched_mg, emd_dyn_solve_mg,
    emd_dyn_solve_noalloc, emd_lsd, emd_mg_workspace_size, emd_misfit_batched_host,
    emd_misfit_batched_host_workspace_size, emd_prolong_time, emd_restrict_time,
    emd_status_string, emd_tile_count, emd_workspace_size, lib, new_workspace,
)

__all__ = [
    "emd", "emd_batched", "emd_loss", "emd_loss_batched", "EMDFunction", "EMDBatchFunction", "emd_decompose", "emd_dyn_solve",
    "emd_dyn_solve_batched", "emd_dyn_solve_noalloc", "emd_adjoint", "emd_default_params", "emd_workspace_size",
    "emd_batched_workspace_size", "emd_status_string", "emd_tile_count", "EmdError",
    "emd_dyn_solve_mg", "emd_dyn_solve_batched_mg", "emd_default_mg_params", "emd_mg_workspace_size",
    "emd_batched_mg_workspace_size", "emd_restrict_time", "emd_prolong_time", "emd_lsd", "lsd_loss",
    "LSDFunction", "emd_adjoint_batched", "emd_batched_adjoint_workspace_size", "emd_misfit_host",
    "emd_misfit_batched_host", "emd_misfit_batched_host_workspace_size",
]


def emd(f_obs, f_pred, dt, dx, workspace=None, stream=None, check=True, multigrid=None, **params):
    """One EMD solve.  Returns ``(dist, phi[nr, nt], m[2, nr, nt], info)``.

    ``params`` are ``emd_params`` fields (eps, xi, zeta, delta, alpha0, tol, max_iter,
    check_every, ls_max_trials, linesearch, balance, phi_init, m_init, tile, launch_mode,
    norm: EMD_NORM_ANISO or EMD_NORM_ISO).
    ``multigrid``: None for one solve, or a dict of ``emd_mg_params`` fields (factor,
    coarse_max_iter, coarse_tol, interpolate_phi; ``{}`` = the Sec. 3.3 setting) for the
    two-grid solve of Sec. 2.2/3.3; ``info["coarse"]`` then describes the coarse solve.
    """
    import torch
    nr, nt = f_obs.shape
    p = emd_default_params(**params)
    phi = torch.empty((nr, nt), dtype=torch.float32, device=f_obs.device)
    m = torch.empty((2, nr, nt), dtype=torch.float32, device=f_obs.device)
    if multigrid is not None:
        g = emd_default_mg_params(**multigrid)
        ws = workspace if workspace is not None else new_workspace(
            emd_mg_workspace_size(nt, nr, g.factor), f_obs.device)
        res, cres = emd_dyn_solve_mg(f_obs, f_pred, float(dt), float(dx), p, g, phi, m, ws, stream,
                                     check=check)
        info = res.as_dict()
        info["coarse"] = cres.as_dict()
        return res.dist, phi, m, info
    ws = workspace if workspace is not None else new_workspace(emd_workspace_size(nt, nr), f_obs.device)
    res = emd_dyn_solve(f_obs, f_pred, float(dt), float(dx), p, phi, m, ws, stream, check=check)
    return res.dist, phi, m, res.as_dict()


def emd_batched(f_obs, f_pred, dts, dxs, workspace=None, stream=None, check=True, multigrid=None,
                **params):
    """B independent solves together (by default one persistent launch runs every PDHG
    iteration of every gather, each gather with its own linesearch).  Lists in, lists out:
    ``(dists, phis, ms, infos)``.  ``multigrid`` as for :func:`emd` (both stages batched)."""
    import torch
    B = len(f_obs)
    dts = [float(v) for v in (dts if hasattr(dts, "__len__") else [dts] * B)]
    dxs = [float(v) for v in (dxs if hasattr(dxs, "__len__") else [dxs] * B)]
    p = emd_default_params(**params)
    phis = [torch.empty_like(t) for t in f_obs]
    ms = [torch.empty((2,) + tuple(t.shape), dtype=torch.float32, device=t.device) for t in f_obs]
    nts, nrs = [int(t.shape[1]) for t in f_obs], [int(t.shape[0]) for t in f_obs]
    if multigrid is not None:
        g = emd_default_mg_params(**multigrid)
        ws = workspace if workspace is not None else new_workspace(
            emd_batched_mg_workspace_size(nts, nrs, g.factor), f_obs[0].device)
        res, cres = emd_dyn_solve_batched_mg(f_obs, f_pred, dts, dxs, p, g, phis, ms, ws, stream,
                                             check=check)
        infos = [r.as_dict() for r in res]
        for i, c in zip(infos, cres):
            i["coarse"] = c.as_dict()
        return [r.dist for r in res], phis, ms, infos
    ws = workspace if workspace is not None else new_workspace(
        emd_batched_workspace_size(nts, nrs), f_obs[0].device)
    res = emd_dyn_solve_batched(f_obs, f_pred, dts, dxs, p, phis, ms, ws, stream, check=check)
    return [r.dist for r in res], phis, ms, [r.as_dict() for r in res]


def emd_misfit_host(f_obs, f_pred, dts, dxs, grad_preds=None, adjoint=True, workspace=None,
                    device=None, stream=None, check=True, **params):
    """Distances and adjoint sources of B gathers held in host memory, in one call of the C
    ABI (``emd_misfit_batched_host``): lists of CPU float32 tensors in (page-locked for the
    host link's full rate), ``(dists, grad_preds, infos)`` out.  ``grad_preds``: CPU tensors
    to receive the adjoint sources (allocated page-locked when None and ``adjoint``)."""
    import torch
    B = len(f_obs)
    dts = [float(v) for v in (dts if hasattr(dts, "__len__") else [dts] * B)]
    dxs = [float(v) for v in (dxs if hasattr(dxs, "__len__") else [dxs] * B)]
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    p = emd_default_params(**params)
    if adjoint and grad_preds is None:
        grad_preds = [torch.empty(tuple(t.shape), dtype=torch.float32).pin_memory() for t in f_obs]
    if not adjoint:
        grad_preds = None
    nts, nrs = [int(t.shape[1]) for t in f_obs], [int(t.shape[0]) for t in f_obs]
    ws = workspace if workspace is not None else new_workspace(
        emd_misfit_batched_host_workspace_size(nts, nrs), dev)
    res = emd_misfit_batched_host(f_obs, f_pred, dts, dxs, p, grad_preds, ws, stream, check=check)
    return [r.dist for r in res], grad_preds, [r.as_dict() for r in res]


def _autograd_function():
    import torch

    class EMDFunction(torch.autograd.Function):
        """dist = EMD(f_pred, f_obs); backward returns the adjoint source of Sec. 2.3,
        dx dt (phi - mean phi), from the phi kept by forward (no recomputation)."""

        @staticmethod
        def forward(ctx, f_pred, f_obs, dt, dx, params):
            dist, phi, _m, info = emd(f_obs.detach().contiguous(), f_pred.detach().contiguous(),
                                      dt, dx, **params)
            ctx.save_for_backward(phi)
            ctx.dt, ctx.dx = float(dt), float(dx)
            ctx.balance = params.get("balance", EMD_BAL_MEAN)
            ctx.info = info
            return torch.tensor(dist, dtype=torch.float32, device=f_pred.device)

        @staticmethod
        def backward(ctx, grad_out):
            (phi,) = ctx.saved_tensors
            nr, nt = phi.shape
            gp = torch.empty_like(phi)
            go = torch.empty_like(phi)
            ws = new_workspace(emd_workspace_size(nt, nr), phi.device)
            g = grad_out.detach().to(torch.float32).contiguous()
            emd_adjoint(phi, ctx.dt, ctx.dx, ctx.balance, g, gp, go, ws)
            return gp, go, None, None, None

    return EMDFunction


def _batched_autograd_function():
    import torch

    class EMDBatchFunction(torch.autograd.Function):
        """dists[b] = EMD(f_pred[b], f_obs[b]) for B gathers solved together; backward
        returns each gather's adjoint source from the phi kept by forward."""

        @staticmethod
        def forward(ctx, dts, dxs, params, *tensors):
            B = len(tensors) // 2
            preds = [t.detach().contiguous() for t in tensors[:B]]
            obss = [t.detach().contiguous() for t in tensors[B:]]
            dists, phis, _ms, infos = emd_batched(obss, preds, dts, dxs, **params)
            ctx.save_for_backward(*phis)
            ctx.dts, ctx.dxs = list(dts), list(dxs)
            ctx.balance = params.get("balance", EMD_BAL_MEAN)
            ctx.infos = infos
            return torch.tensor(dists, dtype=torch.float32, device=preds[0].device)

        @staticmethod
        def backward(ctx, grad_out):
            phis = ctx.saved_tensors
            B = len(phis)
            g = grad_out.detach().to(torch.float32).contiguous()
            gps = [torch.empty_like(phi) for phi in phis]
            gos = [torch.empty_like(phi) for phi in phis] if ctx.needs_input_grad[3 + B] else None
            ws = new_workspace(emd_batched_adjoint_workspace_size(B), phis[0].device)
            emd_adjoint_batched(list(phis), ctx.dts, ctx.dxs, ctx.balance, g, gps, gos, ws)
            return (None, None, None, *gps, *(gos if gos is not None else [None] * B))

    return EMDBatchFunction


def _lsd_autograd_function():
    import torch

    class LSDFunction(torch.autograd.Function):
        """The least-squares misfit of Sec. 2.1 with its adjoint source (Sec. 2.3) from the
        library's kernel: forward keeps the adjoint source it computed for backward."""

        @staticmethod
        def forward(ctx, f_pred, f_obs, dt, dx):
            gp = torch.empty_like(f_pred, dtype=torch.float32)
            v = emd_lsd(f_obs.detach().contiguous(), f_pred.detach().contiguous(), float(dt), float(dx),
                        grad_pred=gp)
            ctx.save_for_backward(gp)
            return torch.tensor(v, dtype=torch.float32, device=f_pred.device)

        @staticmethod
        def backward(ctx, grad_out):
            (gp,) = ctx.saved_tensors
            g = grad_out.to(torch.float32) * gp
            return g, -g, None, None

    return LSDFunction


_EMDFunction = None
_EMDBatchFunction = None
_LSDFunction = None


def __getattr__(name):
    global _EMDFunction, _EMDBatchFunction, _LSDFunction
    if name == "LSDFunction":
        if _LSDFunction is None:
            _LSDFunction = _lsd_autograd_function()
        return _LSDFunction
    if name == "EMDFunction":
        if _EMDFunction is None:
            _EMDFunction = _autograd_function()
        return _EMDFunction
    if name == "EMDBatchFunction":
        if _EMDBatchFunction is None:
            _EMDBatchFunction = _batched_autograd_function()
        return _EMDBatchFunction
    raise AttributeError(name)


def emd_loss(f_pred, f_obs, dt, dx, **params):
    """Differentiable EMD misfit (a 0-dim float32 tensor) with the library's adjoint source."""
    return __getattr__("EMDFunction").apply(f_pred, f_obs, dt, dx, params)


def emd_loss_batched(f_preds, f_obss, dts, dxs, **params):
    """Differentiable EMD misfits of B gathers solved in one batched solve: a float32
    tensor of B distances; backward gives each gather its adjoint source."""
    B = len(f_preds)
    dts = [float(v) for v in (dts if hasattr(dts, "__len__") else [dts] * B)]
    dxs = [float(v) for v in (dxs if hasattr(dxs, "__len__") else [dxs] * B)]
    return __getattr__("EMDBatchFunction").apply(dts, dxs, params, *f_preds, *f_obss)


def lsd_loss(f_pred, f_obs, dt, dx):
    """Differentiable least-squares misfit (a 0-dim float32 tensor), the baseline the paper
    compares the EMD with."""
    return __getattr__("LSDFunction").apply(f_pred, f_obs, dt, dx)
