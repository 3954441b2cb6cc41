"""ctypes binding of the C ABI in ``include/emd_gb300.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and takes torch tensors
where the C function takes device pointers.  No arithmetic of the method happens in
Python: if the shared library is missing, loading fails loudly; there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

c_double, c_int, c_size_t, c_void_p = ctypes.c_double, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p

EMD_OK, EMD_ERR_ARG, EMD_ERR_CUDA, EMD_ERR_NONFINITE, EMD_ERR_LINESEARCH, EMD_ERR_TIMEOUT, EMD_ERR_WORKSPACE = range(7)
EMD_BAL_NONE, EMD_BAL_MEAN = 0, 1
EMD_NORM_ANISO, EMD_NORM_ISO = 1, 2

EXPORTS = (
    "emd_default_params", "emd_tile_count", "emd_workspace_size", "emd_decompose",
    "emd_dyn_solve", "emd_batched_workspace_size", "emd_dyn_solve_batched", "emd_adjoint",
    "emd_status_string", "emd_dyn_solve_noalloc", "emd_default_mg_params", "emd_mg_workspace_size",
    "emd_batched_mg_workspace_size", "emd_restrict_time", "emd_prolong_time", "emd_dyn_solve_mg",
    "emd_dyn_solve_batched_mg", "emd_lsd", "emd_batched_adjoint_workspace_size", "emd_adjoint_batched",
    "emd_misfit_batched_host_workspace_size", "emd_misfit_batched_host",
)


class EmdParams(ctypes.Structure):
    """Mirror of ``emd_params``."""

    _fields_ = [
        ("eps", c_double), ("xi", c_double), ("zeta", c_double), ("delta", c_double),
        ("alpha0", c_double), ("tol", c_double),
        ("max_iter", c_int), ("check_every", c_int), ("ls_max_trials", c_int),
        ("linesearch", c_int), ("ls_norm", c_int), ("balance", c_int),
        ("phi_init", c_void_p), ("m_init", c_void_p),
        ("tile", c_int), ("launch_mode", c_int), ("debug_fault", c_int),
        ("trace", c_void_p), ("norm", c_int),
    ]


class EmdMgParams(ctypes.Structure):
    """Mirror of ``emd_mg_params``."""

    _fields_ = [
        ("factor", c_int), ("coarse_max_iter", c_int), ("coarse_tol", c_double),
        ("interpolate_phi", c_int),
    ]


class EmdResult(ctypes.Structure):
    """Mirror of ``emd_result``."""

    _fields_ = [
        ("dist", c_double), ("dist_l1", c_double), ("mass_mu", c_double), ("mass_nu", c_double),
        ("imbalance", c_double), ("residual", c_double), ("r_feas", c_double), ("r_step", c_double),
        ("duality_gap", c_double), ("alpha", c_double), ("theta", c_double),
        ("iters", c_int), ("ls_trials", c_int), ("status", c_int), ("launches", c_int),
        ("tile", c_int),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class EmdError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} (status {status})")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (built in-tree by ``paper_1808_07284_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it first (python -m paper_1808_07284_gb300.build "
                "or __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.emd_default_params.argtypes = [P(EmdParams)]
        L.emd_default_params.restype = None
        L.emd_tile_count.argtypes = []
        L.emd_tile_count.restype = c_int
        L.emd_workspace_size.argtypes = [c_int, c_int]
        L.emd_workspace_size.restype = c_size_t
        L.emd_decompose.argtypes = [c_void_p, c_void_p, c_int, c_int, c_double, c_double, c_void_p,
                                    c_void_p, P(c_double), c_void_p, c_size_t, c_void_p]
        L.emd_decompose.restype = c_int
        L.emd_dyn_solve.argtypes = [c_void_p, c_void_p, c_int, c_int, c_double, c_double,
                                    P(EmdParams), c_void_p, c_void_p, P(EmdResult), c_void_p,
                                    c_size_t, c_void_p]
        L.emd_dyn_solve.restype = c_int
        L.emd_batched_workspace_size.argtypes = [c_int, P(c_int), P(c_int)]
        L.emd_batched_workspace_size.restype = c_size_t
        L.emd_dyn_solve_batched.argtypes = [c_int, P(c_void_p), P(c_void_p), P(c_int), P(c_int),
                                            P(c_double), P(c_double), P(EmdParams), P(c_void_p),
                                            P(c_void_p), P(EmdResult), c_void_p, c_size_t, c_void_p]
        L.emd_dyn_solve_batched.restype = c_int
        L.emd_adjoint.argtypes = [c_void_p, c_int, c_int, c_double, c_double, c_int, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
        L.emd_adjoint.restype = c_int
        L.emd_batched_adjoint_workspace_size.argtypes = [c_int]
        L.emd_batched_adjoint_workspace_size.restype = c_size_t
        L.emd_adjoint_batched.argtypes = [c_int, P(c_void_p), P(c_int), P(c_int), P(c_double),
                                          P(c_double), c_int, c_void_p, P(c_void_p), P(c_void_p),
                                          c_void_p, c_size_t, c_void_p]
        L.emd_adjoint_batched.restype = c_int
        L.emd_misfit_batched_host_workspace_size.argtypes = [c_int, P(c_int), P(c_int)]
        L.emd_misfit_batched_host_workspace_size.restype = c_size_t
        L.emd_misfit_batched_host.argtypes = [c_int, P(c_void_p), P(c_void_p), P(c_int), P(c_int),
                                              P(c_double), P(c_double), P(EmdParams), P(c_void_p),
                                              P(EmdResult), c_void_p, c_size_t, c_void_p]
        L.emd_misfit_batched_host.restype = c_int
        L.emd_dyn_solve_noalloc.argtypes = [c_void_p, c_void_p, c_int, c_int, c_double, c_double,
                                            P(EmdParams), c_void_p, c_void_p, P(EmdResult), c_void_p]
        L.emd_dyn_solve_noalloc.restype = c_int
        L.emd_default_mg_params.argtypes = [P(EmdMgParams)]
        L.emd_default_mg_params.restype = None
        L.emd_mg_workspace_size.argtypes = [c_int, c_int, c_int]
        L.emd_mg_workspace_size.restype = c_size_t
        L.emd_batched_mg_workspace_size.argtypes = [c_int, P(c_int), P(c_int), c_int]
        L.emd_batched_mg_workspace_size.restype = c_size_t
        L.emd_restrict_time.argtypes = [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]
        L.emd_restrict_time.restype = c_int
        L.emd_prolong_time.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_int,
                                       c_void_p, c_void_p]
        L.emd_prolong_time.restype = c_int
        L.emd_dyn_solve_mg.argtypes = [c_void_p, c_void_p, c_int, c_int, c_double, c_double,
                                       P(EmdParams), P(EmdMgParams), c_void_p, c_void_p,
                                       P(EmdResult), P(EmdResult), c_void_p, c_size_t, c_void_p]
        L.emd_dyn_solve_mg.restype = c_int
        L.emd_dyn_solve_batched_mg.argtypes = [c_int, P(c_void_p), P(c_void_p), P(c_int), P(c_int),
                                               P(c_double), P(c_double), P(EmdParams),
                                               P(EmdMgParams), P(c_void_p), P(c_void_p),
                                               P(EmdResult), P(EmdResult), c_void_p, c_size_t,
                                               c_void_p]
        L.emd_dyn_solve_batched_mg.restype = c_int
        L.emd_lsd.argtypes = [c_void_p, c_void_p, c_int, c_int, c_double, c_double, P(c_double),
                              c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
        L.emd_lsd.restype = c_int
        L.emd_status_string.argtypes = [c_int]
        L.emd_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


# ------------------------------------------------------------------------------ marshalling

def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check_grid(t, nr, nt, name, planes=1):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.numel() != planes * nr * nt:
        raise ValueError(f"{name} must hold {planes} x {nr} x {nt} elements, got {t.numel()}")


def emd_default_params(**overrides) -> EmdParams:
    p = EmdParams()
    lib().emd_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        if k in ("phi_init", "m_init", "trace"):
            v = _ptr(v)
        setattr(p, k, v)
    return p


def emd_default_mg_params(**overrides) -> EmdMgParams:
    g = EmdMgParams()
    lib().emd_default_mg_params(ctypes.byref(g))
    for k, v in overrides.items():
        if not hasattr(g, k):
            raise TypeError(f"unknown two-grid parameter {k}")
        setattr(g, k, v)
    return g


def emd_mg_workspace_size(nt: int, nr: int, factor: int) -> int:
    return lib().emd_mg_workspace_size(nt, nr, factor)


def emd_batched_mg_workspace_size(nts, nrs, factor: int) -> int:
    B = len(nts)
    return lib().emd_batched_mg_workspace_size(B, (c_int * B)(*nts), (c_int * B)(*nrs), factor)


def emd_tile_count() -> int:
    return lib().emd_tile_count()


def emd_workspace_size(nt: int, nr: int) -> int:
    return lib().emd_workspace_size(nt, nr)


def emd_batched_workspace_size(nts, nrs) -> int:
    B = len(nts)
    return lib().emd_batched_workspace_size(B, (c_int * B)(*nts), (c_int * B)(*nrs))


def emd_status_string(status: int) -> str:
    return lib().emd_status_string(status).decode()


status_string = emd_status_string


def emd_decompose(f_obs, f_pred, dt, dx, mu=None, nu=None, workspace=None, stream=None):
    """Returns (masses[2] on the host) and fills mu, nu if given (Sec. 2.1)."""
    nr, nt = f_obs.shape
    _check_grid(f_obs, nr, nt, "f_obs")
    _check_grid(f_pred, nr, nt, "f_pred")
    ws = workspace if workspace is not None else new_workspace(emd_workspace_size(nt, nr), f_obs.device)
    masses = (c_double * 2)()
    st = lib().emd_decompose(_ptr(f_obs), _ptr(f_pred), nt, nr, dt, dx, _ptr(mu), _ptr(nu), masses,
                             _ptr(ws), ws.numel(), _stream(stream))
    if st != EMD_OK:
        raise EmdError(st, "emd_decompose")
    return masses[0], masses[1]


def new_workspace(nbytes: int, device):
    import torch
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def emd_dyn_solve(f_obs, f_pred, dt, dx, params: EmdParams, phi, m, workspace, stream=None,
                  check: bool = True) -> EmdResult:
    """One solve through the C ABI; phi [nr, nt] and m [2, nr, nt] are written in place."""
    nr, nt = f_obs.shape
    _check_grid(f_obs, nr, nt, "f_obs")
    _check_grid(f_pred, nr, nt, "f_pred")
    _check_grid(phi, nr, nt, "phi")
    _check_grid(m, nr, nt, "m", planes=2)
    res = EmdResult()
    st = lib().emd_dyn_solve(_ptr(f_obs), _ptr(f_pred), nt, nr, dt, dx, ctypes.byref(params),
                             _ptr(phi), _ptr(m), ctypes.byref(res), _ptr(workspace),
                             workspace.numel(), _stream(stream))
    if check and st not in (EMD_OK,):
        raise EmdError(st, "emd_dyn_solve")
    return res


def emd_dyn_solve_batched(f_obs, f_pred, dts, dxs, params: EmdParams, phis, ms, workspace,
                          stream=None, check: bool = True):
    """B solves through the C ABI; lists of tensors; returns a list of EmdResult."""
    B = len(f_obs)
    nts, nrs = [int(t.shape[1]) for t in f_obs], [int(t.shape[0]) for t in f_obs]
    for b in range(B):
        _check_grid(f_obs[b], nrs[b], nts[b], f"f_obs[{b}]")
        _check_grid(f_pred[b], nrs[b], nts[b], f"f_pred[{b}]")
        _check_grid(phis[b], nrs[b], nts[b], f"phi[{b}]")
        _check_grid(ms[b], nrs[b], nts[b], f"m[{b}]", planes=2)
    P = c_void_p * B
    res = (EmdResult * B)()
    st = lib().emd_dyn_solve_batched(
        B, P(*[_ptr(t) for t in f_obs]), P(*[_ptr(t) for t in f_pred]), (c_int * B)(*nts),
        (c_int * B)(*nrs), (c_double * B)(*dts), (c_double * B)(*dxs), ctypes.byref(params),
        P(*[_ptr(t) for t in phis]), P(*[_ptr(t) for t in ms]), res, _ptr(workspace),
        workspace.numel(), _stream(stream))
    if check and st != EMD_OK:
        raise EmdError(st, "emd_dyn_solve_batched")
    return list(res)


def emd_adjoint(phi, dt, dx, balance, grad_out, grad_pred, grad_obs, workspace, stream=None):
    """d dist / d Pcal (and its negative for Pobs) from phi (Sec. 2.3); grad_out is a device scalar or None."""
    nr, nt = phi.shape
    _check_grid(phi, nr, nt, "phi")
    _check_grid(grad_pred, nr, nt, "grad_pred")
    if grad_obs is not None:
        _check_grid(grad_obs, nr, nt, "grad_obs")
    st = lib().emd_adjoint(_ptr(phi), nt, nr, dt, dx, balance, _ptr(grad_out), _ptr(grad_pred),
                           _ptr(grad_obs), _ptr(workspace), workspace.numel(), _stream(stream))
    if st != EMD_OK:
        raise EmdError(st, "emd_adjoint")


def emd_batched_adjoint_workspace_size(B: int) -> int:
    return lib().emd_batched_adjoint_workspace_size(B)


def emd_adjoint_batched(phis, dts, dxs, balance, grad_out, grad_preds, grad_obss, workspace, stream=None):
    """Adjoint sources of B gathers in two launches (Sec. 2.3); grad_out is a device vector of B
    floats or None; grad_obss a list (entries may be None) or None."""
    B = len(phis)
    nts, nrs = [int(t.shape[1]) for t in phis], [int(t.shape[0]) for t in phis]
    for b in range(B):
        _check_grid(phis[b], nrs[b], nts[b], f"phi[{b}]")
        _check_grid(grad_preds[b], nrs[b], nts[b], f"grad_pred[{b}]")
        if grad_obss is not None and grad_obss[b] is not None:
            _check_grid(grad_obss[b], nrs[b], nts[b], f"grad_obs[{b}]")
    if grad_out is not None and (grad_out.numel() != B or not grad_out.is_contiguous()):
        raise ValueError("grad_out must be a contiguous device vector of B floats")
    P = c_void_p * B
    go = None if grad_obss is None else P(*[_ptr(t) for t in grad_obss])
    st = lib().emd_adjoint_batched(B, P(*[_ptr(t) for t in phis]), (c_int * B)(*nts), (c_int * B)(*nrs),
                                   (c_double * B)(*dts), (c_double * B)(*dxs), balance, _ptr(grad_out),
                                   P(*[_ptr(t) for t in grad_preds]), go, _ptr(workspace),
                                   workspace.numel(), _stream(stream))
    if st != EMD_OK:
        raise EmdError(st, "emd_adjoint_batched")


def emd_misfit_batched_host_workspace_size(nts, nrs) -> int:
    B = len(nts)
    return lib().emd_misfit_batched_host_workspace_size(B, (c_int * B)(*nts), (c_int * B)(*nrs))


def _check_host_grid(t, nr, nt, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CPU tensor")
    if t.numel() != nr * nt:
        raise ValueError(f"{name} must hold {nr} x {nt} elements, got {t.numel()}")


def emd_misfit_batched_host(f_obs, f_pred, dts, dxs, params: EmdParams, grad_preds, workspace,
                            stream=None, check: bool = True):
    """Distances and adjoint sources of B gathers held in host memory (CPU tensors, pinned
    for full speed); grad_preds: list of CPU tensors (entries may be None) or None.
    Returns a list of EmdResult."""
    B = len(f_obs)
    nts, nrs = [int(t.shape[1]) for t in f_obs], [int(t.shape[0]) for t in f_obs]
    for b in range(B):
        _check_host_grid(f_obs[b], nrs[b], nts[b], f"f_obs[{b}]")
        _check_host_grid(f_pred[b], nrs[b], nts[b], f"f_pred[{b}]")
        if grad_preds is not None and grad_preds[b] is not None:
            _check_host_grid(grad_preds[b], nrs[b], nts[b], f"grad_pred[{b}]")
    P = c_void_p * B
    gp = None if grad_preds is None else P(*[_ptr(t) for t in grad_preds])
    res = (EmdResult * B)()
    st = lib().emd_misfit_batched_host(
        B, P(*[_ptr(t) for t in f_obs]), P(*[_ptr(t) for t in f_pred]), (c_int * B)(*nts),
        (c_int * B)(*nrs), (c_double * B)(*dts), (c_double * B)(*dxs), ctypes.byref(params), gp,
        res, _ptr(workspace), workspace.numel(), _stream(stream))
    if check and st != EMD_OK:
        raise EmdError(st, "emd_misfit_batched_host")
    return list(res)


def emd_dyn_solve_noalloc(f_obs, f_pred, dt, dx, params: EmdParams, phi, m, stream=None,
                          check: bool = True) -> EmdResult:
    """emd_dyn_solve on the library's built-in scratch array (no workspace, no allocation)."""
    nr, nt = f_obs.shape
    _check_grid(f_obs, nr, nt, "f_obs")
    _check_grid(f_pred, nr, nt, "f_pred")
    _check_grid(phi, nr, nt, "phi")
    _check_grid(m, nr, nt, "m", planes=2)
    res = EmdResult()
    st = lib().emd_dyn_solve_noalloc(_ptr(f_obs), _ptr(f_pred), nt, nr, dt, dx, ctypes.byref(params),
                                     _ptr(phi), _ptr(m), ctypes.byref(res), _stream(stream))
    if check and st != EMD_OK:
        raise EmdError(st, "emd_dyn_solve_noalloc")
    return res


def emd_restrict_time(x, factor: int, out, stream=None):
    """Time restriction of a [nr, nt] gather into out [nr, ceil(nt / factor)] (block means)."""
    nr, nt = x.shape
    _check_grid(x, nr, nt, "in")
    _check_grid(out, nr, -(-nt // factor), "out")
    st = lib().emd_restrict_time(_ptr(x), nt, nr, factor, _ptr(out), _stream(stream))
    if st != EMD_OK:
        raise EmdError(st, "emd_restrict_time")


def emd_prolong_time(x, factor: int, out, staggered: bool, zero_row0=False, zero_col0=False,
                     stream=None):
    """Sinc interpolation of coarse rows x [nr, nc] onto out [nr, nt]."""
    nr, nc = x.shape
    nt = int(out.shape[-1])
    _check_grid(x, nr, nc, "in")
    _check_grid(out, nr, nt, "out")
    st = lib().emd_prolong_time(_ptr(x), nc, nr, factor, nt, int(staggered), int(zero_row0),
                                int(zero_col0), _ptr(out), _stream(stream))
    if st != EMD_OK:
        raise EmdError(st, "emd_prolong_time")


def emd_dyn_solve_mg(f_obs, f_pred, dt, dx, params: EmdParams, mg: EmdMgParams, phi, m, workspace,
                     stream=None, check: bool = True):
    """Two-grid solve through the C ABI; returns (fine EmdResult, coarse EmdResult)."""
    nr, nt = f_obs.shape
    _check_grid(f_obs, nr, nt, "f_obs")
    _check_grid(f_pred, nr, nt, "f_pred")
    _check_grid(phi, nr, nt, "phi")
    _check_grid(m, nr, nt, "m", planes=2)
    res, cres = EmdResult(), EmdResult()
    st = lib().emd_dyn_solve_mg(_ptr(f_obs), _ptr(f_pred), nt, nr, dt, dx, ctypes.byref(params),
                                ctypes.byref(mg), _ptr(phi), _ptr(m), ctypes.byref(res),
                                ctypes.byref(cres), _ptr(workspace), workspace.numel(),
                                _stream(stream))
    if check and st != EMD_OK:
        raise EmdError(st, "emd_dyn_solve_mg")
    return res, cres


def emd_dyn_solve_batched_mg(f_obs, f_pred, dts, dxs, params: EmdParams, mg: EmdMgParams, phis, ms,
                             workspace, stream=None, check: bool = True):
    """B two-grid solves through the C ABI; returns (fine results, coarse results)."""
    B = len(f_obs)
    nts, nrs = [int(t.shape[1]) for t in f_obs], [int(t.shape[0]) for t in f_obs]
    for b in range(B):
        _check_grid(f_obs[b], nrs[b], nts[b], f"f_obs[{b}]")
        _check_grid(f_pred[b], nrs[b], nts[b], f"f_pred[{b}]")
        _check_grid(phis[b], nrs[b], nts[b], f"phi[{b}]")
        _check_grid(ms[b], nrs[b], nts[b], f"m[{b}]", planes=2)
    P = c_void_p * B
    res, cres = (EmdResult * B)(), (EmdResult * B)()
    st = lib().emd_dyn_solve_batched_mg(
        B, P(*[_ptr(t) for t in f_obs]), P(*[_ptr(t) for t in f_pred]), (c_int * B)(*nts),
        (c_int * B)(*nrs), (c_double * B)(*dts), (c_double * B)(*dxs), ctypes.byref(params),
        ctypes.byref(mg), P(*[_ptr(t) for t in phis]), P(*[_ptr(t) for t in ms]), res, cres,
        _ptr(workspace), workspace.numel(), _stream(stream))
    if check and st != EMD_OK:
        raise EmdError(st, "emd_dyn_solve_batched_mg")
    return list(res), list(cres)


def emd_lsd(f_obs, f_pred, dt, dx, grad_pred=None, grad_obs=None, workspace=None, stream=None) -> float:
    """Least-squares misfit (Sec. 2.1) on the host; fills the adjoint sources if given."""
    nr, nt = f_obs.shape
    _check_grid(f_obs, nr, nt, "f_obs")
    _check_grid(f_pred, nr, nt, "f_pred")
    for t, name in ((grad_pred, "grad_pred"), (grad_obs, "grad_obs")):
        if t is not None:
            _check_grid(t, nr, nt, name)
    ws = workspace if workspace is not None else new_workspace(256, f_obs.device)
    v = c_double()
    st = lib().emd_lsd(_ptr(f_obs), _ptr(f_pred), nt, nr, dt, dx, ctypes.byref(v), _ptr(grad_pred),
                       _ptr(grad_obs), _ptr(ws), ws.numel(), _stream(stream))
    if st != EMD_OK:
        raise EmdError(st, "emd_lsd")
    return v.value
