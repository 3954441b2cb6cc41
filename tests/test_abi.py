"""The C-ABI library loads, exports every symbol the header declares, agrees with the
ctypes mirrors on struct layout, and validates arguments (host-only calls; no GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emd_gb300.h")


@pytest.fixture(scope="module")
def B():
    from paper_1808_07284_gb300 import build
    build.build()
    import paper_1808_07284_gb300._binding as B
    B.lib()
    return B


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emd_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(B):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(B.lib(), n), n
    assert set(names) == set(B.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_struct_layout_matches_header(B, tmp_path):
    """Compile a probe against the header with gcc and compare sizes and offsets."""
    probe = tmp_path / "probe.c"
    fields_p = [f for f, _ in B.EmdParams._fields_]
    fields_r = [f for f, _ in B.EmdResult._fields_]
    fields_g = [f for f, _ in B.EmdMgParams._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "emd_gb300.h"', "int main(void){"]
    lines.append('printf("%zu %zu %zu\\n", sizeof(emd_params), sizeof(emd_result), sizeof(emd_mg_params));')
    for f in fields_p:
        lines.append(f'printf("p {f} %zu\\n", offsetof(emd_params, {f}));')
    for f in fields_r:
        lines.append(f'printf("r {f} %zu\\n", offsetof(emd_result, {f}));')
    for f in fields_g:
        lines.append(f'printf("g {f} %zu\\n", offsetof(emd_mg_params, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(probe), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sp, sr, sg = map(int, out[0].split())
    assert sp == ctypes.sizeof(B.EmdParams) and sr == ctypes.sizeof(B.EmdResult)
    assert sg == ctypes.sizeof(B.EmdMgParams)
    for line in out[1:]:
        if not line:
            continue
        kind, name, off = line.split()
        cls = {"p": B.EmdParams, "r": B.EmdResult, "g": B.EmdMgParams}[kind]
        assert getattr(cls, name).offset == int(off), name


def test_defaults_are_the_papers_constants(B):
    p = B.emd_default_params()
    assert (p.eps, p.xi, p.zeta, p.delta) == (1e-4, 0.5, 0.99, 1e5)
    assert p.max_iter == 2000 and p.linesearch == 1 and p.ls_norm == 2 and p.balance == B.EMD_BAL_MEAN
    assert p.tol == 0.0 and p.check_every == 10 and p.ls_max_trials == 40
    assert B.emd_tile_count() >= 1


def test_workspace_size(B):
    n = B.emd_workspace_size(3000, 400)
    assert n >= 36 * 3000 * 400
    assert B.emd_workspace_size(1, 5) == 0 and B.emd_workspace_size(5, 0) == 0
    nb = B.emd_batched_workspace_size([100, 200], [3, 4])
    assert nb >= B.emd_workspace_size(100, 3) + 36 * 200 * 4 - 4096


def test_argument_errors_need_no_gpu(B):
    """Invalid arguments come back as EMD_ERR_ARG / EMD_ERR_WORKSPACE before any CUDA call."""
    L = B.lib()
    res = B.EmdResult()
    p = B.emd_default_params()
    fake = ctypes.c_void_p(256)
    # nt < 2
    assert L.emd_dyn_solve(fake, fake, 1, 4, 1e-3, 10.0, ctypes.byref(p), fake, fake, ctypes.byref(res),
                           fake, 1 << 20, None) == B.EMD_ERR_ARG
    # dt <= 0
    assert L.emd_dyn_solve(fake, fake, 8, 4, 0.0, 10.0, ctypes.byref(p), fake, fake, ctypes.byref(res),
                           fake, 1 << 20, None) == B.EMD_ERR_ARG
    # null input
    assert L.emd_dyn_solve(None, fake, 8, 4, 1e-3, 10.0, ctypes.byref(p), fake, fake, ctypes.byref(res),
                           fake, 1 << 20, None) == B.EMD_ERR_ARG
    for bad in [dict(xi=1.0), dict(zeta=0.0), dict(delta=-1.0), dict(eps=-1e-4), dict(max_iter=0),
                dict(ls_norm=1), dict(balance=7), dict(tile=99), dict(linesearch=2)]:
        q = B.emd_default_params(**bad)
        assert L.emd_dyn_solve(fake, fake, 8, 4, 1e-3, 10.0, ctypes.byref(q), fake, fake,
                               ctypes.byref(res), fake, 1 << 20, None) == B.EMD_ERR_ARG, bad
    # workspace too small / misaligned
    assert L.emd_dyn_solve(fake, fake, 8, 4, 1e-3, 10.0, ctypes.byref(p), fake, fake, ctypes.byref(res),
                           fake, 16, None) == B.EMD_ERR_WORKSPACE
    assert L.emd_dyn_solve(fake, fake, 8, 4, 1e-3, 10.0, ctypes.byref(p), fake, fake, ctypes.byref(res),
                           ctypes.c_void_p(264), 1 << 20, None) == B.EMD_ERR_WORKSPACE
    assert L.emd_adjoint(fake, 8, 4, 1e-3, 10.0, 3, None, fake, None, fake, 1 << 20, None) == B.EMD_ERR_ARG
    assert L.emd_decompose(fake, None, 8, 4, 1e-3, 10.0, None, None, None, fake, 1 << 20, None) == B.EMD_ERR_ARG
    assert B.emd_status_string(B.EMD_ERR_LINESEARCH) == "linesearch did not terminate"


def test_two_grid_defaults_sizes_and_argument_errors(B):
    """Sec. 3.3 defaults; the two-grid workspace covers the fine solve; bad arguments are
    refused before any CUDA call."""
    g = B.emd_default_mg_params()
    assert (g.factor, g.coarse_max_iter, g.coarse_tol, g.interpolate_phi) == (10, 150, 0.0, 1)
    for f in (1, 2, 10, 1499):
        assert B.emd_mg_workspace_size(3000, 400, f) >= B.emd_workspace_size(3000, 400)
    assert B.emd_mg_workspace_size(3000, 400, 2999) > 0  # two coarse samples: the least there can be
    assert B.emd_mg_workspace_size(3000, 400, 3000) == 0
    assert B.emd_mg_workspace_size(3000, 400, 0) == 0
    assert B.emd_batched_mg_workspace_size([100, 200], [3, 4], 4) >= B.emd_batched_workspace_size([100, 200], [3, 4])
    L = B.lib()
    res, cres = B.EmdResult(), B.EmdResult()
    fake = ctypes.c_void_p(256)
    p = B.emd_default_params()
    ok = B.emd_default_mg_params(factor=4)
    big = 1 << 30

    def call(prm, mg, ws=fake, nbytes=big, nt=64, nr=4):
        return L.emd_dyn_solve_mg(fake, fake, nt, nr, 1e-3, 10.0, ctypes.byref(prm), ctypes.byref(mg), fake,
                                  fake, ctypes.byref(res), ctypes.byref(cres), ws, nbytes, None)

    for bad in [dict(factor=0), dict(coarse_max_iter=0), dict(coarse_tol=-1.0), dict(interpolate_phi=2),
                dict(factor=64)]:  # 64 samples by 64: one coarse sample
        mg = B.emd_default_mg_params(**{"factor": 4, **bad})
        assert call(p, mg, nbytes=16) == B.EMD_ERR_ARG, bad
    assert call(p, B.emd_default_mg_params(factor=63), nbytes=16) == B.EMD_ERR_WORKSPACE
    warm = B.emd_default_params()
    warm.phi_init = 256
    assert call(warm, ok) == B.EMD_ERR_ARG  # the warm start is the coarse solution
    assert call(p, ok, nbytes=16) == B.EMD_ERR_WORKSPACE
    assert call(p, ok, ws=ctypes.c_void_p(264)) == B.EMD_ERR_WORKSPACE
    assert L.emd_restrict_time(None, 64, 4, 4, fake, None) == B.EMD_ERR_ARG
    assert L.emd_restrict_time(fake, 64, 4, 0, fake, None) == B.EMD_ERR_ARG
    assert L.emd_prolong_time(fake, 16, 4, 4, 64, 2, 0, 0, fake, None) == B.EMD_ERR_ARG
    assert L.emd_prolong_time(fake, 0, 4, 4, 64, 0, 0, 0, fake, None) == B.EMD_ERR_ARG
    assert L.emd_prolong_time(fake, 1 << 20, 4, 1 << 10, 64, 0, 0, 0, fake, None) == B.EMD_ERR_ARG


def test_lsd_argument_errors(B):
    L = B.lib()
    fake = ctypes.c_void_p(256)
    v = ctypes.c_double()
    assert L.emd_lsd(None, fake, 8, 4, 1e-3, 10.0, ctypes.byref(v), fake, None, fake, 256, None) == B.EMD_ERR_ARG
    assert L.emd_lsd(fake, fake, 8, 4, -1.0, 10.0, ctypes.byref(v), fake, None, fake, 256, None) == B.EMD_ERR_ARG
    assert L.emd_lsd(fake, fake, 8, 4, 1e-3, 10.0, ctypes.byref(v), fake, None, fake, 128, None) == B.EMD_ERR_WORKSPACE
    assert L.emd_lsd(fake, fake, 8, 4, 1e-3, 10.0, ctypes.byref(v), fake, None, None, 256, None) == B.EMD_ERR_WORKSPACE


def test_product_path_has_no_oracle_or_fallback():
    """The package and the CUDA sources never reach into the oracle or the input generators."""
    pkg = os.path.join(ROOT, "paper_1808_07284_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+(oracle|synth)\b", text, flags=re.M), f


def test_batched_adjoint_argument_errors_need_no_gpu(B):
    """emd_adjoint_batched refuses bad sizes, spacings, balance, null pointers and a short or
    misaligned workspace before any CUDA call."""
    L = B.lib()
    P2, I2, D2 = ctypes.c_void_p * 2, ctypes.c_int * 2, ctypes.c_double * 2
    phis, gps = P2(256, 512), P2(768, 1024)
    nbytes = B.emd_batched_adjoint_workspace_size(2)
    assert B.emd_batched_adjoint_workspace_size(0) == 0 and nbytes >= 2 * 8
    fake = ctypes.c_void_p(256)

    def call(Bn=2, phi=phis, nt=(8, 8), nr=(4, 4), dt=(1e-3, 1e-3), dx=(10.0, 10.0), bal=1, gp=gps,
             ws=fake, n=nbytes):
        return L.emd_adjoint_batched(Bn, phi, I2(*nt), I2(*nr), D2(*dt), D2(*dx), bal, None, gp, None, ws, n,
                                     None)

    assert call(Bn=0) == B.EMD_ERR_ARG
    assert call(bal=3) == B.EMD_ERR_ARG
    assert call(phi=P2(256, None)) == B.EMD_ERR_ARG
    assert call(gp=P2(None, 512)) == B.EMD_ERR_ARG
    assert call(nt=(8, 1)) == B.EMD_ERR_ARG
    assert call(dt=(1e-3, 0.0)) == B.EMD_ERR_ARG
    assert call(dx=(float("nan"), 10.0)) == B.EMD_ERR_ARG
    assert call(n=nbytes - 8) == B.EMD_ERR_WORKSPACE
    assert call(ws=ctypes.c_void_p(264)) == B.EMD_ERR_WORKSPACE
    assert call(ws=None) == B.EMD_ERR_WORKSPACE


def test_host_misfit_argument_errors_need_no_gpu(B):
    """emd_misfit_batched_host sizes its workspace as the solve's plus the adjoint's plus the
    staging of each gather, and refuses bad sizes, spacings, parameters, warm starts, null
    pointers, B > 65535 and a short or misaligned workspace before any CUDA call."""
    L = B.lib()
    P2, I2, D2 = ctypes.c_void_p * 2, ctypes.c_int * 2, ctypes.c_double * 2
    nts, nrs = (8, 300), (4, 7)
    nbytes = B.emd_misfit_batched_host_workspace_size(list(nts), list(nrs))

    def a256(n):
        return (n + 255) // 256 * 256

    staging = sum(3 * a256(4 * t * r) + a256(8 * t * r) for t, r in zip(nts, nrs))
    assert nbytes == (a256(B.emd_batched_workspace_size(list(nts), list(nrs)))
                      + a256(B.emd_batched_adjoint_workspace_size(2)) + staging)
    assert B.emd_misfit_batched_host_workspace_size([8, 1], [4, 4]) == 0
    host = [(ctypes.c_float * (t * r))() for t, r in zip(nts, nrs)]
    ptrs = P2(*[ctypes.addressof(h) for h in host])
    res = (B.EmdResult * 2)()
    fake = ctypes.c_void_p(256)

    def call(Bn=2, obs=ptrs, pred=ptrs, nt=nts, nr=nrs, dt=(1e-3, 1e-3), dx=(10.0, 10.0), prm=None,
             ws=fake, n=nbytes, results=res):
        p = B.emd_default_params()
        for k, v in (prm or {}).items():
            setattr(p, k, v)
        return L.emd_misfit_batched_host(Bn, obs, pred, I2(*nt), I2(*nr), D2(*dt), D2(*dx), ctypes.byref(p),
                                         None, results, ws, n, None)

    assert call(Bn=0) == B.EMD_ERR_ARG
    assert call(Bn=65536) == B.EMD_ERR_ARG
    assert call(obs=P2(ptrs[0], None)) == B.EMD_ERR_ARG
    assert call(pred=None) == B.EMD_ERR_ARG
    assert call(results=None) == B.EMD_ERR_ARG
    assert call(nt=(8, 1)) == B.EMD_ERR_ARG
    assert call(dt=(1e-3, 0.0)) == B.EMD_ERR_ARG
    assert call(dx=(float("inf"), 10.0)) == B.EMD_ERR_ARG
    assert call(prm=dict(xi=1.5)) == B.EMD_ERR_ARG
    assert call(prm=dict(max_iter=0)) == B.EMD_ERR_ARG
    assert call(prm=dict(phi_init=256)) == B.EMD_ERR_ARG
    assert call(n=nbytes - 8) == B.EMD_ERR_WORKSPACE
    assert call(ws=ctypes.c_void_p(264)) == B.EMD_ERR_WORKSPACE
    assert call(ws=None) == B.EMD_ERR_WORKSPACE
