"""The no-allocation solve entry point against the regular one (needs a GPU).

emd_dyn_solve_noalloc serves callers that cannot allocate device memory (code whose host
framework owns every device allocation, loops that must not block on an allocation); it
runs on a scratch array built into the library.  Two calls in a row must each give the
regular entry point's result, within the parity tolerances of the other GPU tests.  This
file sorts last so that a run stopping at the first failure has run every other test
before it.
"""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07284_gb300 import build
    build.build()
    import paper_1808_07284_gb300 as P
    return P


def _rel_l2(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_workspace_entry_twice(P):
    dev = torch.device("cuda:0")
    obs, pred = synth.gather_pair_hyperbolic()  # 256 x 64
    o = torch.from_numpy(obs).to(dev)
    p = torch.from_numpy(pred).to(dev)
    nr, nt = obs.shape
    params = P.emd_default_params(max_iter=500)
    phi_ref = torch.empty((nr, nt), dtype=torch.float32, device=dev)
    m_ref = torch.empty((2, nr, nt), dtype=torch.float32, device=dev)
    ws = P.new_workspace(P.emd_workspace_size(nt, nr), dev)
    ref = P.emd_dyn_solve(o, p, 2e-3, 10.0, params, phi_ref, m_ref, ws)
    for call in range(2):
        phi = torch.full((nr, nt), float("nan"), dtype=torch.float32, device=dev)
        m = torch.full((2, nr, nt), float("nan"), dtype=torch.float32, device=dev)
        res = P.emd_dyn_solve_noalloc(o, p, 2e-3, 10.0, params, phi, m)
        torch.cuda.synchronize()
        assert res.status == P.EMD_OK, call
        assert res.iters == ref.iters == 500
        assert res.ls_trials == ref.ls_trials
        assert res.dist == pytest.approx(ref.dist, rel=1e-4)
        assert _rel_l2(phi, phi_ref) <= 1e-3
        assert _rel_l2(m, m_ref) <= 1e-3


def test_noalloc_rejects_gathers_beyond_its_scratch(P):
    dev = torch.device("cuda:0")
    nr, nt = 400, 3000  # 43 MB of solver state, beyond the 16 MiB built-in scratch
    o = torch.zeros((nr, nt), dtype=torch.float32, device=dev)
    phi = torch.empty_like(o)
    m = torch.empty((2, nr, nt), dtype=torch.float32, device=dev)
    with pytest.raises(P.EmdError) as err:
        P.emd_dyn_solve_noalloc(o, o, 1e-3, 12.5, P.emd_default_params(), phi, m)
    assert err.value.status == P.EMD_ERR_WORKSPACE
    st = P.lib().emd_dyn_solve_noalloc(o.data_ptr(), o.data_ptr(), nt, nr, 1e-3, 12.5, None,
                                       phi.data_ptr(), m.data_ptr(), None, None)
    assert st == P.EMD_ERR_WORKSPACE
