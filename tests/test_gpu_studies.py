"""The time / receiver weighting study of Sec. 3.3 on GPU results.

The paper compares EMD adjoint sources for Omega = [0, T] x [0, 1] with X = 1 and
T in {0.1, 1, 10}: a larger T makes transport along time dearer, so more of the mass is
moved across receivers.  Measured here as distances per unit of transported mass, which
the cell area and the data scale cancel out of: Dx = sum |u^x| / sum mu (mean distance
moved across receivers) grows with T, and Dt / T = sum |u^t| / sum mu / T (mean distance
moved along time, in units of the record length) shrinks.
"""

import numpy as np
import pytest
import torch

from oracle import emd_oracle as O
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


def test_larger_time_extent_moves_transport_across_receivers(P):
    obs, pred = synth.gather_pair_reflective(nt=4000, nr=480)
    o, p = obs[100:124, 1000:1128], pred[100:124, 1000:1128]  # 24 receivers x 128 samples
    nr, nt = o.shape
    dev = torch.device("cuda:0")
    to = torch.from_numpy(np.ascontiguousarray(o)).to(dev)
    tp = torch.from_numpy(np.ascontiguousarray(p)).to(dev)
    f = (p.astype(np.float64) - o) - (p.astype(np.float64) - o).mean()
    mu = np.maximum(f, 0).sum()
    dx_, dt_ = [], []
    for T in (0.1, 1.0, 10.0):
        _, _, m, info = P.emd(to, tp, T / (nt - 1), 1.0 / (nr - 1), max_iter=200000, tol=1e-4)
        assert info["status"] == P.EMD_OK
        m = m.double().cpu().numpy()
        dx_.append(np.abs(m[0]).sum() / mu)
        dt_.append(np.abs(m[1]).sum() / mu / T)
    assert dx_[0] < dx_[1] < dx_[2]
    assert dt_[0] > dt_[1] > dt_[2]
    # the FP64 oracle's figures for the same crop at T = 1 and 10 (T = 0.1 converges too
    # slowly on the CPU to run here)
    for n, T in ((1, 1.0), (2, 10.0)):
        r = O.pdhg(o, p, T / (nt - 1), 1.0 / (nr - 1), max_iter=40000, tol=1e-4)
        assert dx_[n] == pytest.approx(np.abs(r["ux"]).sum() / mu, rel=3e-2)
        assert dt_[n] == pytest.approx(np.abs(r["ut"]).sum() / mu / T, rel=3e-2)
