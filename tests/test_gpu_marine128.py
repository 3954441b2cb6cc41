"""The large marine-streamer batch at full size: 128 shots of 8000 x 648 (dt = 2 ms,
dx = 25 m; 663 M cells, 24 GB of solver state) solved and differentiated in one batched
call, as the batched training step would run it.  Four sampled shots are checked against
the FP64 oracle after the same 12 iterations: distance, potential and adjoint source.
"""

import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

from oracle import emd_oracle as O
import synth

pytestmark = pytest.mark.gpu

N_SHOTS = 128
SAMPLED = (0, 41, 86, 127)
K = 12
DT, DX = 2e-3, 25.0


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_07284_gb300 import build
    build.build()
    import paper_1808_07284_gb300 as P
    return P


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_128_shot_batch_forward_backward_sampled_against_oracle(P):
    # generating 128 gathers takes ~1.6 s each: a spawn pool (safe after CUDA is up)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        pairs = pool.map(synth.marine_shot, range(N_SHOTS))
    dev = torch.device("cuda:0")
    obs = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    preds = [torch.from_numpy(p).to(dev).requires_grad_(True) for _, p in pairs]
    d = P.emd_loss_batched(preds, obs, DT, DX, max_iter=K)
    assert d.shape == (N_SHOTS,) and torch.isfinite(d).all()
    d.sum().backward()
    for b in SAMPLED:
        o, p = pairs[b]
        r = O.pdhg(o, p, DT, DX, max_iter=K)
        g_ref, _ = O.adjoint_source(r["phi"], DT, DX)
        assert d[b].item() == pytest.approx(r["dist"], rel=1e-4)
        assert _rel_l2(preds[b].grad.double().cpu().numpy(), g_ref) <= 1e-3
