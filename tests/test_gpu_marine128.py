"""The large marine-streamer batch at full size: 128 shots of 8000 x 648 (dt = 2 ms,
dx = 25 m; 663 M cells, 24 GB of solver state) solved and differentiated in one batched
call at 200 iterations, as the batched training step runs it.  Four sampled shots are
checked against the FP64 oracle, which replays the GPU's linesearch decisions (every
contradicted decision must be a near tie): distance, potential and adjoint source.
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
K = 200
DT, DX = 2e-3, 25.0
NEAR_TIE = 1e-3


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


def _replay(shot, trials):
    """The oracle on one shot with the GPU's trial counts (a spawn-pool worker)."""
    obs, pred = synth.gather_pair_marine(shot=shot)
    r = O.pdhg(obs, pred, DT, DX, max_iter=K, record=True, force_trials=np.asarray(trials, np.int64))
    g, _ = O.adjoint_source(r["phi"], DT, DX)
    return r["dist"], g.astype(np.float32), r["trace"]


def test_128_shot_batch_forward_backward_sampled_against_oracle(P):
    # generating 128 gathers takes ~1.6 s each: a spawn pool (safe after CUDA is up)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        pairs = pool.map(synth.marine_shot, range(N_SHOTS))
    dev = torch.device("cuda:0")
    obs = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    preds = [torch.from_numpy(p).to(dev).requires_grad_(True) for _, p in pairs]
    del pairs
    trace = torch.full((N_SHOTS, K, 4), float("nan"), dtype=torch.float64, device=dev)
    d = P.emd_loss_batched(preds, obs, DT, DX, max_iter=K, trace=trace)
    assert d.shape == (N_SHOTS,) and torch.isfinite(d).all()
    d.sum().backward()
    tr = trace.cpu().numpy()
    assert np.isfinite(tr[:, :, 2]).all()  # every gather ran all K iterations
    with mp.get_context("spawn").Pool(len(SAMPLED)) as pool:
        jobs = {b: pool.apply_async(_replay, (b, tr[b, :, 2].astype(int).tolist())) for b in SAMPLED}
        for b, job in jobs.items():
            dist, g_ref, otr = job.get()
            assert otr[:, 6].max() < NEAR_TIE, (b, int(np.argmax(otr[:, 6])))
            np.testing.assert_allclose(tr[b, :, 0], otr[:, 0], rtol=1e-9)
            assert d[b].item() == pytest.approx(dist, rel=1e-4)
            assert _rel_l2(preds[b].grad.double().cpu().numpy(), g_ref.astype(np.float64)) <= 1e-3
