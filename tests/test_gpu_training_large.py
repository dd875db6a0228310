"""Force matching of the learned draft on frames larger than one block (the frame's atoms as rows of the batched
neighbour, descriptor and force kernels, then the residual, the descriptor JVP and the per-weight sums of the
double backward), against the oracle's FP64 loss and exact gradient; and online retraining during lsd_step on the
target-verified frames the verification captures."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W
from parity_bounds import rel

pytestmark = pytest.mark.gpu


def _system(kind):
    if kind == "cells":
        # 512 atoms, 32 A box: a cell grid of five cells per axis, so each frame's lists come from the Verlet kernels
        pos = W.jitter(W.simple_cubic(8, 4.0), 4.0, seed=13)
        sp = (np.arange(512) % 3 == 0).astype(np.int32)
        masses = np.array([12.0, 16.0])
        L = 32.0
    else:
        # 512 atoms at the dense configurations' density: no cell grid, lists from every atom
        L = (512 / 0.1) ** (1.0 / 3.0)
        pos = W.jitter(W.simple_cubic(8, L / 8), L / 8, seed=13)
        sp = (np.arange(512) % 2).astype(np.int32)
        masses = np.array([12.0, 16.0])
    s = W.System(positions=pos, momenta=W.mb_momenta(masses[sp], 300.0, 17), species=sp, masses=masses,
                 box=np.array([L] * 3), seed=23)
    lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=5.0)
    target = W.Potential(**lj, n_rbf=8, n_ang=0, n_layers=1, width=32, desc_cutoff=4.0, head="tanh",
                         head_scale=0.5, weights=W.mlp_weights(W.input_dim(2, 8, 0), 1, 32, 29))
    draft = W.learned_draft(W.Potential(**lj, desc_cutoff=4.0), 2)
    draft = W.replace(draft, weights=W.mlp_weights(W.input_dim(2, 8, 0), 1, 32, seed=3))
    return s, draft, target


@pytest.mark.parametrize("kind", ["cells", "all_atoms"])
def test_large_frame_force_matching_matches_oracle(kind):
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, target = _system(kind)
    h = lsd.LSD(s, draft, target, W.Integrator(1.0, 0.01, 300.0, 8))
    rng = np.random.default_rng(77)
    fq = np.stack([s.positions + 0.1 * rng.standard_normal(s.positions.shape) for _ in range(4)])
    fF = np.stack([O.forces(s, target, q) for q in fq]).astype(np.float32)
    loss, g = h.force_match(torch.tensor(fq, device="cuda"), torch.tensor(fF, device="cuda"))
    rl, rg = O.force_match(s, draft, fq, fF.astype(np.float64))
    assert abs(loss - rl) / rl < 1e-4, (loss, rl)
    assert rel(g.cpu().numpy(), rg) < 1e-4, rel(g.cpu().numpy(), rg)
    h.close()


def test_online_retraining_during_lsd_step():
    """Every 150 accepted steps lsd_step retrains the draft on the captured frames (512 atoms: the large-frame path);
    the run commits exactly the requested steps, retrains once per 150 accepted steps, and the retrained draft's mean
    |delta| per step (Eq. 6) falls below the starting draft's."""
    from paper_2606_02455_b300 import lsd
    s, draft, target = _system("cells")
    draft = W.learned_draft(W.Potential(lj_eps=draft.lj_eps, lj_sigma=draft.lj_sigma, lj_cutoff=5.0,
                                        desc_cutoff=4.0), 2)
    h = lsd.LSD(s, draft, target, W.Integrator(1.0, 0.01, 300.0, 8))
    h.set_frame_capture(512)
    st0 = h.step(200)
    before = st0["sum_delta"] / st0["committed"]
    h.set_online_training(150, n_iters=60, lr=3e-3, frames_per_iter=16)
    st1 = h.step(600)
    n, loss = h.online_status()
    assert st1["committed"] - st0["committed"] == 600
    accepted = (st1["committed"] - st0["committed"]) - (st1["rejected"] - st0["rejected"])
    # one retraining per 150 accepted steps, taken at the first batch boundary after each crossing
    assert n >= 2 and accepted // 150 - 1 <= n <= accepted // 150, (n, accepted)
    st2 = h.step(200)
    after = (st2["sum_delta"] - st1["sum_delta"]) / (st2["committed"] - st1["committed"])
    assert after < 0.8 * before, (before, after)
    h.close()
