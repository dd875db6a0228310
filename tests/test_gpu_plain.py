"""The fused plain-target step (one cooperative launch for every step of a call) against the FP64 oracle's plain ABOBA
run and against the multi-kernel graph path of the same library, on the small workloads it serves.  Both GPU paths
evaluate the FP32 target network (the fused kernel on the CUDA cores, the graph path on the tensor cores at FP32
accuracy); states agree with the oracle and with each other within the bounds of parity_bounds.state_tols."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W
from parity_bounds import state_tols

pytestmark = pytest.mark.gpu


def _ragged27():
    pos = W.jitter(W.simple_cubic(3, 3.1), 3.1, seed=5)
    sp = np.arange(27) % 2
    s = W.System(positions=pos, momenta=W.mb_momenta(np.array([12.0, 16.0])[sp], 300.0, 7), species=sp.astype(np.int32),
                 masses=np.array([12.0, 16.0]), box=np.array([9.3] * 3), seed=99)
    lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=4.6)
    target = W.Potential(**lj, n_rbf=16, n_ang=16, n_layers=2, width=64, desc_cutoff=4.0, head="tanh",
                         head_scale=0.3, weights=W.mlp_weights(W.input_dim(2, 16, 16), 2, 64, 11))
    return W.Workload("ragged27", s, W.Potential(**lj), target, W.Integrator(1.0, 0.01, 300.0, 8), 100)


WORKLOADS = {"c1": lambda: W.config1(), "c2": lambda: W.config2(), "ragged27": _ragged27,
             "c1_lj_target": lambda: W.replace(W.config1(), target=W.config1().draft)}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fused_plain_matches_oracle_and_graph_path(name):
    from paper_2606_02455_b300 import lsd
    w = WORKLOADS[name]()
    s = w.system
    target = W.replace(w.target, head_scale=1.0) if w.target.n_layers else w.target
    n = 20
    h = lsd.LSD(s, w.draft, target, w.integ)
    assert h.launch_counts()["plain"] == 0, "the fused plain step is not in use"
    h.plain_step(n)
    qf, pf, step = h.get_state()
    assert step == n
    h.set_plain_fused(False)
    assert h.launch_counts()["plain"] > 0
    h.set_state(s.positions, s.momenta, 0)
    h.plain_step(n)
    qg, pg, _ = h.get_state()
    h.close()
    ref = O.plain_run(s, target, w.integ, s.seed, n, s.positions, s.momenta)
    ptol, qtol = state_tols(w, target, n)
    assert np.abs(pf - ref["p"]).max() < ptol and np.abs(qf - ref["q"]).max() < qtol
    assert np.abs(pf - pg).max() < ptol and np.abs(qf - qg).max() < qtol


def test_fused_plain_runs_exactly_the_requested_steps_across_calls():
    """Steps split over several calls (and one enqueued call) give the same state as one call: the kernel reads the
    step and the stop step from device memory and the noise is keyed by the step index."""
    from paper_2606_02455_b300 import lsd
    w = W.config2()
    s = w.system
    a = lsd.LSD(s, w.draft, w.target, w.integ)
    a.plain_step(24)
    qa, pa, sa = a.get_state()
    b = lsd.LSD(s, w.draft, w.target, w.integ)
    for n in (5, 1, 10, 8):
        b.plain_step(n)
    qb, pb, sb = b.get_state()
    assert sa == sb == 24 and np.array_equal(qa, qb) and np.array_equal(pa, pb)
    a.close()
    b.close()


def test_large_system_keeps_the_graph_plain_step():
    from paper_2606_02455_b300 import lsd
    w = W.config4()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    assert h.launch_counts()["plain"] > 0
    with pytest.raises(lsd.LSDError):
        h.set_plain_fused(True)
    h.close()
