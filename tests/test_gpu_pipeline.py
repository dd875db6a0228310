"""The pipelined window loop (lsd_set_pipelining: the draft of window w+1 overlaps the verification of window w,
speculatively from w's last drafted state, and is drafted again when w had a rejection) commits exactly the
trajectory of the unpipelined loop: same steps, same bits."""
import numpy as np
import pytest

from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(w, target, n, pipelined, **kw):
    from paper_2606_02455_b300 import lsd
    h = lsd.LSD(w.system, w.draft, target, w.integ)
    if pipelined:
        h.set_pipelining(True)
    st = h.step(n)
    q, p, step = h.get_state()
    h.close()
    return q, p, step, st


@pytest.mark.parametrize("cfg,scale,n", [(1, 1.0, 96), (2, 1.5, 80), (4, None, 96)])
def test_pipelined_equals_unpipelined_bitwise(cfg, scale, n):
    w = W.CONFIGS[cfg]()
    target = w.target if scale is None else W.replace(w.target, head_scale=scale)
    qa, pa, sa, sta = _run(w, target, n, False)
    qb, pb, sb, stb = _run(w, target, n, True)
    assert sa == sb == n
    assert sta["rejected"] == stb["rejected"] and sta["rejected"] > 0
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)


def test_pipelined_equals_unpipelined_bitwise_cell_grid_lists():
    """The same on a box with a cell grid: each window's Verlet lists come from their own kernels (the redraft
    rebuilds them only when the speculative draft does not stand) and are staged in the draft's shared memory."""
    from test_gpu_parity import _dilute_lists
    w = _dilute_lists()
    target = W.replace(w.target, head_scale=1.5)
    qa, pa, sa, sta = _run(w, target, 64, False)
    qb, pb, sb, stb = _run(w, target, 64, True)
    assert sa == sb == 64
    assert sta["rejected"] == stb["rejected"] and sta["rejected"] > 0
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)


def test_pipelined_obabo_equals_unpipelined():
    w = W.config1()
    w = W.replace(w, integ=W.replace(w.integ, scheme="obabo"))
    target = W.replace(w.target, head_scale=1.0)
    qa, pa, sa, sta = _run(w, target, 64, False)
    qb, pb, sb, stb = _run(w, target, 64, True)
    assert sa == sb == 64 and sta["rejected"] == stb["rejected"]
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)


def test_pipelined_survives_state_changes_between_runs():
    """set_state and plain steps between pipelined runs: each run starts from the state it is given."""
    from paper_2606_02455_b300 import lsd
    w = W.config1()
    target = W.replace(w.target, head_scale=1.0)
    s = w.system
    a = lsd.LSD(s, w.draft, target, w.integ)
    b = lsd.LSD(s, w.draft, target, w.integ)
    b.set_pipelining(True)
    for h in (a, b):
        h.step(24)
        h.plain_step(5)
        h.step(16)
        h.set_state(s.positions, s.momenta, 3)
        h.step(24)
    qa, pa, sa = a.get_state()
    qb, pb, sb = b.get_state()
    assert sa == sb == 27 and np.array_equal(qa, qb) and np.array_equal(pa, pb)
    a.close()
    b.close()


def test_pipelining_excludes_error_correction():
    from paper_2606_02455_b300 import lsd
    w = W.config1()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    h.set_error_correction(True)
    with pytest.raises(lsd.LSDError):
        h.set_pipelining(True)
    h.set_error_correction(False)
    h.set_pipelining(True)
    with pytest.raises(lsd.LSDError):
        h.set_error_correction(True)
    h.close()


def test_launch_counts_follow_the_configuration():
    """The kernels a window, a pipelined round and a plain step launch: all-pairs candidates and a one-launch
    transport for the 256-atom workload, whose plain steps run in the fused kernel (0 per step: one launch per call;
    7 per step on the graph path); Verlet-list builds (four kernels on a grid of cells) and a two-launch transport
    for 4096 atoms, whose plain steps also launch the kept-list check (the list kernels return at once while the
    lists stay valid)."""
    from paper_2606_02455_b300 import lsd
    w = W.config2()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    assert h.launch_counts() == dict(window=7, round=9, plain=0)
    h.set_plain_fused(False)
    assert h.launch_counts() == dict(window=7, round=9, plain=7)
    h.close()
    w = W.config4()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    assert h.launch_counts() == dict(window=12, round=19, plain=12)
    h.close()


@pytest.mark.parametrize("joint", [True, False])
def test_window_host_equals_the_per_window_calls(joint):
    """lsd_window_host (state in, one window, state out, one synchronisation) commits bit for bit what
    lsd_set_state + lsd_draft_window + lsd_verify_window + lsd_get_state commit, over windows with and without
    rejections, with the output buffers aliasing the inputs; positions and momenta in one pinned buffer (one copy
    each way) or in two."""
    import torch
    from paper_2606_02455_b300 import lsd
    w = W.config2()
    s = w.system
    a = lsd.LSD(s, w.draft, w.target, w.integ)
    b = lsd.LSD(s, w.draft, w.target, w.integ)
    if joint:
        buf = torch.empty((2, s.n_atoms, 3), dtype=torch.float64, pin_memory=True).numpy()
        pos, mom = buf[0], buf[1]
    else:
        pos = torch.empty((s.n_atoms, 3), dtype=torch.float64, pin_memory=True).numpy()
        mom = torch.empty((s.n_atoms, 3), dtype=torch.float64, pin_memory=True).numpy()
    pos[:] = s.positions
    mom[:] = s.momenta
    q, p, step = s.positions.copy(), s.momenta.copy(), 0
    rejected = 0
    for _ in range(12):
        b.set_state(q, p, step)
        b.draft_window()
        nc_b, first = b.verify_window()
        q, p, step_b = b.get_state()
        step_a, nc_a = a.window_host(pos, mom, step)
        assert (step_a, nc_a) == (step_b, nc_b)
        assert np.array_equal(pos, q) and np.array_equal(mom, p)
        rejected += first != -1
        step = step_b
    assert rejected > 0
    a.close()
    b.close()
