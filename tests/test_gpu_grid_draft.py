"""The grid form of the draft (lsd_set_grid_draft: one cooperative launch of one CTA per SM with a bounded grid-wide
barrier per step) against the cluster form (one thread-block cluster of at most 16 CTAs): both compute every atom's
draft force in the same order, so windows, committed trajectories and early window ends agree bit for bit."""
import numpy as np
import pytest

from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _handle(w, draft, grid, d_max=0.0):
    from paper_2606_02455_b300 import lsd
    h = lsd.LSD(w.system, draft, w.target, w.integ)
    h.set_grid_draft(grid)
    if d_max:
        h.set_max_displacement(d_max)
    return h


def _run_both(w, draft, n, d_max=0.0):
    out = []
    for grid in (True, False):
        h = _handle(w, draft, grid, d_max)
        st = h.step(n)
        q, p, step = h.get_state()
        out.append((q, p, step, st))
        h.close()
    return out


@pytest.mark.parametrize("learned", [False, True])
def test_grid_draft_equals_cluster_draft_config4(learned):
    """4,096 atoms, K = 32: 96 committed steps from the seeded state with each form, the pair draft and the learned
    draft (LJ + MLP on radial basis functions, two grid barriers per step)."""
    w = W.config4()
    draft = W.learned_draft(w.target, w.system.n_species) if learned else w.draft
    (qa, pa, sa, sta), (qb, pb, sb, stb) = _run_both(w, draft, 96)
    assert sa == sb == 96
    assert sta["rejected"] == stb["rejected"] and sta["windows"] == stb["windows"]
    assert sta["sum_delta"] == stb["sum_delta"]
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)


def test_grid_draft_window_arrays_equal_cluster_config5():
    """32,768 atoms, K = 64: one drafted window's half-step positions, momenta and draft forces, bit for bit."""
    w = W.config5()
    wins = []
    for grid in (True, False):
        h = _handle(w, w.draft, grid)
        h.draft_window()
        wins.append(h.get_window())
        h.close()
    a, b = wins
    for key in ("q_mid", "p_draft", "F_draft"):
        assert np.array_equal(a[key], b[key]), key


def test_grid_draft_ends_windows_early_like_the_cluster():
    """With a displacement bound of 0.05 A every window ends early (k_eff < K, the grid-wide flag of the earliest
    step at which an atom left the bound); both forms end at the same steps and commit the same trajectory."""
    w = W.config4()
    res = []
    for grid in (True, False):
        h = _handle(w, w.draft, grid, d_max=0.05)
        h.draft_window()
        nc, _ = h.verify_window()
        win = h.get_window()
        st = h.step(64)
        q, p, step = h.get_state()
        res.append((nc, win, st, q, p, step))
        h.close()
    (nca, wa, sta, qa, pa, stpa), (ncb, wb, stb, qb, pb, stpb) = res
    assert nca == ncb and 1 <= nca < w.integ.K
    assert sta["windows"] == stb["windows"] and sta["windows"] > 64 // w.integ.K + 1
    assert np.array_equal(wa["q_mid"][:nca], wb["q_mid"][:nca])
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb) and stpa == stpb


def test_grid_draft_pipelined_equals_cluster_unpipelined():
    """The pipelined loop (speculative drafts in the cluster form, redrafts in the grid form) commits the
    trajectory of the unpipelined loop with cluster drafts only."""
    from paper_2606_02455_b300 import lsd
    w = W.config4()
    target = w.target
    a = lsd.LSD(w.system, w.draft, target, w.integ)
    a.set_grid_draft(False)
    b = lsd.LSD(w.system, w.draft, target, w.integ)
    b.set_pipelining(True)
    sta, stb = a.step(96), b.step(96)
    qa, pa, _ = a.get_state()
    qb, pb, _ = b.get_state()
    assert sta["rejected"] == stb["rejected"] and sta["rejected"] > 0
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    a.close()
    b.close()


def test_grid_draft_unavailable_for_small_systems():
    from paper_2606_02455_b300 import lsd
    w = W.config2()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    with pytest.raises(lsd.LSDError):
        h.set_grid_draft(True)
    h.set_grid_draft(False)
    h.close()
