"""Verlet lists kept across windows (lsd_set_list_reuse): rebuilt only when the committed state has moved more than
half the draft's displacement bound from the lists' base, or when the last draft stopped at the bound.  Kept lists
are complete for every drafted step (the draft checks each step against the same base), so a window drafted on kept
lists matches the oracle like one drafted on fresh lists; staged and one-pass windows make the same rebuild
decisions, so they still agree bit for bit."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _handle(w, reuse=True, stages=0, d_max=0.0):
    from paper_2606_02455_b300 import lsd
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    if d_max:
        h.set_max_displacement(d_max)
    h.set_list_reuse(reuse)
    h.set_window_stages(stages)
    return h


def test_window_on_kept_lists_matches_oracle():
    """Lists built around the seeded state q0 (one window), then a window from q1 = q0 + 0.02 A seeded noise: the
    lists are kept (no second build) and the first step's draft and target forces at sampled atoms match the
    oracle's at q1's half-step positions.  K = 8: the first window's draft stays inside the displacement bound."""
    w = W.config4(8)
    s = w.system
    h = _handle(w)
    q0, p0 = s.positions.copy(), s.momenta.copy()
    h.set_state(q0, p0, 0)
    h.draft_window()
    h.verify_window()
    assert h.stats()["list_builds"] == 1
    q1 = q0 + 0.02 * np.random.default_rng(11).standard_normal(q0.shape)
    h.set_state(q1, p0, 0)
    h.draft_window()
    nc, _ = h.verify_window()
    win = h.get_window()
    st = h.stats()
    h.close()
    assert st["list_builds"] == 1 and 1 <= nc <= w.integ.K
    c1, aF, hm, sg = O.coefficients(s, w.integ)
    qm = q1 + p0 * hm[s.species][:, None]
    assert np.array_equal(win["q_mid"][0], qm)
    sel = np.sort(np.random.default_rng(12).choice(s.n_atoms, 24, replace=False))
    refd = O.forces_subset(s, w.draft, qm, sel)
    assert _rel(win["F_draft"][0][sel], refd) < 1e-5, _rel(win["F_draft"][0][sel], refd)
    reft = O.forces_subset(s, w.target, qm, sel)
    assert _rel(win["F_target"][0][sel], reft) < 2e-2


def test_kept_lists_staged_equals_one_pass():
    """Config 4 with kept lists: staged (8 steps) and one-pass windows commit the same trajectory and rebuild the
    lists at the same windows; the lists are rebuilt far less often than once per window."""
    w = W.config4()
    out = []
    for S in (0, 8):
        h = _handle(w, stages=S)
        st = h.step(32 * 4 + 9)
        q, p, step = h.get_state()
        out.append((q, p, step, st))
        h.close()
    (qa, pa, sa, sta), (qb, pb, sb, stb) = out
    assert sa == sb == 32 * 4 + 9
    for k in ("windows", "committed", "rejected", "sum_delta", "list_builds"):
        assert sta[k] == stb[k], k
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    assert 1 <= sta["list_builds"] < sta["windows"]


def test_displacement_stop_forces_a_rebuild():
    """With a 0.05 A displacement bound most windows' drafts stop at the bound before any rejection, and each such
    window has the next one rebuild the lists (a window that commits nothing included: the run still advances)."""
    w = W.config4()
    h = _handle(w, d_max=0.05)
    st = h.step(64)
    h.close()
    assert st["committed"] == 64 and st["windows"] > 64 // w.integ.K + 1
    assert st["list_builds"] > st["windows"] // 2


def test_list_reuse_off_by_default_and_exclusive_with_pipelining():
    from paper_2606_02455_b300 import lsd
    w = W.config4()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    st = h.step(40)
    assert st["list_builds"] == 0
    lc = h.launch_counts()["window"]
    h.set_list_reuse(True)
    assert h.launch_counts()["window"] == lc + 1   # the check kernel
    with pytest.raises(lsd.LSDError):
        h.set_pipelining(True)
    h.set_list_reuse(False)
    h.set_pipelining(True)
    with pytest.raises(lsd.LSDError):
        h.set_list_reuse(True)
    h.close()


def test_plain_steps_keep_lists_and_their_trajectory():
    """Plain target steps keep their Verlet lists while the half-step positions stay within the displacement bound
    of the lists' base.  A 1e-4 A bound rebuilds them every step; the trajectory is bit for bit the same (the
    neighbour keys are canonical, so the forces do not depend on which complete lists hold them), with far fewer
    builds under the default bound."""
    from paper_2606_02455_b300 import lsd
    w = W.config4()
    out = []
    for d_max in (0.0, 1e-4):
        h = lsd.LSD(w.system, w.draft, w.target, w.integ)
        if d_max:
            h.set_max_displacement(d_max)
        h.plain_step(60)
        q, p, step = h.get_state()
        out.append((q, p, step, h.stats()["list_builds"]))
        h.close()
    (qa, pa, sa, ba), (qb, pb, sb, bb) = out
    assert sa == sb == 60
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    assert bb == 60 and 1 <= ba < 20


def test_list_skin_can_shrink_only():
    """A smaller Verlet skin (the lists' capacity and cells stay those of the planned one): the run still commits
    every requested step with kept lists; a larger skin than planned is refused."""
    from paper_2606_02455_b300 import lsd
    w = W.config4()
    h = _handle(w, stages=8)
    skin0 = h.list_skin()
    assert skin0 >= 1.0
    with pytest.raises(lsd.LSDError):
        h.set_list_skin(skin0 + 0.5)
    h.set_list_skin(0.8)
    assert h.list_skin() == 0.8
    st = h.step(120)
    h.close()
    assert st["committed"] == 120 and st["list_builds"] >= 1
