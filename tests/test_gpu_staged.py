"""Windows verified in stages (lsd_set_window_stages): stage s drafts and verifies steps sS .. sS + S - 1 and the
next stage runs (a conditional node of the window's graph) only while every step so far was accepted.  The window
then commits what a one-pass window commits (Alg. 1: the first rejection and the steps before it), so trajectories
and statistics agree bit for bit with one-pass windows, while the steps past the first rejection's stage are never
drafted or verified."""
import numpy as np
import pytest

from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu

SAME = ("windows", "committed", "rejected", "sum_delta", "pred_rejected", "step")


def _handle(w, target=None, draft=None, stages=0, d_max=0.0, integrator=None, ec=False):
    from paper_2606_02455_b300 import lsd
    h = lsd.LSD(w.system, draft or w.draft, target or w.target, w.integ)
    if integrator:
        h.set_integrator(integrator)
    if ec:
        h.set_error_correction(True)
    if d_max:
        h.set_max_displacement(d_max)
    h.set_window_stages(stages)
    return h


def _run(w, n, stages, **kw):
    h = _handle(w, stages=stages, **kw)
    st = h.step(n)
    q, p, step = h.get_state()
    h.close()
    return q, p, step, st


def _check_same(a, b, n_stages):
    qa, pa, sa, sta = a
    qb, pb, sb, stb = b
    assert sa == sb
    for k in SAME:
        assert sta[k] == stb[k], (k, sta[k], stb[k])
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    # one pass: one verification per window; staged: between one and n_stages per window, never more steps
    assert sta["stages"] == sta["windows"]
    assert stb["windows"] <= stb["stages"] <= n_stages * stb["windows"]
    assert stb["verified"] <= sta["verified"]


CASES = {
    # name: (workload, target head scale (rejections), steps per stage, steps run)
    "c1_S3": (W.config1, 1.0, 3, 8 * 9 + 5),      # K = 8: stages of 3, 3 and 2 steps; the cap inside a window
    "c2_S4": (W.config2, 1.5, 4, 16 * 5 + 7),     # 256 atoms, K = 16, rejections in most windows
    "c2_S5": (W.config2, 1.5, 5, 16 * 4 + 3),     # stages of 5, 5, 5 and 1 steps
    "c4_S8": (W.config4, 1.0, 8, 32 * 3 + 11),    # 4,096 atoms, K = 32: moments, the grid draft
}


@pytest.mark.parametrize("name", list(CASES))
def test_staged_windows_commit_what_one_pass_commits(name):
    make, head, S, n = CASES[name]
    w = make()
    target = W.replace(w.target, head_scale=head) if head != 1.0 else w.target
    K = w.integ.K
    one = _run(w, n, 0, target=target)
    staged = _run(w, n, S, target=target)
    _check_same(one, staged, -(-K // S))
    assert one[3]["rejected"] > 0 or name in ("c1_S3", "c4_S8")


def test_staged_windows_with_early_ends():
    """A displacement bound of 0.05 A ends every window early (k_eff < K), inside some stage: the draft's flag and
    the stage decision agree with the one-pass window."""
    w = W.config4()
    one = _run(w, 80, 0, d_max=0.05)
    staged = _run(w, 80, 8, d_max=0.05)
    _check_same(one, staged, 4)
    assert one[3]["windows"] > 80 // w.integ.K + 1


def test_staged_windows_obabo_and_error_correction():
    w = W.config2()
    target = W.replace(w.target, head_scale=1.5)
    for kw in (dict(integrator="obabo"), dict(ec=True)):
        one = _run(w, 16 * 4 + 1, 0, target=target, **kw)
        staged = _run(w, 16 * 4 + 1, 4, target=target, **kw)
        _check_same(one, staged, 4)


def test_staged_frames_are_the_verified_prefix_of_each_window():
    """Frame capture: each staged window captures the first `verified` steps of the frames the one-pass window
    captures (the same half-step positions and target forces)."""
    w = W.config2()
    target = W.replace(w.target, head_scale=1.5)
    frames, counts = {}, {}
    for S in (0, 4):
        h = _handle(w, target=target, stages=S)
        h.set_frame_capture(16 * 8)
        per = []
        for _ in range(5):
            v0 = h.stats()["verified"]
            h.enqueue_windows(1)
            per.append(h.stats()["verified"] - v0)
        n = h.frame_count()
        frames[S] = h.get_frames(0, n)
        counts[S] = per
        h.close()
    assert sum(counts[0]) == frames[0][0].shape[0] and sum(counts[4]) == frames[4][0].shape[0]
    assert sum(counts[4]) < sum(counts[0])
    o0 = o4 = 0
    for a, b in zip(counts[0], counts[4]):
        assert b <= a and b % 4 == 0
        for t in range(2):
            assert np.array_equal(frames[0][t][o0:o0 + b], frames[4][t][o4:o4 + b])
        o0 += a
        o4 += b


def test_staged_window_host_and_launch_counts():
    from paper_2606_02455_b300 import lsd
    w = W.config2()
    target = W.replace(w.target, head_scale=1.5)
    res = []
    for S in (0, 4):
        h = _handle(w, target=target, stages=S)
        lc, sc = h.launch_counts(), h.stage_launch_counts()
        if S == 0:
            assert sc == dict(first=lc["window"], later=0)
        else:
            assert sc["first"] == lc["window"] and 0 < sc["later"] <= sc["first"]   # later stages rebuild no lists
        q = np.ascontiguousarray(w.system.positions, dtype=np.float64)
        p = np.ascontiguousarray(w.system.momenta, dtype=np.float64)
        qo, po = np.empty_like(q), np.empty_like(p)
        step, nc = h.window_host(q, p, 0, qo, po)
        res.append((step, nc, qo, po))
        h.close()
    (sa, na, qa, pa), (sb, nb, qb, pb) = res
    assert sa == sb and na == nb and np.array_equal(qa, qb) and np.array_equal(pa, pb)


def test_stages_and_pipelining_are_exclusive():
    from paper_2606_02455_b300 import lsd
    w = W.config2()
    h = _handle(w, stages=4)
    with pytest.raises(lsd.LSDError):
        h.set_pipelining(True)
    h.set_window_stages(0)
    h.set_pipelining(True)
    with pytest.raises(lsd.LSDError):
        h.set_window_stages(4)
    h.set_window_stages(16)   # S >= K: one pass, allowed
    h.close()


def test_profile_window_follows_the_stage_length():
    """lsd_profile_window of a staged handle profiles one stage-length window: at most S steps verified, every
    phase timed, the Verlet lists as their own phase."""
    from paper_2606_02455_b300 import lsd
    w = W.config4()
    h = _handle(w, stages=8)
    a = h.stats()
    ph = h.profile_window()
    b = h.stats()
    h.close()
    assert tuple(ph) == lsd.LSD.PHASES and all(v >= 0.0 for v in ph.values()) and ph["verlet_lists"] > 0.0
    assert b["windows"] - a["windows"] == 1 and 1 <= b["verified"] - a["verified"] <= 8
