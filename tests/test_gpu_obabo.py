"""GPU parity of OBABO through the staggered frame (App. E) against the oracle.

The GPU enters the frame with its own FP32 target forces and FP32 Box-Muller noise, so its staggered state differs
from the oracle's by the same per-step bounds as the ABOBA draft (sigma 1e-6 of the noise, 1e-5 of the force);
decisions, committed counts and step indices are identical; states agree within those bounds."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
TIE = 1e-6


def _wl(cfg):
    w = W.CONFIGS[cfg]()
    return W.replace(w, integ=W.replace(w.integ, scheme="obabo"))


def _tols(w, n):
    """(momentum bound after n staggered steps, dt/m): each step adds the FP32 noise (<= 1e-6 sigma) and FP32
    force (<= 1e-5 |F|) errors of the B kicks, plus the frame entry's half-step (sigma_1/2, (dt/2) kappa F)."""
    c1, aF, hm, sg = O.coefficients(w.system, w.integ)
    fmax = np.abs(O.forces(w.system, w.target, w.system.positions)).max() + \
        np.abs(O.forces(w.system, w.draft, w.system.positions)).max()
    per = sg.max() * 1e-6 + aF * 1e-5 * 10 * fmax
    return (n + 1) * per, 2 * hm.max()


@pytest.mark.parametrize("cfg", [1, 2])
def test_obabo_window_matches_oracle(cfg):
    from paper_2606_02455_b300 import lsd
    w = _wl(cfg)
    s = w.system
    target = W.replace(w.target, head_scale=1.5)
    h = lsd.LSD(s, w.draft, target, w.integ)
    h.draft_window()
    nc, first = h.verify_window()
    win = h.get_window()
    pbar = O.obabo_enter(s, target, w.integ, s.seed, 0, s.positions, s.momenta)
    ref = O.lsd_window(s, w.draft, target, w.integ, s.seed, 0, w.integ.K, s.positions, pbar)
    K = w.integ.K
    for j in range(K):
        ptol, hmf = _tols(w, j + 1)
        assert np.abs(win["p_draft"][j] - ref["pdraft"][j]).max() < ptol, ("p_draft", j)
        assert np.abs(win["q_mid"][j] - ref["qmid"][j]).max() < (j + 1) * hmf * ptol + 1e-12, ("q_mid", j)
        assert np.abs(win["F_target"][j] - ref["Ftarget"][j]).max() <= FORCE_TOL * 10 * np.abs(ref["Ftarget"][j]).max()
    margin = np.abs(ref["logu"] - np.minimum(ref["logr"], 0.0))
    assert not (margin < TIE).any()
    assert np.array_equal(win["accept"], ref["accept"])
    assert nc == ref["n_committed"]
    assert first == (-1 if ref["accept"].all() else int(np.argmin(ref["accept"])) + 1)
    q, p, step = h.get_state()                     # OBABO output state
    assert step == nc
    ptol, hmf = _tols(w, nc)
    sgh = np.sqrt(O.coefficients(s, w.integ)[3].max() ** 2)   # sigma bounds sigma_1/2
    ptol += 1e-4 * sgh
    assert np.abs(q - ref["q"]).max() < (nc + 1) * hmf * ptol + 1e-12
    assert np.abs(p - ref["p_obabo"]).max() < 2 * ptol
    h.close()


def test_obabo_free_running_and_plain_match_oracle():
    from paper_2606_02455_b300 import lsd
    w = _wl(1)
    s = w.system
    target = W.replace(w.target, head_scale=1.0)
    h = lsd.LSD(s, w.draft, target, w.integ)
    st = h.step(20)
    q, p, step = h.get_state()
    pbar = O.obabo_enter(s, target, w.integ, s.seed, 0, s.positions, s.momenta)
    ref = O.lsd_run(s, w.draft, target, w.integ, s.seed, 20, w.integ.K, s.positions, pbar)
    assert step == 20 == st["committed"]
    assert st["rejected"] == ref["stats"]["rejected"]
    ptol, hmf = _tols(w, 20)
    ptol = 10 * ptol + 1e-4 * O.coefficients(s, w.integ)[3].max() * (ref["stats"]["rejected"] + 1)
    assert np.abs(p - ref["p_obabo"]).max() < ptol
    assert np.abs(q - ref["q"]).max() < 40 * hmf * ptol
    # plain target OBABO from the same OBABO state
    h.set_state(s.positions, s.momenta, 0)
    h.plain_step(20)
    q, p, step = h.get_state()
    refp = O.plain_run(s, target, w.integ, s.seed, 20, s.positions, pbar)
    assert step == 20
    assert np.abs(p - refp["p_obabo"]).max() < ptol
    assert np.abs(q - refp["q"]).max() < 400 * hmf * ptol
    h.close()


def test_obabo_checkpoint_resume_is_bitwise():
    from paper_2606_02455_b300 import lsd
    w = _wl(1)
    s = w.system
    target = W.replace(w.target, head_scale=1.0)
    a = lsd.LSD(s, w.draft, target, w.integ)
    a.step(40)
    qa, pa, _ = a.get_state()
    b = lsd.LSD(s, w.draft, target, w.integ)
    b.step(16)
    blob = b.checkpoint()
    b.close()
    c = lsd.LSD(s, w.draft, target, W.replace(w.integ, scheme="aboba"))
    c.restore(blob)                                 # the checkpoint carries the integrator
    c.step(24)
    qc, pc, stc = c.get_state()
    assert stc == 40 and np.array_equal(qa, qc) and np.array_equal(pa, pc)
    a.close()
    c.close()


def test_integrator_switch_round_trip():
    """Switching to OBABO takes the current state as the OBABO state; switching back returns it unchanged."""
    from paper_2606_02455_b300 import lsd
    w = W.config1()
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    h.step(8)
    q0, p0, s0 = h.get_state()
    h.set_integrator("obabo")
    q1, p1, s1 = h.get_state()
    assert s1 == s0 and np.array_equal(q1, q0) and np.array_equal(p1, p0)
    h.step(8)
    q2, p2, s2 = h.get_state()
    assert s2 == s0 + 8 and not np.array_equal(q2, q0)
    h.set_integrator("aboba")
    q3, p3, _ = h.get_state()
    assert np.array_equal(q3, q2) and np.array_equal(p3, p2)
    h.close()
