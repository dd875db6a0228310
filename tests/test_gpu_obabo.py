"""GPU parity of OBABO through the staggered frame (App. E) against the oracle.

The GPU enters the frame with its own FP32 target forces and FP32 Box-Muller noise, so its staggered state differs
from the oracle's by the same per-step bounds as the ABOBA draft (sigma 1e-6 of the noise, 1e-5 of the force);
decisions, committed counts and step indices are identical; states agree within those bounds."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W
from parity_bounds import FORCE_TOL, REFLECT_ERR, XI_ERR, elem, logr_tol

pytestmark = pytest.mark.gpu


def _wl(cfg):
    w = W.CONFIGS[cfg]()
    return W.replace(w, integ=W.replace(w.integ, scheme="obabo"))


def _tols(w, target, n, n_refl=0):
    """(momentum bound, position bound) after n staggered steps.  Each step adds the FP32 noise (XI_ERR sigma) and
    the FP32 force error (per element at most 1e-5 of max|F|, bounded with twice the starting max|F~| + max|F|) of
    its B kicks; the frame entry's half-step counts as one more step; a reflection adds REFLECT_ERR sigma.  Staggered
    positions advance by full steps, q_n = q_{n-1} + dt p_n/m, so their error is dt/m times the sum of the momentum
    errors of the steps so far."""
    c1, aF, hm, sg = O.coefficients(w.system, w.integ)
    fmax = np.abs(O.forces(w.system, target, w.system.positions)).max() + \
        np.abs(O.forces(w.system, w.draft, w.system.positions)).max()
    per = sg.max() * XI_ERR + aF * FORCE_TOL * 2.0 * fmax
    e_refl = REFLECT_ERR * sg.max()
    ptol = (n + 1) * per + n_refl * e_refl
    qtol = 2 * hm.max() * ((n + 1) * (n + 2) / 2 * per + n * n_refl * e_refl)
    return ptol, qtol + 1e-13 * np.abs(w.system.positions).max()


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
        ptol, qtol = _tols(w, target, j + 1)
        assert np.abs(win["p_draft"][j] - ref["pdraft"][j]).max() < ptol, ("p_draft", j)
        assert np.abs(win["q_mid"][j] - ref["qmid"][j]).max() < qtol, ("q_mid", j)
        assert elem(win["F_target"][j], ref["Ftarget"][j]) < FORCE_TOL, j
    tol = logr_tol(ref["logr"])
    assert (np.abs(win["log_ratio"] - ref["logr"]) <= tol).all()
    margin = np.abs(ref["logu"] - np.minimum(ref["logr"], 0.0))
    assert not (margin <= tol).any()
    assert np.array_equal(win["accept"], ref["accept"])
    assert nc == ref["n_committed"]
    assert first == (-1 if ref["accept"].all() else int(np.argmin(ref["accept"])) + 1)
    q, p, step = h.get_state()                     # OBABO output state
    assert step == nc
    # the recovered output momentum adds the conditional half-step draw: its FP32 noise and force errors once more
    ptol, qtol = _tols(w, target, nc, 0 if ref["accept"][:nc].all() else 1)
    assert np.abs(q - ref["q"]).max() < qtol
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
    ptol, qtol = _tols(w, target, 20, int(ref["stats"]["rejected"]))
    assert np.abs(p - ref["p_obabo"]).max() < 2 * ptol
    assert np.abs(q - ref["q"]).max() < qtol
    # plain target OBABO from the same OBABO state
    h.set_state(s.positions, s.momenta, 0)
    h.plain_step(20)
    q, p, step = h.get_state()
    refp = O.plain_run(s, target, w.integ, s.seed, 20, s.positions, pbar)
    assert step == 20
    ptol, qtol = _tols(w, target, 20)
    assert np.abs(p - refp["p_obabo"]).max() < 2 * ptol
    assert np.abs(q - refp["q"]).max() < qtol
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
