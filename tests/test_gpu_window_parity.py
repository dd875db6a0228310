"""GPU parity of the transport, frames, early window ends and the pipelined loop against the FP64 oracle.

Every input is the oracle's (or the seeded workload's); nothing the GPU produced is fed to the oracle.

* The transport on its own (Eq. 5; Alg. 1's commit), through lsd_transport_window: the oracle drafts a window
  and evaluates both potentials in FP64; both sides then take the same FP32-rounded forces.  delta.delta is then
  an FP64 sum of identical FP64 terms on both sides (bar: 1e-11 relative; an FP32 sum would miss it by ~1e-6).
  log r differs only through the noise z = xi: the GPU's FP32 Box-Muller is within 1e-6 of the exact normal per
  component, so |dlog r| <= 1e-6 sum_c |delta_c| (+ FP64 rounding).  Decisions are compared outside that band and
  no decision may fall inside it at the test seeds.
* Frames (a12): the captured (q_mid_j, F_j) equal the window's own arrays bit for bit, in capture order, through a
  ring buffer that wraps.
* Early window end (reading 15): a displacement bound small enough to stop most windows after a few steps; noise
  keyed by the step index makes the committed trajectory independent of where windows end, so it is compared with
  the oracle's lsd_run.
* The pipelined loop (the bench's loop) against the oracle's lsd_run directly, over several windows with
  rejections.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W
from parity_bounds import XI_ERR, state_tols

pytestmark = pytest.mark.gpu


def _lsd():
    from paper_2606_02455_b300 import lsd
    return lsd


def _small_ragged():
    pos = W.jitter(W.simple_cubic(3, 3.1), 3.1, seed=5)
    sp = np.arange(27) % 2
    s = W.System(positions=pos, momenta=W.mb_momenta(np.array([12.0, 16.0])[sp], 300.0, 7), species=sp.astype(np.int32),
                 masses=np.array([12.0, 16.0]), box=np.array([9.3] * 3), seed=99)
    lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=4.6)
    d0 = W.input_dim(2, 16, 16)
    target = W.Potential(**lj, n_rbf=16, n_ang=16, n_layers=2, width=64, desc_cutoff=4.0, head="tanh",
                         head_scale=0.3, weights=W.mlp_weights(d0, 2, 64, 11))
    return W.Workload("ragged27", s, W.Potential(**lj), target, W.Integrator(1.0, 0.01, 300.0, 8), 100)


WORKLOADS = {"c1": lambda: W.config1(), "c2": lambda: W.config2(), "ragged27": _small_ragged}


def _given_window(w, target, n0, q0, p0):
    """The oracle's window (its own FP64 draft and forces) and, from it, the window handed to both transports:
    forces rounded to FP32, draft means and momenta rebuilt from them with the oracle's noise, and the oracle's
    reflectionVerify of every step."""
    s, K = w.system, w.integ.K
    ref = O.lsd_window(s, w.draft, target, w.integ, s.seed, n0, K, q0, p0)
    c1, aF, hm, sg = O.coefficients(s, w.integ)
    sig = np.repeat(sg[s.species][:, None], 3, axis=1)
    hma = np.repeat(hm[s.species][:, None], 3, axis=1)
    Fd = ref["Fdraft"].astype(np.float32)
    Ft = ref["Ftarget"].astype(np.float32)
    pdraft = np.zeros((K, s.n_atoms, 3))
    out = []
    pprev = p0
    for j in range(K):
        n = n0 + j + 1
        xi = np.stack([O.normals(s.seed, n, i, 0) for i in range(s.n_atoms)])
        mud = c1 * pprev + aF * Fd[j].astype(np.float64)
        mut = c1 * pprev + aF * Ft[j].astype(np.float64)
        pdraft[j] = mud + sig * xi
        acc, p_out, lr, zd, dd = O.transport_terms(sig.ravel(), O.uniform(s.seed, n), pdraft[j].ravel(), mud.ravel(),
                                                   mut.ravel())
        delta = (mud - mut) / sig
        out.append(dict(acc=acc, p=p_out.reshape(-1, 3), lr=lr, zd=zd, dd=dd, logu=np.log(O.uniform(s.seed, n)),
                        l1=np.abs(delta).sum(), dmax=np.abs(delta).max()))
        pprev = pdraft[j]
    return ref, Fd, Ft, pdraft, out, sig, hma


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("head_scale", [None, 1.5])
def test_transport_matches_oracle_on_the_same_window(name, head_scale):
    lsd = _lsd()
    w = WORKLOADS[name]()
    s, K = w.system, w.integ.K
    target = w.target if head_scale is None else W.replace(w.target, head_scale=head_scale)
    ref, Fd, Ft, pdraft, out, sig, hma = _given_window(w, target, 0, s.positions, s.momenta)
    h = lsd.LSD(s, w.draft, target, w.integ)
    nc, first = h.transport_window(ref["qmid"], pdraft, Fd, Ft)
    win = h.get_window()
    tol = np.array([XI_ERR * o["l1"] + 1e-12 * (1.0 + abs(o["lr"])) for o in out])
    lr_o = np.array([o["lr"] for o in out])
    margin = np.abs(np.array([o["logu"] for o in out]) - np.minimum(lr_o, 0.0))
    assert (margin > tol).all(), "a decision within the log-ratio bound at the test seed: %s" % np.nonzero(margin <= tol)
    assert np.array_equal(win["accept"], np.array([o["acc"] for o in out]))
    assert (np.abs(win["log_ratio"] - lr_o) <= tol).all(), np.abs(win["log_ratio"] - lr_o) / tol
    dd = np.array([o["dd"] for o in out])
    assert np.allclose(win["delta_norm"] ** 2, dd, rtol=1e-11, atol=1e-300)
    assert np.allclose(win["log_u"], [o["logu"] for o in out], rtol=1e-15, atol=0)
    # committed prefix and the new state
    acc = np.array([o["acc"] for o in out])
    l_exp = K if acc.all() else int(np.argmin(acc)) + 1
    assert nc == l_exp and first == (-1 if acc.all() else l_exp)
    q, p, step = h.get_state()
    assert step == l_exp
    j = l_exp - 1
    if acc[j]:
        assert np.array_equal(p, pdraft[j])                    # the draft's own bits
        assert np.array_equal(q, ref["qmid"][j] + hma * pdraft[j])
    else:
        # the reflection: <p> + sigma (z - 2 (z.delta / delta.delta) delta), with z and z.delta off by the noise error
        o = out[j]
        ptol = sig.max() * (XI_ERR + 2.0 * tol[j] / o["dd"] * o["dmax"]) + 1e-14 * np.abs(o["p"]).max()
        assert np.abs(p - o["p"]).max() < ptol
        assert np.abs(q - (ref["qmid"][j] + hma * o["p"])).max() < hma.max() * ptol + 1e-13 * np.abs(q).max()
    h.close()


def test_transport_rejections_present_at_the_test_seed():
    """The head_scale 1.5 cases above exercise reflections: at least one rejected step in the config-2 window."""
    w = W.config2()
    target = W.replace(w.target, head_scale=1.5)
    _, _, _, _, out, _, _ = _given_window(w, target, 0, w.system.positions, w.system.momenta)
    assert not all(o["acc"] for o in out)


def test_frames_equal_the_window_arrays_bitwise():
    """Frame capture (the learned draft's training labels): each verified window step j appends (q_mid_j, F_j) in
    step order; the ring keeps the last `capacity` frames."""
    lsd = _lsd()
    w = W.config1()
    s, K = w.system, w.integ.K
    target = W.replace(w.target, head_scale=1.5)
    h = lsd.LSD(s, w.draft, target, w.integ)
    cap = 3 * K
    h.set_frame_capture(cap)
    wins = []
    for _ in range(4):
        h.draft_window()
        h.verify_window()
        wins.append(h.get_window())
    assert h.frame_count() == cap
    q, F = h.get_frames(K, 3 * K)
    for t in range(3):
        assert np.array_equal(q[t * K:(t + 1) * K], wins[t + 1]["q_mid"])
        assert np.array_equal(F[t * K:(t + 1) * K], wins[t + 1]["F_target"])
    with pytest.raises(lsd.LSDError):
        h.get_frames(K - 1, 1)            # overwritten by the fourth window
    with pytest.raises(lsd.LSDError):
        h.get_frames(3 * K, K + 1)        # not captured yet
    h.close()


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_windows_ending_early_match_the_oracle_run(name):
    """k_eff < K: with a 0.02 A displacement bound the draft ends most windows after a few steps; the committed
    trajectory is still the oracle's lsd_run (K-independent by the step-keyed noise).  The verification builds no
    neighbour list for the steps past k_eff (their positions are the previous window's, or were never written)."""
    lsd = _lsd()
    w = WORKLOADS[name]()
    s, K = w.system, w.integ.K
    target = W.replace(w.target, head_scale=1.0)
    h = lsd.LSD(s, w.draft, target, w.integ)
    h.set_max_displacement(0.02)
    n = 20
    st = h.step(n)
    q, p, step = h.get_state()
    assert step == n
    assert st["verified"] < st["windows"] * K, "no window ended early"
    ref = O.lsd_run(s, w.draft, target, w.integ, s.seed, n, K, s.positions, s.momenta)
    assert st["rejected"] == ref["stats"]["rejected"]
    ptol, qtol = state_tols(w, target, n, int(ref["stats"]["rejected"]))
    assert np.abs(p - ref["p"]).max() < ptol
    assert np.abs(q - ref["q"]).max() < qtol
    h.set_max_displacement(0.0)
    h.close()


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_pipelined_loop_matches_the_oracle_run(name):
    """The pipelined round (speculative draft of window w+1 during the verification of w, kept or redrafted on
    the device) against the oracle's lsd_run over several windows with rejections."""
    lsd = _lsd()
    w = WORKLOADS[name]()
    s, K = w.system, w.integ.K
    target = W.replace(w.target, head_scale=1.5)
    n = 3 * K if name == "c1" else K
    ref = O.lsd_run(s, w.draft, target, w.integ, s.seed, n, K, s.positions, s.momenta)
    assert ref["stats"]["rejected"] >= 2 and ref["stats"]["windows"] >= 4
    h = lsd.LSD(s, w.draft, target, w.integ)
    h.set_pipelining(True)
    st = h.step(n)
    q, p, step = h.get_state()
    assert step == n and st["committed"] == n
    assert st["rejected"] == ref["stats"]["rejected"] and st["windows"] == ref["stats"]["windows"]
    ptol, qtol = state_tols(w, target, n, int(ref["stats"]["rejected"]))
    assert np.abs(p - ref["p"]).max() < ptol
    assert np.abs(q - ref["q"]).max() < qtol
    h.close()
