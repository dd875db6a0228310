"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (each per result against FP64, derived in tests/parity_bounds.py): neighbour lists and accept/reject
decisions identical; FP32 forces, descriptors and dE/dX within 1e-5 relative, as a norm ratio per configuration
and per element (relative to the configuration's largest |value|); BF16 paths within 2e-2.  The end-to-end log
ratio is within 1e-4 max(1, |log r|), and decisions are compared outside exactly that band (a decision inside it
would be a near-tie; none occurs at the test seeds).  States after a window or a free run are within the
momentum and position bounds of parity_bounds.state_tols."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W
from parity_bounds import BF16_TOL, FORCE_TOL, elem, logr_tol, rel as _rel, state_tols

pytestmark = pytest.mark.gpu

LOGR_DN = 1e-4   # |delta|: the FP32 force error relative to the force difference it is built from


def _lsd():
    from paper_2606_02455_b300 import lsd
    return lsd


def _configs(system, n, scale, seed):
    rng = np.random.default_rng(seed)
    return np.stack([system.positions + scale * rng.standard_normal(system.positions.shape) for _ in range(n)])


def _small_ragged():
    """27 atoms of two species (not a multiple of a warp), simple cubic 3^3 in a 9.3 A box."""
    pos = W.jitter(W.simple_cubic(3, 3.1), 3.1, seed=5)
    sp = np.arange(27) % 2
    s = W.System(positions=pos, momenta=W.mb_momenta(np.array([12.0, 16.0])[sp], 300.0, 7), species=sp.astype(np.int32),
                 masses=np.array([12.0, 16.0]), box=np.array([9.3] * 3), seed=99)
    lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=4.6)
    d0 = W.input_dim(2, 16, 16)
    target = W.Potential(**lj, n_rbf=16, n_ang=16, n_layers=2, width=64, desc_cutoff=4.0, head="tanh",
                         head_scale=0.3, weights=W.mlp_weights(d0, 2, 64, 11))
    return W.Workload("ragged27", s, W.Potential(**lj), target, W.Integrator(1.0, 0.01, 300.0, 8), 100)


def _dilute_lists():
    """512 atoms of two species, simple cubic 8^3 at 4 A in a 32 A box: with a 6 A list radius the cell grid has
    five cells per axis, so the window's Verlet lists come from their own kernels (cell count, scan, fill, list)
    and, short enough to fit, are copied into the draft CTAs' shared memory (the config-2 box has no cell grid:
    there the draft lists its own atoms' candidates)."""
    pos = W.jitter(W.simple_cubic(8, 4.0), 4.0, seed=13)
    sp = (np.arange(512) % 3 == 0).astype(np.int32)
    masses = np.array([12.0, 16.0])
    s = W.System(positions=pos, momenta=W.mb_momenta(masses[sp], 300.0, 17), species=sp, masses=masses,
                 box=np.array([32.0] * 3), seed=23)
    lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=5.0)
    d0 = W.input_dim(2, 8, 0)
    target = W.Potential(**lj, n_rbf=8, n_ang=0, n_layers=1, width=32, desc_cutoff=4.0, head="tanh",
                         head_scale=0.3, weights=W.mlp_weights(d0, 1, 32, 29))
    return W.Workload("dilute512_lists", s, W.Potential(**lj), target, W.Integrator(1.0, 0.01, 300.0, 8), 100)


WORKLOADS = {"c1": lambda: W.config1(), "c2": lambda: W.config2(), "ragged27": _small_ragged,
             "dilute512": _dilute_lists}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def wl(request):
    return WORKLOADS[request.param]()


def test_target_neighbors_descriptors_forces(wl):
    """K configurations in one batched call: neighbour lists identical to the oracle's brute force; X, dE/dX,
    forces and energies within FP32 tolerance of FP64."""
    import torch
    lsd = _lsd()
    s = wl.system
    K = wl.integ.K
    h = lsd.LSD(s, wl.draft, wl.target, wl.integ)
    qs = _configs(s, K, 0.08, seed=123)
    F, E = h.target_forces(torch.tensor(qs, device="cuda"), energies=True)
    F, E = F.cpu().numpy(), E.cpu().numpy()
    X, G = h.descriptors(K)
    for c in range(K):
        ref = O.energy_forces(s, wl.target, qs[c], want=("F", "X", "dEdX", "E_atom"))
        desc, ljl = h.neighbors(c)
        od = O.neighbors(s, qs[c], wl.target.desc_cutoff)
        ol = O.neighbors(s, qs[c], wl.target.lj_cutoff)
        for i in range(s.n_atoms):
            assert np.array_equal(desc[i], od[i]), ("desc list", c, i)
            assert np.array_equal(ljl[i], ol[i]), ("lj list", c, i)
        assert _rel(X[c], ref["X"]) < FORCE_TOL and elem(X[c], ref["X"]) < FORCE_TOL
        assert _rel(G[c], ref["dEdX"]) < FORCE_TOL and elem(G[c], ref["dEdX"]) < FORCE_TOL
        assert _rel(F[c], ref["F"]) < FORCE_TOL, (c, _rel(F[c], ref["F"]))
        assert elem(F[c], ref["F"]) < FORCE_TOL, (c, elem(F[c], ref["F"]))
        assert abs(E[c].astype(np.float64).sum() - ref["E"]) < FORCE_TOL * np.abs(ref["E_atom"]).sum()
    h.close()


def _window_compare(win, ref, K, wl, target):
    assert np.array_equal(win["q_mid"][0], ref["qmid"][0]), "first half step is not bit-identical"
    for j in range(K):
        ptol, qtol = state_tols(wl, target, j + 1)
        assert np.abs(win["p_draft"][j] - ref["pdraft"][j]).max() < ptol, ("p_draft", j)
        # q_mid_j = q'_{j-1} + (dt/2) p'_{j-1}/m: within the position bound of step j
        assert np.abs(win["q_mid"][j] - ref["qmid"][j]).max() < qtol, ("q_mid", j)
    for j in range(K):
        for key_g, key_o in (("F_draft", "Fdraft"), ("F_target", "Ftarget")):
            assert _rel(win[key_g][j], ref[key_o][j]) < FORCE_TOL, (key_g, j)
            assert elem(win[key_g][j], ref[key_o][j]) < FORCE_TOL, (key_g, j, elem(win[key_g][j], ref[key_o][j]))
    tol = logr_tol(ref["logr"])
    assert (np.abs(win["log_ratio"] - ref["logr"]) <= tol).all(), np.abs(win["log_ratio"] - ref["logr"]) / tol
    assert np.allclose(win["delta_norm"], ref["delta_norm"], rtol=LOGR_DN, atol=1e-7)
    assert np.allclose(win["log_u"], ref["logu"], rtol=1e-15, atol=0)
    margin = np.abs(ref["logu"] - np.minimum(ref["logr"], 0.0))
    ties = margin <= tol
    assert not ties.any(), "decisions within the log-ratio tolerance at the test seed: %s" % np.nonzero(ties)
    assert np.array_equal(win["accept"], ref["accept"])


@pytest.mark.parametrize("head_scale", [None, 1.5])
def test_window_matches_oracle(wl, head_scale):
    """One window (Alg. 1, L = K) from the same base state: draft arrays, target forces, log ratios, accept
    decisions, committed count and the new state."""
    lsd = _lsd()
    s = wl.system
    target = wl.target if head_scale is None else W.replace(wl.target, head_scale=head_scale)
    h = lsd.LSD(s, wl.draft, target, wl.integ)
    h.draft_window()
    nc, first = h.verify_window()
    win = h.get_window()
    ref = O.lsd_window(s, wl.draft, target, wl.integ, s.seed, 0, wl.integ.K, s.positions, s.momenta)
    _window_compare(win, ref, wl.integ.K, wl, target)
    assert nc == ref["n_committed"]
    assert first == (-1 if ref["accept"].all() else int(np.argmin(ref["accept"])) + 1)
    q, p, step = h.get_state()
    assert step == nc
    ptol, qtol = state_tols(wl, target, nc, 0 if ref["accept"][:nc].all() else 1)
    assert np.abs(p - ref["p"]).max() < ptol
    assert np.abs(q - ref["q"]).max() < qtol
    h.close()


def test_free_running_matches_oracle_20_steps(wl):
    """lsd_step (the CUDA-graph window loop) and plain target ABOBA stay within tolerance of the oracle for 20
    steps; the committed step count is exact."""
    lsd = _lsd()
    s = wl.system
    target = W.replace(wl.target, head_scale=1.0)
    h = lsd.LSD(s, wl.draft, target, wl.integ)
    st = h.step(20)
    q, p, step = h.get_state()
    ref = O.lsd_run(s, wl.draft, target, wl.integ, s.seed, 20, wl.integ.K, s.positions, s.momenta)
    assert step == 20 == st["committed"]
    assert st["rejected"] == ref["stats"]["rejected"]
    ptol, qtol = state_tols(wl, target, 20, int(ref["stats"]["rejected"]))
    assert np.abs(p - ref["p"]).max() < ptol
    assert np.abs(q - ref["q"]).max() < qtol
    h.set_state(s.positions, s.momenta, 0)
    h.plain_step(20)
    q, p, step = h.get_state()
    refp = O.plain_run(s, target, wl.integ, s.seed, 20, s.positions, s.momenta)
    assert step == 20
    ptol, qtol = state_tols(wl, target, 20)
    assert np.abs(p - refp["p"]).max() < ptol
    assert np.abs(q - refp["q"]).max() < qtol
    h.close()


def test_error_correction_window_matches_oracle():
    """Alg. 3 on the GPU: two windows with the error-correction cache, decisions and states as the oracle's."""
    lsd = _lsd()
    w = W.config1()
    s = w.system
    target = W.replace(w.target, head_scale=1.0)
    h = lsd.LSD(s, w.draft, target, w.integ)
    h.set_error_correction(True)
    q, p, dF, step = s.positions.copy(), s.momenta.copy(), np.zeros_like(s.positions), 0
    for _ in range(3):
        h.draft_window()
        nc, _ = h.verify_window()
        win = h.get_window()
        ref = O.lsd_window(s, w.draft, target, w.integ, s.seed, step, w.integ.K, q, p, ec_dF=dF)
        assert nc == ref["n_committed"]
        assert np.array_equal(win["accept"], ref["accept"])
        gq, gp, gstep = h.get_state()
        q, p, dF = ref["q"], ref["p"], ref["ec_dF"]
        step += nc
        assert gstep == step
        ptol, qtol = state_tols(w, target, nc, 0 if ref["accept"][:nc].all() else 1)
        assert np.abs(gp - p).max() < ptol and np.abs(gq - q).max() < qtol
        h.set_state(q, p, step)    # keep both sides on the oracle's state
    h.close()


def test_draft_equal_target_accepts_everything():
    """T3 on the GPU: LJ draft and LJ target give delta ~ 0; every step is accepted and LSD follows plain target
    ABOBA to rounding."""
    lsd = _lsd()
    w = W.config2()
    s = w.system
    h = lsd.LSD(s, w.draft, w.draft, w.integ)
    st = h.step(64)
    assert st["rejected"] == 0 and st["committed"] == 64
    q1, p1, _ = h.get_state()
    h.set_state(s.positions, s.momenta, 0)
    h.plain_step(64)
    q2, p2, _ = h.get_state()
    # both runs use the same FP32 forces of the same potential: only the summation of the draft kernel and of the
    # verification kernels differs (~1e-6 of |F| per element), far inside the oracle bound used here
    ptol, qtol = state_tols(w, w.draft, 64, draft=w.draft)
    assert np.abs(p1 - p2).max() < ptol and np.abs(q1 - q2).max() < qtol
    h.close()


def test_checkpoint_resume_is_bitwise():
    """2 x 24 steps with a checkpoint/restore in between equal 48 uninterrupted steps bit for bit."""
    lsd = _lsd()
    w = W.config1()
    s = w.system
    target = W.replace(w.target, head_scale=1.0)
    a = lsd.LSD(s, w.draft, target, w.integ)
    a.step(48)
    qa, pa, _ = a.get_state()
    b = lsd.LSD(s, w.draft, target, w.integ)
    b.step(24)
    blob = b.checkpoint()
    b.close()
    c = lsd.LSD(s, w.draft, target, w.integ)
    c.restore(blob)
    c.step(24)
    qc, pc, stc = c.get_state()
    assert stc == 48 and np.array_equal(qa, qc) and np.array_equal(pa, pc)
    a.close()
    c.close()


def test_single_atom_and_window_of_one():
    """Degenerate cases: one atom interacting only with its own images, window length 1."""
    lsd = _lsd()
    s = W.System(positions=np.array([[1.0, 2.0, 3.0]]), momenta=np.array([[0.01, -0.02, 0.03]]),
                 species=np.array([0], np.int32), masses=np.array([40.0]), box=np.array([6.0] * 3), seed=3)
    lj = W.Potential(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=5.9)
    tgt = W.Potential(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=5.9, n_rbf=4, n_ang=16,
                      n_layers=1, width=32, desc_cutoff=5.5, head="tanh", head_scale=0.05,
                      weights=W.mlp_weights(W.input_dim(1, 4, 16), 1, 32, 2))
    integ = W.Integrator(2.0, 0.01, 300.0, 1)
    h = lsd.LSD(s, lj, tgt, integ)
    h.draft_window()
    nc, _ = h.verify_window()
    win = h.get_window()
    ref = O.lsd_window(s, lj, tgt, integ, s.seed, 0, 1, s.positions, s.momenta)
    assert nc == ref["n_committed"] == 1
    assert np.array_equal(win["accept"], ref["accept"])
    assert np.allclose(win["F_target"][0], ref["Ftarget"][0], atol=1e-7)
    h.close()


def test_target_energy_autograd_is_minus_forces():
    import torch
    lsd = _lsd()
    w = W.config1()
    s = w.system
    h = lsd.LSD(s, w.draft, w.target, w.integ)
    q = torch.tensor(_configs(s, 3, 0.05, 9), device="cuda", requires_grad=True)
    E = lsd.target_energy(q, h)
    E.sum().backward()
    F = h.target_forces(q.detach())
    assert torch.allclose(q.grad, -F.double(), rtol=0, atol=0)
    for c in range(3):
        ref = O.energy(s, w.target, q[c].detach().cpu().numpy())
        assert abs(E[c].item() - ref) < 1e-5 * 32
    h.close()


# ---------------------------------------------------------------------------------------------------------------
# learned draft
# ---------------------------------------------------------------------------------------------------------------

def test_learned_draft_bf16_forces_within_tolerance():
    """BF16 inference of the learned draft inside the draft kernel: draft forces of the window within 2e-2 of
    the oracle's FP64 forces of the same draft (weights scaled up so the MLP term is not negligible)."""
    lsd = _lsd()
    w = W.config3()
    s = w.system
    draft = W.replace(w.draft, weights=W.mlp_weights(W.input_dim(1, 8, 0), 1, 32, seed=3))
    h = lsd.LSD(s, draft, w.target, w.integ)
    h.draft_window()
    h.verify_window()
    win = h.get_window()
    ref = O.lsd_window(s, draft, w.target, w.integ, s.seed, 0, w.integ.K, s.positions, s.momenta)
    lj_only = W.Potential(lj_eps=draft.lj_eps, lj_sigma=draft.lj_sigma, lj_cutoff=draft.lj_cutoff)
    for j in range(w.integ.K):
        mlp_part = ref["Fdraft"][j] - O.forces(s, lj_only, ref["qmid"][j])
        assert np.linalg.norm(mlp_part) > 0.05 * np.linalg.norm(ref["Fdraft"][j])
        assert _rel(win["F_draft"][j], ref["Fdraft"][j]) < BF16_TOL, j
    h.close()


def test_force_matching_gradient_matches_oracle():
    """The GPU's hand-written double backward (loss and dL/dtheta of force matching) against the oracle's FP64."""
    import torch
    lsd = _lsd()
    w = W.config3()
    s = w.system
    draft = W.replace(w.draft, weights=W.mlp_weights(W.input_dim(1, 8, 0), 1, 32, seed=3))
    h = lsd.LSD(s, draft, w.target, w.integ)
    fq = _configs(s, 6, 0.1, seed=77)
    fF = np.stack([O.forces(s, w.target, q) for q in fq]).astype(np.float32)
    loss, g = h.force_match(torch.tensor(fq, device="cuda"), torch.tensor(fF, device="cuda"))
    rl, rg = O.force_match(s, draft, fq, fF.astype(np.float64))
    assert abs(loss - rl) / rl < 1e-4
    g = g.cpu().numpy()
    assert _rel(g, rg) < 1e-4, _rel(g, rg)
    h.close()


def test_learned_draft_training_reduces_rejections():
    """Frames captured by verification train the learned draft (Adam on the force-matching loss); the loss
    drops and the mean Mahalanobis distance |delta| (Eq. 6) falls below the untrained draft's."""
    lsd = _lsd()
    w = W.config3(K=8)
    s = w.system
    target = W.replace(w.target, head_scale=0.5)
    h = lsd.LSD(s, w.draft, target, w.integ)
    h.set_frame_capture(4096)
    st0 = h.step(400)
    assert h.frame_count() > 100
    l0 = h.train_draft(1, 1e-3)
    l1 = h.train_draft(300, 3e-3)
    assert l1 < 0.5 * l0, (l0, l1)
    before = st0["sum_delta"] / st0["committed"]
    st1 = h.step(400)
    after = (st1["sum_delta"] - st0["sum_delta"]) / (st1["committed"] - st0["committed"])
    assert after < 0.8 * before, (before, after)
    h.close()


@pytest.mark.parametrize("name", ["c2", "dilute512"])
def test_forces_do_not_depend_on_batch_or_launch_shape(name):
    """The adjoint is a fixed-order gather (pair gradients by diagonals, no atomics): a configuration's forces and
    energies are bit-identical whether it is evaluated alone or as one row block of a K-configuration batch (other
    grids, other tiles of the MLP), and the window's target forces equal the explicit entry point's on the window's
    own half-step positions."""
    import torch
    lsd = _lsd()
    w = WORKLOADS[name]()
    s = w.system
    K = w.integ.K
    h = lsd.LSD(s, w.draft, w.target, w.integ)
    qs = torch.tensor(_configs(s, K, 0.08, seed=321), device="cuda")
    F_all, E_all = h.target_forces(qs, energies=True)
    for c in (0, K // 2, K - 1):
        F_one, E_one = h.target_forces(qs[c:c + 1], energies=True)
        assert torch.equal(F_one[0], F_all[c]) and torch.equal(E_one[0], E_all[c]), c
    h.draft_window()
    h.verify_window()
    win = h.get_window()
    k_eff = h.stats()["verified"]
    F_win = h.target_forces(torch.tensor(win["q_mid"][:k_eff], device="cuda")).cpu().numpy()
    assert np.array_equal(F_win, win["F_target"][:k_eff])
    h.close()
