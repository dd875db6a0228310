"""Oracle pins for the integrator and the speculative protocol: draft == target reproduces plain ABOBA bit for
bit (Eq. 5, Eq. 6), the committed trajectory does not depend on the window length (Alg. 1 with step-indexed
noise), the harmonic ABOBA chain matches its exact stationary covariance (Eq. 2; discrete Lyapunov equation) and
LSD with a wrong draft converges to the target's, and error correction (Alg. 3) removes a constant draft error."""
import numpy as np
import pytest
from scipy import linalg

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W


def _stronger_target(w, scale=0.6):
    t = W.replace(w.target, head_scale=scale)
    return t


def test_draft_equal_target_reproduces_plain_aboba_bitwise():
    """T3: with F~ = F every step is accepted and the LSD trajectory equals plain target ABOBA bit for bit."""
    w = W.config1()
    s = w.system
    lsd = O.lsd_run(s, w.target, w.target, w.integ, s.seed, 24, 8, s.positions, s.momenta, traj=True)
    plain = O.plain_run(s, w.target, w.integ, s.seed, 24, s.positions, s.momenta, traj=True)
    assert lsd["stats"]["rejected"] == 0
    assert np.array_equal(lsd["traj_q"], plain["traj_q"])
    assert np.array_equal(lsd["traj_p"], plain["traj_p"])


@pytest.mark.parametrize("K", [1, 3, 8, 16])
def test_trajectory_is_independent_of_window_length(K):
    """T4: committed trajectories for window lengths K are identical (noise keyed by step index; the first
    rejected step is reflected, later ones flushed), and rejections do occur."""
    w = W.config1()
    s = w.system
    target = _stronger_target(w)
    ref = O.lsd_run(s, w.draft, target, w.integ, s.seed, 40, 1, s.positions, s.momenta, traj=True)
    run = O.lsd_run(s, w.draft, target, w.integ, s.seed, 40, K, s.positions, s.momenta, traj=True)
    assert ref["stats"]["rejected"] >= 2
    assert np.array_equal(run["traj_q"], ref["traj_q"])
    assert np.array_equal(run["traj_p"], ref["traj_p"])
    assert run["stats"]["rejected"] == ref["stats"]["rejected"]


def test_resume_equals_uninterrupted_run():
    """Checkpoint/resume: two runs of 20 steps from the saved (q, p, step) equal one run of 40 steps."""
    w = W.config1()
    s = w.system
    target = _stronger_target(w)
    full = O.lsd_run(s, w.draft, target, w.integ, s.seed, 40, 8, s.positions, s.momenta)
    a = O.lsd_run(s, w.draft, target, w.integ, s.seed, 20, 8, s.positions, s.momenta)
    b = O.lsd_run(s, w.draft, target, w.integ, s.seed, 20, 8, a["q"], a["p"], step=a["step"])
    assert b["step"] == 40
    assert np.array_equal(b["q"], full["q"]) and np.array_equal(b["p"], full["p"])


def test_window_commits_prefix_and_reflection():
    """Alg. 1: the window commits exactly the accepted prefix plus the first rejected step, whose state is the
    reflected one; accepted states are the draft's bits."""
    w = W.config1()
    s = w.system
    target = _stronger_target(w, 2.0)
    out = O.lsd_window(s, w.draft, target, w.integ, s.seed, 0, 8, s.positions, s.momenta)
    acc = out["accept"]
    l = int(np.argmin(acc)) + 1 if not acc.all() else 8
    assert out["n_committed"] == l
    c1, aF, hm, sg = O.coefficients(s, w.integ)
    if not acc.all():
        j = l - 1
        p_prev = s.momenta if j == 0 else out["pdraft"][j - 1]
        mu_t = c1 * p_prev + aF * out["Ftarget"][j]
        sig = sg[s.species][:, None]
        z = (out["pdraft"][j] - out["mudraft"][j]) / sig
        dl = (out["mudraft"][j] - mu_t) / sig
        p_ref = mu_t + sig * (z - 2 * (z * dl).sum() / (dl * dl).sum() * dl)
        assert np.allclose(out["p"], p_ref, rtol=1e-12, atol=1e-15)
    else:
        assert np.array_equal(out["p"], out["pdraft"][7])


def _harmonic_system(n_atoms=64, k=0.05, mass=12.0):
    pos = np.random.default_rng(0).uniform(0, 20, (n_atoms, 3))
    s = W.System(positions=pos, momenta=np.zeros((n_atoms, 3)), species=np.zeros(n_atoms, np.int32),
                 masses=np.array([mass]), box=np.array([20.0] * 3), seed=77)
    return s


def _aboba_stationary_cov(k, m, integ):
    """Exact stationary covariance of (x, p) for ABOBA on U = k x^2/2 from C = M C M^T + n n^T."""
    kappa, kB = O.kappa(), O.kboltz()
    h = integ.dt / 2
    c1 = np.exp(-integ.gamma * integ.dt)
    sig = np.sqrt(m * kB * integ.temperature * kappa * (1 - np.exp(-2 * integ.gamma * integ.dt)))
    A = np.array([[1, h / m], [0, 1]])
    B = np.array([[1, 0], [-h * kappa * k, 1]])
    Om = np.array([[1, 0], [0, c1]])
    M = A @ B @ Om @ B @ A
    n = A @ B @ np.array([0, sig])
    return linalg.solve_discrete_lyapunov(M, np.outer(n, n))


@pytest.mark.slow
def test_harmonic_stationary_covariance_plain_and_lsd():
    """T8: plain target ABOBA on a harmonic tether matches the exact discrete stationary covariance; LSD with a
    draft of a different stiffness samples the target's covariance, not the draft's."""
    k_t, k_d, m = 2.0, 3.0, 12.0
    s = _harmonic_system(mass=m)
    integ = W.Integrator(dt=2.0, gamma=0.05, temperature=300.0, K=4)
    q_ref = s.positions.copy()
    target = W.Potential(k_harm=k_t, q_ref=q_ref)
    draft = W.Potential(k_harm=k_d, q_ref=q_ref)
    C_t = _aboba_stationary_cov(k_t, m, integ)
    C_d = _aboba_stationary_cov(k_d, m, integ)
    assert C_d[0, 0] < 0.75 * C_t[0, 0]
    kappa, kB = O.kappa(), O.kboltz()
    # start from the stationary law so no burn-in is needed
    rng = np.random.default_rng(1)
    L = np.linalg.cholesky(C_t)
    z = rng.standard_normal((s.n_atoms * 3, 2)) @ L.T
    q0 = q_ref + z[:, 0].reshape(-1, 3)
    p0 = z[:, 1].reshape(-1, 3)
    n_steps = 3000
    for name, runner in (("plain", lambda: O.plain_run(s, target, integ, s.seed, n_steps, q0, p0, traj=True)),
                         ("lsd", lambda: O.lsd_run(s, draft, target, integ, s.seed, n_steps, 4, q0, p0, traj=True))):
        r = runner()
        x = (r["traj_q"][::10] - q_ref).reshape(-1)
        p = r["traj_p"][::10].reshape(-1)
        # effective sample count: samples decorrelate over ~2/gamma = 40 fs (20 steps); one kept per 10 steps
        n_eff = x.size / 2.0
        for est, ref in ((np.mean(x * x), C_t[0, 0]), (np.mean(p * p), C_t[1, 1])):
            assert abs(est / ref - 1) < 5 * np.sqrt(2 / n_eff), (name, est, ref)
        assert np.mean(x * x) > 0.9 * C_t[0, 0], name
    # equipartition of momenta up to O(dt^2): <p^2/m> = kB T kappa
    assert C_t[1, 1] / m == pytest.approx(kB * 300.0 * kappa, rel=0.02)


def test_error_correction_removes_constant_error():
    """Alg. 3: a draft whose force differs from the target's by a constant gets delta = 0 after the first
    commit with error correction, so every later step is accepted; without it rejections persist."""
    s = _harmonic_system(n_atoms=8)
    integ = W.Integrator(dt=2.0, gamma=0.01, temperature=300.0, K=4)
    q_ref = s.positions.copy()
    target = W.Potential(k_harm=0.05, q_ref=q_ref)
    draft = W.Potential(k_harm=0.05, q_ref=q_ref + 1.0)
    p0 = np.zeros_like(q_ref)
    no_ec = O.lsd_run(s, draft, target, integ, s.seed, 200, 4, q_ref, p0, use_ec=False)
    ec = O.lsd_run(s, draft, target, integ, s.seed, 200, 4, q_ref, p0, use_ec=True)
    assert no_ec["stats"]["rejected"] > 20
    assert ec["stats"]["rejected"] <= 1
    # |delta| is the same on every uncorrected step; with EC only the steps committed by the first window
    # (drafted before the cache held an error) carry it
    per_step = no_ec["stats"]["sum_delta"] / no_ec["stats"]["committed"]
    ratio = ec["stats"]["sum_delta"] / per_step
    assert 1 <= round(ratio) <= integ.K and ratio == pytest.approx(round(ratio), rel=1e-9)


def test_predicted_rejections_match_observed():
    """Eq. 6 along a trajectory: the number of rejections is consistent with the sum of erf(|delta_n|/sqrt 8)
    over committed steps (binomial z-test)."""
    w = W.config1()
    s = w.system
    target = _stronger_target(w, 0.6)
    r = O.lsd_run(s, w.draft, target, w.integ, s.seed, 300, 8, s.positions, s.momenta)
    st = r["stats"]
    mean = st["pred_rejected"]
    var = mean * (1 - mean / st["committed"])
    assert abs(st["rejected"] - mean) < 4 * np.sqrt(var) + 1


def test_window_parallel_verification_equals_serial():
    """The oracle's window-parallel variant (the K target evaluations of a window on several threads, the CPU
    analogue of the batched verification) gives the serial result bit for bit."""
    w = W.config1()
    s = w.system
    target = W.replace(w.target, head_scale=1.5)
    O.set_threads(1)
    a = O.lsd_window(s, w.draft, target, w.integ, s.seed, 0, w.integ.K, s.positions, s.momenta)
    O.set_threads(4)
    try:
        b = O.lsd_window(s, w.draft, target, w.integ, s.seed, 0, w.integ.K, s.positions, s.momenta)
    finally:
        O.set_threads(1)
    for k in ("qmid", "pdraft", "Ftarget", "logr", "accept", "q", "p"):
        assert np.array_equal(a[k], b[k]), k
    assert a["n_committed"] == b["n_committed"]
