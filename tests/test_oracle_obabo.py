"""Oracle pins for OBABO through the staggered frame (App. E).

- The recovery of the OBABO output momentum (the conditional draw of the first half-step noise given the staggered
  result) against the closed-form joint law of the two O half-steps: with u = p_mid - e^(-g dt/2) p_in and
  v = p_new - (dt/2) k F - e^(-g dt) p_in, Var(u) = S_1/2, Var(v) = (1 + e^(-g dt)) S_1/2, Cov(u, v) =
  e^(-g dt/2) S_1/2.
- The harmonic tether: the OBABO map is linear, so its exact stationary covariance solves a discrete Lyapunov
  equation; the literal integrator, the staggered plain chain and staggered LSD with a draft of another stiffness
  all reach the target's covariance.
- Draft equal to target reproduces the plain staggered chain bit for bit (T3); the committed trajectory does not
  depend on the window length (T4)."""
import numpy as np
import pytest
from scipy import linalg

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W


def _coefs(m, integ):
    kappa, kB = O.kappa(), O.kboltz()
    ch = np.exp(-integ.gamma * integ.dt / 2)
    sh = np.sqrt(m * kB * integ.temperature * kappa * (1 - np.exp(-integ.gamma * integ.dt)))
    return ch, sh, integ.dt / 2 * kappa


def test_recovered_momentum_has_the_half_step_joint_law():
    n = 60000
    m = 12.0
    s = W.System(positions=np.zeros((n, 3)), momenta=np.zeros((n, 3)), species=np.zeros(n, np.int32),
                 masses=np.array([m]), box=np.array([100.0] * 3), seed=5)
    integ = W.Integrator(dt=2.0, gamma=0.05, temperature=300.0, K=1, scheme="obabo")
    ch, sh, bF = _coefs(m, integ)
    c1 = ch * ch
    rng = np.random.default_rng(3)
    p_prev = rng.normal(0, 3.0, (n, 3))
    F = rng.normal(0, 0.5, (n, 3))
    p_in = p_prev + bF * F
    xi1, xi2 = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    p_mid_true = ch * p_in + sh * xi1
    p_new = ch * p_mid_true + sh * xi2 + bF * F                     # the staggered momentum after the block
    p_mid = O.obabo_output(s, integ, s.seed, 17, p_prev, F, p_new)
    u = (p_mid - ch * p_in).ravel()
    v = (p_new - bF * F - c1 * p_in).ravel()
    tol = 5 * np.sqrt(2.0 / u.size)
    assert np.var(u) / sh ** 2 == pytest.approx(1.0, abs=tol)
    assert np.mean(u * v) / (ch * sh ** 2) == pytest.approx(1.0, abs=2 * tol)
    assert np.var(v) / ((1 + c1) * sh ** 2) == pytest.approx(1.0, abs=tol)
    # and the recovered momentum is distributed as the true one
    assert np.var(p_mid - p_mid_true) > 0                           # not a copy: a fresh conditional draw
    assert np.mean(p_mid) == pytest.approx(np.mean(p_mid_true), abs=5 * sh / np.sqrt(u.size))


def _obabo_stationary_cov(k, m, integ):
    """Exact stationary covariance of (x, p) for literal OBABO on U = k x^2 / 2."""
    ch, sh, bF = _coefs(m, integ)
    Oh = np.array([[1, 0], [0, ch]])
    B = np.array([[1, 0], [-bF * k, 1]])
    A = np.array([[1, integ.dt / m], [0, 1]])
    M = Oh @ B @ A @ B @ Oh
    n1 = Oh @ B @ A @ B @ np.array([0, sh])
    n2 = np.array([0, sh])
    return linalg.solve_discrete_lyapunov(M, np.outer(n1, n1) + np.outer(n2, n2))


def _harmonic(n_atoms=64, m=12.0):
    pos = np.random.default_rng(0).uniform(0, 20, (n_atoms, 3))
    return W.System(positions=pos, momenta=np.zeros((n_atoms, 3)), species=np.zeros(n_atoms, np.int32),
                    masses=np.array([m]), box=np.array([20.0] * 3), seed=91)


@pytest.mark.slow
def test_harmonic_stationary_covariance_literal_staggered_and_lsd():
    k_t, k_d, m = 2.0, 3.0, 12.0
    s = _harmonic(m=m)
    integ = W.Integrator(dt=2.0, gamma=0.05, temperature=300.0, K=4, scheme="obabo")
    q_ref = s.positions.copy()
    target = W.Potential(k_harm=k_t, q_ref=q_ref)
    draft = W.Potential(k_harm=k_d, q_ref=q_ref)
    C_t = _obabo_stationary_cov(k_t, m, integ)
    C_d = _obabo_stationary_cov(k_d, m, integ)
    assert C_d[0, 0] < 0.75 * C_t[0, 0]
    rng = np.random.default_rng(2)
    z = rng.standard_normal((s.n_atoms * 3, 2)) @ np.linalg.cholesky(C_t).T
    q0 = q_ref + z[:, 0].reshape(-1, 3)
    p0 = z[:, 1].reshape(-1, 3)
    pbar0 = O.obabo_enter(s, target, integ, s.seed, 0, q0, p0)      # into the staggered frame
    n_steps = 3000
    runs = {
        "literal": lambda: O.obabo_literal(s, target, integ, s.seed, n_steps, q0, p0, traj=True),
        "staggered": lambda: O.plain_run(s, target, integ, s.seed, n_steps, q0, pbar0, traj=True),
        "lsd": lambda: O.lsd_run(s, draft, target, integ, s.seed, n_steps, 4, q0, pbar0, traj=True),
    }
    for name, run in runs.items():
        r = run()
        x = (r["traj_q"][::10] - q_ref).reshape(-1)
        p = r["traj_p"][::10].reshape(-1)
        n_eff = x.size / 2.0
        for est, ref in ((np.mean(x * x), C_t[0, 0]), (np.mean(p * p), C_t[1, 1]), (np.mean(x * p), C_t[0, 1])):
            scale = np.sqrt(C_t[0, 0] * C_t[1, 1]) if ref is C_t[0, 1] else ref
            assert abs(est - ref) / scale < 5 * np.sqrt(2 / n_eff), (name, est, ref)
        if name == "lsd":
            assert r["stats"]["rejected"] > 10


def test_draft_equal_target_is_the_plain_staggered_chain_bitwise():
    w = W.config1()
    s = w.system
    integ = W.replace(w.integ, scheme="obabo")
    pbar = O.obabo_enter(s, w.target, integ, s.seed, 0, s.positions, s.momenta)
    lsd = O.lsd_run(s, w.target, w.target, integ, s.seed, 24, 8, s.positions, pbar, traj=True)
    plain = O.plain_run(s, w.target, integ, s.seed, 24, s.positions, pbar, traj=True)
    assert lsd["stats"]["rejected"] == 0
    for key in ("traj_q", "traj_p", "q", "p", "p_obabo"):
        assert np.array_equal(lsd[key], plain[key]), key


@pytest.mark.parametrize("K", [1, 5, 8])
def test_staggered_trajectory_is_independent_of_window_length(K):
    w = W.config1()
    s = w.system
    integ = W.replace(w.integ, scheme="obabo")
    target = W.replace(w.target, head_scale=0.6)
    pbar = O.obabo_enter(s, target, integ, s.seed, 0, s.positions, s.momenta)
    ref = O.lsd_run(s, w.draft, target, integ, s.seed, 32, 1, s.positions, pbar, traj=True)
    run = O.lsd_run(s, w.draft, target, integ, s.seed, 32, K, s.positions, pbar, traj=True)
    assert ref["stats"]["rejected"] >= 2
    for key in ("traj_q", "traj_p", "p_obabo"):
        assert np.array_equal(run[key], ref[key]), key


def test_staggered_positions_advance_by_full_steps():
    """The staggered transition's A is the full step q_n = q_(n-1) + dt p_(n-1) / m (App. E)."""
    w = W.config1()
    s = w.system
    integ = W.replace(w.integ, scheme="obabo")
    out = O.lsd_window(s, w.draft, w.target, integ, s.seed, 0, 4, s.positions, s.momenta)
    m = s.masses[s.species][:, None]
    assert np.array_equal(out["qmid"][0], s.positions + s.momenta * (integ.dt / m))
    assert np.array_equal(out["qmid"][1], out["qmid"][0] + out["pdraft"][0] * (integ.dt / m))
