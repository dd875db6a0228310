"""The rejection-law and speedup-bound tooling (paper_2606_02455_b300/analysis.py) against closed forms, Monte Carlo
and the oracle.  T11 (the scaling law of Eq. 9 fitted at one system size and used at another) is reported, not
gated."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2606_02455_b300 import analysis as A


def test_rejection_law_is_total_variation_of_unit_gaussians():
    """Eq. 6: the reflection coupling rejects with the total-variation distance of N(0,1) and N(|delta|,1),
    integrated numerically here."""
    for d in (0.0, 0.1, 0.5, 1.3, 3.0):
        tv, _ = integrate.quad(lambda x: 0.5 * abs(stats.norm.pdf(x) - stats.norm.pdf(x, loc=d)), -12, 12 + d,
                               points=[d / 2], limit=200)
        assert A.rejection_probability(d) == pytest.approx(tv, abs=1e-9)


def test_expected_committed_matches_bernoulli_windows():
    rng = np.random.default_rng(0)
    for beta, K in ((0.0, 8), (0.05, 16), (0.3, 4), (1.0, 6)):
        rej = rng.random((200000, K)) < beta
        first = np.where(rej.any(axis=1), rej.argmax(axis=1) + 1, K)   # accepted prefix + reflected step
        assert A.expected_committed(beta, K) == pytest.approx(first.mean(), rel=5e-3, abs=5e-3)


def test_speedup_bounds_limits_and_order():
    c = 0.05
    assert A.speedup_async(0.0, c) == pytest.approx(1.0 / c)             # full draft throughput at a -> 1
    assert A.speedup_sync(0.3, c, 0) == pytest.approx(1.0)               # no lookahead, no gain
    for L in (1, 4, 16, 64):
        assert A.speedup_sync(0.0, c, L) == pytest.approx((L + 1) / (L * c + 1))
        for beta in (0.0, 0.01, 0.2):
            assert A.speedup_sync(beta, c, L) <= (L + 1) / (L * c + 1) + 1e-12 < 1.0 / c
            # the sum form of the truncated geometric series
            a = 1 - beta
            assert A.speedup_sync(beta, c, L) == pytest.approx(sum(a ** k for k in range(L + 1)) / (L * c + 1))


def test_scaling_law_fit_and_prediction():
    eps = A.fit_scaling_eps(0.2, 256, 100.0, 1.0, 300.0)
    assert A.predict_beta(eps, 256, 100.0, 1.0, 300.0) == pytest.approx(0.2)
    # the argument grows like sqrt(N tau dt / T)
    assert A.scaling_argument(512, 100.0, 1.0, 300.0) / A.scaling_argument(256, 100.0, 1.0, 300.0) == pytest.approx(
        math.sqrt(2.0))
    assert A.predict_beta(eps, 256, 100.0, 1.0, 600.0) < 0.2            # hotter: errors hidden under more noise
    with pytest.raises(ValueError):
        A.fit_scaling_eps(0.0, 1, 1.0, 1.0, 1.0)


def test_window_model_optimum():
    costs = A.WindowCosts(t_draft=1.0, verify_fixed=50.0, verify_per_step=2.0, t_plain=40.0)
    assert costs.c == pytest.approx(1.0 / 40.0)
    k, s = A.best_window(0.0, costs, K_max=64)                             # no rejections: longest window wins
    assert k == 64 and s == pytest.approx(64 * 40.0 / (64 * 3.0 + 50.0))
    assert A.best_window(1.0, costs)[0] == 1                               # every step rejected: one per window
    k, _ = A.best_window(0.05, costs, K_max=256)
    assert 1 < k < 256
    ks = np.arange(1, 257)
    assert k == ks[np.argmax(A.speedup_window(0.05, costs, ks))]
    fixed, per = A.fit_verify_costs([4, 8, 16, 32], [58.0, 66.0, 82.0, 114.0])
    assert fixed == pytest.approx(50.0) and per == pytest.approx(2.0)


def test_t11_scaling_law_report():
    """T11: fit eps from the oracle's measured <beta> at 32 atoms and predict 108 atoms of the same density and
    potentials; reported (Eq. 9 is a model), only sanity is asserted."""
    import oracle.oracle as O
    from paper_2606_02455_b300 import workloads as W
    rows = []
    for cells in (2, 3):
        s = W.small_system(n_cells=cells, a=5.0, n_species=2, seed=1)
        d0 = O.input_dim(2, 16, 0)
        lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=4.9)
        tgt = W.Potential(**lj, n_rbf=16, n_ang=0, n_layers=1, width=32, desc_cutoff=4.9, head="tanh",
                          head_scale=0.05, weights=W.mlp_weights(d0, 1, 32, seed=1))
        integ = W.Integrator(2.0, 0.01, 300.0, 8)
        p = O.mb_momenta(s, integ, 3)
        r = O.lsd_run(s, W.Potential(**lj), tgt, integ, 11, 160, 8, s.positions, p)["stats"]
        rows.append((s.n_atoms, r["rejected"] / r["verified"]))
    (n1, b1), (n2, b2) = rows
    eps = A.fit_scaling_eps(min(max(b1, 1e-3), 0.999), n1, 100.0, 2.0, 300.0)
    pred = float(A.predict_beta(eps, n2, 100.0, 2.0, 300.0))
    print("T11: <beta> measured %.4f at N=%d, %.4f at N=%d; Eq. 9 predicts %.4f" % (b1, n1, b2, n2, pred))
    assert 0.0 <= b1 <= 1.0 and 0.0 <= b2 <= 1.0 and 0.0 < pred < 1.0


def test_staged_window_model_against_bernoulli_windows_and_limits():
    """Windows verified in stages: the mean stages run and steps verified against simulated Bernoulli windows; S = 1
    verifies exactly the committed steps, S >= K is the one-pass window (and the staged cost model then reduces to
    the one-pass window model)."""
    rng = np.random.default_rng(1)
    for beta, K, S in ((0.2, 64, 2), (0.05, 32, 4), (0.5, 16, 3), (0.0, 8, 3)):
        rej = rng.random((200000, K)) < beta
        first = np.where(rej.any(axis=1), rej.argmax(axis=1) + 1, K)       # committed steps
        n_st = -(-first // S)                                              # the stage holding the last committed step
        verified = np.minimum(n_st * S, K)
        assert A.expected_stages(beta, K, S) == pytest.approx(n_st.mean(), rel=5e-3, abs=5e-3)
        assert A.expected_verified(beta, K, S) == pytest.approx(verified.mean(), rel=5e-3, abs=5e-3)
        assert A.expected_verified(beta, K, 1) == pytest.approx(float(A.expected_committed(beta, K)))
        assert A.expected_stages(beta, K, K) == 1.0 and A.expected_verified(beta, K, K + 5) == K
    one = A.WindowCosts(t_draft=0.2, verify_fixed=0.3, verify_per_step=0.5, t_plain=0.55)
    staged = A.StageCosts(per_step=0.7, per_stage=0.1, per_window=0.2, t_plain=0.55)
    assert A.speedup_staged(0.2, staged, 64, 64) == pytest.approx(float(A.speedup_window(0.2, one, 64)))
    S, sp = A.best_stage_length(0.2, staged, 64)
    assert 1 <= S < 64 and sp > A.speedup_staged(0.2, staged, 64, 64)
    # a free stage makes S = 1 optimal: no step past the first rejection is paid for
    assert A.best_stage_length(0.2, A.StageCosts(0.7, 0.0, 0.2, 0.55), 64)[0] == 1
