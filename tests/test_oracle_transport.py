"""Oracle pins for reflectionVerify (Eq. 5): the 1-D picture of Fig. 2, the closed-form rejection rate of
Eq. 6, and the coupling property (Eq. 3): transported draft samples are target distributed."""
import numpy as np
import pytest
from scipy import special, stats

import oracle.oracle as O


def test_one_dimensional_reflection():
    """Fig. 2: in 1-D the reflection through the equal-likelihood point maps p~ to <p> + <p~> - p~,
    and acceptance is u <= min(1, N(p~;<p>,s)/N(p~;<p~>,s))."""
    mu_d, mu_t, sig = 0.3, -0.4, 0.7
    rng = np.random.default_rng(0)
    for _ in range(200):
        pd = mu_d + sig * rng.standard_normal()
        u = rng.uniform(1e-9, 1.0)
        acc, p, lr = O.transport([sig], u, [pd], [mu_d], [mu_t])
        ratio = stats.norm.pdf(pd, mu_t, sig) / stats.norm.pdf(pd, mu_d, sig)
        assert lr == pytest.approx(np.log(ratio), abs=1e-12)
        assert acc == (u <= min(1.0, ratio))
        if acc:
            assert p[0] == pd
        else:
            assert p[0] == pytest.approx(mu_t + mu_d - pd, abs=1e-14)


def _mc_transport(D, delta_norm, n, seed):
    rng = np.random.default_rng(seed)
    sig = rng.uniform(0.5, 2.0, D)
    mu_t = rng.standard_normal(D)
    direction = rng.standard_normal(D)
    direction /= np.linalg.norm(direction)
    mu_d = mu_t + sig * direction * delta_norm      # |S^-1/2 (mu_d - mu_t)| = delta_norm
    acc = np.zeros(n, bool)
    out = np.zeros((n, D))
    for k in range(n):
        pd = mu_d + sig * rng.standard_normal(D)
        u = 1.0 - rng.uniform()                       # (0, 1]
        a, p, _ = O.transport(sig, u, pd, mu_d, mu_t)
        acc[k] = a
        out[k] = (p - mu_t) / sig
    return acc, out, direction


@pytest.mark.parametrize("D,delta_norm", [(1, 0.5), (6, 0.8), (30, 2.0)])
def test_rejection_rate_is_erf(D, delta_norm):
    """Eq. 6: the rejection rate equals erf(|delta| / sqrt(8)) (binomial 4-sigma band)."""
    n = 12000
    acc, _, _ = _mc_transport(D, delta_norm, n, seed=D)
    beta = special.erf(delta_norm / np.sqrt(8.0))
    se = np.sqrt(beta * (1 - beta) / n)
    assert abs((1 - acc.mean()) - beta) < 4 * se + 1e-4


@pytest.mark.parametrize("D,delta_norm", [(6, 1.2), (30, 2.5)])
def test_transported_samples_are_target_distributed(D, delta_norm):
    """Eq. 3 / Thm 3.1 (coupling): S^-1/2 (p - <p>) is N(0, I).  KS on the delta direction (the only
    direction the reflection acts on) and on a random orthogonal direction; means and variances too."""
    n = 12000
    _, z, e = _mc_transport(D, delta_norm, n, seed=100 + D)
    proj = z @ e
    assert stats.kstest(proj, "norm").pvalue > 1e-3
    rng = np.random.default_rng(5)
    o = rng.standard_normal(D)
    o -= (o @ e) * e
    o /= np.linalg.norm(o)
    assert stats.kstest(z @ o, "norm").pvalue > 1e-3
    assert np.all(np.abs(z.mean(0)) < 5 / np.sqrt(n))
    assert np.all(np.abs(z.var(0) - 1) < 6 * np.sqrt(2 / n))


def test_draft_equal_target_always_accepts():
    """delta = 0 gives log ratio 0 and acceptance for every u in (0, 1] (Eq. 5; Eq. 6 gives erf(0) = 0)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        mu = rng.standard_normal(4)
        sig = rng.uniform(0.1, 1, 4)
        pd = mu + sig * rng.standard_normal(4)
        acc, p, lr = O.transport(sig, 1.0, pd, mu, mu)
        assert acc and lr == 0.0 and np.array_equal(p, pd)


def test_rejected_sample_is_householder_reflection():
    """On rejection, z -> z - 2 (z.delta / delta.delta) delta preserves |z| and flips the delta component."""
    rng = np.random.default_rng(3)
    D = 9
    sig = rng.uniform(0.5, 1.5, D)
    mu_t = rng.standard_normal(D)
    mu_d = mu_t + sig * rng.standard_normal(D)
    found = 0
    for _ in range(400):
        pd = mu_d + sig * rng.standard_normal(D)
        acc, p, _ = O.transport(sig, 1.0, pd, mu_d, mu_t)
        if acc:
            continue
        found += 1
        z = (pd - mu_d) / sig
        zr = (p - mu_t) / sig
        dl = (mu_d - mu_t) / sig
        assert np.linalg.norm(zr) == pytest.approx(np.linalg.norm(z), rel=1e-12)
        assert zr @ dl == pytest.approx(-(z @ dl), rel=1e-10, abs=1e-12)
    assert found > 20


def test_transport_terms_give_the_log_ratio_in_closed_form():
    """Eq. 5: with z = S^-1/2 (p~ - <p~>) and delta = S^-1/2 (<p~> - <p>), the log density ratio of the two
    Gaussians at p~ is -z.delta - |delta|^2/2.  The oracle forms log r from the two Gaussian exponents and the
    sums z.delta, delta.delta separately; scipy's densities fix both."""
    rng = np.random.default_rng(4)
    for D in (1, 3, 12, 96):
        sig = rng.uniform(0.5, 2.0, D)
        mu_d, mu_t = rng.standard_normal(D), rng.standard_normal(D)
        pd = mu_d + sig * rng.standard_normal(D)
        acc, p, lr, zd, dd = O.transport_terms(sig, 0.5, pd, mu_d, mu_t)
        logpdf = stats.norm.logpdf(pd, mu_t, sig).sum() - stats.norm.logpdf(pd, mu_d, sig).sum()
        assert lr == pytest.approx(logpdf, rel=1e-12, abs=1e-12)
        assert -zd - 0.5 * dd == pytest.approx(logpdf, rel=1e-12, abs=1e-12)
        # |delta|^2 is the squared Mahalanobis distance of the two means; z.delta its projection
        assert dd == pytest.approx(float(np.sum(((mu_d - mu_t) / sig) ** 2)), rel=1e-13)
        assert acc == (np.log(0.5) <= min(0.0, logpdf))
        assert np.array_equal(p, O.transport(sig, 0.5, pd, mu_d, mu_t)[1])
