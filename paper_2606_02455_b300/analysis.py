"""Rejection-law and speedup-bound analysis of Langevin speculative dynamics (host side, no GPU).

Everything here is the paper's analysis restated as functions, plus the one-GPU window model this
implementation runs:

- rejection law (Eq. 6): a verified step is rejected with probability erf(|delta| / sqrt(8));
- scaling law (Eq. 9): the mean rejection rate <beta>(N, tau, dt, T) ~ erf(sqrt(N tau dt / T) eps) with one
  constant eps per draft/target pair, fitted from one measurement and used to extrapolate;
- speedup bounds: the pipelined bound 1 / (c + <beta>) (Eq. 8, Prop. 3.2) and the synchronous bound
  F_sync(L) = (1 - a^(L+1)) / ((1 - a)(L c + 1)) with a = 1 - <beta> (the lookahead comparison of App. D);
- the one-GPU synchronous window of this implementation, in which the K target evaluations of a window are one
  batched launch instead of K parallel target models: a window of K steps commits (1 - a^K) / (1 - a) steps on
  average (the accepted prefix plus the reflected step) and costs K t_draft + t_verify(K), so the throughput
  against plain target Langevin is F_window(K) = t_plain (1 - a^K) / ((1 - a)(K t_draft + t_verify(K)));
- the same window verified in stages of S steps (the next stage runs only while every step so far was accepted):
  stage s runs with probability a^(s S) and drafts and verifies min(S, K - s S) steps, so a window runs
  sum_s a^(s S) stages and verifies sum_s a^(s S) min(S, K - s S) steps on average, and commits as many steps as
  the one-pass window.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

import numpy as np
from scipy.special import erf, erfinv


def rejection_probability(delta_norm):
    """Eq. 6: probability that reflectionVerify rejects a step whose draft and target momentum Gaussians are
    |delta| apart in Mahalanobis distance."""
    return erf(np.asarray(delta_norm, dtype=np.float64) / math.sqrt(8.0))


def expected_rejections(delta_norms: Iterable[float]) -> float:
    """Expected number of rejections over verified steps with the given |delta| (the sum of Eq. 6)."""
    return float(np.sum(rejection_probability(np.fromiter(delta_norms, dtype=np.float64))))


def scaling_argument(n_atoms, tau_fs, dt_fs, temperature_k):
    """The argument of Eq. 9 without eps: sqrt(N tau dt / T)."""
    return np.sqrt(np.asarray(n_atoms, np.float64) * tau_fs * dt_fs / temperature_k)


def fit_scaling_eps(beta, n_atoms, tau_fs, dt_fs, temperature_k) -> float:
    """Inverts Eq. 9 for eps from one measured mean rejection rate <beta> in (0, 1)."""
    if not 0.0 < beta < 1.0:
        raise ValueError("the mean rejection rate must lie in (0, 1)")
    return float(erfinv(beta) / scaling_argument(n_atoms, tau_fs, dt_fs, temperature_k))


def predict_beta(eps, n_atoms, tau_fs, dt_fs, temperature_k):
    """Eq. 9: the mean rejection rate at another (N, tau, dt, T) for the same draft/target pair."""
    return erf(scaling_argument(n_atoms, tau_fs, dt_fs, temperature_k) * eps)


def speedup_async(beta, c):
    """Eq. 8: the pipelined speedup bound 1 / (c + <beta>)."""
    return 1.0 / (np.asarray(c, np.float64) + np.asarray(beta, np.float64))


def speedup_sync(beta, c, lookahead):
    """The synchronous speedup with lookahead L (App. D, after Leviathan et al.): (1 - a^(L+1)) / ((1 - a)(L c + 1)),
    a = 1 - <beta>; its a -> 1 limit is (L + 1) / (L c + 1)."""
    a = 1.0 - np.asarray(beta, np.float64)
    L = np.asarray(lookahead, np.float64)
    geo = np.where(np.isclose(a, 1.0), L + 1.0, (1.0 - a ** (L + 1.0)) / np.where(np.isclose(a, 1.0), 1.0, 1.0 - a))
    return geo / (L * c + 1.0)


def expected_committed(beta, K):
    """Expected committed steps of one synchronous window of K drafted steps with i.i.d. rejections at rate <beta>:
    the accepted prefix plus the reflected step, sum_{j=1..K} a^(j-1) = (1 - a^K) / (1 - a)."""
    a = 1.0 - np.asarray(beta, np.float64)
    K = np.asarray(K, np.float64)
    return np.where(np.isclose(a, 1.0), K, (1.0 - a ** K) / np.where(np.isclose(a, 1.0), 1.0, 1.0 - a))


@dataclass
class WindowCosts:
    """Measured costs of the one-GPU window: t_draft per drafted step, t_verify(K) = verify_fixed + verify_per_step K
    for the batched verification of K steps, and t_plain per plain target step (all in the same unit)."""
    t_draft: float
    verify_fixed: float
    verify_per_step: float
    t_plain: float

    def window(self, K):
        return np.asarray(K, np.float64) * (self.t_draft + self.verify_per_step) + self.verify_fixed

    @property
    def c(self) -> float:
        """The paper's draft-to-target cost ratio per step."""
        return self.t_draft / self.t_plain


def speedup_window(beta, costs: WindowCosts, K):
    """Throughput of the one-GPU synchronous window against plain target Langevin: expected committed steps per
    window time, times t_plain."""
    return expected_committed(beta, K) * costs.t_plain / costs.window(K)


def best_window(beta, costs: WindowCosts, K_max: int = 256) -> Tuple[int, float]:
    """The window length K in 1..K_max with the largest predicted speedup, and that speedup."""
    Ks = np.arange(1, K_max + 1)
    s = speedup_window(beta, costs, Ks)
    i = int(np.argmax(s))
    return int(Ks[i]), float(s[i])


def fit_verify_costs(K_values: Sequence[int], t_verify: Sequence[float]) -> Tuple[float, float]:
    """Least-squares line t_verify(K) = fixed + per_step K through measured batched verification times."""
    A = np.stack([np.ones(len(K_values)), np.asarray(K_values, np.float64)], axis=1)
    (fixed, per), *_ = np.linalg.lstsq(A, np.asarray(t_verify, np.float64), rcond=None)
    return float(fixed), float(per)


def summarize(beta: float, costs: WindowCosts, K: int) -> Dict[str, float]:
    """The bounds and the window model at one operating point, for reports."""
    kb, sb = best_window(beta, costs)
    return {
        "c": costs.c,
        "beta": beta,
        "speedup_async_bound": float(speedup_async(beta, costs.c)),
        "speedup_sync_bound": float(speedup_sync(beta, costs.c, K)),
        "expected_committed_per_window": float(expected_committed(beta, K)),
        "speedup_window_model": float(speedup_window(beta, costs, K)),
        "best_K_window_model": kb,
        "speedup_at_best_K": sb,
    }


def expected_stages(beta, K: int, S: int) -> float:
    """Mean number of stages a window of K steps verified in stages of S runs, with i.i.d. rejections at rate <beta>:
    stage s (0-based) runs when the s S steps before it were all accepted, with probability a^(s S)."""
    a = 1.0 - float(beta)
    S = min(int(S), int(K))
    return float(sum(a ** (s * S) for s in range(-(-int(K) // S))))


def expected_verified(beta, K: int, S: int) -> float:
    """Mean number of steps such a window drafts and verifies: sum_s a^(s S) min(S, K - s S).  S = 1 gives the
    expected committed steps (no step past the first rejection is verified); S >= K gives K."""
    a = 1.0 - float(beta)
    S = min(int(S), int(K))
    return float(sum(a ** (s * S) * min(S, int(K) - s * S) for s in range(-(-int(K) // S))))


@dataclass
class StageCosts:
    """Costs of the staged window: per drafted and verified step (draft step plus one verified configuration), per
    stage (its launches' fixed part) and per window (lists, the first stage's extras); t_plain per plain step."""
    per_step: float
    per_stage: float
    per_window: float
    t_plain: float


def speedup_staged(beta, costs: StageCosts, K: int, S: int) -> float:
    """Throughput of staged windows against plain target Langevin: expected committed steps per expected window
    time, times t_plain."""
    t = (costs.per_window + expected_stages(beta, K, S) * costs.per_stage +
         expected_verified(beta, K, S) * costs.per_step)
    return float(expected_committed(beta, K)) * costs.t_plain / t


def best_stage_length(beta, costs: StageCosts, K: int) -> Tuple[int, float]:
    """The stage length S in 1..K with the largest predicted speedup, and that speedup."""
    best = max(((speedup_staged(beta, costs, K, S), S) for S in range(1, int(K) + 1)))
    return best[1], best[0]
