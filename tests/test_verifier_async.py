"""T12: the host-side bookkeeping of the pipelined protocol (Alg. 2) among CPU threads.

A Gaussian AR(1) chain stands in for the dynamics: target x' ~ N(a x + b_t, s^2 I), draft y' ~ N(a x + b_d, s^2 I),
coupled by the reflection map of Eq. 5 (the oracle's transport).  Workers sleep a random time before returning, so
results arrive out of submission order.  Checked: every verified state was drawn from the target kernel given the
verified state before it (recursive correctness, by provenance); flushed results are ignored; the run halts with
n + 1 states; the final states follow the target chain's closed-form law, not the draft's; a worker that raises, or
that does not return within the bound, ends the run with an error instead of a trajectory."""
import threading
import time

import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import verifier as VF

A, S, B_T, B_D, DIM = 0.8, 1.0, 0.0, 0.45, 24


def _chain(seed, sleep_max=1e-3, fail_sid=None, hang_sid=None, hang=2.0, bias=B_D):
    rng_draft = np.random.default_rng(seed)
    tag = {"n": 0}
    base_of = {}
    lock = threading.Lock()

    def draft_step(y):
        tag["n"] += 1
        return {"v": A * y["v"] + bias + S * rng_draft.standard_normal(DIM), "tag": ("draft", tag["n"])}

    def verify_step(y, y_new, sid):
        with lock:
            base_of[sid] = y["tag"]
        r = np.random.default_rng([seed, sid])
        if sid == fail_sid:
            raise RuntimeError("injected worker failure")
        time.sleep(hang if sid == hang_sid else r.uniform(0, sleep_max))
        mu_d = A * y["v"] + bias
        mu_t = A * y["v"] + B_T
        acc, p, _ = O.transport(np.full(DIM, S), r.uniform(1e-12, 1.0), y_new["v"], mu_d, mu_t)
        if acc:
            return y_new, False                  # accepted: the draft's own state
        return {"v": p, "tag": ("reflected", sid)}, True

    x0 = {"v": np.zeros(DIM), "tag": "x0"}
    return x0, draft_step, verify_step, base_of


def test_out_of_order_returns_keep_recursive_correctness():
    x0, draft, verify, base_of = _chain(1)
    st = VF.run_pipelined(x0, 40, draft, verify, n_workers=6)
    assert len(st.V) == 41 and st.V[0][1] == 0
    ids = [sid for _, sid in st.V]
    assert ids == sorted(ids) and len(set(ids)) == len(ids)
    for k in range(1, len(st.V)):
        x, sid = st.V[k]
        assert base_of[sid] == st.V[k - 1][0]["tag"], k      # drawn given the previous verified state
    assert st.rejections > 0 and st.ignored > 0 and not st.CV


def test_verified_states_follow_the_target_chain():
    n, runs = 12, 60
    finals = []
    for seed in range(runs):
        x0, draft, verify, _ = _chain(100 + seed, sleep_max=3e-4)
        finals.append(VF.run_pipelined(x0, n, draft, verify, n_workers=4).V[-1][0]["v"])
    x = np.concatenate(finals)
    mean_t = B_T * (1 - A ** n) / (1 - A)
    mean_d = B_D * (1 - A ** n) / (1 - A)
    var = S ** 2 * (1 - A ** (2 * n)) / (1 - A ** 2)
    se = np.sqrt(var / x.size)
    assert abs(x.mean() - mean_t) < 5 * se
    assert abs(mean_d - mean_t) > 20 * se                      # the draft chain would be detected
    assert x.var() / var == pytest.approx(1.0, abs=5 * np.sqrt(2.0 / x.size))


def test_single_worker_is_the_sequential_protocol():
    x0, draft, verify, base_of = _chain(7, sleep_max=0.0)
    st = VF.run_pipelined(x0, 25, draft, verify, n_workers=1)
    # the next step is submitted before a return is processed (Alg. 2), so a rejection flushes at most that one
    assert len(st.V) == 26 and st.ignored <= st.rejections
    for k in range(1, 26):
        assert base_of[st.V[k][1]] == st.V[k - 1][0]["tag"]


def test_worker_failure_is_detected():
    x0, draft, verify, _ = _chain(3, fail_sid=5)
    with pytest.raises(VF.WorkerError):
        VF.run_pipelined(x0, 30, draft, verify, n_workers=3)


def test_worker_that_does_not_return_times_out():
    # draft equal to target: nothing is rejected, so the hung step is never flushed and holds V back
    x0, draft, verify, _ = _chain(4, hang_sid=4, hang=2.0, bias=B_T)
    t0 = time.monotonic()
    with pytest.raises(TimeoutError):
        VF.run_pipelined(x0, 30, draft, verify, n_workers=3, timeout=0.3)
    assert time.monotonic() - t0 < 1.5
