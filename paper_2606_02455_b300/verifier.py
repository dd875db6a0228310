"""The pipelined verifier protocol of Alg. 2 (host side): a producer-consumer loop in which the draft proposes steps
one at a time, each step is verified asynchronously by the next idle target worker, and results may return out of
submission order.

State (the verifier state of Alg. 2):
  EP  eligible_pending        {id: y'}   submitted, not returned, not flushed
  CV  conditionally_verified  {id: x'}   returned, not flushed, some predecessor not yet final
  V   verified                [(x, id)]  final, in order; V[0] = (x0, 0)

Per returned step (y', x', id'):
  - if id' is not in EP it was flushed by an upstream rejection: ignore it;
  - else move it from EP to CV (accepted or not);
  - if x' != y' (rejected): drop every id > id' from EP and CV and roll the draft back to x';
  - then move the smallest id of CV to V while it is smaller than every id still in EP.

Every entry appended to V was drawn from the target kernel given the entry before it (Thm. D.2 of the paper's
appendix), so V is a target-distributed trajectory whatever the return order.  On one GPU this implementation runs
the synchronous window form (Alg. 1) and its pipelined single-GPU variant (lsd_set_pipelining); this module is the
asynchronous form for a pool of target workers (threads here, one per device in a multi-device pool).

Failure detection: a worker that raises ends the run with WorkerError; a worker that does not return within
`timeout` seconds ends it with TimeoutError (no result of a failed run is committed past what V already holds).
"""
from __future__ import annotations

import concurrent.futures as cf
import time
from dataclasses import dataclass, field
from typing import Any, Callable, Dict, List, Optional, Tuple


class WorkerError(RuntimeError):
    pass


@dataclass
class VerifierState:
    """EP, CV and V of Alg. 2, with the counters the tests read."""
    V: List[Tuple[Any, int]]
    EP: Dict[int, Any] = field(default_factory=dict)
    CV: Dict[int, Any] = field(default_factory=dict)
    next_id: int = 1
    ignored: int = 0       # returns of flushed steps
    rejections: int = 0

    def submit(self, y_new) -> int:
        """Registers a new draft step as eligible-pending and returns its id."""
        sid = self.next_id
        self.EP[sid] = y_new
        self.next_id += 1
        return sid

    def process(self, y_new, x_new, sid: int, rejected: bool) -> Optional[Any]:
        """One returned step.  Returns the state the draft rolls back to on a rejection, else None."""
        if sid not in self.EP:          # flushed by an upstream rejection
            self.ignored += 1
            return None
        del self.EP[sid]
        self.CV[sid] = x_new
        rollback = None
        if rejected:
            self.rejections += 1
            for k in [k for k in self.EP if k > sid]:
                del self.EP[k]
            for k in [k for k in self.CV if k > sid]:
                del self.CV[k]
            rollback = x_new
        while self.CV and min(self.CV) < min(self.EP, default=float("inf")):
            k = min(self.CV)
            self.V.append((self.CV.pop(k), k))
        return rollback


def run_pipelined(x0, n_steps: int, draft_step: Callable, verify_step: Callable, n_workers: int,
                  timeout: float = 30.0, poll: float = 1e-4) -> VerifierState:
    """Alg. 2's main loop until V holds n_steps + 1 states.

    draft_step(y) -> y'            proposes the next draft state (synchronous, in the main loop)
    verify_step(y, y', sid) -> (x', rejected)
                                   the reflection-coupled target state of y' given y (runs on a worker)

    As in Alg. 2, waiting for an idle worker does not process returns: the new step is submitted first (its
    draft base is the current y), and the returns are processed after it, so a rejection flushes it too.
    """
    st = VerifierState(V=[(x0, 0)])
    y = x0
    pending: Dict[cf.Future, Tuple[Any, int, float]] = {}
    pool = cf.ThreadPoolExecutor(max_workers=n_workers)
    try:
        while len(st.V) < n_steps + 1:
            y_new = draft_step(y)
            # fetch_idle_worker: block (bounded) while every worker is busy
            while sum(not f.done() for f in pending) >= n_workers:
                _check_timeout(pending, timeout)
                time.sleep(poll)
            sid = st.submit(y_new)
            pending[pool.submit(verify_step, y, y_new, sid)] = (y_new, sid, time.monotonic())
            y = y_new
            # process_new_returns: everything that has returned, in whatever order
            for f in [f for f in pending if f.done()]:
                y_sub, sid_r, _ = pending.pop(f)
                exc = f.exception()
                if exc is not None:
                    raise WorkerError("target worker failed on step %d: %r" % (sid_r, exc))
                x_new, rejected = f.result()
                rb = st.process(y_sub, x_new, sid_r, bool(rejected))
                if rb is not None:
                    y = rb
            _check_timeout(pending, timeout)
    finally:
        pool.shutdown(wait=False, cancel_futures=True)
    del st.V[n_steps + 1:]
    return st


def _check_timeout(pending, timeout):
    running = [t0 for f, (_, _, t0) in pending.items() if not f.done()]
    if running and time.monotonic() - min(running) > timeout:
        raise TimeoutError("a target worker did not return within %.1f s" % timeout)
