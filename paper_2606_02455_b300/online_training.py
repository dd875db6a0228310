"""Online retraining of the learned draft on a dense workload (the 32,768-atom configuration by default).

    python -m paper_2606_02455_b300.online_training [--config 5] [--every 200] [--rounds 3] [--iters 40]
                                                    [--frames 128] [--fpi 16] [--windows 20] [--K 0]

1. Equilibrates with plain target Langevin and times `windows` windows with the pair (LJ) draft.
2. Starts LSD with the learned draft (LJ + MLP on 8 radial basis functions per species, BF16 inference, started
   near the pair draft), captures the target-verified frames of every window into a ring of `frames` frames, and
   retrains the draft online every `every` accepted steps (lsd_set_online_training: `iters` Adam steps of `fpi`
   frames each, the large-frame force-matching path), for `rounds` retrainings.
3. Times `windows` windows with the retrained draft, and `windows` x K plain target steps.

Reports per-step rejection rates, committed steps per window, ns/day, the retrainings' losses and the time spent
per phase.  Every kernel runs in the CUDA library; this module only drives it.  Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import time

from . import lsd, workloads as W

NS_PER_DAY = 86400.0 * 1e-6


def _stream(h):
    import torch
    s = torch.cuda.Stream()
    h.set_stream(s)
    return s


def _timed_windows(h, s, n, dt):
    import torch
    a = h.stats()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    h.enqueue_windows(n)
    e1.record(s)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    b = h.stats()
    c = b["committed"] - a["committed"]
    rj = b["rejected"] - a["rejected"]
    return {"ns_per_day": c * dt / sec * NS_PER_DAY, "beta": rj / max(c, 1), "committed_per_window": c / n,
            "ms_per_window": sec * 1e3 / n, "mean_delta": (b["sum_delta"] - a["sum_delta"]) / max(c, 1)}


def run(cfg=5, every=200, rounds=3, iters=40, frames=128, fpi=16, windows=20, K=0, equil=200):
    import torch
    w = W.CONFIGS[cfg](K) if K else W.CONFIGS[cfg]()
    s, dt = w.system, w.integ.dt
    out = {"workload": w.name, "every_accepted": every, "iters": iters, "frames": frames, "frames_per_iter": fpi}
    # pair draft and plain target
    h = lsd.LSD(s, w.draft, w.target, w.integ)
    st = _stream(h)
    h.plain_step(equil)
    q0, p0, n0 = h.get_state()
    h.set_pipelining(True)
    h.enqueue_windows(2)
    out["lj"] = _timed_windows(h, st, windows, dt)
    h.set_state(q0, p0, n0)
    h.plain_step(2)
    h.set_state(q0, p0, n0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_plain = max(32, windows * 4)
    e0.record(st)
    h.enqueue_plain(n_plain)
    e1.record(st)
    torch.cuda.synchronize()
    out["plain_ns_per_day"] = n_plain * dt / (e0.elapsed_time(e1) * 1e-3) * NS_PER_DAY
    h.close()
    # learned draft, online retraining
    draft = W.learned_draft(w.target, s.n_species)
    h = lsd.LSD(s, draft, w.target, w.integ)
    st = _stream(h)
    h.set_state(q0, p0, n0)
    h.set_pipelining(True)
    h.enqueue_windows(2)
    out["learned_start"] = _timed_windows(h, st, windows, dt)
    h.set_frame_capture(frames)
    h.set_online_training(every, n_iters=iters, lr=3e-3, frames_per_iter=fpi)
    t0 = time.perf_counter()
    a = h.stats()
    log = []
    while h.online_status()[0] < rounds:
        b0 = h.stats()
        h.step(max(every // 4, 8))
        b1 = h.stats()
        n, loss = h.online_status()
        if not log or log[-1]["retrains"] != n:
            log.append({"retrains": n, "loss": loss, "step": b1["step"],
                        "beta_segment": (b1["rejected"] - b0["rejected"]) / max(b1["committed"] - b0["committed"], 1)})
    b = h.stats()
    out["online"] = {"wall_s": time.perf_counter() - t0, "committed": b["committed"] - a["committed"],
                     "windows": b["windows"] - a["windows"], "log": log}
    h.set_online_training(0)
    out["learned_trained"] = _timed_windows(h, st, windows, dt)
    h.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--every", type=int, default=200)
    ap.add_argument("--rounds", type=int, default=3)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--frames", type=int, default=128)
    ap.add_argument("--fpi", type=int, default=16)
    ap.add_argument("--windows", type=int, default=20)
    ap.add_argument("--K", type=int, default=0)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.config, a.every, a.rounds, a.iters, a.frames, a.fpi, a.windows, a.K)))


if __name__ == "__main__":
    main()
