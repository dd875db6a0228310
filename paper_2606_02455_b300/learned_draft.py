"""The learned-draft experiment of the 32-atom workload: frames, training, and the window-length sweep.

    python -m paper_2606_02455_b300.learned_draft [--frames 50000] [--rounds 2] [--K 4 8 16 32 64] [--steps 10000]

1. Equilibrates the 32-atom LJ + MLP target with plain target Langevin.
2. Collects target-labelled frames (q_mid_j, F_target(q_mid_j)) from the method's own LSD trajectories with the
   learned draft (LJ + MLP 9->32->1 on 8 radial basis functions, BF16 inference, starting near the pure pair draft):
   `rounds` rounds of frames/rounds frames each, every round followed by force-matching training (Adam on
   mean |F~ - F_target|^2 over all frames so far, the library's double-backward kernels), so later rounds draft
   with the improved network.
3. For each K: `steps` committed LSD steps with the LJ draft and with the trained learned draft, and `steps` plain
   target steps, from the same equilibrated state, timed with CUDA events on the library's stream: acceptance
   (1 - rejections / committed), per-step rejection rate <beta> over tested steps, ns/day, speedup over plain.

Prints one JSON object.  Every kernel runs in the CUDA library; this module only drives it.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import lsd, workloads as W

NS_PER_DAY = 86400.0 * 1e-6


def _stream(h):
    """A stream of the caller's own for the handle (not the legacy default stream, which would hand the library
    its own non-blocking stream); set before any warm-up, since a new stream rebuilds the handle's graphs."""
    import torch
    s = torch.cuda.Stream()
    h.set_stream(s)
    return s


def _timed(s, fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def _lsd_rate(w, draft, weights, q0, p0, n0, steps, pipelined=True):
    h = lsd.LSD(w.system, draft, w.target, w.integ)
    s = _stream(h)
    if weights is not None:
        h.set_draft_weights(weights)
    h.set_state(q0, p0, n0)
    h.set_pipelining(pipelined)
    h.step(w.integ.K)                        # warm-up: graphs built, first window drafted
    h.set_state(q0, p0, n0)
    a = h.stats()
    sec = _timed(s, lambda: h.step(steps))
    b = h.stats()
    h.close()
    committed = b["committed"] - a["committed"]
    rejected = b["rejected"] - a["rejected"]
    return {"ns_per_day": committed * w.integ.dt / sec * NS_PER_DAY, "acceptance": 1.0 - rejected / committed,
            "beta": rejected / committed, "committed_per_window": committed / max(b["windows"] - a["windows"], 1),
            "mean_delta": (b["sum_delta"] - a["sum_delta"]) / committed, "us_per_step": sec / committed * 1e6}


def run(frames=50000, rounds=2, Ks=(4, 8, 16, 32, 64), steps=10000, iters=1500, lr=3e-3, frames_per_iter=512,
        equil=2000, K_collect=8):
    w = W.config3(K_collect)
    s = w.system
    h = lsd.LSD(s, w.draft, w.target, w.integ)
    h.plain_step(equil)
    q0, p0, n0 = h.get_state()
    h.set_frame_capture(frames)
    log = []
    loss0 = None
    for r in range(rounds):
        want = (r + 1) * frames // rounds
        st0 = h.stats()
        while h.frame_count() < want:
            h.step(K_collect * 64)
        st1 = h.stats()
        if loss0 is None:
            loss0 = h.train_draft(1, 0.0, frames_per_iter)   # loss of the starting network (no update)
        loss = h.train_draft(iters, lr, frames_per_iter)
        log.append({"round": r, "frames": h.frame_count(),
                    "beta_while_collecting": (st1["rejected"] - st0["rejected"]) / max(st1["committed"] - st0["committed"], 1),
                    "loss_after": loss})
    trained = h.get_draft_weights()
    h.close()
    lj = W.Potential(lj_eps=w.draft.lj_eps, lj_sigma=w.draft.lj_sigma, lj_cutoff=w.draft.lj_cutoff)
    rows = []
    for K in Ks:
        wk = W.config3(K)
        r_lj = _lsd_rate(wk, lj, None, q0, p0, n0, steps)
        r_ln = _lsd_rate(wk, wk.draft, trained, q0, p0, n0, steps)
        hp = lsd.LSD(s, lj, wk.target, wk.integ)
        sp = _stream(hp)
        hp.set_state(q0, p0, n0)
        hp.plain_step(8)
        hp.set_state(q0, p0, n0)
        t_plain = _timed(sp, lambda: hp.enqueue_plain(steps))
        hp.close()
        plain = steps * wk.integ.dt / t_plain * NS_PER_DAY
        rows.append({"K": K, "lj": r_lj, "learned": r_ln, "plain_ns_per_day": plain,
                     "speedup_lj": r_lj["ns_per_day"] / plain, "speedup_learned": r_ln["ns_per_day"] / plain})
    return {"workload": "learned_draft_32atoms", "frames": frames, "rounds": log, "loss_start": loss0,
            "train": {"iters_per_round": iters, "lr": lr, "frames_per_iter": frames_per_iter},
            "steps_per_K": steps, "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--frames", type=int, default=50000)
    ap.add_argument("--rounds", type=int, default=2)
    ap.add_argument("--K", type=int, nargs="+", default=[4, 8, 16, 32, 64])
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--lr", type=float, default=3e-3)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.frames, a.rounds, tuple(a.K), a.steps, a.iters, a.lr)))


if __name__ == "__main__":
    main()
