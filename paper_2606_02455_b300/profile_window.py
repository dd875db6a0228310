"""Runs LSD windows of a benchmark configuration, for profilers (ncu) and quick timing.

    python -m paper_2606_02455_b300.profile_window --config 4 [--K 32] [--windows 2] [--equil 0] [--pipelined]
                                                   [--plain 0] [--learned] [--stages S]

Builds one handle for the configuration (window length K overridable, to keep a profiled footprint small),
optionally runs `equil` plain target steps, then `windows` windows through lsd_enqueue_windows on the handle's
stream, prints the per-phase CUDA-event times of one more window (lsd_profile_window) and the run's counters, and
then runs `plain` plain target steps in one call.  --learned drafts with the learned draft (LJ + MLP on radial
basis functions, untrained weights: the kernels' cost does not depend on them); --stages S verifies the windows in
stages of S steps (lsd_set_window_stages; the profiled window is then one stage long).  Windows verified in
stages run as graphs with conditional nodes, whose kernel nodes ncu does not profile; --windows 0 --profiles N
issues N stage-shaped windows kernel by kernel instead (the shape the bench's roofline pass times).
The first kernels a handle launches are its set-up (the FP8 and FP32-split calibration runs the MLP once on N
rows); window kernels follow.
"""
from __future__ import annotations

import argparse
import json

from . import lsd, workloads as W


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--K", type=int, default=0, help="window length (0: the configuration's)")
    ap.add_argument("--windows", type=int, default=2)
    ap.add_argument("--equil", type=int, default=0)
    ap.add_argument("--pipelined", action="store_true")
    ap.add_argument("--plain", type=int, default=0, help="plain target steps after the windows (one call)")
    ap.add_argument("--learned", action="store_true", help="the learned draft instead of the configuration's")
    ap.add_argument("--stages", type=int, default=0, help="steps per verification stage (0: one pass)")
    ap.add_argument("--profiles", type=int, default=1,
                    help="profiled windows (lsd_profile_window: kernels issued one by one, no graph)")
    a = ap.parse_args()
    w = W.CONFIGS[a.config](a.K) if a.K else W.CONFIGS[a.config]()
    draft = W.learned_draft(w.target, w.system.n_species) if a.learned else w.draft
    h = lsd.LSD(w.system, draft, w.target, w.integ)
    if a.equil:
        h.plain_step(a.equil)
    h.set_pipelining(a.pipelined)
    h.set_window_stages(a.stages)
    if a.windows:
        h.enqueue_windows(a.windows)
    st = h.stats()
    for _ in range(a.profiles):
        ph = h.profile_window()
    if a.plain:
        h.plain_step(a.plain)
    print(json.dumps({"workload": w.name, "windows": st["windows"], "committed": st["committed"],
                      "phases_ms": {k: round(v, 4) for k, v in ph.items()}, "plain_steps": a.plain}))
    h.close()


if __name__ == "__main__":
    main()
