"""Window-length sweep on one GPU: measures, for each K, the drafted-step time, the batched verification time, the
per-step rejection rate and the LSD throughput; fits t_verify(K) = a + b K; and compares the best K predicted by
the window model of paper_2606_02455_b300.analysis with the measured one.

    python -m paper_2606_02455_b300.ksweep --config 2 --K 4 8 16 32 64 --windows 60

Prints one JSON object.  Inputs are the synthetic workloads of workloads.py, equilibrated with plain target steps.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import analysis as A
from . import workloads as W

NS_PER_DAY = 86400.0 * 1e-6   # fs of simulated time per second -> ns per day


def _measure(cfg: int, K: int, windows: int, equil: int):
    import torch
    from . import lsd
    w = W.CONFIGS[cfg](K)
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    # a stream of its own (set before the warm-up: a new stream rebuilds the graphs): the legacy default stream
    # would hand the library its own non-blocking stream, which the events below would not see
    stream = torch.cuda.Stream()
    h.set_stream(stream)
    h.plain_step(equil)
    for _ in range(3):
        h.profile_window()
    ph = {}
    for _ in range(10):
        for k, v in h.profile_window().items():
            ph[k] = ph.get(k, 0.0) + v / 10
    t_draft = ph["draft"] * 1e-3 / K
    t_verify = sum(v for k, v in ph.items() if k != "draft") * 1e-3
    h.enqueue_windows(2)   # graphs of the window loop built before the timed region
    torch.cuda.synchronize()
    st0 = h.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.enqueue_windows(windows)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    st1 = h.stats()
    committed = st1["committed"] - st0["committed"]
    verified = st1["verified"] - st0["verified"]
    # per tested step: every committed step was tested in order; steps after a window's first rejection were not
    beta = (st1["rejected"] - st0["rejected"]) / max(committed, 1)
    n_plain = 200
    e0.record(stream)
    h.enqueue_plain(n_plain)
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) * 1e-3 / n_plain
    h.close()
    return dict(K=K, t_draft=t_draft, t_verify=t_verify, beta=beta, committed=committed, verified=verified, seconds=sec,
                ns_per_day=committed * w.integ.dt / sec * NS_PER_DAY, t_plain=t_plain,
                plain_ns_per_day=w.integ.dt / t_plain * NS_PER_DAY)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--K", type=int, nargs="+", default=[4, 8, 16, 32, 64])
    ap.add_argument("--windows", type=int, default=60)
    ap.add_argument("--equil", type=int, default=300)
    args = ap.parse_args(argv)
    rows, failed = [], {}
    for K in args.K:
        try:
            rows.append(_measure(args.config, K, args.windows, args.equil))
        except RuntimeError as e:   # reported, not fatal: the other window lengths still run
            failed[K] = str(e)
    if len(rows) < 2:
        print(json.dumps({"config": args.config, "failed": failed}))
        return
    fixed, per = A.fit_verify_costs([r["K"] for r in rows], [r["t_verify"] for r in rows])
    t_draft = float(np.mean([r["t_draft"] for r in rows]))
    t_plain = float(np.mean([r["t_plain"] for r in rows]))
    tested = sum(r["committed"] for r in rows)
    beta = float(sum(r["beta"] * r["committed"] for r in rows) / max(tested, 1))
    costs = A.WindowCosts(t_draft=t_draft, verify_fixed=max(fixed, 0.0), verify_per_step=per, t_plain=t_plain)
    k_best, s_best = A.best_window(beta, costs, K_max=max(args.K) * 2)
    for r in rows:
        r["speedup_measured"] = r["ns_per_day"] / r["plain_ns_per_day"]
        r["speedup_model"] = float(A.speedup_window(r["beta"], costs, r["K"]))
    measured_best = max(rows, key=lambda r: r["ns_per_day"])["K"]
    out = {"config": args.config, "fit": {"t_draft_us": t_draft * 1e6, "verify_fixed_us": fixed * 1e6,
                                          "verify_per_step_us": per * 1e6, "t_plain_us": t_plain * 1e6,
                                          "beta": beta, "c": costs.c},
           "bounds": A.summarize(beta, costs, int(np.median(args.K))),
           "best_K_predicted": k_best, "speedup_predicted_at_best": s_best, "best_K_measured": measured_best,
           "rows": [{k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()} for r in rows],
           "failed": failed}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
