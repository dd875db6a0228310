"""Benchmark: target-distributed ns/day of LSD on one B300 against plain target Langevin, and acceptance rate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config 2]

A step is one LSD window: K drafted steps (persistent draft kernel), one batched target evaluation on all K*N
atoms (neighbours, descriptors, MLP, adjoint), transport and commit; the window runs as one CUDA graph.
`value` = committed steps x dt / device time, in ns/day, with the state resident in HBM.  L2 is flushed
between timed windows.  `e2e` is the same metric through the public one-call window (lsd_window_host) with the state
copied host->device before and device->host after every window.  The plain-target baseline (the same
kernels, one ABOBA step per graph launch) is timed the same way in the same process.  `roofline` is the
dominant kernel, timed live with CUDA events on the library's stream.  `cpu_baseline` is the FP64 oracle on a
bounded sample of the same workload on the host.

Multi-GPU: the method does not shard on one node here (replicas only): with torchrun each rank runs an
independent replica and `value` sums them over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "target-distributed ns/day vs plain target Langevin on 1 B300; acceptance rate"
NS_PER_DAY = 86400.0 * 1e-6   # steps * dt[fs] / seconds -> ns/day


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
            "fallback"


def _workload(cfg):
    from paper_2606_02455_b300 import workloads as W
    return W.CONFIGS[cfg]()


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce_over_ranks(x, world, op, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _max_over_ranks(x, world, device="cuda"):
    return _reduce_over_ranks(x, world, "max", device)


def _sum_over_ranks(x, world, device="cuda"):
    return _reduce_over_ranks(x, world, "sum", device)


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_seed(base_seed, rank):
    """Replicas only: rank r runs an independent copy of the workload with its own noise key."""
    return base_seed + rank


def whole_job_rate(units_local, seconds_local, world, device="cuda"):
    """Whole-job throughput of independent replicas: the units all ranks processed over the slowest rank's time."""
    return _sum_over_ranks(units_local, world, device) / _max_over_ranks(seconds_local, world, device)


# ------------------------------------------------------------------------------------------------------------------
# roofline of the dominant kernel
# ------------------------------------------------------------------------------------------------------------------

def _lj_pairs_per_atom(w, q):
    """Mean number of LJ partners per atom (r < LJ cutoff, minimum image; every cutoff here is below half the box)
    at positions q: brute force up to 4,096 atoms, the density estimate above."""
    s = w.system
    rc = w.draft.lj_cutoff
    N = s.n_atoms
    if N > 4096:
        return N / float(np.prod(s.box)) * 4.0 / 3.0 * np.pi * rc ** 3
    tot = 0
    for i0 in range(0, N, 512):
        d = q[None, :, :] - q[i0:i0 + 512, None, :]
        d -= s.box * np.round(d / s.box)
        r2 = (d * d).sum(-1)
        tot += int(((r2 < rc * rc) & (r2 > 0)).sum())
    return tot / N


# DRAM bytes (read + write) of one launch, from one ncu capture of the kernel as it is now (the summaries under
# profiles/ give the command); a kernel changed since its capture has no entry here.
NCU_TRAFFIC = {
    ("lj_mlp_angular_256atoms_K16", "draft"): 70144,       # draft_window_cluster_kernel, K = 16
    ("lj_mlp_angular_256atoms_K16", "mlp"): 1419520,       # mlp_tc_kernel<F16x3>, 4096 rows
}


def _algorithmic_work(w, phase, q):
    """Algorithmic work of one launch of a phase, with its bound: (amount, unit, bound, detail).

    mlp:   2 FLOP per multiply-add of the forward chain plus the input-gradient chain (no weight gradient):
           2 * M * sum(d_in * d_out) * 2, M = K N rows.  FP32 targets run it as three TF32 tensor-core
           products per term (3x the algorithmic MACs executed); BF16 targets as one BF16 product.
    draft: per drafted step, every LJ pair within the cutoff costs 8 FLOP of distance and 15 of force
           (gather form: each ordered pair once), plus 24 FP64 FLOP per atom of BOB + A;
           K steps per launch, serial.
    transport: bytes that must cross HBM once per window."""
    s, t, K = w.system, w.target, w.integ.K
    N = s.n_atoms
    M = K * N
    if phase == "mlp":
        d0p = ((s.n_species * t.n_rbf + t.n_ang + s.n_species) + 31) // 32 * 32
        macs = d0p * t.width + (t.n_layers - 1) * t.width * t.width + t.width
        return 2.0 * 2.0 * M * macs, "FLOP", "tensor", {"precision": t.precision, "rows": M}
    if phase == "draft":
        nb = _lj_pairs_per_atom(w, q)
        flop = K * (N * nb * (8 + 15) + N * 24)
        return flop, "FLOP", "alu", {"lj_pairs_per_atom": round(nb, 1), "steps_per_launch": K}
    if phase in ("transport_reduce",):
        return M * 3 * (4 + 4), "B", "hbm", {}
    if phase in ("transport_commit",):
        return N * 3 * (8 + 8 + 4 + 4 + 8 + 8 + 8), "B", "hbm", {}
    return None


def _analysis(st1, st0, rl, K, t_plain_step):
    """The paper's bounds at the measured operating point (paper_2606_02455_b300.analysis): per-step rejection
    rate <beta> = rejections / tested steps (every committed step was tested, in order; steps after a window's
    first rejection are flushed untested), cost ratio c = drafted-step time / plain-step time, the pipelined
    bound 1 / (c + <beta>) (Eq. 8) and the synchronous lookahead-K bound."""
    from paper_2606_02455_b300 import analysis as A
    tested = max(st1["committed"] - st0["committed"], 1)
    beta = (st1["rejected"] - st0["rejected"]) / tested
    ph = rl["phases_ms"]
    t_draft = ph["draft"] * 1e-3 / K
    c = t_draft / t_plain_step
    return {"beta": round(beta, 5), "c": round(c, 5),
            "speedup_async_bound": round(float(A.speedup_async(beta, c)), 3),
            "speedup_sync_bound_K": round(float(A.speedup_sync(beta, c, K)), 3),
            "expected_committed_per_window": round(float(A.expected_committed(beta, K)), 3)}


def roofline(h, w, peaks, peak_kind, q, n_rep=20):
    """Per-phase CUDA-event times of the window (live, on the library's stream), the dominant phase, and its
    achieved rate against the peak that bounds it."""
    phases = None
    for _ in range(3):
        h.profile_window()
    acc = {}
    for _ in range(n_rep):
        ph = h.profile_window()
        for k, v in ph.items():
            acc[k] = acc.get(k, 0.0) + v / n_rep
    phases = acc
    dom = max(phases, key=lambda k: phases[k])
    share = phases[dom] / sum(phases.values())
    work = _algorithmic_work(w, dom, q)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s: 148 SMs x 128 FP32 lanes x FMA
    out = {"kernel": dom, "share": round(share, 3), "ms": round(phases[dom], 5),
           "phases_ms": {k: round(v, 5) for k, v in phases.items()}}
    if work is None:
        out.update({"bound": "alu", "achieved": None, "peak": round(fp32_peak, 1), "unit": "TFLOP/s", "frac": None,
                    "traffic": None, "note": "no algorithmic model for this phase"})
        return out
    amount, unit, bound, detail = work
    sec = phases[dom] * 1e-3
    out.update(detail)
    traffic = NCU_TRAFFIC.get((w.name, dom))
    if bound == "alu":
        ach = amount / sec / 1e12
        out.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                    "frac": round(ach / fp32_peak, 5), "traffic": traffic,
                    "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz" % sm_max})
        if dom == "draft":
            out["us_per_step"] = round(phases[dom] * 1e3 / w.integ.K, 3)
            out["note"] = ("serial chain of K drafted steps in one thread-block cluster (at most 16 SMs); "
                           "latency-bound: the per-step time, not FLOP/s, is the figure of merit")
    elif bound == "tensor":
        ach = amount / sec / 1e12
        bf16 = peaks["bf16_tflops"]
        if w.target.precision in ("bf16", "fp32"):
            # BF16 and the FP16 split of FP32 targets: the FP16 dense rate equals the BF16 one
            pk, src = bf16, "%s bf16 burst (FP16 dense = BF16 dense)" % peak_kind
        else:
            # TF32 dense = bf16 x (1.1 / 2.25), the nominal ratio
            pk, src = bf16 * 1.1 / 2.25, "%s bf16 burst x 1.1/2.25 (nominal TF32:BF16)" % peak_kind
        out.update({"bound": "tensor", "achieved": round(ach, 2), "peak": round(pk, 1), "unit": "TFLOP/s",
                    "frac": round(ach / pk, 5), "traffic": traffic, "peak_source": src})
        if w.target.precision in ("fp32", "fp32-tf32"):
            out["tensor_flop_executed_per_algorithmic"] = 3
    else:
        ach = amount / sec / 1e9
        pk = peaks["hbm_gbs"]
        out.update({"bound": "hbm", "achieved": round(ach, 1), "peak": pk, "unit": "GB/s", "frac": round(ach / pk, 4),
                    "traffic": traffic, "peak_source": peak_kind})
    return out


# ------------------------------------------------------------------------------------------------------------------
# our implementation
# ------------------------------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_2606_02455_b300 import lsd

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = _workload(args.config)
    s = w.system
    s.seed = replica_seed(s.seed, rank)   # independent replicas
    K = w.integ.K
    peaks, peak_kind = _peaks()
    h = lsd.LSD(s, w.draft, w.target, w.integ)
    stream = torch.cuda.Stream()
    h.set_stream(stream)
    # equilibrate with plain target dynamics, then warm up both graphs
    h.plain_step(args.equil)
    q_eq, p_eq, step_eq = h.get_state()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.add_(1.0)

    pipelined = not args.no_pipeline
    h.set_pipelining(pipelined)
    for _ in range(args.warmup):
        h.step(K)
        h.plain_step(1)

    def timed_windows(n):
        """n windows from the equilibrated state, each enqueue bracketed by events, L2 flushed in between."""
        h.set_state(q_eq, p_eq, step_eq)
        a = h.stats()
        _barrier(world)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush_l2()
            ev[k][0].record(stream)
            h.enqueue_windows(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        _barrier(world)
        b = h.stats()
        return (sum(x.elapsed_time(y) for x, y in ev) * 1e-3, b["committed"] - a["committed"],
                b["rejected"] - a["rejected"], b["windows"] - a["windows"], a, b)

    clocks = Clocks(local)
    clocks.start()
    # ---- LSD: `steps` windows (pipelined: each enqueue verifies one window while drafting the next) ----
    t_lsd, committed, rejected, windows, st0, st1 = timed_windows(args.steps)
    if args.only_lsd:
        # profiling mode: the LSD windows alone (no baseline, e2e or roofline pass)
        clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "mode": "only-lsd", "windows": windows, "committed": committed,
                              "ms_per_step": round(t_lsd * 1e3 / args.steps, 5)}), flush=True)
        h.close()
        return
    # ---- the same windows without the draft/verify overlap, for comparison ----
    value_unpipelined = None
    if pipelined:
        h.set_pipelining(False)
        h.step(K)
        t_u, c_u, _, _, _, _ = timed_windows(args.steps)
        value_unpipelined = whole_job_rate(c_u, t_u, world) * w.integ.dt * NS_PER_DAY
        h.set_pipelining(True)
    # ---- plain target Langevin: the same number of steps as committed, one graph launch per step ----
    h.set_state(q_eq, p_eq, step_eq)
    n_plain = max(committed, 16)
    evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_plain)]
    torch.cuda.synchronize()
    for k in range(n_plain):
        flush_l2()
        evp[k][0].record(stream)
        h.enqueue_plain(1)
        evp[k][1].record(stream)
    torch.cuda.synchronize()
    t_plain = sum(a.elapsed_time(b) for a, b in evp) * 1e-3
    clk = clocks.stop()

    t_lsd_max = _max_over_ranks(t_lsd, world)
    value = whole_job_rate(committed, t_lsd, world) * w.integ.dt * NS_PER_DAY
    plain_value = whole_job_rate(n_plain, t_plain, world) * w.integ.dt * NS_PER_DAY

    # ---- e2e: the public one-call window with host buffers (pinned): every window uploads its state, runs,
    # and reads the committed state back ----
    h.set_state(q_eq, p_eq, step_eq)
    state = torch.empty((2, s.n_atoms, 3), dtype=torch.float64, pin_memory=True).numpy()
    pos, mom = state[0], state[1]   # adjacent, as on the device: one copy each way
    pos[:] = q_eq
    mom[:] = p_eq
    n_e2e = args.steps
    step = step_eq
    for _ in range(max(args.warmup, 3)):   # untimed: first-call costs of the one-call path
        step, nc = h.window_host(pos, mom, step)
    stats_a = h.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        step, nc = h.window_host(pos, mom, step)
    t_e2e = time.perf_counter() - t0
    stats_b = h.stats()
    e2e_committed = stats_b["committed"] - stats_a["committed"]
    e2e_val = whole_job_rate(e2e_committed, t_e2e, world) * w.integ.dt * NS_PER_DAY
    D = 3 * s.n_atoms

    rl = roofline(h, w, peaks, peak_kind, pos)
    # this library's kernels per window / pipelined round / plain step, for the handle's configuration
    lc = h.launch_counts()
    launches_per_window = lc["round"] if pipelined else lc["window"]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "ns/day", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_lsd_max * 1e3 / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "dtype_detail": ("FP32 forces and descriptors; MLP %s; FP64 integrator state, z.delta, delta.delta and "
                         "log ratio" % {"fp32": "at FP32 accuracy as three FP16 tensor-core products per term "
                                                "(exact power-of-two scales)",
                                        "fp32-tf32": "at FP32 accuracy as three TF32 tensor-core products per term",
                                        "bf16": "in BF16 on the tensor cores with FP32 accumulation",
                                        "fp8": "in FP32 on the CUDA cores (FP8 not built)",
                                        "fp32-cuda-cores": "in FP32 on the CUDA cores"}[w.target.precision]),
        "data": "synthetic",
        "config": {"workload": w.name, "n_atoms": s.n_atoms, "K": K, "dt_fs": w.integ.dt, "T_K": w.integ.temperature,
                   "gamma_per_fs": w.integ.gamma, "target": "LJ + 0.05 eV tanh(MLP %d->%dx%d->1)" % (
                       s.n_species * w.target.n_rbf + w.target.n_ang + s.n_species, w.target.width,
                       w.target.n_layers),
                   "draft": "LJ", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (256 MB write) between timed windows"},
        "acceptance_rate": round(1.0 - rejected / max(committed, 1), 5),
        "analysis": _analysis(st1, st0, rl, K, t_plain / n_plain),
        "committed_per_window": round(committed / max(windows, 1), 3),
        "plain_target_ns_per_day": round(plain_value, 3),
        "speedup_vs_plain": round(value / plain_value, 3),
        "pipelined": pipelined,
        "value_unpipelined": None if value_unpipelined is None else round(value_unpipelined, 3),
        "plain_ms_per_step": round(t_plain * 1e3 / n_plain, 5),
        "gpu_launches": int(windows * launches_per_window + n_plain * lc["plain"]),
        "e2e": {"value": round(e2e_val, 3), "unit": "ns/day", "h2d_bytes_per_step": 2 * D * 8 + 16,
                "d2h_bytes_per_step": 2 * D * 8 + 32, "calls": "lsd_window_host (pinned host state in and out)"},
        "roofline": rl,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------------------------
# the oracle on the host (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------------------------------

def cpu_baseline(w, seconds):
    from oracle import oracle as O
    s = w.system
    K = w.integ.K
    q, p, step = s.positions.copy(), s.momenta.copy(), 0
    t0 = time.perf_counter()
    committed = 0
    windows = 0
    while time.perf_counter() - t0 < seconds:
        out = O.lsd_window(s, w.draft, w.target, w.integ, s.seed, step, K, q, p)
        q, p = out["q"], out["p"]
        step += out["n_committed"]
        committed += out["n_committed"]
        windows += 1
    dt = time.perf_counter() - t0
    return {"value": round(committed * w.integ.dt * NS_PER_DAY / dt, 6), "unit": "ns/day", "cores": 1,
            "kind": "oracle", "sample": "%d windows (%d committed steps) of %s, single-threaded FP64 C" % (
                windows, committed, w.name)}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    w = _workload(args.config)
    from oracle import oracle as O
    O.build()
    s = w.system
    K = w.integ.K
    q, p, step = s.positions.copy(), s.momenta.copy(), 0
    for _ in range(max(1, min(args.warmup, 1))):
        out = O.lsd_window(s, w.draft, w.target, w.integ, s.seed, step, K, q, p)
    times, committed = [], 0
    n = max(1, min(args.steps, args.ref_windows))
    for _ in range(n):
        t0 = time.perf_counter()
        out = O.lsd_window(s, w.draft, w.target, w.integ, s.seed, step, K, q, p)
        times.append(time.perf_counter() - t0)
        q, p = out["q"], out["p"]
        step += out["n_committed"]
        committed += out["n_committed"]
    tot = sum(times)
    val = committed * w.integ.dt * NS_PER_DAY / tot
    sample = "%d windows (%d committed steps) of %s, single-threaded FP64 C oracle" % (n, committed, w.name)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": "ns/day", "n_gpus": world,
        "steps": n, "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / n, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_atoms": s.n_atoms, "K": K, "dt_fs": w.integ.dt},
        "cpu_baseline": {"value": round(val, 6), "unit": "ns/day", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 6), "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--equil", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-windows", type=int, default=6)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true", help="time the unpipelined window loop only")
    ap.add_argument("--only-lsd", action="store_true", help="time the LSD windows only (for profiler runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
