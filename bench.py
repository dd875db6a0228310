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


# The dense configurations draft with a learned draft (the 4,096-atom one: "learned BF16 draft"; the 32,768-atom
# one: "learned draft retrained online every 10,000 accepted steps"): LJ + a per-atom MLP on 8 radial basis
# functions per species in BF16, trained during the untimed set-up by the library's online force matching on the
# target-verified frames of its own LSD run (`train_rounds` retrainings, one every `train_every` accepted steps),
# then timed with the trained draft; online retraining stays on at the configuration's cadence where it has one.
LEARNED_ONLINE = {4: 0, 5: 10000}   # configuration -> retraining cadence (accepted steps) during the timed run
# configuration -> steps per verification stage of the timed windows (lsd_set_window_stages: the next stage runs
# only while every step so far was accepted), from a sweep of S on a B300; the other configurations verify their
# windows in one pass, pipelined
WINDOW_STAGES = {4: 4, 5: 1}


def _workload(cfg, pair_draft=False):
    from paper_2606_02455_b300 import workloads as W
    w = W.CONFIGS[cfg]()
    if cfg in LEARNED_ONLINE and not pair_draft:
        w.draft = W.learned_draft(w.target, w.system.n_species)
    w.cfg = cfg
    return w


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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from ncu captures of the kernels as they
# are now (the summaries under profiles/ give the commands); a kernel changed since its capture has no entry here.
# Per verified row for the kernels whose traffic grows with the rows (scaled to the profiled launch's K N rows):
NCU_TRAFFIC_PER_ROW = {
    # desc_mom_kernel: 501,708,288 B per launch of 262,144 rows (the 32,768-atom workload shortened to K = 8: the
    # moments written, 1,344 B per row, and the staged geometry); 199,167,744 B per 131,072 rows at 4,096 atoms
    ("fp8_mlp_32768atoms_K64", "descriptors"): 501708288 / 262144,
    ("bf16_mlp_4096atoms_K32", "descriptors"): 199167744 / 131072,
    # pairgrad_mom_kernel: the moments read back, the pair gradients written
    ("fp8_mlp_32768atoms_K64", "pair_grad"): 873477120 / 262144,
    ("bf16_mlp_4096atoms_K32", "pair_grad"): 368440576 / 131072,
}
# Per launch of a given number of drafted steps (the draft kernel: its lists and weights are read once per launch,
# so its traffic does not grow with the steps): (workload, phase, steps per launch) -> bytes
NCU_TRAFFIC_PER_LAUNCH = {
    # the learned grid draft, 2 drafted steps at 32,768 atoms (a stage of the staged windows): 37,615,360 B read
    # (lists, positions, first-layer weights), 941,568 B written
    ("fp8_mlp_32768atoms_K64", "draft", 2): 37615360 + 941568,
    # one drafted step (stages of 1 step): 37,255,168 B read, 339,712 B written
    ("fp8_mlp_32768atoms_K64", "draft", 1): 37255168 + 339712,
}


# FP32 operations of one unordered angular neighbour pair (all 16 terms): the descriptor's forward (cosine, the
# powers (1 +- c)^zeta, 16 weighted accumulations) and the pair gradient's backward (the same powers, the value and
# derivative sums S0, S1 per eta, and the two displacement gradients), counted from the formulas each kernel
# evaluates; and per (neighbour, radial basis function): exp argument, exp, cutoff product, accumulation.
FLOP_ANG_DESC = 64
FLOP_ANG_GRAD = 132
FLOP_RAD_DESC = 8
FLOP_RAD_GRAD = 12
FLOP_LJ_PAIR = 23


def _mom_horner_fma():
    """Fused multiply-adds of one eta's nested Horner evaluation of the moment adjoint (value and gradient of a
    degree-8 polynomial in three variables, 165 coefficients), counted from its loops: per x-power 2 (value and
    x-derivative; the first derivative step is a copy), per further y-power 3, per further z-power 4."""
    n = 0
    for c in range(8, -1, -1):
        cols = 9 - c
        for bi in range(cols):
            L = 9 - (8 - c - bi) - c
            n += 2 * (L - 1) - (1 if L >= 2 else 0)
            if bi > 0:
                n += 3 - (1 if bi == 1 else 0)
        if c < 8:
            n += 4 - (1 if c == 7 else 0)
    return n


# The angular block by moments (165 monomials x^a y^b z^c of degree <= 8 per neighbour): per neighbour, the
# descriptor pass forms 24 powers, the unit vector and two weights (5), the monomials (165) and two weighted
# accumulations per monomial (660); per row it squares and scales the 330 moments (990) and forms 16 features
# from 9 sums each (288).  The pair-gradient pass runs the Horner evaluation for both etas (2 FLOP per FMA) and
# its per-neighbour epilogue (42); per row it scales the 330 moments (990) and forms 20 adjoint scalars (960).
FLOP_MOM_DESC_NB = 24 + 5 + 165 + 660
FLOP_MOM_DESC_ROW = 990 + 288
FLOP_MOM_GRAD_NB = 2 * 2 * _mom_horner_fma() + 42
FLOP_MOM_GRAD_ROW = 990 + 960


def _neighbours_per_atom(w, rc):
    s = w.system
    return s.n_atoms / float(np.prod(s.box)) * 4.0 / 3.0 * np.pi * rc ** 3


def _algorithmic_work(w, phase, q, moments=False, K=None):
    """Algorithmic work of one launch of a phase, with its bound: (amount, unit, bound, detail).

    mlp:   2 FLOP per multiply-add of the forward chain plus the input-gradient chain (no weight gradient):
           2 * M * sum(d_in * d_out) * 2, M = K N rows.  FP32 targets run it as three FP16 tensor-core
           products per term (3x the algorithmic MACs executed); BF16 and FP8 targets as one product.
    draft: per drafted step, every LJ pair within the cutoff costs 8 FLOP of distance and 15 of force
           (gather form: each ordered pair once), plus 24 FP64 FLOP per atom of BOB + A;
           K steps per launch, serial.
    descriptors / pair_grad: FP32 ALU work per row, from the mean neighbour count nb within the descriptor cutoff:
           nb (nb - 1) / 2 angular pairs x FLOP_ANG_* (pair sums) or nb x FLOP_MOM_*_NB + FLOP_MOM_*_ROW
           (moments), + nb x n_rbf x FLOP_RAD_* (+ LJ pairs for pair_grad).
    transport: bytes that must cross HBM once per window."""
    s, t, K = w.system, w.target, K or w.integ.K
    N = s.n_atoms
    M = K * N
    if phase == "mlp":
        d0p = ((s.n_species * t.n_rbf + t.n_ang + s.n_species) + 31) // 32 * 32
        macs = d0p * t.width + (t.n_layers - 1) * t.width * t.width + t.width
        return 2.0 * 2.0 * M * macs, "FLOP", "tensor", {"precision": t.precision, "rows": M}
    if phase == "draft":
        nb = _lj_pairs_per_atom(w, q)
        flop = K * (N * nb * FLOP_LJ_PAIR + N * 24)
        detail = {"lj_pairs_per_atom": round(nb, 1), "steps_per_launch": K}
        d = w.draft
        if d.n_layers:
            # the learned draft per atom and step: the radial basis of every descriptor neighbour (forward 8 FLOP,
            # adjoint 12 per basis function), the MLP forward and its input gradient (4 d_in W)
            nbd = _neighbours_per_atom(w, d.desc_cutoff)
            d0 = w.system.n_species * d.n_rbf + d.n_ang + w.system.n_species
            flop += K * N * (nbd * d.n_rbf * (FLOP_RAD_DESC + FLOP_RAD_GRAD) + 4 * d0 * d.width)
            detail["descriptor_neighbours_per_atom"] = round(nbd, 1)
        return flop, "FLOP", "alu", detail
    if phase in ("descriptors", "pair_grad") and t.n_layers:
        nb = _neighbours_per_atom(w, t.desc_cutoff)
        ang = nb * (nb - 1) / 2 if t.n_ang else 0.0
        if phase == "descriptors":
            ang_f = (nb * FLOP_MOM_DESC_NB + FLOP_MOM_DESC_ROW) if moments else ang * FLOP_ANG_DESC
            per_row = (ang_f if t.n_ang else 0.0) + nb * t.n_rbf * FLOP_RAD_DESC
        else:
            nlj = _neighbours_per_atom(w, t.lj_cutoff) if t.lj_cutoff else 0.0
            ang_f = (nb * FLOP_MOM_GRAD_NB + FLOP_MOM_GRAD_ROW) if moments else ang * FLOP_ANG_GRAD
            per_row = (ang_f if t.n_ang else 0.0) + nb * t.n_rbf * FLOP_RAD_GRAD + nlj * FLOP_LJ_PAIR
        return M * per_row, "FLOP", "alu", {"neighbours_per_atom": round(nb, 1), "rows": M,
                                            "flop_per_row": round(per_row),
                                            "angular": "moments" if moments else "pair sums"}
    if phase in ("transport_reduce",):
        return M * 3 * (4 + 4), "B", "hbm", {}
    if phase in ("transport_commit",):
        return N * 3 * (8 + 8 + 4 + 4 + 8 + 8 + 8), "B", "hbm", {}
    return None


def _analysis(st1, st0, rl, K, t_plain_step, Kp=None, S=None):
    """The paper's bounds at the measured operating point (paper_2606_02455_b300.analysis): per-step rejection
    rate <beta> = rejections / tested steps (every committed step was tested, in order; steps after a window's
    first rejection are flushed untested), cost ratio c = drafted-step time / plain-step time, the pipelined
    bound 1 / (c + <beta>) (Eq. 8) and the synchronous lookahead-K bound."""
    from paper_2606_02455_b300 import analysis as A
    tested = max(st1["committed"] - st0["committed"], 1)
    beta = (st1["rejected"] - st0["rejected"]) / tested
    ph = rl["phases_ms"]
    t_draft = ph["draft"] * 1e-3 / (Kp or K)   # the profiled window drafts Kp steps (a stage of a staged window)
    c = t_draft / t_plain_step
    out = {"beta": round(beta, 5), "c": round(c, 5),
           "speedup_async_bound": round(float(A.speedup_async(beta, c)), 3),
           "speedup_sync_bound_K": round(float(A.speedup_sync(beta, c, K)), 3),
           "expected_committed_per_window": round(float(A.expected_committed(beta, K)), 3)}
    if S:
        # windows verified in stages: the i.i.d.-rejection model's stages and verified steps per window, beside the
        # measured ones (stages_per_window)
        out["expected_stages_per_window"] = round(A.expected_stages(beta, K, S), 3)
        out["expected_verified_per_window"] = round(A.expected_verified(beta, K, S), 3)
    return out


def roofline(h, w, peaks, peak_kind, q, n_rep=20, Kp=None):
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
    Kp = Kp or w.integ.K   # steps of the profiled window: K, or the stage length of staged windows
    work = _algorithmic_work(w, dom, q, h.angular_moments(), K=Kp)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s: 148 SMs x 128 FP32 lanes x FMA
    out = {"kernel": dom, "share": round(share, 3), "ms": round(phases[dom], 5), "window_steps_profiled": Kp,
           "phases_ms": {k: round(v, 5) for k, v in phases.items()}}
    if work is None:
        out.update({"bound": "alu", "achieved": None, "peak": round(fp32_peak, 1), "unit": "TFLOP/s", "frac": None,
                    "traffic": None, "note": "no algorithmic model for this phase"})
        return out
    amount, unit, bound, detail = work
    sec = phases[dom] * 1e-3
    out.update(detail)
    per_row = NCU_TRAFFIC_PER_ROW.get((w.name, dom))
    traffic = (round(per_row * Kp * w.system.n_atoms) if per_row is not None
               else NCU_TRAFFIC_PER_LAUNCH.get((w.name, dom, Kp)))
    if bound == "alu":
        ach = amount / sec / 1e12
        out.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                    "frac": round(ach / fp32_peak, 5), "traffic": traffic,
                    "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz" % sm_max})
        if dom == "draft":
            out["us_per_step"] = round(phases[dom] * 1e3 / Kp, 3)
            out["note"] = ("serial chain of K drafted steps (one cooperative grid with a barrier per step for systems of "
                           "2048 atoms or more, else one thread-block cluster of at most 16 SMs); latency-bound: the "
                           "per-step time, not FLOP/s, is the figure of merit")
        elif h.angular_moments():
            out["note"] = ("FP32 operations counted from the kernel's formulas (angular block by moments: %d / %d "
                           "FLOP per neighbour and %d / %d per row; radial term %d / %d FLOP; for descriptors / pair "
                           "gradients) over the derived FP32 FMA peak" % (
                               FLOP_MOM_DESC_NB, FLOP_MOM_GRAD_NB, FLOP_MOM_DESC_ROW, FLOP_MOM_GRAD_ROW,
                               FLOP_RAD_DESC, FLOP_RAD_GRAD))
        else:
            out["note"] = ("FP32 operations counted from the kernel's formulas (angular pair %d / %d FLOP, radial "
                           "term %d / %d FLOP for descriptors / pair gradients) over the derived FP32 FMA peak" % (
                               FLOP_ANG_DESC, FLOP_ANG_GRAD, FLOP_RAD_DESC, FLOP_RAD_GRAD))
    elif bound == "tensor":
        ach = amount / sec / 1e12
        bf16 = peaks["bf16_tflops"]
        if w.target.precision in ("bf16", "fp32"):
            # BF16 and the FP16 split of FP32 targets: the FP16 dense rate equals the BF16 one
            pk, src = bf16, "%s bf16 burst (FP16 dense = BF16 dense)" % peak_kind
        elif w.target.precision == "fp8":
            # FP8 dense = bf16 x (4.5 / 2.25), the nominal ratio
            pk, src = bf16 * 2.0, "%s bf16 burst x 4.5/2.25 (nominal FP8:BF16)" % peak_kind
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

L2_BYTES = 126 * 2 ** 20


def _working_set_bytes(w, K=None):
    """Device bytes one window's verification touches (neighbour keys and pair gradients at ~2x the mean count,
    descriptors and dE/dX, window arrays) for K verified steps (a stage of a staged window; default the window's
    K): decides whether L2 must be flushed between timed windows."""
    s, t, K = w.system, w.target, K or w.integ.K
    N = s.n_atoms
    rc = max(t.desc_cutoff or 0.0, t.lj_cutoff or 0.0)
    nb = 2.0 * N / float(np.prod(s.box)) * 4.0 / 3.0 * np.pi * rc ** 3 + 32
    d0p = ((s.n_species * t.n_rbf + t.n_ang + s.n_species) + 31) // 32 * 32
    return K * N * (nb * (4 + 16) + 2 * 4 * d0p + 3 * (8 + 8 + 4 + 4 + 4))


def measure_workload(w, args, world, rank, full):
    """LSD windows and plain target steps of one workload on this rank's GPU.  `full`: also the unpipelined
    comparison, e2e through the public one-call window, the live per-phase roofline and the clocks."""
    import torch
    from paper_2606_02455_b300 import lsd

    s = w.system
    s.seed = replica_seed(s.seed, rank)   # independent replicas
    K = w.integ.K
    cfg = getattr(w, "cfg", None)
    S = args.stages if args.stages >= 0 else WINDOW_STAGES.get(cfg, 0)
    S = S if S < K else 0
    h = lsd.LSD(s, w.draft, w.target, w.integ)

    reuse = bool(S) and not args.no_list_reuse   # staged windows keep their Verlet lists while they stay valid

    def set_mode(stages, pipe, keep=False):
        h.set_window_stages(0)   # pipelining excludes stages and kept lists
        h.set_list_reuse(False)
        h.set_pipelining(pipe)
        h.set_window_stages(stages)
        h.set_list_reuse(keep)
    stream = torch.cuda.Stream()
    h.set_stream(stream)
    # equilibrate with plain target dynamics
    h.plain_step(args.equil)
    train = None
    pipelined = not args.no_pipeline and S == 0
    if cfg in LEARNED_ONLINE and w.draft.n_layers:
        # the learned draft, trained online on the run's own frames (untimed set-up)
        t0 = time.perf_counter()
        a = h.stats()
        set_mode(S, pipelined, reuse)
        h.set_frame_capture(args.train_frames)
        h.set_online_training(args.train_every, n_iters=args.train_iters, lr=3e-3, frames_per_iter=args.train_fpi)
        while h.online_status()[0] < args.train_rounds:
            h.step(max(args.train_every // 4, 8))
        n_rt, loss = h.online_status()
        b = h.stats()
        cad = LEARNED_ONLINE[cfg]
        if cad:
            h.set_online_training(cad, n_iters=args.train_iters, lr=3e-3, frames_per_iter=args.train_fpi)
        else:
            h.set_online_training(0)
            h.set_frame_capture(0)
        train = {"retrainings": n_rt, "last_loss": loss, "accepted_steps": b["committed"] - a["committed"],
                 "beta_while_training": round((b["rejected"] - a["rejected"]) / max(b["committed"] - a["committed"], 1), 4),
                 "wall_s": round(time.perf_counter() - t0, 2), "every_accepted": args.train_every,
                 "iters": args.train_iters, "frames": args.train_frames, "frames_per_iter": args.train_fpi,
                 "timed_run_cadence": cad or None}
    q_eq, p_eq, step_eq = h.get_state()
    flush_needed = _working_set_bytes(w, S or K) < 4 * L2_BYTES
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda") if flush_needed else None

    def flush_l2():
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.add_(1.0)

    set_mode(S, pipelined, reuse)
    for _ in range(args.warmup):
        h.step(K)
        h.plain_step(1)

    def timed_windows(n):
        """n windows from the equilibrated state on the library's stream.  Small working sets: each window
        bracketed by its own events, L2 flushed before it; otherwise (inputs larger than L2) one event pair."""
        h.set_state(q_eq, p_eq, step_eq)
        a = h.stats()
        _barrier(world)
        torch.cuda.synchronize()
        if flush is not None:
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
            for k in range(n):
                flush_l2()
                ev[k][0].record(stream)
                h.enqueue_windows(1)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            t = sum(x.elapsed_time(y) for x, y in ev) * 1e-3
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.enqueue_windows(n)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
        _barrier(world)
        b = h.stats()
        return (t, b["committed"] - a["committed"], b["rejected"] - a["rejected"], b["windows"] - a["windows"], a, b)

    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0"))) if full else None
    if clocks:
        clocks.start()
    t_lsd, committed, rejected, windows, st0, st1 = timed_windows(args.steps)
    value_unpipelined = value_one_pass = None
    if pipelined and full:
        set_mode(0, False)
        h.step(K)
        t_u, c_u, _, _, _, _ = timed_windows(args.steps)
        value_unpipelined = whole_job_rate(c_u, t_u, world) * w.integ.dt * NS_PER_DAY
        set_mode(0, True)
    if S and full:
        # the same windows verified in one pass (pipelined unless --no-pipeline), for comparison
        set_mode(0, not args.no_pipeline)
        h.step(K)
        t_o, c_o, _, _, _, _ = timed_windows(args.steps)
        value_one_pass = whole_job_rate(c_o, t_o, world) * w.integ.dt * NS_PER_DAY
        set_mode(S, False, reuse)
    # plain target Langevin: the same number of steps as committed, back to back (one graph launch per step)
    h.set_state(q_eq, p_eq, step_eq)
    n_plain = max(committed, 32)
    h.plain_step(2)
    h.set_state(q_eq, p_eq, step_eq)
    torch.cuda.synchronize()
    flush_l2()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.enqueue_plain(n_plain)
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) * 1e-3
    clk = clocks.stop() if clocks else None

    value = whole_job_rate(committed, t_lsd, world) * w.integ.dt * NS_PER_DAY
    plain_value = whole_job_rate(n_plain, t_plain, world) * w.integ.dt * NS_PER_DAY
    lc = h.launch_counts()
    out = {
        "workload": w.name, "value": round(value, 4), "ms_per_window": round(t_lsd * 1e3 / args.steps, 5),
        "acceptance_rate": round(1.0 - rejected / max(committed, 1), 5),
        "committed_per_window": round(committed / max(windows, 1), 3),
        "list_builds_per_window": (round((st1["list_builds"] - st0["list_builds"]) / max(windows, 1), 3)
                                   if reuse else None),
        "stages_per_window": round((st1["stages"] - st0["stages"]) / max(windows, 1), 3) if S else None,
        "plain_target_ns_per_day": round(plain_value, 4), "plain_ms_per_step": round(t_plain * 1e3 / n_plain, 5),
        "speedup_vs_plain": round(value / plain_value, 4),
        "l2": "flushed (256 MB write) before every timed window and once before the plain steps" if flush is not None
        else "not flushed: the window's working set (%.2f GB) is larger than L2" % (_working_set_bytes(w, S or K) / 1e9),
        "draft": _draft_label(w) + (" trained online before timing" if train else ""),
    }
    if train:
        out["draft_training"] = train
    if not full:
        h.close()
        return out
    out.update({
        "t_lsd": t_lsd, "committed": committed, "windows": windows, "n_plain": n_plain, "st0": st0, "st1": st1,
        "t_plain": t_plain, "pipelined": pipelined, "window_stages": S or None,
        "value_unpipelined": None if value_unpipelined is None else round(value_unpipelined, 4),
        "value_one_pass": None if value_one_pass is None else round(value_one_pass, 4),
        # the fused plain step (lc["plain"] == 0) is one launch for all n_plain steps
        "gpu_launches": int(_window_launches(h, lc, pipelined, S, windows, st0, st1) +
                            (1 if lc["plain"] == 0 else n_plain * lc["plain"])),
        "clocks": clk,
    })
    # ---- e2e: the public one-call window with host buffers (pinned): every window uploads its state, runs, and
    # reads the committed state back ----
    h.set_state(q_eq, p_eq, step_eq)
    state = torch.empty((2, s.n_atoms, 3), dtype=torch.float64, pin_memory=True).numpy()
    pos, mom = state[0], state[1]   # adjacent, as on the device: one copy each way
    pos[:] = q_eq
    mom[:] = p_eq
    step = step_eq
    for _ in range(max(args.warmup, 3)):   # untimed: first-call costs of the one-call path
        step, nc = h.window_host(pos, mom, step)
    stats_a = h.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step, nc = h.window_host(pos, mom, step)
    t_e2e = time.perf_counter() - t0
    stats_b = h.stats()
    e2e_committed = stats_b["committed"] - stats_a["committed"]
    D = 3 * s.n_atoms
    out["e2e"] = {"value": round(whole_job_rate(e2e_committed, t_e2e, world) * w.integ.dt * NS_PER_DAY, 4),
                  "unit": "ns/day", "h2d_bytes_per_step": 2 * D * 8 + 16, "d2h_bytes_per_step": 2 * D * 8 + 32,
                  "calls": "lsd_window_host (pinned host state in and out)"}
    out["roofline"] = roofline(h, w, _peaks()[0], _peaks()[1], pos, Kp=S or K)
    h.close()
    return out


def _window_launches(h, lc, pipelined, S, windows, st0, st1):
    """Kernels the timed windows launched: per round (pipelined), per window, or per stage run (staged)."""
    if S:
        sc = h.stage_launch_counts()
        return windows * sc["first"] + (st1["stages"] - st0["stages"] - windows) * sc["later"]
    return windows * (lc["round"] if pipelined else lc["window"])


def run_ours(args):
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = _workload(args.config, getattr(args, "pair_draft", False))
    K = w.integ.K
    m = measure_workload(w, args, world, rank, full=True)
    st0, st1 = m["st0"], m["st1"]
    extra = {}
    for cfg in args.extra:
        if cfg == args.config:
            continue
        extra["config%d" % cfg] = measure_workload(_workload(cfg, args.pair_draft), args, world, rank, full=False)
    t = w.target
    line = {
        "metric": METRIC, "value": m["value"], "unit": "ns/day", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(_max_over_ranks(m["t_lsd"], world) * 1e3 / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "dtype_detail": ("FP32 forces and descriptors; MLP %s; FP64 integrator state, z.delta, delta.delta and "
                         "log ratio" % {"fp32": "at FP32 accuracy as three FP16 tensor-core products per term "
                                                "(exact power-of-two scales)",
                                        "fp32-tf32": "at FP32 accuracy as three TF32 tensor-core products per term",
                                        "bf16": "in BF16 on the tensor cores with FP32 accumulation",
                                        "fp8": "in FP8 e4m3 on the tensor cores (per-tensor scales) with FP32 "
                                               "accumulation",
                                        "fp32-cuda-cores": "in FP32 on the CUDA cores"}[t.precision]),
        "data": "synthetic",
        "config": {"workload": w.name, "n_atoms": w.system.n_atoms, "K": K, "dt_fs": w.integ.dt,
                   "T_K": w.integ.temperature, "gamma_per_fs": w.integ.gamma,
                   "target": "LJ + 0.05 eV tanh(MLP %d->%dx%d->1, %s)" % (
                       w.system.n_species * t.n_rbf + t.n_ang + w.system.n_species, t.width, t.n_layers,
                       t.precision),
                   "draft": m["draft"], "parallelism": "replicas" if world > 1 else "single",
                   "l2": m["l2"]},
        "acceptance_rate": m["acceptance_rate"],
        "analysis": _analysis(st1, st0, m["roofline"], K, m["t_plain"] / m["n_plain"],
                              m["roofline"]["window_steps_profiled"], m["window_stages"]),
        "committed_per_window": m["committed_per_window"],
        "plain_target_ns_per_day": m["plain_target_ns_per_day"],
        "speedup_vs_plain": m["speedup_vs_plain"],
        "pipelined": m["pipelined"],
        "window_stages": m["window_stages"],
        "list_builds_per_window": m["list_builds_per_window"],
        "stages_per_window": m["stages_per_window"],
        "value_unpipelined": m["value_unpipelined"],
        "value_one_pass": m["value_one_pass"],
        "plain_ms_per_step": m["plain_ms_per_step"],
        "gpu_launches": m["gpu_launches"],
        "e2e": m["e2e"],
        "roofline": m["roofline"],
        "clocks": m["clocks"],
        "workloads": extra,
    }
    if "draft_training" in m:
        line["draft_training"] = m["draft_training"]
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _draft_label(w):
    d = w.draft
    if not d.n_layers:
        return "LJ"
    d0 = w.system.n_species * d.n_rbf + d.n_ang + w.system.n_species
    return "LJ + learned MLP %d->%s->1 (%s, linear head)" % (d0, "x".join([str(d.width)] * d.n_layers), d.precision)


# ------------------------------------------------------------------------------------------------------------------
# the oracle on the host (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------------------------------

def _oracle_threads():
    return os.cpu_count() or 1


def oracle_window_rate(w, seconds, threads):
    """Whole oracle windows (Alg. 1, the window-parallel variant: a window's K target evaluations on `threads`
    threads) from the workload's initial state for about `seconds`: (ns/day, sample description)."""
    from oracle import oracle as O
    s = w.system
    K = w.integ.K
    O.set_threads(threads)
    q, p, step = s.positions.copy(), s.momenta.copy(), 0
    t0 = time.perf_counter()
    committed = windows = 0
    while time.perf_counter() - t0 < seconds or windows == 0:
        out = O.lsd_window(s, w.draft, w.target, w.integ, s.seed, step, K, q, p)
        q, p = out["q"], out["p"]
        step += out["n_committed"]
        committed += out["n_committed"]
        windows += 1
    dt = time.perf_counter() - t0
    O.set_threads(1)
    return committed * w.integ.dt * NS_PER_DAY / dt, "%d windows (%d committed steps) of %s" % (
        windows, committed, w.name)


def oracle_slice_rate(w, threads, rows_target, rows_draft, seed=0):
    """A bounded slice of one oracle window when whole windows take hours: the target's energy and forces of
    centre atoms [0, rows_target) in all K window configurations (one configuration per thread, as in the
    window-parallel verification) and the draft's of centre atoms [0, rows_draft) of one configuration; one window
    is extrapolated as (N / rows) times each, the draft K times, and every drafted step is counted as committed (an
    upper bound on the oracle's LSD rate).  The K configurations are the initial state with a seeded 0.01 A jitter
    standing in for the drafted half-step positions.  Returns (ns/day, seconds spent, sample description)."""
    from oracle import oracle as O
    s = w.system
    K, N = w.integ.K, s.n_atoms
    rng = np.random.default_rng(seed)
    qs = s.positions[None] + 0.01 * rng.standard_normal((K, N, 3))
    O.set_threads(threads)
    t0 = time.perf_counter()
    O.eval_range(s, w.target, qs, 0, rows_target)
    t_v = time.perf_counter() - t0
    t1 = time.perf_counter()
    O.eval_range(s, w.draft, qs[:1], 0, rows_draft)
    t_d = time.perf_counter() - t1
    O.set_threads(1)
    window = t_v * N / rows_target + K * t_d * N / rows_draft
    rate = K * w.integ.dt * NS_PER_DAY / window
    desc = ("slice of one window of %s: target energy/forces of centre atoms [0, %d) of %d in all %d configurations "
            "(%.2f s on %d threads) and %s draft of centre atoms [0, %d) of one configuration (%.2f s); one window "
            "extrapolated to %.0f s (verification x %.0f, draft x %d x %.0f), every drafted step counted as committed "
            "(upper bound)" % (w.name, rows_target, N, K, t_v, threads, _draft_label(w), rows_draft, t_d, window,
                               N / rows_target, K, N / rows_draft))
    return rate, t_v + t_d, desc


def _slice_rows(w, seconds, threads):
    """Centre-atom rows of the slice sized so that it takes about `seconds` (about 2/3 target, 1/3 draft),
    from a small timed calibration slice of each."""
    from oracle import oracle as O
    s = w.system
    K, N = w.integ.K, s.n_atoms
    qs = np.repeat(s.positions[None], K, axis=0)
    O.set_threads(threads)
    r0 = min(N, 2)
    t0 = time.perf_counter()
    O.eval_range(s, w.target, qs, 0, r0)
    per_t = (time.perf_counter() - t0) / r0
    r1 = min(N, 32)
    t0 = time.perf_counter()
    O.eval_range(s, w.draft, qs[:1], 0, r1)
    per_d = (time.perf_counter() - t0) / r1
    O.set_threads(1)
    rows_t = int(max(1, min(N, 0.65 * seconds / max(per_t, 1e-9))))
    rows_d = int(max(1, min(N, 0.35 * seconds / max(per_d, 1e-9))))
    return rows_t, rows_d


def cpu_baseline(w, seconds):
    threads = _oracle_threads()
    if w.system.n_atoms <= 256:
        val, sample = oracle_window_rate(w, seconds, threads)
        sample += ", window-parallel FP64 C oracle on %d threads" % threads
    else:
        rt, rd = _slice_rows(w, seconds, threads)
        val, _, sample = oracle_slice_rate(w, threads, rt, rd)
    return {"value": val, "unit": "ns/day", "cores": threads, "kind": "oracle", "sample": sample}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    w = _workload(args.config, getattr(args, "pair_draft", False))
    from oracle import oracle as O
    O.build()
    threads = _oracle_threads()
    K = w.integ.K
    small = w.system.n_atoms <= 256
    rt, rd = (None, None) if small else _slice_rows(w, args.ref_seconds, threads)
    vals, times, desc = [], [], ""
    for k in range(args.warmup + args.steps):
        if small:
            t0 = time.perf_counter()
            v, desc = oracle_window_rate(w, args.ref_seconds, threads)
            dt = time.perf_counter() - t0
        else:
            v, dt, desc = oracle_slice_rate(w, threads, rt, rd, seed=k)
        if k >= args.warmup:
            vals.append(v)
            times.append(dt)
    val = float(np.mean(vals))
    sample = "each step: " + desc + (", window-parallel FP64 C oracle on %d threads" % threads if small else "")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "ns/day", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(float(np.mean(times)) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_atoms": w.system.n_atoms, "K": K, "dt_fs": w.integ.dt},
        "cpu_baseline": {"value": val, "unit": "ns/day", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--extra", type=int, nargs="*", default=[2, 4],
                    help="configurations measured as well (value, plain, acceptance) under `workloads`")
    ap.add_argument("--equil", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=4.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true", help="time the unpipelined window loop only")
    ap.add_argument("--pair-draft", action="store_true", help="the dense configurations with the bare LJ draft")
    ap.add_argument("--no-list-reuse", action="store_true",
                    help="staged windows rebuild their Verlet lists every window")
    ap.add_argument("--stages", type=int, default=-1,
                    help="steps per verification stage (0: one pass; default: per configuration, WINDOW_STAGES)")
    ap.add_argument("--train-rounds", type=int, default=16, help="online retrainings of the learned draft before timing")
    ap.add_argument("--train-every", type=int, default=200, help="accepted steps between retrainings before timing")
    ap.add_argument("--train-iters", type=int, default=40)
    ap.add_argument("--train-frames", type=int, default=128)
    ap.add_argument("--train-fpi", type=int, default=16)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
