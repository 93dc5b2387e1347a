#!/usr/bin/env python
"""Benchmark: atom-steps/s of the RBSOG + RBL MD step (force evaluation of
stages a-d + the BAOAB integrator of stage e) on molten NaCl, N = 64,000
(20^3 rock-salt cells, L = 126 A, P_R = 20, P_F = 500, r_core = 6 A,
r_shell = 12 A, Langevin 1200 K, dt = 1 fs), mixed precision.

One JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead (the reference arm).

Timing: W warm-up steps, then K steps, each preceded by an L2 flush (a
512 MiB memset, then a read of 256 MiB so that the memset's dirty lines are
written back before the step rather than inside it; both outside the timed
interval) and timed with CUDA events on the
stream the library runs on; per-stage times come from the event nodes the
library records inside its step graph.  Multi-GPU (torchrun): every rank runs
an independent replica (weak scaling, no collective on the data path); the
time is the max over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20
L2_CLEAN_BYTES = 256 << 20
L2_DESC = "flushed before every step (512 MiB memset, then a 256 MiB read that leaves L2 clean)"


class L2Flush:
    """Evicts the step's data from L2 (126 MB on GB300) before a timed step:
    writes a buffer larger than L2, then reads another one larger than L2, so
    that the lines the write left dirty are written back here and not by the
    first kernels of the step."""

    def __init__(self, torch, dev):
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.r = torch.zeros(L2_CLEAN_BYTES // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.sum()
SFU_LANES_PER_SM = 16      # MUFU lanes per SM per clock (sin, cos, ex2, rsq ...)
ISSUE_PER_SM = 4           # warp instructions per SM per clock (4 schedulers)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="nacl_64k")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--P_F", type=int, default=None)
    ap.add_argument("--P_R", type=int, default=None)
    ap.add_argument("--list-every", type=int, default=None,
                    help="0: per-step random batch lists; n >= 1: kept (skin) lists rebuilt every n steps; "
                         "-1: rebuilt when an atom has moved by skin/2 (default: the workload's, -1)")
    ap.add_argument("--skin", type=float, default=None, help="skin of kept lists [A] (default: the workload's)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="kept lists rebuilt when needed: use the workload's skin instead of timing candidates")
    ap.add_argument("--no-per-step-lists", action="store_true",
                    help="skip the second measurement with lists rebuilt at every step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-force-error", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU form beside the line")
    ap.add_argument("--schedule", default=None,
                    help="schedule rho_variant,rho_blocks_per_sm,far_atoms_per_thread,far_segments,"
                         "far_packed,near_blocks_per_sm,rho_tile_atoms,near_wide,rho_reduce (default: tuned, or the library's with "
                         "--no-autotune)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-replica ensemble beside the line")
    ap.add_argument("--sweep", action="store_true",
                    help="shell batch x P_F sweep of the configuration (one JSON line each)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def pause(self):
        """End of the timed region: later samples are not used."""
        self.n_keep = len(self.lines)

    def stop(self):
        if self.proc is None:
            return None
        if getattr(self, "n_keep", None) is not None:
            self.lines = self.lines[:self.n_keep]
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# kernels of one MD step: main branch k_prepare, k_rowscan, k_cellstart, k_scatter, k_rank,
# k_near, k_finish (F^corr from the near field's fixed-point totals); side branch k_ksample,
# k_rho, k_reduce (rho), k_farforce (the histogram clear is a memset node)
KERNELS_PER_STEP = 11
# kept lists: the near field is the batch draw (k_sample_batch) and the pair
# sums (k_near_kept); a build step adds the list build to the per-step graph;
# a step that reuses the lists has no binning (4 kernels) and no build
KERNELS_BUILD_STEP = 13
KERNELS_KEEP_STEP = 8
# automatic kept lists: every step's graph holds the binning and build
# kernels (they return at once unless the step rebuilds)
KERNELS_AUTO_STEP = 13
KERNEL_LABEL = {"near": "k_near", "rho": "k_rho", "farforce": "k_farforce"}


METRIC = "atom-steps/s of RBSOG+RBL force step at <=1e-5 RMS rel. force err, mixed vs FP64"

# Algorithmic work per unit (the minimal operation model of the design notes):
# lane multiply-add / FP32 operations on the FMA pipe, and issue slots when
# two FP32 lanes share one packed FP32x2 instruction (integer multiply-adds
# take a slot per lane).
OPS_PAIR = 25.0            # one near-field pair (FP32 pair force, tabulated SOG part)
OPS_TEST = 8.0             # one list-predicate test
OPS_RHO = 3.0 + 10.0 + 2.0     # per (atom, k): phase (3 IMAD), sin + cos (10), 2 FMA into rho
OPS_FAR = 3.0 + 5.0 + 3.0      # per (atom, k): phase (3 IMAD), one sine (5), 3 FMA into the force
SLOTS_RHO = 3.0 + 12.0 / 2.0
SLOTS_FAR = 3.0 + 8.0 / 2.0
# the plain FP64 form, FP64 multiply-adds: per pair M+1 = 65 Gaussians (exp ~ 11 + 1
# each) plus the BMH terms; per (atom, k) an FP64 sincospi (~15) plus 2 (rho) or 5 (force)
DFMA_PAIR = 65 * 12.0 + 20.0
DFMA_RHO = 15.0 + 2.0
DFMA_FAR = 15.0 + 5.0


def algorithmic_ops(w, P_F, P_R, r_core=6.0, r_shell=12.0, list_every=0, skin=0.0, builds_per_step=None):
    """Algorithmic FMA-pipe lane operations of one force evaluation, per stage:
    near field = OPS_TEST per list test of every neighbour inside the list
    radius, performed at every step with per-step lists and at each build
    (r_shell + skin) with kept lists, charged by the builds actually made per
    step, plus OPS_PAIR per evaluated pair (core + P_R shell); structure factor
    OPS_RHO and far force OPS_FAR per (atom, k).  Also the packed issue-slot
    count of the two far-field kernels."""
    rho_n = w.n / float(np.prod(w.box))
    if list_every == 0:
        tests = 4.0 / 3.0 * np.pi * r_shell ** 3 * rho_n
    else:
        bps = builds_per_step if builds_per_step is not None else 1.0 / max(list_every, 1)
        tests = 4.0 / 3.0 * np.pi * (r_shell + skin) ** 3 * rho_n * bps
    n_core = 4.0 / 3.0 * np.pi * r_core ** 3 * rho_n
    ops = {"near": w.n * (OPS_TEST * tests + OPS_PAIR * (n_core + P_R)),
           "rho": OPS_RHO * w.n * P_F, "farforce": OPS_FAR * w.n * P_F}
    slots = {"rho": SLOTS_RHO * w.n * P_F, "farforce": SLOTS_FAR * w.n * P_F}
    return ops, slots, tests


def fp64_dfma(w, P_F, P_R, r_core=6.0):
    rho_n = w.n / float(np.prod(w.box))
    n_core = 4.0 / 3.0 * np.pi * r_core ** 3 * rho_n
    return w.n * (DFMA_PAIR * (n_core + P_R) + (DFMA_RHO + DFMA_FAR) * P_F)


def measured_peaks(rbsog, local):
    """Multiply-add lane operations per second of the FP32 (scalar and packed),
    FP64 and integer pipes, measured on this GPU (rbsog_probe_peak)."""
    out = {}
    for name, kind in (("fp32", rbsog.PROBE_FP32), ("fp32x2", rbsog.PROBE_FP32X2), ("fp64", rbsog.PROBE_FP64),
                       ("imad", rbsog.PROBE_IMAD)):
        out[name] = max(rbsog.probe_peak(local, kind) for _ in range(3))
    return out


def profiled_traffic(stage, kept=False):
    """DRAM bytes per launch of the stage's kernels (with kept lists the near
    field is the batch draw and the pair sums) from the committed ncu summary,
    only while the kernels' source is the one that was profiled (else None)."""
    import hashlib
    src = {"near": "k_near.cu", "rho": "k_far.cu", "farforce": "k_far.cu"}.get(stage)
    names = ["k_sample_batch", "k_near_kept"] if (stage == "near" and kept) else [KERNEL_LABEL.get(stage)]
    summ = os.path.join(ROOT, "profiles", "traffic_nacl64k.txt")
    if src is None or not os.path.exists(summ):
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2512_24970_gb300", "csrc", src), "rb").read()).hexdigest()[:16]
    found = {}
    for line in open(summ):
        f = line.split()
        if len(f) >= 3 and f[0] in names and f[1] == h:
            found[f[0]] = float(f[2])
    return sum(found.values()) if len(found) == len(names) else None


def force_error(rbsog, w, prm, dev):
    """RMS relative force error of the mixed-precision path against the FP64
    GPU path, eps = sqrt(sum |F_mixed - F_FP64|^2 / sum |F_FP64|^2), from the
    same positions, seed and step (so the same shell batches and k-batch), and
    the largest per-atom relative error."""
    import dataclasses
    F = {}
    for name, pr in (("mixed", rbsog.MIXED), ("fp64", rbsog.FP64)):
        c = rbsog.Context(dev)
        c.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, dataclasses.replace(prm, precision=pr))
        c.set_state(w.pos, None, 1)
        F[name] = c.compute_forces()
        c.close()
    d = F["mixed"] - F["fp64"]
    eps = float(np.sqrt((d ** 2).sum() / (F["fp64"] ** 2).sum()))
    per = np.sqrt((d ** 2).sum(1)) / np.maximum(np.sqrt((F["fp64"] ** 2).sum(1)), 1e-30)
    return {"rms_rel": eps, "max_atom_rel": float(per.max()), "median_atom_rel": float(np.median(per)),
            "what": "mixed vs FP64 GPU path, same state, seed and step (identical samples)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
def oracle_sample(w, cfg, P_F, P_R, budget_s=15.0):
    """Oracle (FP64 CPU) atom-steps/s on a bounded sample of the workload: the
    structure factor over all N atoms for all P_F modes, then the near + far
    field of successive blocks of atoms (cycling through the box, one RNG step
    per pass) until about budget_s seconds of work; the per-atom cost is scaled
    to N.  Returns (value, seconds, sample text)."""
    import oracle
    S = oracle.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=P_R, P_F=P_F, seed=cfg.seed)
    N = w.n
    t0 = time.perf_counter()
    m, c, _ = S.kbatch()
    t1 = time.perf_counter()
    rho = S.rho(m)
    t_rho = time.perf_counter() - t1
    block = 1024
    done, t_atoms, start = 0, 0.0, 0
    while True:
        sel = (start + np.arange(block, dtype=np.int64)) % N
        t2 = time.perf_counter()
        S.near(sel)
        S.far(m, c, rho, sel)
        t_atoms += time.perf_counter() - t2
        done += block
        start += block
        if start >= N:
            start -= N
            S.step += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    T = t_rho + N * t_atoms / done
    wall = time.perf_counter() - t0
    sample = ("force evaluation of %s: structure factor of all %d atoms x %d modes, near + far field of "
              "%d atom evaluations (scaled to N), %.1f s of oracle work" % (cfg.key, N, P_F, done, wall))
    return N / T, wall, sample


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2512_24970_gb300 import workloads as W
    w, cfg = W.make(args.config)
    P_F = args.P_F or cfg.P_F
    P_R = args.P_R or cfg.P_R
    oracle.build()
    nthreads = oracle.num_threads()
    total = max(1, args.steps + args.warmup)
    budget = float(np.clip(150.0 / total, 1.0, 15.0))      # the whole run stays within a few minutes
    vals = []
    for k in range(args.warmup + args.steps):
        v, wall, sample = oracle_sample(w, cfg, P_F, P_R, budget_s=budget)
        if k >= args.warmup:
            vals.append(v)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "atom-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * w.n / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg.description, "P_F": P_F, "P_R": P_R},
        "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2512_24970_gb300 import build, rbsog, workloads as W
    from paper_2512_24970_gb300.replicas import aggregate, replica_seed
    build.build()
    w, cfg = W.make(args.config)
    P_F = args.P_F or cfg.P_F
    P_R = args.P_R or cfg.P_R
    prec = rbsog.MIXED if args.precision == "mixed" else rbsog.FP64
    list_every = cfg.list_every if args.list_every is None else args.list_every
    skin = (cfg.skin if args.skin is None else args.skin) if list_every != 0 else 0.0
    prm = rbsog.MethodParams(P_R=P_R, P_F=P_F, seed=replica_seed(cfg.seed, rank), precision=prec,
                             integrator=rbsog.LANGEVIN_BAOAB if cfg.integrator == "langevin" else rbsog.NVE_VV,
                             T=cfg.T, dt=0.001, gamma=cfg.gamma, list_every=list_every, skin=skin)
    stream = torch.cuda.Stream(device=dev)
    flush = L2Flush(torch, dev)
    K, Wm = args.steps, args.warmup
    # the skin of automatically rebuilt kept lists: timed candidates (outside
    # the timed region), unless given
    tuning = None
    if list_every < 0 and args.skin is None and not args.no_autotune:
        from paper_2512_24970_gb300 import autotune
        # 500 steps per candidate at N = 64,000, fewer for larger systems (at
        # least 100): at P_F = 1000 the N = 216,000 and 1,024,000 workloads
        # heat up, or blow up, within a few hundred Langevin steps at 1/ps
        skin_steps = max(100, int(500 * 64000 / w.n))
        skin, table, rejected = autotune.tune_skin(w, prm, device=local, stream=stream, flush=flush,
                                                   steps=skin_steps)
        prm = dataclasses.replace(prm, skin=skin)
        tuning = {"chosen_skin": skin, "candidates": [{"skin": a, "ms_per_step": b, "list_builds": c}
                                                      for a, b, c in table],
                  "rejected": [{"skin": a, "why": r} for a, r in rejected],
                  "how": "%d steps per candidate after 20 warm-up, each after an L2 flush and timed alone with CUDA events (autotune.tune_skin)" % skin_steps}

    sched, sched_tuning = None, None
    if args.schedule:
        sched = tuple(int(x) for x in args.schedule.split(","))
    elif prec == rbsog.MIXED and not args.no_autotune:
        from paper_2512_24970_gb300 import autotune
        sched, table = autotune.tune_schedule(w, prm, device=local, stream=stream, flush=flush)
        sched_tuning = {"chosen": dict(zip(("rho_variant", "rho_blocks_per_sm", "far_atoms_per_thread",
                                             "far_segments", "far_packed", "near_blocks_per_sm", "rho_tile_atoms", "near_wide",
                                             "rho_reduce"), sched)),
                        "candidates": [{"schedule": list(q), "ms_per_step": t} for q, t in table],
                        "how": "100 MD steps per candidate after 10 warm-up, every candidate from the same initial "
                               "state, each step after an L2 flush and timed alone with CUDA events, coordinate "
                               "search (autotune.tune_schedule)"}

    def timed_run(params, clocks=None, k_stage=None):
        """Wm untimed steps, then K steps timed with CUDA events on the
        launching stream (L2 flushed before each; no event inside the step
        graph), then k_stage more steps with the stage events on (they add
        event nodes to the graph, so they stay out of the timed steps).
        Returns the context, the per-step ms and the mean stage times."""
        c = rbsog.Context(local, stream.cuda_stream)
        c.set_workload(w, params)
        if sched is not None:
            c.set_schedule(*sched)
        with torch.cuda.stream(stream):
            for _ in range(Wm):
                flush()
                c.step(1)
            torch.cuda.synchronize()
            if ws > 1:
                dist.barrier()
            b0 = c.list_builds()
            if clocks:
                clocks.start()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            torch.cuda.synchronize()
            for k in range(K):
                flush()
                ev[k][0].record(stream)
                c.step(1)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            if ws > 1:
                dist.barrier()
            if clocks:
                clocks.pause()
            builds_timed = c.list_builds() - b0
            ks = min(K, 500) if k_stage is None else k_stage
            st = np.zeros(rbsog.NSTAGE)
            mk = np.zeros(rbsog.NMARK)
            c.set_profiling(True)
            for k in range(ks):
                flush()
                c.step(1)
                st += c.stage_times()          # waits for this step's last event
                mk += c.stage_marks()
            c.set_profiling(False)
        c.sync()
        return c, np.array([a.elapsed_time(b) for a, b in ev]), st / max(ks, 1), mk / max(ks, 1), builds_timed

    peak_ops = measured_peaks(rbsog, local)
    clocks = Clocks(local)
    ctx, ms, stage_ms, marks, builds_timed = timed_run(prm, clocks)
    clk = clocks.stop()
    value, t_total, _ = aggregate(float(ms.sum()), float(w.n * K), dist if ws > 1 else None, dev)
    # the same steps with the random batch lists rebuilt from scratch at every step
    per_step = None
    if list_every != 0 and not args.no_per_step_lists:
        c1, ms1, st1, mk1, _ = timed_run(dataclasses.replace(prm, list_every=0, skin=0.0), k_stage=min(K, 200))
        c1.close()
        v1, t1, _ = aggregate(float(ms1.sum()), float(w.n * K), dist if ws > 1 else None, dev)
        per_step = {"value": v1, "unit": "atom-steps/s", "ms_per_step": t1 / K,
                    "stage_ms": {n: float(t) for n, t in zip(rbsog.STAGES, st1)},
                    "timeline_us": {n: round(float(t) * 1e3, 2) for n, t in zip(rbsog.MARKS, mk1)},
                    "what": "same workload and steps, random batch lists rebuilt from the positions at every step"}
    # ---- roofline of the dominant kernel -------------------------------------
    # denominators measured on this GPU in this run (rbsog_probe_peak): the
    # FP32 FMA pipe in lane multiply-adds per second (packed or not, the larger),
    # and the issue rate (4 warp instructions per clock per SM at the clock the
    # probe ran, i.e. the scalar FP32 probe's rate, one lane-op per slot)
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    names = rbsog.STAGES
    bps = (builds_timed / K) if list_every != 0 else None
    alg, slots, tests = algorithmic_ops(w, P_F, P_R, list_every=list_every, skin=prm.skin, builds_per_step=bps)
    fma_peak = max(peak_ops["fp32"], peak_ops["fp32x2"])
    issue_peak = peak_ops["fp32"]
    label = dict(KERNEL_LABEL)
    if list_every != 0:
        label["near"] = ("k_sample_batch + k_near_kept (+ list builds by k_near, charged per build made in the "
                         "timed steps)")
    # every hot kernel against the FMA-pipe peak, from its own live events (the
    # near field on the main stream, k_rho and k_farforce on the side stream,
    # running concurrently, so a live duration includes time spent sharing
    # the SMs); the dominant kernel is the one with the longest live time
    kern = {}
    for kname in ("near", "rho", "farforce"):
        t = stage_ms[names.index(kname)] * 1e-3
        kern[kname] = {"kernel": label[kname], "ms": t * 1e3, "achieved": alg[kname] / t / 1e9,
                       "frac": alg[kname] / t / fma_peak}
        if kname in slots:
            kern[kname]["issue_frac"] = slots[kname] / t / issue_peak
    # the kept near field reads its lists from HBM: algorithmic bytes per atom-step
    # = the entries of A and of the batch (4 B each), |A| and |B| (8 B), its own
    # slot record and each member's coordinates once (16 B + 16 B), its force (12 B)
    pk_json, pk_kind = peaks()
    hbm_peak = float(pk_json.get("hbm_gbs", 6800.0)) * 1e9
    rho_n = w.n / float(np.prod(w.box))
    n_core = 4.0 / 3.0 * np.pi * 6.0 ** 3 * rho_n
    if list_every != 0:
        kb = w.n * (4.0 * (n_core + P_R) + 8.0 + 16.0 + 16.0 + 12.0)
        t = kern["near"]["ms"] * 1e-3
        kern["near"].update({"algorithmic_bytes": kb, "achieved_gbs": kb / t / 1e9, "hbm_frac": kb / t / hbm_peak,
                             "hbm_peak_gbs": hbm_peak / 1e9, "hbm_peak_source": pk_kind + " (MEASURED_PEAKS.json)"})
    dom = max(kern, key=lambda k: kern[k]["ms"])
    near_hbm = dom == "near" and list_every != 0 and kern["near"]["algorithmic_bytes"] / hbm_peak > alg["near"] / fma_peak
    if near_hbm:
        roof = {"bound": "hbm", "kernel": label[dom], "achieved": kern[dom]["achieved_gbs"], "peak": hbm_peak / 1e9,
                "unit": "GB/s", "frac": kern[dom]["hbm_frac"],
                "traffic": profiled_traffic(dom, kept=True),
                "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs, %s)" % pk_kind,
                "bytes_per_unit": {"atom_step": kern[dom]["algorithmic_bytes"] / w.n},
                "units": {"atoms": w.n},
                "alu_frac": kern[dom]["frac"]}
    else:
        roof = {"bound": "alu", "kernel": label[dom], "achieved": kern[dom]["achieved"], "peak": fma_peak / 1e9,
            "unit": "Glane-op/s", "frac": kern[dom]["frac"],
            "traffic": profiled_traffic(dom, kept=list_every != 0),
            "peak_source": "measured in this run: FP32 multiply-add pipe, %d SMs (rbsog_probe_peak)" % nsm,
            "ops_per_unit": {"near_pair": OPS_PAIR, "list_test": OPS_TEST, "rho_atom_k": OPS_RHO,
                             "far_atom_k": OPS_FAR},
            "units": {"atoms": w.n, "P_F": P_F, "list_tests_per_atom_step": tests}}
        if "issue_frac" in kern[dom]:
            roof["issue_frac"] = kern[dom]["issue_frac"]
    step_ops = sum(alg.values())
    step_roof = {"ops_per_step": step_ops, "t_roof_us": step_ops / fma_peak * 1e6,
                 "frac": (step_ops / fma_peak) / (t_total / K * 1e-3),
                 "what": "all algorithmic FMA-pipe work of the step at the measured FP32 multiply-add rate"}
    # ---- the plain FP64 GPU form on the same workload ---------------------------
    fp64 = None
    if prec == rbsog.MIXED and not args.no_fp64:
        Kd = max(3, min(K, 20))
        cd = rbsog.Context(local, stream.cuda_stream)
        cd.set_workload(w, dataclasses.replace(prm, precision=rbsog.FP64))
        with torch.cuda.stream(stream):
            cd.step(2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cd.step(Kd)
            e1.record(stream)
            torch.cuda.synchronize()
        cd.sync()
        td = e0.elapsed_time(e1) / Kd
        cd.close()
        dfma = fp64_dfma(w, P_F, P_R)
        fp64 = {"value": w.n / (td * 1e-3), "unit": "atom-steps/s", "ms_per_step": td, "steps": Kd,
                "dfma_per_step": dfma, "peak_dfma_per_s": peak_ops["fp64"],
                "frac": dfma / (td * 1e-3) / peak_ops["fp64"],
                "mixed_over_fp64": (t_total / K) ** -1 / td ** -1 if td > 0 else None,
                "what": "same workload, lists and integrator in the plain FP64 form (analytic pair terms with "
                        "all M+1 Gaussians, FP64 sincospi, FP64 sums); DFMA model per pair %.0f, per (atom, k) "
                        "%.0f; peak = measured FP64 multiply-add rate" % (DFMA_PAIR, DFMA_RHO + DFMA_FAR)}
    # ---- end to end through the public API (host buffers) --------------------
    e2e = None
    if not args.no_e2e:
        # a caller that integrates on its side: every step hands the positions
        # over from pinned host memory and reads the forces back.  The positions
        # are those of this run's own next steps, recorded beforehand, so the
        # kept lists are rebuilt (by the device's skin/2 check) as often as in
        # the run itself.
        Ke = args.e2e_steps
        traj = torch.empty((Ke, w.n, 3), dtype=torch.float64, pin_memory=True).numpy()
        frc_h = torch.empty((w.n, 3), dtype=torch.float64, pin_memory=True).numpy()
        ctx.set_profiling(False)
        with torch.cuda.stream(stream):
            p0, v0s, s0 = ctx.get_state()
            for k in range(Ke):
                ctx.step(1)
                ctx.get_state(pos=traj[k])
            ctx.set_state(p0, v0s, s0)
            for k in range(3):
                ctx.forces_at(traj[k], s0 + 1 + k, frc_h)
            ctx.set_state(p0, v0s, s0)
            ctx.compute_forces(frc_h)
            b0 = ctx.list_builds()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(Ke):
                # H2D positions (pinned), force evaluation, D2H forces (pinned)
                ctx.forces_at(traj[k], s0 + 1 + k, frc_h)
            torch.cuda.synchronize()
            te = time.perf_counter() - t0
            nb = ctx.list_builds() - b0
        e2e = {"value": w.n * Ke / te, "unit": "atom-steps/s", "h2d_bytes_per_step": 24 * w.n,
               "d2h_bytes_per_step": 24 * w.n,
               "what": "rbsog_forces_at(host positions of %d recorded steps of this run, host forces) "
                       "per step, i.e. rbsog_move_atoms + rbsog_compute_forces in one call%s" %
                       (Ke, "; kept lists rebuilt by the device check: %d builds" % nb if list_every != 0 else "")}
    # ---- mixed vs FP64 force error on identical state and samples ---------------
    ferr = None
    if not args.no_force_error and prec == rbsog.MIXED and ws == 1:
        ferr = force_error(rbsog, w, prm, local)
    # ---- CPU baseline (oracle) ---------------------------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = oracle.num_threads()
        v, wall, sample = oracle_sample(w, cfg, P_F, P_R)
        oracle.set_num_threads(1)                 # and on one core, a shorter sample
        v1, wall1, sample1 = oracle_sample(w, cfg, P_F, P_R, budget_s=5.0)
        oracle.set_num_threads(cores)
        cpu = {"value": v, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
               "sample": sample, "wall_s": wall,
               "single_core": {"value": v1, "unit": "atom-steps/s", "cores": 1, "sample": sample1,
                               "wall_s": wall1}}
    if list_every < 0:
        launches = KERNELS_AUTO_STEP * K
    elif list_every > 0:
        builds = sum(1 for s in range(Wm + 1, Wm + K + 1) if s % list_every == 0)
        launches = KERNELS_BUILD_STEP * builds + KERNELS_KEEP_STEP * (K - builds)
    else:
        launches = KERNELS_PER_STEP * K
    if rank == 0:
        ens = None
        if ws == 1 and not args.no_ensemble and args.config == "nacl_64k":
            ens = ensemble_measure(args, K, Wm, with_sequential=True)
        line = {
            "metric": METRIC,
            "value": value, "unit": "atom-steps/s", "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": t_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == rbsog.MIXED else "f64", "data": "synthetic",
            "config": {"workload": cfg.description, "N": w.n, "P_F": P_F, "P_R": P_R, "r_core": 6.0,
                       "r_shell": 12.0, "precision": args.precision, "langevin_gamma_per_ps": cfg.gamma, "l2": L2_DESC,
                       "lists": ("per step" if not list_every else
                                 ("kept: skin %.2f A, rebuilt when an atom has moved by skin/2 (%d builds in the "
                                  "%d timed steps)" % (prm.skin, builds_timed, K)) if list_every < 0 else
                                 "kept: skin %.2f A, rebuilt every %d steps (%d builds in the %d timed steps)" %
                                 (prm.skin, list_every, builds_timed, K)),
                       "list_builds_timed": builds_timed if list_every != 0 else K,
                       "skin_tuning": tuning, "schedule_tuning": sched_tuning,
                       "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "stage_ms": {n: float(t) for n, t in zip(names, stage_ms)},
            "timeline_us": {n: round(float(t) * 1e3, 2) for n, t in zip(rbsog.MARKS, marks)},
            "roofline": roof, "kernel_rooflines": kern, "step_roofline": step_roof, "per_step_lists": per_step,
            "peaks": {"measured_here": {k: v / 1e9 for k, v in peak_ops.items()}, "unit": "G lane multiply-adds/s",
                      "how": "rbsog_probe_peak, best of 3"},
            "clocks": clk, "e2e": e2e, "fp64_gpu": fp64, "ensemble": ens,
            "gpu_launches": launches, "cpu_baseline": cpu, "force_error": ferr,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def ensemble_measure(args, K, Wm, with_sequential=True):
    """The replica ensemble (64 replicas of uneven size and composition, one
    ensemble step = one MD step of every replica, all overlapping on the GPU)
    against the same replicas stepped one after another on one stream."""
    import torch
    from paper_2512_24970_gb300 import build, rbsog, workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    reps = W.ensemble(n_rep=64, seed=5)
    stream = torch.cuda.Stream(device=dev)
    ens = rbsog.Ensemble(0, stream.cuda_stream, max_replicas=len(reps))
    natoms = 0
    list_every = -1 if args.list_every is None else args.list_every

    def params(r, w, T):
        # kept lists rebuilt when needed, with the skin each box allows (at most
        # 1 A; L >= 2 (r_shell + skin)); or per-step lists with --list-every 0
        skin = min(1.0, 0.5 * float(w.box.min()) - 12.0 - 0.01) if list_every else 0.0
        return rbsog.MethodParams(P_R=20, P_F=500, seed=5000 + r, precision=rbsog.MIXED,
                                  integrator=rbsog.LANGEVIN_BAOAB, T=T, list_every=list_every, skin=skin)

    for r, (w, T) in enumerate(reps):
        prm = params(r, w, T)
        c = ens.add_workload(w, prm)
        c.set_velocities(w.vel)
        natoms += w.n
    flush = L2Flush(torch, dev)
    def timed(step_fn):
        with torch.cuda.stream(stream):
            for _ in range(Wm):
                flush()
                step_fn()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            for k in range(K):
                flush()
                ev[k][0].record(stream)
                step_fn()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in ev))

    tuning = None
    if args.schedule:
        q = tuple(int(x) for x in args.schedule.split(","))
        for c in ens.replicas:
            c.set_schedule(*q)
        tuning = {"chosen": list(q), "how": "given (--schedule)"}
    elif not args.no_autotune:
        from paper_2512_24970_gb300 import autotune
        best, table = autotune.tune_ensemble_schedule(ens, stream=stream, flush=flush)
        tuning = {"chosen": {"schedule": list(best[0]), "groups": best[1]},
                  "candidates": [{"schedule": list(q), "groups": g, "ms_per_step": t} for (q, g), t in table],
                  "how": "20 ensemble steps per candidate after 3 warm-up, each after an L2 flush and timed alone, "
                         "coordinate search (autotune.tune_ensemble_schedule); groups = replicas dealt into that "
                         "many packed groups run as parallel graph branches, 0 = child graphs"}
    t_ens = timed(lambda: ens.step(1))
    ens.sync()
    out = {"value": natoms * K / (t_ens / 1000.0), "unit": "atom-steps/s", "ms_per_step": t_ens / K, "steps": K,
           "workload": "64 replicas: N = 8 n^3, n in [4, 16] (N 512..32768), NaCl / LiCl / LiCl-NaCl, "
                       "T 1100-1300 K, P_F = 500, P_R = 20", "atoms": natoms,
           "lists": ("per step" if not list_every else
                     "kept, rebuilt when an atom has moved by skin/2; skin min(1 A, L/2 - r_shell)"),
           "launch": ens.launch_kind(), "l2": L2_DESC,
           "schedule_tuning": tuning}
    # the same ensemble with every replica in one packed group, and as child
    # graphs (each replica's own step graph), beside the tuned plan
    used = ens.used_mode()
    for name, mode, groups in (("one_packed_group", rbsog.ENSEMBLE_PACKED, 1), ("child_graphs", rbsog.ENSEMBLE_GRAPHS, 1)):
        ens.set_mode(mode)
        ens.set_groups(groups)
        t_g = timed(lambda: ens.step(1))
        ens.sync()
        out[name] = {"value": natoms * K / (t_g / 1000.0), "ms_per_step": t_g / K, "launch": ens.launch_kind()}
    if with_sequential:
        # the same replicas one after another, each step on the ensemble's stream
        solo = []
        for r, (w, T) in enumerate(reps):
            c = rbsog.Context(0, stream.cuda_stream)
            c.set_workload(w, params(r, w, T))
            solo.append(c)

        def seq():
            for c in solo:
                c.step(1)

        t_seq = timed(seq)
        out["sequential"] = {"value": natoms * K / (t_seq / 1000.0), "ms_per_step": t_seq / K,
                             "what": "the same replicas stepped one after another on one stream"}
        for c in solo:
            c.close()
    ens.close()
    return out


def run_ensemble(args):
    K, Wm = args.steps, args.warmup
    e = ensemble_measure(args, K, Wm)
    line = {"metric": "atom-steps/s of RBSOG+RBL force step, replica ensemble", "value": e["value"],
            "unit": "atom-steps/s", "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": e["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {k: e[k] for k in ("workload", "atoms", "lists", "launch", "l2", "schedule_tuning")},
            "sequential": e.get("sequential"), "child_graphs": e.get("child_graphs"),
            "one_packed_group": e.get("one_packed_group")}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "ensemble_64":
        run_ensemble(args)
    elif args.sweep:
        # shell batch x Fourier batch sweep of one configuration, one line each
        for P_R in (10, 20, 40):
            for P_F in (500, 1000, 2000):
                args.P_R, args.P_F = P_R, P_F
                args.no_cpu_baseline = args.no_e2e = True
                run_ours(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
