"""Benchmark: batched fitness evaluation of one GOM/FOS step on GB300.

One step = one batched evaluation of every trial of one FOS step (pack,
batched forward, finalise), replayed as a CUDA graph, on the largest
workload, "large-16384xh6-1000000x10": 16,384 trials of height 6 (127
nodes, full function set), X 1,000,000 x 10 ~ U[-1, 1], y from a seeded
height-6 tree plus 1 % noise.  Inputs are resident in HBM when the timed
region starts; L2 is flushed (a 512 MB write) between timed steps.
Reported:

  value      node-row evals/s (active nodes x rows x trials / s), graph form;
             the library folds each feature-free subtree into one constant
             (bit-identical outputs), so fewer nodes run per row than the
             active count: config.nodes_evaluated_per_row_per_step; a trial
             stops once one of its tiles is non-finite (+inf fitness):
             config.trials_with_infinite_fitness
  e2e        the same through the C ABI with pinned HOST buffers: the H2D
             copy of the trial arrays and the D2H copy of the fitness inside
             every step
  plain      the one-launch-per-trial form (multi-block per trial + a
             second-stage reduction launch per trial)
  roofline   the batched forward kernel's algorithmic FP32 and SFU
             operations (of the folded programs) per second against the
             FP32 and SFU issue rates measured in the same process
             (ggeval_pipe_rates); the pipe with the larger fraction bounds
             the kernel and gives the headline fields
  parity     the timed outputs of a sample of trials against the FP64 oracle
  cpu_baseline  the FP64 oracle on one host core, on a sample of trials
  cpu_baseline_all_cores  the same oracle over every host core (process pool)
  also       the FOS-step (4,096 x h4 over 100,000 x 8) and uneven-heights
             (8,192 x h3..7 over 200,000 x 10) workloads: graph form,
             roofline and parity

The oracle leg (the target y of each workload, the parity sample and the
CPU baselines) is the only part that runs the oracle package; the timed
path runs the CUDA library alone.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = ("node-row evals/sec and trial fitness evals/sec at scaled-MSE rel err ≤1e-4, "
          "batched vs plain")
UNIT = "node-row evals/s"
CFG = "c5"
EXTRA_CFGS = ("c2", "c3")
SMS, FP32_LANES, SFU_LANES = 152, 128, 16
# operations per evaluated node (by class) and per row-trial for the
# fitness sums (shift, sum d, sum d^2, sum d*y).  FP32: the algorithmic
# count (the operator's own arithmetic, as if sin / cos / log were one SFU
# operation plus a range reduction).  SFU: the MUFU instructions the kernels
# issue: rsqrt (AQ, sqrt), ex2 (exp), one reciprocal in log's reduction and
# in division, lg2 + ex2 for pow; sin and cos run as FMA polynomials and
# issue none.
OPS_FP32 = {"term": 0, "addsubmul": 1, "aq": 2, "div": 1, "sincos": 2, "exp": 1, "log": 1,
            "sqrt": 0, "square": 1, "pow": 1}
OPS_SFU = {"term": 0, "addsubmul": 0, "aq": 1, "div": 1, "sincos": 0, "exp": 1, "log": 1,
           "sqrt": 1, "square": 0, "pow": 2}
ACC_FP32 = 4
# the adjoint's reverse sweep, per node by class: the local derivatives and
# the adjoint times each of them (one per operand); the forward recompute
# counts as OPS_FP32 / OPS_SFU on the unfolded program
OPS_REV_FP32 = {"term": 0, "addsubmul": 2, "aq": 6, "div": 3, "sincos": 3, "exp": 2, "log": 1,
                "sqrt": 2, "square": 2, "pow": 3}
OPS_REV_SFU = {"term": 0, "addsubmul": 0, "aq": 1, "div": 1, "sincos": 0, "exp": 1, "log": 1,
               "sqrt": 1, "square": 0, "pow": 4}
TUNE_STEPS = 20  # Adam steps of the constant-tuning report (grad mode)
PARITY_TRIALS = 64  # timed trials compared with the oracle per workload
# DRAM bytes (read + write) of one batched-forward launch from an ncu
# capture, keyed by (workload, hash of the forward kernel's sources at the
# time of the capture, FWD_SOURCES); reported only while they still match
NCU_TRAFFIC: dict = {
    # dram__bytes_read.sum 196,295,680 + dram__bytes_write.sum 487,198,720: X and
    # y from HBM (44 MB, re-read by later trial groups through L2) and the
    # per-(trial, tile) partial records (16,384 x 977 x 32 B = 512 MB)
    ("large-16384xh6-1000000x10", "8cffde60a4ef550f"): 683_494_400,
    # 4,984,320 + 2,560: X, y and programs once; partial records stay in L2
    ("fos-step-4096xh4-100000x8", "8cffde60a4ef550f"): 4_986_880,
}
STAT_COLS = {"term": 1, "addsubmul": 2, "aq": 3, "div": 4, "sincos": 5, "exp": 6, "log": 7,
             "sqrt": 8, "square": 9, "pow": 12}
# the same classes after constant folding (the nodes evaluated on every row)
EXEC_COLS = {"term": 14, "addsubmul": 15, "aq": 16, "div": 17, "sincos": 18, "exp": 19,
             "log": 20, "sqrt": 21, "square": 22, "pow": 23}


# the sources the batched forward kernel is compiled from (its includes and
# the generator of its PTX interpreter)
FWD_SOURCES = ("kernels.cuh", "device.cuh", "gmath.cuh", "isa.h", "fwd.cu", "fwd_pow.cu",
               "interp_gen.py")


def source_hash(names=None):
    """Hash of the CUDA sources and the C header the library is built from
    (or of the named files of csrc/ only)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2605_30954_gb300", "csrc")
    if names is None:
        files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc)
                       if f.endswith((".cu", ".cuh", ".h", ".py")))
        files.append(os.path.join(ROOT, "include", "ggeval.h"))
    else:
        files = [os.path.join(csrc, f) for f in names]
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


_PEAKS = {}


def measured_peaks(gg, dev):
    """FP32 and SFU issue rates (Gop/s) measured in this process by the
    library's microbenchmarks (ggeval_pipe_rates): FP32 = the faster of
    FFMA and FFMA2 chains, SFU = the median of the rsqrt, ex2, lg2 and sin
    chains."""
    if dev not in _PEAKS:
        r = gg.pipe_rates(dev)
        sfu = sorted(r[k] for k in ("rsqrt", "ex2", "lg2", "sin"))
        _PEAKS[dev] = {"fp32": max(r["ffma"], r["ffma2"]) / 1e9,
                       "sfu": 0.5 * (sfu[1] + sfu[2]) / 1e9,
                       "rates_gops": {k: v / 1e9 for k, v in r.items()}}
    return _PEAKS[dev]


def pipe_roofline(alg_fp32, alg_sfu, ms, peaks, sm_mhz):
    """Two-pipe roofline of an interpreter kernel: the achieved rate of the
    algorithmic FP32 and SFU operations against the measured peaks; the
    pipe with the larger fraction bounds the kernel and gives the headline
    fields."""
    fp = alg_fp32 / (ms * 1e-3) / 1e9
    sf = alg_sfu / (ms * 1e-3) / 1e9
    out = {"fp32": {"achieved": fp, "peak": peaks["fp32"], "frac": fp / peaks["fp32"]},
           "sfu": {"achieved": sf, "peak": peaks["sfu"], "frac": sf / peaks["sfu"]}}
    pipe = "sfu" if out["sfu"]["frac"] > out["fp32"]["frac"] else "fp32"
    return {"bound": "alu", "pipe": pipe, "achieved": out[pipe]["achieved"],
            "peak": out[pipe]["peak"], "unit": "Gop/s", "frac": out[pipe]["frac"],
            **out,
            "peak_basis": ("measured in this process by ggeval_pipe_rates (FP32: faster of "
                           "FFMA / FFMA2 chains; SFU: median of rsqrt, ex2, lg2, sin chains); "
                           f"nominal at the sampled {sm_mhz:.0f} MHz: "
                           f"{SMS * FP32_LANES * sm_mhz / 1e3:.0f} / "
                           f"{SMS * SFU_LANES * sm_mhz / 1e3:.0f} Gop/s"),
            "pipe_rates_gops": peaks["rates_gops"]}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=CFG, choices=sorted(synth.CONFIGS))
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baselines")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads")
    ap.add_argument("--mode", default="eval", choices=["eval", "grad", "sweep"],
                    help="eval: one batched FOS-step evaluation per step (the headline); "
                         "grad: fitness + adjoint + one Adam step per step; "
                         "sweep: a whole FOS sweep on the device per step")
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(step_ms_total, steps, nodes, trials, rows, allreduce, ops):
    """Whole-job numbers over all ranks: the step time is the MAX over ranks
    (the slowest rank bounds the job), the work is the SUM (every rank
    evaluates its own FOS step of trials; no data moves between ranks)."""
    t_max = allreduce(float(step_ms_total), ops["max"])
    n_sum = allreduce(float(nodes), ops["sum"])
    p_sum = allreduce(float(trials), ops["sum"])
    ms = t_max / steps
    return {"ms_per_step": ms, "node_row_evals_per_s": n_sum * rows / (ms * 1e-3),
            "trial_evals_per_s": p_sum / (ms * 1e-3), "nodes": n_sum, "trials": p_sum}


# ------------------------------------------------------------ oracle leg --
# Everything in this section runs the FP64 oracle on the host: the target of
# each workload (the same computation the parity tests use), the parity
# sample of the timed outputs and the CPU baselines.

def oracle_workload(cfg, rep):
    """Seeded workload with its target y from the oracle's evaluation of the
    first usable generator tree (as in the parity tests)."""
    import oracle.parity as OP
    w = synth.workload(cfg, rep)
    if "y" not in w:
        w["y"], _ = OP.target_from_oracle(w)
    return w


def oracle_parity(w, smse, mse, n=PARITY_TRIALS, seed=5):
    """The timed outputs of n sampled trials against the oracle at the full
    row count (spawn-started process pool over the host cores)."""
    import oracle.parity as OP
    trials = sorted(np.random.default_rng(seed).choice(w["P"], min(n, w["P"]),
                                                       replace=False).tolist())
    t0 = time.perf_counter()
    t = OP.check_fitness(w, trials, smse, mse)
    d = t.as_dict()
    d.update(trials_sampled=len(trials), seconds=round(time.perf_counter() - t0, 1),
             tolerance="|g - r| <= 1e-4 r + 1e-8 Var(y)", ok=t.failed == 0)
    if t.msgs:
        d["first_failures"] = t.msgs[:3]
    return d


_POOL_W = None


def _pool_init(w):
    global _POOL_W
    _POOL_W = w


def _oracle_trials(idx):
    """Worker of the all-cores oracle timing: fitness of the given trials."""
    import oracle as O
    w = _POOL_W
    nodes = 0
    for p in idx:
        t = O.Template(w["op"][p], w["cval"][p], int(w["heights"][p]), w["layout"], w["F"])
        try:
            O.fitness(O.eval_tree(t, w["X"]), w["y"])
            nodes += int(O.active_mask(t).sum())
        except O.InvalidTemplate:
            pass
    return nodes


def cpu_baseline_all_cores(w, per_trial_s, seconds):
    """The same oracle on every host core: a spawn-started process pool (safe
    after GPU work in this process), trials split evenly, sized so the timed
    part takes about `seconds`."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = int(min(w["P"], max(cores, seconds * cores / max(per_trial_s, 1e-9))))
    idx = np.arange(n)
    chunks = [c.tolist() for c in np.array_split(idx, cores) if len(c)]
    ww = {k: w[k] for k in ("op", "cval", "heights", "layout", "F", "X", "y")}
    with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn"),
                                initializer=_pool_init, initargs=(ww,)) as ex:
        list(ex.map(_oracle_trials, [[0]] * cores))  # start-up (imports) outside the timing
        t0 = time.perf_counter()
        nodes = sum(ex.map(_oracle_trials, chunks))
        el = time.perf_counter() - t0
    return {"value": nodes * w["N"] / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "trial_evals_per_s": n / el,
            "sample": f"first {n} of {w['P']} trials at all {w['N']} rows split over {cores} "
                      f"processes ({el:.1f} s, FP64 numpy)"}


def cpu_baseline(w, seconds, torch):
    """Time the FP64 oracle (as it stands) on a sample of the workload's
    trials at the full row count, on one host core."""
    import oracle as O
    torch.set_num_threads(1)
    P, N = w["P"], w["N"]
    y = w["y"]
    t0 = time.perf_counter()
    done = nodes = 0
    while done < P and time.perf_counter() - t0 < seconds:
        t = O.Template(w["op"][done], w["cval"][done], int(w["heights"][done]), w["layout"], w["F"])
        try:
            O.fitness(O.eval_tree(t, w["X"]), y)
            nodes += int(O.active_mask(t).sum())
        except O.InvalidTemplate:
            pass
        done += 1
    el = time.perf_counter() - t0
    return {"value": nodes * N / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "trial_evals_per_s": done / el,
            "sample": f"first {done} of {P} trials at all {N} rows ({el:.1f} s, FP64 numpy)"}


def run_reference(a):
    """The reference arm: the FP64 oracle on the host cores, each step a
    bounded sample of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    import torch
    torch.set_num_threads(1)
    w = oracle_workload(a.config, 0)
    y = w["y"]
    per_step = 1
    idx = 0

    def step():
        nonlocal idx
        nodes = 0
        for _ in range(per_step):
            p = idx % w["P"]
            idx += 1
            t = O.Template(w["op"][p], w["cval"][p], int(w["heights"][p]), w["layout"], w["F"])
            O.fitness(O.eval_tree(t, w["X"]), y)
            nodes += int(O.active_mask(t).sum())
        return nodes

    t0 = time.perf_counter()
    step()
    per_trial = time.perf_counter() - t0
    # size each step so the whole run takes about cpu_seconds of host time
    per_step = max(1, int(a.cpu_seconds / max(a.steps + a.warmup, 1) / per_trial))
    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    nodes = sum(step() for _ in range(a.steps))
    el = time.perf_counter() - t0
    v = nodes * w["N"] / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "trials_per_step": per_step,
                                        "rows": w["N"], "flush_l2": False},
        "trial_evals_per_s": per_step * a.steps / el,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} trials per step at all {w['N']} rows"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# -------------------------------------------------------------- GPU legs --
def node_counts(gg, torch, w):
    st = gg.batch_stats(torch.from_numpy(w["op"]), torch.from_numpy(w["cval"]),
                        torch.from_numpy(w["heights"]) if "h_min" in synth.CONFIGS[w["cfg"]] else None,
                        n_features=w["F"]).numpy()
    ok = st[:, 0] >= 0
    nodes = int(st[ok, 0].sum())
    # algorithmic operations of what runs per row: the program after folding
    fp32 = sum(OPS_FP32[k] * int(st[ok, c].sum()) for k, c in EXEC_COLS.items())
    sfu = sum(OPS_SFU[k] * int(st[ok, c].sum()) for k, c in EXEC_COLS.items())
    return nodes, fp32, sfu, int(ok.sum()), int(st[ok, 13].sum())


class Runner:
    """One workload on one GPU: dataset, device batch, side stream, timing."""

    def __init__(self, gg, torch, w, dev, barrier):
        self.gg, self.torch, self.w, self.dev, self.barrier = gg, torch, w, dev, barrier
        self.PF = gg.F_POW if w["uses_pow"] else 0  # kernels with pow, for a pow function set
        self.ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]), device=dev)
        self.op = torch.from_numpy(w["op"]).cuda(dev)
        self.cv = torch.from_numpy(w["cval"]).cuda(dev)
        self.hs = (torch.from_numpy(w["heights"]).cuda(dev)
                   if "h_min" in synth.CONFIGS[w["cfg"]] else None)
        self.st = torch.cuda.Stream(dev)
        self.outs = [torch.empty(w["P"], device=f"cuda:{dev}") for _ in range(4)]
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32,
                                 device=f"cuda:{dev}")
        self.ds.autotune(self.op, self.cv, self.hs, flags=self.PF)
        self.cfg = self.ds.tile_config(self.op, self.cv, self.hs, flags=self.PF)
        torch.cuda.synchronize()

    def graph_step(self):
        self.ds.eval_batch(self.op, self.cv, self.hs, flags=self.gg.F_GRAPH | self.PF,
                           stream=self.st, out=self.outs)

    def prof_step(self):
        self.ds.eval_batch(self.op, self.cv, self.hs, flags=self.gg.F_PROFILE | self.PF,
                           stream=self.st, out=self.outs)

    def timed(self, fn, steps, clocks=None, name="timed"):
        """Sum of per-step CUDA-event times (ms) on the side stream, L2
        flushed before every step."""
        torch = self.torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        self.barrier()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        torch.cuda.nvtx.range_push(name)
        for i in range(steps):
            with torch.cuda.stream(self.st):
                self.flush.fill_(float(i))
                ev[i][0].record(self.st)
                fn()
                ev[i][1].record(self.st)
        self.st.synchronize()
        torch.cuda.nvtx.range_pop()
        self.barrier()
        ck = clocks.stop() if clocks else None
        return float(np.sum([e0.elapsed_time(e1) for e0, e1 in ev])), ck

    def warm(self, fn, n):
        for _ in range(n):
            with self.torch.cuda.stream(self.st):
                fn()
        self.st.synchronize()

    def roofline(self, steps, fp32_ops, sfu_ops, valid, fallback_ck):
        """The batched forward kernel alone: CUDA events around it on its
        launching stream (GGEVAL_F_PROFILE), eager launches."""
        self.warm(self.prof_step, 2)
        self.ds.profile_read()
        clocks = Clocks(self.dev)
        eager_ms, ck = self.timed(self.prof_step, steps, clocks, "timed_eager")
        fwd_ms, launches = self.ds.profile_read()
        fwd_avg = fwd_ms / max(launches, 1)
        w = self.w
        N = w["N"]
        sm_mhz = (ck or fallback_ck or {}).get("sm_mhz") or 1477.0
        alg_fp32 = (fp32_ops + ACC_FP32 * valid) * N  # per launch
        alg_sfu = sfu_ops * N
        x_bytes = (w["F"] + 1) * N * 4
        traffic = NCU_TRAFFIC.get((w["name"], source_hash(FWD_SOURCES)))
        roof = pipe_roofline(alg_fp32, alg_sfu, fwd_avg, measured_peaks(self.gg, self.dev), sm_mhz)
        return {**roof, "traffic": traffic,
                "kernel": "fwd_kernel (batched forward)", "kernel_ms": fwd_avg,
                "algorithmic_fp32_ops_per_launch": alg_fp32,
                "algorithmic_sfu_ops_per_launch": alg_sfu,
                "hbm_gbs": x_bytes / (fwd_avg * 1e-3) / 1e9,
                "eager_ms_per_step": eager_ms / steps, "clocks": ck}

    def close(self):
        self.ds.close()


def extra_workload(gg, torch, cfg, a, dev, barrier):
    """A smaller workload in the same process: graph-form throughput,
    roofline and parity (no plain form, end-to-end or CPU legs)."""
    w = oracle_workload(cfg, 0)
    nodes, fp32_ops, sfu_ops, valid, nodes_eval = node_counts(gg, torch, w)
    r = Runner(gg, torch, w, dev, barrier)
    r.warm(r.graph_step, a.warmup)
    clocks = Clocks(dev)
    tot_ms, ck = r.timed(r.graph_step, a.steps, clocks, "timed_graph_" + cfg)
    ms = tot_ms / a.steps
    smse, mse = r.outs[0].cpu().numpy(), r.outs[3].cpu().numpy()
    r.ds.sync(r.st)
    roof = r.roofline(a.steps, fp32_ops, sfu_ops, valid, ck)
    cfg_used = r.cfg
    r.close()
    return {"workload": w["name"], "value": nodes * w["N"] / (ms * 1e-3), "unit": UNIT,
            "trial_evals_per_s": w["P"] / (ms * 1e-3), "ms_per_step": ms,
            "nodes_evaluated_per_row_per_step": nodes_eval,
            "tile_config": {"variant": cfg_used[0], "tile_rows": cfg_used[1],
                            "group": cfg_used[2], "warps": cfg_used[3]},
            "roofline": roof, "clocks": ck, "parity": oracle_parity(w, smse, mse)}


def fos_csr(stride):
    """One FOS subset per template node: the node and its children."""
    subsets = [[i] + [c for c in (2 * i + 1, 2 * i + 2) if c < stride] for i in range(stride)]
    off = np.cumsum([0] + [len(x) for x in subsets]).astype(np.int32)
    return off, np.concatenate(subsets).astype(np.int32)


def run_extra_mode(a, gg, torch):
    """--mode grad / sweep on one GPU (documentation lines, not the headline)."""
    dev = 0
    torch.cuda.set_device(dev)
    w = oracle_workload(a.config, 0)
    PF = gg.F_POW if w["uses_pow"] else 0  # kernels with pow, for a pow function set
    nodes, _, _, valid, _ = node_counts(gg, torch, w)
    N, P = w["N"], w["P"]
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]), device=dev)
    op = torch.from_numpy(w["op"]).cuda(dev)
    cv = torch.from_numpy(w["cval"]).cuda(dev)
    hs = torch.from_numpy(w["heights"]).cuda(dev) if "h_min" in synth.CONFIGS[a.config] else None
    ds.autotune(op, cv, hs, flags=PF)
    st = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "trials_per_step": P, "rows": N,
                       "active_nodes": nodes, "mode": a.mode}}
    if a.mode == "grad":
        m = torch.zeros_like(cv)
        v = torch.zeros_like(cv)
        smse = torch.empty(P, device="cuda")
        dc = torch.empty_like(cv)
        # the adjoint kernel alone: CUDA events around it (roofline)
        st_ = gg.batch_stats(torch.from_numpy(w["op"]), torch.from_numpy(w["cval"]),
                             torch.from_numpy(w["heights"]) if hs is not None else None,
                             n_features=w["F"]).numpy()
        ok = st_[:, 0] >= 0
        alg_fp32 = sum((OPS_FP32[k] + OPS_REV_FP32[k]) * int(st_[ok, c].sum())
                       for k, c in STAT_COLS.items()) * N
        alg_sfu = sum((OPS_SFU[k] + OPS_REV_SFU[k]) * int(st_[ok, c].sum())
                      for k, c in STAT_COLS.items()) * N
        with torch.cuda.stream(st):
            for _ in range(2):
                ds.grad_batch(op, cv.clone(), hs, flags=PF | gg.F_PROFILE, stream=st,
                              smse=smse, dcval=dc)
        st.synchronize()
        ds.profile_read()
        clocks = Clocks(dev)
        clocks.start()
        time.sleep(0.3)
        with torch.cuda.stream(st):
            for _ in range(a.steps):
                ds.grad_batch(op, cv.clone(), hs, flags=PF | gg.F_PROFILE, stream=st,
                              smse=smse, dcval=dc)
        st.synchronize()
        ck = clocks.stop()
        adj_ms, launches = ds.profile_read()
        adj_avg = adj_ms / max(launches, 1)
        sm_mhz = (ck or {}).get("sm_mhz") or 1477.0
        roof = pipe_roofline(alg_fp32, alg_sfu, adj_avg, measured_peaks(gg, dev), sm_mhz)
        line["roofline"] = {
            **roof, "kernel": "adjoint (bin + one launch per length class: forward recompute + "
                              "reverse sweep)",
            "kernel_ms": adj_avg,
            "algorithmic_fp32_ops_per_launch": alg_fp32,
            "algorithmic_sfu_ops_per_launch": alg_sfu,
            "traffic": None, "clocks": ck}

        def step(t):
            ds.grad_batch(op, cv, hs, flags=PF, stream=st, smse=smse, dcval=dc)
            gg.adam_step(op, cv, dc, m, v, t, lr=0.05, stream=st)
        with torch.cuda.stream(st):
            s0 = ds.eval_batch(op, cv, hs, flags=PF, stream=st)[0].clone()
            for t in range(1, a.warmup + 1):
                step(t)
        st.synchronize()
        e0, e1 = ev(), ev()
        with torch.cuda.stream(st):
            e0.record(st)
            for t in range(a.warmup + 1, a.warmup + 1 + a.steps):
                step(t)
            e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        # constant tuning runs 20 Adam steps per trial in all (untimed past the
        # timed region) before the improvement is reported
        t_done = a.warmup + a.steps
        with torch.cuda.stream(st):
            for t in range(t_done + 1, TUNE_STEPS + 1):
                step(t)
        st.synchronize()
        t_done = max(t_done, TUNE_STEPS)
        s1 = ds.eval_batch(op, cv, hs, flags=PF)[0]
        ds.sync()
        fin = torch.isfinite(s0) & torch.isfinite(s1)
        line.update(value=nodes * N / (ms * 1e-3), ms_per_step=ms,
                    gradient_trial_evals_per_s=P / (ms * 1e-3),
                    note="node-row evals of the forward pass; each step also runs the "
                         "adjoint (forward recompute + reverse sweep) and one Adam step",
                    tuning={"adam_steps": t_done,
                            "trials_improved": int((s1[fin] < s0[fin]).sum().item()),
                            "median_smse_ratio": float((s1[fin & (s0 > 0)] / s0[fin & (s0 > 0)])
                                                       .median().item())})
    else:  # sweep
        stride = op.shape[1]
        off, fnodes = fos_csr(stride)
        rng = np.random.default_rng(1)
        order = torch.from_numpy(np.argsort(rng.random((stride, P)), axis=0).astype(np.int32)).cuda()
        donors = torch.from_numpy(rng.integers(0, P, (stride, P)).astype(np.int32)).cuda()
        off_d, nodes_d = torch.from_numpy(off).cuda(), torch.from_numpy(fnodes).cuda()
        pop_op, pop_cv = op.clone(), cv.clone()
        O_op, O_cv, B_op, B_cv = op.clone(), cv.clone(), op.clone(), cv.clone()
        f_b = ds.eval_batch(O_op, O_cv, hs, flags=PF)[0].clone()
        f_new = torch.empty(P, device="cuda")
        changed_total = torch.zeros((), dtype=torch.int64, device="cuda")

        def sweep():
            chs = []  # each step's changed flags (distinct buffers), counted once per sweep
            for i in range(stride):
                gg.gom_donate(O_op, O_cv, pop_op, pop_cv, donors[i], order[i], off_d, nodes_d,
                              stream=st)
                ch = gg.gom_changed(O_op, O_cv, B_op, B_cv, w["F"], hs, stream=st)
                chs.append(ch)
                ds.eval_batch_masked(O_op, O_cv, ch, hs, flags=PF, stream=st,
                                     out=[f_new, None, None, None])
                gg.gom_accept(O_op, O_cv, B_op, B_cv, f_new, f_b, ch, stream=st)
            changed_total.add_(torch.stack(chs).sum())
        with torch.cuda.stream(st):
            sweep()  # sizes the workspace and tunes the plan outside the capture
        st.synchronize()
        # the whole sweep (one GOM step per FOS subset) as one CUDA graph
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            sweep()
        st.synchronize()
        changed_total.zero_()
        e0, e1 = ev(), ev()
        with torch.cuda.stream(st):
            e0.record(st)
            for _ in range(a.steps):
                graph.replay()
            e1.record(st)
        st.synchronize()
        ds.sync(st)
        ms = e0.elapsed_time(e1) / a.steps
        evals = changed_total.item() / a.steps
        line.update(value=evals * (nodes / P) * N / (ms * 1e-3), ms_per_step=ms,
                    fos_steps_per_s=stride / (ms * 1e-3),
                    changed_trial_evals_per_s=evals / (ms * 1e-3),
                    note="one step = a full FOS sweep (%d subsets) on the device, replayed "
                         "as one CUDA graph: donor copy, changed test, masked evaluation of "
                         "the changed trials, accept or revert; value counts node-rows of the "
                         "evaluated trials with the batch's mean active size" % stride)
    ds.close()
    print(json.dumps(line))


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import torch
    import paper_2605_30954_gb300 as gg
    if a.mode != "eval":
        return run_extra_mode(a, gg, torch)

    rank, world, local = dist_env()
    dev = local
    torch.cuda.set_device(dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    def allreduce(x, op):
        if not pg:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=op)
        return t.item()

    ops = {"max": pg.ReduceOp.MAX if pg else None, "sum": pg.ReduceOp.SUM if pg else None}

    w = oracle_workload(a.config, rank)
    nodes, fp32_ops, sfu_ops, valid, nodes_eval = node_counts(gg, torch, w)
    N, P = w["N"], w["P"]
    r = Runner(gg, torch, w, dev, barrier)

    # ---- batched form, graph replay (the headline) ----
    r.warm(r.graph_step, a.warmup)
    clocks = Clocks(dev)
    tot_ms, ck = r.timed(r.graph_step, a.steps, clocks, "timed_graph")
    agg = aggregate(tot_ms, a.steps, nodes, P, N, allreduce, ops)
    ms_step = agg["ms_per_step"]
    all_nodes, all_trials = agg["nodes"], agg["trials"]
    r.ds.sync(r.st)
    timed_smse, timed_mse = r.outs[0].cpu().numpy(), r.outs[3].cpu().numpy()
    # trials whose fitness is +inf: the batched form stops evaluating such a
    # trial after its first non-finite tile (node-rows still count them all)
    nonfinite = int((~np.isfinite(timed_smse)).sum())

    # ---- forward kernel alone: live CUDA events around it (roofline) ----
    roof = r.roofline(a.steps, fp32_ops, sfu_ops, valid, ck)

    # ---- plain form: one launch per trial ----
    def plain_step():
        r.ds.eval_plain(r.op, r.cv, r.hs, flags=r.PF, stream=r.st, out=r.outs)
    r.warm(plain_step, 1)
    plain_ms, _ = r.timed(plain_step, a.plain_steps, name="timed_plain")
    plain_step_ms = allreduce(plain_ms, ops["max"]) / a.plain_steps
    plain_trials = all_trials / (plain_step_ms * 1e-3)

    # ---- end to end through the C ABI with pinned host buffers ----
    hop = torch.from_numpy(w["op"]).pin_memory()
    hcv = torch.from_numpy(w["cval"]).pin_memory()
    hhs = torch.from_numpy(w["heights"]).pin_memory() if r.hs is not None else None
    hout = [torch.empty(P, dtype=torch.float32).pin_memory(), None, None, None]

    def e2e_step():
        r.ds.eval_batch(hop, hcv, hhs, flags=r.PF, stream=r.st, out=hout)
    r.warm(e2e_step, a.warmup)
    e2e_ms, _ = r.timed(e2e_step, a.steps, name="timed_e2e")
    e2e_ms = allreduce(e2e_ms, ops["max"]) / a.steps
    h2d = w["op"].nbytes + w["cval"].nbytes + (w["heights"].nbytes if r.hs is not None else 0)
    r.ds.sync(r.st)
    cfg_used = r.cfg
    r.close()

    line = {
        "metric": METRIC, "value": agg["node_row_evals_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "trials_per_step": P, "rows": N,
                   "features": w["F"], "template_height": w["h_max"],
                   "active_nodes_per_step": nodes,
                   "nodes_evaluated_per_row_per_step": nodes_eval,
                   "trials_with_infinite_fitness": nonfinite,
                   "flush_l2": "512 MB write between steps",
                   "form": "persistent batched kernel, CUDA graph replay, autotuned tiles",
                   "tile_config": {"variant": cfg_used[0], "tile_rows": cfg_used[1],
                                   "group": cfg_used[2], "warps": cfg_used[3]},
                   "parallelism": f"replicas x{world} (independent FOS steps)"},
        "trial_evals_per_s": agg["trial_evals_per_s"],
        "plain": {"trial_evals_per_s": plain_trials, "ms_per_step": plain_step_ms,
                  "node_row_evals_per_s": all_nodes * N / (plain_step_ms * 1e-3),
                  "launches_per_step": 2 * P + 2},
        "batched_over_plain": agg["trial_evals_per_s"] / plain_trials,
        "e2e": {"value": all_nodes * N / (e2e_ms * 1e-3), "unit": UNIT,
                "trial_evals_per_s": all_trials / (e2e_ms * 1e-3), "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(4 * P)},
        "roofline": roof,
        "gpu_launches": 3 * a.steps,
        "clocks": ck,
        "kernel_sources": source_hash(),
    }
    if rank == 0:
        line["parity"] = oracle_parity(w, timed_smse, timed_mse)
    if rank == 0 and world == 1 and not a.no_cpu:
        line["cpu_baseline"] = cb = cpu_baseline(w, a.cpu_seconds, torch)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(
            w, 1.0 / cb["trial_evals_per_s"], a.cpu_seconds)
    if world == 1 and not a.no_extra:
        line["also"] = [extra_workload(gg, torch, c, a, dev, barrier)
                        for c in EXTRA_CFGS if c != a.config]
    if pg:
        pg.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
