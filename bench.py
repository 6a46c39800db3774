"""Benchmark of the unbinned-likelihood hot path on GB300.

Workload (one GPU): the 4D decay-time x helicity-angle model on 1e6 FP64 SoA
events (t, cos thK, cos thmu, phi) distributed like the PDF at the truth
(generated by ipa_toygen before the timed region), 10 parameters.  One step = one
ipa_nll_grad call: parameter constants + fused PDF / log / analytic adjoint +
deterministic FP64 reduction, i.e. one minimiser iteration's event pass.
The metric is NLL+grad Gevents/s.  Inputs (32 MB) are smaller than L2, so L2
is flushed (256 MB write) before every timed step.

Also reported on the same JSON line:
  e2e           the same metric through the C ABI with host buffers
                (ipa_nll_grad_host: the step's pinned host columns copied in
                chunks overlapped with the event pass) and the device -> host
                copy of NLL and gradient, every step;
  roofline      FP64-pipe roofline of the fused kernel (bound "alu");
  cpu_baseline  the CPU oracle on a bounded sample of the same workload;
  fit / toygen / batch   full fit of the 1e6-event sample, 4D toy generation
                of the 4096-toy batch, batched toy fits vs one-fit-at-a-time;
  large / serve large weighted event sets, the fit server under load;
  tagged        the flavour-tagged model with B_s oscillation (1e6 events):
                NLL+grad rate and roofline, generator, batched fits, CPU oracle;
  errors / cls  HESSE and MINOS of the toy batch; Example 4's CLs toys;
  phis          the time-dependent angular model with tagging (1e6 events);
  phis_joint    Example 2's twelve-category simultaneous fit at 1e4 and 1e7
                events generated from the model: joint NLL+grad rate and the
                whole fit's wall time.

`--impl reference` times the CPU oracle on the same workload and metric.
Multi-GPU (torchrun): every rank runs an independent replica (the path is one
GPU; there is no data-path collective); value = total events / max time.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EVENTS = 1_000_000
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
METRIC = "NLL+grad Gevents/s"
WORKLOAD = "4D angular+time unbinned NLL+grad, 1e6 FP64 SoA events, 10 params"

# FP64 operations of the fused 4D NLL+gradient kernel, counted from the formula
# as nll.cu evaluates it on whole tiles (FMA = 2 flops; each FP64 function call
# counts its cost in DFMA issue slots measured live by ipa_calibrate_fp64, times
# 2 flops).  The angular basis (sin/cos, the ten products, the square root,
# the amplitude sum A'), the Gaussian's exp, the ten angular adjoint sums S_k
# (64-bit fixed point) and the lane's product of the P mantissas run on the
# integer pipe and count no FP64 operation; only their arguments and results do:
#   every event: tau, the exponent of 2E and 2E itself (the table-driven FP64
#     exp, its measured slots), T2 = 2E - X (computed for every
#     event, selected for the near-peak ones), P, 1/P (an FP32 seed and one
#     FP64 Newton step: 2 FMA), sum r, r T2 (then fixed point), r A', u = r A'
#     tau and the three sums u T2, r A' Gx, u Gx (Gx = 0 away from the peak);
#   unweighted: the lane's product of the P mantissas (one multiply);
#     weighted: w log P, w / P and the product (by 1 or P);
#   events near the resolution peak (t <= mu + Gamma sigma^2 + 6.25 sqrt2 sigma,
#     packed 32 to a warp pass): tau, the Gaussian's exponent (tau^2 k_g), the
#     erfcx argument ((Gs2 - tau) k_z), erfcx (FP64 polynomial) and g X;
#   once per lane and 512-event tile (16 events): the log of the product and
#     its exponent term.
# (Angles within 2^-17 of |cos| = 1, about 1.5e-5 of the events, take the FP64
# basis instead; they are not counted.)
OPS_EVENT_4D = {"fma": 7, "mul": 3, "add": 3, "exp_fast": 1}
OPS_UNWEIGHTED = {"mul": 1}
OPS_WEIGHTED = {"fma": 1, "mul": 2, "log_fast": 1}
OPS_NEAR_PEAK = {"mul": 4, "add": 2, "erfcx_poly": 1}
OPS_LANE_TILE = {"fma": 2, "log_fast": 1}


# The same formula evaluated with CUDA's FP64 library functions (what the paper's
# kernels call: exp, erfc and log per event, sincos and sqrt for the angles),
# each charged its measured cost: the FP64 work the kernel avoids by moving
# functions to the integer pipe and by the algebra above.
OPS_LIBRARY_4D = {"fma": 32, "mul": 30, "add": 6, "exp": 2, "erfc": 1, "log": 1, "sincos": 1, "sqrt": 1, "rcp": 1}


# The flavour-tagged model (IPA_MODEL_TAGGED1D, tagged.cu), counted the same way:
#   every event: tau, three exponents (integer-pipe exp), the oscillation phase
#     (its sine and cosine on the integer pipe), 2 gH, 2 gL, 2 g (complex),
#     q qD and P, 1/P, and the 12 adjoint sums;
#   events with t <= tcut (mu + max(Gamma_H, Gamma_L, Gamma) sigma^2 +
#     sqrt(39.1 + (Dm sigma)^2 / 2) sqrt2 sigma): the Gaussian's exponent, three
#     erfc arguments, the Faddeeva function's division, Z and final
#     combination, and the five products stored for the event (two erfcx and
#     the Faddeeva function's 39 complex Horner steps run on the integer pipe).
OPS_TAG_EVENT = {"fma": 17, "mul": 8, "add": 9}
OPS_TAG_SLOW = {"fma": 8, "mul": 19, "add": 5, "rcp": 1}
TH_TAG = np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.8, 0.3])


def tag_slow_fraction(t, theta) -> float:
    Gamma, sigma, mu, _, DG, Dm = (float(v) for v in theta[:6])
    rmax = max(Gamma - DG / 2, Gamma + DG / 2, Gamma)
    beta = Dm * sigma / math.sqrt(2.0)
    tcut = mu + rmax * sigma * sigma + math.sqrt(39.1 + beta * beta) * math.sqrt(2.0) * sigma
    return float(np.mean(np.asarray(t) <= tcut))


def _flops(ops: dict, cal: dict) -> float:
    f = 0.0
    for k, v in ops.items():
        f += v * (2.0 if k == "fma" else 1.0 if k in ("mul", "add") else 2.0 * cal[k])
    return f


def _slots(ops: dict, cal: dict) -> float:
    return sum(v * (1.0 if k in ("fma", "mul", "add") else cal[k]) for k, v in ops.items())


def slots_per_event(cal: dict, near: float, weighted: bool = False) -> float:
    """FP64 issue slots per event of the same count (each FMA, multiply or add is
    one slot; functions their measured slots): the pipe's own roofline, which a
    flop count understates for multiplies and adds (one flop, one slot)."""
    f = _slots(OPS_EVENT_4D, cal) + near * _slots(OPS_NEAR_PEAK, cal)
    if weighted:
        return f + _slots(OPS_WEIGHTED, cal)
    return f + _slots(OPS_UNWEIGHTED, cal) + _slots(OPS_LANE_TILE, cal) / 16.0


def near_peak_fraction(t, theta) -> float:
    """Fraction of events whose decay time needs the Gaussian and erfcx."""
    Gamma, sigma, mu = float(theta[0]), float(theta[1]), float(theta[2])
    cut = mu + Gamma * sigma * sigma + 6.25 * math.sqrt(2.0) * sigma
    return float(np.mean(np.asarray(t) <= cut))


def flops_per_event(cal: dict, near: float, weighted: bool = False) -> float:
    f = _flops(OPS_EVENT_4D, cal) + near * _flops(OPS_NEAR_PEAK, cal)
    if weighted:
        return f + _flops(OPS_WEIGHTED, cal)
    return f + _flops(OPS_UNWEIGHTED, cal) + _flops(OPS_LANE_TILE, cal) / 16.0


def kernel_traffic(n_events: int, kernel: str = "nll_kernel<4D, grad>"):
    """DRAM bytes per launch of a kernel (read + write, from the committed ncu
    capture in profiles/kernel_counts.json) scaled by events; None if the
    kernel's sources changed since the capture."""
    counts = kernel_counts(kernel)
    return None if counts is None else counts["dram_bytes"] * n_events


def kernel_counts(kernel: str):
    """Per-event counts of a kernel from the committed ncu capture
    (profiles/kernel_counts.json): warp instructions issued, FP64 lane
    operations and DRAM bytes per event; None if the record is missing or the
    kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "kernel_counts.json")
    try:
        rec = json.load(open(path))[kernel]
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, "paper_1706_01420_gb300", "csrc", f), "rb").read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return rec["per_event"]
    except (OSError, ValueError, KeyError):
        return None


# ---- profiles/kernel_counts.json: per-event counts of the likelihood kernels ----
# From the CSV logs of these ncu captures (each after the same command exited
# 0 without ncu):
#   ncu --metrics <COUNT_METRICS> --clock-control none -k regex:<kernel> -s 2 -c 1 --csv \
#       --log-file <dir>/counts_<name>.csv python bench.py --profile-case[-phis|-tagged]
# `python bench.py --write-kernel-counts <dir>` writes the record with a SHA-256
# of the sources each count belongs to; kernel_counts() uses a record only while
# that hash matches.
COUNT_METRICS = ("smsp__inst_executed.sum,smsp__inst_executed_pipe_fp64.sum,"
                 "sm__sass_thread_inst_executed_op_dfma_pred_on.sum,sm__sass_thread_inst_executed_op_dmul_pred_on.sum,"
                 "sm__sass_thread_inst_executed_op_dadd_pred_on.sum,dram__bytes_read.sum,dram__bytes_write.sum,"
                 "gpu__time_duration.sum,smsp__cycles_active.sum,smsp__issue_active.sum")
COUNT_COMMON = ["tile_reduce.cuh", "fp64_math.cuh", "fp64_tables.cuh", "int_math.cuh", "ipa_internal.cuh"]
COUNT_CAPTURES = {
    "nll_kernel<4D, grad>": ("counts_4d.csv", "bench.py --profile-case", 8_000_000,
                             ["nll.cu", "angular.cuh"] + COUNT_COMMON),
    "phis_kernel<grad>": ("counts_phis.csv", "bench.py --profile-case-phis", 8_000_000,
                          ["phis.cu", "phis_consts.cuh", "angular.cuh", "tagged.cuh", "faddeeva.cuh", "consts.cuh",
                           "philox.cuh"] + COUNT_COMMON),
    "tag_kernel<grad>": ("counts_tag.csv", "bench.py --profile-case-tagged", 8_000_000,
                         ["tagged.cu", "tagged.cuh", "faddeeva.cuh", "consts.cuh"] + COUNT_COMMON),
}


def _csv_metrics(path):
    rows = list(csv.reader(open(path)))
    hdr, out = None, {}
    for r in rows:
        if r and r[0] == "ID":
            hdr = r
            continue
        if hdr and len(r) == len(hdr):
            d = dict(zip(hdr, r))
            out[d["Metric Name"]] = float(d["Metric Value"].replace(",", ""))
    return out


def write_kernel_counts(src_dir: str) -> int:
    rec = {}
    for kernel, (fname, cmd, n, files) in COUNT_CAPTURES.items():
        m = _csv_metrics(os.path.join(src_dir, fname))
        h = hashlib.sha256()
        for f in files:
            h.update(open(os.path.join(ROOT, "paper_1706_01420_gb300", "csrc", f), "rb").read())
        fp64 = (m["sm__sass_thread_inst_executed_op_dfma_pred_on.sum"] +
                m["sm__sass_thread_inst_executed_op_dmul_pred_on.sum"] +
                m["sm__sass_thread_inst_executed_op_dadd_pred_on.sum"])
        rec[kernel] = {
            "capture": f"ncu --metrics {COUNT_METRICS} --clock-control none -k regex:{kernel.split('<')[0]} -s 2 -c 1 "
                       f"--csv --log-file {fname} python {cmd}",
            "events": n,
            "duration_us": m["gpu__time_duration.sum"] / 1e3,
            "issue_active_frac": m["smsp__issue_active.sum"] / m["smsp__cycles_active.sum"],
            "per_event": {"warp_inst": m["smsp__inst_executed.sum"] / n,
                          "fp64_warp_inst": m["smsp__inst_executed_pipe_fp64.sum"] / n,
                          "fp64_lane_ops": fp64 / n,
                          "dram_bytes": (m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"]) / n},
            "source_files": files,
            "source_sha256": h.hexdigest(),
        }
    json.dump(rec, open(os.path.join(ROOT, "profiles", "kernel_counts.json"), "w"), indent=1)
    print(json.dumps({k: v["per_event"] for k, v in rec.items()}, indent=1))
    return 0



def max_over_ranks(x: float, device) -> float:
    """Max of a per-rank number over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def cpu_reference_step(O, model, cols, th):
    f, g = O.nll_grad(model, cols, th)
    return f, g


def run_reference(args):
    """The oracle timed on the host cores: same workload, metric and unit."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import ipa_oracle as O
    from paper_1706_01420_gb300 import synth
    n_sample = 100_000
    cols = synth.events_4d(n_sample, 0)
    model = O.Model("4d", 0.0, 15.0)
    for _ in range(args.warmup):
        cpu_reference_step(O, model, cols, TH4)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_reference_step(O, model, cols, TH4)
    dt = time.perf_counter() - t0
    value = n_sample * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gevents/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_events_per_step": n_sample},
            "cpu_baseline": {"value": value, "unit": "Gevents/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n_sample} events of the 4D workload per step (numpy/scipy FP64, "
                                       "single thread)"},
            "e2e": {"value": value, "unit": "Gevents/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- the CPU oracle on the host cores (one worker process per core, spawned) ----
_W = {}


def _w_init(kind: str, n: int, seed: int, chunk: int, n_chunks: int):
    """A worker's chunk [chunk n / n_chunks, (chunk + 1) n / n_chunks) of a seeded
    synthetic workload (each chunk drawn with its own seed; generation untimed)."""
    from oracle import ipa_oracle as O
    from paper_1706_01420_gb300 import synth
    _W.clear()
    m = (chunk + 1) * n // n_chunks - chunk * n // n_chunks
    if kind in ("4d", "4dw"):
        _W.update(model=O.Model("4d", 0.0, 15.0), cols=synth.events_4d(m, seed + chunk, weighted=kind == "4dw"),
                  th=TH4)
    else:
        _W.update(model=O.Model("1d", 0.3, 15.0), cols={"t": synth.events_1d(m, seed + chunk)},
                  th=np.array([0.66, 0.045, 0.0, 0.1]))


def _w_pass():
    from oracle import ipa_oracle as O
    f, g = O.nll_grad(_W["model"], _W["cols"], _W["th"])
    return f, list(g)


def _w_toy(k: int):
    """Toy k of the batched workload (Poisson(2e4) events, seed 0): the oracle's
    generator, then the oracle's fit with all ten parameters free."""
    from oracle import ipa_oracle as O
    from paper_1706_01420_gb300 import synth
    m = O.Model("4d", 0.0, 15.0)
    n_sig, n_bkg = synth.toy_sizes(k + 1, 2e4, TH4[3], seed=0)
    toy = O.toy_one(m, TH4, 0, k, int(n_sig[k]), int(n_bkg[k]))
    lo = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
    hi = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2])
    r = O.fit(m, toy, TH4, list(range(10)), lo, hi, tol=1e-8)
    return r.status


def _w_loop(inq, outq):
    """A worker: runs the commands of its queue until None."""
    while True:
        cmd = inq.get()
        if cmd is None:
            return
        if cmd[0] == "init":
            _w_init(*cmd[1:])
            outq.put(("init", None))
        elif cmd[0] == "pass":
            outq.put(("pass", _w_pass()))
        else:
            outq.put(("toy", _w_toy(cmd[1])))


class _Workers:
    """One spawned process per host core (spawn: safe after CUDA was initialised)."""

    def __init__(self, n: int):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.out = ctx.Queue()
        self.ins = [ctx.Queue() for _ in range(n)]
        self.procs = [ctx.Process(target=_w_loop, args=(q, self.out), daemon=True) for q in self.ins]
        for p in self.procs:
            p.start()

    def run(self, cmds_per_worker: list) -> list:
        for q, cmds in zip(self.ins, cmds_per_worker):
            for c in cmds:
                q.put(c)
        return [self.out.get(timeout=600)[1] for _ in range(sum(len(c) for c in cmds_per_worker))]

    def close(self):
        for q in self.ins:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)


def cpu_baseline(budget_s: float = 12.0) -> dict:
    """The oracle (numpy/scipy FP64, untuned) on the host cores, on bounded
    samples of the workloads: one core and all cores on the 4D workload, the 1D
    workload (passes and a full fit), a 64-toy subset of the batched toys
    (generation and fit per toy, all cores), one pass over the 5e7-event
    weighted workload (all cores), and the tagged model on one core."""
    from oracle import ipa_oracle as O
    from paper_1706_01420_gb300 import synth
    cores = os.cpu_count() or 1
    n = 200_000
    cols = synth.events_4d(n, 0)
    model = O.Model("4d", 0.0, 15.0)
    O.nll_grad(model, cols, TH4)
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s * 0.5:
        O.nll_grad(model, cols, TH4)
        reps += 1
    dt = time.perf_counter() - t0
    out = {"value": n * reps / dt / 1e9, "unit": "Gevents/s", "cores": 1, "kind": "oracle",
           "sample": f"{reps} NLL+grad passes over {n} events of the 4D workload "
                     f"({dt:.1f} s, numpy/scipy FP64, single thread)", "host_cores": cores}
    # the 1D workload on one core: NLL+grad passes and a full fit (Gamma, f_b free)
    t1d = synth.events_1d(100_000, 0)
    m1 = O.Model("1d", 0.3, 15.0)
    th1 = np.array([0.66, 0.045, 0.0, 0.1])
    r1, t0 = 0, time.perf_counter()
    while r1 == 0 or time.perf_counter() - t0 < 1.5:
        O.nll_grad(m1, {"t": t1d}, th1)
        r1 += 1
    d1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    f1 = O.fit(m1, {"t": t1d}, th1 + np.array([0.03, 0, 0, -0.02]), [0, 3], np.array([0.3, 0.01, -0.1, 0.0]),
               np.array([1.5, 0.2, 0.1, 0.5]), tol=1e-10)
    out["config1_1d"] = {"events": 100_000, "cores": 1, "nll_grad_Mevents_per_s": 1e5 * r1 / d1 / 1e6,
                         "fit_wall_s": time.perf_counter() - t0, "fit_status": f1.status}
    # all cores: the 4D workload split over one worker process per core
    ncore = max(1, cores)
    w = _Workers(ncore)
    try:
        w.run([[("init", "4d", n * ncore, 100, i, ncore)] for i in range(ncore)])
        w.run([[("pass",)] for _ in range(ncore)])
        rm, t0 = 0, time.perf_counter()
        while rm == 0 or time.perf_counter() - t0 < budget_s * 0.3:
            w.run([[("pass",)] for _ in range(ncore)])
            rm += 1
        dm = time.perf_counter() - t0
        out["all_cores"] = {"value": n * ncore * rm / dm / 1e9, "unit": "Gevents/s", "cores": ncore,
                            "sample": f"{rm} NLL+grad passes over {n * ncore} events of the 4D workload, "
                                      f"{n} per worker process"}
        # 64 toys of the batched workload, oracle generation + fit, dealt round-robin
        t0 = time.perf_counter()
        st = w.run([[("toy", k) for k in range(i, 64, ncore)] for i in range(ncore)])
        dtoy = time.perf_counter() - t0
        out["config3_toys"] = {"toys": 64, "cores": ncore, "wall_s": dtoy, "toys_per_s": 64 / dtoy,
                               "converged": sum(1 for x in st if x == "CONVERGED"),
                               "sample": "toys 0-63 of Poisson(2e4) events (seed 0): the oracle's generator "
                                         "and fit of all ten parameters per toy"}
        # one NLL+grad pass over 5e7 weighted events, split over the workers
        n5 = 50_000_000
        w.run([[("init", "4dw", n5, 200, i, ncore)] for i in range(ncore)])
        t0 = time.perf_counter()
        w.run([[("pass",)] for _ in range(ncore)])
        d5 = time.perf_counter() - t0
        out["config5_pass"] = {"events": n5, "weighted": True, "cores": ncore, "wall_s": d5,
                               "Gevents_per_s": n5 / d5 / 1e9}
    finally:
        w.close()
    # the tagged model's oracle on 2e4 events (about a second)
    from oracle import tagged as T
    cols_t = synth.events_tagged(20_000, 0)
    model_t = O.Model("tag", 0.0, 15.0)
    reps_t, t1 = 0, time.perf_counter()
    while reps_t == 0 or time.perf_counter() - t1 < 1.0:
        T.nll_grad(model_t, cols_t, TH_TAG)
        reps_t += 1
    dt_t = time.perf_counter() - t1
    out["tagged"] = {"value": 20_000 * reps_t / dt_t / 1e9, "unit": "Gevents/s", "cores": 1,
                     "sample": f"{reps_t} NLL+grad passes over 20000 events of the tagged workload"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip fit/toygen/batch sub-benchmarks")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of single-core oracle timing (0: no CPU baseline, for profiling runs)")
    ap.add_argument("--profile-case", action="store_true",
                    help="untimed: 4 ipa_nll_grad calls on 8e6 4D events (256 MB, > L2), for ncu")
    ap.add_argument("--write-kernel-counts", metavar="DIR",
                    help="write profiles/kernel_counts.json from the ncu CSV logs in DIR and exit")
    ap.add_argument("--profile-events", type=int, default=8_000_000,
                    help="events of --profile-case (1000000: the headline workload's size)")
    ap.add_argument("--profile-case-tagged", action="store_true",
                    help="untimed: 4 ipa_nll_grad calls on 8e6 tagged events (128 MB, > L2), for ncu")
    ap.add_argument("--profile-case-phis", action="store_true",
                    help="untimed: 4 ipa_nll_grad calls on 8e6 phi_s-model events (320 MB, > L2), for ncu")
    ap.add_argument("--profile-case-joint", action="store_true",
                    help="untimed: Example 2's twelve-category fit of 1e4 events, twice, for an ncu launch list")
    args = ap.parse_args()
    if args.write_kernel_counts:
        return write_kernel_counts(args.write_kernel_counts)
    if args.profile_case:
        return profile_case(args.profile_events)
    if args.profile_case_tagged:
        return profile_case_tagged()
    if args.profile_case_phis:
        return profile_case_phis()
    if args.profile_case_joint:
        return profile_case_joint()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_01420_gb300 import api, synth

    cal = api.ipa_calibrate_fp64()
    m = api.model_4d(0.0, 15.0)
    theta = torch.tensor(TH4, device=dev)
    # 1e6 events per GPU distributed like the 4D PDF at the truth: 50 pseudo-
    # experiments of 2e4 events (10 % background) from the library's generator.
    # With N > 1 GPUs the job is ONE likelihood over N x 1e6 events: rank r holds
    # the events shard_bounds(N x 1e6, r, N) (group-aligned, about 1e6 each) and a
    # step is the event-sharded pass (ipa_nll_grad_shard, an all-gather of the
    # group partials, ipa_nll_grad_combine), bitwise the one-GPU result.
    n_total = N_EVENTS * ws
    sharded = None
    if ws > 1:
        from paper_1706_01420_gb300 import shard
        lo, hi = shard.shard_bounds(n_total, rank, ws)
        full = gen_sample(api, torch, dev, m, theta, (hi - lo + 19999) // 20000, 20000, seed=1000 + rank)
        ev = {k: v[:hi - lo].clone() for k, v in full.items()}
        del full
        sharded = shard.ShardedNLL(m, ev, n_total, rank, ws)
    else:
        ev = gen_sample(api, torch, dev, m, theta, 50, 20000, seed=rank)
    cols_h = {k: v.cpu().numpy() for k, v in ev.items()}
    out = torch.empty(11, dtype=torch.float64, device=dev)

    def step():
        if sharded is None:
            api.ipa_nll_grad(m, ev, theta, out)
        else:
            sharded.nll_grad(theta, out)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    api.ipa_reserve(N_EVENTS, 4096)

    # launch geometry: time the built-in default, then let the autotuner pick
    def mean_ms(reps=30):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        api.ipa_nll_grad(m, ev, theta, out)
        a.record(stream)
        for _ in range(reps):
            api.ipa_nll_grad(m, ev, theta, out)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    default_ms = mean_ms()
    picked = api.ipa_autotune(m, ev, theta, grad=True, stream=stream)
    launch = {"picked": picked, "default": api.ipa_launch_config_get(m, 0), "default_step_ms": default_ms,
              "tuned_step_ms": mean_ms()}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(dev.index if dev.index is not None else 0) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                        # evict the 32 MB of inputs from L2
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, dev)
    value = n_total / (ms_max * 1e-3) / 1e9

    # kernel-only time of the dominant kernel, measured with events on its stream:
    # the step is [constants kernel (one block for the fit), fused NLL+grad kernel];
    # a constants-only call (n = 0) is timed alone and subtracted.
    k_ev0, k_ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cons = []
    for i in range(20):
        flush.fill_(float(i))
        k_ev0.record(stream)
        api.ipa_nll(api.model_1d(0.3, 15.0), {"t": ev["t"][:0]}, theta[:4], out)   # consts only (n = 0)
        k_ev1.record(stream)
        torch.cuda.synchronize()
        cons.append(k_ev0.elapsed_time(k_ev1))
    kernel_ms = max(ms - statistics.median(cons), 1e-6)
    near = near_peak_fraction(cols_h["t"], TH4)
    fpe = flops_per_event(cal, near)
    spe = slots_per_event(cal, near)
    peak_dfma_derived = 2.0 * 152 * 2070e6          # DFMA/s: 2 per clock per SM x 152 SMs x 2070 MHz
    achieved = fpe * N_EVENTS / (kernel_ms * 1e-3) / 1e12
    peak = 2.0 * peak_dfma_derived / 1e12
    ops_achieved = spe * N_EVENTS / (kernel_ms * 1e-3) / 1e9
    traffic = kernel_traffic(N_EVENTS)

    # e2e: pinned host columns in, result out, every step, through the host-memory
    # entry point (ipa_nll_grad_host: chunked copies overlapped with the event pass)
    pinned = {k: torch.tensor(v).pin_memory() for k, v in cols_h.items()}
    res_h = torch.empty(11, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in pinned.values())
    ev_copy = {k: torch.empty_like(v) for k, v in ev.items()} if sharded is not None else None

    def e2e_step():
        if sharded is None:
            api.ipa_nll_grad_host(m, pinned, theta, out)
        else:
            for k in ev_copy:
                ev_copy[k].copy_(pinned[k], non_blocking=True)
            sharded.ev = ev_copy
            sharded.nll_grad(theta, out)
        res_h.copy_(out, non_blocking=True)
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = max(20, args.steps // 4)
    e2e_steps = []
    for i in range(n_e2e):
        flush.fill_(float(i))                            # no step reads host lines cached in L2
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_steps.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(sum(e2e_steps) / n_e2e, dev)
    e2e_val = n_total / (e2e_ms * 1e-3) / 1e9

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(api, synth, torch, dev, m, ev, theta, cal)

    clocks = clk.summary()
    counts = kernel_counts("nll_kernel<4D, grad>")
    inst_pe = counts["warp_inst"] if counts else None
    fp64_pe = counts["fp64_lane_ops"] if counts else None
    if counts and traffic is None:
        traffic = counts["dram_bytes"] * N_EVENTS
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    issue_peak = 4.0 * 152 * sm_mhz * 1e6 / 1e9
    issue_achieved = inst_pe * N_EVENTS / (kernel_ms * 1e-3) / 1e9 if inst_pe else None
    line = {
        "metric": METRIC, "value": value, "unit": "Gevents/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "events": n_total, "events_per_gpu": int(ev["t"].numel()),
                   "step": "ipa_nll_grad (a1-a6)" if ws == 1 else
                           "ipa_nll_grad_shard + all-gather of group partials + ipa_nll_grad_combine (a1-a6)",
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "one GPU" if ws == 1 else f"events sharded over {ws} GPUs",
                   "launch": launch},
        "gpu_launches": (2 if ws == 1 else 5) * args.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "Gevents/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 88,
                "ms_per_step": e2e_ms, "l2": "flushed (256 MB write) before every step"},
        "roofline": {"bound": "alu", "resource": "instruction issue (all pipes)",
                     "achieved": issue_achieved, "peak": issue_peak, "unit": "G warp instructions/s",
                     "frac": issue_achieved / issue_peak if issue_achieved is not None else None,
                     "traffic": traffic, "kernel": "nll_kernel<4D, grad>", "kernel_ms": kernel_ms,
                     "warp_instructions_per_event": inst_pe,
                     "peak_note": "4 warp instructions/clk/SM x 152 SMs x the SM clock sampled during the timed "
                                  "region; instructions per event from the ncu capture of the current source "
                                  "(profiles/kernel_counts.json)",
                     "fp64": {"achieved": ops_achieved, "peak": peak_dfma_derived / 1e9, "unit": "G FP64 op/s",
                              "frac": ops_achieved * 1e9 / peak_dfma_derived, "fp64_ops_per_event": spe,
                              "fp64_lane_ops_per_event_ncu": fp64_pe, "near_peak_fraction": near,
                              "peak_note": "FP64 pipe: 2 operations/clk/SM x 152 SMs x 2070 MHz (derived); DFMA loop "
                                           f"measured {cal['dfma_per_s'] * 1e-9:.0f} G/s at {cal['sm_mhz']:.0f} MHz, "
                                           f"{cal['dfma_per_clk_per_sm']:.2f} DFMA/clk/SM"},
                     "flops": {"per_event": fpe, "achieved_tflops": achieved, "peak_tflops": peak,
                               "frac": achieved / peak},
                     "library_formula": {"flops_per_event": _flops(OPS_LIBRARY_4D, cal),
                                         "equivalent_tflops": _flops(OPS_LIBRARY_4D, cal) * N_EVENTS
                                         / (kernel_ms * 1e-3) / 1e12,
                                         "note": "the formula with CUDA FP64 library functions; above the "
                                                 "FP64 peak because the kernel does not evaluate it that way"},
                     "fp64_costs_dfma_slots": {k: round(cal[k], 2) for k in
                                               ("exp_fast", "erfcx_poly", "sincos_fast", "log_fast", "sqrt",
                                                "rcp", "exp", "erfc", "log", "sincos")},
                     "int_pipe_calls_per_event": {"exp_int": near, "angular_basis_q62": 1.0},
                     "int_pipe_time_alone_dfma_slots": {k: round(cal[k], 2) for k in ("exp_int", "sincos_int")}},
        "wall_s_timed_region": wall,
    }
    line.update(extras)
    if "large" in line:
        lg = line["large"]
        near_l = lg.pop("near_peak_fraction")
        spe_w = slots_per_event(cal, near_l, weighted=True)
        lg["fp64_ops_per_event"] = spe_w
        lg["roofline_frac"] = spe_w * lg["events"] / (lg["nll_grad_ms"] * 1e-3) / peak_dfma_derived
        lg["flops_frac"] = flops_per_event(cal, near_l, weighted=True) * lg["events"] / (
            lg["nll_grad_ms"] * 1e-3) / 1e12 / peak
    if rank == 0:
        if args.cpu_budget > 0:
            line["cpu_baseline"] = cpu_baseline(args.cpu_budget)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def gen_sample(api, torch, dev, m, theta, n_toys: int, per: int, seed: int) -> dict:
    """n_toys x per events of the 4D PDF at theta (per // 10 background each), contiguous."""
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
    n_bkg = np.full(n_toys, per // 10, dtype=np.int64)
    n_sig = np.full(n_toys, per, dtype=np.int64) - n_bkg
    off = np.arange(n_toys, dtype=np.int64) * per
    cols = {k: torch.empty(n_toys * per, dtype=torch.float64, device=dev) for k in ("t", "ck", "cl", "phi")}
    api.ipa_toygen(m, theta, seed, d64(n_sig), d64(n_bkg), d64(off), cols)
    torch.cuda.synchronize()
    return cols


def profile_case(n: int = 8_000_000) -> int:
    """A small fixed case for Nsight Compute: 8e6 events (inputs larger than L2)
    or the headline workload's 1e6 (drawn from the 4D PDF like the bench's), few
    launches."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_01420_gb300 import api, synth
    if n == N_EVENTS:
        ev = gen_sample(api, torch, torch.device("cuda"), api.model_4d(0.0, 15.0), torch.tensor(TH4, device="cuda"),
                        50, 20000, seed=0)
    else:
        ev = {k: torch.tensor(v, device="cuda") for k, v in synth.events_4d(n, 3).items()}
    m = api.model_4d(0.0, 15.0)
    theta = torch.tensor(TH4, device="cuda")
    for _ in range(4):
        out = api.ipa_nll_grad(m, ev, theta)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "ipa_nll_grad 4D", "events": n, "nll": float(out[0])}))
    return 0


def profile_case_tagged() -> int:
    """The tagged model's small fixed case for Nsight Compute (inputs larger than L2)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_01420_gb300 import api, synth
    n = 8_000_000
    ev = {k: torch.tensor(v, device="cuda") for k, v in synth.events_tagged(n, 3).items()}
    m = api.model_tagged(0.0, 15.0)
    theta = torch.tensor(TH_TAG, device="cuda")
    for _ in range(4):
        out = api.ipa_nll_grad(m, ev, theta)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "ipa_nll_grad tagged", "events": n, "nll": float(out[0]),
                      "slow_fraction": tag_slow_fraction(ev["t"].cpu().numpy(), TH_TAG)}))
    return 0


def profile_case_phis() -> int:
    """The phi_s model's small fixed case for Nsight Compute (inputs larger than L2)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_01420_gb300 import api, synth
    n = 8_000_000
    ev = {k: torch.tensor(v, device="cuda") for k, v in synth.events_phis(n, 3).items()}
    m = api.model_phis(0.0, 15.0)
    theta = torch.tensor(TH_PHIS, device="cuda")
    for _ in range(4):
        out = api.ipa_nll_grad(m, ev, theta)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "ipa_nll_grad phi_s model", "events": n, "nll": float(out[0])}))
    return 0


def profile_case_joint() -> int:
    """Example 2's fit of 1e4 events (twelve categories), run twice: the launch
    list of one simultaneous fit at a latency-bound size."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1706_01420_gb300 import api
    dev = torch.device("cuda")
    m = api.model_phis(0.0, 15.0)
    jmap, value = joint_map_phis()
    joint = api.Joint(jmap, value)
    ev, seg = joint_events(api, torch, dev, m, jmap, value, TRUTH_JOINT, 10_000, seed=31 + 10_000)
    start = TRUTH_JOINT * np.where(np.arange(TRUTH_JOINT.size) < 8, 1.02, 1.0)
    params = [api.Param(float(start[j]), float(LO_JOINT[j]), float(HI_JOINT[j]),
                        float((HI_JOINT[j] - LO_JOINT[j]) / 100)) for j in range(TRUTH_JOINT.size)]
    for _ in range(2):
        r = api.ipa_fit_joint(m, ev, seg, joint, params, torch.tensor(start[None, :], device=dev), max_iter=500,
                              tol=1e-6)
    # five joint passes outside a graph: the kernels of one pass, one launch each
    th = torch.tensor(TRUTH_JOINT[None, :], device=dev)
    for _ in range(5):
        api.ipa_nll_grad_joint(m, ev, seg, joint, th)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "ipa_fit_joint, 12 categories, 1e4 events", "passes": int(r["passes"].item()),
                      "status": int(r["status"].item())}))
    return 0


def run_extras(api, synth, torch, dev, m, ev, theta, cal) -> dict:
    """Fit of the 1e6 sample, 4096-toy generation, batched vs one-at-a-time toy fits."""
    out = {}
    lo = [0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2]
    hi = [1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2]
    step = [0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2]
    params = [api.Param(float(TH4[i]), lo[i], hi[i], step[i] / 7.0) for i in range(10)]
    # full fit of the 1e6-event sample from a displaced start
    start = TH4 + np.array([0.01, 0.002, 0.001, 0.01, 0.01, -0.01, 0.05, -0.05, 0.01, 0.1])
    off1 = torch.tensor([0, N_EVENTS], dtype=torch.int64, device=dev)
    th1 = torch.tensor(start[None, :], device=dev)
    tune = {"fit_1e6": api.ipa_autotune(m, dict(ev, fk=api.ipa_angular_basis(m, ev)), th1, seg_off=off1)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    evc = dict(ev, fk=api.ipa_angular_basis(m, ev))        # cached angular basis, inside the timing
    r = api.ipa_fit_batch(m, evc, off1, params, th1, max_iter=200, tol=1e-8)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    npass = int(r["passes"][0])
    out["fit"] = {"events": N_EVENTS, "wall_s": dt, "status": int(r["status"][0]),
                  "iterations": int(r["iters"][0]), "passes": npass,
                  "Gevents_per_s": N_EVENTS * npass / dt / 1e9, "angular_basis": "cached"}
    del evc

    # toy generation: 4096 toys of Poisson(2e4) events
    n_toys = 4096
    n_sig, n_bkg = synth.toy_sizes(n_toys, 2e4, TH4[3], seed=0)
    sizes = n_sig + n_bkg
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(off[-1])
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
    cols = {k: torch.empty(total, dtype=torch.float64, device=dev) for k in ("t", "ck", "cl", "phi")}
    api.ipa_toygen(m, theta, 0, d64(n_sig[:8]), d64(n_bkg[:8]), d64(off[:8]), cols)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.ipa_toygen(m, theta, 0, d64(n_sig), d64(n_bkg), d64(off[:-1]), cols)
    e1.record()
    torch.cuda.synchronize()
    tg = e0.elapsed_time(e1) * 1e-3
    out["toygen"] = {"toys": n_toys, "events": total, "s": tg, "Mevents_per_s": total / tg / 1e6}

    # batched fits of all toys vs the plain loop (one fit per call) on a subset; both
    # read the cached angular basis, computed once for all toys
    e0.record()
    cols["fk"] = api.ipa_angular_basis(m, cols)
    e1.record()
    torch.cuda.synchronize()
    t_basis = e0.elapsed_time(e1) * 1e-3
    thb = torch.tensor(np.tile(TH4, (n_toys, 1)), device=dev)
    tune["batch"] = api.ipa_autotune(m, cols, thb, seg_off=d64(off))
    tune["plain_loop"] = api.ipa_autotune(m, cols, thb[:1], seg_off=d64(off[:2]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rb = api.ipa_fit_batch(m, cols, d64(off), params, thb, max_iter=200, tol=1e-8)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    st = rb["status"].cpu().numpy()
    n_plain = 32
    t0 = time.perf_counter()
    for k in range(n_plain):
        th_k = torch.tensor(TH4[None, :], device=dev)
        api.ipa_fit_batch(m, cols, d64([off[k], off[k + 1]]), params, th_k, max_iter=200, tol=1e-8)
    torch.cuda.synchronize()
    tp = (time.perf_counter() - t0) / n_plain
    thn = rb["theta"].cpu().numpy()
    ern = rb["err"].cpu().numpy()
    ok = st == 0
    pulls = {}
    names = ["Gamma", "sigma", "mu", "f_b", "A0sq", "Apesq", "delta_pa", "delta_pe", "F_S", "delta_S"]
    for j, nm in enumerate(names):
        p = (thn[ok, j] - TH4[j]) / ern[ok, j]
        pulls[nm] = [round(float(p.mean()), 4), round(float(p.std(ddof=1)), 4)]
    passes_b = rb["passes"].cpu().numpy()
    out["batch"] = {"toys": n_toys, "events": total, "batched_fits_per_s": n_toys / tb, "batched_s": tb,
                    "batched_Gevents_per_s": float((sizes * passes_b).sum()) / tb / 1e9,
                    "plain_loop_fits_per_s": 1.0 / tp, "plain_loop_sample": n_plain,
                    "angular_basis_s": t_basis,
                    "converged": int(ok.sum()), "status_counts": np.bincount(st, minlength=5).tolist(),
                    "pull_mean_width": pulls}
    out["autotuned"] = tune
    out["errors"] = run_errors(api, torch, dev, m, cols, off, params, rb)
    del cols, rb, thb
    out["large"] = run_large(api, synth, torch, dev, m, theta, params)
    out["serve"] = run_serve(api, synth, torch, dev, m, theta, params)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out["tagged"] = run_tagged(api, synth, torch, dev, cal, flush)
    out["cls"] = run_cls(api, torch, dev)
    out["phis"] = run_phis(api, synth, torch, dev, flush)
    out["phis_joint"] = run_phis_joint(api, torch, dev, flush)
    return out


def run_tagged(api, synth, torch, dev, cal, flush, steps: int = 50) -> dict:
    """The flavour-tagged model with B_s oscillation: 1e6 events of its PDF (50
    toys of 2e4 from ipa_toygen, timed), NLL+grad per step with L2 flushed, its
    FP64-pipe roofline, and batched fits of the 50 toys (omega held).  The CPU
    oracle's rate on this model is part of cpu_baseline."""
    m = api.model_tagged(0.0, 15.0)
    theta = torch.tensor(TH_TAG, device=dev)
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
    n_toys, per = 50, 20000
    n_bkg = np.full(n_toys, per // 10, dtype=np.int64)
    n_sig = np.full(n_toys, per, dtype=np.int64) - n_bkg
    off = np.arange(n_toys + 1, dtype=np.int64) * per
    n = n_toys * per
    ev = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in ("t", "q")}
    api.ipa_toygen(m, theta, 7, d64(n_sig[:2]), d64(n_bkg[:2]), d64(off[:2]), ev)   # warm-up
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    api.ipa_toygen(m, theta, 7, d64(n_sig), d64(n_bkg), d64(off[:-1]), ev)
    e1.record(stream)
    torch.cuda.synchronize()
    toygen_s = e0.elapsed_time(e1) * 1e-3
    picked = api.ipa_autotune(m, ev, theta, grad=True, stream=stream)
    out = torch.empty(9, dtype=torch.float64, device=dev)
    for _ in range(3):
        api.ipa_nll_grad(m, ev, theta, out)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        api.ipa_nll_grad(m, ev, theta, out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))
    cons = []
    empty = {"t": ev["t"][:0], "q": ev["q"][:0]}
    for i in range(20):
        flush.fill_(float(i))
        e0.record(stream)
        api.ipa_nll(m, empty, theta, out)                 # constants kernel only (n = 0)
        e1.record(stream)
        torch.cuda.synchronize()
        cons.append(e0.elapsed_time(e1))
    kernel_ms = max(ms - statistics.median(cons), 1e-6)
    t_h = ev["t"].cpu().numpy()
    slow = tag_slow_fraction(t_h, TH_TAG)
    spe = (_slots(OPS_TAG_EVENT, cal) + slow * _slots(OPS_TAG_SLOW, cal) + _slots(OPS_UNWEIGHTED, cal)
           + _slots(OPS_LANE_TILE, cal) / 16.0)
    peak = 2.0 * 152 * 2070e6
    ops = spe * n / (kernel_ms * 1e-3)
    # batched fits of the 50 toys: Gamma, f_b, DG, Dm, phi_s free; sigma, mu, omega held
    lo = [0.3, 0.01, -0.1, 0.0, -0.5, 10.0, -3.1, 0.0]
    hi = [1.5, 0.2, 0.1, 0.5, 0.5, 25.0, 3.1, 0.5]
    step = [0.01, 0.003, 0.002, 0.005, 0.02, 0.05, 0.1, 0.01]
    free = (0, 3, 4, 5, 6)
    params = [api.Param(float(TH_TAG[i]), lo[i], hi[i], step[i], fixed=i not in free) for i in range(8)]
    thb = torch.tensor(np.tile(TH_TAG, (n_toys, 1)), device=dev)
    api.ipa_fit_batch(m, ev, d64(off[:3]), params, thb[:2].clone(), max_iter=200, tol=1e-8)   # graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = api.ipa_fit_batch(m, ev, d64(off), params, thb, max_iter=200, tol=1e-8)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    st = r["status"].cpu().numpy()
    return {"workload": "flavour-tagged decay time with B_s oscillation, 1e6 FP64 SoA events (t, q), "
                        "8 params, ipa_nll_grad", "events": n, "launch": picked,
            "nll_grad_ms": ms, "Gevents_per_s": n / (ms * 1e-3) / 1e9, "kernel_ms": kernel_ms,
            "slow_fraction": slow, "fp64_ops_per_event": spe,
            "roofline": {"bound": "alu", "achieved": ops / 1e9, "peak": peak / 1e9, "unit": "G FP64 op/s",
                         "frac": ops / peak, "kernel": "tag_kernel<grad>"},
            "toygen": {"toys": n_toys, "events": n, "s": toygen_s, "Mevents_per_s": n / toygen_s / 1e6},
            "batch_fit": {"toys": n_toys, "s": fit_s, "fits_per_s": n_toys / fit_s,
                          "status_counts": np.bincount(st, minlength=5).tolist(),
                          "passes_mean": float(r["passes"].float().mean())}}


def run_errors(api, torch, dev, m, cols, off, params, rb, n_minos: int = 64) -> dict:
    """HESSE of every fit of the toy batch, and MINOS of all ten parameters of
    the first n_minos toys, at the batch's minima (ipa_hesse, ipa_minos)."""
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
    n_toys = int(rb["theta"].shape[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs = api.ipa_hesse(m, cols, d64(off), params, rb["theta"])
    torch.cuda.synchronize()
    t_h = time.perf_counter() - t0
    st_h = hs["status"].cpu().numpy()
    # agreement of the HESSE errors with the minimiser's own (both from the Hessian at the minimum)
    ok = (rb["status"] == 0).cpu().numpy() & (st_h == 0)
    rel = (hs["err"][ok] / rb["err"][ok] - 1).abs().max().item() if ok.any() else float("nan")
    sub = d64(off[:n_minos + 1])
    t0 = time.perf_counter()
    mn = api.ipa_minos(m, cols, sub, params, rb["theta"][:n_minos].contiguous(), rb["nll"][:n_minos].contiguous(),
                       hs["cov"][:n_minos].contiguous(), list(range(10)))
    torch.cuda.synchronize()
    t_m = time.perf_counter() - t0
    st_m = mn["status"].cpu().numpy().ravel()
    asym = (mn["hi"] + mn["lo"]).abs() / (mn["hi"] - mn["lo"]).clamp_min(1e-300)
    return {"hesse": {"fits": n_toys, "s": t_h, "fits_per_s": n_toys / t_h,
                      "status_counts": np.bincount(st_h, minlength=4).tolist(),
                      "max_rel_diff_vs_fit_errors": rel},
            "minos": {"fits": n_minos, "parameters": 10, "probes": n_minos * 20, "s": t_m,
                      "intervals_per_s": n_minos * 10 / t_m,
                      "status_counts": np.bincount(st_m, minlength=6).tolist(),
                      "median_asymmetry": float(asym.median())}}


TH_PHIS = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.8, 0.3, 0.8, 0.0])


def run_phis(api, synth, torch, dev, flush, steps: int = 30) -> dict:
    """The time-dependent angular model with tagging (16 parameters) on 1e6
    synthetic events (t, angles, tag): NLL+grad per step with L2 flushed, the
    raw and the cached angular basis."""
    m = api.model_phis(0.0, 15.0)
    ev = {k: torch.tensor(v, device=dev) for k, v in synth.events_phis(1_000_000, 11).items()}
    theta = torch.tensor(TH_PHIS, device=dev)
    out = torch.empty(1 + m.n_par, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    res = {"workload": "time-dependent angular model with tagging, 1e6 FP64 SoA events (t, 3 angles, q), "
                       "16 params, ipa_nll_grad", "events": 1_000_000}
    for name, evx in (("raw", ev), ("cached_basis", dict(ev, fk=api.ipa_angular_basis(m, ev)))):
        res["launch_" + name] = api.ipa_autotune(m, evx, theta, grad=True, stream=stream)
        for _ in range(3):
            api.ipa_nll_grad(m, evx, theta, out)
        torch.cuda.synchronize()
        a = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            a[i].record(stream)
            api.ipa_nll_grad(m, evx, theta, out)
            b[i].record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(x.elapsed_time(y) for x, y in zip(a, b))
        res["nll_grad_ms_" + name] = ms
        res["Gevents_per_s_" + name] = 1e6 / (ms * 1e-3) / 1e9
    counts = kernel_counts("phis_kernel<grad>")
    if counts:
        ops = counts["fp64_lane_ops"] * 1e6 / (res["nll_grad_ms_raw"] * 1e-3)
        peak = 2.0 * 152 * 2070e6
        res["roofline"] = {"bound": "alu", "resource": "FP64 pipe", "kernel": "phis_kernel<grad>",
                           "achieved": ops / 1e9, "peak": peak / 1e9, "unit": "G FP64 op/s", "frac": ops / peak,
                           "fp64_lane_ops_per_event": counts["fp64_lane_ops"],
                           "note": "FP64 lane operations per event from the ncu capture of the current source "
                                   "(profiles/kernel_counts.json); step time of the raw-basis call"}
    return res


# Example 2's simultaneous fit: six m(KK) bins times two B flavours, the
# physics parameters shared, F_S and delta_S per bin, C_SP per bin (synthetic
# values of the usual size), each flavour normalised over its own tag; events
# from the model's own generator (no background, perfect tagging, as the
# paper's generated sample without experimental effects).
CSP_BINS = (0.96, 0.93, 0.88, 0.90, 0.95, 0.97)
TRUTH_JOINT = np.array([0.66, 0.52, 0.25, 3.2, 3.1, 0.085, 17.77, 0.8,
                        0.02, 0.035, 0.05, 0.06, 0.04, 0.03, 1.2, 0.7, 0.2, -0.3, -0.8, -1.3])
LO_JOINT = np.array([0.3, 0.35, 0.1, 0.0, 0.0, -0.5, 10.0, -3.1] + [1e-3] * 6 + [-3.2] * 6)
HI_JOINT = np.array([1.5, 0.6, 0.35, 6.3, 6.3, 0.5, 25.0, 3.1] + [0.5] * 6 + [3.2] * 6)


def joint_map_phis(n_bins: int = 6):
    """Category 2 b + (q < 0): joint 0 Gamma, 1 A0sq, 2 Apesq, 3 delta_pa,
    4 delta_pe, 5 DG, 6 Dm, 7 phi_s, 8.. F_S of each bin, 8 + n_bins.. delta_S;
    sigma, mu, f_b, omega, C_SP and the tag selector constant."""
    jmap, value = [], []
    for b in range(n_bins):
        for q in (1.0, -1.0):
            jmap.append([0, -1, -1, -1, 1, 2, 3, 4, 8 + b, 8 + n_bins + b, 5, 6, 7, -1, -1, -1])
            value.append([0, 0.045, 0.0, 0.0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0.0, CSP_BINS[b], q])
    return jmap, value


def joint_events(api, torch, dev, m, jmap, value, theta_joint, n_total: int, seed: int, sub: int = 8192):
    """Events of every category (n_total / n_cat each), generated by ipa_toygen
    in sub-toys of at most `sub` events (one block each), back to back; returns
    the columns and the category offsets."""
    n_cat = len(jmap)
    per = n_total // n_cat
    cols = {k: [] for k in ("t", "ck", "cl", "phi", "q")}
    for c in range(n_cat):
        th = np.array([theta_joint[jmap[c][p]] if jmap[c][p] >= 0 else value[c][p] for p in range(len(jmap[c]))])
        k = max(1, -(-per // sub))
        n_sig = np.full(k, per // k, dtype=np.int64)
        n_sig[: per - int(n_sig.sum())] += 1
        off = np.concatenate([[0], np.cumsum(n_sig)[:-1]]).astype(np.int64)
        out = {name: torch.empty(per, dtype=torch.float64, device=dev) for name in cols}
        d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
        api.ipa_toygen(m, torch.tensor(th, device=dev), seed + 1000 * c, d64(n_sig), d64(np.zeros(k, np.int64)),
                       d64(off), out)
        for name in cols:
            cols[name].append(out[name])
    ev = {name: torch.cat(v) for name, v in cols.items()}
    seg = torch.tensor(np.arange(n_cat + 1, dtype=np.int64) * per, device=dev)
    return ev, seg


def run_phis_joint(api, torch, dev, flush, sizes=(10_000, 10_000_000), steps: int = 20) -> dict:
    """Example 2 (Table 2: 1e4 and 1e7 events): the twelve-category phi_s fit.
    Per size: events from the model (ipa_toygen), the joint NLL+grad pass
    (ipa_nll_grad_joint, L2 flushed, CUDA events) and the whole fit to
    convergence (ipa_fit_joint, all 20 joint parameters free, started 2 % off
    the truth), wall time on the host clock around the blocking call."""
    m = api.model_phis(0.0, 15.0)
    jmap, value = joint_map_phis()
    joint = api.Joint(jmap, value)
    stream = torch.cuda.current_stream()
    res = {"workload": "phi_s model, 12 categories (6 m(KK) bins x 2 flavours), 20 joint parameters; "
                       "events from the model (ipa_toygen), FP64"}
    for n in sizes:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, seg = joint_events(api, torch, dev, m, jmap, value, TRUTH_JOINT, n, seed=31 + n)
        torch.cuda.synchronize()
        t_gen = time.perf_counter() - t0
        n_ev = int(ev["t"].numel())
        theta = torch.tensor(TRUTH_JOINT[None, :], device=dev)
        for _ in range(3):
            api.ipa_nll_grad_joint(m, ev, seg, joint, theta)
        torch.cuda.synchronize()
        a = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            a[i].record(stream)
            api.ipa_nll_grad_joint(m, ev, seg, joint, theta)
            b[i].record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(x.elapsed_time(y) for x, y in zip(a, b))
        start = TRUTH_JOINT * np.where(np.arange(TRUTH_JOINT.size) < 8, 1.02, 1.0)
        params = [api.Param(float(start[j]), float(LO_JOINT[j]), float(HI_JOINT[j]),
                            float((HI_JOINT[j] - LO_JOINT[j]) / 100)) for j in range(TRUTH_JOINT.size)]
        fit_s = []
        for rep in range(2):        # the first call captures the fit's graph
            th = torch.tensor(start[None, :], device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = api.ipa_fit_joint(m, ev, seg, joint, params, th, max_iter=500, tol=1e-6)
            torch.cuda.synchronize()
            fit_s.append(time.perf_counter() - t0)
        th_fit = r["theta"].cpu().numpy()[0]
        err = r["err"].cpu().numpy()[0]
        pulls = (th_fit - TRUTH_JOINT) / np.where(err > 0, err, np.inf)
        res[f"events_{n}"] = {
            "events": n_ev, "generate_s": t_gen, "nll_grad_ms": ms, "Gevents_per_s": n_ev / (ms * 1e-3) / 1e9,
            "fit_wall_s": fit_s[1], "fit_wall_s_first_call": fit_s[0], "status": int(r["status"].item()),
            "iterations": int(r["iters"].item()), "passes": int(r["passes"].item()),
            "fit_Gevents_per_s": n_ev * int(r["passes"].item()) / fit_s[1] / 1e9,
            "max_abs_pull": float(np.max(np.abs(pulls))), "phi_s": [float(th_fit[7]), float(err[7])]}
    return res


def run_cls(api, torch, dev, n_bins: int = 10000, n_toys: int = 10000) -> dict:
    """Example 4's configuration: 10 000 bins on [5179, 5379], a Gaussian signal
    peak smeared by a Gaussian (ipa_binned_smear) over the exponential
    background exp(0.001 m), ns = 70, nb = 5000; CL_b, CL_s+b, CL_s from
    10 000 toys per hypothesis (ipa_cls), timed with CUDA events."""
    lo, hi = 5179.0, 5379.0
    width = (hi - lo) / n_bins
    c = lo + (np.arange(n_bins) + 0.5) * width
    sig = np.exp(-0.5 * ((c - 5279.6) / 5.0) ** 2)
    bkg = np.exp(0.001 * c)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_raw = torch.tensor(sig / sig.sum() * 70.0, device=dev)
    b = torch.tensor(bkg / bkg.sum() * 5000.0, device=dev)
    e0.record(stream)
    s = api.ipa_binned_smear(s_raw, width, 8.0)
    e1.record(stream)
    torch.cuda.synchronize()
    smear_ms = e0.elapsed_time(e1)
    data = api.ipa_binned_generate(s + b, seed=78, n_toys=1, hypothesis=1)[0].contiguous()
    api.ipa_cls(s, b, data, 64, 9)                      # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    r = api.ipa_cls(s, b, data, n_toys, 9)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    draws = 2 * n_toys * n_bins
    return {"bins": n_bins, "toys_per_hypothesis": n_toys, "ms": ms, "toys_per_s": 2 * n_toys / (ms * 1e-3),
            "poisson_draws_per_s": draws / (ms * 1e-3), "smear_ms": smear_ms,
            "cl_b": float(r["cl_b"]), "cl_sb": float(r["cl_sb"]), "cl_s": float(r["cl_s"])}


SERVE_PLAN = {200.0: (2000, 2000), 100.0: (1000, 500), 50.0: (1000, 500), 25.0: (1000, 500)}


def run_serve(api, synth, torch, dev, m, theta, params, plan: dict | None = None) -> dict:
    """Fit requests arriving Poisson at each rate, sizes log-uniform on [1e3, 1e7],
    weights Normal(1, 0.2), events of the 4D PDF: latency (arrival -> result) and
    throughput of the continuous-batching server vs plain sequential fits (one
    ipa_fit_batch call per request, first come first served).  plan: rate ->
    (requests served, requests of the plain loop, the first of the same stream);
    2000 requests at the configuration's 200/s, so that p99 is a percentile of
    2000 latencies."""
    plan = SERVE_PLAN if plan is None else plan
    pool_n = 20_000_000
    cols = gen_sample(api, torch, dev, m, theta, pool_n // 20000, 20000, seed=9)
    pool = {k: v.cpu().numpy() for k, v in cols.items()}
    del cols
    pool["w"] = synth.weights(pool_n, 13)
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
    out = {"requests": {str(int(r)): {"served": a, "plain": b} for r, (a, b) in plan.items()},
           "sizes": "log-uniform [1e3, 1e7]", "weights": "Normal(1, 0.2)"}

    def slices(rate, n_req):
        reqs = synth.request_stream(n_req, rate, seed=int(rate))
        rng = np.random.default_rng(int(rate) + 1)
        return [(r.arrival_s, int(rng.integers(0, pool_n - r.n_events)), r.n_events) for r in reqs]

    for rate in sorted(plan, reverse=True):
        n_served, n_plain = plan[rate]
        full = slices(rate, n_served)
        plan_r = full
        srv = api.ipa_server_create(m, 16 << 30, max_slots=64, max_iter=200, tol=1e-8)
        lat, done_t = {}, {}
        try:
            pending = {}
            t0 = time.perf_counter()
            i = 0
            while len(lat) < len(plan_r):
                now = time.perf_counter() - t0
                while i < len(plan_r) and plan_r[i][0] <= now:
                    arr, a, n = plan_r[i]
                    ev = {k: v[a:a + n] for k, v in pool.items()}
                    pending[api.ipa_serve_submit(srv, ev, params)] = (i, arr)
                    i += 1
                for tk in list(pending):
                    r = api.ipa_serve_poll(srv, tk, 10)
                    if r is not None:
                        k, arr = pending.pop(tk)
                        tnow = time.perf_counter() - t0
                        lat[k] = tnow - arr
                        done_t[k] = tnow
                time.sleep(0.0005)
        finally:
            api.ipa_server_destroy(srv)
        ls = np.array([lat[k] for k in range(len(plan_r))])
        span = max(done_t.values()) - plan_r[0][0]
        # plain sequential: one fit call per request, first come first served
        plat = []
        t0 = time.perf_counter()
        for arr, a, n in full[:n_plain]:
            now = time.perf_counter() - t0
            if now < arr:
                time.sleep(arr - now)
            ev = {k: torch.tensor(v[a:a + n], device=dev) for k, v in pool.items()}
            th = torch.tensor(TH4[None, :], device=dev)
            api.ipa_fit_batch(m, ev, d64([0, n]), params, th, max_iter=200, tol=1e-8)
            torch.cuda.synchronize()
            plat.append(time.perf_counter() - t0 - arr)
        pspan = time.perf_counter() - t0 - plan_r[0][0]
        pl = np.array(plat)
        out[f"rate_{int(rate)}"] = {
            "served": {"p50_s": float(np.percentile(ls, 50)), "p99_s": float(np.percentile(ls, 99)),
                       "fits_per_s": len(plan_r) / span, "requests": len(plan_r)},
            "plain_sequential": {"p50_s": float(np.percentile(pl, 50)), "p99_s": float(np.percentile(pl, 99)),
                                 "fits_per_s": n_plain / pspan, "requests": n_plain}}
    return out


def run_large(api, synth, torch, dev, m, theta, params) -> dict:
    """5e7 events of the 4D PDF (generated on the GPU) with a Normal(1, 0.2) weight
    column, 2 GB: NLL+grad throughput and one full fit."""
    n_toys, per = 2500, 20000
    n = n_toys * per
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device=dev)
    cols = gen_sample(api, torch, dev, m, theta, n_toys, per, seed=5)
    cols["w"] = torch.tensor(synth.weights(n, 11), device=dev)
    out = torch.empty(11, dtype=torch.float64, device=dev)
    tuned = {"raw": api.ipa_autotune(m, cols, theta)}
    for _ in range(2):
        api.ipa_nll_grad(m, cols, theta, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        api.ipa_nll_grad(m, cols, theta, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    start = TH4 + np.array([0.002, 0.0005, 0.0003, 0.002, 0.002, -0.002, 0.01, -0.01, 0.002, 0.02])
    th1 = torch.tensor(start[None, :], device=dev)
    big = [api.Param(p.value, p.lo, p.hi, p.step / 7.0) for p in params]
    tuned["cached_basis"] = api.ipa_autotune(m, dict(cols, fk=api.ipa_angular_basis(m, cols)), theta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cols["fk"] = api.ipa_angular_basis(m, cols)              # inside the fit timing
    r = api.ipa_fit_batch(m, cols, d64([0, n]), big, th1, max_iter=200, tol=1e-8)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    npass = int(r["passes"][0])
    e0.record()
    for _ in range(reps):
        api.ipa_nll_grad(m, cols, theta, out)
    e1.record()
    torch.cuda.synchronize()
    ms_c = e0.elapsed_time(e1) / reps
    # the same pass with the 2 GB of columns in page-locked host memory, read in
    # place by the kernel (ipa_nll_grad_host)
    host = {k: cols[k].cpu().pin_memory() for k in ("t", "ck", "cl", "phi", "w")}
    api.ipa_nll_grad_host(m, host, theta, out)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        api.ipa_nll_grad_host(m, host, theta, out)
    e1.record()
    torch.cuda.synchronize()
    ms_h = e0.elapsed_time(e1) / reps
    del host
    return {"events": n, "weighted": True, "near_peak_fraction": near_peak_fraction(cols["t"].cpu().numpy(), TH4),
            "nll_grad_ms": ms, "Gevents_per_s": n / (ms * 1e-3) / 1e9,
            "nll_grad_ms_cached_basis": ms_c, "Gevents_per_s_cached_basis": n / (ms_c * 1e-3) / 1e9,
            "host_columns": {"nll_grad_ms": ms_h, "Gevents_per_s": n / (ms_h * 1e-3) / 1e9,
                             "h2d_bytes": 40 * n, "note": "page-locked host columns read in place"},
            "fit": {"wall_s": dt, "status": int(r["status"][0]), "iterations": int(r["iters"][0]),
                    "passes": npass, "Gevents_per_s": n * npass / dt / 1e9},
            "autotuned": tuned}


if __name__ == "__main__":
    sys.exit(main())
