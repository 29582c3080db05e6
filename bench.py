#!/usr/bin/env python
"""Benchmark: twisted Wilson flow of a batch of SU(3) configurations on GB300 (one JSON line).

A bench step is one pass of the whole hot path over one batch: pack the resident FP64
canonical links into device storage, flow every configuration with RK3 (eps = 0.01) to its
t_end measuring E, Q, P every step (one CUDA graph), read the records back and form
lambda_TGF on the host.  The metric is flowed site-RK3-steps per second.  The default
workload is 4 configurations of 16x16x48x48 flowed to t = c^2 l^2/8 = 2.88 (288 steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64|fp32_r12]
                    [--workload l16x4|l8x16|l12x8|l12x8_c04|l4|mixed256|...] [--impl tgf|reference]

Besides the headline (the FP32 form with FP64 sums), the line carries a `forms` record with
every precision form (FP64, FP32-18, FP32-12) flowed on the same workload: site-steps/s, the
stage kernel's roofline fraction, its DRAM traffic from the committed ncu capture, the achieved
HBM GB/s and the error of E and lambda_TGF against the FP64 flow; a `batched` record (256
mixed-size configurations in one graph against a loop of single-configuration FP64 flows); and
the CPU oracle timed on the host's cores (`cpu_baseline`).

Under torchrun (N > 1) each rank flows its own batch (seeds offset by rank): weak scaling,
no data-path collective; the time is the max over ranks.

`--profile-stages PREC` runs only the three RK3 stage kernels of the workload a few times (the
command the committed ncu traffic captures under profiles/ were taken with).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# flop model (site counts): per RK3 stage 13.4 kflop, per measurement 15.1 kflop
STAGE_FLOP = 13.4e3
MEAS_FLOP = 15.1e3
EPS = 0.01
L2_BYTES = 129e6
# algorithmic HBM bytes per site of one stage launch (stage 1, 2, 3): links read, X read/written,
# links written (fused double-buffered stage, X as 8 reals per link)
STAGE_BYTES = {
    "fp64": (1408, 1664, 1408),
    "fp32": (704, 832, 704),
    "fp32_r12": (512, 640, 512),
}
# a measured step also writes and re-reads the clover halves and plaquette traces (114 reals/site)
MEAS_BYTES = {"fp64": 2 * 114 * 8, "fp32": 2 * 114 * 4, "fp32_r12": 2 * 114 * 4}
PREC_NAMES = ("fp64", "fp32", "fp32_r12")

WORKLOADS = {
    "l4": dict(l=[4], n=1, amp=0.3, c=0.3,
               desc="1 x SU(3) 4x4x12x12, twist n01=1, links exp(i 0.3 omega T) seed 0, RK3 eps=0.01 to t=0.18"),
    "l8x16": dict(l=[8], n=16, amp=0.3, c=0.3,
                  desc="16 x SU(3) 8x8x24x24, twist n01=1, links exp(i 0.3 omega T) seeds 0-15, RK3 eps=0.01 to "
                       "t=c^2 l^2/8=0.72 (72 steps), E/Q/P every step"),
    "l12x8": dict(l=[12], n=8, amp=0.5, c=0.3,
                  desc="8 x SU(3) 12x12x36x36, twist n01=1, links exp(i 0.5 omega T) seeds 0-7, RK3 eps=0.01 to "
                       "t=c^2 l^2/8=1.62 (162 steps), E/Q/P every step"),
    "l12x8_c04": dict(l=[12], n=8, amp=0.5, c=0.4,
                      desc="8 x SU(3) 12x12x36x36, twist n01=1, links exp(i 0.5 omega T) seeds 0-7, RK3 eps=0.01 to "
                           "t=c^2 l^2/8=2.88 with c=0.4 (288 steps), E/Q/P every step"),
    "l16x4": dict(l=[16], n=4, amp=0.4, c=0.3,
                  desc="4 x SU(3) 16x16x48x48, twist n01=1, links exp(i 0.4 omega T) seeds 0-3, RK3 eps=0.01 to "
                       "t=c^2 l^2/8=2.88 (288 steps), E/Q/P every step"),
    "mixed256": dict(l=[4, 6, 8], n=256, amp=None, c=0.3,
                     desc="256 x SU(3) mixed l in {4,6,8} (l x l x 3l x 3l), twist n01=1, amp U[0.2,0.6], RK3 eps=0.01 "
                          "to t=c^2 l^2/8 each"),
    "l16x4_paper": dict(l=[16], n=4, amp=0.4, c=0.3, long=True,
                        desc="4 x SU(3) 16x16x48x48, twist n01=1, links exp(i 0.4 omega T) seeds 0-3, RK3 eps=0.01 to "
                             "the coupling's own scale sqrt(8t)=0.3*3l, t=25.92 (2592 steps), E/Q/P every step"),
    "l8x16_paper": dict(l=[8], n=16, amp=0.3, c=0.3, long=True,
                        desc="16 x SU(3) 8x8x24x24, twist n01=1, links exp(i 0.3 omega T) seeds 0-15, RK3 eps=0.01 to "
                             "the coupling's own scale sqrt(8t)=0.3*3l, t=6.48 (648 steps), E/Q/P every step"),
}


def workload_members(name, rank=0):
    """[(extent, seed, amplitude, t_end)] of one rank's batch."""
    w = WORKLOADS[name]
    out = []
    for i in range(w["n"]):
        l = w["l"][i % len(w["l"])]
        seed = rank * w["n"] + i
        # t = c^2 l^2 / 8 with the short extent, or the paper's sqrt(8t) = c * 3l
        scale = 3 * l if w.get("long") else l
        t_end = w["c"] ** 2 * scale * scale / 8.0
        out.append(((l, l, 3 * l, 3 * l), seed, w["amp"], t_end))
    return out


def make_field(member, device="cpu"):
    from paper_2107_03747_gb300 import inputs as I

    L, seed, amp, _ = member
    if amp is None:
        return I.batched_member(seed, L, device=device)[1]
    return I.random_links(L, seed, amp, device=device)


def make_fields(members, device):
    return [make_field(m, device) for m in members]


def n_steps(t_end):
    n = int(math.floor(t_end / EPS + 1e-9))
    rest = t_end - n * EPS
    return n, (1 if rest > 1e-12 * EPS else 0)


def site_steps(members):
    tot = 0
    for L, _, _, t_end in members:
        n, extra = n_steps(t_end)
        tot += L[0] * L[1] * L[2] * L[3] * (n + extra)
    return tot


def launches_per_flow(members):
    """Kernels one flow enqueues: 3 stages per step, measure + reduce per distinct record set, + pack."""
    steps = [sum(n_steps(m[3])) for m in members]
    maxT = max(steps)
    k = 1  # pack
    if any(s == 0 for s in steps):
        k += 2
    for i in range(maxT):
        act = [s for s in steps if i < s]
        k += 2 + 3  # measure+reduce (measure_every = 1), 3 stages
        if any(s == i + 1 for s in act):
            k += 2
    return k


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"tgf_bench_clocks_{os.getpid()}_gpu{index}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


STAGE_SOURCES = ["stage_kernel.cuh", "stage.cu", "stage_tiles.cu", "su3.cuh", "expm.cuh", "lattice.cuh"]


def stage_source_hash():
    """sha256 of the stage kernel's code with comments and whitespace removed: a capture stays
    valid across comment edits and goes stale when the code changes."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        src = open(os.path.join(ROOT, "paper_2107_03747_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).strip().encode())
    return h.hexdigest()


def traffic_path(workload, prec):
    return os.path.join(ROOT, "profiles", f"k_stage_traffic_{prec}_{workload}.json")


def stored_traffic(workload, prec):
    """DRAM bytes per stage launch (mean of stages 1-3) from the committed ncu capture of this
    workload and precision, or None if there is none or it was taken on another kernel source."""
    try:
        d = json.load(open(traffic_path(workload, prec)))
    except Exception:
        return None
    if d.get("stage_source_sha256") != stage_source_hash():
        return None
    b = d.get("dram_bytes_per_launch")
    return float(sum(b) / len(b)) if b else None


def dist_init():
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    from paper_2107_03747_gb300 import replicas

    return replicas.max_over_ranks(x)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------------

def oracle_unit(member):
    """One unit of the workload on the oracle, single-threaded: a measurement and one RK3 step of
    one configuration (what the flow does at every step).  Returns (site-steps, seconds)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    from oracle import tgf_oracle as O
    from paper_2107_03747_gb300 import inputs as I

    L = member[0]
    U = make_field(member, "cpu")
    tw = I.default_twist(1)
    t0 = time.perf_counter()
    O.measure(U, tw)
    O.rk3_step(U, EPS, tw)
    return L[0] * L[1] * L[2] * L[3], time.perf_counter() - t0


def oracle_workers(member, want):
    """Worker processes for the oracle pool: at most the host's cores and as many as its free
    memory holds (about 9 KB per site per worker, measured on the full-size oracle step)."""
    cores = os.cpu_count() or 1
    L = member[0]
    need = 9e3 * L[0] * L[1] * L[2] * L[3] + 0.5e9
    try:
        import psutil

        avail = psutil.virtual_memory().available
    except Exception:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    by_mem = max(1, int(0.7 * avail // need))
    return max(1, min(cores, want, by_mem)), cores


def oracle_pool(members, n_units):
    """`n_units` oracle units (configurations of the workload, cycled) on a spawn pool; returns
    (site-steps, wall seconds, per-unit seconds, workers, host cores)."""
    import multiprocessing as mp

    units = [members[i % len(members)] for i in range(n_units)]
    workers, cores = oracle_workers(units[0], n_units)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(oracle_unit, units, chunksize=1)
    wall = time.perf_counter() - t0
    return sum(r[0] for r in res), wall, [r[1] for r in res], workers, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    members = workload_members(args.workload)
    # warm-up: imports and numpy set-up on the smallest lattice (a CPU program has no device to warm)
    small = ((4, 4, 12, 12), 0, 0.3, 0.18)
    for _ in range(args.warmup):
        oracle_unit(small)
    sites, wall, per, workers, cores = oracle_pool(members, args.steps)
    v = sites / wall
    L = members[0][0]
    sample = (f"{args.steps} units, each one measurement + one RK3 step of one {L[0]}x{L[1]}x{L[2]}x{L[3]} "
              f"configuration of the workload (seeds cycled), numpy FP64, on a spawn pool of {workers} single-threaded "
              f"workers ({cores} host cores); wall {wall:.1f} s, {np.mean(per):.1f} s per unit")
    line = {"impl": "reference", "metric": "flowed site-RK3-steps/s", "value": v, "unit": "site-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]["desc"], "oracle": "numpy FP64"},
            "cpu_baseline": {"value": v, "unit": "site-steps/s", "cores": workers, "kind": "oracle",
                             "sample": sample, "host_cores": cores,
                             "single_core_value": float(np.mean([sites / args.steps / t for t in per]))},
            "e2e": {"value": v, "unit": "site-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def time_stages(tgf, b, prec_name, nrep=10, flags=0):
    """Mean device time (ms) of each RK3 stage kernel launch on `b` (CUDA events on the stream the
    kernels are launched on; `flags` selects the launch tile) and of one measurement.

    Each repetition runs stages 1, 2, 3 in order on the same input field, as one RK3 step does, so
    that every stage sees the accumulator X of a real step (a stage repeated on its own output X
    would grow it, and the exponential's scaling would then time work a flow never does)."""
    import torch

    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * nrep)]
    tile = flags & (0x7 << 13)
    for s in (1, 2, 3):  # warm-up step
        tgf.tgf_stage(b.prec, b.lat, b.links, b.links_tmp, b.accum, s, EPS, 0, tile)
    torch.cuda.synchronize()
    for r in range(nrep):
        ev[4 * r].record(stream)
        for s in (1, 2, 3):
            tgf.tgf_stage(b.prec, b.lat, b.links, b.links_tmp, b.accum, s, EPS, 0, tile)
            ev[4 * r + s].record(stream)
    torch.cuda.synchronize()
    out = {s: sum(ev[4 * r + s - 1].elapsed_time(ev[4 * r + s]) for r in range(nrep)) / nrep for s in (1, 2, 3)}
    e0, e1 = ev[0], ev[1]
    obs1 = torch.zeros(b.ncfg * 5, dtype=torch.float64, device=b.device)
    e0.record(stream)
    for _ in range(nrep):
        tgf.tgf_measure(b.prec, b.lat, b.links, b.scratch, obs1, 1, 0, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    return [out[1], out[2], out[3]], e0.elapsed_time(e1) / nrep


def roofline_of(tgf, prec_name, V, stage_ms, meas_ms, workload, peaks, hbm_peak):
    """Roofline record of the fused stage kernel: flops of the flop model per launch over its mean
    launch time against the measured FMA peak of its precision; algorithmic bytes per launch over
    the same time against the measured HBM copy bandwidth."""
    stage_avg = sum(stage_ms) / 3
    peak = peaks["fp64" if prec_name == "fp64" else "fp32"]
    achieved = STAGE_FLOP * V / (stage_avg * 1e-3) / 1e12
    alg_bytes = sum(STAGE_BYTES[prec_name]) / 3.0 * V
    gbs = alg_bytes / (stage_avg * 1e-3) / 1e9
    return {"kernel": "k_stage (fused staples+force+RK3+exp+update)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"measured {'FP64' if prec_name == 'fp64' else 'FP32'} FMA-pipe peak (tgf_fma_peak)",
            "traffic": stored_traffic(workload, prec_name), "traffic_unit": "DRAM bytes per stage launch (ncu, mean of stages 1-3)",
            "algorithmic_bytes_per_launch": alg_bytes, "hbm_gbs": gbs, "hbm_peak_gbs": hbm_peak,
            "hbm_frac": gbs / hbm_peak if hbm_peak else None,
            "flop_per_site": STAGE_FLOP, "sites_per_launch": V, "stage_ms": stage_ms,
            "measure_ms": meas_ms, "measure_tflops": MEAS_FLOP * V / (meas_ms * 1e-3) / 1e12}


def tune_setting(flags):
    from paper_2107_03747_gb300 import tune

    return tune.flags_setting(flags)


def hbm_peak_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0  # the profiling recipe's fallback copy bandwidth


def flow_bytes(prec_name, members):
    """Algorithmic HBM bytes of one flow: the three stage launches of every step and the clover
    halves of every measured step (written by stage 1, re-read by the clover sum)."""
    tot = 0
    for L, _, _, t_end in members:
        V = L[0] * L[1] * L[2] * L[3]
        n, extra = n_steps(t_end)
        tot += V * (n + extra) * (sum(STAGE_BYTES[prec_name]) + MEAS_BYTES[prec_name])
    return tot


def lam_of(tgf, o, nrec, Ls):
    """lambda_TGF per box size l~ = 3l from the last record of every configuration; o: (ncfg, cap, 5)."""
    lt = [3 * L[0] for L in Ls]
    lams = {}
    for key in sorted(set(lt)):
        idx = [i for i in range(len(Ls)) if lt[i] == key]
        E = [float(o[i, nrec[i] - 1, 1]) for i in idx]
        Q = [float(o[i, nrec[i] - 1, 2]) for i in idx]
        t = float(o[idx[0], nrec[idx[0]] - 1, 0])
        lams[key] = tgf.tgf_lambda(math.sqrt(8 * t) / key, key, t, E, Q)
    return lams


def accuracy_vs(o, o64, nrec, lam, lam64):
    """max |dE/E| over every record (all configurations and those kept by |Q| < 1/2), max |dQ|,
    |dlambda/lambda| against the FP64 flow's records."""
    rel, dq, rel_kept = 0.0, 0.0, 0.0
    for i in range(o.shape[0]):
        n = nrec[i]
        ri = float(np.max(np.abs(o[i, :n, 1] / o64[i, :n, 1] - 1)))
        rel = max(rel, ri)
        if abs(o64[i, n - 1, 2]) < 0.5:
            rel_kept = max(rel_kept, ri)
        dq = max(dq, float(np.max(np.abs(o[i, :n, 2] - o64[i, :n, 2]))))
    dl = [abs(lam[k][0] / lam64[k][0] - 1) for k in lam if lam[k][0] and lam64[k][0]]
    return {"max_rel_dE_vs_fp64": rel, "max_rel_dE_vs_fp64_kept": rel_kept, "max_abs_dQ_vs_fp64": dq,
            "rel_dlambda_vs_fp64": max(dl) if dl else None, "target_rel_dE": 1e-6}


def profile_stages(args):
    """Only the three stage kernels of the workload in one precision, a few times each: the command
    under which the per-launch DRAM traffic of profiles/k_stage_traffic_*.json is captured."""
    import torch

    from paper_2107_03747_gb300 import build

    build.build()
    from paper_2107_03747_gb300 import binding as tgf

    torch.cuda.set_device(0)
    members = workload_members(args.workload)
    Ls = [m[0] for m in members]
    canon = torch.from_numpy(np.concatenate([f.view(np.float64).reshape(-1) for f in make_fields(members, "cuda")]))
    canon = canon.to("cuda")
    b = tgf.FlowBatch(Ls, args.profile_stages)
    tgf.tgf_pack(b.prec, b.lat, canon, b.links)
    del canon
    from paper_2107_03747_gb300 import tune

    flags = tune.tune_flags(0, False, args.tile or 0)
    for _ in range(args.steps):
        for s in (1, 2, 3):
            tgf.tgf_stage(b.prec, b.lat, b.links, b.links_tmp, b.accum, s, EPS, 0, flags)
    torch.cuda.synchronize()
    print(json.dumps({"profile_stages": args.profile_stages, "workload": args.workload, "tile": args.tile,
                      "launches": 3 * args.steps}))
    return 0


def run_tgf(args):
    import torch

    ws, rank, local = dist_init()
    from paper_2107_03747_gb300 import build

    if rank == 0:
        build.build()
    barrier(ws)
    from paper_2107_03747_gb300 import binding as tgf

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    members = workload_members(args.workload, rank)
    Ls = [m[0] for m in members]
    t_end = [m[3] for m in members]
    canon_host = torch.from_numpy(
        np.concatenate([f.view(np.float64).reshape(-1) for f in make_fields(members, str(dev))])).pin_memory()
    canon_dev = canon_host.to(dev)
    prec = tgf.PRECISIONS[args.prec]
    b = tgf.FlowBatch(Ls, prec, device=dev)
    cap = max(tgf.tgf_flow_records(EPS, t, 1) for t in t_end)
    obs = torch.zeros(len(Ls) * cap * 5, dtype=torch.float64, device=dev)
    obs_host = torch.zeros(len(Ls) * cap * 5, dtype=torch.float64).pin_memory()
    V = sum(L[0] * L[1] * L[2] * L[3] for L in Ls)

    reunit = args.reunit if prec != tgf.TGF_FP64 else 0
    flags = 0
    if args.launch_flags is not None:
        flags = args.launch_flags
    elif args.tune:
        # launch settings of tgf_flow timed on this workload (results are the same for all of them)
        from paper_2107_03747_gb300 import tune

        tgf.tgf_pack(prec, b.lat, canon_dev, b.links)
        flags = tune.tune(b, eps=EPS, steps=4, measure_every=1, force=True)

    def step():
        tgf.tgf_pack(prec, b.lat, canon_dev, b.links)
        nrec = tgf.tgf_flow(prec, b.lat, b.links, b.links_tmp, b.accum, b.scratch, EPS, t_end, obs, cap, 1,
                            reunit, flags)
        obs_host.copy_(obs, non_blocking=True)
        stream.synchronize()
        return lam_of(tgf, obs_host.view(len(Ls), cap, 5), nrec, Ls), nrec

    for _ in range(args.warmup):
        lams, nrec = step()
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            lams, nrec = step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, ws)
    work = site_steps(members)
    value = work * ws / (ms * 1e-3)
    res_obs = obs_host.view(len(Ls), cap, 5).numpy().copy()

    # ---- e2e: host canonical links -> C ABI upload -> flow -> records back -> lambda -------------
    # Two buffer sets, double-buffered as a production caller would run a stream of batches: the
    # upload of step k+1 (tgf_upload on a copy stream) overlaps the flow of step k.  Every step's
    # host->device copy of its inputs and device->host read of its records are inside the timed
    # region.  (The first large copy after the host link has idled runs at ~1/4 of its 211 GB/s,
    # which the overlap hides behind the flow.)
    b2 = tgf.FlowBatch(Ls, prec, device=dev)
    bufs, obs_b = [b, b2], [obs, torch.zeros_like(obs)]
    staging = [torch.empty(max(L[0] * L[1] * L[2] * L[3] for L in Ls) * 72, dtype=torch.float64, device=dev)
               for _ in range(2)]
    up_stream = torch.cuda.Stream(device=dev)
    up_done = [torch.cuda.Event(), torch.cuda.Event()]
    flow_done = [torch.cuda.Event(), torch.cuda.Event()]
    for ev_ in flow_done:
        ev_.record(stream)

    def upload(k):
        i = k % 2
        up_stream.wait_event(flow_done[i])  # the buffer set's previous flow has finished with it
        tgf.tgf_upload(prec, bufs[i].lat, canon_host, staging[i], bufs[i].links, stream=up_stream)
        up_done[i].record(up_stream)

    def run_e2e(nsteps, start=None):
        if start is not None:
            up_stream.wait_event(start)
        upload(0)
        lams_ = None
        for k in range(nsteps):
            i = k % 2
            stream.wait_event(up_done[i])
            nrec_ = tgf.tgf_flow(prec, bufs[i].lat, bufs[i].links, bufs[i].links_tmp, bufs[i].accum, bufs[i].scratch,
                                 EPS, t_end, obs_b[i], cap, 1, reunit, flags, stream=stream)
            flow_done[i].record(stream)
            if k + 1 < nsteps:
                upload(k + 1)
            obs_host.copy_(obs_b[i], non_blocking=True)
            stream.synchronize()
            lams_ = lam_of(tgf, obs_host.view(len(Ls), cap, 5), nrec_, Ls)
        return lams_

    e2e_steps = max(2, min(args.steps, 6))
    run_e2e(2)  # captures the flow graph of each buffer set
    torch.cuda.synchronize()
    barrier(ws)
    e0.record(stream)
    run_e2e(e2e_steps, start=e0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, ws)
    e2e_value = work * ws / (ms_e2e * 1e-3)
    del b2, bufs, obs_b, staging
    torch.cuda.empty_cache()

    # ---- dominant kernel: the fused stage kernel, timed live on the same workload ------------------
    peaks = {"fp32": tgf.tgf_fma_peak(tgf.TGF_FP32), "fp64": tgf.tgf_fma_peak(tgf.TGF_FP64),
             "fp32_packed": tgf.tgf_fma_peak(tgf.TGF_FMA_PEAK_FP32X2)}
    hbm = hbm_peak_gbs()
    tgf.tgf_pack(prec, b.lat, canon_dev, b.links)
    stage_ms, meas_ms = time_stages(tgf, b, args.prec, flags=flags)
    roof = roofline_of(tgf, args.prec, V, stage_ms, meas_ms, args.workload, peaks, hbm)
    roof["launch_tile"] = (flags >> 13) & 0x7

    # ---- the other precision forms on the same workload, and the FP64 reference flow ---------------
    forms = {}
    main_rec = {"value": value, "ms_per_step": ms, "roofline_frac": roof["frac"], "stage_ms": stage_ms,
                "launch_tuning": tune_setting(flags) if prec != tgf.TGF_FP64 else None,
                "stage_hbm_gbs": roof["hbm_gbs"], "traffic_per_launch": roof["traffic"],
                "flow_hbm_gbs": flow_bytes(args.prec, members) / (ms * 1e-3) / 1e9,
                "flow_bytes_per_step": flow_bytes(args.prec, members), "link_bytes": tgf.tgf_links_bytes(prec, b.lat)}
    forms[args.prec] = main_rec
    o64 = None
    if not args.no_forms:
        del b
        torch.cuda.empty_cache()
        for pn in PREC_NAMES:
            if pn == args.prec:
                continue
            bf = tgf.FlowBatch(Ls, pn, device=dev)
            of = torch.zeros_like(obs)
            ru = args.reunit if pn != "fp64" else 0
            # FP64: one run with direct launches (no graph to capture, ~26 ms kernels); FP32 forms:
            # the launch setting tuned for this form, the first run captures the graph, the second
            # is timed
            fl = tgf.TGF_NO_GRAPH
            if pn != "fp64":
                fl = 0
                if args.tune and args.launch_flags is None:
                    from paper_2107_03747_gb300 import tune

                    tgf.tgf_pack(bf.prec, bf.lat, canon_dev, bf.links)
                    fl = tune.tune(bf, eps=EPS, steps=4, measure_every=1, force=True)
                elif args.launch_flags is not None:
                    fl = args.launch_flags
            for r in range(1 if pn == "fp64" else 2):
                tgf.tgf_pack(bf.prec, bf.lat, canon_dev, bf.links)
                torch.cuda.synchronize()
                e0.record(stream)
                nr = tgf.tgf_flow(bf.prec, bf.lat, bf.links, bf.links_tmp, bf.accum, bf.scratch, EPS, t_end, of,
                                  cap, 1, ru, fl)
                e1.record(stream)
                torch.cuda.synchronize()
            msf = e0.elapsed_time(e1)
            oo = of.view(len(Ls), cap, 5).cpu().numpy()
            tgf.tgf_pack(bf.prec, bf.lat, canon_dev, bf.links)
            sm, mm = time_stages(tgf, bf, pn, nrep=3 if pn == "fp64" else 10, flags=fl & ~tgf.TGF_NO_GRAPH)
            rf = roofline_of(tgf, pn, V, sm, mm, args.workload, peaks, hbm)
            forms[pn] = {"value": work / (msf * 1e-3), "ms_per_step": msf, "roofline_frac": rf["frac"],
                         "stage_ms": sm, "stage_hbm_gbs": rf["hbm_gbs"], "traffic_per_launch": rf["traffic"],
                         "flow_hbm_gbs": flow_bytes(pn, members) / (msf * 1e-3) / 1e9,
                         "flow_bytes_per_step": flow_bytes(pn, members),
                         "link_bytes": tgf.tgf_links_bytes(bf.prec, bf.lat), "_obs": oo, "_nrec": nr,
                         "launch_tuning": tune_setting(fl & ~tgf.TGF_NO_GRAPH) if pn != "fp64" else None}
            if pn == "fp64":
                o64 = oo
            del bf
            torch.cuda.empty_cache()
        forms[args.prec]["_obs"], forms[args.prec]["_nrec"] = res_obs, nrec
        if o64 is not None:
            lam64 = lam_of(tgf, o64, forms["fp64"]["_nrec"], Ls)
            for pn in PREC_NAMES:
                f = forms[pn]
                if pn != "fp64":
                    f["accuracy"] = accuracy_vs(f["_obs"], o64, f["_nrec"], lam_of(tgf, f["_obs"], f["_nrec"], Ls),
                                                lam64)
                    f["speedup_vs_fp64_gpu"] = forms["fp64"]["ms_per_step"] / f["ms_per_step"]
                    f["reunit_every"] = args.reunit
        for pn in PREC_NAMES:
            forms[pn].pop("_obs", None)
            forms[pn].pop("_nrec", None)
    acc = forms.get(args.prec, {}).get("accuracy")

    # ---- batched mixed-size ensemble vs a per-configuration FP64 loop ------------------------------
    batched = None
    if args.batched and args.workload != "mixed256":
        batched = run_batched(tgf, dev, stream, args)

    clocks = clk.summary()
    lam_all = {}
    if ws > 1:
        from paper_2107_03747_gb300 import replicas

        o = torch.from_numpy(res_obs)
        for key in sorted(set(3 * L[0] for L in Ls)):
            idx = [i for i in range(len(Ls)) if 3 * Ls[i][0] == key]
            E = [float(o[i, nrec[i] - 1, 1]) for i in idx]
            Q = [float(o[i, nrec[i] - 1, 2]) for i in idx]
            t = float(o[idx[0], nrec[idx[0]] - 1, 0])
            lam_all[key] = replicas.ensemble_lambda(math.sqrt(8 * t) / key, key, t, E, Q)
    else:
        lam_all = lams
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            units = max(1, args.cpu_units)
            sites, wall, per, workers, cores = oracle_pool(members, units)
            L0 = members[0][0]
            cpu = {"value": sites / wall, "unit": "site-steps/s", "cores": workers, "kind": "oracle",
                   "host_cores": cores, "single_core_value": float(np.mean([sites / units / t for t in per])),
                   "sample": f"{units} units on a spawn pool of {workers} single-threaded workers ({cores} host cores): "
                             f"each a measurement + one RK3 step of one {L0[0]}x{L0[1]}x{L0[2]}x{L0[3]} "
                             f"configuration of the workload, numpy FP64; wall {wall:.1f} s, "
                             f"{np.mean(per):.1f} s per unit"}
        canon_bytes = canon_host.numel() * 8
        link_bytes = main_rec["link_bytes"]
        line = {
            "metric": "flowed site-RK3-steps/s", "value": value, "unit": "site-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp32_r12": "f32"}[args.prec], "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "precision": args.prec,
                       "sums": "f64", "configs_per_gpu": len(Ls), "sites_per_gpu": V,
                       "site_steps_per_gpu": work, "link_bytes": link_bytes,
                       "l2": ("inputs larger than L2" if link_bytes > L2_BYTES else "inputs smaller than L2") +
                             f" ({link_bytes / 1e6:.0f} MB links, {canon_bytes / 1e6:.0f} MB canonical)",
                       "parallelism": f"replicas x{ws}", "graph": True,
                       "launch_tuning": dict(flags=flags, tuned=bool(args.tune and args.launch_flags is None),
                                             **tune_setting(flags))},
            "e2e": {"value": e2e_value, "unit": "site-steps/s", "h2d_bytes_per_step": canon_bytes,
                    "d2h_bytes_per_step": obs_host.numel() * 8, "ms_per_step": ms_e2e, "steps": e2e_steps,
                    "how": "tgf_upload of each step's canonical FP64 host fields (pinned) on a copy stream, "
                           "overlapping the previous step's tgf_flow; records read back every step"},
            "gpu_launches": launches_per_flow(members) * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "peaks": {"fp32_fma_tflops": peaks["fp32"], "fp32_packed_fma_tflops": peaks["fp32_packed"],
                      "fp64_fma_tflops": peaks["fp64"], "hbm_gbs": hbm},
            "lambda_tgf": {str(k): {"lambda": v[0], "kept": v[1]} for k, v in lam_all.items()},
            "forms": forms,
        }
        if acc:
            line["accuracy"] = acc
        if batched:
            line["batched"] = batched
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_batched(tgf, dev, stream, args):
    """256 mixed-size configurations (l in {4,6,8}) flowed in FP32 in one CUDA graph against the same
    configurations flowed one at a time in FP64 with direct launches; lambda_TGF per box size from both."""
    import torch

    members = workload_members("mixed256")
    Ls = [m[0] for m in members]
    t_end = [m[3] for m in members]
    canon = torch.from_numpy(np.concatenate([f.view(np.float64).reshape(-1) for f in make_fields(members, str(dev))]))
    canon = canon.to(dev)
    b = tgf.FlowBatch(Ls, "fp32", device=dev)
    cap = max(tgf.tgf_flow_records(EPS, t, 1) for t in t_end)
    obs = torch.zeros(len(Ls) * cap * 5, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flags = 0
    if args.tune:
        from paper_2107_03747_gb300 import tune

        tgf.tgf_pack(b.prec, b.lat, canon, b.links)
        flags = tune.tune(b, eps=EPS, steps=4, measure_every=1, force=True)
    times = []
    for r in range(4):
        tgf.tgf_pack(b.prec, b.lat, canon, b.links)
        torch.cuda.synchronize()
        e0.record(stream)
        nrec = tgf.tgf_flow(b.prec, b.lat, b.links, b.links_tmp, b.accum, b.scratch, EPS, t_end, obs, cap, 1,
                            args.reunit, flags)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    o = obs.view(len(Ls), cap, 5).cpu().numpy()
    del b
    # per-configuration FP64 loop
    o64 = np.zeros_like(o)
    nrec64 = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    off = 0
    for i, L in enumerate(Ls):
        bi = tgf.FlowBatch([L], "fp64", device=dev)
        n72 = L[0] * L[1] * L[2] * L[3] * 72
        tgf.tgf_pack(bi.prec, bi.lat, canon[off:off + n72], bi.links)
        off += n72
        oi = torch.zeros(cap * 5, dtype=torch.float64, device=dev)
        nr = tgf.tgf_flow(bi.prec, bi.lat, bi.links, bi.links_tmp, bi.accum, bi.scratch, EPS, [t_end[i]], oi, cap, 1,
                          0, tgf.TGF_NO_GRAPH)
        o64[i] = oi.view(cap, 5).cpu().numpy()
        nrec64.append(nr[0])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    work = site_steps(members)
    acc = accuracy_vs(o, o64, nrec, lam_of(tgf, o, nrec, Ls), lam_of(tgf, o64, nrec64, Ls))
    return {"workload": WORKLOADS["mixed256"]["desc"], "precision": "fp32", "launch_flags": flags,
            "launch_tuning": tune_setting(flags),
            "value": work / (ms * 1e-3), "ms_per_step": ms, "fp64_loop_value": work / dt, "fp64_loop_seconds": dt,
            "speedup_vs_fp64_loop": dt / (ms * 1e-3),
            "fp64_loop": "each configuration flowed alone in FP64, kernels launched directly (no graph), host clock",
            "accuracy": acc}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tgf", choices=["tgf", "reference"])
    ap.add_argument("--prec", default="fp32", choices=list(PREC_NAMES))
    ap.add_argument("--workload", default="l16x4", choices=sorted(WORKLOADS))
    ap.add_argument("--reunit", type=int, default=20, help="FP32 forms: re-project onto SU(3) every R steps")
    ap.add_argument("--no-forms", action="store_true", help="skip the other precision forms (and the FP64 flow)")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the mixed-size batched ensemble against the per-configuration FP64 loop")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="use the default launch settings instead of timing the candidates first")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timing")
    ap.add_argument("--launch-flags", type=int, default=None,
                    help="tgf_flow launch flags to use instead of tuning (reproduces a tuned run under a profiler)")
    ap.add_argument("--cpu-units", type=int, default=0,
                    help="oracle units in the cpu_baseline pool (default: one per host core, memory permitting)")
    ap.add_argument("--profile-stages", default=None, choices=list(PREC_NAMES),
                    help="only run the stage kernels of the workload in this precision (ncu traffic captures)")
    ap.add_argument("--tile", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="with --profile-stages: launch the stage kernels with this launch tile")
    args = ap.parse_args()
    if args.cpu_units <= 0:
        args.cpu_units = os.cpu_count() or 1
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_stages:
        return profile_stages(args)
    return run_tgf(args)


if __name__ == "__main__":
    sys.exit(main())
