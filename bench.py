#!/usr/bin/env python
"""Benchmark: twisted Wilson flow of a batch of SU(3) configurations on GB300 (one JSON line).

A bench step is one pass of the whole hot path over one batch: pack the resident FP64
canonical links into device storage, flow every configuration with RK3 (eps = 0.01) to its
t_end measuring E, Q, P every step (one CUDA graph), read the records back and form
lambda_TGF on the host.  The metric is flowed site-RK3-steps per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64|fp32_r12]
                    [--workload l8x16|l16x4|l12x8|l4|mixed256] [--impl tgf|reference]

Under torchrun (N > 1) each rank flows its own batch (seeds offset by rank): weak scaling,
no data-path collective; the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# flop model (site counts): per RK3 stage 13.4 kflop, per measurement 15.1 kflop
STAGE_FLOP = 13.4e3
MEAS_FLOP = 15.1e3
EPS = 0.01
L2_BYTES = 129e6

WORKLOADS = {
    # name: (list of (extent, seed offset, amplitude), t_end per config, description)
    "l4": dict(l=[4], n=1, amp=0.3, c=0.3,
               desc="1 x SU(3) 4x4x12x12, twist n01=1, links exp(i 0.3 omega T) seed 0, RK3 eps=0.01 to t=0.18"),
    "l8x16": dict(l=[8], n=16, amp=0.3, c=0.3,
                  desc="16 x SU(3) 8x8x24x24, twist n01=1, links exp(i 0.3 omega T) seeds 0-15, RK3 eps=0.01 to "
                       "t=c^2 l^2/8=0.72 (72 steps), E/Q/P every step"),
    "l12x8": dict(l=[12], n=8, amp=0.5, c=0.3,
                  desc="8 x SU(3) 12x12x36x36, twist n01=1, links exp(i 0.5 omega T) seeds 0-7, RK3 eps=0.01 to t=1.62"),
    "l16x4": dict(l=[16], n=4, amp=0.4, c=0.3,
                  desc="4 x SU(3) 16x16x48x48, twist n01=1, links exp(i 0.4 omega T) seeds 0-3, RK3 eps=0.01 to t=2.88"),
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


def make_fields(members, device):
    from paper_2107_03747_gb300 import inputs as I

    fields = []
    for L, seed, amp, _ in members:
        if amp is None:
            _, U = I.batched_member(seed, L, device=device)
        else:
            U = I.random_links(L, seed, amp, device=device)
        fields.append(U)
    return fields


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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


STAGE_SOURCES = ["stage.cu", "su3.cuh", "expm.cuh", "lattice.cuh"]


def stage_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2107_03747_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def stored_traffic(workload, prec):
    """DRAM bytes per stage launch from the committed ncu capture, or None if that capture is of
    another workload, precision or kernel source."""
    path = os.path.join(ROOT, "profiles", "k_stage_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("workload") != workload or d.get("precision") != prec or d.get("stage_source_sha256") != stage_source_hash():
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

def oracle_sample(members, nsteps=1):
    """Oracle on a bounded sample: `nsteps` RK3 steps (each with a measurement) of the first
    configuration of the workload.  Returns (site-steps, seconds)."""
    from oracle import tgf_oracle as O
    from paper_2107_03747_gb300 import inputs as I

    L, seed, amp, _ = members[0]
    U = make_fields([members[0]], "cpu")[0]
    tw = I.default_twist(1)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        O.measure(U, tw)
        U = O.rk3_step(U, EPS, tw)
    dt = time.perf_counter() - t0
    return L[0] * L[1] * L[2] * L[3] * nsteps, dt


def run_reference(args):
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    members = workload_members(args.workload)
    for _ in range(args.warmup):
        oracle_sample(members, 1)
    tot_sites, tot_t = 0, 0.0
    for _ in range(args.steps):
        s, t = oracle_sample(members, 1)
        tot_sites += s
        tot_t += t
    v = tot_sites / tot_t
    L = members[0][0]
    sample = (f"one RK3 step + one measurement of configuration seed {members[0][1]} "
              f"({L[0]}x{L[1]}x{L[2]}x{L[3]}) per bench step")
    line = {"impl": "reference", "metric": "flowed site-RK3-steps/s", "value": v, "unit": "site-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]["desc"], "oracle": "numpy FP64"},
            "cpu_baseline": {"value": v, "unit": "site-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "site-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def run_tgf(args):
    import torch

    ws, rank, local = dist_init()
    from paper_2107_03747_gb300 import build

    if rank == 0:
        build.build()
    barrier(ws)
    from paper_2107_03747_gb300 import binding as tgf

    dev = torch.device("cuda", torch.cuda.current_device())
    members = workload_members(args.workload, rank)
    Ls = [m[0] for m in members]
    t_end = [m[3] for m in members]
    fields = make_fields(members, str(dev))
    canon_host = torch.from_numpy(
        np.concatenate([f.view(np.float64).reshape(-1) for f in fields])).pin_memory()
    canon_dev = canon_host.to(dev)
    del fields
    prec = tgf.PRECISIONS[args.prec]
    b = tgf.FlowBatch(Ls, prec, device=dev)
    stream = torch.cuda.current_stream()
    cap = max(tgf.tgf_flow_records(EPS, t, 1) for t in t_end)
    obs = torch.zeros(len(Ls) * cap * 5, dtype=torch.float64, device=dev)
    obs_host = torch.zeros(len(Ls) * cap * 5, dtype=torch.float64).pin_memory()
    lt = [3 * L[0] for L in Ls]

    def lam_of(o, nrec):
        o = o.view(len(Ls), cap, 5)
        lams = {}
        for key in sorted(set(lt)):
            idx = [i for i in range(len(Ls)) if lt[i] == key]
            E = [float(o[i, nrec[i] - 1, 1]) for i in idx]
            Q = [float(o[i, nrec[i] - 1, 2]) for i in idx]
            t = float(o[idx[0], nrec[idx[0]] - 1, 0])
            c_eff = math.sqrt(8 * t) / key
            lams[key] = tgf.tgf_lambda(c_eff, key, t, E, Q)
        return lams

    reunit = args.reunit if prec != tgf.TGF_FP64 else 0
    flags = 0
    if args.tune:
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
        return lam_of(obs_host, nrec), nrec

    for _ in range(args.warmup):
        lams, nrec = step()
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            lams, nrec = step()
        e1.record()
        torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, ws)
    work = site_steps(members)
    value = work * ws / (ms * 1e-3)
    res_obs = obs_host.view(len(Ls), cap, 5).numpy().copy()

    # ---- e2e: host canonical links -> C ABI upload -> flow -> records back -> lambda -------------
    staging = torch.empty(max(L[0] * L[1] * L[2] * L[3] for L in Ls) * 72, dtype=torch.float64, device=dev)

    def step_e2e():
        tgf.tgf_upload(prec, b.lat, canon_host, staging, b.links)
        nrec = tgf.tgf_flow(prec, b.lat, b.links, b.links_tmp, b.accum, b.scratch, EPS, t_end, obs, cap, 1,
                            reunit, flags)
        obs_host.copy_(obs, non_blocking=True)
        stream.synchronize()
        return lam_of(obs_host, nrec)

    e2e_steps = max(1, min(args.steps, 5))
    step_e2e()
    torch.cuda.synchronize()
    barrier(ws)
    e0.record()
    for _ in range(e2e_steps):
        step_e2e()
    e1.record()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, ws)
    e2e_value = work * ws / (ms_e2e * 1e-3)

    # ---- dominant kernel: the fused stage kernel, timed live on the same workload ------------------
    tgf.tgf_pack(prec, b.lat, canon_dev, b.links)
    nrep = 10
    stage_ms = {}
    for s in (1, 2, 3):
        tgf.tgf_stage(prec, b.lat, b.links, b.links_tmp, b.accum, s, EPS, 0)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(nrep):
            tgf.tgf_stage(prec, b.lat, b.links, b.links_tmp, b.accum, s, EPS, 0)
        e1.record()
        torch.cuda.synchronize()
        stage_ms[s] = e0.elapsed_time(e1) / nrep
    obs1 = torch.zeros(len(Ls) * 5, dtype=torch.float64, device=dev)
    e0.record()
    for _ in range(nrep):
        tgf.tgf_measure(prec, b.lat, b.links, b.scratch, obs1, 1, 0, 0.0)
    e1.record()
    torch.cuda.synchronize()
    meas_ms = e0.elapsed_time(e1) / nrep
    V = sum(L[0] * L[1] * L[2] * L[3] for L in Ls)
    stage_avg = sum(stage_ms.values()) / 3
    peak_prec = tgf.TGF_FP64 if prec == tgf.TGF_FP64 else tgf.TGF_FP32
    peak = tgf.tgf_fma_peak(peak_prec)
    achieved = STAGE_FLOP * V / (stage_avg * 1e-3) / 1e12
    roof = {"kernel": "k_stage (fused staples+force+RK3+exp+update)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"measured {'FP64' if peak_prec == tgf.TGF_FP64 else 'FP32'} FMA-pipe peak (tgf_fma_peak)",
            "traffic": stored_traffic(args.workload, args.prec), "traffic_unit": "bytes per stage launch (ncu)",
            "algorithmic_bytes_per_launch": (2240 if prec != tgf.TGF_FP64 else 4480) / 3.0 * V *
                                             (1.0 if prec != tgf.TGF_FP32_R12 else 1664.0 / 2240.0),
            "flop_per_site": STAGE_FLOP, "sites_per_launch": V,
            "stage_ms": [stage_ms[1], stage_ms[2], stage_ms[3]],
            "measure_ms": meas_ms, "measure_tflops": MEAS_FLOP * V / (meas_ms * 1e-3) / 1e12}

    # ---- accuracy of the reduced-precision forms against the FP64 GPU flow -------------------------
    acc = None
    fp64 = None
    if prec != tgf.TGF_FP64 and not args.no_fp64:
        b64 = tgf.FlowBatch(Ls, tgf.TGF_FP64, device=dev)
        obs64 = torch.zeros_like(obs)
        tgf.tgf_pack(tgf.TGF_FP64, b64.lat, canon_dev, b64.links)
        torch.cuda.synchronize()
        e0.record()
        tgf.tgf_flow(tgf.TGF_FP64, b64.lat, b64.links, b64.links_tmp, b64.accum, b64.scratch, EPS, t_end, obs64,
                     cap, 1, 0, 0)
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        o64 = obs64.view(len(Ls), cap, 5).cpu().numpy()
        rel, dq, rel_kept = 0.0, 0.0, 0.0
        for i in range(len(Ls)):
            n = nrec[i]
            ri = float(np.max(np.abs(res_obs[i, :n, 1] / o64[i, :n, 1] - 1)))
            rel = max(rel, ri)
            if abs(o64[i, n - 1, 2]) < 0.5:  # configurations that enter lambda_TGF
                rel_kept = max(rel_kept, ri)
            dq = max(dq, float(np.max(np.abs(res_obs[i, :n, 2] - o64[i, :n, 2]))))
        lam64 = lam_of(torch.from_numpy(o64.reshape(-1)), nrec)
        dlam = max(abs(lams[k][0] / lam64[k][0] - 1) for k in lams if lams[k][0] and lam64[k][0])
        acc = {"max_rel_dE_vs_fp64": rel, "max_rel_dE_vs_fp64_kept": rel_kept, "max_abs_dQ_vs_fp64": dq,
               "rel_dlambda_vs_fp64": dlam,
               "target_rel_dE": 1e-6, "reunit_every": reunit}
        fp64 = {"value": work / (ms64 * 1e-3), "ms_per_step": ms64, "speedup_of_this_form": ms64 / ms}
        del b64

    # ---- batched flow vs a per-configuration FP64 loop (mixed-size ensembles) ----------------------
    loop = None
    if args.fp64_loop:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(len(Ls)):
            bi = tgf.FlowBatch([Ls[i]], tgf.TGF_FP64, device=dev)
            off = sum(L[0] * L[1] * L[2] * L[3] * 72 for L in Ls[:i])
            n72 = Ls[i][0] * Ls[i][1] * Ls[i][2] * Ls[i][3] * 72
            tgf.tgf_pack(tgf.TGF_FP64, bi.lat, canon_dev[off:off + n72], bi.links)
            oi = torch.zeros(tgf.tgf_flow_records(EPS, t_end[i], 1) * 5, dtype=torch.float64, device=dev)
            tgf.tgf_flow(tgf.TGF_FP64, bi.lat, bi.links, bi.links_tmp, bi.accum, bi.scratch, EPS, [t_end[i]], oi,
                         tgf.tgf_flow_records(EPS, t_end[i], 1), 1, 0, tgf.TGF_NO_GRAPH)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        loop = {"value": work / dt, "seconds": dt, "speedup_of_this_form": dt / (ms * 1e-3),
                "what": "each configuration flowed alone in FP64, kernels launched directly (no graph)"}

    clocks = clk.summary()
    lam_all = {}
    if ws > 1:
        from paper_2107_03747_gb300 import replicas

        o = torch.from_numpy(res_obs)
        for key in sorted(set(lt)):
            idx = [i for i in range(len(Ls)) if lt[i] == key]
            E = [float(o[i, nrec[i] - 1, 1]) for i in idx]
            Q = [float(o[i, nrec[i] - 1, 2]) for i in idx]
            t = float(o[idx[0], nrec[idx[0]] - 1, 0])
            lam_all[key] = replicas.ensemble_lambda(math.sqrt(8 * t) / key, key, t, E, Q)
    else:
        lam_all = lams
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            s, t = oracle_sample(members, 3)
            L0 = members[0][0]
            cpu = {"value": s / t, "unit": "site-steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"three RK3 steps, each with a measurement, of one {L0[0]}x{L0[1]}x{L0[2]}x{L0[3]} "
                             f"configuration ({s} site-steps, {t:.1f} s, numpy FP64 single-threaded)"}
        canon_bytes = canon_host.numel() * 8
        link_bytes = tgf.tgf_links_bytes(prec, b.lat)
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
                       "launch_tuning": {"flags": flags, "grid_k": (flags >> 8) & 0xF,
                                         "size_order": bool(flags & (1 << 12)), "tuned": bool(args.tune)}},
            "e2e": {"value": e2e_value, "unit": "site-steps/s", "h2d_bytes_per_step": canon_bytes,
                    "d2h_bytes_per_step": obs_host.numel() * 8, "ms_per_step": ms_e2e},
            "gpu_launches": launches_per_flow(members) * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "lambda_tgf": {str(k): {"lambda": v[0], "kept": v[1]} for k, v in lam_all.items()},
        }
        if acc:
            line["accuracy"] = acc
        if fp64:
            line["fp64_gpu"] = fp64
        if loop:
            line["fp64_per_config_loop"] = loop
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tgf", choices=["tgf", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "fp32_r12"])
    ap.add_argument("--workload", default="l8x16", choices=sorted(WORKLOADS))
    ap.add_argument("--reunit", type=int, default=20, help="FP32 forms: re-project onto SU(3) every R steps")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison flow")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="use the default launch settings instead of timing the candidates first")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timing")
    ap.add_argument("--fp64-loop", action="store_true",
                    help="also time the ensemble as a loop of single-configuration FP64 flows")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_tgf(args)


if __name__ == "__main__":
    sys.exit(main())
