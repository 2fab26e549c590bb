#!/usr/bin/env python3
"""Benchmark: QPs solved per second on the dense few-equalities QP
(n=2000, m_eq=200, m_in=4000, seed 1), mixed precision vs plain FP64.

A step is one whole solve through the C ABI: qp_create from inputs resident in
HBM (device-to-device copy), qp_factor_K0 (the setup phase), qp_ipm_solve (all
IPM iterations with their reduced PCG solves), qp_destroy.  A step counts as a
solved QP when its objective is within 1e-6 (relative) of the FP64 oracle's.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank solves its own replica of
the QP: the method has no data-parallel exchange for a single QP.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qpgen  # noqa: E402

WORKLOAD = "dense convex QP n=2000 m_eq=200 m_in=4000 (Lambda log-uniform [1e-3,1e3], seed 1)"
METRIC = "QPs solved/s at 1e-6 obj err (mixed precision; FP64 path alongside)"
CONFIG_ID = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the FP64 comparison line")
    ap.add_argument("--profile-pcg", type=int, default=0, metavar="ITERS",
                    help="only factor the QP and run ITERS PCG iterations (a short run for ncu)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"], help="precision of --profile-pcg")
    ap.add_argument("--pcg-form", type=int, default=0, choices=[0, 1],
                    help="--profile-pcg, batch, serving: 0 the implicit K_F product, 1 the W-form")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serving"],
                    help="batch: the 512 batched QPs through qp_batch_solve; "
                         "serving: a Poisson stream of the served workload's QPs through qp_server_*")
    ap.add_argument("--batch", type=int, default=512, help="batch: number of QPs")
    ap.add_argument("--concurrency", type=int, default=16, help="batch: QPs in flight")
    ap.add_argument("--requests", type=int, default=64, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=50.0, help="serving: arrival rate (requests/s)")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: HBM admission budget")
    ap.add_argument("--slots", type=int, default=64, help="serving: QPs in flight at most")
    ap.add_argument("--max-n", type=int, default=4096, help="serving: skip requests with n above this")
    return ap.parse_args()


def golden():
    with open(os.path.join(ROOT, "tests", "golden", f"oracle_config{CONFIG_ID}.json")) as fh:
        return json.load(fh)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(total_ms, solved, device=None):
    """Whole-job figures of a replicated run: the slowest rank's timed total and
    the QPs solved by all ranks (a no-op without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), int(solved)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    k = torch.tensor([int(solved)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(k, op=dist.ReduceOp.SUM)
    return float(t.item()), int(k.item())


# ---------------------------------------------------------------- CPU baseline
def oracle_sample(qp, ipm_iters_full, sample_iters=2):
    """Time the FP64 oracle (3x3 LDL^T variant) on a bounded sample of the same
    workload: its setup plus `sample_iters` IPM iterations, scaled to a full solve
    by the oracle's own iteration count."""
    from oracle import ipm
    t0 = time.perf_counter()
    ipm.start_point(qp.H, qp.c, qp.A, qp.b, qp.C, qp.d)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    ipm.solve_qp(qp, variant="kkt3", max_ipm=sample_iters)
    t_iters = time.perf_counter() - t0 - t_setup
    per_iter = t_iters / sample_iters
    t_full = t_setup + per_iter * ipm_iters_full
    cores = len(os.sched_getaffinity(0))
    return dict(value=1.0 / t_full, unit="QPs/s", cores=cores, kind="oracle",
                sample=f"start point + {sample_iters} of {ipm_iters_full} IPM iterations of the FP64 "
                       f"3x3-LDL^T oracle on the same QP, scaled to the full solve "
                       f"({per_iter:.2f} s/iteration, {t_full:.1f} s/QP)")


# ---------------------------------------------------------------------- clocks
REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 3:
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), int(parts[2], 16)))
                except ValueError:
                    pass

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        mask = 0
        for _, _, m in self.samples:
            mask |= m
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "reasons": [name for bit, name in REASONS.items() if mask & bit],
                "samples": len(self.samples)}


# ------------------------------------------------------------------ our solver
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    B.load()
    gold = golden()
    qp = qpgen.config_qp(CONFIG_ID)
    dev = torch.device("cuda", local)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Hd, cd, Ad, bd, Cd, dd = t(qp.H), t(qp.c), t(qp.A), t(qp.b), t(qp.C), t(qp.d)
    xd = torch.zeros(qp.n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2
    # The solver runs on this (non-default) stream: PCG graphs are captured on it and
    # the CUDA events below are recorded on it.
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)

    def opts(prec):
        o = B.qp_opts_default()
        o.precision = prec
        o.stream = stream.cuda_stream
        return o

    def step(prec, out):
        h = B.qp_create(Hd, cd, Ad, bd, Cd, dd, opts(prec))
        try:
            st, f, its, pits = B.qp_ipm_solve(h, xd, allow=(B.QP_OK, B.QP_EMAXIT, B.QP_ENUMERIC))
            out.append(dict(status=st, f=f, ipm=its, pcg=pits, stats=B.qp_get_stats(h)))
        finally:
            B.qp_destroy(h)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, steps, warmup):
        res = []
        for _ in range(warmup):
            step(prec, [])
        barrier()
        total_ms = 0.0
        l0 = B.qp_kernel_launches()
        for _ in range(steps):
            flush.fill_(1.0)                     # evict L2 between timed steps (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec, res)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
        barrier()
        launches = B.qp_kernel_launches() - l0
        ok = [abs(r["f"] - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6 and r["status"] == 0 for r in res]
        total_ms, solved_all = reduce_over_ranks(total_ms, sum(ok), dev)
        return res, total_ms, ok, launches, solved_all

    with ClockSampler(local) as clk:
        res, total_ms, ok, launches, solved = timed(B.QP_PREC_FP32, args.steps, args.warmup)
    res64, total64, ok64, _, solved64 = timed(B.QP_PREC_FP64, args.fp64_steps, 1)

    value = solved / (total_ms / 1e3)
    value64 = solved64 / (total64 / 1e3)

    # ---- roofline of the dominant kernel chain: one PCG iteration (a6-a10)
    o = opts(B.QP_PREC_FP32)
    o.mixed_fallback = 0          # the FP32 hot path itself (the mixed solve's first phase)
    h = B.qp_create(Hd, cd, Ad, bd, Cd, dd, o)
    B.qp_factor_K0(h)
    # an early-IPM D (s, nu of order one): the FP32 P_H factor applies, so this times
    # the FP32 hot path (the bytes and work per iteration do not depend on D's values)
    Dmid = np.exp(np.random.default_rng(7).uniform(np.log(1e-1), np.log(1e1), qp.m2))
    ms_it = B.qp_time_pcg_iteration(h, Dmid, precond=B.QP_PC_AUTO, warmup=16, iters=128)
    by_it = B.qp_pcg_bytes_per_iter(h, B.QP_PC_AUTO)
    B.qp_destroy(h)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = by_it / (ms_it * 1e-3) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "pcg_iteration_traffic.json")) as fh:
            tr = json.load(fh)
        from paper_2104_12916_gb300 import build as _b
        if tr.get("source_hash") == source_hash():
            traffic = tr.get("dram_bytes_per_iteration")
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "one PCG iteration on K_F (C'p, K0 solve, C y + D p, update, P_H solve): "
                          f"{by_it / 1e6:.1f} MB algorithmic, {ms_it * 1e3:.1f} us",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback"}

    # ---- the same path with pcg_form = 1 (K_F through B = L^-1[C'; 0], two matrix phases)
    o = opts(B.QP_PREC_FP32)
    o.mixed_fallback, o.pcg_form = 0, 1
    h = B.qp_create(Hd, cd, Ad, bd, Cd, dd, o)
    B.qp_factor_K0(h)
    ms_w = B.qp_time_pcg_iteration(h, Dmid, precond=B.QP_PC_AUTO, warmup=16, iters=128)
    by_w = B.qp_pcg_bytes_per_iter(h, B.QP_PC_AUTO)
    B.qp_destroy(h)
    def step_w(out):
        ow = opts(B.QP_PREC_FP32)
        ow.pcg_form = 1
        hw = B.qp_create(Hd, cd, Ad, bd, Cd, dd, ow)
        try:
            st_, f_, its_, pits_ = B.qp_ipm_solve(hw, xd, allow=(B.QP_OK, B.QP_EMAXIT, B.QP_ENUMERIC))
            out.append(dict(status=st_, f=f_, ipm=its_, pcg=pits_))
        finally:
            B.qp_destroy(hw)
    step_w([])
    torch.cuda.synchronize()
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rw = []
    e0.record(stream)
    step_w(rw)
    e1.record(stream)
    e1.synchronize()
    ms_wsolve = e0.elapsed_time(e1)
    ok_w = abs(rw[0]["f"] - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6 and rw[0]["status"] == 0
    wform = {"what": "pcg_form=1: K_F p = D p + B1'(B1 p) - B2'(B2 p), B = L^-1[C'; 0] formed once per QP",
             "pcg_iteration_us": round(ms_w * 1e3, 1), "algorithmic_MB": round(by_w / 1e6, 1),
             "achieved_GBps": round(by_w / (ms_w * 1e-3) / 1e9, 1),
             "frac": round(by_w / (ms_w * 1e-3) / 1e9 / peak, 4),
             "qps_per_s": round((1.0 if ok_w else 0.0) / (ms_wsolve / 1e3), 4), "ms_per_solve": round(ms_wsolve, 1),
             "ipm_iters": rw[0]["ipm"], "pcg_iters": rw[0]["pcg"], "obj_rel_err": abs(rw[0]["f"] - gold["f"]) / abs(gold["f"]),
             "traffic": None}
    try:
        with open(os.path.join(ROOT, "profiles", "pcg_iteration_traffic_wform.json")) as fh:
            trw = json.load(fh)
        if trw.get("source_hash") == source_hash():
            wform["traffic"] = trw.get("dram_bytes_per_iteration")
    except Exception:
        pass

    # ---- end to end through host buffers (H2D of the inputs and D2H of x inside)
    e2e_ms = 0.0
    xh = np.zeros(qp.n)
    Cdense = np.ascontiguousarray(qp.C)
    nsteps_e2e = max(1, min(args.steps, 2))
    e2e_ok = 0
    torch.cuda.synchronize()
    for _ in range(nsteps_e2e):
        t0 = time.perf_counter()
        o = B.qp_opts_default()
        o.precision = B.QP_PREC_FP32
        hh = B.qp_create(qp.H, qp.c, qp.A, qp.b, Cdense, qp.d, o)
        st, f, its, pits = B.qp_ipm_solve(hh, xh, allow=(B.QP_OK, B.QP_EMAXIT, B.QP_ENUMERIC))
        B.qp_destroy(hh)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_ok += int(abs(f - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6 and st == 0)
    h2d = 8 * (qp.n * qp.n + qp.m1 * qp.n + qp.m2 * qp.n + qp.n + qp.m1 + qp.m2)
    d2h = 8 * qp.n + 8
    e2e_ms, e2e_solved = reduce_over_ranks(e2e_ms, e2e_ok, dev)
    e2e = {"value": e2e_solved / (e2e_ms / 1e3), "unit": "QPs/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    if rank == 0:
        cpu = oracle_sample(qp, gold["ipm_iters"]) if world == 1 else None
        st0 = res[-1]["stats"] if res else {}
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "QPs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "mixed (FP32 operator and P_H, FP64 refinement)",
                       "preconditioner": "auto -> P_H (few equalities)", "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write, untimed)"},
            "solved": f"{sum(ok)}/{len(ok)} per rank", "obj_rel_err": [abs(r["f"] - gold["f"]) / abs(gold["f"]) for r in res],
            "ipm_iters": [r["ipm"] for r in res], "pcg_iters": [r["pcg"] for r in res],
            "oracle_ipm_iters": gold["ipm_iters"],
            "breakdown_ms": {k: round(st0.get(k, 0.0), 1) for k in ("t_factor_ms", "t_pcg_ms", "t_precond_ms", "t_solve_ms")},
            "fp64": {"value": round(value64, 4), "unit": "QPs/s", "ms_per_step": round(total64 / max(1, args.fp64_steps), 2),
                     "dtype": "f64", "solved": f"{sum(ok64)}/{len(ok64)}",
                     "ipm_iters": [r["ipm"] for r in res64], "pcg_iters": [r["pcg"] for r in res64]},
            "roofline": roofline, "wform": wform, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def source_hash():
    """Hash of the sources of the persistent PCG kernel (the kernel whose DRAM
    traffic profiles/pcg_iteration_traffic.json records)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2104_12916_gb300", "csrc")
    for fn in ("common.cuh", "vec.cuh", "pcg_fused.cuh"):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The reference arm is the FP64 CPU oracle (the paper ships no code): each
    step is a bounded sample (start point + 2 IPM iterations of the 3x3 LDL^T
    oracle) scaled to a full solve by the oracle's iteration count."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    gold = golden()
    qp = qpgen.config_qp(CONFIG_ID)
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up state; warm-up steps are not repeated work
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(qp, gold["ipm_iters"]))
    wall = time.perf_counter() - t0
    v = statistics.median(r["value"] for r in vals)
    cpu = dict(vals[0])
    cpu["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "QPs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 / v, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "cpu"}, "impl": "reference",
            "cpu_baseline": cpu, "e2e": {"value": v, "unit": "QPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Factor the workload's QP and time `--profile-pcg` PCG iterations (P_H,
    mid-IPM D); prints the per-iteration time.  Used as the ncu target."""
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    qp = qpgen.config_qp(CONFIG_ID)
    o = B.qp_opts_default()
    o.precision = B.QP_PREC_FP32 if args.precision == "fp32" else B.QP_PREC_FP64
    o.mixed_fallback = 0          # time the FP32 kernels themselves
    o.pcg_form = args.pcg_form
    h = B.qp_create(qp.H, qp.c, qp.A, qp.b, np.ascontiguousarray(qp.C), qp.d, o)
    B.qp_factor_K0(h)
    Dmid = np.exp(np.random.default_rng(7).uniform(np.log(1e-1), np.log(1e1), qp.m2))
    ms = B.qp_time_pcg_iteration(h, Dmid, precond=B.QP_PC_AUTO, warmup=8, iters=args.profile_pcg)
    by = B.qp_pcg_bytes_per_iter(h, B.QP_PC_AUTO)
    print(json.dumps({"pcg_iteration_us": ms * 1e3, "algorithmic_MB": by / 1e6,
                      "GBps": by / (ms * 1e-3) / 1e9, "precision": args.precision, "pcg_form": args.pcg_form}))
    B.qp_destroy(h)


BATCH_WORKLOAD = ("512 dense QPs, n uniform [64,512], m_eq uniform [0.1n,0.5n], m_in uniform [n,3n], "
                  "Lambda log-uniform [1e-2,1e2], seeds 1e6+i")


def run_batch(args):
    """The batched workload through qp_batch_solve: every QP created from host
    buffers, solved with many in flight (each QP's persistent PCG kernel on 8-16
    blocks launched as one cluster, host waits yielding), the solution read back.  One step = the whole batch,
    timed on the host clock around qp_batch_solve (inputs already on the device);
    e2e includes the creation (H2D) and the solution copies.  QPs with n <= 160
    are checked against the FP64 oracle."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    B.load()
    qps = [qpgen.batch_qp(i) for i in range(args.batch)]
    out = {}
    for prec in (B.QP_PREC_FP32, B.QP_PREC_FP64):
        o = B.qp_opts_default()
        o.precision, o.blocking_wait, o.pcg_form = prec, 1, args.pcg_form
        l0 = B.qp_kernel_launches()
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            hs = [B.QP.from_qpgen(q, o) for q in qps]
            t1 = time.perf_counter()
            st, res = B.qp_batch_solve([h.h for h in hs], max_concurrent=args.concurrency)
            t2 = time.perf_counter()
            xs = []
            for q, h in zip(qps, hs):
                x = np.zeros(q.n)
                B.qp_get_solution(h.h, x)
                xs.append(x)
            t3 = time.perf_counter()
        for h in hs:
            h.close()
        ok = [r["status"] == 0 for r in res]
        out[prec] = dict(res=res, ok=ok, solve_s=t2 - t1, e2e_s=t3 - t0, launches=B.qp_kernel_launches() - l0,
                         clocks=clk.summary())
    from oracle import ipm
    errs = []
    r32 = out[B.QP_PREC_FP32]["res"]
    for i, q in enumerate(qps):
        if q.n <= 160:
            ref = ipm.solve_qp(q, variant="kkt3")
            errs.append(abs(r32[i]["obj"] - ref.f) / max(abs(ref.f), 1.0))
    m = out[B.QP_PREC_FP32]
    m64 = out[B.QP_PREC_FP64]
    h2d = sum(8 * (q.n * q.n + q.m1 * q.n + q.m2 * q.n + q.n + q.m1 + q.m2) for q in qps)
    line = {"metric": "QPs solved/s on the 512-QP batch (mixed precision; FP64 path alongside)",
            "value": round(sum(m["ok"]) / m["solve_s"], 3), "unit": "QPs/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": round(m["solve_s"] * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "qps": len(qps), "in_flight": args.concurrency,
                       "precision": "mixed (FP32 operator and P_H, FP64 refinement)",
                       "pcg_form": "W-form" if args.pcg_form else "implicit"},
            "solved": f"{sum(m['ok'])}/{len(qps)}",
            "fp64": {"value": round(sum(m64["ok"]) / m64["solve_s"], 3), "unit": "QPs/s",
                     "solved": f"{sum(m64['ok'])}/{len(qps)}"},
            "oracle_checked": len(errs), "oracle_max_rel_err": max(errs) if errs else None,
            "latency_ms": {"p50": round(float(np.percentile([r["solve_ms"] for r in m["res"]], 50)), 1),
                           "p99": round(float(np.percentile([r["solve_ms"] for r in m["res"]], 99)), 1)},
            "e2e": {"value": round(sum(m["ok"]) / m["e2e_s"], 3), "unit": "QPs/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": sum(8 * q.n for q in qps)},
            "gpu_launches": int(m["launches"]), "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)


SERVING_WORKLOAD = ("served stream: n log-uniform [64,4096], m_eq = n U(0.05,0.9), m_in = n U(1,3), "
                    "C CSR 8 nnz/row, Lambda log-uniform [1e-2,1e2], Poisson arrivals")


def run_serving(args):
    """A Poisson stream of the served workload through qp_server_*: requests are
    submitted at their arrival times (host buffers: the submission copies them,
    the server moves them to the device when it admits them), results polled as
    they complete.  value = solved QPs / (last completion - first arrival); a QP
    counts as solved when it converged to the IPM tolerances (FP64 residuals);
    the requests with n <= 256 are also checked against the FP64 oracle."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    B.load()
    idx = [i for i in range(10 * args.requests) if qpgen.serving_dims(i)[0] <= args.max_n][:args.requests]
    qps = [qpgen.serving_qp(i) for i in idx]
    arrive = qpgen.arrival_times(len(qps), args.rate)
    o = B.qp_opts_default()
    o.blocking_wait, o.pcg_form = 1, args.pcg_form
    srv = B.Server(budget_bytes=int(args.budget_gb * 1e9), max_slots=args.slots, opts=o)
    l0 = B.qp_kernel_launches()
    results = {}
    pending = {}
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        k = 0
        while k < len(qps) or pending:
            now = time.perf_counter() - t0
            while k < len(qps) and arrive[k] <= now:
                pending[srv.submit(qps[k])] = k
                k += 1
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    results[pending.pop(t)] = (r[0], r[1], time.perf_counter() - t0)
            if k < len(qps):
                time.sleep(max(0.0, min(0.002, arrive[k] - (time.perf_counter() - t0))))
            else:
                time.sleep(0.001)
        wall = max(v[2] for v in results.values()) - arrive[0]
    st = srv.stats()
    srv.close()
    launches = B.qp_kernel_launches() - l0
    lat = np.array([results[i][0]["latency_ms"] for i in range(len(qps))])
    ok = [results[i][0]["status"] == 0 for i in range(len(qps))]
    # oracle check of the small requests
    from oracle import ipm
    errs = []
    for i, q in enumerate(qps):
        if q.n <= 256 and ok[i]:
            ref = ipm.solve_qp(q, variant="kkt3")
            errs.append(abs(results[i][0]["obj"] - ref.f) / max(abs(ref.f), 1.0))
    line = {"metric": "QPs solved/s on a served Poisson stream, with p50/p99 latency",
            "value": round(sum(ok) / wall, 3), "unit": "QPs/s", "n_gpus": 1, "steps": len(qps), "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SERVING_WORKLOAD, "rate_per_s": args.rate, "requests": len(qps),
                       "max_n": args.max_n, "budget_gb": args.budget_gb, "slots": args.slots,
                       "precision": "mixed (FP32 operator and P_H, FP64 refinement)",
                       "pcg_form": "W-form" if args.pcg_form else "implicit"},
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 1), "p99": round(float(np.percentile(lat, 99)), 1),
                           "max": round(float(lat.max()), 1)},
            "wait_ms_p50": round(float(np.percentile([results[i][0]["wait_ms"] for i in range(len(qps))], 50)), 1),
            "solved": f"{sum(ok)}/{len(ok)}", "wall_s": round(wall, 2),
            "oracle_checked": len(errs), "oracle_max_rel_err": max(errs) if errs else None,
            "n_range": [min(q.n for q in qps), max(q.n for q in qps)],
            "server": {k2: st[k2] for k2 in ("peak_reserved_bytes", "peak_device_bytes", "failed")},
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.workload == "serving" and a.impl == "ours":
        run_serving(a)
    elif a.workload == "batch" and a.impl == "ours":
        run_batch(a)
    elif a.profile_pcg:
        run_profile(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
