"""Benchmark: time to the stationary vector of a 256 x 256 tandem queue.

Workload (one "step" = the whole hot path): bootstrap setup (Algorithm 1:
test-vector relaxation, LS fits of P and Q, Q B P, coarsest triplets) and
V-cycle-preconditioned flexible GMRES to ||B x||_1 / ||x||_1 <= 1e-10, on the
tandem queueing network with 65,536 states (arrival 10/31, service 11/31 and
10/31), r = 16 test vectors, 5 levels, GMRES(20).  The headline runs the
mixed-precision path (FP32 V-cycle and setup relaxation inside FP64 GMRES);
the plain FP64 GPU path is timed beside it on the same chain.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  With --impl reference the CPU oracle is timed on the
host cores instead (the reference arm of the comparison).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("solve time to ‖Bx‖₁/‖x‖₁≤1e-10, mixed/learned vs FP64 plain; "
          "% of HBM peak")
WORKLOAD = {"workload": "tandem queue 256x256 (65,536 states, nnz(B)=261,121), rates 10/31, 11/31, 10/31",
            "r": 16, "levels": 5, "gmres_restart": 20, "tol": 1e-10, "nu": "3+3 Jacobi omega=0.7",
            "setup_relaxations": 5}
SIDE = 256
KW = dict(r=16, max_levels=5, coarse_min=1, seed=2)


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- GPU arm
def gpu_arm(args, rank: int, world: int):
    import numpy as np
    import torch

    import chaingen as cg
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api

    dev = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    ch = cg.tandem(SIDE)
    rp = torch.from_numpy(ch.row_ptr).cuda()
    ci = torch.from_numpy(ch.col).cuda()
    va = torch.from_numpy(ch.val).cuda()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step(prec):
        p = api.bamg_params_default(precision=prec, **KW)
        h = api.bamg_setup(rp, ci, va, ch.n, p, nx=SIDE, ny=SIDE, stream=stream)
        x, info = api.bamg_solve(h, restart=20, tol=1e-10, stream=stream)
        return h, x, info

    def timed(prec, steps, warmup, count_launches=False):
        times, infos = [], []
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                h, x, info = one_step(prec)
                h.destroy()
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            l0 = api.launch_count()
            for _ in range(steps):
                flush.fill_(1.0)                     # evict the 129 MB L2 between steps
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h, x, info = one_step(prec)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                infos.append(info)
                last = (h, x)
            torch.cuda.synchronize()
            launches = api.launch_count() - l0
        return times, infos, last, launches

    with ClockSampler(dev) as clk:
        t_mix, i_mix, (h_mix, x_mix), launches = timed("mixed", args.steps, args.warmup, True)
    t_64, i_64, (h_64, x_64), _ = timed("fp64", max(3, args.steps // 2), 2)

    ms = statistics.mean(t_mix)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    err_vs_fp64 = float((x_mix - x_64).abs().sum().item())

    # end to end through host buffers (pinned), copies inside the timed region
    hrp = torch.from_numpy(ch.row_ptr).pin_memory().numpy()
    hci = torch.from_numpy(ch.col).pin_memory().numpy()
    hva = torch.from_numpy(ch.val).pin_memory().numpy()
    e2e = []
    with torch.cuda.stream(stream):
        for k in range(max(3, args.steps // 2) + 1):
            p = api.bamg_params_default(precision="mixed", **KW)
            t0 = time.perf_counter()
            xh, _ = api.bamg_solve_host(hrp, hci, hva, ch.n, p, nx=SIDE, ny=SIDE, restart=20, tol=1e-10,
                                        stream=stream)
            if k:
                e2e.append((time.perf_counter() - t0) * 1e3)
    h2d = hrp.nbytes + hci.nbytes + hva.nbytes
    d2h = xh.nbytes

    roof = roofline(api, torch, np, ch, stream, h_mix)
    return {
        "ms": ms, "t_mix": t_mix, "i_mix": i_mix, "t_64": t_64, "i_64": i_64, "launches": launches,
        "clocks": clk.summary(), "err_vs_fp64": err_vs_fp64, "e2e_ms": statistics.mean(e2e),
        "h2d": h2d, "d2h": d2h, "roofline": roof,
    }


def roofline(api, torch, np, ch, stream, h):
    """Live CUDA-event timing of the dominant kernel on the bench's data.

    The dominant kernel of a step (by the ncu launch list) is the cooperative
    coarsest-level solver; it is latency bound.  Its figure is reported
    against the FP32 ALU peak; the finest-level block relaxation (the hot
    sparse kernel) is timed too and reported against the HBM peak.
    """
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        hbm, src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        hbm, src = 6800.0, "fallback"
    # finest-level FP32 block relaxation: n x 16 block, B of the tandem chain
    lev = h.level(0)
    B = lev["B"]
    n, ld = ch.n, 16
    rp, ci = B["row_ptr"], B["col"]
    va = B["val"].float()
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    rows = torch.repeat_interleave(torch.arange(n, device="cuda"), (rp[1:] - rp[:-1]).long())
    diag = (B["col"].long() == rows)
    d[rows[diag]] = B["val"][diag]
    dinv = (1.0 / d).float()
    X = torch.rand((n, ld), device="cuda", dtype=torch.float32)
    nb = 64   # > L2 in total: cycle through distinct X/Y pairs
    Xs = [torch.rand((n, ld), device="cuda", dtype=torch.float32) for _ in range(nb)]
    with torch.cuda.stream(stream):
        for k in range(5):
            api.bamg_step_relax_block(rp, ci, va, dinv, Xs[k % nb], stream=stream)
        reps = 200
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            api.bamg_step_relax_block(rp, ci, va, dinv, Xs[k % nb], stream=stream)
        e1.record(stream)
        e1.synchronize()
    dur_s = e0.elapsed_time(e1) / reps / 1e3
    nnz = int(B["nnz"])
    alg_bytes = nnz * 8 + (n + 1) * 4 + n * 4 + 2 * n * ld * 4
    achieved = alg_bytes / dur_s / 1e9
    return {"bound": "hbm", "kernel": "relax_block_kernel<float,16> (finest level)",
            "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": None, "peak_source": src,
            "launch_us": round(dur_s * 1e6, 3), "alg_bytes": alg_bytes}


# ---------------------------------------------------------------- CPU baseline
def cpu_oracle_step(side=SIDE):
    """One oracle setup + solve of the same workload (plain numpy/scipy)."""
    import chaingen as cg
    from oracle import setup as S
    from oracle import solve as So
    ch = cg.tandem(side)
    t0 = time.perf_counter()
    H = S.bamg_setup(ch.csr(), S.Params(**KW), grid=(side, side))
    x, its, _ = So.bamg_solve(H, tol=1e-10, restart=20)
    return (time.perf_counter() - t0) * 1e3, its


def cpu_baseline_subprocess(steps=1):
    """Time the oracle in a child process with BLAS pinned to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r=[bench.cpu_oracle_step() for _ in range(%d)]; print(json.dumps(r))" % (ROOT, steps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)

    if args.impl == "reference":
        if rank != 0:
            return
        res = cpu_baseline_subprocess(args.warmup + args.steps)
        if res is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle run failed"}))
            return
        times = [t for t, _ in res[args.warmup:]]
        v = statistics.mean(times)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism="host cores, 1 thread"),
            "cpu_baseline": {"value": round(v, 3), "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": "full workload: oracle setup + GMRES solve of the 256x256 tandem chain"},
            "e2e": {"value": round(v, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iterations": res[-1][1]}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = gpu_arm(args, rank, world)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        res = cpu_baseline_subprocess(1)
        if res:
            cpu = {"value": round(res[0][0], 1), "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": "one full step: oracle setup + GMRES solve of the 256x256 tandem chain "
                             "(BLAS threads pinned to 1)"}
    it_mix = [i["iterations"] for i in r["i_mix"]]
    line = {
        "metric": METRIC, "value": round(r["ms"], 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(r["ms"], 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(WORKLOAD, precision="mixed: FP32 V-cycle and setup relaxation, FP64 GMRES",
                       l2="flushed (512 MB write) before every step", parallelism="replicas" if world > 1 else "1 GPU"),
        "setup_ms": round(statistics.mean(i["setup_ms"] for i in r["i_mix"]), 3),
        "solve_ms": round(statistics.mean(i["solve_ms"] for i in r["i_mix"]), 3),
        "iterations": it_mix[-1], "iters_to_1e7": r["i_mix"][-1]["iters_to_1e7"],
        "rel_res_1": r["i_mix"][-1]["rel_res_1"], "err_l1_vs_fp64_gpu": r["err_vs_fp64"],
        "fp64_plain": {"ms_per_step": round(statistics.mean(r["t_64"]), 3),
                       "setup_ms": round(statistics.mean(i["setup_ms"] for i in r["i_64"]), 3),
                       "solve_ms": round(statistics.mean(i["solve_ms"] for i in r["i_64"]), 3),
                       "iterations": r["i_64"][-1]["iterations"]},
        "op_cplx": r["i_mix"][-1]["op_cplx"], "grid_cplx": r["i_mix"][-1]["grid_cplx"],
        "e2e": {"value": round(r["e2e_ms"], 3), "unit": "ms", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"],
        "roofline": r["roofline"],
        "cpu_baseline": cpu,
        "clocks": r["clocks"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
