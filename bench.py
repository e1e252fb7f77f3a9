"""Benchmark: time to the stationary vector of a 256 x 256 tandem queue.

Workload (one "step" = the whole hot path): bootstrap setup (Algorithm 1:
test-vector relaxation, LS fits of P and Q, Q B P, coarsest triplets) and
V-cycle-preconditioned flexible GMRES to ||B x||_1 / ||x||_1 <= 1e-10, on the
tandem queueing network with 65,536 states (arrival 10/31, service 11/31 and
10/31), r = 16 test vectors, 5 levels, GMRES(20).  The headline runs the
mixed-precision path (FP32 V-cycle and setup relaxation inside FP64 GMRES);
the plain FP64 GPU path is timed beside it on the same chain.

Beside the headline line the same JSON object reports, on the same GPU:
  mcgs_smoother     the same step with multicolour Gauss-Seidel as the
                    V-cycle smoother instead of weighted Jacobi
  roofline          the dominant kernel of a step (coarsest-level solver),
                    timed live with CUDA events
  roofline_sparse   the finest-level block relaxation on a 2048 x 2048
                    tandem queue (4.2M states, inputs far above L2) vs HBM
  learned           network fits vs LS fits on the 2048 x 2048 tandem queue
  batched           256 seeded chains of 1k-65k states, batched vs a loop
  delaunay          random walk on the Delaunay graph of 2^20 points (MIS),
                    plus sets of 3-8 points with the penalised LS fit
  birthdeath        the paper's birth-death table: BAMG, BAMG^2 and
                    GMRES(50) without preconditioning, n = 2^k + 1

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--sections all|none|learned,batched,...] [--no-cpu-baseline]
                  [--no-headline] [--sparse-side S]

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
SECTIONS = ("learned", "batched", "delaunay", "sparse", "birthdeath", "kernels", "mlpfwd")
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (4 partitions x 32)
# DRAM bytes (read + write) of one coarsest_kernel<float> launch of this
# workload from an ncu capture, valid only while the kernel's source file is
# byte-identical to the one captured (else the roofline reports null)
COARSEST_TRAFFIC = {"source": "paper_1402_4005_gb300/csrc/dense.cu",
                    "sha256": "7a303679a004cf5f97f794f4e7196d0602a73bf5c61f156c5e0e3fa5756ae1a1",
                    "bytes": 1741568 + 0}
# the same for one relax_block_kernel<float,16> launch on the 2048 x 2048
# tandem queue (ncu reports MB to two decimals)
SPARSE_TRAFFIC = {"source": "paper_1402_4005_gb300/csrc/blockops.cu",
                  "sha256": "e4ddb26dd524f4c4e237597f9bc1e406775e40abf13a66ebd9de981b5d2752dd",
                  "bytes": 436_170_000 + 239_300_000, "side": 2048}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def load_peaks():
    """HBM GB/s from MEASURED_PEAKS.json (else the fallback figure)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        return float(peaks["hbm_gbs"]), "measured", peaks
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback", {}


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


def max_over_ranks(torch, value: float, world: int) -> float:
    """The slowest rank's value (every rank gets it); NCCL tensors live on
    the GPU, gloo ones on the host."""
    if world <= 1:
        return value
    dist = torch.distributed
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def event_ms(torch, stream, fn, reps=1):
    """Mean CUDA-event time of fn() on `stream` over reps calls (ms)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps, out


def chain_tensors(torch, ch):
    return tuple(torch.from_numpy(a).cuda() for a in (ch.row_ptr, ch.col, ch.val))


# ---------------------------------------------------------------- headline
def gpu_arm(args, rank: int, world: int):
    import torch

    import chaingen as cg
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api

    dev = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    if args.no_headline:                          # sections alone (profiling runs)
        return run_sections(args, api, torch, stream, {})
    ch = cg.tandem(SIDE)
    rp, ci, va = chain_tensors(torch, ch)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step(prec, **extra):
        p = api.bamg_params_default(precision=prec, **KW, **extra)
        h = api.bamg_setup(rp, ci, va, ch.n, p, nx=SIDE, ny=SIDE, stream=stream)
        x, info = api.bamg_solve(h, restart=20, tol=1e-10, stream=stream)
        return h, x, info

    def timed(prec, steps, warmup, **extra):
        times, infos = [], []
        with torch.cuda.stream(stream):
            # at least `warmup` steps and at least a second of them: a GPU
            # that sat idle (e.g. during the build) needs that long to reach
            # its clocks
            t_w, k = time.perf_counter(), 0
            while k < warmup or time.perf_counter() - t_w < 1.0:
                h, x, info = one_step(prec, **extra)
                h.destroy()
                k += 1
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            l0 = api.launch_count()
            for _ in range(steps):
                flush.fill_(1.0)                     # evict the 129 MB L2 between steps
                torch.cuda.synchronize()
                ms, (h, x, info) = event_ms(torch, stream, lambda: one_step(prec, **extra))
                times.append(ms)
                infos.append(info)
                last = (h, x)
            torch.cuda.synchronize()
            launches = api.launch_count() - l0
        return times, infos, last, launches

    with ClockSampler(dev) as clk:
        # nvidia-smi's start-up (driver initialisation) stalls CUDA calls of
        # this process for a moment: let it pass before the warm-up steps
        time.sleep(1.0)
        t_mix, i_mix, (h_mix, x_mix), launches = timed("mixed", args.steps, args.warmup)
    t_64, i_64, (h_64, x_64), _ = timed("fp64", max(3, args.steps // 2), 3)
    # the Gauss-Seidel splitting of Section 3 in multicolour order as the
    # V-cycle smoother (same hierarchy construction)
    try:
        t_gs, i_gs, (h_gs, x_gs), _ = timed("mixed", 3, 3, smoother="mcgs")
        gs = {"ms_per_step": round(statistics.mean(t_gs), 3),
              "setup_ms": round(statistics.mean(i["setup_ms"] for i in i_gs), 3),
              "solve_ms": round(statistics.mean(i["solve_ms"] for i in i_gs), 3),
              "iterations": i_gs[-1]["iterations"], "rel_res_1": i_gs[-1]["rel_res_1"],
              "err_l1_vs_jacobi": None}
        h_gs.destroy()
    except Exception as exc:          # a variant failure must not lose the headline
        gs, x_gs = {"error": f"{type(exc).__name__}: {exc}"[:300]}, None

    ms = max_over_ranks(torch, statistics.mean(t_mix), world)
    err_vs_fp64 = float((x_mix - x_64).abs().sum().item())
    if x_gs is not None:
        gs["err_l1_vs_jacobi"] = float((x_gs - x_mix).abs().sum().item())

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
    out = {
        "ms": ms, "t_mix": t_mix, "i_mix": i_mix, "t_64": t_64, "i_64": i_64, "launches": launches,
        "x_mix": x_mix.cpu().numpy(), "x_64": x_64.cpu().numpy(),
        "clocks": clk.summary(), "err_vs_fp64": err_vs_fp64, "e2e_ms": statistics.mean(e2e),
        "h2d": hrp.nbytes + hci.nbytes + hva.nbytes, "d2h": xh.nbytes,
        "roofline": roofline_coarsest(api, torch, stream, h_mix), "mcgs": gs,
    }
    h_mix.destroy()
    h_64.destroy()
    return run_sections(args, api, torch, stream, out)


def run_sections(args, api, torch, stream, out):
    for name, fn in (("sparse", lambda *a: roofline_sparse(*a, side=args.sparse_side)),
                     ("kernels", kernel_rooflines),
                     ("mlpfwd", lambda a, t, st: mlp_forward_roofline(a, t, st) if "kernels" not in args.sections
                      else {"in": "roofline_kernels"}),
                     ("learned", learned_section), ("batched", batched_section),
                     ("delaunay", delaunay_section), ("birthdeath", birthdeath_section)):
        if name in args.sections:
            try:
                out[name] = fn(api, torch, stream)
            except Exception as exc:          # a section failure must not lose the headline
                out[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- rooflines
def _dense(torch, lv_csr, n):
    rp, col, val = lv_csr["row_ptr"].long(), lv_csr["col"].long(), lv_csr["val"]
    rows = torch.repeat_interleave(torch.arange(n, device="cuda"), rp[1:] - rp[:-1])
    D = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    D[rows, col] = val
    return D


def _max_sm_mhz():
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return 2070.0


def coarsest_flops(n: int) -> float:
    """Algorithmic flops of one coarsest solve (leading terms): Cholesky of M
    and N (2 n^3/3), L_M^{-1} B and L_N^{-1} X^T (2 n^3), two-sided
    Householder bidiagonalization (8 n^3/3), Gauss-Jordan on [B + e w^T | I]
    (3 n^3); the triplet solves are lower order."""
    return (2.0 / 3.0 + 2.0 + 8.0 / 3.0 + 3.0) * n ** 3


def captured_traffic(rec):
    import hashlib
    try:
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            same = hashlib.sha256(f.read()).hexdigest() == rec["sha256"]
    except OSError:
        return None
    return rec["bytes"] if same else None


def roofline_coarsest(api, torch, stream, h):
    """The dominant kernel of a step: the dense coarsest-level solver (one
    16-block cluster, FP32 on the mixed path), timed with CUDA events on the
    stream it is launched on, on the bench hierarchy's own coarsest level."""
    L = h.num_levels - 1
    lv = h.level(L)
    n = lv["n"]
    B, M, N = (_dense(torch, lv[k], n) for k in ("B", "M", "N"))
    r = KW["r"]
    with torch.cuda.stream(stream):
        for _ in range(2):
            api.bamg_step_coarsest(B, M, N, r, prec="mixed", stream=stream)
        torch.cuda.synchronize()
        ms, _ = event_ms(torch, stream, lambda: api.bamg_step_coarsest(B, M, N, r, prec="mixed", stream=stream),
                         reps=5)
    flops = coarsest_flops(n)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = _max_sm_mhz()
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": f"coarsest_kernel<float> (n={n} dense coarsest level, 16-block cluster, "
                                      f"rows in shared memory)",
            "achieved": round(achieved, 4), "peak": round(peak, 1), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 6), "traffic": captured_traffic(COARSEST_TRAFFIC),
            "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {mhz:.0f} MHz",
            "launch_ms": round(ms, 3), "alg_flops": flops,
            "frac_of_cluster_sms": round(achieved / (peak * 16 / sms), 5)}


_CHAIN_CACHE = {}


def _tandem(side):
    import chaingen as cg
    if side not in _CHAIN_CACHE:
        _CHAIN_CACHE[side] = cg.tandem(side)
    return _CHAIN_CACHE[side]


def roofline_sparse(api, torch, stream, side=2048, ld=16):
    """Finest-level FP32 block relaxation (setup hot loop, Algorithm 1) on a
    2048 x 2048 tandem queue: n = 4,194,304 rows, X and Y blocks of 268 MB
    (above L2), two alternating input blocks, CUDA events on the stream."""
    hbm, src, _ = load_peaks()
    ch = _tandem(side)
    rp, ci, va = chain_tensors(torch, ch)
    with torch.cuda.stream(stream):
        Brp, Bci, Bva = api.bamg_step_build_B(rp, ci, va, stream=stream)
        n = ch.n
        rows = torch.repeat_interleave(torch.arange(n, device="cuda"), (Brp[1:] - Brp[:-1]).long())
        diag = Bci.long() == rows
        d = torch.zeros(n, dtype=torch.float64, device="cuda")
        d[rows[diag]] = Bva[diag]
        dinv = (1.0 / d).float()
        va32 = Bva.float()
        Xs = [torch.rand((n, ld), device="cuda", dtype=torch.float32) for _ in range(2)]
        for k in range(4):
            api.bamg_step_relax_block(Brp, Bci, va32, dinv, Xs[k % 2], stream=stream)
        torch.cuda.synchronize()
        reps = 20
        state = {"k": 0}

        def one():
            state["k"] += 1
            return api.bamg_step_relax_block(Brp, Bci, va32, dinv, Xs[state["k"] % 2], stream=stream)
        ms, _ = event_ms(torch, stream, one, reps=reps)
    nnz = int(Bci.numel())
    alg = nnz * (4 + 4) + 4 * (n + 1) + 2 * n * ld * 4 + n * 4
    achieved = alg / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "relax_block_kernel<float,16> (finest level, r=16)",
            "workload": f"tandem queue {side}x{side} (n={n}, nnz(B)={nnz})",
            "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": captured_traffic(SPARSE_TRAFFIC) if side == SPARSE_TRAFFIC["side"] else None,
            "peak_source": src, "launch_us": round(ms * 1e3, 2), "alg_bytes": alg}


# ---------------------------------------------------------------- kernel rooflines (configs 3 and 5)
def per_launch_ms(torch, stream, fn, reps, flush=None):
    """Mean CUDA-event duration of single launches of fn() on `stream`; with
    `flush` (two tensors, each larger than L2) the first is overwritten and
    the second read before every launch, outside the timed interval: each
    launch starts from DRAM, and the read has already written the flush's
    dirty lines back, so they do not compete with the timed kernel."""
    ts = []
    with torch.cuda.stream(stream):
        for _ in range(reps):
            if flush is not None:
                flush[0].fill_(1.0)
                flush[1].sum()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts[1:]) if len(ts) > 1 else ts[0]


def kernel_rooflines(api, torch, stream):
    """Sparse kernels of the config-3 and config-5 steps against the measured
    HBM copy bandwidth: algorithmic bytes per launch (each input read once,
    each output written once; neighbour reuse from L2) over the mean
    CUDA-event duration of single launches, L2 flushed before each.

      relax_block  Delaunay 2^20 walk, FP32 block of 16 (setup relaxation)
      csr_vec      Jacobi sweep of the V-cycle, FP32, and the FGMRES SpMV,
                   FP64, on the finest levels of configs 3 and 5
      ls_fit       P-row fits of the finest Delaunay level (MIS, sets of at
                   most 3 points; FP32 pass plus FP64 refits of flagged rows)
      mlp_forward  network inference on 3.1M fine points (config 5)"""
    import numpy as np
    import chaingen as cg
    hbm, src, _ = load_peaks()
    flush = (torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda"),
             torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda"))
    out = {"peak_gbs": hbm, "peak_source": src,
           "l2": "flushed before every launch (512 MB write, then 256 MB read so no dirty line is left)"}

    def rec(name, alg, ms, **kw):
        gbs = alg / (ms * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "achieved": round(gbs, 1), "frac": round(gbs / hbm, 4), "unit": "GB/s",
                     "launch_us": round(ms * 1e3, 2), "alg_bytes": int(alg), **kw}

    def build(ch):
        rp, ci, va = chain_tensors(torch, ch)
        Brp, Bci, Bva = api.bamg_step_build_B(rp, ci, va, stream=stream)
        n = ch.n
        rows = torch.repeat_interleave(torch.arange(n, device="cuda"), (Brp[1:] - Brp[:-1]).long())
        d = torch.zeros(n, dtype=torch.float64, device="cuda")
        dg = Bci.long() == rows
        d[rows[dg]] = Bva[dg]
        return Brp, Bci, Bva, d

    with torch.cuda.stream(stream):
        for label, ch in (("delaunay_2^20", cg.delaunay_walk(1 << 20, seed=3)), ("tandem_2048^2", _tandem(2048))):
            Brp, Bci, Bva, d = build(ch)
            n, nnz = ch.n, int(Bci.numel())
            wl = f"{label} (n={n}, nnz(B)={nnz})"
            va32, dinv32, dinv64 = Bva.float(), (1.0 / d).float(), 1.0 / d
            if label.startswith("delaunay"):
                ld = 16
                X = torch.rand((n, ld), device="cuda", dtype=torch.float32)
                ms = per_launch_ms(torch, stream, lambda: api.bamg_step_relax_block(
                    Brp, Bci, va32, dinv32, X, keep_col0=True, stream=stream), 8, flush)
                rec("relax_block_fp32_" + label, nnz * 8 + 4 * (n + 1) + 2 * n * ld * 4 + n * 4, ms,
                    kernel="relax_block_kernel<float,16,2>", workload=wl)
            x32, b32, y32 = (torch.rand(n, device="cuda") for _ in range(3))
            ms = per_launch_ms(torch, stream, lambda: api.bamg_step_csr_vec(
                "jacobi", Brp, Bci, va32, x=x32, b=b32, dinv=dinv32, y=y32, stream=stream), 10, flush)
            rec("csr_vec_jacobi_fp32_" + label, nnz * 8 + 4 * (n + 1) + 4 * n * 4, ms,
                kernel="csr_vec_kernel<float,G,kJacobi>", workload=wl)
            x64, y64 = torch.rand(n, device="cuda", dtype=torch.float64), torch.empty(n, device="cuda",
                                                                                     dtype=torch.float64)
            ms = per_launch_ms(torch, stream, lambda: api.bamg_step_csr_vec(
                "spmv", Brp, Bci, Bva, x=x64, y=y64, stream=stream), 10, flush)
            rec("csr_vec_spmv_fp64_" + label, nnz * 12 + 4 * (n + 1) + 2 * n * 8, ms,
                kernel="csr_vec_kernel<double,G,kSpmv>", workload=wl)
            if label.startswith("delaunay"):
                Btrp, Btci, Btva = api.bamg_step_transpose(Brp, Bci, Bva, n, n, stream=stream)
                cf, cmap, nc = api.bamg_step_coarsen_mis(Brp, Bci, Btrp, Btci, 3, 0, stream=stream)
                jrp, jci = api.bamg_step_graph_sets(Brp, Bci, Bva, Btrp, Btci, Btva, cf, 1, 3, stream=stream)
                V = (torch.rand((n, 16), device="cuda") - 0.5).contiguous()
                w = np.ones(16)
                ms = per_launch_ms(torch, stream, lambda: api.bamg_step_ls_fit(jrp, jci, V, w, 16, stream=stream),
                                   6, flush)
                nj = int(jci.numel())
                rec("ls_fit_fp32_" + label, n * 16 * 4 + 4 * (n + 1) + nj * (4 + 8), ms,
                    kernel="ls_fit_kernel<float,float,16,false,false> (+ FP64 refit launch)", workload=wl,
                    fine_points=int(n - nc), set_entries=nj,
                    note="step call: two launches (FP32 pass, FP64 refit of flagged rows) and a host read")
            X = V = None
            torch.cuda.empty_cache()
    out.update(mlp_forward_roofline(api, torch, stream, flush))
    return out


def mlp_forward_roofline(api, torch, stream, flush=None):
    """Network inference (tcgen05) on the 3,145,728 fine points of the
    2048 x 2048 tandem queue (random BF16 features), against HBM."""
    hbm, src, _ = load_peaks()
    if flush is None:
        flush = (torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda"),
                 torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda"))
    with torch.cuda.stream(stream):
        params = api.bamg_mlp_init(seed=5, stream=stream)
        npts = 3 * 2048 * 2048 // 4
        Xf = (torch.rand((npts, 64), device="cuda") * 2 - 1).to(torch.bfloat16)
        ms = per_launch_ms(torch, stream, lambda: api.bamg_mlp_forward(params, Xf, stream=stream), 8, flush)
    alg = npts * (64 * 2 + 16 * 4)
    flops = npts * 2 * (64 * 64 * 2 + 64 * 16)
    gbs = alg / (ms * 1e-3) / 1e9
    return {"mlp_forward_config5": {
        "bound": "hbm", "achieved": round(gbs, 1), "frac": round(gbs / hbm, 4), "unit": "GB/s",
        "launch_us": round(ms * 1e3, 2), "alg_bytes": int(alg), "kernel": "mlp_forward_tc_kernel (tcgen05)",
        "workload": f"{npts} fine points", "flops": flops, "tflops": round(flops / (ms * 1e-3) / 1e12, 2),
        "note": "CUDA events around the step call: the kernel plus its host part (flag set/read, tensor map)"}}


# ---------------------------------------------------------------- learned (config 5)
def learned_section(api, torch, stream, eval_side=2048, train_count=512, rows_per_level=2048):
    """Network fits against LS fits on a 2048 x 2048 tandem queue.  The
    network is trained first, on the LS weights of bootstrap setups of 512
    seeded chains (tandem queues and weighted lattices, sides 64-512; at
    most 2048 seeded rows per level and chain).  Every variant's x is
    compared with an FP64 LS solve run to stagnation (the oracle does not
    finish at 4.2M states), at 1e-10 and at the tolerance that brings the
    1-norm error to 1e-8."""
    import numpy as np
    t0 = time.perf_counter()
    import chaingen as cg
    train = cg.training_mix(train_count, seed=6)
    t_gen = time.perf_counter() - t0
    Xs, Ts, Ms = [], [], []
    dropped = 0
    g = torch.Generator(device="cpu").manual_seed(7)
    with torch.cuda.stream(stream):
        for k, ch in enumerate(train):
            p = api.bamg_params_default(r=16, seed=5 + k, precision="mixed")
            h = api.bamg_setup(*chain_tensors(torch, ch), ch.n, p, nx=ch.nx, ny=ch.ny, stream=stream)
            for l in range(h.num_levels - 1):
                X, T, M = api.bamg_mlp_harvest(h, l, stream=stream)
                # rows whose LS weights blew up (ill-determined fits) are not
                # targets to learn: keep |w| <= 4 on the used slots
                ok = (T.abs() * M).amax(dim=1) <= 4.0
                dropped += int((~ok).sum().item())
                X, T, M = X[ok], T[ok], M[ok]
                if X.shape[0] > rows_per_level:
                    sel = torch.randperm(X.shape[0], generator=g)[:rows_per_level].cuda()
                    X, T, M = X[sel], T[sel], M[sel]
                Xs.append(X); Ts.append(T); Ms.append(M)
            h.destroy()
        X, T, M = torch.cat(Xs), torch.cat(Ts), torch.cat(Ms)
        del Xs, Ts, Ms
        perm = torch.from_numpy(np.random.default_rng(6).permutation(X.shape[0])).cuda()
        X, T, M = X[perm].contiguous(), T[perm].contiguous(), M[perm].contiguous()
        t_h = time.perf_counter()
        params = api.bamg_mlp_init(seed=5, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        losses = api.bamg_mlp_train(params, X, T, M, epochs=40, batch=4096, lr=2e-3, stream=stream)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
    ch = _tandem(eval_side)
    rp, ci, va = chain_tensors(torch, ch)
    res = {"train_rows": int(X.shape[0]), "train_rows_dropped": dropped, "train_chains": len(train),
           "generate_s": round(t_gen, 1),
           "harvest_s": round(t_h - t0 - t_gen, 2), "train_s": round(t_train, 2), "epochs": 40,
           "loss_first": losses[0], "loss_last": losses[-1],
           "workload": f"tandem queue {eval_side}x{eval_side} ({ch.n} states)"}
    del X, T, M
    # reference: FP64 LS fits (tuned to converge) solved to stagnation
    with torch.cuda.stream(stream):
        p = api.bamg_params_default(seed=2, precision="fp64", r=32, max_levels=7, nu_setup=20)
        href = api.bamg_setup(rp, ci, va, ch.n, p, nx=eval_side, ny=eval_side, stream=stream)
        xref, iref = api.bamg_solve(href, restart=20, tol=1e-14, max_iter=3000, stream=stream,
                                    allow_not_converged=True)
        href.destroy()
    res["reference"] = {"how": "FP64 LS hierarchy (r=32, 20 setup relaxations, 7 levels) solved to stagnation",
                        "rel_res_1": iref["rel_res_1"], "iterations": iref["iterations"]}
    err = lambda x: float((x - xref).abs().sum().item())
    # 7 levels (32 x 32 coarsest, solved densely): network fits with the
    # default parameters, and the LS fits with the same parameters and tuned
    # to converge (r = 32, 20 setup relaxations); at the default depth (8
    # levels) both stall, because the deepest levels get b_ii <= 0 rows
    variants = (("learned_mixed", dict(precision="mixed", r=16, max_levels=7, interp="mlp"), 2),
                ("learned_fp64", dict(precision="fp64", r=16, max_levels=7, interp="mlp"), 1),
                ("ls_mixed", dict(precision="mixed", r=16, max_levels=7), 1),
                ("ls_tuned_mixed", dict(precision="mixed", r=32, max_levels=7, nu_setup=20), 2),
                ("learned_default_depth_mixed", dict(precision="mixed", r=16, interp="mlp"), 1),
                ("ls_default_depth_mixed", dict(precision="mixed", r=16), 1))
    for name, kw, reps in variants:
        rows = []
        with torch.cuda.stream(stream):
            for k in range(reps + 1):
                p = api.bamg_params_default(seed=2, mlp_params=params, **kw)
                torch.cuda.synchronize()
                ms, (h, x, info) = event_ms(torch, stream, lambda: (lambda hh: (hh, *api.bamg_solve(
                    hh, restart=20, tol=1e-10, max_iter=400, stream=stream, allow_not_converged=True)))(
                        api.bamg_setup(rp, ci, va, ch.n, p, nx=eval_side, ny=eval_side, stream=stream)))
                if k:
                    rows.append((ms, info))
                if k < reps:
                    h.destroy()
            f = api.bamg_vcycle_factor(h, iters=12, stream=stream)
            info = rows[-1][1]
            res[name] = {"ms_per_step": round(statistics.mean(m for m, _ in rows), 2),
                         "setup_ms": round(statistics.mean(i["setup_ms"] for _, i in rows), 2),
                         "solve_ms": round(statistics.mean(i["solve_ms"] for _, i in rows), 2),
                         "iterations": info["iterations"], "levels": info["levels"],
                         "rel_res_1": info["rel_res_1"], "converged": info["rel_res_1"] <= 1e-10,
                         "vcycle_factor": round(f, 4), "params": {k: v for k, v in kw.items()},
                         "err_l1_vs_reference": err(x)}
            if name in ("learned_mixed", "ls_tuned_mixed", "learned_fp64") and info["rel_res_1"] <= 1e-10:
                res[name]["to_err_1e-8"] = tighten(api, torch, h, stream, err, restart=20)
        h.destroy()
    return res


# ---------------------------------------------------------------- birth-death (Table birthdeath)
def birthdeath_section(api, torch, stream, sizes=(1025, 2049, 4097, 8193, 16385)):
    """The paper's birth-death table: n = 2^k + 1, mu = 0.96, geometric
    coarsening while n > 29, c = 2, r = 8, 3+3 Jacobi; one and two bootstrap
    cycles against GMRES(50) without preconditioning (at most 1000
    iterations).  Iterations to the paper's ||Bx||_2/||x||_2 <= 1e-7 (2-norm
    estimate) and to ||Bx||_1/||x||_1 <= 1e-10, FP64."""
    import chaingen as cg
    out = {"paper_context": {"gmres50": ">1000", "bamg": [3, 3, 3, 4, 4, 4, 5], "bamg2": [1, 1, 1, 1, 1, 2, 2],
                             "sizes": [1025, 2049, 4097, 8193, 16385, 32769, 65537],
                             "note": "the paper counts iterations to 1e-7 in its own norm"}}
    for n in sizes:
        ch = cg.birth_death(n)
        rp, ci, va = chain_tensors(torch, ch)
        row = {}
        with torch.cuda.stream(stream):
            for name, kw in (("bamg", {}), ("bamg2", {"setup_cycles": 2})):
                p = api.bamg_params_default(r=8, coarse_min=29, seed=2, **kw)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = api.bamg_setup(rp, ci, va, ch.n, p, nx=n, ny=1, stream=stream)
                x, info = api.bamg_solve(h, restart=20, tol=1e-10, stream=stream, allow_not_converged=True)
                torch.cuda.synchronize()
                row[name] = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "iters_to_1e7": info["iters_to_1e7"],
                             "iterations": info["iterations"], "levels": info["levels"],
                             "rel_res_1": info["rel_res_1"], "converged": info["rel_res_1"] <= 1e-10}
                if name == "bamg":
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, pinfo = api.bamg_solve(h, restart=50, tol=1e-7, max_iter=1000, plain=True, stream=stream,
                                              allow_not_converged=True)
                    torch.cuda.synchronize()
                    row["gmres50"] = {"ms": round((time.perf_counter() - t0) * 1e3, 2),
                                      "iterations": pinfo["iterations"], "rel_res_1": pinfo["rel_res_1"],
                                      "converged_1e7": pinfo["rel_res_1"] <= 1e-7}
                h.destroy()
        out[str(n)] = row
    return out


# ---------------------------------------------------------------- batched (config 4)
def batched_section(api, torch, stream, count=256):
    """256 seeded chains (weighted lattices and tandem queues of side 32-256,
    Delaunay walks of 1k-64k states, sizes log-uniform: about 4.3M states):
    one batched setup + lock-step FGMRES against a loop of per-chain setups
    and solves, FP32 V-cycle (chains that stall continue with FP64
    V-cycles).  Every chain's x is compared with its reference: the closed
    form (weighted degree for lattices, degree for Delaunay walks) or the
    oracle's direct solve (tandem queues, computed on the host cores while
    the GPU runs)."""
    import numpy as np
    import chaingen as cg
    t0 = time.perf_counter()
    chains = cg.chain_mix(count, seed=4, log_sizes=True)
    t_gen = time.perf_counter() - t0
    p = api.bamg_params_default(r=16, coarse_min=150, coarsening="mis", c_min=1, c_max=3, nu_pre=5, nu_post=5,
                                seed=3, precision="mixed")
    specs = [(c.row_ptr, c.col, c.val, c.n, c.nx, c.ny) for c in chains]
    res = {"chains": count, "states": int(sum(c.n for c in chains)), "generate_s": round(t_gen, 1),
           "size_mix": "log-uniform sides 32-256 (lattices, tandem queues), points 1k-64k (Delaunay)"}
    with torch.cuda.stream(stream):
        b = api.bamg_setup_batched(specs[:8], p, stream=stream)    # warm-up
        api.bamg_solve_batched(b, restart=30, tol=1e-10, stream=stream)
        b.destroy()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        b = api.bamg_setup_batched(specs, p, stream=stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        x, infos = api.bamg_solve_batched(b, restart=30, tol=1e-10, stream=stream)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        off = b.offsets.copy()
        # the same batch solved to 1e-12 (slowly mixing members need a smaller
        # residual for a 1e-8 error)
        x12, infos12 = api.bamg_solve_batched(b, restart=30, tol=1e-12, max_iter=1500, stream=stream)
        torch.cuda.synchronize()
        t12 = (time.perf_counter() - t3) * 1e3
        b.destroy()
        loop_setup = loop_solve = 0.0
        its = []
        for c in chains:
            s0 = time.perf_counter()
            h = api.bamg_setup(c.row_ptr, c.col, c.val, c.n, p, nx=c.nx, ny=c.ny, stream=stream)
            torch.cuda.synchronize()
            s1 = time.perf_counter()
            _, info = api.bamg_solve(h, restart=30, tol=1e-10, stream=stream)
            torch.cuda.synchronize()
            s2 = time.perf_counter()
            loop_setup += s1 - s0
            loop_solve += s2 - s1
            its.append(info["iterations"])
            h.destroy()
    # the oracle's direct solves of the tandem members (error references) run
    # on the host cores only now, after the timed regions
    pool = oracle_pool()
    futs = {k: pool.submit(_tandem_direct, c.nx) for k, c in enumerate(chains) if c.kind == "tandem"}
    bt = (t3 - t1) * 1e3
    lt = (loop_setup + loop_solve) * 1e3
    xh, xh12 = x.cpu().numpy(), x12.cpu().numpy()
    t4 = time.perf_counter()
    worst, worst12 = {}, {}
    for k, c in enumerate(chains):
        if c.kind == "lattice":
            ref = c.meta["wdeg"] / c.meta["wdeg"].sum()
        elif c.kind == "delaunay":
            ref = c.meta["deg"] / c.meta["deg"].sum()
        else:
            ref = futs[k].result()
        for xx, inf, wd in ((xh, infos, worst), (xh12, infos12, worst12)):
            e = float(np.abs(xx[off[k]:off[k + 1]] - ref).sum())
            w = wd.setdefault(c.kind, {"err_l1_max": -1.0})
            if e > w["err_l1_max"]:
                w.update(err_l1_max=e, chain=k, n=c.n, rel_res_1=inf[k]["rel_res_1"],
                         iterations=inf[k]["iterations"])
    pool.shutdown()
    for wd in (worst, worst12):
        for kind, w in wd.items():
            w["reference"] = {"lattice": "closed form (weighted degree)", "delaunay": "closed form (degree)",
                              "tandem": "oracle direct solve (sparse LU of the definition)"}[kind]
    res.update({"batched_ms": round(bt, 1), "batched_setup_ms": round((t2 - t1) * 1e3, 1),
                "batched_solve_ms": round((t3 - t2) * 1e3, 1), "loop_ms": round(lt, 1),
                "loop_setup_ms": round(loop_setup * 1e3, 1), "loop_solve_ms": round(loop_solve * 1e3, 1),
                "speedup": round(lt / bt, 2), "max_rel_res_1": max(i["rel_res_1"] for i in infos),
                "iterations_max": max(i["iterations"] for i in infos),
                "fp64_fallback_chains": sum(1 for i in infos if i.get("fallback_iterations", 0) > 0),
                "loop_iterations_max": max(its), "worst_err_by_kind": worst,
                "err_l1_max": max(w["err_l1_max"] for w in worst.values()),
                "tol_1e-12": {"solve_ms": round(t12, 1), "worst_err_by_kind": worst12,
                              "err_l1_max": max(w["err_l1_max"] for w in worst12.values()),
                              "max_rel_res_1": max(i["rel_res_1"] for i in infos12),
                              "iterations_max": max(i["iterations"] for i in infos12)},
                "reference_wait_s": round(time.perf_counter() - t4, 1)})
    return res


# ---------------------------------------------------------------- Delaunay (config 3)
TIGHTEN = (1e-11, 3e-12, 1e-12, 3e-13, 1e-13)


def tighten(api, torch, h, stream, err_fn, target=1e-8, restart=30):
    """Solve again with tighter tolerances until the 1-norm error against
    the reference is at most `target`; the first tolerance that reaches it,
    with its true residual, iterations and solve time (CUDA events)."""
    rows = []
    for tol in TIGHTEN:
        ms, (x, info) = event_ms(torch, stream, lambda: api.bamg_solve(
            h, restart=restart, tol=tol, max_iter=1500, stream=stream, allow_not_converged=True))
        e = err_fn(x)
        rows.append({"tol": tol, "rel_res_1": info["rel_res_1"], "iterations": info["iterations"],
                     "solve_ms": round(ms, 2), "err_l1": e})
        if e <= target:
            return {"reached": True, **rows[-1]}
    return {"reached": False, "tried": rows}


def delaunay_section(api, torch, stream, npts=1 << 20):
    """Random walk on the Delaunay graph of 2^20 uniform points: MIS
    coarsening, up to 3 interpolation points (the paper's planar-graph
    setting; with the plain fit, sets of 3-8 points give coarse operators
    with b_ii <= 0 at this size and GMRES stalls), r = 16, 5+5 sweeps,
    coarse_min 500.  The variant "mixed_c3to8_ridge" runs sets of 3-8 points
    with the penalised fit (ls_ridge = 0.03).  Each variant reports its
    error against the closed form x ~ degree at ||Bx||_1/||x||_1 <= 1e-10
    and the tolerance that brings that error to 1e-8 (the chain mixes
    slowly, so a 1e-10 residual admits a larger error)."""
    import chaingen as cg
    t0 = time.perf_counter()
    ch = cg.delaunay_walk(npts, seed=3)
    t_gen = time.perf_counter() - t0
    deg = torch.from_numpy(ch.meta["deg"]).cuda()
    xstar = deg / deg.sum()
    err = lambda x: float((x - xstar).abs().sum().item())
    rp, ci, va = chain_tensors(torch, ch)
    res = {"workload": f"Delaunay walk, {npts} points (nnz(A)={ch.nnz})", "generate_s": round(t_gen, 1),
           "reference": "closed form x ~ degree (uniform walk, detailed balance)"}
    for name, prec, reps, extra in (("mixed", "mixed", 2, dict(c_min=1, c_max=3)),
                                    ("fp64", "fp64", 1, dict(c_min=1, c_max=3)),
                                    ("mixed_c3to8_ridge", "mixed", 2, dict(c_min=3, c_max=8, ls_ridge=0.03))):
        p = api.bamg_params_default(r=16, coarsening="mis", nu_pre=5, nu_post=5, coarse_min=500,
                                    seed=3, precision=prec, **extra)
        rows = []
        h = None
        try:
            with torch.cuda.stream(stream):
                for k in range(reps + 1):
                    if h is not None:
                        h.destroy()
                    torch.cuda.synchronize()
                    ms, (h, x, info) = event_ms(torch, stream, lambda: (lambda hh: (hh, *api.bamg_solve(
                        hh, restart=30, tol=1e-10, stream=stream, allow_not_converged="ls_ridge" in extra)))(
                        api.bamg_setup(rp, ci, va, ch.n, p, stream=stream)))
                    if k:
                        rows.append((ms, info))
                info = rows[-1][1]
                res[name] = {"ms_per_step": round(statistics.mean(m for m, _ in rows), 2),
                             "setup_ms": round(statistics.mean(i["setup_ms"] for _, i in rows), 2),
                             "solve_ms": round(statistics.mean(i["solve_ms"] for _, i in rows), 2),
                             "iterations": info["iterations"], "levels": info["levels"],
                             "rel_res_1": info["rel_res_1"],
                             "op_cplx": round(info["op_cplx"], 3), "grid_cplx": round(info["grid_cplx"], 3),
                             "err_l1_vs_closed_form": err(x)}
                res[name]["to_err_1e-8"] = tighten(api, torch, h, stream, err)
                h.destroy()
        except Exception as exc:          # a variant failure keeps the other rows
            res[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.synchronize()
            continue
        if "ls_ridge" in extra:
            res[name]["ls_ridge"] = extra["ls_ridge"]
            res[name]["sets"] = "3-8 points"
    return res


# ---------------------------------------------------------------- CPU baseline
def cpu_oracle_step(side=SIDE, xpath=None):
    """One oracle setup + solve of the same workload (plain numpy/scipy);
    with xpath the oracle's x is saved there (.npy)."""
    import numpy as np
    import chaingen as cg
    from oracle import setup as S
    from oracle import solve as So
    ch = cg.tandem(side)
    t0 = time.perf_counter()
    H = S.bamg_setup(ch.csr(), S.Params(**KW), grid=(side, side))
    x, its, _ = So.bamg_solve(H, tol=1e-10, restart=20)
    ms = (time.perf_counter() - t0) * 1e3
    if xpath:
        np.save(xpath, x)
    return ms, its


def direct_reference(side=SIDE, xpath=None):
    """The stationary vector from its definition (sparse LU, oracle)."""
    import numpy as np
    import chaingen as cg
    from oracle import solve as So
    t0 = time.perf_counter()
    x = So.direct_nullvector(cg.tandem(side).csr())
    if xpath:
        np.save(xpath, x)
    return (time.perf_counter() - t0) * 1e3


def cpu_baseline_subprocess(steps=1, threads=1, xpath=None, timeout=900):
    """Time the oracle in a child process with `threads` BLAS threads."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r=[bench.cpu_oracle_step(xpath=%r if k == 0 else None) for k in range(%d)]; print(json.dumps(r))"
            % (ROOT, xpath, steps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
    if out.returncode != 0:
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


def _tandem_direct(side):
    """Worker of the spawn pool: oracle stationary vector of a tandem queue."""
    import chaingen as cg
    from oracle import solve as So
    return So.direct_nullvector(cg.tandem(side).csr())


def oracle_pool(workers=None):
    """Process pool for oracle work that overlaps the GPU sections (spawned,
    so no child inherits a CUDA context)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(max_workers=workers or max(1, min(8, (os.cpu_count() or 2) - 1)),
                               mp_context=mp.get_context("spawn"))


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--sections", default="all",
                    help="comma list of " + ",".join(SECTIONS) + ", or all / none")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-headline", action="store_true",
                    help="run the selected sections only and print their JSON (for profiling)")
    ap.add_argument("--sparse-side", type=int, default=2048,
                    help="grid side of the tandem queue of the sparse roofline section")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.sections = (set(SECTIONS) if args.sections == "all" else set() if args.sections == "none"
                     else set(args.sections.split(",")))
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
    if rank != 0:
        args.sections = set()               # replicas time the headline only
    r = gpu_arm(args, rank, world)
    if rank != 0:
        return
    if args.no_headline:
        print(json.dumps({"sections_only": True, **r}))
        return
    cpu = cpu_all = None
    acc = {}
    if not args.no_cpu_baseline and world == 1:
        import numpy as np
        import tempfile
        tmp = tempfile.mkdtemp(prefix="bamg_bench_")
        xo_path, xd_path = os.path.join(tmp, "x_oracle.npy"), os.path.join(tmp, "x_direct.npy")
        res = cpu_baseline_subprocess(1, threads=1, xpath=xo_path)
        if res:
            cpu = {"value": round(res[0][0], 1), "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": "one full step: oracle setup + GMRES solve of the 256x256 tandem chain "
                             "(BLAS threads pinned to 1)"}
        ncores = os.cpu_count() or 1
        res_all = cpu_baseline_subprocess(1, threads=ncores)
        if res_all:
            cpu_all = {"value": round(res_all[0][0], 1), "unit": "ms", "cores": ncores, "kind": "oracle",
                       "sample": "the same step with BLAS on every host core (the sparse parts of the oracle "
                                 "stay single-threaded)"}
        # accuracy of the GPU results against the oracle (same workload)
        t_direct = direct_reference(xpath=xd_path)
        xd = np.load(xd_path)
        acc = {"err_l1_vs_direct": {"mixed": float(np.abs(r["x_mix"] - xd).sum()),
                                    "fp64": float(np.abs(r["x_64"] - xd).sum()),
                                    "reference": "oracle direct solve of B x = 0, sum 1 (sparse LU)",
                                    "reference_ms": round(t_direct, 1)}}
        if os.path.exists(xo_path):
            xo = np.load(xo_path)
            acc["err_l1_vs_oracle"] = {"mixed": float(np.abs(r["x_mix"] - xo).sum()),
                                       "fp64": float(np.abs(r["x_64"] - xo).sum()),
                                       "oracle_vs_direct": float(np.abs(xo - xd).sum())}
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
        "mcgs_smoother": r["mcgs"],
        "e2e": {"value": round(r["e2e_ms"], 3), "unit": "ms", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"],
        "roofline": r["roofline"],
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        **acc,
        "clocks": r["clocks"],
    }
    for k in ("sparse", "kernels", "learned", "batched", "delaunay", "birthdeath"):   # mlpfwd: profiling runs only
        if k in r:
            line["roofline_sparse" if k == "sparse" else "roofline_kernels" if k == "kernels" else k] = r[k]
    print(json.dumps(line))


if __name__ == "__main__":
    main()
