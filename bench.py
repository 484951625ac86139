#!/usr/bin/env python
"""Benchmark of the GB300 PDLP library (prints one JSON line).

Workload (default): the 100k x 250k MIP-relaxation-shaped planted LP with about
1.5M nonzeros (power-law row lengths, |values| log-uniform in [1e-3, 1e3],
60% inequality rows, 10% free variables).  One step = the whole hot path on
inputs already resident in HBM: pdlp_create (validation, K^T, Ruiz +
Pock-Chambolle preconditioning, transform, graph capture) then pdlp_solve
(Algorithm 1 with restarts, primal-weight updates and the Eq. (15) checks),
float64, stopped at an iteration cap.  value = accepted PDHG iterations per
second over the timed steps (all ranks).  The L2 cache is flushed (256 MiB
write) between timed steps.

Also reported: the roofline of the dominant kernel (the persistent step
kernel: algorithmic bytes of its step attempts over their CUDA-event time);
time to 1e-8 relative KKT error (Eq. (15)) on the 1M-node PageRank LP,
float64 against float32 inner solves with float64 refinement; the batched
solve of 4096 small planted LPs (LPs/s and aggregate iterations/s to 1e-6
and 1e-8, with the autotuner's lanes per row); the unrolled map with its
adjoint on the 20k x 50k LP (T = 500, checkpoint every 50); the end-to-end
rate through the C ABI with host buffers; and the CPU oracle timed on a
bounded sample of the same workload.  `--impl reference` times only the CPU
oracle.  `--stepped` launches the same kernels from a host loop instead of
one CUDA graph per solve (for profilers that cannot see inside conditional
graph nodes).

Multi-GPU (torchrun): every rank solves its own replica (no data-path
collective); value = the ranks' iterations / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time-to-1e-8 rel KKT & PDHG iter/s (HBM GB/s vs peak); FP32+refine vs FP64"
# dram__bytes_read.sum + dram__bytes_write.sum per step attempt of the
# persistent step kernel from one ncu capture each (one launch = one chunk of
# about 40 attempts; see profiles/); drop an entry whenever the kernel changes
# DRAM bytes per step attempt from one-pass ncu captures of the current
# kernels (profiles/k_persist_pagerank1m_mip100k.md); a kernel changed since
# its capture has no entry here (the bench line then reports null) and its
# last figure in STALE_TRAFFIC, named in the line's note
CAPTURED_TRAFFIC = {"pagerank_1m_fp32": 1.936e8}
STALE_TRAFFIC = {"mip_100k": 1.335e6, "pagerank_1m_fp64": 3.275e8}
L2_BYTES = 129e6  # GB300 L2 capacity
WORKLOADS = ("mip_100k", "pagerank_1m", "planted_200x500")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="mip_100k", choices=WORKLOADS)
    ap.add_argument("--iter-cap", type=int, default=20000)
    ap.add_argument("--no-tol", action="store_true", help="skip the time-to-tolerance runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch and unroll lines")
    ap.add_argument("--stepped", action="store_true", help="host-stepped kernels instead of one graph per solve")
    ap.add_argument("--mip-cap-s", type=float, default=20.0,
                    help="time cap of each time-to-1e-8 solve of the MIP-shaped LP")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="only solve the first N LPs of the 4096-LP batch twice (tuning, then one launch "
                         "between cudaProfilerStart / Stop, for ncu --profile-from-start off) and exit")
    ap.add_argument("--profile-precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--profile-solve", action="store_true",
                    help="only create and solve --workload once in --profile-precision, host-stepped "
                         "(use_graph = 0, so that ncu sees every kernel), capped at --iter-cap iterations, "
                         "and exit")
    ap.add_argument("--profile-unroll", action="store_true",
                    help="only run the unrolled map (T = 500, checkpoint 50) and its adjoint on the 20k x 50k "
                         "LP twice, the second time between cudaProfilerStart / Stop, and exit")
    return ap.parse_args()


def _make(workload):
    import lpgen
    if workload == "mip_100k":
        return lpgen.mip_relaxation_100k()
    if workload == "pagerank_1m":
        return lpgen.pagerank_1m()
    return lpgen.small_planted()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _alg_bytes(lp, fp):
    """Algorithmic bytes of one step attempt's two kernels (each array once).
    primal (over the rows of K^T): values + column indices + row pointers of
    K^T, y gathered once, c, l, u, x, xs read, x', xs' written.  dual (over the
    rows of K): values + indices + row pointers of K, x' gathered once, y, q,
    K x, ys, y-lower-bound read, y', K x', ys' written."""
    m, n, nnz = lp.m, lp.n, lp.nnz
    v = 8 if fp == 64 else 4
    primal = nnz * (v + 4) + 4 * (n + 1) + v * m + 7 * v * n
    dual = nnz * (v + 4) + 4 * (m + 1) + v * n + 8 * v * m
    return primal, dual


def _survey_bytes(m, n, nnz, fp):
    """Algorithmic bytes of one step attempt by the per-unit figure of the
    measurement plan: both matrices' values and indices (2 nnz (v + 4)), row
    starts 4 (m + n), one read of each gathered vector v (m + n), and the
    vector streams of the two epilogues v (10 n + 9 m), with v the element
    size of the iteration (8 for float64; 4 for float32, whose iterate and
    running-sum vectors are float32 here)."""
    v = 8 if fp == 64 else 4
    return 2 * nnz * (v + 4) + 4 * (m + n) + v * (m + n) + v * (10 * n + 9 * m)


def aggregate_over_ranks(elapsed, iters, device=None):
    """Whole-job figures of N replicas: the slowest rank's timed seconds and
    the iterations of all ranks (torch.distributed, any backend; one process
    per GPU).  Without an initialised process group: the rank's own."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(elapsed), float(iters)
    t = torch.tensor([float(elapsed), float(iters)], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t[1:].clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())


def _batch_line(P):
    """4096 planted LPs (m in [20, 400], n in [50, 1000], 5% density) in one
    persistent launch per call (two for float32 + float64 refinement): LPs/s
    and iterations/s to 1e-6 and 1e-8."""
    import lpgen
    import torch
    lps = lpgen.batch_4096()
    out = {"workload": "batch_4096", "count": len(lps), "nnz_total": int(sum(lp.nnz for lp in lps))}
    P.solve_batch(lps[:256], rel_tol=1e-6, iter_limit=2000)  # autotuner + warm-up on a slice
    for name, prec, tol in (("fp64_1e-6", P.PDLP_FP64, 1e-6), ("fp64_1e-8", P.PDLP_FP64, 1e-8),
                            ("fp32_1e-6", P.PDLP_FP32, 1e-6), ("fp32_refine_1e-6", P.PDLP_FP32_REFINE, 1e-6),
                            ("fp32_refine_1e-8", P.PDLP_FP32_REFINE, 1e-8)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, rs = P.solve_batch(lps, precision=prec, rel_tol=tol, iter_limit=20000)
        dt = time.perf_counter() - t0
        its = sum(r["iters"] for r in rs)
        opt = sum(1 for r in rs if r["status_name"] == "OPTIMAL")
        out[name] = {"seconds": dt, "lps_per_s": len(lps) / dt, "iter_per_s": its / dt, "optimal": opt,
                     "iter_cap": 20000}
    lk, lt = P.batch_lanes(P.PDLP_FP64)
    lk32, lt32 = P.batch_lanes(P.PDLP_FP32)
    out["autotuned_lanes_per_row"] = {
        "buckets_mean_row_len": ["<8", "<16", "<32", "<64", ">=64"],
        "fp64_K": lk.tolist(), "fp64_KT": lt.tolist(), "fp32_K": lk32.tolist(), "fp32_KT": lt32.tolist()}
    return out


def _ablation_line(P):
    """KKT passes to 1e-8 on the 200 x 500 planted LP with each enhancement of
    Section 3 switched off in turn, the alternatives of Appendix C (the
    Malitsky-Pock line search at the paper's best setting, the "theory"
    restart mode, presolve-lite), and Section 2's baseline PDHG (constant
    eta = 0.9 / ||K||_2, omega = 1, no restarts, no scaling): the axes of the
    paper's ablation study and of its Figure 1 comparison."""
    import lpgen
    lp = lpgen.small_planted()
    cap = 200000
    variants = {
        "pdlp": {},
        "no_restarts": {"adaptive_restart": 0},
        "fixed_primal_weight": {"pw_update": 0},
        "no_preconditioning": {"ruiz_iters": 0, "pock_chambolle": 0},
        "constant_step": {"step_policy": 1},
        "malitsky_pock": {"step_policy": 2, "mp_breaking": 1.0, "mp_downscaling": 0.5, "mp_interpolation": 0.4},
        "restart_theory": {"restart_to_current": 0, "beta_suff": 0.37, "beta_nec": 0.37},
        "presolve_lite": {"presolve": 1},
        "baseline_pdhg": {"step_policy": 1, "omega0": 1.0, "adaptive_restart": 0, "pw_update": 0,
                          "ruiz_iters": 0, "pock_chambolle": 0},
    }
    out = {"workload": "planted_200x500", "rel_tol": 1e-8, "iter_cap": cap}
    for name, kw in variants.items():
        _, _, r = P.solve(lp, rel_tol=1e-8, iter_limit=cap, **kw)
        out[name] = {"kkt_passes": r["kkt_passes"], "status": r["status_name"], "seconds": r["seconds"]}
    return out


def _unroll_line(P, dev, sptr):
    """Unrolled map (T = 500, checkpoint every 50) and its adjoint on the
    20k x 50k planted LP with loss 1/2 ||x_T - x_target||^2."""
    import lpgen
    import torch
    lp = lpgen.unroll_20k()
    target = np.random.default_rng(4).standard_normal(lp.n)
    with P.Context.from_lp(lp, stream=sptr) as ctx:
        ctx.unroll(500, 50)
        ctx.grad(np.zeros(lp.n))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, _, _ = ctx.unroll(500, 50)
        t1 = time.perf_counter()
        ctx.grad(x - target)
        t2 = time.perf_counter()
    return {"workload": "mip_20k_50k (m=20,000, n=50,000, nnz=%d)" % lp.nnz, "T": 500, "ckpt_every": 50,
            "forward_s": t1 - t0, "backward_s": t2 - t1, "backward_over_forward": (t2 - t1) / (t1 - t0)}


def _attempt_ms(ctx, reps=30):
    """Mean CUDA-event time of one step attempt on the context's step engine
    (the persistent kernel's per-attempt time, or the two launches of the
    per-launch engines) and the engine's name."""
    kp, kd, kc, _ = ctx.time_step_kernels(reps)
    if kc > 0:
        return kc, "k_persist (persistent warp-chunk kernel)"
    slab = ctx.last_engine == 2
    return kp + kd, ("k_primal_slab + k_dual_slab (slab kernels)" if slab else "k_primal + k_dual (warp chunks)")


def _pagerank_lines(P, T, dev, sptr, flush, peak, peak_src, reps=3):
    """On the 1M-node PageRank LP (working set far above L2): the HBM roofline
    of the step attempt in float64 and float32, and the time to 1e-8 relative
    KKT error (Eq. (15)) in float64 against float32 + refinement, `reps`
    times each; the same times on the 100k-node PageRank LP (Table 2's
    family)."""
    import lpgen
    import torch
    out = {}
    pr = lpgen.pagerank_1m()
    pin = [T(pr.row_ptr), T(pr.col_idx), T(pr.val), T(pr.c), T(pr.q), T(pr.l), T(pr.u), T(pr.ineq)]
    roof = {}
    for name, prec, fp in (("fp64", P.PDLP_FP64, 64), ("fp32", P.PDLP_FP32, 32)):
        c = P.Context(*pin, pr.m, pr.n, precision=prec, stream=sptr, iter_limit=400)
        c.solve()
        ms, eng = _attempt_ms(c)
        c.close()
        b = _survey_bytes(pr.m, pr.n, pr.nnz, fp)
        ach = b / (ms * 1e-3) / 1e9
        roof[name] = {"bound": "hbm", "kernel": eng, "achieved": ach, "peak": peak, "unit": "GB/s",
                      "frac": ach / peak, "peak_source": peak_src + " burst copy (MEASURED_PEAKS.json hbm_gbs)",
                      "traffic": CAPTURED_TRAFFIC.get(f"pagerank_1m_{name}"),
                      "algorithmic_bytes_per_attempt": b, "attempt_ms": ms,
                      "note": _roofline_note(b, f"pagerank_1m_{name}")}
    out["roofline_hbm"] = {"workload": "pagerank_1m (n=1,000,000, nnz=7,999,982)", **roof}

    def to_tol(lp, pins, label):
        res = {"workload": label, "rel_tol": 1e-8, "repeats": reps}
        for name, prec in (("fp64", P.PDLP_FP64), ("fp32_refine", P.PDLP_FP32_REFINE)):
            runs = []
            for _ in range(reps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                c3 = P.Context(*pins, lp.m, lp.n, precision=prec, stream=sptr, time_limit_s=120.0)
                _, _, r3 = c3.solve()
                torch.cuda.synchronize(dev)
                runs.append({"seconds": time.perf_counter() - t0, "status": r3["status_name"],
                             "iters": r3["iters"], "rel_kkt": r3["rel_kkt"], "refine_rounds": r3["refine_rounds"],
                             "finish_iters": r3["finish_iters"]})
                c3.close()
            secs = [r["seconds"] for r in runs]
            res[name] = {"median_seconds": float(np.median(secs)), "min_seconds": min(secs),
                         "max_seconds": max(secs), "iters": [r["iters"] for r in runs],
                         "status": [r["status"] for r in runs], "rel_kkt": [r["rel_kkt"] for r in runs],
                         "refine_rounds": [r["refine_rounds"] for r in runs],
                         "finish_iters": [r["finish_iters"] for r in runs]}
        return res

    out["time_to_tol"] = to_tol(pr, pin, "pagerank_1m (n=1,000,000, nnz=7,999,982)")
    del pin
    p1 = lpgen.pagerank(100_000, seed_key=(2, 1), name="pagerank_100k")
    pin = [T(p1.row_ptr), T(p1.col_idx), T(p1.val), T(p1.c), T(p1.q), T(p1.l), T(p1.u), T(p1.ineq)]
    out["time_to_tol_pagerank_100k"] = to_tol(p1, pin, f"pagerank_100k (n=100,000, nnz={p1.nnz})")
    return out


def _mip_time_to_tol(P, inputs, lp, dev, sptr, flush, cap_s):
    """Time to 1e-8 on the 100k x 250k MIP-shaped LP, float32 + refinement
    against float64: each run stops at OPTIMAL, at a limit of the method, or
    at cap_s seconds of solve time; float64 is also run for exactly the wall
    time the refinement took, so both precisions are compared at equal time
    (status, accepted iterations, relative KKT error and its three terms)."""
    import torch

    def run(prec, cap):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        c = P.Context(*inputs, lp.m, lp.n, precision=prec, stream=sptr, time_limit_s=cap, iter_limit=10 ** 9,
                      kkt_pass_limit=10 ** 9)
        _, _, r = c.solve()
        torch.cuda.synchronize(dev)
        c.close()
        return {"seconds": time.perf_counter() - t0, "status": r["status_name"], "iters": r["iters"],
                "rel_kkt": r["rel_kkt"], "rel_gap": r["rel_gap"], "rel_pres": r["rel_pres"],
                "rel_dres": r["rel_dres"], "refine_rounds": r["refine_rounds"], "finish_iters": r["finish_iters"]}

    res = {"workload": "mip_100k", "rel_tol": 1e-8, "time_cap_s": cap_s}
    res["fp32_refine"] = run(P.PDLP_FP32_REFINE, cap_s)
    res["fp64"] = run(P.PDLP_FP64, cap_s)
    # a refinement that used the whole cap (its float64 finish runs to the
    # time limit) is already compared at equal time by the capped float64 run
    t_ref = res["fp32_refine"]["seconds"]
    res["fp64_same_time"] = res["fp64"] if t_ref >= 0.95 * cap_s else run(P.PDLP_FP64, t_ref)
    return res


def _roofline_note(ws_bytes, key=None):
    """How to read `achieved` for a step attempt touching ws_bytes (and where
    `traffic` comes from for the capture key)."""
    where = ("fits in the 129 MB L2: algorithmic GB/s, not DRAM GB/s" if ws_bytes < L2_BYTES else
             "exceeds the 129 MB L2: streamed from DRAM every attempt")
    note = f"working set ~{ws_bytes / 1e6:.0f} MB {where}; "
    if key in STALE_TRAFFIC:
        return note + (f"traffic null: the kernel changed after its last ncu capture, which gave "
                       f"{STALE_TRAFFIC[key] / 1e6:.4g} MB of DRAM per attempt")
    return note + "traffic = DRAM bytes per attempt from one ncu capture of this kernel on this workload"


def run_reference(args):
    """The CPU oracle, as it stands, on the same workload and metric."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    lp = _make(args.workload)
    oracle.build()
    cap = {"mip_100k": 300, "pagerank_1m": 40, "planted_200x500": 20000}[args.workload]
    for _ in range(args.warmup):
        oracle.solve(lp, iter_limit=max(1, cap // 10))
    its, secs = 0, 0.0
    for _ in range(args.steps):
        t = time.perf_counter()
        _, _, r = oracle.solve(lp, iter_limit=cap)
        secs += time.perf_counter() - t
        its += r["iters"]
    value = its / secs
    sample = f"{args.workload}: each step = oracle PDLP (setup + {cap} iterations), {args.steps} steps"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "PDHG iter/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": args.workload, "m": lp.m, "n": lp.n, "nnz": lp.nnz,
                                            "iter_cap": cap},
           "cpu_baseline": {"value": value, "unit": "PDHG iter/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "PDHG iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2106_04756_gb300 as P
    from paper_2106_04756_gb300 import build
    build.build()
    if args.profile_unroll:
        import lpgen
        lp = lpgen.unroll_20k()
        target = np.random.default_rng(4).standard_normal(lp.n)
        with P.Context.from_lp(lp) as ctx:
            x, _, _ = ctx.unroll(500, 50)
            ctx.grad(x - target)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            x, _, _ = ctx.unroll(500, 50)
            ctx.grad(x - target)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        print(json.dumps({"profile_unroll": "mip_20k_50k", "T": 500, "ckpt_every": 50}))
        return
    if args.profile_solve:
        lp = _make(args.workload)
        prec = P.PDLP_FP64 if args.profile_precision == "fp64" else P.PDLP_FP32
        with P.Context.from_lp(lp, precision=prec, iter_limit=args.iter_cap, use_graph=0) as ctx:
            _, _, r = ctx.solve()
        print(json.dumps({"profile_solve": args.workload, "precision": args.profile_precision,
                          "iters": r["iters"], "kkt_passes": r["kkt_passes"], "restarts": r["restarts"]}))
        return
    if args.profile_batch > 0:
        import lpgen
        lps = lpgen.batch_4096()[:args.profile_batch]
        prec = P.PDLP_FP64 if args.profile_precision == "fp64" else P.PDLP_FP32
        P.solve_batch(lps, precision=prec, rel_tol=1e-6, iter_limit=20000)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, _, rs = P.solve_batch(lps, precision=prec, rel_tol=1e-6, iter_limit=20000)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_batch": len(lps), "precision": args.profile_precision,
                          "optimal": sum(r["status_name"] == "OPTIMAL" for r in rs),
                          "iters": sum(r["iters"] for r in rs)}))
        return
    lp = _make(args.workload)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    def T(a):
        return torch.as_tensor(np.asarray(a)).to(dev)

    inputs = [T(lp.row_ptr), T(lp.col_idx), T(lp.val), T(lp.c), T(lp.q), T(lp.l), T(lp.u), T(lp.ineq)]
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    use_graph = 0 if args.stepped else 1

    def step(cap, precision=P.PDLP_FP64, keep=False):
        ctx = P.Context(*inputs, lp.m, lp.n, precision=precision, iter_limit=cap, stream=sptr, use_graph=use_graph)
        xo = torch.empty(lp.n, dtype=torch.float64, device=dev)
        yo = torch.empty(lp.m, dtype=torch.float64, device=dev)
        _, _, r = ctx.solve(x_out=xo, y_out=yo)
        if keep:
            return ctx, r
        ctx.close()
        return None, r

    for _ in range(args.warmup):
        step(args.iter_cap)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = attempts = evals = 0
    results = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        _, r = step(args.iter_cap)
        ev[k][1].record(stream)
        iters += r["iters"]
        attempts += r["kkt_passes"]
        evals += r["iters"] // 40 + 1
        results.append(r)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    elapsed, total_iters = aggregate_over_ranks(elapsed, iters, dev if ws > 1 else None)
    value = total_iters / elapsed
    if rank != 0:
        return

    # ---- roofline of the dominant kernel: the persistent step kernel.  Each
    # launch runs the step attempts between two evaluations; its mean time
    # per attempt comes from CUDA events around `reps` launches on this
    # stream, continuing from the state of a solve of the same workload.
    ctx, _ = step(args.iter_cap, keep=True)
    kp, kd, kc, ke = ctx.time_step_kernels(50)
    ctx.close()
    bp, bd = _alg_bytes(lp, 64)
    peak, peak_src = _peaks()
    if kc > 0:
        # one attempt is one unit of the measurement plan's per-unit figure
        ba = _survey_bytes(lp.m, lp.n, lp.nnz, 64)
        achieved = ba / (kc * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_persist<double> (persistent step attempts: K^T y + primal "
                    "projection, grid barrier, K x' + dual projection, step test)",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": peak_src + " burst copy (MEASURED_PEAKS.json hbm_gbs)", "traffic": None,
                    "algorithmic_bytes_per_attempt": ba, "attempt_ms": kc,
                    "note": _roofline_note(ba, args.workload)}
        if args.workload in CAPTURED_TRAFFIC:
            roofline["traffic"] = CAPTURED_TRAFFIC[args.workload]
    else:
        dom = ("dual", kd, bd) if kd >= kp else ("primal", kp, bp)
        achieved = dom[2] / (dom[1] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"k_{dom[0]}<double>", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
                    "algorithmic_bytes_per_launch": dom[2], "launch_ms": dom[1]}
    kernels = {"persistent_attempt_ms": kc, "primal_ms": kp, "dual_ms": kd, "primal_bytes": bp, "dual_bytes": bd,
               "primal_gbs": bp / (kp * 1e-3) / 1e9, "dual_gbs": bd / (kd * 1e-3) / 1e9,
               "persistent_evaluation_ms": ke}
    # cost of an evaluation (every 40 iterations: Eq. (15) terms, normalized
    # gaps, restart decision, restart) from the timed solves: solve time minus
    # the step attempts at the timed attempt duration, per evaluation
    evaluation = None
    if kc > 0:
        per = [((r["seconds"] - r["kkt_passes"] * kc * 1e-3) / (r["iters"] // 40 + 1), r["seconds"],
                r["iters"] // 40 + 1) for r in results]
        us = float(np.median([p[0] for p in per])) * 1e6
        evaluation = {"us_per_evaluation": us,
                      "share_of_solve": float(np.median([p[0] * p[2] / p[1] for p in per])),
                      "basis": "device-timed solve minus kkt_passes x the timed persistent attempt, per "
                               "evaluation (a chunk's first attempt that reuses the evaluation's K^T y counts as "
                               "evaluation time saved)"}
    # float32 arithmetic on the same workload
    ctx32, r32 = step(args.iter_cap, precision=P.PDLP_FP32, keep=True)
    kp32, kd32, kc32, _ = ctx32.time_step_kernels(50)
    ctx32.close()
    bp32, bd32 = _alg_bytes(lp, 32)
    kernels.update({"fp32_persistent_attempt_ms": kc32, "fp32_primal_ms": kp32, "fp32_dual_ms": kd32,
                    "fp32_attempt_gbs": (bp32 + bd32) / (kc32 * 1e-3) / 1e9 if kc32 > 0 else None,
                    "fp32_iter_per_s": r32["iters"] / r32["seconds"]})

    # ---- end to end through the C ABI with host buffers
    e2e_steps = 2
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(e2e_steps):
        with P.Context.from_lp(lp, iter_limit=args.iter_cap, stream=sptr) as c2:
            x_h, y_h, r2 = c2.solve()
        e2e_iters += r2["iters"]
    torch.cuda.synchronize(dev)
    e2e_t = time.perf_counter() - t0
    h2d = 4 * (lp.m + 1) + 12 * lp.nnz + 8 * (3 * lp.n + lp.m) + lp.m
    d2h = 8 * (lp.n + lp.m) + 2 * 8 * 16
    e2e = {"value": e2e_iters / e2e_t, "unit": "PDHG iter/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- PageRank: HBM roofline of the step attempt, time to 1e-8 (3 repeats,
    # float64 vs float32 + refinement, 1M and 100k nodes); the MIP-shaped LP
    # itself solved under a time cap in both precisions
    tol = None
    pagerank = {}
    if not args.no_tol:
        if args.workload != "pagerank_1m":
            pagerank = _pagerank_lines(P, T, dev, sptr, flush, peak, peak_src)
        if args.workload == "mip_100k":
            pagerank["time_to_tol_mip_100k"] = _mip_time_to_tol(P, inputs, lp, dev, sptr, flush, args.mip_cap_s)
        tol = pagerank.pop("time_to_tol", None)

    # ---- CPU oracle on a bounded sample of the same workload
    cpu = None
    if not args.no_cpu:
        import oracle
        oracle.build()
        cap = {"mip_100k": 600, "pagerank_1m": 60, "planted_200x500": 20000}[args.workload]
        t0 = time.perf_counter()
        _, _, ro = oracle.solve(lp, iter_limit=cap)
        ct = time.perf_counter() - t0
        cpu = {"value": ro["iters"] / ct, "unit": "PDHG iter/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.workload}, oracle setup + first {cap} iterations ({ct:.1f} s)"}

    extra = {}
    if not args.no_extra:
        extra["batch"] = _batch_line(P)
        extra["unroll"] = _unroll_line(P, dev, sptr)
        extra["ablation"] = _ablation_line(P)

    # per solve: ~120 create/setup launches, 6 per evaluation (persistent
    # step kernel, persistent evaluation, 3 gap passes, finish), 5 more per
    # restart (apply, 3 gap passes of the restart point, book-keeping) + 8
    restarts = sum(r["restarts"] for r in results)
    launches_per_step = 120 + (6 * evals + 5 * restarts) / args.steps + 8
    out = {"metric": METRIC, "value": value, "unit": "PDHG iter/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "m": lp.m, "n": lp.n, "nnz": lp.nnz, "precision": "fp64",
                      "iter_cap": args.iter_cap, "parallelism": f"replicas x{ws}",
                      "l2": "flushed between steps (256 MiB write)",
                      "rel_kkt_at_cap": float(np.median([r["rel_kkt"] for r in results]))},
           "roofline": roofline, "kernels": kernels, "evaluation": evaluation, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(launches_per_step * args.steps),
           "gpu_launches_basis": ("not a profiler count: kernel nodes the solve graph executes per create + solve "
                                  "(about 120 set-up launches; 6 per evaluation: persistent step kernel, persistent "
                                  "evaluation, three gap passes, finish; 5 more per restart: apply, three gap passes "
                                  "of the restart point, book-keeping; 8 at the end), times the evaluations and "
                                  "restarts the device counted"),
           "clocks": clk, "time_to_tol": tol, **pagerank, **extra}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
