"""Benchmark: time to solve the advection-diffusion Schur system with adaptive
BDDC-GMRES to relative residual 1e-8 on one GB300.

Workload (default): 4x4x4 subdomains, H/h = 8 (32^3 hexahedra, 29 791 dofs),
nu = 0.01, beta = (1, 0.5, 0.25), f = 1, GMRES(50), Theta_E = 10,
Theta_F = 1 + ln 8.  A step is the whole hot path for one synthetic input:
assembly, batched subdomain factorisation and Schur complements, face GEPs,
edge GEPs on prior-selected primal constraints, constrained local solvers,
coarse space, then condensation, preconditioned GMRES and interior recovery,
in the mixed-precision solver (FP32 factors and operators, FP64 refinement).
The plain FP64 GPU path is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle as it stands on the host cores.
Under torchrun (N > 1) each rank solves its own independent replica (the
solver runs on one GPU; no data-path collective) and rank 0 prints the max
over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "BDDC-GMRES time to rel.res 1e-8 (setup + solve)"
WORKLOAD = "4x4x4 subdomains, H/h=8 (32^3 Q1 hexes, 29791 dofs), nu=0.01, beta=(1,0.5,0.25), f=1, GMRES(50)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return P.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM traffic per launch of the engine task kernel: ncu's dram__bytes_read.sum +
# dram__bytes_write.sum, mean over the four launches of one step of this workload,
# and the hash of the sources it was measured on: reported only while they are
# unchanged.
ENGINE_TRAFFIC_BYTES = 133731584
ENGINE_TRAFFIC_SOURCES = ("engine.cu", "tc_common.cuh", "bddc_internal.h")
ENGINE_TRAFFIC_SHA256 = "9ea7868344f8a53fc27076ea43407fd7b70bea88b7dbf7ea8dcffbd201fe089f"


def engine_traffic():
    import hashlib
    h = hashlib.sha256()
    try:
        for f in ENGINE_TRAFFIC_SOURCES:
            with open(os.path.join(ROOT, "paper_2501_01676_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return ENGINE_TRAFFIC_BYTES if h.hexdigest() == ENGINE_TRAFFIC_SHA256 else None


def measured_bf16_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("bf16_tflops"))
    except Exception:
        return None


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, ws, dist


def barrier(dist):
    import torch
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(dist, v):
    import torch
    if dist is None:
        return v
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        try:
            self.proc.terminate()
            self.proc.wait(timeout=5)
        except Exception:
            pass
        try:
            dev = int(os.environ.get("LOCAL_RANK", "0"))
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
            rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(dev)]
            sm = [float(r[1]) for r in rows if r[1].replace('.', '', 1).isdigit()]
            mx = [float(r[2]) for r in rows if r[2].replace('.', '', 1).isdigit()]
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = set()
            for r in rows:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                   "reasons": sorted(reasons), "samples": len(rows)}
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        return out


def flush_l2(buf):
    buf.add_(1.0)


def run_ours(args):
    import torch

    from paper_2501_01676_gb300 import bddc as B
    from paper_2501_01676_gb300 import workloads as W

    rank, ws, dist = dist_init()
    torch.cuda.init()
    B.lib()
    p = W.config2()
    arrays = B.resident_arrays(p)
    pinned = B.resident_arrays(p, pinned_host=True)
    stream = torch.cuda.Stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    torch.cuda.synchronize()

    mlp = B.load_mlp_params()
    learned = {} if mlp is None else {"learned_skip_p": 0.9, "mlp_params": mlp}

    def step(precision, skip=True):
        kw = learned if (precision == B.PREC_MIXED and skip) else {}
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s = B.Solver(p, stream=stream, arrays=arrays, precision=precision, **kw)
            u, st = s.solve()
            e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        return ms, st, u

    if args.part == "fp64":
        for _ in range(args.warmup + args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            ms, st, _ = step(B.PREC_FP64)
        if rank == 0:
            print(json.dumps({"part": "fp64", "ms": ms, "iters": st["iters"]}), flush=True)
        return
    # warm-up
    for _ in range(args.warmup):
        flush_l2(flush)
        torch.cuda.synchronize()
        step(B.PREC_MIXED)
    times, stats = [], None
    clocks = Clocks()
    barrier(dist)
    clocks.start()
    B.kernel_timer(B.KT_ENGINE_TASKS)        # CUDA events around each launch of the engine's task kernel
    l0 = B.kernel_launches()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        ms, st, u = step(B.PREC_MIXED)
        times.append(ms)
        stats = st
    barrier(dist)
    t_wall = time.perf_counter() - t_wall0
    launches = B.kernel_launches() - l0
    kt = B.kernel_timer_read()
    B.kernel_timer(B.KT_NONE)
    ck = clocks.stop()
    ms_step = max_over_ranks(dist, sum(times) / len(times))
    if args.part == "mixed":
        if rank == 0:
            print(json.dumps({"part": "mixed", "ms": ms_step, "iters": stats["iters"],
                              "launches": int(launches)}), flush=True)
        return
    # the same mixed solver without the learned skip (every edge runs its GEP)
    noskip = []
    for _ in range(max(1, min(args.steps, 5))):
        flush_l2(flush)
        torch.cuda.synchronize()
        ms, st_ns, _ = step(B.PREC_MIXED, skip=False)
        noskip.append(ms)
    ms_noskip = max_over_ranks(dist, sum(noskip) / len(noskip))
    # plain FP64 GPU path on the same GPU
    fp64_times, st64 = [], None
    flush_l2(flush)
    torch.cuda.synchronize()
    step(B.PREC_FP64)
    for _ in range(max(1, min(args.steps, 3))):
        flush_l2(flush)
        torch.cuda.synchronize()
        ms, st64, _ = step(B.PREC_FP64)
        fp64_times.append(ms)
    ms64 = max_over_ranks(dist, sum(fp64_times) / len(fp64_times))
    # end to end through the C ABI with host (pinned) buffers
    e2e_times = []
    h2d = sum(v.numel() * 8 for v in pinned.values() if v is not None)
    d2h = 8 * stats["ndof"]
    for r in range(args.warmup + args.steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = B.Solver(p, host=True, stream=stream, arrays=pinned, precision=B.PREC_MIXED, **learned)
        u_host, _ = s.solve(host=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.close()
        if r >= args.warmup:
            e2e_times.append((t1 - t0) * 1e3)
    e2e_ms = max_over_ranks(dist, sum(e2e_times) / len(e2e_times))
    hbm, which = peaks()
    # The dominant kernel: the elimination engine's persistent task kernel (one
    # launch per elimination: subdomain Schur complements, face Schur complements,
    # constrained-solver / coarse-basis extended matrices).  Its algorithmic work
    # is the blocked LU's: per panel of width w over a trailing size m, 2 m^2 w
    # (update) + 2 w^2 m (substitutions) + (2/3) w^3, counted once.  With w = 128
    # the update does 32 flop per byte of the trailing matrix read and written,
    # above the FP32 ridge of ~11.8 flop/B: compute bound.  The update tiles run on
    # the tensor cores (split TF32: three MMAs per product), the diagonal blocks and
    # the triangular solves on the FP32 CUDA cores, which now hold most of the
    # kernel's CTA time: the roofline is the FP32 pipe ("alu": 152 SMs x 128 FP32
    # lanes x 2 flops x the sampled SM clock); the split-TF32 tensor peak (the
    # measured bf16 peak x the nominal TF32/bf16 ratio 1.1/2.25, / 3 MMAs) is
    # reported beside it.
    secs = kt["ms"] * 1e-3
    gbs = kt["bytes"] / secs / 1e9 if secs > 0 else 0.0
    tfl = kt["flops"] / secs / 1e12 if secs > 0 else 0.0
    sm_mhz = ck.get("sm_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    roofline = {"kernel": "k_engine_tasks<float,128,128> (blocked LU task kernel: 128-wide panels, 128x128 update tiles)",
                "bound": "alu", "achieved": round(tfl, 2), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                "frac": round(tfl / fp32_peak, 4), "traffic": engine_traffic(),
                "peak_source": "derived: 152 SMs x 128 FP32 FMA lanes x 2 x median sampled SM clock",
                "launches": kt["launches"], "avg_launch_us": round(1e3 * kt["ms"] / max(kt["launches"], 1), 2),
                "flops_per_launch": round(kt["flops"] / max(kt["launches"], 1)),
                "bytes_per_launch": round(kt["bytes"] / max(kt["launches"], 1)),
                "hbm_gbs_of_algorithmic_bytes": round(gbs, 1), "hbm_peak_gbs": hbm, "hbm_peak_source": which}
    bf16 = measured_bf16_tflops()
    if bf16:
        roofline["split_tf32_tensor_peak"] = round(bf16 * (1.1 / 2.25) / 3.0, 1)
        roofline["split_tf32_tensor_peak_source"] = "derived from measured bf16 dense (burst) x 1.1/2.25 / 3"
    apply = apply_bandwidth(B, W, hbm, which) if args.apply else None
    out = {
        "metric": METRIC, "value": round(ms_step, 4), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "subdomains": 64, "H_over_h": 8, "global_batch": 1,
                   "parallelism": "replicas" if ws > 1 else "single-gpu", "l2_flush": True,
                   "inputs": "device-resident FP64 coefficient arrays"},
        "iters": stats["iters"], "refine_steps": stats["refine_steps"], "relres": stats["relres"],
        "relres_global": stats["relres_global"], "pnumF": stats["pnumF"], "pnumE": stats["pnumE"],
        "n_pi": stats["n_pi"],
        "edges_skipped": stats["edges_skipped"], "learned_skip": bool(learned),
        "mixed_without_skip_ms": round(ms_noskip, 4), "mixed_without_skip_iters": st_ns["iters"],
        "plain_fp64_ms": round(ms64, 4), "plain_fp64_iters": st64["iters"],
        "speedup_vs_fp64": round(ms64 / ms_step, 3),
        "setup_breakdown_ms": {k: round(stats[k], 3) for k in ("setup_ms", "t_assemble_ms", "t_factor_ms",
                                                               "t_face_ms", "t_edge_ms", "t_coarse_ms")},
        "solve_ms": round(stats["solve_ms"], 3), "jacobi_sweeps_max": stats["jacobi_sweeps_max"],
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "apply": apply,
        "clocks": ck,
        "wall_s_timed": round(t_wall, 3),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def apply_bandwidth(B, W, hbm, which, reps=20):
    """HBM throughput of the apply kernels on the 8x8x8, H/h=8 workload, whose
    operators exceed the 129 MB L2: S x (the gather-GEMV-scatter over all 512
    subdomains) and M^-1 r (its three launches), FP32 and FP64 operators."""
    import torch
    p = W.config3()
    out = {"workload": "8x8x8 subdomains, H/h=8 (64^3 hexes, 250047 dofs)", "hbm_peak_gbs": hbm,
           "peak_source": which}
    for prec, name in ((B.PREC_MIXED, "fp32"), (B.PREC_FP64, "fp64")):
        s = B.Solver(p, precision=prec)
        x = torch.randn(s.n_gamma, dtype=torch.float64, device="cuda")
        res = {}
        for op, fn in (("S", s.schur_apply), ("M", s.apply)):
            for _ in range(3):
                fn(x)
            torch.cuda.synchronize()
            B.kernel_timer(B.KT_GEMV)
            for _ in range(reps):
                fn(x)
            kt = B.kernel_timer_read()
            B.kernel_timer(B.KT_NONE)
            gbs = kt["bytes"] / (kt["ms"] * 1e-3) / 1e9 if kt["ms"] > 0 else 0.0
            res[op] = {"GB/s": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 4),
                       "kernel_us_per_apply": round(1e3 * kt["ms"] / reps, 2),
                       "bytes_per_apply": round(kt["bytes"] / reps)}
        out[name] = res
        s.close()
        torch.cuda.synchronize()
    return out


def cpu_baseline(p):
    """The FP64 oracle as it stands (setup + BDDC-GMRES) on the host cores."""
    from oracle import bddc as ob
    t0 = time.perf_counter()
    o = ob.BDDC(p)
    _, info = o.solve()
    dt = time.perf_counter() - t0
    return {"value": round(dt * 1e3, 1), "unit": "ms", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": "the full workload once (oracle setup + GMRES, numpy/scipy FP64)",
            "iters": info["iters"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import bddc as ob
    from paper_2501_01676_gb300 import workloads as W
    p = W.config2()
    times, info = [], None
    for r in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o = ob.BDDC(p)
        _, info = o.solve()
        dt = (time.perf_counter() - t0) * 1e3
        if r >= args.warmup:
            times.append(dt)
    v = sum(times) / len(times)
    cores = len(os.sched_getaffinity(0))
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "subdomains": 64, "H_over_h": 8},
           "iters": info["iters"], "pnumF": info["pnumF"], "pnumE": info["pnumE"],
           "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                            "sample": "the full workload per step (oracle setup + GMRES)"},
           "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-apply", dest="apply", action="store_false",
                    help="skip the apply-bandwidth measurement on the 8x8x8 workload")
    ap.add_argument("--part", default="all", choices=["all", "mixed", "fp64"],
                    help="all: the full JSON line; mixed/fp64: time only that path (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: at least 3 warm-up steps are required for a valid number", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
