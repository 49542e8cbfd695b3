"""Benchmark: time to solve the advection-diffusion Schur system with adaptive
BDDC-GMRES to relative residual 1e-8 on one GB300.

Workload (the headline): 8x8x8 subdomains, H/h = 8 (64^3 hexahedra, 250 047
dofs), nu per subdomain 10^U(-4,0), rotating beta = (-(y-1/2), x-1/2, 0.1),
f = 1, Theta_E = 10, Theta_F = 1 + ln 8.  A step is the whole hot path for one
synthetic input: assembly, batched subdomain factorisation and Schur
complements, face GEPs, edge GEPs on prior-selected primal constraints (with
the learned skip), constrained local solvers, the coarse problem (sparse LU by
nested dissection), then condensation, preconditioned GMRES and interior
recovery, in the mixed-precision solver (FP32 factors and operators, FP64
refinement).  Beside it, on the same GPU: the same solver without the learned
skip, with the conventional edge GEP, the plain FP64 path, the end-to-end call
with host buffers, the channel workload (8x8x8, nu = 1e-4 with 12 channels of
nu = 1, Fourier velocity) and the 4x4x4 workload (with its error against the
oracle's direct solve), and the apply kernels' bandwidth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle as it stands on the host cores, on
a bounded sample (the first 2 of the 8 subdomain layers of the workload, 128 of
the 512 subdomains, scaled by 4).  Under torchrun (N > 1) each rank solves its own independent replica (the
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
WORKLOAD = ("8x8x8 subdomains, H/h=8 (64^3 Q1 hexes, 250047 dofs), nu per subdomain 10^U(-4,0), "
            "beta=(-(y-1/2),x-1/2,0.1), f=1, GMRES to 1e-8")
WORKLOAD_C5 = ("8x8x8 subdomains, H/h=8, nu=1e-4 with 12 one-element channels of nu=1, "
               "4-mode Fourier beta (|beta|<=1), f=1")
WORKLOAD_C2 = "4x4x4 subdomains, H/h=8 (32^3 Q1 hexes, 29791 dofs), nu=0.01, beta=(1,0.5,0.25), f=1, GMRES(50)"
SAMPLE = ("the oracle's setup + BDDC-GMRES on the first 2 of the 8 subdomain layers of the workload "
          "(128 of the 512 subdomains, the same per-subdomain nu and H/h = 8, as a problem of its own), "
          "timed once per step and scaled by 4")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return P.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM traffic per launch of the engine task kernel on the 8x8x8 workload: ncu's
# dram__bytes_read.sum + dram__bytes_write.sum, mean over the launches of one
# step, and the hash of the sources it was measured on: reported only while
# they are unchanged (None: not measured on the current sources).
ENGINE_TRAFFIC_BYTES = 3617968064
ENGINE_TRAFFIC_SOURCES = ("engine.cu", "tc_common.cuh")
ENGINE_TRAFFIC_SHA256 = "73a3984b49f82cbbee830ed3130993d23bb0a486ad4355d0b87e8fdb9c8c0951"


def engine_traffic(kt=None):
    import hashlib
    if ENGINE_TRAFFIC_BYTES is None:
        return None
    h = hashlib.sha256()
    try:
        for f in ENGINE_TRAFFIC_SOURCES:
            with open(os.path.join(ROOT, "paper_2501_01676_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return ENGINE_TRAFFIC_BYTES if h.hexdigest() == ENGINE_TRAFFIC_SHA256 else None


def measured_bf16_tflops(sustained=False):
    """(dense bf16 TFLOP/s, source): MEASURED_PEAKS.json's burst or sustained
    figure, else the fallback of the profiling recipe."""
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured " + ("sustained" if sustained else "burst")
    except Exception:
        return (1700.0 if sustained else 1900.0), "fallback " + ("sustained" if sustained else "burst")


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


def solve_step(B, p, stream, arrays, precision, flush, **kw):
    """One timed step (setup + solve through the C ABI, inputs resident in HBM);
    returns (ms, stats, u)."""
    import torch
    flush_l2(flush)
    torch.cuda.synchronize()
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


def timed(B, p, stream, arrays, precision, flush, steps, warmup=1, **kw):
    for _ in range(warmup):
        solve_step(B, p, stream, arrays, precision, flush, **kw)
    times, st, u = [], None, None
    for _ in range(steps):
        ms, st, u = solve_step(B, p, stream, arrays, precision, flush, **kw)
        times.append(ms)
    return statistics.median(times), st, u


STAT_KEYS = ("iters", "refine_steps", "relres_global", "kappa_est", "pnumF", "pnumE", "n_pi", "edges_skipped",
             "coarse_path", "coarse_fronts", "coarse_levels")


def summary(ms, st):
    out = {"ms": round(ms, 3)}
    out.update({k: (round(st[k], 12) if isinstance(st[k], float) else st[k]) for k in STAT_KEYS})
    out["setup_ms"] = round(st["setup_ms"], 3)
    out["solve_ms"] = round(st["solve_ms"], 3)
    out["setup_breakdown_ms"] = {k: round(st[k], 3) for k in ("t_mesh_ms", "t_assemble_ms", "t_factor_ms",
                                                             "t_face_ms", "t_edge_ms", "t_basis_ms",
                                                             "t_coarse_ms")}
    return out


# The paper's Tables 4 (m = 6, row nu_1 = 1, nu_2 = 1e-7) and 5 (m = 4, 8, 16):
# iterations (pnumF, pnumE) of ABDDC-OLD and ABDDC-NEW for Tests 1-3 (P1
# tetrahedra, MATLAB) - context only.
EX41_PAPER = {4: {"old": ((8, 4, 12), (9, 3, 10), (7, 0, 18)), "new": ((9, 4, 3), (10, 3, 3), (9, 0, 6))},
              6: {"old": ((9, 4, 20), (9, 3, 17), (7, 0, 30)), "new": ((10, 4, 9), (11, 3, 6), (10, 0, 6))},
              8: {"old": ((10, 4, 28), (10, 3, 24), (7, 0, 42)), "new": ((11, 4, 10), (12, 3, 7), (15, 0, 6))},
              16: {"old": ((12, 6, 61), (11, 5, 55), (8, 4, 90)), "new": ((14, 6, 24), (16, 5, 12), (16, 4, 9))}}


def example41_part(B, W, stream, flush):
    """Example 4.1 (Sect. 4) at m = 4, 6, 8, 16, nu_1 = 1, nu_2 = 1e-7: the P1
    Kuhn-tetrahedron discretisation with u = 1 on z = 0, Tests 1-3, the new and the
    conventional edge GEP, FP64 solver: iterations, (pnumF, pnumE), time to solve
    (one setup + solve; m = 16 has faces of 225 and interiors of 3375 dofs)."""
    try:
        out = {"workload": "Example 4.1: 2x2x2 cubic subdomains of m^3 cubes split into six P1 tetrahedra, "
                           "c = 1, a = (-2 pi y, 2 pi x, sin 2 pi x), u = 1 on z = 0, nu_1 = 1, nu_2 = 1e-7",
               "paper_tables_4_5": {str(m): v for m, v in EX41_PAPER.items()}}
        for m in (4, 6, 8, 16):
            for test in (1, 2, 3):
                p = W.example41(test=test, m=m, nu1=1.0, nu2=1e-7)
                arrays = B.resident_arrays(p)
                for name, mode in (("new", B.EDGE_NEW), ("old", B.EDGE_OLD)):
                    ms, st, _ = timed(B, p, stream, arrays, B.PREC_FP64, flush, 1, warmup=1 if m < 16 else 0,
                                      edge_gep=mode)
                    out[f"m{m}_test{test}_{name}"] = {"ms": round(ms, 3), "iters": st["iters"],
                                                      "pnumF": st["pnumF"], "pnumE": st["pnumE"],
                                                      "relres_global": st["relres_global"]}
        p = W.example41(test=1, m=16, nu1=1.0, nu2=1e-7)
        arrays = B.resident_arrays(p)
        # m = 16 with the dense interior elimination and with one level of local
        # nested dissection (2 x 2 x 2 child boxes per subdomain), FP64 and mixed
        for key, prec, nd in (("m16_test1_new_mixed", B.PREC_MIXED, 0), ("m16_test1_new_fp64_local_nd", B.PREC_FP64, 1),
                              ("m16_test1_new_mixed_local_nd", B.PREC_MIXED, 1)):
            ms, st, _ = timed(B, p, stream, arrays, prec, flush, 1, local_nd=nd)
            out[key] = {"ms": round(ms, 3), "iters": st["iters"], "pnumF": st["pnumF"], "pnumE": st["pnumE"],
                        "relres_global": st["relres_global"], "setup_ms": round(st["setup_ms"], 3),
                        "solve_ms": round(st["solve_ms"], 3), "factor_gflop": round(st["factor_gflop"], 3),
                        "setup_breakdown_ms": {k: round(st[k], 3) for k in ("t_assemble_ms", "t_factor_ms",
                                                                             "t_face_ms", "t_edge_ms",
                                                                             "t_coarse_ms")}}
        return out
    except Exception as e:        # reported in the line, never fatal to the benchmark
        return {"error": repr(e)[:300]}


# The paper's random-viscosity table: n(m) -> OLD and NEW iterations (pnumF, pnumE).
EX41_PAPER_RANDOM = {"2(4)": ((10, 4, 8), (11, 4, 0)), "2(8)": ((12, 14, 33), (15, 14, 0)),
                     "2(12)": ((13, 15, 51), (16, 15, 9)), "3(4)": ((13, 18, 60), (17, 18, 0)),
                     "3(8)": ((17, 64, 201), (25, 64, 18)), "3(12)": ((18, 72, 301), (24, 72, 54)),
                     "4(4)": ((15, 52, 187), (24, 52, 18)), "4(8)": ((19, 181, 593), (36, 181, 112)),
                     "4(12)": ((19, 181, 909), (30, 181, 309))}


def example41_random_part(B, W, stream, flush):
    """Example 4.1's data on n^3 cubic subdomains of m^3 cubes (P1) with a random
    viscosity 10^U(-3,3) per cube, n(m) as in the paper's random-viscosity table, the
    new and the conventional edge GEP, FP64 solver."""
    try:
        out = {"workload": "Example 4.1 data on n^3 subdomains of m^3 cubes (six P1 tetrahedra each), "
                           "nu = 10^U(-3,3) per cube (seeded)", "paper_old_new": EX41_PAPER_RANDOM}
        for n in (2, 3, 4):
            for m in (4, 8, 12):
                p = W.example41_random(n, m)
                arrays = B.resident_arrays(p)
                row = {}
                for name, mode in (("new", B.EDGE_NEW), ("old", B.EDGE_OLD)):
                    ms, st, _ = timed(B, p, stream, arrays, B.PREC_FP64, flush, 1, edge_gep=mode)
                    row[name] = {"ms": round(ms, 3), "iters": st["iters"], "pnumF": st["pnumF"],
                                 "pnumE": st["pnumE"]}
                out[f"{n}({m})"] = row
        return out
    except Exception as e:        # reported in the line, never fatal to the benchmark
        return {"error": repr(e)[:300]}


def run_ours(args):
    import torch

    from paper_2501_01676_gb300 import bddc as B
    from paper_2501_01676_gb300 import workloads as W

    rank, ws, dist = dist_init()
    torch.cuda.init()
    B.lib()
    if args.part == "apply":
        hbm, which = peaks()
        if rank == 0:
            print(json.dumps({"part": "apply", "apply": apply_bandwidth(B, W, hbm, which)}), flush=True)
        return
    p = W.config3()
    arrays = B.resident_arrays(p)
    pinned = B.resident_arrays(p, pinned_host=True)
    stream = torch.cuda.Stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    torch.cuda.synchronize()

    mlp = B.load_mlp_params()
    learned = {} if mlp is None else {"learned_skip_p": 0.9, "mlp_params": mlp}

    for _ in range(args.warmup):
        solve_step(B, p, stream, arrays, B.PREC_MIXED, flush, **learned)
    times, stats = [], None
    clocks = Clocks()
    barrier(dist)
    clocks.start()
    B.kernel_timer(B.KT_ENGINE_TASKS)        # CUDA events around each launch of the engine's task kernel
    l0 = B.kernel_launches()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        ms, stats, u = solve_step(B, p, stream, arrays, B.PREC_MIXED, flush, **learned)
        times.append(ms)
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
    few = max(1, min(args.steps, 3))
    # the same workload: without the learned skip, conventional edge GEP, plain FP64
    ms_ns, st_ns, _ = timed(B, p, stream, arrays, B.PREC_MIXED, flush, few)
    ms_old, st_old, _ = timed(B, p, stream, arrays, B.PREC_MIXED, flush, few, edge_gep=B.EDGE_OLD)
    ms64, st64, _ = timed(B, p, stream, arrays, B.PREC_FP64, flush, max(1, min(args.steps, 2)))
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
    # (update) + 2 w^2 m (substitutions) + (2/3) w^3, counted once.  The dense
    # contraction (the trailing updates, most of the flops) runs on the tensor
    # cores with split-TF32 operands (three MMAs per product), so the roofline is
    # the tensor pipe: the measured dense bf16 peak (sustained: the kernel runs
    # inside a long step) x the nominal TF32/bf16 ratio 1.1/2.25, / 3.  The FP32
    # CUDA-core fraction (diagonal blocks and triangular solves run there) is
    # reported beside it: 152 SMs x 128 FP32 lanes x 2 flops x the sampled clock.
    secs = kt["ms"] * 1e-3
    gbs = kt["bytes"] / secs / 1e9 if secs > 0 else 0.0
    tfl = kt["flops"] / secs / 1e12 if secs > 0 else 0.0
    sm_mhz = ck.get("sm_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    bf16, bf16_src = measured_bf16_tflops(sustained=True)
    tc_peak = bf16 * (1.1 / 2.25) / 3.0
    roofline = {"kernel": "k_engine_tasks<float,128,128> (blocked LU task kernel: 128-wide panels, "
                          "128x128 split-TF32 tensor-core update tiles)",
                "bound": "tensor", "achieved": round(tfl, 2), "peak": round(tc_peak, 1), "unit": "TFLOP/s",
                "frac": round(tfl / tc_peak, 4), "traffic": engine_traffic(kt),
                "peak_source": f"derived: {bf16_src} bf16 dense {bf16:.1f} TFLOP/s x 1.1/2.25 (TF32/bf16) / 3 "
                               f"(split-TF32 products)",
                "fp32_cuda_core_peak": round(fp32_peak, 1), "frac_of_fp32_cuda_core_peak": round(tfl / fp32_peak, 4),
                "launches": kt["launches"], "avg_launch_us": round(1e3 * kt["ms"] / max(kt["launches"], 1), 2),
                "flops_per_launch": round(kt["flops"] / max(kt["launches"], 1)),
                "bytes_per_launch": round(kt["bytes"] / max(kt["launches"], 1)),
                "hbm_gbs_of_algorithmic_bytes": round(gbs, 1), "hbm_peak_gbs": hbm, "hbm_peak_source": which}
    # the channel workload (learned-skip workload) and the 4x4x4 workload
    p5 = W.config5()
    a5 = B.resident_arrays(p5)
    ms5, st5, _ = timed(B, p5, stream, a5, B.PREC_MIXED, flush, max(1, min(args.steps, 5)), **learned)
    ms5_ns, st5_ns, _ = timed(B, p5, stream, a5, B.PREC_MIXED, flush, few)
    ms5_old, st5_old, _ = timed(B, p5, stream, a5, B.PREC_MIXED, flush, few, edge_gep=B.EDGE_OLD)
    p2 = W.config2()
    a2 = B.resident_arrays(p2)
    ms2, st2, u2 = timed(B, p2, stream, a2, B.PREC_MIXED, flush, max(1, min(args.steps, 10)), **learned)
    ms2_64, st2_64, u2_64 = timed(B, p2, stream, a2, B.PREC_FP64, flush, few)
    apply = apply_bandwidth(B, W, hbm, which) if args.apply else None
    ex41 = example41_part(B, W, stream, flush)
    ex41r = example41_random_part(B, W, stream, flush)
    out = {
        "metric": METRIC, "value": round(ms_step, 4), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "subdomains": 512, "H_over_h": 8, "global_batch": 1,
                   "parallelism": "replicas" if ws > 1 else "single-gpu", "l2_flush": True,
                   "inputs": "device-resident FP64 coefficient arrays", "solver": "mixed + learned edge-GEP skip"},
        "iters": stats["iters"], "refine_steps": stats["refine_steps"], "relres": stats["relres"],
        "relres_global": stats["relres_global"], "kappa_est": stats["kappa_est"], "pnumF": stats["pnumF"],
        "pnumE": stats["pnumE"], "n_pi": stats["n_pi"], "edges_skipped": stats["edges_skipped"],
        "learned_skip": bool(learned),
        "setup_ms": round(stats["setup_ms"], 3), "solve_ms": round(stats["solve_ms"], 3),
        "setup_breakdown_ms": summary(ms_step, stats)["setup_breakdown_ms"],
        "coarse": {k: stats[k] for k in ("coarse_path", "coarse_fronts", "coarse_levels", "coarse_factor_gflop")},
        "mixed_without_skip": summary(ms_ns, st_ns),
        "conventional_edge_gep": summary(ms_old, st_old),
        "plain_fp64": summary(ms64, st64),
        "speedup_vs_fp64": round(ms64 / ms_step, 3),
        "channel_workload": {"workload": WORKLOAD_C5, "learned_skip": summary(ms5, st5),
                             "without_skip": summary(ms5_ns, st5_ns), "conventional_edge_gep": summary(ms5_old, st5_old)},
        "workload_4x4x4": {"workload": WORKLOAD_C2, "mixed": summary(ms2, st2), "plain_fp64": summary(ms2_64, st2_64)},
        "example_4_1": ex41,
        "example_4_1_random_nu": ex41r,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "apply": apply,
        "clocks": ck,
        "wall_s_timed": round(t_wall, 3),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["workload_4x4x4"]["err_vs_oracle"] = oracle_error(p2, u2, u2_64)
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def apply_bandwidth(B, W, hbm, which, reps=20):
    """HBM throughput of the per-iteration operators on the 8x8x8 workload,
    whose operators exceed the 129 MB L2: S x (one gather-GEMV-scatter launch
    over all 512 subdomains) and M^-1 r (one persistent launch: local part,
    coarse restriction, nested-dissection coarse sweeps, prolongation), FP32
    and FP64 operators."""
    import torch
    p = W.config3()
    out = {"workload": "8x8x8 subdomains, H/h=8 (64^3 hexes, 250047 dofs)", "hbm_peak_gbs": hbm,
           "peak_source": which}
    for prec, name in ((B.PREC_MIXED, "fp32"), (B.PREC_FP64, "fp64")):
        s = B.Solver(p, precision=prec)
        x = torch.randn(s.n_gamma, dtype=torch.float64, device="cuda")
        res = {}
        for op, fn, kind in (("S", s.schur_apply, B.KT_GEMV), ("M", s.apply, B.KT_APPLY_TASKS)):
            for _ in range(3):
                fn(x)
            torch.cuda.synchronize()
            B.kernel_timer(kind)
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


def oracle_error(p, u_mixed, u_fp64):
    """Relative solution error of the 4x4x4 solves (default stopping rule) against
    the oracle's direct solve of the assembled FP64 system."""
    from oracle import bddc as ob
    from oracle import fem
    o = ob.BDDC(p, edge_gep='none', face_gep=False)
    ustar = fem.direct_solve(o.A, o.F)
    nrm = float(np.linalg.norm(ustar))
    return {"mixed": float(np.linalg.norm(u_mixed.cpu().numpy() - ustar) / nrm),
            "plain_fp64": float(np.linalg.norm(u_fp64.cpu().numpy() - ustar) / nrm),
            "reference": "oracle global assembly + sparse direct solve (FP64)"}


def oracle_sample_ms():
    """The oracle as it stands on the bounded sample; returns (ms scaled to the
    8x8x8 workload, iterations)."""
    from oracle import bddc as ob
    from paper_2501_01676_gb300 import workloads as W
    ps = W.config3_layers(2)
    t0 = time.perf_counter()
    o = ob.BDDC(ps)
    _, info = o.solve()
    dt = (time.perf_counter() - t0) * 1e3
    return 4.0 * dt, info["iters"], dt


def cpu_baseline():
    v, iters, raw = oracle_sample_ms()
    return {"value": round(v, 1), "unit": "ms", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": SAMPLE, "sample_ms": round(raw, 1), "sample_iters": iters}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times, iters, raws = [], None, []
    for r in range(args.warmup + args.steps):
        v, iters, raw = oracle_sample_ms()
        if r >= args.warmup:
            times.append(v)
            raws.append(raw)
    v = sum(times) / len(times)
    cores = len(os.sched_getaffinity(0))
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "subdomains": 512, "H_over_h": 8, "global_batch": 1,
                      "parallelism": "single-gpu", "l2_flush": True,
                      "inputs": "host numpy arrays", "solver": "FP64 CPU oracle"},
           "sample_iters": iters,
           "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                            "sample": SAMPLE, "sample_ms": round(sum(raws) / len(raws), 1)},
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
    ap.add_argument("--part", default="all", choices=["all", "mixed", "apply"],
                    help="all: the full JSON line; mixed: time only the headline solver; apply: only the "
                         "apply-bandwidth measurement (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: at least 3 warm-up steps are required for a valid number", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
