"""Train the edge-count network of the learned edge-GEP skip on the GPU.

Training rows come from the method itself: full setups (every edge runs its
GEP) of seeded problems from the workload generators -- the channel /
Fourier-velocity generator (seeds other than the benchmark's), the
per-subdomain jump generator, the rotating-velocity patterns and
constant-coefficient variants -- each at several thresholds Theta_E (the
GEP selects constraints only at the lower ones on these meshes), give each
edge's features (log10 Theta_E among them) and the number of constraints its
GEP selected.  The network is trained with the library's own forward,
backward and Adam kernels and saved next to this file (edge_mlp_params.npy).
The report gives the class histogram and, on the benchmark workloads' seeds
(never trained on), the false-skip and false-keep rates of the skip rule
P(no constraint) >= 0.9 beside the constant rule that skips every edge.

    python -m paper_2501_01676_gb300.train_edge_mlp [--epochs 600] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import bddc as B
from . import workloads as W

TEST_SEED_OFFSETS = {3, 5}          # the seeds of the benchmark workloads are never trained on


def training_problems():
    probs = []
    for k in range(20):                               # channel + Fourier-velocity generator
        probs.append(W.config5(seed_offset=101 + k))
    for k in range(8):                                # per-subdomain jump generator
        probs.append(W.config3(seed_offset=201 + k))
    for t in (1, 2, 3):                               # rotating velocity, c = 1, nu patterns
        for (nsub, m, lo) in ((2, 6, 1e-7), (3, 6, 1e-5), (4, 4, 1e-3)):
            probs.append(W.rotating_checker(t, nsub, m, 1.0, lo))
    rng = np.random.default_rng(301)
    for k in range(8):                                # constant coefficients, 4x4x4
        beta = tuple(rng.uniform(-1, 1, 3))
        probs.append(W.uniform(4, 8, nu=10.0 ** rng.uniform(-3, 0), beta=beta, f=1.0, name=f"const{k}"))
    return probs


THETAS = (1.25, 1.5, 2.0, 3.0, 5.0, 10.0)


def collect(probs, thetas=THETAS, precision=B.PREC_MIXED):
    X, y = [], []
    for p in probs:
        for th in thetas:
            s = B.Solver(p, precision=precision, theta_E=th)
            F, cnt = s.edge_features()
            s.close()
            X.append(F)
            y.append(np.minimum(cnt, B.MLP_CLASSES - 1))
    return np.concatenate(X), np.concatenate(y).astype(np.int32)


def held_out_report(params, skip_p=0.9):
    """Skip-rule errors on the benchmark workloads' seeds at several thresholds."""
    import torch
    out = []
    for cfg in (3, 5):
        p = W.CONFIGS[cfg]()
        for th in (1.5, 2.0, 3.0, 10.0):
            s = B.Solver(p, precision=B.PREC_MIXED, theta_E=th)
            F, cnt = s.edge_features()
            s.close()
            P = B.mlp_forward(params, torch.from_numpy(F).cuda()).cpu().numpy()
            skip = P[:, 0] >= skip_p
            pos = cnt > 0
            out.append({"workload": cfg, "theta_E": th, "edges": int(len(cnt)), "positives": int(pos.sum()),
                        "skipped": int(skip.sum()), "false_skips": int((skip & pos).sum()),
                        "false_keeps": int((~skip & ~pos).sum()),
                        "skip_all_false_skips": int(pos.sum())})
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=B.MLP_PARAMS_FILE)
    args = ap.parse_args()
    t0 = time.perf_counter()
    X, y = collect(training_problems())
    t1 = time.perf_counter()
    rng = np.random.default_rng(7)
    he = []
    for shape in [(B.MLP_FEATURES, 64), (64,), (64, 64), (64,), (64, 64), (64,), (64, 8), (8,)]:
        he.append(rng.standard_normal(shape) * np.sqrt(2.0 / shape[0]) if len(shape) == 2 else np.zeros(shape))
    th0 = np.concatenate([a.ravel() for a in he]).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    th, hist = B.mlp_train(th0, Xd, yd, args.epochs, lr=args.lr)
    t2 = time.perf_counter()
    P = B.mlp_forward(th, Xd).cpu().numpy()
    acc = float((P.argmax(1) == y).mean())
    np.save(args.out, th)
    rep = {"rows": int(len(y)), "thetas": list(THETAS), "class_counts": np.bincount(y, minlength=8).tolist(),
           "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "train_accuracy": acc,
           "data_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2), "epochs": args.epochs, "out": args.out,
           "held_out": held_out_report(th)}
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
