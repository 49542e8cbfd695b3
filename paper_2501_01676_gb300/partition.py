"""Partition of the subdomains over ranks (one GPU each) for the multi-GPU path.

The BDDC hot path shards by subdomains: every local solve, every Schur
complement and every constraint of a subdomain involves that subdomain's data
only, and the operators of Sect. 3 are sums over subdomains,

    S x    = sum_i R_i^T S^(i) R_i x                              (eq. Schur-complex-sys)
    M^-1 r = sum_i R_i^T D_i (G_i rho_i + Phi_i u_Pi),  rho_i = D_i^T R_i r,
             S_Pi u_Pi = sum_i R_Pi_i^T Psi_i^T rho_i             (M_BDDC^-1, coarse problem)

so one iteration of right-preconditioned GMRES needs exactly three kinds of
exchange:

1. neighbour sums of interface values: each rank sums its subdomains'
   contributions into the interface dofs they touch; a dof shared with
   subdomains of other ranks receives their partial sums (point to point,
   neighbours only);
2. one allreduce of the n_Pi-vector of coarse right-hand-side contributions,
   after which every rank solves the (small, replicated) coarse problem;
3. one allreduce of the j + 1 Arnoldi dot products per Gram-Schmidt pass, each
   rank summing over the interface dofs it owns.

This module holds the host logic: rank blocks (contiguous boxes of the
subdomain grid, so that the interface between ranks is a few planes), dof
ownership, the neighbour lists, and the three exchanges written against a
`torch.distributed`-like object.  The per-rank arithmetic is the library's
kernels on the rank's own subdomains; the tests exercise the partition and
the exchanges with CPU ranks (gloo).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def rank_boxes(nsub: Sequence[int], world: int) -> List[Tuple[Tuple[int, int, int], Tuple[int, int, int]]]:
    """Contiguous boxes [lo, hi) of the subdomain grid, one per rank: recursive
    bisection across the longest direction, sizes proportional to the ranks on
    each side.  Every rank gets at least one subdomain (world <= prod(nsub))."""
    n = [int(v) for v in nsub]
    if world < 1 or world > n[0] * n[1] * n[2]:
        raise ValueError("need 1 <= world <= number of subdomains")

    def split(lo, hi, ranks):
        if ranks == 1:
            return [(tuple(lo), tuple(hi))]
        ext = [hi[d] - lo[d] for d in range(3)]
        d = int(np.argmax(ext))
        left = ranks // 2
        cut = lo[d] + max(1, min(ext[d] - 1, round(ext[d] * left / ranks)))
        if ext[d] < 2:
            raise ValueError("cannot split a single subdomain")
        hl, lr = list(hi), list(lo)
        hl[d] = cut
        lr[d] = cut
        return split(list(lo), hl, left) + split(lr, list(hi), ranks - left)

    return split([0, 0, 0], n, world)


def subdomains_in(box, nsub: Sequence[int]) -> List[int]:
    """Subdomain ids s = sx + nx (sy + ny sz) inside a box, ascending."""
    (x0, y0, z0), (x1, y1, z1) = box
    nx, ny = int(nsub[0]), int(nsub[1])
    return sorted(sx + nx * (sy + ny * sz) for sz in range(z0, z1) for sy in range(y0, y1) for sx in range(x0, x1))


class RankPlan:
    """What one rank holds: its subdomains, the interface dofs they touch (the
    rank's ghosted interface layout, ascending global interface index), which of
    those it owns, and per neighbour rank the local positions they share."""

    def __init__(self, rank: int, subs: List[int], gamma_local: np.ndarray, owned: np.ndarray,
                 neighbours: Dict[int, np.ndarray], sub_pos: Dict[int, np.ndarray]):
        self.rank = rank
        self.subs = subs
        self.gamma_local = gamma_local
        self.owned = owned
        self.neighbours = neighbours
        self.sub_pos = sub_pos

    @property
    def n_local(self) -> int:
        return int(self.gamma_local.size)


def build_plans(sub_gidx: Sequence[np.ndarray], nsub: Sequence[int], world: int) -> List[RankPlan]:
    """Plans of all ranks from each subdomain's interface map R_i (global
    interface indices of its local interface dofs).  A dof is owned by the
    lowest rank whose subdomains touch it."""
    boxes = rank_boxes(nsub, world)
    owner_sub = {}
    rank_subs = []
    for r, b in enumerate(boxes):
        ss = subdomains_in(b, nsub)
        rank_subs.append(ss)
        for s in ss:
            owner_sub[s] = r
    touching: Dict[int, set] = {}
    for s, g in enumerate(sub_gidx):
        r = owner_sub[s]
        for d in np.asarray(g).tolist():
            touching.setdefault(d, set()).add(r)
    plans = []
    for r in range(world):
        gl = np.array(sorted({int(d) for s in rank_subs[r] for d in np.asarray(sub_gidx[s]).tolist()}),
                      dtype=np.int64)
        pos = {int(d): q for q, d in enumerate(gl.tolist())}
        owned = np.array([min(touching[int(d)]) == r for d in gl.tolist()], dtype=bool)
        nb: Dict[int, List[int]] = {}
        for q, d in enumerate(gl.tolist()):
            for o in touching[int(d)]:
                if o != r:
                    nb.setdefault(o, []).append(q)
        neighbours = {o: np.array(v, dtype=np.int64) for o, v in sorted(nb.items())}
        sub_pos = {s: np.array([pos[int(d)] for d in np.asarray(sub_gidx[s]).tolist()], dtype=np.int64)
                   for s in rank_subs[r]}
        plans.append(RankPlan(r, rank_subs[r], gl, owned, neighbours, sub_pos))
    return plans


# ---------------------------------------------------------------------------
# the three exchanges (dist: torch.distributed; vectors: torch CPU or CUDA tensors)
# ---------------------------------------------------------------------------
def neighbour_sum(plan: RankPlan, partial, dist):
    """Interface values from partial sums: every shared dof adds the partial
    sums of the neighbour ranks touching it (one send and one receive per
    neighbour, all posted before any wait).  Returns the summed vector."""
    out = partial.clone()
    reqs, bufs = [], []
    for o, q in plan.neighbours.items():
        idx = _index(q, partial)
        send = partial.index_select(0, idx).contiguous()
        recv = send.new_empty(send.shape)
        reqs.append(dist.isend(send, o))
        reqs.append(dist.irecv(recv, o))
        bufs.append((idx, recv, send))
    for rq in reqs:
        rq.wait()
    for idx, recv, _ in bufs:
        out.index_add_(0, idx, recv)
    return out


def dots(plan: RankPlan, V, w, dist):
    """V^T w over the owned interface dofs of all ranks: one allreduce of the
    rows of V (the Arnoldi basis, k x n_local) against w."""
    import torch
    own = _mask(plan, w)
    h = (V[:, own] @ w[own]).contiguous()
    dist.all_reduce(h, op=dist.ReduceOp.SUM)
    return h


def norm(plan: RankPlan, w, dist) -> float:
    own = _mask(plan, w)
    t = (w[own] @ w[own]).reshape(1).contiguous()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.sqrt().item())


def coarse_sum(v, dist):
    """The coarse right-hand side: the ranks' contributions summed (allreduce)."""
    v = v.contiguous()
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return v


def _index(q, like):
    import torch
    return torch.as_tensor(q, dtype=torch.long, device=like.device)


def _mask(plan: RankPlan, like):
    import torch
    return torch.as_tensor(plan.owned, dtype=torch.bool, device=like.device)
