"""The multi-GPU partition by subdomains on CPU ranks (gloo).

Host logic: rank boxes cover the subdomain grid without overlap; every
interface dof has exactly one owner; neighbour lists are symmetric.  Then
world-size 2 and 3 process groups run one BDDC-GMRES solve through the
partition's three exchanges (neighbour sums, the coarse allreduce, the Arnoldi
allreduces), each rank applying the oracle's operators of its own subdomains
(stand-ins for the rank's kernels), and the results equal the single-process
oracle: S x and M^-1 r to 1e-12 relative, the GMRES solution at rel. residual
1e-12 to 1e-9 of the oracle's, the iteration count at the paper's 1e-8 rule
within one of the oracle's.
"""
import multiprocessing as mp
import socket

import numpy as np
import pytest

from paper_2501_01676_gb300 import partition as P
from paper_2501_01676_gb300 import workloads as W


def problem():
    return W.random_small(1, (4, 2, 2), 3, (-2, 1))


@pytest.mark.parametrize("nsub,world", [((4, 4, 4), 2), ((4, 4, 4), 8), ((3, 2, 2), 3), ((8, 8, 8), 7),
                                        ((4, 2, 2), 16)])
def test_rank_boxes_cover_the_grid(nsub, world):
    boxes = P.rank_boxes(nsub, world)
    assert len(boxes) == world
    seen = np.zeros(nsub[0] * nsub[1] * nsub[2], dtype=int)
    for b in boxes:
        ss = P.subdomains_in(b, nsub)
        assert ss
        seen[ss] += 1
    assert (seen == 1).all()


def test_plans_own_every_interface_dof_once():
    from oracle import bddc as obddc
    o = obddc.BDDC(problem())
    gidx = [o.gidx[s] for s in range(o.mesh.nsd)]
    for world in (2, 3, 4):
        plans = P.build_plans(gidx, (4, 2, 2), world)
        owned = np.zeros(o.nG, dtype=int)
        for pl in plans:
            owned[pl.gamma_local[pl.owned]] += 1
            for nb, q in pl.neighbours.items():
                back = plans[nb].neighbours[pl.rank]
                assert np.array_equal(pl.gamma_local[q], plans[nb].gamma_local[back])
            for s in pl.subs:
                assert np.array_equal(pl.gamma_local[pl.sub_pos[s]], gidx[s])
        assert (owned == 1).all()


# ---------------------------------------------------------------------------
# per-rank operators (oracle stand-ins for the rank's kernels)
# ---------------------------------------------------------------------------
def _apply_S(o, pl, x, dist):
    import torch
    y = np.zeros(pl.n_local)
    xl = x.numpy()
    for s in pl.subs:
        np.add.at(y, pl.sub_pos[s], o.S[s] @ xl[pl.sub_pos[s]])
    return P.neighbour_sum(pl, torch.from_numpy(y), dist)


def _apply_M(o, pl, r, dist):
    import torch
    rl = r.numpy()
    rPi = np.zeros(o.nPi)
    rhos = {}
    for s in pl.subs:
        rhos[s] = o.Dmat[s].T @ rl[pl.sub_pos[s]]
        np.add.at(rPi, o.RPi[s], o.Psi[s].T @ rhos[s])
    rPi = P.coarse_sum(torch.from_numpy(rPi), dist).numpy()
    uPi = np.linalg.solve(o.SPi, rPi)
    z = np.zeros(pl.n_local)
    for s in pl.subs:
        w = o.G_apply(s, rhos[s]) + o.Phi[s] @ uPi[o.RPi[s]]
        np.add.at(z, pl.sub_pos[s], o.Dmat[s] @ w)
    return P.neighbour_sum(pl, torch.from_numpy(z), dist)


def _gmres(o, pl, b, dist, rtol, max_iter=300):
    """Right-preconditioned GMRES on the ranks' interface layouts: CGS2 with one
    allreduce per pass, Givens rotations on every rank (replicated scalars)."""
    import torch
    bn = P.norm(pl, b, dist)
    x = torch.zeros_like(b)
    m = max_iter
    V = torch.zeros((m + 1, b.numel()), dtype=b.dtype)
    H = np.zeros((m + 1, m))
    cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
    beta = bn
    V[0] = b / beta
    g[0] = beta
    k = 0
    for j in range(m):
        w = _apply_S(o, pl, _apply_M(o, pl, V[j], dist), dist)
        h1 = P.dots(pl, V[:j + 1], w, dist)
        w = w - V[:j + 1].T @ h1
        h2 = P.dots(pl, V[:j + 1], w, dist)
        w = w - V[:j + 1].T @ h2
        H[:j + 1, j] = (h1 + h2).numpy()
        H[j + 1, j] = P.norm(pl, w, dist)
        if H[j + 1, j] > 0:
            V[j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if abs(g[j + 1]) <= rtol * bn:
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = _apply_M(o, pl, V[:k].T @ torch.from_numpy(y), dist)
    return x, k


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from oracle import bddc as obddc
    from oracle.krylov import gmres
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        torch.set_default_dtype(torch.float64)
        o = obddc.BDDC(problem())
        plans = P.build_plans([o.gidx[s] for s in range(o.mesh.nsd)], (4, 2, 2), world)
        pl = plans[rank]
        res = {}
        rng = np.random.default_rng(12)
        v = rng.standard_normal(o.nG)
        loc = torch.from_numpy(v[pl.gamma_local])
        y = _apply_S(o, pl, loc, dist).numpy()
        ref = o.apply_S(v)[pl.gamma_local]
        res["S"] = float(np.abs(y - ref).max() / np.abs(ref).max())
        z = _apply_M(o, pl, loc, dist).numpy()
        ref = o.apply_M(v)[pl.gamma_local]
        res["M"] = float(np.abs(z - ref).max() / np.abs(ref).max())
        gfull = o.condense()
        b = torch.from_numpy(gfull[pl.gamma_local])
        x, k = _gmres(o, pl, b, dist, 1e-12)
        uG, _ = gmres(o.apply_S, gfull, o.apply_M, rtol=1e-12)
        ref = uG[pl.gamma_local]
        res["x"] = float(np.linalg.norm(x.numpy() - ref) / np.linalg.norm(ref))
        _, k8 = _gmres(o, pl, b, dist, 1e-8)
        _, info8 = gmres(o.apply_S, gfull, o.apply_M, rtol=1e-8)
        res["iters"] = (k8, info8["iters"])
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, res, None))
    except Exception as e:          # reported to the parent, which fails the test
        q.put((rank, None, repr(e)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_solve_equals_single_process(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, res, err = q.get(timeout=600)
        assert err is None, err
        out[rank] = res
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, res in out.items():
        assert res["S"] < 1e-12 and res["M"] < 1e-12, res
        assert res["x"] < 1e-9, res
        k8, ko = res["iters"]
        assert abs(k8 - ko) <= 1, res
