"""The learned edge-GEP skip on the GPU against the FP64 reference MLP.

Tolerances: features are computed in FP64 and stored in FP32 (relative 1e-6);
the network runs in FP32: probabilities within 1e-5, the gradient within
1e-4 of its largest entry (FP32 sums over a few hundred rows).
"""
import numpy as np
import pytest

from oracle import fem
from oracle import mlp as omlp
from oracle.mesh import Mesh
from paper_2501_01676_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_2501_01676_gb300 import bddc
    return bddc


@pytest.mark.parametrize("prob,theta_E", [
    (lambda: W.random_small(4, (3, 3, 3), 3, (-3, 3)), 10.0),
    (lambda: W.config5(seed_offset=77, nsub=3, m=4), 2.0),
    (lambda: W.uniform(2, 2, nu=0.3, beta=(0.2, -1.0, 0.5)), 10.0),      # one-dof edges
])
def test_edge_features_match_oracle(prob, theta_E):
    p = prob()
    s = B().Solver(p, theta_E=theta_E)
    F, cnt = s.edge_features()
    Fo = omlp.edge_features(Mesh(p.slabs), p.nu_elem, p.beta_node, theta_E=theta_E)
    assert F.shape == Fo.shape
    np.testing.assert_allclose(F, Fo, rtol=1e-6, atol=1e-6)
    k = [g['k'] for g in s.entities(1)]
    assert list(cnt) == k


def test_forward_and_gradient_match_reference():
    import torch
    rng = np.random.default_rng(3)
    th = (omlp.init_params(2) + 0.05 * rng.standard_normal(omlp.NPARAM)).astype(np.float32)
    X = rng.standard_normal((300, omlp.NF)).astype(np.float32)
    y = rng.integers(0, omlp.NC, 300).astype(np.int32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    P = B().mlp_forward(th, Xd).cpu().numpy()
    L, _ = omlp.forward(th.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(P, omlp.softmax(L), atol=1e-5)
    loss, g = B().mlp_loss_grad(th, Xd, yd)
    lo, go = omlp.loss_grad(th.astype(np.float64), X.astype(np.float64), y)
    assert abs(loss - lo) < 1e-5 * max(1.0, lo)
    assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()


def test_training_reduces_loss():
    import torch
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2000, omlp.NF)).astype(np.float32)
    y = (np.clip(np.floor(2 * X[:, 0] + X[:, 1] + 3), 0, 7)).astype(np.int32)   # learnable labels
    th0 = omlp.init_params(9).astype(np.float32)
    th, hist = B().mlp_train(th0, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 200, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    P = B().mlp_forward(th, torch.from_numpy(X).cuda()).cpu().numpy()
    assert (P.argmax(1) == y).mean() > 0.8


def test_learned_skip_gain_on_channel_workload():
    """On the 8x8x8 channel / Fourier-velocity workload (a seed never trained on):
    with the shipped network the edge GEPs predicted to select nothing are
    skipped; the solve still reaches 1e-8 with at most two more GMRES
    iterations, and the edge phase of the setup gets cheaper."""
    params = B().load_mlp_params()
    if params is None:
        pytest.skip("no trained parameters shipped")
    p = W.config5()
    full = B().Solver(p, precision=1)
    u0, st0 = full.solve()
    F, cnt_full = full.edge_features()
    skip = B().Solver(p, precision=1, learned_skip_p=0.9, mlp_params=params)
    u1, st1 = skip.solve()
    _, cnt_skip = skip.edge_features()
    assert st1["edges_skipped"] > 0
    skipped = cnt_skip < 0
    false_skips = int((cnt_full[skipped] > 0).sum())
    print(f"edges {len(cnt_full)} skipped {skipped.sum()} false skips {false_skips} "
          f"pnumE {st0['pnumE']}->{st1['pnumE']} iters {st0['iters']}->{st1['iters']} "
          f"edge phase {st0['t_edge_ms']:.2f}->{st1['t_edge_ms']:.2f} ms "
          f"setup {st0['setup_ms']:.2f}->{st1['setup_ms']:.2f} ms")
    assert st0["converged"] and st1["converged"]
    assert st1["relres"] <= 1e-8
    assert st1["iters"] <= st0["iters"] + 2
    assert st1["t_edge_ms"] < st0["t_edge_ms"]
    d = (u1 - u0).abs().max().item() / u0.abs().max().item()
    assert d < 1e-6


@pytest.mark.parametrize("cfg,theta_E", [(5, 3.0), (3, 2.0)])
def test_learned_skip_keeps_edges_that_select(cfg, theta_E):
    """At a threshold where the full edge GEP selects constraints on part of
    the edges (8x8x8 workloads, seeds never trained on), the shipped network
    runs the GEP on almost every edge that selects: its false skips (skipped
    edges whose full GEP selects) stay below 5 % of those edges -- the constant
    rule that skips every edge misses all of them -- while it still skips
    edges, and the false skips cost at most two GMRES iterations."""
    params = B().load_mlp_params()
    if params is None:
        pytest.skip("no trained parameters shipped")
    p = W.CONFIGS[cfg]()
    full = B().Solver(p, precision=1, theta_E=theta_E)
    u0, st0 = full.solve()
    _, cnt_full = full.edge_features()
    skip = B().Solver(p, precision=1, theta_E=theta_E, learned_skip_p=0.9, mlp_params=params)
    u1, st1 = skip.solve()
    _, cnt_skip = skip.edge_features()
    pos = cnt_full > 0
    skipped = cnt_skip < 0
    false_skips = int((skipped & pos).sum())
    print(f"theta_E {theta_E}: edges {len(cnt_full)} selecting {pos.sum()} skipped {skipped.sum()} "
          f"false skips {false_skips} pnumE {st0['pnumE']}->{st1['pnumE']} iters {st0['iters']}->{st1['iters']}")
    assert pos.sum() > 0 and skipped.sum() > 0
    assert false_skips <= 0.05 * pos.sum()
    assert st0["converged"] and st1["converged"]
    assert st1["iters"] <= st0["iters"] + 2
