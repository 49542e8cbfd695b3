"""Edge features and the reference MLP of the learned edge-GEP skip.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not in the paper: the benchmark pattern trains a small network on the edge
GEP's own outputs (the number of constraints k_E an edge selects, eq. equ-5-21
and the selection below it) to predict k_E from local coefficient features.

Features of an edge E (a line of n_E interior dofs along axis a, shared by
the subdomains n(E)); "touching elements" are the 4 (n_E + 1) elements that
contain the closed edge segment:
  0 min log10 nu, 1 max log10 nu, 2 mean log10 nu   over touching elements
  3 max - min over n(E) of the per-subdomain mean log10 nu (touching elements)
  4 mean |beta . t|, 5 max |beta . t|, 6 mean |beta|  over the n_E edge nodes
  7 edge length (n_E + 1) h_a
  8 H/h / 10 (largest slab element count over n(E), scaled)
  9 log10 of the Peclet number h_a * feature6 / (2 * 10^feature2)
  10 log10 Theta_E (the threshold the edge GEP selects with)
Network: x (11) -> relu(W1 x + b1) (64) -> relu (64) -> relu (64) -> W4 h + b4
(8 logits, class c = min(k_E, 7)); loss = mean softmax cross-entropy.
Flat parameter layout: W1 [11][64], b1, W2 [64][64], b2, W3 [64][64], b3,
W4 [64][8], b4 (row-major, input index first).
"""
from __future__ import annotations

import math

import numpy as np

NF, NH, NC = 11, 64, 8
SHAPES = [(NF, NH), (NH,), (NH, NH), (NH,), (NH, NH), (NH,), (NH, NC), (NC,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n]).reshape(s))
        o += n
    return out


def init_params(seed=0):
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * math.sqrt(2.0 / s[0]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([p.ravel() for p in parts])


def forward(theta, X):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0)
    z3 = h2 @ W3 + b3
    h3 = np.maximum(z3, 0)
    logits = h3 @ W4 + b4
    return logits, (X, z1, h1, z2, h2, z3, h3)


def softmax(L):
    L = L - L.max(axis=1, keepdims=True)
    e = np.exp(L)
    return e / e.sum(axis=1, keepdims=True)


def loss_grad(theta, X, y):
    """Mean cross-entropy and its gradient (manual backpropagation)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    logits, (X, z1, h1, z2, h2, z3, h3) = forward(theta, X)
    B = X.shape[0]
    P = softmax(logits)
    loss = -np.mean(np.log(P[np.arange(B), y]))
    dL = P.copy()
    dL[np.arange(B), y] -= 1.0
    dL /= B
    gW4 = h3.T @ dL
    gb4 = dL.sum(0)
    dh3 = dL @ W4.T
    dz3 = dh3 * (z3 > 0)
    gW3 = h2.T @ dz3
    gb3 = dz3.sum(0)
    dh2 = dz3 @ W3.T
    dz2 = dh2 * (z2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])
    return loss, g


def edge_features(mesh, nu_elem, beta_node, theta_E=10.0):
    """Feature rows for the mesh's edges in the mesh's edge order."""
    logn = np.log10(np.asarray(nu_elem, dtype=float))
    beta = np.asarray(beta_node, dtype=float)
    rows = []
    for e in mesh.edges:
        coords = np.array([mesh.dof_coords(int(d)) for d in e['dofs']])
        a = int(np.nonzero(coords.max(0) != coords.min(0))[0][0]) if len(coords) > 1 else None
        if a is None:
            # a one-dof edge: its axis is the direction in which the owners' slabs agree
            sc = [mesh.sub_coords(s) for s in e['subs']]
            a = [d for d in range(3) if len({c[d] for c in sc}) == 1][0]
        fixed = [d for d in range(3) if d != a]
        lo, hi = int(coords[:, a].min()), int(coords[:, a].max())
        els, owner = [], []
        for ea in range(lo - 1, hi + 1):
            for d1 in (-1, 0):
                for d2 in (-1, 0):
                    idx = [0, 0, 0]
                    idx[a] = ea
                    idx[fixed[0]] = int(coords[0, fixed[0]]) + d1
                    idx[fixed[1]] = int(coords[0, fixed[1]]) + d2
                    els.append(mesh.elem_id(*idx))
                    sxyz = [int(np.searchsorted(mesh.off[d], idx[d], side='right') - 1) for d in range(3)]
                    owner.append(mesh.sub_id(*sxyz))
        ln = logn[np.array(els)]
        owner = np.array(owner)
        means = [ln[owner == s].mean() for s in e['subs']]
        nodes = [mesh.node_id(*c) for c in coords]
        bt = np.abs(beta[nodes, a])
        bn = np.linalg.norm(beta[nodes], axis=1)
        m = max(max(mesh.slabs[d][mesh.sub_coords(s)[d]] for d in range(3)) for s in e['subs'])
        h = mesh.h[a]
        f = [ln.min(), ln.max(), ln.mean(), max(means) - min(means), bt.mean(), bt.max(), bn.mean(),
             (len(e['dofs']) + 1) * h, m / 10.0,
             math.log10(max(h * bn.mean() / (2.0 * 10.0 ** ln.mean()), 1e-30)), math.log10(theta_E)]
        rows.append(f)
    return np.array(rows)
