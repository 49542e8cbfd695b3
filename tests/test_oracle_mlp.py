"""Pins of the reference MLP and the edge features (learned edge-GEP skip)."""
import math

import numpy as np

from oracle import mlp
from oracle.mesh import Mesh
from paper_2501_01676_gb300 import workloads as W


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + 0.05 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((40, mlp.NF))
    y = rng.integers(0, mlp.NC, 40)
    loss, g = mlp.loss_grad(theta, X, y)
    for k in rng.choice(mlp.NPARAM, 80, replace=False):
        e = np.zeros(mlp.NPARAM)
        e[k] = 1e-6
        fd = (mlp.loss_grad(theta + e, X, y)[0] - mlp.loss_grad(theta - e, X, y)[0]) / 2e-6
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-8, (k, fd, g[k])


def test_uniform_logits_give_log_classes():
    theta = np.zeros(mlp.NPARAM)
    X = np.random.default_rng(1).standard_normal((7, mlp.NF))
    loss, g = mlp.loss_grad(theta, X, np.arange(7) % mlp.NC)
    assert abs(loss - math.log(mlp.NC)) < 1e-14


def test_features_constant_coefficients():
    p = W.uniform(3, 4, nu=0.01, beta=(1.0, 0.5, 0.25))
    mesh = Mesh(p.slabs)
    F = mlp.edge_features(mesh, p.nu_elem, p.beta_node)
    assert F.shape == (len(mesh.edges), mlp.NF)
    np.testing.assert_allclose(F[:, 0:3], -2.0, atol=1e-12)
    np.testing.assert_allclose(F[:, 3], 0.0, atol=1e-12)
    bn = math.sqrt(1 + 0.25 + 0.0625)
    for e, f in zip(mesh.edges, F):
        c = np.array([mesh.dof_coords(int(d)) for d in e['dofs']])
        a = int(np.nonzero(c.max(0) != c.min(0))[0][0])
        assert abs(f[4] - (1.0, 0.5, 0.25)[a]) < 1e-12 and abs(f[5] - f[4]) < 1e-12
        assert abs(f[6] - bn) < 1e-12
        assert abs(f[7] - 1.0 / 3.0) < 1e-12          # an edge spans one subdomain: H = 1/3
        assert abs(f[8] - 0.4) < 1e-12
        assert abs(f[9] - math.log10((1.0 / 12.0) * bn / 0.02)) < 1e-12
        assert abs(f[10] - 1.0) < 1e-12                # log10 of the default Theta_E = 10
    F2 = mlp.edge_features(mesh, p.nu_elem, p.beta_node, theta_E=2.0)
    np.testing.assert_allclose(F2[:, 10], math.log10(2.0), atol=1e-15)
    np.testing.assert_array_equal(F2[:, :10], F[:, :10])


def test_features_jump_ratio():
    p = W.uniform(2, 3, nu=1e-4)
    mesh = Mesh(p.slabs)
    sub = W._elem_subdomain(p.slabs)
    p.nu_elem = np.where(sub == 0, 1.0, 1e-4)
    F = mlp.edge_features(mesh, p.nu_elem, p.beta_node)
    for e, f in zip(mesh.edges, F):
        want = 4.0 if 0 in e['subs'] else 0.0
        assert abs(f[3] - want) < 1e-12
        assert abs(f[1] - (0.0 if 0 in e['subs'] else -4.0)) < 1e-12
