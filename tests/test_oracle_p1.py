"""The oracle's P1 discretisation on the six Kuhn tetrahedra of each brick
(Sect. 4) and the non-homogeneous Dirichlet lifting, pinned against facts that do
not come from the oracle itself:

* the six tetrahedra tile the brick (volumes sum to the brick's, barycentric
  gradients sum to zero, every tetrahedron contains the main diagonal);
* the P1 stiffness on the Kuhn split of a uniform grid equals h times the 7-point
  finite-difference Laplacian (the couplings along the face and main diagonals
  vanish);
* the consistent mass: the sum of all entries is the domain's volume;
* with beta = 0 the element matrices are symmetric, and their convective part is
  skew (Sect. 2: z(u, v) = -z(v, u));
* a patch test: for constant nu, beta, c and a linear exact solution u with
  f = beta.grad u + c u, Galerkin plus the residual-based stabilisation
  reproduce u at the nodes exactly, with u's values imposed on the boundary
  through the lifting (this fails for a wrong sign or index in the lifting, a
  dropped term of the stabilisation, or a transposed convection term);
* Example 4.1's data: the subdomain viscosities of Tests 1-3 and the boundary
  values;
* the unit-cube brick matrices (diffusion, reaction, convection with its
  stabilisation) against the exact rational integrals of
  tests/golden/p1_unit_brick.txt (written by make_p1_unit_brick.py from the
  tetrahedra's barycentric gradients alone);
* the advective stabilisation branch is homogeneous of degree one in beta, with
  ||beta||_{K,inf} taken over all four vertices of each tetrahedron.
"""
import numpy as np
import pytest

from oracle import fem
from oracle.mesh import Mesh
from paper_2501_01676_gb300 import workloads as W


def test_kuhn_tetrahedra_tile_the_brick():
    h = (0.3, 0.5, 0.7)
    vid, G, vol, lam = fem.p1_tables(h)
    assert np.isclose(6 * vol, h[0] * h[1] * h[2])
    assert np.abs(G.sum(axis=1)).max() < 1e-12
    assert all(v[0] == 0 and v[3] == 7 for v in vid)
    assert len({tuple(v) for v in vid}) == 6
    assert np.allclose(lam.sum(axis=1), 1.0)
    # gradient of lambda_a at vertex b is the Kronecker delta: grad lambda_a . (x_b - x_0) = delta_ab - delta_a0
    xyz = np.array([[(a & 1) * h[0], ((a >> 1) & 1) * h[1], ((a >> 2) & 1) * h[2]] for a in range(8)])
    for k in range(6):
        P = xyz[vid[k]]
        for a in range(4):
            for b in range(4):
                val = G[k, a] @ (P[b] - P[0]) + (1.0 if a == 0 else 0.0)
                assert abs(val - (1.0 if a == b else 0.0)) < 1e-12


def test_p1_stiffness_is_the_seven_point_laplacian():
    slabs = [[3], [3], [3]]
    mesh = Mesh(slabs)
    n = mesh.nnode[0] * mesh.nnode[1] * mesh.nnode[2]
    Ae, Fe, nodes = fem.element_matrices(mesh, np.ones(mesh.nelem), np.zeros((n, 3)), np.zeros(n), 0.0,
                                         element='p1')
    A, _ = fem.assemble_global(mesh, Ae, Fe, nodes)
    h = mesh.h[0]
    m = 2                                   # free nodes per direction
    I = np.eye(m)
    T = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    L = np.kron(np.kron(I, I), T) + np.kron(np.kron(I, T), I) + np.kron(np.kron(T, I), I)
    assert np.abs(A.toarray() - h * L).max() < 1e-12


def test_p1_mass_sums_to_the_volume_and_convection_is_skew():
    slabs = [[2, 1], [2], [1, 2]]
    mesh = Mesh(slabs)
    n = mesh.nnode[0] * mesh.nnode[1] * mesh.nnode[2]
    rng = np.random.default_rng(7)
    z = np.zeros(n)
    # mass: nu -> 0 leaves only c~ u v (beta = 0: no stabilisation term besides c^2 C)
    Ae, _, _ = fem.element_matrices(mesh, np.full(mesh.nelem, 1e-300), np.zeros((n, 3)), z, 1.0, tau=0.0,
                                    element='p1')
    assert np.isclose(Ae.sum(), 1.0)
    beta = rng.standard_normal((n, 3))
    A1, _, _ = fem.element_matrices(mesh, np.ones(mesh.nelem), beta, z, 0.0, tau=0.0, element='p1')
    A0, _, _ = fem.element_matrices(mesh, np.ones(mesh.nelem), np.zeros((n, 3)), z, 0.0, tau=0.0, element='p1')
    skew = A1 - A0
    assert np.abs(skew + skew.transpose(0, 2, 1)).max() < 1e-13
    assert np.abs(skew).max() > 1e-3
    assert np.abs(A0 - A0.transpose(0, 2, 1)).max() < 1e-13


def test_p1_patch_test_with_lifted_dirichlet_values():
    slabs = [[2, 3], [3, 2], [2, 2]]
    mesh = Mesh(slabs)
    ne, h, X, Y, Z = W._grid(slabs)
    n = X.size
    nu, beta, c = 0.05, np.array([0.7, -0.4, 1.1]), 0.8
    u = 1.0 + 0.5 * X - 2.0 * Y + 1.5 * Z
    f = beta @ np.array([0.5, -2.0, 1.5]) + c * u
    Ae, Fe, nodes = fem.element_matrices(mesh, np.full(mesh.nelem, nu), np.tile(beta, (n, 1)), f, c,
                                         element='p1')
    Fe = fem.lift_dirichlet(mesh, Ae, Fe, nodes, u)
    A, F = fem.assemble_global(mesh, Ae, Fe, nodes)
    uh = fem.direct_solve(A, F)
    free = mesh.free_node_ids()
    assert np.abs(uh - u[free]).max() < 1e-11
    # the homogeneous system (no lifting) does not reproduce u: the lifting carries the boundary
    Ae2, Fe2, _ = fem.element_matrices(mesh, np.full(mesh.nelem, nu), np.tile(beta, (n, 1)), f, c, element='p1')
    A2, F2 = fem.assemble_global(mesh, Ae2, Fe2, nodes)
    assert np.abs(fem.direct_solve(A2, F2) - u[free]).max() > 1e-2


def test_example41_data():
    p = W.example41(test=3, m=2, nu1=1.0, nu2=1e-7)
    sub = W._elem_subdomain(p.slabs)
    nu_sub = np.array([p.nu_elem[sub == s][0] for s in range(8)])
    # Test 3: Omega_1, _3, _6, _8 (a checkerboard of the 2 x 2 x 2 cubes) carry nu_1
    for s in range(8):
        sx, sy, sz = s & 1, (s >> 1) & 1, s >> 2
        assert nu_sub[s] == (1.0 if (sx + sy + sz) % 2 == 0 else 1e-7)
    p1 = W.example41(test=1, m=2)
    sub1 = np.array([p1.nu_elem[sub == s][0] for s in range(8)])
    assert all(sub1[s] == (1.0 if (s & 1) == 0 else 1e-7) for s in range(8))      # x < 0 half
    ne, h, X, Y, Z = W._grid(p.slabs)
    assert np.all(p.dirichlet_node[Z == 0.0] == 1.0) and np.all(p.dirichlet_node[Z > 0.0] == 0.0)
    assert np.allclose(p.beta_node[:, 0], -2 * np.pi * (Y - 0.5))
    assert p.element == 'p1' and p.c == 1.0


def test_example41_random_viscosity_data():
    p = W.example41_random(n=3, m=2)
    assert p.nu_elem.size == 6 ** 3 and p.element == 'p1'
    r = np.log10(p.nu_elem)
    assert r.min() > -3 and r.max() < 3 and r.std() > 1.0          # 10^U(-3,3), std 6/sqrt(12)
    assert np.array_equal(p.nu_elem, W.example41_random(n=3, m=2).nu_elem)
    ne, h, X, Y, Z = W._grid(p.slabs)
    assert np.all(p.dirichlet_node[Z == 0.0] == 1.0) and np.all(p.dirichlet_node[Z > 0.0] == 0.0)


def _golden_p1():
    """The exact P1 unit-cube integrals of tests/golden/p1_unit_brick.txt."""
    from fractions import Fraction
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "p1_unit_brick.txt")
    mats, cur = {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line[1:-1]
                mats[cur] = []
            else:
                mats[cur].append([float(Fraction(v)) for v in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


@pytest.mark.parametrize("case", ["diffusion", "reaction", "convection"])
def test_p1_unit_cube_against_golden_integrals(case):
    """Unit cube, one brick of six tetrahedra: the oracle's P1 brick matrix against
    the stored exact integrals combined by the bilinear form of Sect. 2 (tau = 0.7,
    h_K = sqrt 3, here P_K < 1 on every tetrahedron: C_K = tau h_K^2 / (4 nu))."""
    G = _golden_p1()
    mesh = Mesh([[1], [1], [1]])
    nu, c = 1.0, 0.0
    beta = np.zeros(3)
    if case == "reaction":
        c = 1.0
    if case == "convection":
        beta = np.array([1.0, 0.0, 0.0])
    A, _, _ = fem.element_matrices(mesh, np.full(1, nu), np.tile(beta, (8, 1)), np.zeros(8), c, element='p1')
    CK = 0.7 * 3.0 / (4.0 * nu)
    want = {"diffusion": G["K0"],
            "reaction": G["K0"] + (1.0 + CK) * G["M"],
            "convection": G["K0"] + CK * G["Kx"] + 0.5 * (G["Cx"] - G["Cx"].T)}[case]
    np.testing.assert_allclose(A[0], want, rtol=0, atol=1e-14)


def test_p1_advective_stabilisation_is_homogeneous_of_degree_one():
    """In the advective branch (P_K >= 1) C_K = tau h_K / (2 ||beta||_{K,inf}) and the
    GLS term is C_K int (beta.grad u)(beta.grad v), so with c = 0 the symmetric part of
    the element matrix minus diffusion grows linearly in the size of beta.  Here beta
    is non-zero only at the brick's node 7, a vertex of all six tetrahedra: the
    vertex maximum must see it (a maximum over three of the four vertices would take
    the diffusive branch and grow quadratically)."""
    mesh = Mesh([[1], [1], [1]])
    nu = 1e-8

    def sym_part(scale):
        beta = np.zeros((8, 3))
        beta[7] = scale * np.array([0.6, -0.3, 0.9])
        A, _, _ = fem.element_matrices(mesh, np.full(1, nu), beta, np.zeros(8), 0.0, element='p1')
        return 0.5 * (A[0] + A[0].T)

    S0, S1, S2 = sym_part(0.0), sym_part(1.0), sym_part(2.0)
    assert np.abs(S1 - S0).max() > 1e-3
    np.testing.assert_allclose(S2 - S0, 2.0 * (S1 - S0), rtol=1e-12, atol=1e-15)
