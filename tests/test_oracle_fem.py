"""Pins of the oracle's discretisation (Sect. 2) against closed forms.

* element matrices against exact tensor-product integrals of Q1 functions;
* b symmetric positive definite, z skew (end of Sect. 2);
* constant reproduction of the full row sums when c = 0 and div(beta) = 0;
* convergence on a manufactured solution: L2 rate 2, H1 rate 1.
"""
import math

import numpy as np
import pytest

from oracle import fem
from oracle.mesh import Mesh
from paper_2501_01676_gb300 import workloads as W


def one_d(h):
    m = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])          # int phi_j phi_i
    k = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])        # int phi_j' phi_i'
    c = np.array([[-0.5, 0.5], [-0.5, 0.5]])                  # [i][j] = int phi_j' phi_i
    one = np.array([h / 2.0, h / 2.0])                        # int phi_i
    return m, k, c, one


def t3(X, Y, Z):
    """3D matrix [a][b] with a = ax + 2 ay + 4 az from per-direction factors."""
    return np.kron(Z, np.kron(Y, X))


def exact_element(h, nu, beta, c, f, tau=fem.TAU):
    """Closed-form element matrix/load for constant beta, nu, c, f on an h-box."""
    mx, kx, cx, ox = one_d(h[0])
    my, ky, cy, oy = one_d(h[1])
    mz, kz, cz, oz = one_d(h[2])
    M = t3(mx, my, mz)
    Kd = [t3(kx, my, mz), t3(mx, ky, mz), t3(mx, my, kz)]
    # Cv[d][i][j] = int d_d phi_j phi_i
    Cv = [t3(cx, my, mz), t3(mx, cy, mz), t3(mx, my, cz)]
    ms, ks, cs = [mx, my, mz], [kx, ky, kz], [cx, cy, cz]

    def mixed(d, e):
        # [i][j] = int d_d phi_j * d_e phi_i
        if d == e:
            return Kd[d]
        f3 = []
        for t in range(3):
            if t == d:
                f3.append(cs[t])          # int phi_j' phi_i  in direction d
            elif t == e:
                f3.append(cs[t].T)        # int phi_j phi_i'  in direction e
            else:
                f3.append(ms[t])
        return t3(*f3)

    hK = math.sqrt(sum(x * x for x in h))
    bn = float(np.linalg.norm(beta))
    PK = hK * bn / (2 * nu)
    CK = tau * hK / (2 * bn) if PK >= 1 else tau * hK * hK / (4 * nu)
    BG = sum(beta[d] * Cv[d] for d in range(3))                # int beta.grad phi_j phi_i
    diff = nu * sum(Kd)
    LL = sum(beta[d] * beta[e] * mixed(d, e) for d in range(3) for e in range(3))
    LL = LL + c * BG + c * BG.T + c * c * M                    # int L phi_j L phi_i
    A = diff + CK * LL + c * M + 0.5 * (BG - BG.T)
    one = t3(ox[:, None], oy[:, None], oz[:, None])[:, 0]      # int phi_i
    # int beta.grad phi_i = sum_j int beta.grad phi_i phi_j = column sums of BG
    gi = BG.sum(axis=0)
    F = f * one + CK * f * (gi + c * one)
    return A, F


@pytest.mark.parametrize("nu,beta,c", [
    (1.0, (0.0, 0.0, 0.0), 0.0),
    (0.3, (0.0, 0.0, 0.0), 2.0),
    (1.0, (1.0, 0.5, 0.25), 0.0),         # P_K < 1 branch
    (0.001, (1.0, -0.5, 0.25), 0.7),      # P_K >= 1 branch
])
def test_element_matrix_closed_form(nu, beta, c):
    mesh = Mesh([[2], [3], [4]])             # unequal spacings hx != hy != hz
    nn = np.prod(mesh.nnode)
    beta_node = np.tile(beta, (nn, 1))
    f_node = np.full(nn, 1.7)
    A, F, _ = fem.element_matrices(mesh, np.full(mesh.nelem, nu), beta_node, f_node, c)
    Ax, Fx = exact_element(mesh.h, nu, np.array(beta), c, 1.7)
    for e in range(mesh.nelem):
        np.testing.assert_allclose(A[e], Ax, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(F[e], Fx, rtol=1e-12, atol=1e-14)


def test_laplacian_known_values():
    """Unit-cube Q1 Laplacian: diagonal 1/3, edge neighbours 0, others -1/12."""
    mesh = Mesh([[1], [1], [1]])
    A, _, _ = fem.element_matrices(mesh, np.ones(1), np.zeros((8, 3)), np.zeros(8), 0.0)
    K = A[0]
    for a in range(8):
        for b in range(8):
            dist = bin(a ^ b).count('1')
            want = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[dist]
            assert abs(K[a, b] - want) < 1e-14


def rotating_problem(nsub=2, m=3):
    p = W.uniform(nsub, m, nu=0.05)
    ne, h, X, Y, Z = W._grid(p.slabs)
    p.beta_node = np.stack([-(Y - 0.5), X - 0.5, np.full_like(X, 0.1)], axis=1)
    return p


def test_symmetric_part_spd_and_skew_part():
    p = rotating_problem()
    mesh = Mesh(p.slabs)
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, p.f_node, 0.0)
    A, _ = fem.assemble_global(mesh, Ae, Fe, nodes)
    A = A.toarray()
    Bsym = 0.5 * (A + A.T)
    assert np.linalg.eigvalsh(Bsym).min() > 0
    # the z part alone is skew: element matrices minus their symmetric part
    for e in range(0, mesh.nelem, 7):
        Z = 0.5 * (Ae[e] - Ae[e].T)
        np.testing.assert_allclose(Z, -Z.T, atol=1e-15)


def test_row_sums_vanish_for_interior_supports():
    """a(1, phi_i) = -1/2 int beta.grad phi_i = 0 for interior nodes when c = 0, div beta = 0."""
    p = rotating_problem(2, 3)
    mesh = Mesh(p.slabs)
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, p.f_node, 0.0)
    nn = int(np.prod(mesh.nnode))
    rs = np.zeros(nn)
    cs = np.zeros(nn)
    for e in range(mesh.nelem):
        np.add.at(rs, nodes[e], Ae[e].sum(axis=1))
        np.add.at(cs, nodes[e], Ae[e].sum(axis=0))
    n2d = fem.node_to_dof(mesh)
    interior = n2d >= 0
    scale = np.abs(Ae).max()
    assert np.abs(rs[interior]).max() < 1e-13 * scale
    assert np.abs(cs[interior]).max() < 1e-13 * scale


def mms_errors(m):
    p = W.mms(2, m, nu=1.0, beta=(1.0, 1.0, 1.0))
    mesh = Mesh(p.slabs)
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, p.f_node, 0.0)
    A, F = fem.assemble_global(mesh, Ae, Fe, nodes)
    u = fem.direct_solve(A, F)
    nn = int(np.prod(mesh.nnode))
    un = np.zeros(nn)
    un[mesh.free_node_ids()] = u
    N, G, wq = fem.q1_tables(mesh.h)
    xg, _ = fem.gauss3()
    pts = np.array([(xg[i], xg[j], xg[k]) for k in range(3) for j in range(3) for i in range(3)])
    E = np.arange(mesh.nelem)
    ex, ey, ez = E % mesh.ne[0], (E // mesh.ne[0]) % mesh.ne[1], E // (mesh.ne[0] * mesh.ne[1])
    X = (ex[:, None] + pts[None, :, 0]) * mesh.h[0]
    Y = (ey[:, None] + pts[None, :, 1]) * mesh.h[1]
    Z = (ez[:, None] + pts[None, :, 2]) * mesh.h[2]
    pi = math.pi
    ue = np.sin(pi * X) * np.sin(pi * Y) * np.sin(pi * Z)
    gx = pi * np.cos(pi * X) * np.sin(pi * Y) * np.sin(pi * Z)
    gy = pi * np.sin(pi * X) * np.cos(pi * Y) * np.sin(pi * Z)
    gz = pi * np.sin(pi * X) * np.sin(pi * Y) * np.cos(pi * Z)
    ua = un[nodes]                                            # (E,8)
    uh = ua @ N.T
    gh = np.einsum('ea,qad->eqd', ua, G)
    w = wq * np.prod(mesh.h)
    l2 = math.sqrt(np.sum(w * (uh - ue) ** 2))
    h1 = math.sqrt(np.sum(w * ((gh[..., 0] - gx) ** 2 + (gh[..., 1] - gy) ** 2 + (gh[..., 2] - gz) ** 2)))
    return l2, h1


def test_manufactured_solution_rates():
    e = [mms_errors(m) for m in (4, 8, 16)]
    l2_rates = [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
    h1_rates = [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
    assert 1.8 < l2_rates[-1] < 2.3, l2_rates
    assert 0.9 < h1_rates[-1] < 1.2, h1_rates


def _golden_q1():
    """The exact Q1 unit-cube integrals of tests/golden/q1_unit_cube.txt."""
    from fractions import Fraction
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "q1_unit_cube.txt")
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
def test_unit_cube_against_golden_integrals(case):
    """Unit cube, one element: the oracle's element matrix against the stored exact
    integrals combined by the bilinear form of Sect. 2 (tau = 0.7, h_K = sqrt 3;
    here P_K < 1, so C_K = tau h_K^2 / (4 nu))."""
    G = _golden_q1()
    mesh = Mesh([[1], [1], [1]])
    nu, c = 1.0, 0.0
    beta = np.zeros(3)
    if case == "reaction":
        c = 1.0
    if case == "convection":
        beta = np.array([1.0, 0.0, 0.0])
    A, _, _ = fem.element_matrices(mesh, np.full(1, nu), np.tile(beta, (8, 1)), np.zeros(8), c)
    CK = 0.7 * 3.0 / (4.0 * nu)
    want = {"diffusion": G["K0"],
            "reaction": G["K0"] + (1.0 + CK) * G["M"],
            "convection": G["K0"] + CK * G["Kx"] + 0.5 * (G["Cx"] - G["Cx"].T)}[case]
    np.testing.assert_allclose(A[0], want, rtol=0, atol=1e-14)
