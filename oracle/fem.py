"""Stabilised Q1 (and P1 Kuhn-tetrahedron) finite elements for
-div(nu grad u) + beta.grad u + c u = f.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Sect. 2 of the paper (model problem, Peclet number, stabilisation
weight C(x), effective reaction c~ = c - div(beta)/2, and the stabilised
variational problem a = b + z = g), with these readings:

* Trilinear (Q1) hexahedra instead of the paper's P1 tetrahedra.  The forms are
  element-agnostic; L phi = beta.grad(phi) + c phi elementwise, because the
  second-order term of a Q1 function with elementwise-constant nu vanishes.
* nu is constant per element; beta, f and div(beta) are given at the nodes
  and interpolated trilinearly at the quadrature points.
* h_K = sqrt(hx^2+hy^2+hz^2) (the element diameter); ||beta||_{K,inf} is the
  largest |beta| over the 8 vertices and the 27 quadrature points; when it is
  zero the P_K < 1 branch of C(x) is taken.
* 3x3x3 Gauss-Legendre quadrature on every element.
* Entry (i,j) of an element matrix is a(phi_j, phi_i): trial j, test i.
* P1 (the paper's element, Sect. 4): each brick split into the six Kuhn
  tetrahedra around its main diagonal; per tetrahedron beta, f, div(beta) are
  interpolated linearly from its vertices, ||beta||_{K,inf} is the largest
  vertex |beta|, h_K its diameter (the brick's diagonal), and a 4-point degree-2
  rule integrates every term exactly; the brick's 8 x 8 matrix is the sum.
* Non-homogeneous Dirichlet values g enter through the element loads
  (lift_dirichlet).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

TAU = 0.7


def gauss3():
    """3-point Gauss-Legendre rule on [0,1]."""
    r = np.sqrt(3.0 / 5.0)
    x = 0.5 + 0.5 * np.array([-r, 0.0, r])
    w = np.array([5.0, 8.0, 5.0]) / 18.0
    return x, w


def q1_tables(h):
    """Shape values N[q,a] and physical gradients G[q,a,d] at the 27 points."""
    x, w = gauss3()
    pts, wts = [], []
    for k in range(3):
        for j in range(3):
            for i in range(3):
                pts.append((x[i], x[j], x[k]))
                wts.append(w[i] * w[j] * w[k])
    pts = np.array(pts)
    wts = np.array(wts)
    N = np.zeros((27, 8))
    G = np.zeros((27, 8, 3))
    for q, p in enumerate(pts):
        for a in range(8):
            bits = (a & 1, (a >> 1) & 1, (a >> 2) & 1)
            f1 = [p[d] if bits[d] else 1.0 - p[d] for d in range(3)]
            df = [1.0 if bits[d] else -1.0 for d in range(3)]
            N[q, a] = f1[0] * f1[1] * f1[2]
            G[q, a, 0] = df[0] * f1[1] * f1[2] / h[0]
            G[q, a, 1] = f1[0] * df[1] * f1[2] / h[1]
            G[q, a, 2] = f1[0] * f1[1] * df[2] / h[2]
    return N, G, wts


def element_nodes(mesh):
    """Node ids of all elements, shape (nelem, 8), element-id order."""
    ex, ey, ez = mesh.ne
    E = np.arange(mesh.nelem)
    ix, iy, iz = E % ex, (E // ex) % ey, E // (ex * ey)
    out = np.zeros((mesh.nelem, 8), dtype=int)
    for a in range(8):
        out[:, a] = mesh.node_id(ix + (a & 1), iy + ((a >> 1) & 1), iz + ((a >> 2) & 1))
    return out


def p1_tables(h):
    """The six Kuhn tetrahedra of a brick h[0] x h[1] x h[2] (Sect. 4: each cube
    divided into six tetrahedra): tetrahedron k for the k-th permutation p of the
    axes has the vertices 0, e_p0, e_p0 + e_p1, (1,1,1) (local node a has the
    coordinate bits a & 1, a >> 1 & 1, a >> 2 & 1, so the vertices are the local
    nodes 0, 1 << p0, 1 << p0 | 1 << p1, 7); all six share the main diagonal, and
    the same split in every brick is conforming.  Returns vid (6,4) local node ids,
    G (6,4,3) gradients of the barycentric coordinates, the volume of one
    tetrahedron, and the 4-point degree-2 rule: lam (4 points, 4 barycentric
    coordinates) with equal weights volume / 4."""
    import itertools
    vid = np.zeros((6, 4), dtype=int)
    G = np.zeros((6, 4, 3))
    xyz = np.array([[(a & 1) * h[0], ((a >> 1) & 1) * h[1], ((a >> 2) & 1) * h[2]] for a in range(8)])
    vol = 0.0
    for k, p in enumerate(itertools.permutations(range(3))):
        v1 = 1 << p[0]
        v2 = v1 | (1 << p[1])
        vid[k] = [0, v1, v2, 7]
        P = xyz[vid[k]]
        D = P[1:] - P[0]                                      # rows P_k - P_0
        Dit = np.linalg.inv(D).T                               # row k-1: grad lambda_k
        G[k, 1:] = Dit
        G[k, 0] = -Dit.sum(axis=0)
        vol = abs(np.linalg.det(D)) / 6.0
    a = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
    b = (5.0 - np.sqrt(5.0)) / 20.0
    lam = np.full((4, 4), b)
    np.fill_diagonal(lam, a)
    return vid, G, vol, lam


def _p1_element_matrices(mesh, nu, beta, fa, dva, c, tau):
    """Brick matrices of the P1 discretisation on the six Kuhn tetrahedra of each
    brick: the tetrahedra's 4 x 4 matrices and loads summed into the brick's 8
    nodes.  Per tetrahedron, as for Q1 (Sect. 2 forms): nu from the brick, beta, f
    and div(beta) interpolated linearly from its 4 vertices, ||beta||_{K,inf} the
    largest |beta| over its vertices, h_K its diameter (the brick's diagonal),
    the 4-point degree-2 rule (exact: every integrand is at most quadratic)."""
    hx, hy, hz = mesh.h
    vid, G, vol, lam = p1_tables(mesh.h)
    E = beta.shape[0]
    hK = np.sqrt(hx * hx + hy * hy + hz * hz)
    A = np.zeros((E, 8, 8))
    F = np.zeros((E, 8))
    w = np.full(4, vol / 4.0)
    for k in range(6):
        v = vid[k]
        bv = beta[:, v, :]                                     # (E,4,3)
        bq = np.einsum('qa,ead->eqd', lam, bv)
        fq = np.einsum('qa,ea->eq', lam, fa[:, v])
        dq = np.einsum('qa,ea->eq', lam, dva[:, v])
        bmax = np.linalg.norm(bv, axis=2).max(axis=1)
        PK = hK * bmax / (2.0 * nu)
        with np.errstate(divide='ignore', invalid='ignore'):
            C_adv = tau * hK / (2.0 * bmax)
        C_dif = tau * hK * hK / (4.0 * nu)
        CK = np.where(PK >= 1.0, C_adv, C_dif)
        bg = np.einsum('eqd,ad->eqa', bq, G[k])                # beta.grad lambda_a at q
        Lphi = bg + c * lam[None, :, :]
        ct = c - 0.5 * dq
        diff = nu[:, None, None] * vol * (G[k] @ G[k].T)[None, :, :]
        stab = np.einsum('e,q,eqj,eqi->eij', CK, w, Lphi, Lphi)
        reac = np.einsum('q,eq,qj,qi->eij', w, ct, lam, lam)
        skew = 0.5 * (np.einsum('q,eqj,qi->eij', w, bg, lam) - np.einsum('q,eqi,qj->eij', w, bg, lam))
        At = diff + stab + reac + skew
        Ft = np.einsum('q,eq,qi->ei', w, fq, lam) + np.einsum('e,q,eq,eqi->ei', CK, w, fq, Lphi)
        A[:, v[:, None], v[None, :]] += At
        F[:, v] += Ft
    return A, F


def lift_dirichlet(mesh, Ae, Fe, nodes, g_node):
    """Non-homogeneous Dirichlet values: u = g on the boundary nodes enters as the
    load correction F_i -= sum_j a(phi_j, phi_i) g_j over the boundary nodes j of
    each element (the free-dof system of u - (the boundary interpolant of g))."""
    if g_node is None:
        return Fe
    bnd = node_to_dof(mesh)[nodes] < 0                          # (E,8)
    gb = np.where(bnd, np.asarray(g_node, dtype=float)[nodes], 0.0)
    return Fe - np.einsum('eij,ej->ei', Ae, gb)


def element_matrices(mesh, nu_elem, beta_node, f_node, c=0.0, divb_node=None, tau=TAU,
                     elems=None, element='q1'):
    """Element matrices A[e,i,j] = a_K(phi_j, phi_i) and loads F[e,i] = g_K(phi_i).

    Sect. 2: b(u,v) = int nu grad u.grad v + C Lu Lv + c~ u v,
    z(u,v) = 1/2 int (beta.grad u v - beta.grad v u),
    g(v) = int f v + C f Lv, with P_K and C(x) as defined there.
    element 'q1': trilinear bricks; 'p1': linear elements on the six Kuhn
    tetrahedra of each brick (Sect. 4), returned per brick.
    """
    nodes = element_nodes(mesh)
    if elems is not None:
        nodes = nodes[elems]
        nu = np.asarray(nu_elem, dtype=float)[elems]
    else:
        nu = np.asarray(nu_elem, dtype=float)
    hx, hy, hz = mesh.h
    if element == 'p1':
        fa = np.asarray(f_node, dtype=float)[nodes]
        dva = np.zeros_like(fa) if divb_node is None else np.asarray(divb_node, dtype=float)[nodes]
        A, F = _p1_element_matrices(mesh, nu, np.asarray(beta_node, dtype=float)[nodes], fa, dva, c, tau)
        return A, F, nodes
    N, G, wq = q1_tables(mesh.h)
    detJ = hx * hy * hz
    beta = np.asarray(beta_node, dtype=float)[nodes]          # (E,8,3)
    fa = np.asarray(f_node, dtype=float)[nodes]               # (E,8)
    if divb_node is None:
        dva = np.zeros_like(fa)
    else:
        dva = np.asarray(divb_node, dtype=float)[nodes]
    bq = np.einsum('qa,ead->eqd', N, beta)                     # beta at quad points
    fq = np.einsum('qa,ea->eq', N, fa)
    dq = np.einsum('qa,ea->eq', N, dva)
    bmax = np.maximum(np.linalg.norm(beta, axis=2).max(axis=1),
                      np.linalg.norm(bq, axis=2).max(axis=1))
    hK = np.sqrt(hx * hx + hy * hy + hz * hz)
    PK = hK * bmax / (2.0 * nu)
    with np.errstate(divide='ignore', invalid='ignore'):
        C_adv = tau * hK / (2.0 * bmax)
    C_dif = tau * hK * hK / (4.0 * nu)
    CK = np.where(PK >= 1.0, C_adv, C_dif)
    bg = np.einsum('eqd,qad->eqa', bq, G)                      # beta.grad phi_a
    Lphi = bg + c * N[None, :, :]
    ct = c - 0.5 * dq
    w = wq * detJ
    diff = np.einsum('e,q,qjd,qid->eij', nu, w, G, G, optimize=True)
    stab = np.einsum('e,q,eqj,eqi->eij', CK, w, Lphi, Lphi, optimize=True)
    reac = np.einsum('q,eq,qj,qi->eij', w, ct, N, N, optimize=True)
    skew = 0.5 * (np.einsum('q,eqj,qi->eij', w, bg, N, optimize=True) - np.einsum('q,eqi,qj->eij', w, bg, N, optimize=True))
    A = diff + stab + reac + skew
    F = np.einsum('q,eq,qi->ei', w, fq, N) + np.einsum('e,q,eq,eqi->ei', CK, w, fq, Lphi)
    return A, F, nodes


def node_to_dof(mesh):
    """Array mapping node id -> dof id (-1 for Dirichlet nodes)."""
    nn = mesh.nnode[0] * mesh.nnode[1] * mesh.nnode[2]
    m = -np.ones(nn, dtype=int)
    m[mesh.free_node_ids()] = np.arange(mesh.ndof)
    return m


def assemble_global(mesh, Ae, Fe, nodes):
    """Global sparse matrix and load on the free dofs (Dirichlet rows/cols dropped)."""
    n2d = node_to_dof(mesh)
    dofs = n2d[nodes]                                          # (E,8)
    rows = np.repeat(dofs[:, :, None], 8, axis=2)
    cols = np.repeat(dofs[:, None, :], 8, axis=1)
    mask = (rows >= 0) & (cols >= 0)
    A = sp.coo_matrix((Ae[mask], (rows[mask], cols[mask])), shape=(mesh.ndof, mesh.ndof)).tocsr()
    F = np.zeros(mesh.ndof)
    fm = dofs >= 0
    np.add.at(F, dofs[fm], Fe[fm])
    return A, F


def direct_solve(A, F):
    """u* = A^{-1} F by sparse LU (the reference result)."""
    return spla.splu(A.tocsc()).solve(F)


def assemble_subdomain(mesh, s, Ae, Fe, nodes):
    """Dense local matrix A^(i) and load f^(i) over the local dofs of subdomain s.

    Sect. 3: a_i = b_i + z_i integrated over Omega_i only (the Robin-type
    local form); dofs ordered interior first, then interface.
    """
    n2d = node_to_dof(mesh)
    loc = -np.ones(mesh.ndof, dtype=int)
    loc[mesh.sub_dofs[s]] = np.arange(len(mesh.sub_dofs[s]))
    el = mesh.sub_elems[s]
    d = n2d[nodes[el]]                                         # (e,8) dof or -1
    dl = np.where(d >= 0, loc[np.maximum(d, 0)], -1)           # local index or -1
    n = len(mesh.sub_dofs[s])
    A = np.zeros((n, n))
    F = np.zeros(n)
    ri = np.repeat(dl[:, :, None], 8, axis=2)
    cj = np.repeat(dl[:, None, :], 8, axis=1)
    m = (ri >= 0) & (cj >= 0)
    np.add.at(A, (ri[m], cj[m]), Ae[el][m])
    fm = dl >= 0
    np.add.at(F, dl[fm], Fe[el][fm])
    return A, F
