"""The P1 discretisation on the six Kuhn tetrahedra of each brick (Sect. 4) and
non-homogeneous Dirichlet values on the GPU, against the oracle:

* S^(i) of every subdomain of a small random P1 case (FP64 path, 1e-10 relative);
* the solution with lifted boundary values against the oracle's direct solve
  (FP64 and mixed solvers, residual 1e-12, 1e-8 relative);
* the patch test: a linear exact solution reproduced at the nodes;
* Example 4.1 at m = 4 (Tests 1-3, nu_1 = 1, nu_2 = 1e-7, the paper's Table 5 row),
  new and conventional edge GEPs: the constraint counts (pnumF, pnumE) equal the
  oracle's and the iteration counts are within one of the oracle's GMRES;
* the same on the random-viscosity variant (2^3 and 3^3 subdomains of 4^3 cubes);
* Example 4.1 at m = 16 (the paper's Table 5 row): faces of 225 dofs (the face
  GEP kernel's global-memory path) and 3375 interior dofs per subdomain: the
  large face eigenvalues, constraint counts and iterations against the oracle
  (FP64), and the mixed solver's global residual.
"""
import numpy as np
import pytest

from oracle import bddc as obddc
from oracle import fem
from oracle.mesh import Mesh
from paper_2501_01676_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_2501_01676_gb300 import bddc
    return bddc


def random_p1(seed=11, slabs=((3, 2), (2, 3), (3, 2))):
    rng = np.random.default_rng(seed)
    slabs = [list(s) for s in slabs]
    ne, h, X, Y, Z = W._grid(slabs)
    nel = ne[0] * ne[1] * ne[2]
    nu = 10.0 ** rng.uniform(-2, 1, nel)
    beta = np.stack([np.sin(3 * Y) + 0.5, np.cos(2 * X), 0.3 * Z - 0.1], axis=1)
    f = rng.standard_normal(X.size)
    g = rng.standard_normal(X.size)
    return W.Problem("p1_random", slabs, nu, beta, f, c=0.4, element='p1', dirichlet_node=g)


def system(p):
    mesh = Mesh(p.slabs)
    f = p.f_node if p.f_node is not None else np.zeros(p.beta_node.shape[0])
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, f, p.c, element=p.element)
    Fe = fem.lift_dirichlet(mesh, Ae, Fe, nodes, p.dirichlet_node)
    A, F = fem.assemble_global(mesh, Ae, Fe, nodes)
    return mesh, Ae, Fe, nodes, A, F


def test_p1_schur_complements_match_the_oracle():
    p = random_p1()
    mesh, Ae, Fe, nodes, A, F = system(p)
    s = B().Solver(p)
    for sd in range(mesh.nsd):
        Asub, _ = fem.assemble_subdomain(mesh, sd, Ae, Fe, nodes)
        nI = mesh.sub_nI[sd]
        So = Asub[nI:, nI:] - Asub[nI:, :nI] @ np.linalg.solve(Asub[:nI, :nI], Asub[:nI, nI:])
        S = s.schur(sd)
        assert np.abs(S - So).max() < 1e-10 * np.abs(So).max(), sd
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_p1_solution_with_dirichlet_values_matches_the_direct_solve(precision):
    p = random_p1(seed=12)
    mesh, Ae, Fe, nodes, A, F = system(p)
    ustar = fem.direct_solve(A, F)
    s = B().Solver(p, precision=precision, rtol=1e-12)
    u, st = s.solve()
    u = u.cpu().numpy()
    assert st["converged"]
    assert np.linalg.norm(u - ustar) / np.linalg.norm(ustar) < 1e-8
    s.close()


def test_p1_patch_test_on_the_gpu():
    slabs = [[3, 2], [2, 3], [2, 2]]
    ne, h, X, Y, Z = W._grid(slabs)
    beta, c = np.array([0.7, -0.4, 1.1]), 0.8
    u = 1.0 + 0.5 * X - 2.0 * Y + 1.5 * Z
    f = beta @ np.array([0.5, -2.0, 1.5]) + c * u
    p = W.Problem("p1_patch", slabs, np.full(ne[0] * ne[1] * ne[2], 0.05), np.tile(beta, (X.size, 1)), f, c=c,
                  element='p1', dirichlet_node=u)
    s = B().Solver(p, rtol=1e-13)
    uh, st = s.solve()
    free = Mesh(slabs).free_node_ids()
    assert np.abs(uh.cpu().numpy() - u[free]).max() < 1e-9
    s.close()


@pytest.mark.parametrize("test", [1, 2, 3])
@pytest.mark.parametrize("edge", ["new", "old"])
def test_example41_counts_and_iterations_match_the_oracle(test, edge):
    p = W.example41(test=test, m=4, nu1=1.0, nu2=1e-7)
    o = obddc.BDDC(p, edge_gep=edge)
    _, info = o.solve()
    s = B().Solver(p, edge_gep=B().EDGE_NEW if edge == "new" else B().EDGE_OLD)
    st = s.stats()
    assert (st["pnumF"], st["pnumE"]) == (o.pnumF, o.pnumE)
    _, sv = s.solve()
    assert sv["converged"] and abs(sv["iters"] - info["iters"]) <= 1
    s.close()


@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("edge", ["new", "old"])
def test_example41_random_viscosity_matches_the_oracle(n, edge):
    p = W.example41_random(n=n, m=4)
    o = obddc.BDDC(p, edge_gep=edge)
    _, info = o.solve()
    s = B().Solver(p, edge_gep=B().EDGE_NEW if edge == "new" else B().EDGE_OLD)
    st = s.stats()
    assert (st["pnumF"], st["pnumE"]) == (o.pnumF, o.pnumE)
    _, sv = s.solve()
    assert sv["converged"] and abs(sv["iters"] - info["iters"]) <= 1
    s.close()


def _face_lambdas(s, o):
    ge = s.entities(2)
    by = {e['subs']: i for i, e in enumerate(o.mesh.entities) if e['kind'] == 'F'}
    return [(g, o.face_info[by[g['subs']]]) for g in ge]


@pytest.mark.parametrize("edge", ["new", "old"])
def test_example41_m16_large_faces_match_the_oracle(edge):
    p = W.example41(test=1, m=16, nu1=1.0, nu2=1e-7)
    o = obddc.BDDC(p, edge_gep=edge)
    _, info = o.solve()
    s = B().Solver(p, edge_gep=B().EDGE_NEW if edge == "new" else B().EDGE_OLD)
    for g, ref in _face_lambdas(s, o):
        assert len(g['dofs']) == 225
        lo, lg = ref['lam'], g['lam']
        big = np.isfinite(lo) & (lo > 0.5)
        np.testing.assert_allclose(lg[big], lo[big], rtol=1e-6)
        assert g['k'] == ref['Q'].shape[1]
    st = s.stats()
    assert (st['pnumF'], st['pnumE']) == (o.pnumF, o.pnumE)
    _, sv = s.solve()
    assert sv["converged"] and abs(sv["iters"] - info["iters"]) <= 1
    s.close()


def test_example41_m16_mixed_precision_reaches_the_global_residual():
    p = W.example41(test=2, m=16, nu1=1.0, nu2=1e-7)
    s = B().Solver(p, precision=B().PREC_MIXED)
    _, sv = s.solve()
    assert sv["converged"] and sv["relres_global"] <= 1e-8
    s.close()
