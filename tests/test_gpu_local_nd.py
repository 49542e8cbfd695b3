"""Local nested dissection on the GPU (opts.local_nd = 1: each subdomain's box
split into up to 2 x 2 x 2 child boxes whose interiors are eliminated first, then
the separator planes), against the oracle, which eliminates each subdomain's
interior in one dense step (Sect. 3: S^(i) = A_BB - A_BI A_II^{-1} A_IB):

* S^(i) of every subdomain (uneven slabs with odd and 1-element slabs, Q1 and
  P1), FP64, 1e-10 relative;
* the solution against the oracle's direct solve (FP64 and mixed solvers,
  residual 1e-12, 1e-8 relative), one load and three loads in one call (the
  batched path condenses and recovers through the children as well);
* Example 4.1 at m = 16: constraint counts and iterations as with the dense
  elimination and the oracle, with fewer elimination flops.
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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _uneven(element='q1', seed=9):
    p = W.random_small(5, (2, 3, 2), 4, (-2, 1))
    p.slabs = [[3, 5], [4, 1, 3], [6, 4]]
    ne = [sum(s) for s in p.slabs]
    _, _, X, Y, Z = W._grid(p.slabs)
    rng = np.random.default_rng(seed)
    p.nu_elem = 10.0 ** rng.uniform(-2, 1, ne[0] * ne[1] * ne[2])
    p.beta_node = np.stack([-(Y - 0.5), X - 0.5, np.full_like(X, 0.1)], axis=1)
    p.f_node = rng.standard_normal(X.size)
    p.c = 0.3
    p.element = element
    if element == 'p1':
        p.dirichlet_node = rng.standard_normal(X.size)
    return p


def _system(p):
    mesh = Mesh(p.slabs)
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, p.f_node, p.c, element=p.element)
    Fe = fem.lift_dirichlet(mesh, Ae, Fe, nodes, p.dirichlet_node)
    return fem.assemble_global(mesh, Ae, Fe, nodes)


@pytest.mark.parametrize("element", ["q1", "p1"])
def test_local_nd_schur_complements_match_the_oracle(element):
    p = _uneven(element)
    o = obddc.BDDC(p)
    s = B().Solver(p, local_nd=1)
    st = s.stats()
    assert st["nd_children"] > o.mesh.nsd
    for sd in range(o.mesh.nsd):
        assert rel(s.schur(sd), o.S[sd]) < 1e-10, sd
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_local_nd_solution_matches_the_direct_solve(precision):
    p = _uneven('p1', seed=10)
    A, F = _system(p)
    ustar = fem.direct_solve(A, F)
    s = B().Solver(p, precision=precision, rtol=1e-12, local_nd=1)
    u, st = s.solve()
    assert st["converged"]
    assert np.linalg.norm(u.cpu().numpy() - ustar) / np.linalg.norm(ustar) < 1e-8
    # three loads in one call (batched condensation and recovery)
    rng = np.random.default_rng(11)
    L = rng.standard_normal((F.size, 3))
    U, sb = s.solve(load=L)
    U = U.cpu().numpy()
    for c in range(3):
        x = fem.direct_solve(A, L[:, c])
        assert np.linalg.norm(U[:, c] - x) / np.linalg.norm(x) < 1e-8, c
    s.close()


def test_local_nd_example41_m16_matches_the_dense_elimination():
    p = W.example41(test=2, m=16, nu1=1.0, nu2=1e-7)
    o = obddc.BDDC(p, edge_gep='new')
    _, info = o.solve()
    s = B().Solver(p, local_nd=1)
    st = s.stats()
    assert st["nd_children"] == 64
    assert (st["pnumF"], st["pnumE"]) == (o.pnumF, o.pnumE)
    _, sv = s.solve()
    assert sv["converged"] and abs(sv["iters"] - info["iters"]) <= 1
    d = B().Solver(p)
    assert st["factor_gflop"] < 0.25 * d.stats()["factor_gflop"]
    for sd in (0, 7):
        assert rel(s.schur(sd), d.schur(sd)) < 1e-9
    s.close()
    d.close()


def test_local_nd_full_size_jump_workload():
    """The 8 x 8 x 8-subdomain jump workload (H/h = 8, 4096 child boxes) in the
    mixed solver: the same constraint counts as the dense elimination, the global
    FP64 residual at the 1e-8 rule, sampled S^(i) equal to the dense path's to
    FP32 rounding."""
    p = W.config3()
    mesh = Mesh(p.slabs)
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, p.f_node, p.c)
    A, F = fem.assemble_global(mesh, Ae, Fe, nodes)
    d = B().Solver(p, precision=1)
    s = B().Solver(p, precision=1, local_nd=1)
    sd, ss = d.stats(), s.stats()
    assert ss["nd_children"] == 4096
    assert (ss["pnumF"], ss["pnumE"], ss["n_pi"]) == (sd["pnumF"], sd["pnumE"], sd["n_pi"])
    for k in (0, 73, 292, 511):
        assert rel(s.schur(k), d.schur(k)) < 1e-4, k
    u, st = s.solve()
    u = u.cpu().numpy()
    assert st["converged"] and np.linalg.norm(F - A @ u) / np.linalg.norm(F) <= 1e-8
    s.close()
    d.close()
    for nd in (0, 1):                       # warm second setups, for the record
        t = B().Solver(p, precision=1, local_nd=nd)
        _, sv = t.solve()
        tt = t.stats()
        print(f"local_nd={nd}: setup {tt['setup_ms']:.1f} ms (eliminations {tt['factor_gflop']:.1f} GFLOP, "
              f"assembly phase {tt['t_assemble_ms']:.2f} ms, factor phase {tt['t_factor_ms']:.2f} ms) "
              f"solve {sv['solve_ms']:.1f} ms, {sv['iters']} iterations")
        t.close()
