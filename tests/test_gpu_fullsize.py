"""Full-size workloads on the GPU, checked on sampled outputs the oracle computes
one by one and through properties that hold at any size.

* 8x8x8 subdomains, H/h = 8 (250 047 dofs), per-subdomain jumps: S^(i) of sampled
  subdomains against the oracle (FP64 path, 1e-10 relative); the global FP64
  residual of the mixed solution recomputed on the host from the oracle's
  assembled matrix (<= 1e-8 relative).
* the channel / Fourier-velocity workload at the same size: global residual.
* uneven slabs (H/h drawn from 6..10 per slab) with several load vectors:
  every column against the oracle's direct solve, FP64 and mixed paths.
* the 6x6x6 uneven-slab workload with 64 N(0,1) nodal loads: a sample of the
  columns solved in one call, each column's global FP64 residual recomputed on
  the host from the oracle's assembled matrix (<= 1e-8 relative).
"""
import numpy as np
import pytest

from oracle import fem
from oracle.mesh import Mesh
from paper_2501_01676_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_2501_01676_gb300 import bddc
    return bddc


def global_system(p):
    mesh = Mesh(p.slabs)
    f = p.f_node if p.f_node is not None else np.zeros(p.beta_node.shape[0])
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, f, p.c)
    A, F = fem.assemble_global(mesh, Ae, Fe, nodes)
    return mesh, Ae, Fe, nodes, A, F


def schur_of(mesh, s, Ae, Fe, nodes):
    A, _ = fem.assemble_subdomain(mesh, s, Ae, Fe, nodes)
    nI = mesh.sub_nI[s]
    return A[nI:, nI:] - A[nI:, :nI] @ np.linalg.solve(A[:nI, :nI], A[:nI, nI:])


def test_config3_sampled_schur_and_global_residual():
    p = W.config3()
    mesh, Ae, Fe, nodes, A, F = global_system(p)
    s64 = B().Solver(p)
    for sd in (0, 73, 292, 511):
        S = s64.schur(sd)
        So = schur_of(mesh, sd, Ae, Fe, nodes)
        assert np.abs(S - So).max() < 1e-10 * np.abs(So).max()
    s64.close()
    s = B().Solver(p, precision=1)
    u, st = s.solve()
    u = u.cpu().numpy()
    assert st["converged"]
    assert np.linalg.norm(F - A @ u) / np.linalg.norm(F) <= 1e-8


def test_config5_global_residual():
    p = W.config5()
    mesh, Ae, Fe, nodes, A, F = global_system(p)
    s = B().Solver(p, precision=1)
    u, st = s.solve()
    u = u.cpu().numpy()
    assert st["converged"]
    assert np.linalg.norm(F - A @ u) / np.linalg.norm(F) <= 1e-8


def uneven_problem(nrhs=3):
    rng = np.random.default_rng(20250103 + 4)
    slabs = [list(rng.integers(6, 11, size=3)) for _ in range(3)]
    ne, h, X, Y, Z = W._grid(slabs)
    p = W.Problem("uneven_3x3x3", slabs, np.full(ne[0] * ne[1] * ne[2], 1e-2),
                  np.tile(np.array([1.0, 1.0, 0.0]), (X.size, 1)), None,
                  load=rng.standard_normal((W.ndof_of(slabs), nrhs)))
    return p


@pytest.mark.parametrize("precision", [0, 1])
def test_uneven_slabs_multiple_loads(precision):
    p = uneven_problem()
    mesh, Ae, Fe, nodes, A, F = global_system(p)
    ustar = np.stack([fem.direct_solve(A, p.load[:, c]) for c in range(p.load.shape[1])], 1)
    s = B().Solver(p, precision=precision, rtol=1e-12)
    u, st = s.solve(p.load)
    u = u.cpu().numpy()
    for c in range(p.load.shape[1]):
        assert np.linalg.norm(u[:, c] - ustar[:, c]) / np.linalg.norm(ustar[:, c]) < 1e-8


def test_config4_multiple_loads_global_residual():
    p = W.config4()
    mesh = Mesh(p.slabs)
    zero = np.zeros(p.beta_node.shape[0])
    Ae, Fe, nodes = fem.element_matrices(mesh, p.nu_elem, p.beta_node, zero, p.c)
    A, _ = fem.assemble_global(mesh, Ae, Fe, nodes)
    cols = [0, 17, 42, 63]
    loads = np.ascontiguousarray(p.load[:, cols])
    s = B().Solver(p, precision=1)
    u, st = s.solve(loads)
    u = u.cpu().numpy()
    assert st["converged"]
    for c in range(len(cols)):
        r = loads[:, c] - A @ u[:, c]
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(loads[:, c]), cols[c]
