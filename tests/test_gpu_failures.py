"""Failure paths of the C ABI on the GPU, none of which faults or hangs it.

* invalid inputs are rejected with BDDC_EINVAL before any solver work: a
  viscosity <= 0 or NaN (host and device arrays), a non-finite velocity, a
  slab without elements, a subdomain interior above 8192 dofs, a face above
  256 dofs;
* a solve that reaches its iteration cap returns BDDC_NOT_CONVERGED with the
  iterate written (finite, the residual reduced);
* the bounded device waits end by themselves: the one-launch apply's wait,
  run on a counter that nothing increments, gives up and reports
  BDDC_ETIMEOUT, and the device keeps working (a setup and apply right after
  it match the oracle).
"""
import numpy as np
import pytest

from paper_2501_01676_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EINVAL, ETIMEOUT, NOT_CONVERGED = -1, -5, 1


def B():
    from paper_2501_01676_gb300 import bddc
    return bddc


def _expect_einval(p, **kw):
    with pytest.raises(B().BDDCError) as ei:
        B().Solver(p, **kw)
    assert ei.value.code == EINVAL


@pytest.mark.parametrize("host", [True, False])
@pytest.mark.parametrize("bad", ["zero", "negative", "nan"])
def test_rejects_invalid_viscosity(host, bad):
    p = W.random_small(1, (2, 2, 2), 3, (-2, 0))
    p.nu_elem = p.nu_elem.copy()
    p.nu_elem[17] = {"zero": 0.0, "negative": -1e-3, "nan": np.nan}[bad]
    _expect_einval(p, host=host)


def test_rejects_non_finite_velocity():
    p = W.random_small(1, (2, 2, 2), 3, (-2, 0))
    p.beta_node = p.beta_node.copy()
    p.beta_node[5, 1] = np.inf
    _expect_einval(p)


def test_rejects_empty_slab():
    p = W.random_small(1, (2, 2, 2), 3, (-2, 0))
    p.slabs = [[3, 0], [3, 3], [3, 3]]
    _expect_einval(p)


def _box_problem(slabs):
    ne = [sum(s) for s in slabs]
    n = (ne[0] + 1) * (ne[1] + 1) * (ne[2] + 1)
    return W.Problem("box", slabs, np.ones(ne[0] * ne[1] * ne[2]), np.tile([1.0, 0.5, 0.25], (n, 1)), np.ones(n))


def test_rejects_too_large_interior_and_face():
    _expect_einval(_box_problem([[22], [22], [22]]))          # 21^3 = 9261 interior dofs
    _expect_einval(_box_problem([[2, 2], [18, 18], [18, 18]]))  # x-faces of 17 x 17 = 289 dofs
    s = B().Solver(_box_problem([[2, 2], [17, 17], [17, 17]]))  # 16 x 16 = 256: accepted
    assert s.stats()["pnumF"] >= 0
    s.close()


def test_iteration_cap_returns_not_converged_with_result():
    import torch
    p = W.random_small(2, (3, 3, 3), 3, (-3, 1))
    s = B().Solver(p, max_iter=2)
    u, st = s.solve()
    assert st["rc"] == NOT_CONVERGED and st["converged"] == 0 and st["iters"] == 2
    u = u.cpu().numpy()
    assert np.isfinite(u).all() and np.abs(u).max() > 0
    assert 0 < st["relres_global"] < 1.0


def test_bounded_wait_gives_up_and_device_stays_usable():
    import torch

    from oracle import bddc as obddc
    assert B().wait_selftest(2000) == ETIMEOUT
    p = W.random_small(3, (2, 2, 2), 3, (-2, 1))
    s = B().Solver(p)
    o = obddc.BDDC(p)
    r = np.random.default_rng(1).standard_normal(o.nG)
    z = s.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = o.apply_M(r)
    assert np.abs(z - zo).max() <= 1e-9 * np.abs(zo).max()
