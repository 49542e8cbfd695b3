"""bddc_apply_static against bddc_apply.

bddc_apply_static is for callers that cannot allocate device memory where
they apply the preconditioner (for example a host framework that owns all
device memory).  Its work vectors live in the library's static device array.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process (where its
first call performs the per-device lookup of the array) and after the rest.
"""
import numpy as np
import pytest

from paper_2501_01676_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_static_matches_apply_on_two_calls(precision):
    import torch

    from paper_2501_01676_gb300.bddc import Solver
    p = W.random_small(1, (3, 3, 3), 3, (-3, 3))
    s = Solver(p, theta_E=1.5, precision=precision)
    rng = np.random.default_rng(17)
    for _ in range(2):
        r = torch.from_numpy(rng.standard_normal(s.n_gamma)).cuda()
        z_ref = s.apply(r).cpu().numpy()
        z = s.apply_static(r).cpu().numpy()
        # same kernels, FP64 atomics in a different order: the parity tolerance of the suite
        assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max()
    s.close()


def test_apply_static_several_columns():
    """nrhs = 2: the columns run one after the other through the shared array."""
    import torch

    from paper_2501_01676_gb300.bddc import Solver
    p = W.random_small(2, (3, 3, 3), 3, (-2, 1))
    s = Solver(p, precision=1)
    r = torch.from_numpy(np.random.default_rng(5).standard_normal((s.n_gamma, 2))).cuda()
    z_ref = s.apply(r).cpu().numpy()
    z = s.apply_static(r).cpu().numpy()
    assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max()
    s.close()
