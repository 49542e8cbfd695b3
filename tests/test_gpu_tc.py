"""The tcgen05 (split TF32) trailing update against FP64 products.

Split TF32 represents each FP32 operand as hi + lo (both TF32) and drops the
lo*lo term: the error per product is about 2^-21 relative, so K = 32 terms stay
within 1e-5 of the largest partial sum; the test allows 1e-4.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def B():
    from paper_2501_01676_gb300 import bddc
    return bddc


@pytest.mark.parametrize("nr,nc,K", [(128, 128, 32), (97, 45, 32), (128, 128, 17), (5, 128, 3)])
def test_tile_against_fp64(nr, nc, K):
    rng = np.random.default_rng(nr * 1000 + nc + K)
    A = rng.standard_normal((128, 32)).astype(np.float32)
    Bm = rng.standard_normal((32, 128)).astype(np.float32)
    C = rng.standard_normal((128, 128)).astype(np.float32)
    out = B().tc_selftest(A, Bm, C, nr, nc, K)
    ref = C.astype(np.float64).copy()
    ref[:nr, :nc] -= A[:nr, :K].astype(np.float64) @ Bm[:K, :nc].astype(np.float64)
    scale = np.abs(A[:nr, :K]).max() * np.abs(Bm[:K, :nc]).max() * K
    assert np.abs(out - ref).max() <= 1e-4 * scale
    # entries outside the nr x nc block are untouched
    assert np.array_equal(out[nr:, :], C[nr:, :]) and np.array_equal(out[:, nc:], C[:, nc:])


def test_engine_tensor_cores_match_cuda_cores():
    """Schur complements of the mixed path: tcgen05 trailing updates vs FP32 CUDA cores."""
    from paper_2501_01676_gb300 import workloads as W
    p = W.random_small(2, (3, 3, 3), 4, (-2, 1))
    a = B().Solver(p, precision=1, tensor_cores=1)
    b = B().Solver(p, precision=1, tensor_cores=0)
    for sd in range(27):
        Sa, Sb = a.schur(sd), b.schur(sd)
        assert np.abs(Sa - Sb).max() <= 2e-5 * np.abs(Sb).max()
    ua, sa = a.solve()
    ub, sb = b.solve()
    assert sa["converged"] and sb["converged"]
    assert (ua - ub).abs().max().item() <= 1e-7 * ub.abs().max().item()


def test_bf16_updates_schur_and_refined_solution():
    """precision 2: the trailing updates of the FP32 eliminations on the tensor cores
    with BF16 operands (FP32 accumulation).  The Schur complements carry a BF16-level
    error, clearly above the split-TF32 path's (so the BF16 tiles did run), and the
    FP64 refinement still reaches the 1e-8 residual and the FP64 solution."""
    from paper_2501_01676_gb300 import workloads as W
    p = W.uniform(2, 8, nu=0.05, beta=(1.0, 0.5, 0.25))
    bf = B().Solver(p, precision=2)
    tf = B().Solver(p, precision=1, tensor_cores=1)
    f64 = B().Solver(p, precision=0)
    e_bf = e_tf = 0.0
    for sd in range(f64.stats()["nsub"]):
        S = f64.schur(sd)
        nS = np.linalg.norm(S)
        e_bf = max(e_bf, np.linalg.norm(bf.schur(sd) - S) / nS)
        e_tf = max(e_tf, np.linalg.norm(tf.schur(sd) - S) / nS)
    assert e_bf <= 5e-2
    assert e_bf >= 10 * e_tf
    u, st = bf.solve()
    assert st["converged"] and st["relres"] <= 1e-8
    u64, _ = f64.solve()
    assert (u - u64).abs().max().item() <= 1e-6 * u64.abs().max().item()
