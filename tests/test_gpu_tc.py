"""The tensor-core building block of the projector contractions (tcgen05 kind::tf32 MMAs from
shared-memory descriptors, TMEM accumulators, three-product TF32 split) against an FP64 product.

Bound: with a_hi = a rounded to TF32 and a_lo the rounded remainder, a_hi b_hi + a_hi b_lo + a_lo b_hi
differs from a b by at most about 3 x 2^-22 |a b|; the FP32 accumulation over K terms adds at most
K x 2^-24 sum |a b|.  Each element is held to (3.01 x 2^-22 + K x 2^-24) (|A| |B|^T)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")


@pytest.mark.parametrize("M,N,K", [(128, 48, 256), (56, 16, 64), (128, 128, 32), (100, 64, 1024)])
def test_tf32_split_product(M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = (rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, 1)))).astype(np.float32)
    D = P.selftest_tc(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    bound = (3.01 * 2.0 ** -22 + K * 2.0 ** -24) * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    assert np.all(np.abs(D - ref) <= bound)


def test_descriptor_reading():
    """The operand descriptors' leading-byte offset steps along K and the stride-byte offset across
    8-row groups: exchanging the two fields (an in-bounds reading of the same tiles) gives a wrong
    product."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    B = rng.standard_normal((32, 64)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    good = P.selftest_tc(A, B, lbo_swap=0)
    bad = P.selftest_tc(A, B, lbo_swap=1)
    assert np.abs(good - ref).max() < 1e-5 * np.abs(ref).max()
    assert np.abs(bad - ref).max() > 1e-2 * np.abs(ref).max()
