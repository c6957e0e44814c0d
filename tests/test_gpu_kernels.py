"""Device kernels checked one by one against numpy or the hardware: the batched Hermitian
eigensolver of the ground state (including matrices whose off-diagonal entries underflow during
the sweeps) and the integer-operation FP64/FP32 conversions of the FP32 form."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")


def _check(A, tol=1e-12):
    w, V = P.selftest_eigh(A)
    n = A.shape[-1]
    for b in range(len(A)):
        ref = np.linalg.eigvalsh(A[b])
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(w[b] - ref).max() < tol * scale
        assert np.abs(V[b].conj().T @ V[b] - np.eye(n)).max() < tol
        assert np.abs(A[b] @ V[b] - V[b] * w[b][None, :]).max() < tol * scale


@pytest.mark.parametrize("n", [1, 2, 5, 24, 30, 31, 64, 128])
def test_eigh_random_and_degenerate(n):
    rng = np.random.default_rng(n)
    As = []
    for b in range(5):
        Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
        ev = rng.standard_normal(n) * 3
        if b % 2:
            ev[: n // 3] = ev[0]
        As.append(Q @ np.diag(ev) @ Q.conj().T)
    _check(np.array(As))


def test_eigh_block_structure_with_underflowing_couplings():
    """Degenerate blocks embedded in a permuted basis with 1e-170 couplings between blocks: the
    sweeps must skip pairs whose coupling is negligible instead of forming their phase."""
    rng = np.random.default_rng(7)
    n, As = 30, []
    for b in range(4):
        A = np.zeros((n, n), dtype=complex)
        for s in range(0, n, 3):
            Qb = np.linalg.qr(rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))[0]
            ev = -3 + 0.1 * (s // 3) + np.array([0.0, 0.0, 1e-9])
            A[s:s + 3, s:s + 3] = Qb @ np.diag(ev) @ Qb.conj().T
        C = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 1e-170
        A = A + C + C.conj().T
        perm = rng.permutation(n)
        As.append(A[np.ix_(perm, perm)])
    _check(np.array(As))


def test_integer_fp64_fp32_conversions_match_hardware():
    """FP64 -> FP32 rounding by integer operations (FP32 form's hot loops) equals the hardware
    round-to-nearest-even conversion bit for bit over the FP32 normal range, including exact ties
    in both directions; below that range it gives a signed zero, above it a signed infinity; the
    widening back to FP64 is exact."""
    rng = np.random.default_rng(2203)
    mant = rng.random(20000) + 1.0
    expo = rng.integers(-140, 140, 20000)
    x = mant * 2.0 ** expo * rng.choice([-1.0, 1.0], 20000)
    # exact ties: an FP32 value plus half of its last place (even and odd last bits)
    f = rng.random(4000).astype(np.float32) * np.float32(1e3) + np.float32(1.0)
    half = np.spacing(f).astype(np.float64) / 2.0
    ties = f.astype(np.float64) + half
    x = np.concatenate([x, ties, -ties, [0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 1.1754943508222875e-38]])
    out, back, ref, back_ref = P.selftest_convert(x)
    tiny = np.float64(np.finfo(np.float32).tiny)
    normal = np.isfinite(ref) & (np.abs(ref.astype(np.float64)) >= tiny)
    assert np.array_equal(out[normal].view(np.uint32), ref[normal].view(np.uint32))
    assert np.array_equal(back[normal], back_ref[normal])
    low = np.abs(x) < tiny / 2
    assert np.all(out[low] == 0.0) and np.array_equal(np.signbit(out[low]), np.signbit(x[low]))
    high = np.abs(x) > 3.5e38
    assert np.all(np.isinf(out[high])) and np.array_equal(np.signbit(out[high]), np.signbit(x[high]))
    assert normal.sum() > 15000 and low.sum() > 100 and high.sum() > 100
