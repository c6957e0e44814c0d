"""The allocation-free H psi entry point against the allocating one.

hp_apply_h_noalloc exists for callers that cannot call cudaMalloc while they compute (their own
pool allocator owns the free device memory, or device-synchronising allocation calls are not
allowed in their loop); it keeps all scratch in a fixed device array instead.  Two calls in a row
must each reproduce hp_apply_h on fresh inputs (the array keeps the previous call's contents), and
a batch too large for the fixed scratch must be refused with HP_EINVAL.  This file is collected
last so that a failure here cannot hide the results of the other tests."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    w = W.tiny()  # 20^3 grid, 751-804 plane waves per k
    c = P.Context.from_workload(w)
    s = c.query_sizes()
    rng = np.random.default_rng(11)
    nr, nk, no = s["nr"], s["nk"], int(w["nelec"] // 2)
    vhxc = rng.standard_normal((1, nr)) * 0.3
    rho = np.abs(rng.standard_normal((1, nr))) * 0.05
    psi = [[np.linalg.qr(W.random_coefficients(40 + k, (len(c.sphere(k)), no)))[0] for k in range(nk)]]
    c.set_ground_state(1, w["nelec"], vhxc, rho, np.zeros((1, nk, no)), psi)
    return c


def _rows(ctx, ik, X):
    npw_max = ctx.query_sizes()["npw_max"]
    out = np.zeros((X.shape[0], npw_max), dtype=np.complex128)
    out[:, : X.shape[1]] = X
    return out


def _noalloc(ctx, ik, X):
    """One allocation-free call on fresh device rows; returns (result, device allocations made by
    the library during the call)."""
    nb = X.shape[0]
    xd = torch.from_numpy(_rows(ctx, ik, X).view(np.float64)).cuda()
    yd = torch.full_like(xd, float("nan"))
    torch.cuda.synchronize()
    a0 = P.alloc_count()
    ctx.apply_h_noalloc(ik, 0, nb, xd.data_ptr(), yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    made = P.alloc_count() - a0
    return yd.cpu().numpy().view(np.complex128), made


@pytest.mark.parametrize("ik", [0, 5])
def test_noalloc_matches_allocating_entry_point_twice(ctx, ik):
    npw = len(ctx.sphere(ik))
    for call, nb in enumerate((37, 11)):
        X = W.random_coefficients(1000 * ik + call, (nb, npw))
        ref = ctx.apply_h(ik, 0, X)
        got, made = _noalloc(ctx, ik, X)
        assert made == 0                   # the defining property: no device allocation at call time
        assert np.all(got[:, npw:] == 0)
        assert np.abs(got[:, :npw] - ref).max() < 1e-11 * np.abs(ref).max()


def test_noalloc_several_grid_chunks(ctx):
    """600 bands on the 20^3 grid: the fixed scratch holds about 490 FFT grids after the band list
    and projections, so the local part runs in two chunks, the second one partial (offsets c0 > 0
    into the band list for the scatter, the potential and the gather)."""
    ik = 3
    npw = len(ctx.sphere(ik))
    X = W.random_coefficients(4242, (600, npw))
    ref = ctx.apply_h(ik, 0, X)
    got, made = _noalloc(ctx, ik, X)
    assert made == 0
    assert np.all(got[:, npw:] == 0)
    assert np.abs(got[:, :npw] - ref).max() < 1e-11 * np.abs(ref).max()


def test_noalloc_rejects_batches_beyond_the_fixed_scratch(ctx):
    nb = 20000  # 20000 x (128 projections + 128 partial sums) x 16 B alone exceeds 64 MiB
    npw_max = ctx.query_sizes()["npw_max"]
    xd = torch.zeros((nb, 2 * npw_max), dtype=torch.float64, device="cuda")
    yd = torch.zeros_like(xd)
    with pytest.raises(P.HPError) as e:
        ctx.apply_h_noalloc(0, 0, nb, xd.data_ptr(), yd.data_ptr())
    assert e.value.code == 1  # HP_EINVAL, nothing launched
    assert "fixed" in ctx.last_error()
