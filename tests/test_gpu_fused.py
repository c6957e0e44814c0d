"""The three routes between the wavefunction sphere and real space give the oracle's response.

Routes: fused column/plane transforms with register-resident line FFTs (the default), the same
fused transforms with shared-memory line FFTs (HP_FUSED_SMEM), and the batched 3D FFT with
scatter/gather (HP_NO_FUSED, and any grid the fused kernels do not cover).  Grids: a cube, a grid
whose z size differs from x and y (fused, non-cubic columns), and one with a z size the fused
kernels do not cover (falls back to the 3D FFT).  q != 0, so the k+q spheres are shifted copies.
FP64 at 1e-8 relative to max|Delta n| (the FP64 parity bar)."""

import numpy as np
import pytest

import workloads as W
from oracle import groundstate as G, response as R
from oracle.model import Model
from tests.bridge import import_ground_state, oracle_dn_padded

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")

ROUTES = {"register": {}, "shared": {"HP_FUSED_SMEM": "1"}, "fft3d": {"HP_NO_FUSED": "1"}}
GRIDS = [(12, 12, 12), (12, 12, 15), (12, 12, 25)]

_cache = {}


def _reference(grid):
    if grid not in _cache:
        w = W.tiny_q(ecut=8.0, grid=grid, kmesh=(2, 2, 2), qmesh=(2, 1, 1))
        m = Model(w)
        gs = G.scf(m, tol=1e-12)
        J = m.hub_atoms[0]
        ref = R.solve_column(m, gs, 1, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
        _cache[grid] = (w, m, gs, J, ref)
    return _cache[grid]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("route", list(ROUTES))
def test_route_matches_oracle(monkeypatch, grid, route):
    w, m, gs, J, ref = _reference(grid)
    for k, v in ROUTES[route].items():
        monkeypatch.setenv(k, v)
    ctx = P.Context.from_workload(w, cg_tol=1e-12, scf_tol=1e-11, conv_thr_chi=1e-11)
    import_ground_state(ctx, m, gs)
    dn0, dn, info = ctx.response(1, J)
    r0 = oracle_dn_padded(m, ref["dn0"])
    r1 = oracle_dn_padded(m, ref["dn"])
    assert np.abs(dn0 - r0).max() < 1e-8 * np.abs(r0).max()
    assert np.abs(dn - r1).max() < 1e-8 * np.abs(r1).max()
    assert info["iterations"] > 2


@pytest.mark.parametrize("route", ["register", "shared", "fft3d"])
def test_mixed_routes_agree_with_fp64(monkeypatch, route):
    """Mixed form through both fused routes: Delta n within 1e-5 of max|Delta n| of the FP64
    oracle, the bar the mixed form's chi is held to."""
    w, m, gs, J, ref = _reference(GRIDS[1])
    for k, v in ROUTES[route].items():
        monkeypatch.setenv(k, v)
    ctx = P.Context.from_workload(w, precision=1)
    import_ground_state(ctx, m, gs)
    _, dn, _ = ctx.response(1, J)
    r1 = oracle_dn_padded(m, ref["dn"])
    assert np.abs(dn - r1).max() < 1e-5 * np.abs(r1).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_two_pass_projection_matches_oracle(monkeypatch, precision):
    """beta and P_v rows projected in two passes (as when nproj + nocc exceeds one projection's
    128 rows), forced here with HP_PROJ_ROWS on the small cell: FP64 at 1e-8, mixed at 1e-5."""
    w, m, gs, J, ref = _reference(GRIDS[0])
    monkeypatch.setenv("HP_PROJ_ROWS", "4")
    kw = dict(cg_tol=1e-12, scf_tol=1e-11, conv_thr_chi=1e-11) if precision == 0 else {}
    ctx = P.Context.from_workload(w, precision=precision, **kw)
    import_ground_state(ctx, m, gs)
    _, dn, _ = ctx.response(1, J)
    r1 = oracle_dn_padded(m, ref["dn"])
    assert np.abs(dn - r1).max() < (1e-8 if precision == 0 else 1e-5) * np.abs(r1).max()
