"""CUDA path against the oracle, element by element, on identical seeded inputs (FP64).

Tolerances: the operator (H psi) is compared at 1e-11 relative to its largest element (round-off
of two FP64 FFT routes); response matrices and U/V at 1e-8 relative to max|chi| (the bar the FP64
path is held to), with both sides converged to 1e-11 or tighter."""

import numpy as np
import pytest

import workloads as W
from oracle import groundstate as G, hubbard as HB, response as R
from oracle.hamiltonian import apply_h
from oracle.model import Model
from tests.bridge import import_ground_state, oracle_dn_padded, order_map

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")


def _ctx(w, **kw):
    kw.setdefault("cg_tol", 1e-12)
    kw.setdefault("scf_tol", 1e-11)
    kw.setdefault("conv_thr_chi", 1e-11)
    return P.Context.from_workload(w, **kw)


@pytest.fixture(scope="module")
def tiny_low():
    w = W.tiny_lowcut(ecut=10.0, grid=(12, 12, 12))
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    ctx = _ctx(w)
    import_ground_state(ctx, m, gs)
    return w, m, gs, ctx


def test_sizes_match_oracle(tiny_low):
    w, m, gs, ctx = tiny_low
    s = ctx.query_sizes()
    assert s["grid"] == m.grid
    assert s["nk"] == len(m.kpts) and s["nq"] == len(m.qpts)
    for ik in range(len(m.kpts)):
        assert len(ctx.sphere(ik)) == m.kdata(m.kpts[ik]).npw
    atoms, mdim = ctx.hubbard_atoms()
    assert list(atoms) == m.hub_atoms


@pytest.mark.parametrize("ik", [0, 3, 7])
def test_apply_h_matches_oracle(tiny_low, ik):
    w, m, gs, ctx = tiny_low
    perm, kd = order_map(ctx, m, ik)
    X = W.random_coefficients(100 + ik, (5, kd.npw))            # rows in the library's order
    Xo = np.zeros_like(X)
    Xo[:, perm] = X
    ref = apply_h(m, kd, gs.vr(0), Xo.T).T[:, perm]
    got = ctx.apply_h(ik, 0, X)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_apply_h_full_tiny_grid():
    """Full config-0 grid (20^3) and sphere (751-804 plane waves), several tiles and a ragged tail."""
    w = W.tiny()
    m = Model(w)
    rng = np.random.default_rng(5)
    vhxc = rng.standard_normal((1, m.nr)) * 0.3
    rho = np.abs(rng.standard_normal((1, m.nr))) * 0.05
    ctx = _ctx(w)
    no = m.nocc
    psi = [[np.linalg.qr(W.random_coefficients(7 + k, (m.kdata(m.kpts[k]).npw, no)))[0] for k in range(len(m.kpts))]]
    ctx.set_ground_state(1, m.nelec, vhxc, rho, np.zeros((1, len(m.kpts), no)), psi)
    vr = m.vloc_r() + vhxc[0]
    for ik in (0, 5):
        perm, kd = order_map(ctx, m, ik)
        X = W.random_coefficients(200 + ik, (37, kd.npw))
        Xo = np.zeros_like(X)
        Xo[:, perm] = X
        ref = apply_h(m, kd, vr, Xo.T).T[:, perm]
        got = ctx.apply_h(ik, 0, X)
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_response_matches_oracle_tiny_low(tiny_low):
    w, m, gs, ctx = tiny_low
    J = m.hub_atoms[0]
    ref = R.solve_column(m, gs, 0, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
    dn0, dn, info = ctx.response(0, J)
    r0 = oracle_dn_padded(m, ref["dn0"])
    r1 = oracle_dn_padded(m, ref["dn"])
    assert np.abs(dn0 - r0).max() < 1e-8 * np.abs(r0).max()
    assert np.abs(dn - r1).max() < 1e-8 * np.abs(r1).max()
    assert info["iterations"] > 2 and info["hpsi"] > 0


def test_hubbard_matrix_tiny_q():
    """Two Hubbard atoms, q mesh 2x1x1: every (q, J) column, chi_0, chi and U/V."""
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1))
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    ctx = _ctx(w)
    import_ground_state(ctx, m, gs)
    c0, c = {}, {}
    for iq in range(len(m.qpts)):
        rctx = R.ResponseContext(m, gs, iq)
        for J in m.hub_atoms:
            res = R.solve_column(m, gs, iq, J, ctx=rctx, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
            c0[(iq, J)] = HB.trace_column(m, res["dn0"])
            c[(iq, J)] = HB.trace_column(m, res["dn"])
            ctx.response(iq, J)
    chi0_ref = HB.assemble_chi(m, c0).real
    chi_ref = HB.assemble_chi(m, c).real
    hub_ref = HB.hubbard_matrix(chi0_ref, chi_ref)
    r = ctx.hubbard_parameters()
    chi0, chi, hub = r["chi0"], r["chi"], r["hub"]
    assert np.abs(chi0 - chi0_ref).max() < 1e-8 * np.abs(chi0_ref).max()
    assert np.abs(chi - chi_ref).max() < 1e-8 * np.abs(chi_ref).max()
    assert np.abs(hub - hub_ref).max() < 1e-8 * np.abs(hub_ref).max()
    # U per Hubbard atom and the nearest-neighbour V list (reading c17), against the oracle's shell
    nh = len(m.hub_atoms)
    assert np.abs(r["U"] - np.diag(hub_ref)[:nh]).max() < 1e-8 * np.abs(hub_ref).max()
    expect = [(s, j) for s in range(nh) for j in HB.neighbours(m, s)]
    assert [(s, j) for s, j, _, _ in r["V"]] == expect
    for s, j, dist, v in r["V"]:
        assert abs(v - hub_ref[s, j]) < 1e-8 * np.abs(hub_ref).max()
        assert 0 < dist < 8.0


def test_response_spin_polarised():
    """nspin = 2 rocksalt cell (8 atoms, 8 Hubbard atoms, 20 bands per spin), q = 0 and q != 0."""
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 1, 1), qmesh=(2, 1, 1))
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    ctx = _ctx(w)
    import_ground_state(ctx, m, gs)
    for iq, J in ((0, m.hub_atoms[0]), (1, m.hub_atoms[5])):
        ref = R.solve_column(m, gs, iq, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
        dn0, dn, info = ctx.response(iq, J)
        r0 = oracle_dn_padded(m, ref["dn0"])
        r1 = oracle_dn_padded(m, ref["dn"])
        assert np.abs(dn0 - r0).max() < 1e-8 * np.abs(r0).max()
        assert np.abs(dn - r1).max() < 1e-8 * np.abs(r1).max()


def test_errors_are_reported_not_raised_on_device():
    w = W.tiny_lowcut(ecut=6.0, grid=(10, 10, 10))
    ctx = _ctx(w)
    with pytest.raises(P.HPError) as e:
        ctx.response(0, 0)
    assert e.value.code == 3  # HP_ESTATE: no ground state
    with pytest.raises(P.HPError) as e:
        ctx.hubbard()
    assert e.value.code == 3
