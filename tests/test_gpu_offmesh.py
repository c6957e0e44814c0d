"""k+q off the k mesh (q mesh 3x1x1 on a 2x2x2 k mesh): the CUDA path computes the occupied states
at k+q non-self-consistently with the ground-state potential, evaluates the projector and Hubbard
rows there, and must give the oracle's response columns (FP64, 1e-8 relative to max|Delta n|),
chi, U and V (FP64 1e-8; mixed form within 1 meV)."""

import numpy as np
import pytest

import workloads as W
from oracle import groundstate as G, hubbard as HB, response as R
from oracle.model import Model
from tests.bridge import import_ground_state, oracle_dn_padded

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")
MEV = 1e-3


@pytest.fixture(scope="module")
def offmesh():
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(3, 1, 1))
    m = Model(w)
    assert m.kq_map(0, 1) == (None, None)  # the case under test: k+q off the mesh
    gs = G.scf(m, tol=1e-12)
    cols, c0, c = {}, {}, {}
    for iq in range(len(m.qpts)):
        rctx = R.ResponseContext(m, gs, iq)
        for J in m.hub_atoms:
            res = R.solve_column(m, gs, iq, J, ctx=rctx, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
            cols[(iq, J)] = res
            c0[(iq, J)] = HB.trace_column(m, res["dn0"])
            c[(iq, J)] = HB.trace_column(m, res["dn"])
    chi0 = HB.assemble_chi(m, c0).real
    chi = HB.assemble_chi(m, c).real
    return w, m, gs, cols, chi0, chi, HB.hubbard_matrix(chi0, chi)


def test_offmesh_columns_fp64(offmesh):
    w, m, gs, cols, chi0_ref, chi_ref, hub_ref = offmesh
    ctx = P.Context.from_workload(w, cg_tol=1e-12, scf_tol=1e-11, conv_thr_chi=1e-11)
    import_ground_state(ctx, m, gs)
    for iq in range(len(m.qpts)):
        for J in m.hub_atoms:
            dn0, dn, _ = ctx.response(iq, J)
            r0 = oracle_dn_padded(m, cols[(iq, J)]["dn0"])
            r1 = oracle_dn_padded(m, cols[(iq, J)]["dn"])
            assert np.abs(dn0 - r0).max() < 1e-8 * np.abs(r0).max()
            assert np.abs(dn - r1).max() < 1e-8 * np.abs(r1).max()
    chi0, chi, hub = ctx.hubbard()
    assert np.abs(chi0 - chi0_ref).max() < 1e-8 * np.abs(chi0_ref).max()
    assert np.abs(chi - chi_ref).max() < 1e-8 * np.abs(chi_ref).max()
    assert np.abs(hub - hub_ref).max() < 1e-8 * np.abs(hub_ref).max()


def test_offmesh_mixed_within_1mev(offmesh):
    w, m, gs, cols, chi0_ref, chi_ref, hub_ref = offmesh
    ctx = P.Context.from_workload(w, precision=1)
    import_ground_state(ctx, m, gs)
    for iq in range(len(m.qpts)):
        for J in m.hub_atoms:
            ctx.response(iq, J)
    chi0, chi, hub = ctx.hubbard()
    assert np.abs(chi - chi_ref).max() < 1e-5 * np.abs(chi_ref).max()
    assert np.abs(hub - hub_ref).max() < MEV
