"""Pins of the oracle's Loewdin ortho-atomic Hubbard projectors (Sec. 2.2, Eq. OAO_def) and of the
DFPT response built on them.

The orthogonalisation itself: the new orbitals are orthonormal, span the same manifold as the atomic
orbitals, are the orthonormal set closest to them (Loewdin's least-squares property, against
Gram-Schmidt and random nearby orthonormal sets), and leave an already orthonormal set unchanged.
The response: with ortho-atomic projectors chi_0 still equals the sum over states, chi the finite
differences of SCF occupations under lambda sum_m |phi~^J_m><phi~^J_m|, and the q-sum the explicit
supercell (whose ortho-atomic orbitals at the folded k points are those of the primitive cell at
the unfolded ones)."""

import numpy as np
import pytest

import workloads as W
from oracle import fd, groundstate as G, hubbard as HB, response as R, sos
from oracle.model import Model, lowdin_orthonormalize


def _rocksalt_phi():
    m = Model(W.medium_small(ecut=8.0, grid=(18, 18, 18), kmesh=(2, 1, 1), qmesh=(1, 1, 1)))
    return m, m.kdata(m.kpts[1])


def test_lowdin_orthonormal_and_same_span():
    m, kd = _rocksalt_phi()
    phi = kd.phi                                    # atomic (not orthogonalised) rows
    O = phi.conj() @ phi.T
    assert np.abs(O - np.diag(np.diag(O))).max() > 1e-2   # the metal d and ligand p orbitals overlap
    t = lowdin_orthonormalize(phi)
    assert np.abs(t.conj() @ t.T - np.eye(len(phi))).max() < 1e-12
    # same manifold: the projectors onto the span agree, P = phi^T O^-1 phi^*
    P_atomic = phi.T @ np.linalg.solve(O.T, phi.conj())
    P_ortho = t.T @ t.conj()
    assert np.abs(P_atomic - P_ortho).max() < 1e-11


def test_lowdin_is_the_closest_orthonormal_set():
    m, kd = _rocksalt_phi()
    phi = kd.phi
    t = lowdin_orthonormalize(phi)
    d_lowdin = np.linalg.norm(t - phi) ** 2
    # Gram-Schmidt in the given order (QR of the columns phi^T)
    q, r = np.linalg.qr(phi.T)
    q = q * np.sign(np.diag(r).real)[None, :]
    assert d_lowdin < np.linalg.norm(q.T - phi) ** 2
    # random orthonormal sets of the same span near the Loewdin one
    rng = np.random.default_rng(4)
    n = len(phi)
    for _ in range(5):
        a = 0.05 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        u = np.linalg.qr(np.eye(n) + a - a.conj().T)[0]      # close to the identity, unitary
        assert d_lowdin < np.linalg.norm(u.T @ t - phi) ** 2


def test_lowdin_leaves_orthonormal_rows_unchanged():
    rng = np.random.default_rng(5)
    q = np.linalg.qr(rng.standard_normal((300, 12)) + 1j * rng.standard_normal((300, 12)))[0].T
    assert np.abs(lowdin_orthonormalize(q) - q).max() < 1e-13


def _oao(w):
    return W.with_projectors(w, "ortho-atomic")


def test_oao_bare_response_equals_sum_over_states():
    m = Model(_oao(W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 1, 1), qmesh=(2, 1, 1))))
    gs = G.scf(m, tol=1e-12)
    for iq in range(len(m.qpts)):
        for J in m.hub_atoms:
            r = R.solve_column(m, gs, iq, J, hxc=False)
            ref = sos.bare_column(m, gs, iq, J)
            got = HB.trace_column(m, r["dn0"])
            assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def test_oao_response_equals_finite_differences():
    m = Model(_oao(W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 1, 1), qmesh=(1, 1, 1))))
    gs = G.scf(m, tol=1e-12)
    for J in m.hub_atoms:
        r = R.solve_column(m, gs, 0, J)
        chi0 = HB.trace_column(m, r["dn0"]).real
        chi = HB.trace_column(m, r["dn"]).real
        assert np.abs(chi0 - fd.fd_column(m, J, lam=5e-4, gs0=gs, bare=True)).max() < 1e-8 * np.abs(chi0).max()
        assert np.abs(chi - fd.fd_column(m, J, lam=5e-4, gs0=gs)).max() < 1e-8 * np.abs(chi).max()


@pytest.mark.slow
def test_oao_q_sum_equals_supercell_and_differs_from_atomic():
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 1, 1), qmesh=(2, 1, 1))

    def full(wl):
        m = Model(wl)
        gs = G.scf(m, tol=1e-12)
        c0, c = {}, {}
        for iq in range(len(m.qpts)):
            ctx = R.ResponseContext(m, gs, iq)
            for J in m.hub_atoms:
                res = R.solve_column(m, gs, iq, J, ctx=ctx)
                c0[(iq, J)] = HB.trace_column(m, res["dn0"])
                c[(iq, J)] = HB.trace_column(m, res["dn"])
        return HB.assemble_chi(m, c0).real, HB.assemble_chi(m, c).real

    chi0, chi = full(_oao(w))
    schi0, schi = full(_oao(W.supercell(w, (2, 1, 1))))
    assert np.abs(schi0 - chi0).max() < 1e-9 * np.abs(chi0).max()
    assert np.abs(schi - chi).max() < 1e-9 * np.abs(chi).max()
    a0, a = full(w)
    # the projector choice changes U (Sec. 2.2): ortho-atomic and atomic U differ
    U_oao = np.diag(HB.hubbard_matrix(chi0, chi))
    U_at = np.diag(HB.hubbard_matrix(a0, a))
    assert np.abs(U_oao - U_at).max() > 1e-3
