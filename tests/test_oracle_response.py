"""Method-level pins of the oracle's DFPT response (Sec. 2.3): sum over states, finite differences
of SCF occupations, the q-sum against an explicit supercell, symmetries and invariances."""

import copy

import numpy as np
import pytest

import workloads as W
from oracle import fd, groundstate as G, hubbard as HB, response as R, sos
from oracle.hamiltonian import dense_h
from oracle.model import Model


@pytest.fixture(scope="module")
def tiny_low():
    m = Model(W.tiny_lowcut(ecut=10.0, grid=(12, 12, 12)))
    gs = G.scf(m, tol=1e-12)
    J = m.hub_atoms[0]
    r = R.solve_column(m, gs, 0, J)
    return m, gs, J, r


def test_ground_state_insulating_and_d_filled(tiny_low):
    m, gs, _, _ = tiny_low
    assert gs.gap() > 0.1
    n = gs.occupations()[0]
    assert 4.0 < np.trace(n[0]) < 5.0                      # d shell nearly full per spin
    assert np.allclose(n[0], n[0].T, atol=1e-12)


def test_bare_response_equals_sum_over_states(tiny_low):
    m, gs, J, r = tiny_low
    ref = sos.bare_column(m, gs, 0, J)
    got = HB.trace_column(m, r["dn0"])
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(ref.imag).max() < 1e-12


def test_response_equals_finite_differences(tiny_low):
    m, gs, J, r = tiny_low
    chi0_fd = fd.fd_column(m, J, gs0=gs, bare=True)
    chi_fd = fd.fd_column(m, J, gs0=gs)
    chi0 = HB.trace_column(m, r["dn0"]).real
    chi = HB.trace_column(m, r["dn"]).real
    assert np.abs(chi0 - chi0_fd).max() < 1e-8 * np.abs(chi0).max()
    assert np.abs(chi - chi_fd).max() < 1e-8 * np.abs(chi).max()
    # screening: the self-consistent response is smaller than the bare one, both negative
    assert chi0[0] < chi[0] < 0


def test_alpha_and_preconditioner_independence(tiny_low):
    m, gs, J, r = tiny_low
    ctx = R.ResponseContext(m, gs, 0)
    ctx.alpha *= 3.0
    r2 = R.solve_column(m, gs, 0, J, ctx=ctx)
    for s in m.hub_atoms:
        assert np.abs(r2["dn"][s] - r["dn"][s]).max() < 1e-9


def test_hxc_switched_off_gives_zero_u(tiny_low):
    m, gs, J, r = tiny_low
    r0 = R.solve_column(m, gs, 0, J, hxc=False)
    c0 = HB.trace_column(m, r0["dn0"]).real
    c = HB.trace_column(m, r0["dn"]).real
    U = HB.hubbard_matrix(np.array([[c0[0]]]), np.array([[c[0]]]))
    assert abs(U[0, 0]) < 1e-12
    chi0 = HB.trace_column(m, r["dn0"]).real
    chi = HB.trace_column(m, r["dn"]).real
    U = HB.hubbard_matrix(np.array([[chi0[0]]]), np.array([[chi[0]]]))
    assert 1.0 < U[0, 0] < 20.0                                 # a few eV, as for a 3d metal


def test_rigid_shift_invariance(tiny_low):
    """Translating every atom by a vector of the real-space grid leaves chi unchanged (the
    structure-factor phases exp(-iG.tau) and the grid quadrature move together).  A shift that is
    not a grid vector changes the grid sampling of the non-linear xc potential slightly (the
    egg-box effect of a real-space grid, 1e-5 relative here), so it is not used as a pin."""
    m, gs, J, r = tiny_low
    w = copy.deepcopy(m.w)
    shift = [3.0 / m.grid[0], 5.0 / m.grid[1], 7.0 / m.grid[2]]
    w["atoms"] = [(s, tuple((x + d) % 1.0 for x, d in zip(p, shift))) for s, p in w["atoms"]]
    m2 = Model(w)
    gs2 = G.scf(m2, tol=1e-12)
    r2 = R.solve_column(m2, gs2, 0, m2.hub_atoms[0])
    a = HB.trace_column(m, r["dn"]).real
    b = HB.trace_column(m2, r2["dn"]).real
    assert np.abs(a - b).max() < 1e-8 * np.abs(a).max()


@pytest.fixture(scope="module")
def q_pair():
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1))

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
        return m, gs, HB.assemble_chi(m, c0), HB.assemble_chi(m, c)

    return full(w), full(W.supercell(w, (2, 1, 1)))


def test_q_sum_equals_supercell(q_pair):
    (m, _, chi0, chi), (_, _, schi0, schi) = q_pair
    assert np.abs(schi0 - chi0).max() < 1e-9 * np.abs(chi0).max()
    assert np.abs(schi - chi).max() < 1e-9 * np.abs(chi).max()


def test_chi_symmetric_real_and_negative_definite(q_pair):
    (m, _, chi0, chi), _ = q_pair
    for X in (chi0, chi):
        assert np.abs(X.imag).max() < 1e-10 * np.abs(X).max()
        assert np.abs(X - X.T).max() < 1e-9 * np.abs(X).max()
    assert np.linalg.eigvalsh(chi0.real).max() < 0
    assert np.linalg.eigvalsh(chi.real).max() < 0


def test_minus_q_is_complex_conjugate(q_pair):
    """With time reversal, Delta_{-q} n = conj(Delta_q n).  On the 2x1x1 mesh -q = q + G, so the
    q = b1/2 column must itself be real up to solver tolerance, and the q = 0 column real too."""
    (m, gs, _, _), _ = q_pair
    for iq in range(len(m.qpts)):
        res = R.solve_column(m, gs, iq, m.hub_atoms[0])
        col = HB.trace_column(m, res["dn"])
        assert np.abs(col.imag).max() < 1e-9 * np.abs(col).max()


def test_neighbours_and_v_sign(q_pair):
    (m, _, chi0, chi), _ = q_pair
    UV = HB.hubbard_matrix(chi0.real, chi.real)
    nb = HB.neighbours(m, 0)
    assert len(nb) >= 1
    for j in nb:
        assert UV[0, j] > 0.0        # inter-site V positive between the metal and its ligand


@pytest.mark.slow
def test_spin_polarised_sos_and_symmetry():
    """nspin = 2 rocksalt cell (AFM start): bare response = sum over states, spin channels summed."""
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(1, 1, 1), qmesh=(1, 1, 1))
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    J = m.hub_atoms[0]
    r = R.solve_column(m, gs, 0, J)
    ref = sos.bare_column(m, gs, 0, J)
    got = HB.trace_column(m, r["dn0"])
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()
    # the four H sites of the rocksalt cell are equivalent: on-site responses equal
    cols = {}
    for Jx in m.hub_atoms[:4]:
        cols[Jx] = HB.trace_column(m, R.solve_column(m, gs, 0, Jx)["dn"]).real
    diag = [cols[Jx][i] for i, Jx in enumerate(m.hub_atoms[:4])]
    assert np.ptp(diag) < 1e-8 * abs(diag[0])
    # chi_IJ = chi_JI
    for a in range(4):
        for b in range(4):
            assert abs(cols[m.hub_atoms[b]][a] - cols[m.hub_atoms[a]][b]) < 1e-8 * abs(diag[0])


def test_off_mesh_branch_equals_mapped_states(monkeypatch):
    """The non-self-consistent k+q branch (used when k+q is off the k mesh) forced on an on-mesh q
    gives the same response column as the states mapped from k' = k+q - G0: same occupied
    energies, and Delta n equal up to the gauge of the states (traces and the full matrices, which
    do not depend on it)."""
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1))
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    J = m.hub_atoms[0]
    mapped = R.solve_column(m, gs, 1, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
    e_mapped = [G.kq_states(m, gs, ik, 1)[2] for ik in range(len(m.kpts))]
    monkeypatch.setattr(Model, "kq_map", lambda self, ik, iq: (None, None))
    e_nscf = [G.kq_states(m, gs, ik, 1)[2] for ik in range(len(m.kpts))]
    nscf = R.solve_column(m, gs, 1, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
    assert max(np.abs(a - b).max() for a, b in zip(e_mapped, e_nscf)) < 1e-9
    for key in ("dn0", "dn"):
        a, b = mapped[key], nscf[key]
        assert set(a) == set(b)
        scale = max(np.abs(np.asarray(v)).max() for v in a.values())
        for atom in a:
            assert np.abs(np.asarray(a[atom]) - np.asarray(b[atom])).max() < 1e-8 * scale


def test_neighbours_rocksalt_shell_of_six():
    """Reading c17: in the rocksalt cell every metal (H) has six ligand (L) neighbours tied at a/2
    and every ligand six metals; on the 2x2x2 q mesh the six are distinct atoms of the supercell
    (+-x, +-y, +-z).  A shell rule that kept one of a tied set, or took the wrong species, fails."""
    m = Model(W.medium())
    a = 8.4
    R = m.supercell_R()
    nh = len(m.hub_atoms)
    n = np.array(m.qmesh, dtype=float)
    for si, ia in enumerate(m.hub_atoms):
        nb = HB.neighbours(m, si)
        assert len(nb) == 6 and len(set(nb)) == 6
        for j in nb:
            l, sj = divmod(j, nh)
            ja = m.hub_atoms[sj]
            assert m.atom_species[ja] != m.atom_species[ia]
            d = (m.frac[ja] + R[l] - m.frac[ia]) / n
            d -= np.round(d)
            assert abs(np.linalg.norm(d * n * a) - a / 2) < 1e-12


def test_sternheimer_operator_equals_dense_matrix():
    """The Sternheimer operator through the FFT route equals the dense aliased H plus alpha Cq Cq^H
    minus the shift, on random vectors at a k+q point of the q = (1/2, 0, 0) column."""
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1))
    m = Model(w)
    rng = np.random.default_rng(3)
    vr = m.vloc_r() + 0.2 * rng.standard_normal(m.nr)
    kdq = m.kdata(m.kpts[3] + m.qpts[1])
    Cq = np.linalg.qr(rng.standard_normal((kdq.npw, 5)) + 1j * rng.standard_normal((kdq.npw, 5)))[0]
    X = rng.standard_normal((kdq.npw, 4)) + 1j * rng.standard_normal((kdq.npw, 4))
    eps = np.array([-0.7, -0.5, -0.2, 0.1])
    got = R.sternheimer_operator(m, kdq, vr, Cq, 1.3, eps, X)
    Hd = dense_h(m, kdq, vr) + 1.3 * (Cq @ Cq.conj().T)
    ref = np.stack([(Hd - e * np.eye(kdq.npw)) @ X[:, j] for j, e in enumerate(eps)], axis=1)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
