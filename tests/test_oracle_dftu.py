"""Pins of the oracle's Hubbard-corrected ground state (DFT+U+V, Sec. 2.1, Eqs. occ_matrix_0,
Edftu, Hub_pot_0) and of the DFPT response on top of it.

1. The Hubbard potential is the derivative of the corrective energy: for random states C and a
   random variation D, d E_{U+V}(C + e D)/de at e = 0 (central differences) equals
   (f/N_k) sum 2 Re <D|V_Hub|C>, for on-site U and inter-site V with lattice-vector phases.
2. The primitive cell with a k mesh and the explicit supercell at the folded k points give the same
   self-consistent DFT+U+V ground state (occupation matrices, on-site and inter-site), on a cell
   without inversion symmetry, so that the sign of the k.R phases is fixed.
3. U = V = 0 listed explicitly gives the plain ground state.
4. On a DFT+U+V ground state, chi_0 equals the sum over states of its Hamiltonian and chi equals
   finite differences of SCF occupations with the Hubbard potential held fixed (the response of
   the Hubbard potential is not part of the linear-response problem, Sec. 2.3)."""

import copy

import numpy as np

import workloads as W
from oracle import dftu, fd, groundstate as G, hubbard as HB, response as R, sos
from oracle.model import Model


def _cell(kmesh=(2, 1, 1)):
    """Two atoms carrying orbitals (H d at the origin, L p off-centre), low cutoff."""
    w = W.tiny_q(ecut=6.0, grid=(10, 10, 10), kmesh=kmesh, qmesh=(1, 1, 1))
    w["atoms"] = [(0, (0.0, 0.0, 0.0)), (1, (0.42, 0.37, 0.31))]
    return w


def _with_uv(w, U=(4.0, 2.5), V=0.8):
    """U on both atoms; V between the H atom and its three nearest L images (and the reverse)."""
    w = copy.deepcopy(w)
    w["hubbard_U"] = [(0, U[0]), (1, U[1])]
    pairs = []
    for R in ((0, 0, 0), (-1, 0, 0), (0, -1, 0)):
        pairs.append((0, 1, R, V))
        pairs.append((1, 0, tuple(-x for x in R), V))
    w["hubbard_V"] = pairs
    return w


def test_potential_is_the_energy_derivative():
    m = Model(_with_uv(_cell()))
    kds = [m.kdata(k) for k in m.kpts]
    rng = np.random.default_rng(1)
    C = [[rng.standard_normal((kd.npw, m.nocc)) + 1j * rng.standard_normal((kd.npw, m.nocc)) for kd in kds]]
    D = [[rng.standard_normal((kd.npw, m.nocc)) + 1j * rng.standard_normal((kd.npw, m.nocc)) for kd in kds]]
    occ = dftu.occupations(m, C, kds)
    f = 2.0 if m.nspin == 1 else 1.0
    grad = 0.0
    for ik, kd in enumerate(kds):
        Wk = dftu.w_matrix(m, kd, occ, 0)
        grad += f / len(kds) * 2.0 * np.real(np.sum(D[0][ik].conj() * dftu.apply(m, kd, Wk, C[0][ik])))
    h = 1e-4

    def E(e):
        Ce = [[C[0][ik] + e * D[0][ik] for ik in range(len(kds))]]
        return dftu.energy(m, dftu.occupations(m, Ce, kds))

    def rich(fn):  # Richardson-extrapolated central difference (E is quartic in e)
        d = lambda t: (fn(t) - fn(-t)) / (2 * t)
        return (4 * d(h / 2) - d(h)) / 3

    assert abs(rich(E) - grad) < 1e-9 * abs(grad)
    # the inter-site part alone is exercised too
    w2 = _with_uv(_cell(), U=(0.0, 0.0))
    m2 = Model(w2)
    occ2 = dftu.occupations(m2, C, kds)
    g2 = sum(f / len(kds) * 2.0 * np.real(np.sum(D[0][ik].conj() * dftu.apply(m2, kd, dftu.w_matrix(m2, kd, occ2, 0),
                                                                              C[0][ik]))) for ik, kd in enumerate(kds))
    E2 = lambda e: dftu.energy(m2, dftu.occupations(m2, [[C[0][ik] + e * D[0][ik] for ik in range(len(kds))]], kds))
    assert abs(rich(E2) - g2) < 1e-9 * abs(g2)
    assert abs(g2) > 1e-3 * abs(grad)


def _supercell_uv(w, n):
    sc = W.supercell(w, n)
    nat = len(w["atoms"])
    cells = [(l1, l2, l3) for l1 in range(n[0]) for l2 in range(n[1]) for l3 in range(n[2])]
    sc["hubbard_U"] = [(ci * nat + a, u) for ci in range(len(cells)) for a, u in w["hubbard_U"]]
    pairs = []
    for ci, l in enumerate(cells):
        for i, j, R, v in w["hubbard_V"]:
            t = [l[d] + R[d] for d in range(3)]
            lj = tuple(t[d] % n[d] for d in range(3))
            Rs = tuple(t[d] // n[d] for d in range(3))
            pairs.append((ci * nat + i, cells.index(lj) * nat + j, Rs, v))
    sc["hubbard_V"] = pairs
    return sc


def test_dftu_ground_state_equals_supercell():
    w = _with_uv(_cell())
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    sc = _supercell_uv(w, (2, 1, 1))
    ms = Model(sc)
    gss = G.scf(ms, tol=1e-12)
    on, pairs = gs.hub_occ
    on_s, pairs_s = gss.hub_occ
    for ci in range(2):
        for a in m.hub_atoms:
            assert np.abs(on_s[ci * m.nat + a] - on[a]).max() < 1e-9
        for p in range(len(pairs)):
            assert np.abs(pairs_s[ci * len(pairs) + p] - pairs[p]).max() < 1e-9
    # the correction matters: the occupations differ from the uncorrected ground state's
    plain = G.scf(Model(_cell()), tol=1e-12).occupations()
    assert max(np.abs(on[a] - plain[a]).max() for a in m.hub_atoms) > 1e-3


def test_zero_parameters_give_the_plain_ground_state():
    w = _with_uv(_cell(), U=(0.0, 0.0), V=0.0)
    gs = G.scf(Model(w), tol=1e-12)
    ref = G.scf(Model(_cell()), tol=1e-12)
    assert np.abs(gs.eps - ref.eps).max() < 1e-10


def test_response_on_dftu_ground_state_sos_and_fd():
    m = Model(_with_uv(_cell()))
    gs = G.scf(m, tol=1e-12)
    for J in m.hub_atoms[:1]:
        r = R.solve_column(m, gs, 0, J)
        chi0 = HB.trace_column(m, r["dn0"])
        assert np.abs(chi0 - sos.bare_column(m, gs, 0, J)).max() < 1e-10 * np.abs(chi0).max()
        chi = HB.trace_column(m, r["dn"]).real
        assert np.abs(chi0.real - fd.fd_column(m, J, lam=5e-4, gs0=gs, bare=True)).max() < 1e-8 * np.abs(chi0).max()
        assert np.abs(chi - fd.fd_column(m, J, lam=5e-4, gs0=gs)).max() < 1e-8 * np.abs(chi).max()
