"""Pins of the oracle's symmetry reductions (oracle/symmetry.py; Sec. 2.4 "Symmetry", Sec. 3.2 and
the hp.x input table: find_atpert, docc_thr, dist_thr, skip_equivalence_q).

The pins rest on symmetries the model crystals have exactly:
- the rocksalt cell's four H sites (and its four L sites) are images of each other under the fcc
  translations (1/2, 1/2, 0) etc. of the cubic cell, which the Hamiltonian and any k mesh of the cubic
  cell respect: their ground-state occupations agree to the SCF tolerance, and the response column of
  one site is the column of another with the atoms relabelled, which the distance rule must find;
- time reversal of a real Hamiltonian: Delta_{-q} n = conj(Delta_q n), so the q-summed chi built
  from one q of each pair {q, -q} equals the one built from the whole mesh.
A site displaced off its lattice position loses the equivalence and must form a class of its own.
"""

import copy

import numpy as np
import pytest

import workloads as W
from oracle import groundstate as G
from oracle import hubbard as H
from oracle import response as R
from oracle import symmetry as S
from oracle.model import Model

TOL = dict(tol_cg=1e-12, scf_tol=1e-11, conv_chi=1e-12)


@pytest.fixture(scope="module")
def rocksalt():
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(1, 1, 1))
    m = Model(w)
    return m, G.scf(m, tol=1e-11)


def test_rocksalt_classes(rocksalt):
    m, gs = rocksalt
    tr = S.total_traces(m, gs)
    assert max(abs(tr[i] - tr[0]) for i in (1, 2, 3)) < 1e-8
    assert max(abs(tr[i] - tr[4]) for i in (5, 6, 7)) < 1e-8
    for mode in (1, 2):
        pert, rep = S.perturbed_atoms(m, gs, mode)
        assert pert == [0, 4]
        assert rep == {0: 0, 1: 0, 2: 0, 3: 0, 4: 4, 5: 4, 6: 4, 7: 4}
    pert, rep = S.perturbed_atoms(m, gs, 4)
    assert pert == list(range(8)) and all(rep[i] == i for i in range(8))
    pert, rep = S.perturbed_atoms(m, gs, 3)  # the same orbits under the 192 operations
    assert pert == [0, 4] and rep == {0: 0, 1: 0, 2: 0, 3: 0, 4: 4, 5: 4, 6: 4, 7: 4}
    # the antiferromagnetic start relaxes to zero moments (reading of the medium cell)
    assert set(S.orientations(m, gs).values()) == {0}


def test_displaced_site_is_its_own_class():
    w = copy.deepcopy(W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(1, 1, 1)))
    s, p = w["atoms"][1]
    w["atoms"][1] = (s, (p[0] + 0.03, p[1], p[2]))
    m = Model(w)
    gs = G.scf(m, tol=1e-10)
    pert, rep = S.perturbed_atoms(m, gs, 1)
    assert rep[1] == 1 and 1 in pert and 0 in pert
    pert2, _ = S.perturbed_atoms(m, gs, 2)
    assert pert2 == [0, 4]
    _, rep3 = S.perturbed_atoms(m, gs, 3)
    assert rep3[1] == 1


def test_rebuilt_columns_equal_computed_ones(rocksalt):
    """Columns of atoms 1 (H) and 5 (L) rebuilt from the representatives 0 and 4 by the distance rule
    equal the columns computed for them, for chi_0 and chi."""
    m, gs = rocksalt
    ctx = R.ResponseContext(m, gs, 0)
    tr = {}
    for J in (0, 1, 4, 5):
        r = R.solve_column(m, gs, 0, J, ctx=ctx, **TOL)
        tr[J] = (H.trace_column(m, r["dn0"]), H.trace_column(m, r["dn"]))
    pert, rep = S.perturbed_atoms(m, gs, 1)
    orient = S.orientations(m, gs)
    for k in (0, 1):
        rs = {J: S.realspace_column(m, [tr[J][k]]) for J in pert}
        full = S.reconstruct_columns(m, rs, rep, orient)
        for J in (1, 5):
            direct = S.realspace_column(m, [tr[J][k]])
            assert np.abs(full[J] - direct).max() < 1e-8 * np.abs(direct).max()
        with pytest.raises(ValueError):  # no distance within the threshold: no entry to take
            S.reconstruct_columns(m, rs, rep, orient, dist_thr=-1.0)


def test_rebuilt_columns_in_an_elongated_supercell():
    """On a 2 x 1 x 1 q mesh the supercell is no longer cubic: atoms at one distance from a site are
    not all equivalent, and the distance alone picks a wrong entry (1.5 % off here); the separation
    vector finds the translation image.  Gamma-only k (the L orbitals carry no occupation there), the
    H columns."""
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(1, 1, 1), qmesh=(2, 1, 1))
    m = Model(w)
    gs = G.scf(m, tol=1e-11)
    tr = {J: [H.trace_column(m, R.solve_column(m, gs, iq, J, **TOL)["dn"]) for iq in range(2)] for J in (0, 1)}
    _, rep = S.perturbed_atoms(m, gs, 1)
    orient = S.orientations(m, gs)
    rs = {0: S.realspace_column(m, tr[0]), 4: np.zeros(len(m.supercell_R()) * len(m.hub_atoms), dtype=complex)}
    direct = S.realspace_column(m, tr[1])
    got = S.reconstruct_columns(m, rs, rep, orient)[1]
    assert np.abs(got - direct).max() < 1e-8 * np.abs(direct).max()


def test_space_group_orders():
    """The conventional cubic cell of rocksalt has the 48 point operations of m-3m times the 4 fcc
    centring translations (192); the 2 x 1 x 1 supercell keeps the 16 that leave the x axis on +-x
    (times 4); the mirror cell has {1, m_xy, m_z, m_xy m_z}; a displaced H site leaves fewer."""
    m = Model(W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(2, 1, 1)))
    ops = S.space_group(m)
    assert len(ops) == 192
    assert len(S._supercell_ops(m, ops)) == 64
    for Wm, t, perm in ops:  # every operation keeps the metric and maps each species onto itself
        assert sorted(perm) == list(range(8)) and all(m.atom_species[perm[a]] == m.atom_species[a] for a in range(8))
    mm = Model(W.mirror())
    assert len(S.space_group(mm)) == 4
    w = copy.deepcopy(W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(1, 1, 1)))
    s, p = w["atoms"][1]
    w["atoms"][1] = (s, (p[0] + 0.03, p[1], p[2]))
    assert len(S.space_group(Model(w))) < 192


@pytest.fixture(scope="module")
def mirror():
    """The mirror cell's ground state and every (q, J) trace column of chi (q mesh 2 x 2 x 1)."""
    m = Model(W.mirror())
    gs = G.scf(m, tol=1e-11)
    cols = {}
    for iq in range(len(m.qpts)):
        ctx = R.ResponseContext(m, gs, iq)
        for J in m.hub_atoms:
            cols[(iq, J)] = H.trace_column(m, R.solve_column(m, gs, iq, J, ctx=ctx, **TOL)["dn"])
    return m, gs, cols


def test_mirror_images_by_operation(mirror):
    """find_atpert 3 on the mirror cell puts the two H sites in one orbit; the column of the second,
    rebuilt from the first through the mirror, equals its computed column on a 2 x 2 x 1 q mesh (the
    two are images under no translation, so the separation vectors do not match)."""
    m, gs, cols = mirror
    pert, rep = S.perturbed_atoms(m, gs, 3)
    assert pert == [0, 2] and rep == {0: 0, 1: 0, 2: 2}
    nq = len(m.qpts)
    tr = {J: [cols[(iq, J)] for iq in range(nq)] for J in (0, 1)}
    orient = S.orientations(m, gs)
    ops = S.space_group(m, orient)
    rs = {0: S.realspace_column(m, tr[0]), 2: np.zeros(len(m.supercell_R()) * len(m.hub_atoms), dtype=complex)}
    direct = S.realspace_column(m, tr[1])
    got = S.reconstruct_columns(m, rs, rep, orient, ops=ops)[1]
    assert np.abs(got - direct).max() < 1e-8 * np.abs(direct).max()


def test_star_of_q(mirror):
    """The (q, J) pairs of the mirror cell reduce to 7 of 12 under its four operations (the mirror
    takes (1/2, 0, 0) to (0, 1/2, 0) and one H site to the other); the 5 others, derived from the
    computed 7 with the lattice-shift phases, equal their computed trace columns, and chi follows.
    The rocksalt cell's 64 pairs on a 2 x 2 x 2 mesh reduce to 8 (one H and one L at the four classes
    of q)."""
    m, gs, cols = mirror
    ops = S.space_group(m, S.orientations(m, gs))
    irr = S.irreducible_pairs(m, ops)
    assert len(irr) == 7 and all(p in cols for p in irr)
    full = S.fill_pairs(m, {p: cols[p] for p in irr}, ops)
    assert set(full) == set(cols)
    for p in cols:
        if p not in irr:
            assert np.abs(full[p] - cols[p]).max() < 1e-9 * np.abs(cols[p]).max()
    assert np.abs(H.assemble_chi(m, full) - H.assemble_chi(m, cols)).max() < 1e-9 * np.abs(H.assemble_chi(m, cols)).max()
    mr = Model(W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(2, 2, 2)))
    assert S.irreducible_pairs(mr, S.space_group(mr)) == [(0, 0), (1, 0), (3, 0), (7, 0), (0, 4), (1, 4), (3, 4), (7, 4)]


def test_star_of_q_phases():
    """The lattice-shift phases at q = (1/3, 0, 0), where they are not +-1: in the Gamma-only rocksalt
    cell on a 3 x 1 x 1 q mesh the fcc translation (1/2, 1/2, 0) takes H site 1 onto site 0 of the next
    cell; the column of site 1 derived from that of site 0 equals its computed column (H entries; the L
    orbitals carry no occupation at Gamma), and so does the q = 2/3 column by time reversal."""
    m = Model(W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(1, 1, 1), qmesh=(3, 1, 1)))
    gs = G.scf(m, tol=1e-11)
    cols = {}
    for J in (0, 1):
        for iq in (1, 2):
            cols[(iq, J)] = H.trace_column(m, R.solve_column(m, gs, iq, J, **TOL)["dn"])
    ops = S.space_group(m, S.orientations(m, gs))
    full = S.fill_pairs(m, {(1, 0): cols[(1, 0)]}, ops)
    hsl = slice(0, 4)
    for p in ((1, 1), (2, 0), (2, 1)):
        assert np.abs(full[p][hsl] - cols[p][hsl]).max() < 1e-9 * np.abs(cols[p][hsl]).max()
    # the phases matter here: without them site 1's column is off
    assert np.abs(cols[(1, 1)][hsl] - cols[(1, 0)][[1, 0, 3, 2]]).max() > 1e-6 * np.abs(cols[(1, 1)]).max()


def test_columns_to_matrix_matches_q_sum():
    """chi from the real-space columns (lattice periodicity of the supercell) equals the q-summed
    assembly, on a 3 x 1 x 1 q mesh with random columns (index conventions only)."""
    m = Model(W.tiny_q(qmesh=(3, 1, 1)))
    rng = np.random.default_rng(7)
    nh = len(m.hub_atoms)
    cols = {(iq, J): rng.standard_normal(nh) + 1j * rng.standard_normal(nh)
            for iq in range(len(m.qpts)) for J in m.hub_atoms}
    ref = H.assemble_chi(m, cols)
    rs = {J: S.realspace_column(m, [cols[(iq, J)] for iq in range(len(m.qpts))]) for J in m.hub_atoms}
    assert np.abs(S.chi_from_columns(m, rs) - ref).max() < 1e-12


def test_time_reversal_pairs():
    m = Model(W.tiny_q(qmesh=(3, 1, 1)))
    irr, partner = S.irreducible_q(m)
    assert irr == [0, 1] and partner == [0, 1, 1]
    m4 = Model(W.tiny_q(qmesh=(2, 2, 1)))
    assert S.irreducible_q(m4)[0] == [0, 1, 2, 3]  # every q of a 2 x 2 mesh is its own -q


def test_time_reversal_response():
    """Delta_{-q} n = conj(Delta_q n) at q = (1/3, 0, 0) and (2/3, 0, 0), elementwise for dn0 and dn
    (complex entries on the second atom), and chi from the irreducible q with the conjugate pairs
    equals chi from the whole mesh."""
    m = Model(W.tiny_q(qmesh=(3, 1, 1)))
    gs = G.scf(m, tol=1e-11)
    cols, res = {}, {}
    for J in m.hub_atoms:
        for iq in range(3):
            res[(iq, J)] = R.solve_column(m, gs, iq, J, **TOL)
            cols[(iq, J)] = H.trace_column(m, res[(iq, J)]["dn"])
    J = m.hub_atoms[0]
    for key in ("dn0", "dn"):
        for s in res[(1, J)][key]:
            a, b = res[(1, J)][key][s], res[(2, J)][key][s]
            assert np.abs(b - a.conj()).max() < 1e-9 * np.abs(a).max()
    assert max(np.abs(res[(1, J)]["dn"][s].imag).max() for s in res[(1, J)]["dn"]) > 1e-6  # not trivially real
    _, partner = S.irreducible_q(m)
    red = {(iq, J): (cols[(iq, J)] if partner[iq] == iq else cols[(partner[iq], J)].conj())
           for iq in range(3) for J in m.hub_atoms}
    full, half = H.assemble_chi(m, cols), H.assemble_chi(m, red)
    assert np.abs(full - half).max() < 1e-9 * np.abs(full).max()
