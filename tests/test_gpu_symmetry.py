"""Symmetry reductions on the GPU (hp_perturbed_atoms, hp_irreducible_q and the reconstruction in
hp_hubbard; Sec. 2.4 "Symmetry", Sec. 3.2): the classes (find_atpert 1 to 4) and occupations against
the oracle, and chi from the reduced set of responses against chi from every response.

The rocksalt cell's four H (and four L) sites are images of each other under fcc translations of the
cubic cell, so their columns are relabellings of one another (pinned in the oracle tests); a 3 x 1 x 1
q mesh pairs q = 1/3 with -q = 2/3, whose response is the conjugate one.
"""

import numpy as np
import pytest

import workloads as W
from oracle import groundstate as G
from oracle import symmetry as S
from oracle.model import Model
from tests.bridge import import_ground_state

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")


def _chi(ctx, atoms, qs):
    for J in atoms:
        for iq in qs:
            ctx.response(iq, int(J))
    return ctx.hubbard()


def test_classes_and_traces_match_oracle():
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(1, 1, 1))
    m = Model(w)
    gs = G.scf(m, tol=1e-11)
    ctx = P.Context.from_workload(w)
    import_ground_state(ctx, m, gs)
    ref = S.spin_traces(m, gs)
    for mode in (1, 2, 3, 4):
        atoms, rep, tr = ctx.perturbed_atoms(mode)
        ref_atoms, ref_rep = S.perturbed_atoms(m, gs, mode)
        assert atoms == ref_atoms
        assert rep == [ref_rep[a] for a in m.hub_atoms]
    for i, a in enumerate(m.hub_atoms):
        assert np.abs(tr[i, :m.nspin] - np.array(ref[a])).max() < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_reduced_atoms_give_the_full_chi(precision):
    """find_atpert = 1 on the rocksalt cell (q mesh 2 x 1 x 1): 2 of the 8 atoms perturbed, the other
    columns rebuilt; chi_0, chi and U/V equal those from all 8 atoms (FP64: 1e-9 relative; mixed form:
    1e-5 relative, the mixed form's bar, and 0.1 meV: the rebuilt columns copy the representative's, the
    computed ones carry their own FP32 noise)."""
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(2, 1, 1))
    full = P.Context.from_workload(w, precision=precision)
    full.ground_state(w["nelec"], w["nspin"], w.get("moments"))
    atoms, _ = full.hubbard_atoms()
    c0, c, hub = _chi(full, atoms, range(2))
    red = P.Context.from_workload(w, precision=precision)
    red.ground_state(w["nelec"], w["nspin"], w.get("moments"))
    pert, rep, _ = red.perturbed_atoms(1)
    assert pert == [0, 4] and rep == [0, 0, 0, 0, 4, 4, 4, 4]
    r0, r, rhub = _chi(red, pert, range(2))
    rel = 1e-9 if precision == 0 else 1e-5
    assert np.abs(r0 - c0).max() < rel * np.abs(c0).max()
    assert np.abs(r - c).max() < rel * np.abs(c).max()
    assert np.abs(rhub - hub).max() < (1e-6 if precision == 0 else 1e-4)
    # without classes the missing columns are an error
    red.perturbed_atoms(4)
    with pytest.raises(P.HPError):
        red.hubbard()


def test_space_group_orbits_give_the_full_chi():
    """find_atpert 3 on the mirror cell (its two H sites are images under the mirror x <-> y and under
    no translation): the library's orbits equal the oracle's, and chi with the second H column rebuilt
    through the mirror equals chi from both columns (FP64, q mesh 2 x 2 x 1)."""
    w = W.mirror()
    m = Model(w)
    gs = G.scf(m, tol=1e-11)
    ref_pert, ref_rep = S.perturbed_atoms(m, gs, 3)
    full = P.Context.from_workload(w)
    import_ground_state(full, m, gs)
    atoms, _ = full.hubbard_atoms()
    c0, c, hub = _chi(full, atoms, range(len(m.qpts)))
    red = P.Context.from_workload(w)
    import_ground_state(red, m, gs)
    pert, rep, _ = red.perturbed_atoms(3)
    assert pert == ref_pert == [0, 2] and rep == [ref_rep[a] for a in m.hub_atoms]
    r0, r, rhub = _chi(red, pert, range(len(m.qpts)))
    assert np.abs(r0 - c0).max() < 1e-9 * np.abs(c0).max()
    assert np.abs(r - c).max() < 1e-9 * np.abs(c).max()
    assert np.abs(rhub - hub).max() < 1e-6


@pytest.mark.parametrize("cell", ["mirror", "rocksalt"])
def test_star_of_q_gives_the_full_chi(cell):
    """find_atpert 3 with the star of q: only the irreducible (q, J) pairs computed (the oracle's list:
    7 of 12 in the mirror cell, 8 of 64 in the rocksalt cell on a 2 x 2 x 2 q mesh), the other trace
    columns derived with the lattice-shift phases; chi_0, chi and U/V equal those from every pair
    (FP64, 1e-9 relative)."""
    if cell == "mirror":
        w = W.mirror()
    else:
        w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 2, 2), qmesh=(2, 2, 2))
    m = Model(w)
    gs = G.scf(m, tol=1e-11)
    full = P.Context.from_workload(w)
    import_ground_state(full, m, gs)
    atoms, _ = full.hubbard_atoms()
    c0, c, hub = _chi(full, atoms, range(len(m.qpts)))
    red = P.Context.from_workload(w)
    import_ground_state(red, m, gs)
    red.perturbed_atoms(3)
    pairs = red.irreducible_pairs()
    assert pairs == S.irreducible_pairs(m, S.space_group(m, S.orientations(m, gs)), atoms=S.perturbed_atoms(m, gs, 3)[0])
    for iq, J in pairs:
        red.response(iq, J)
    r0, r, rhub = red.hubbard()
    assert np.abs(r0 - c0).max() < 1e-9 * np.abs(c0).max()
    assert np.abs(r - c).max() < 1e-9 * np.abs(c).max()
    assert np.abs(rhub - hub).max() < 1e-6


def test_time_reversal_gives_the_full_chi():
    w = W.tiny_q(qmesh=(3, 1, 1))
    full = P.Context.from_workload(w)
    full.ground_state(w["nelec"], w["nspin"])
    atoms, _ = full.hubbard_atoms()
    c0, c, hub = _chi(full, atoms, range(3))
    half = P.Context.from_workload(w)
    half.ground_state(w["nelec"], w["nspin"])
    irr, partner = half.irreducible_q()
    assert irr == [0, 1] and partner == [0, 1, 1]
    h0, h, hhub = _chi(half, atoms, irr)
    assert np.abs(h0 - c0).max() < 1e-9 * np.abs(c0).max()
    assert np.abs(h - c).max() < 1e-9 * np.abs(c).max()
    assert np.abs(hhub - hub).max() < 1e-6
