"""Oracle post-processing: q-sum with phases, chi_0 and chi, Hubbard U and V.

Test infrastructure only (see the package docstring).

  chi_{(l,s),(l',s')} = (1/N_q) sum_q exp(i q.(R_l - R_l')) sum_sigma sum_m Delta^{s'}_q n^{s sigma}_mm
                                                      (Eqs. chi and occ_matrix_response_lp_1)
  U^I = (chi_0^-1 - chi^-1)_II,   V^IJ = (chi_0^-1 - chi^-1)_IJ           (Eqs. U_def, V_def)

with R_l the cells of the supercell that the q mesh images (index l = (l1 n2 + l2) n3 + l3) and
the spin sum of a nspin = 1 run taken as twice the per-spin trace.  Results in eV (1 Ha =
27.211386245988 eV).  Neighbours for V: every (l', s') whose minimum-image distance from (0, s) is
within d_min + dist_thr (dist_thr = 6e-4 bohr, Appendix B), d_min the shortest distance from s to
an atom of another Hubbard type class.
"""

from __future__ import annotations

import numpy as np

from .model import HA_TO_EV


def trace_column(model, dn):
    """{s: (nspin, m, m)} -> vector over Hubbard atoms of sum_sigma sum_m Delta n_mm."""
    f = 2.0 if model.nspin == 1 else 1.0
    return np.array([f * np.trace(dn[s], axis1=1, axis2=2).sum() for s in model.hub_atoms])


def assemble_chi(model, columns):
    """columns[(iq, J)] = trace vector over the primitive cell's Hubbard atoms.  Returns the complex
    supercell matrix (N_H N_q, N_H N_q), index (l, s) -> l * N_H + s."""
    nh = len(model.hub_atoms)
    R = model.supercell_R()
    nq = len(model.qpts)
    ncell = len(R)
    chi = np.zeros((ncell * nh, ncell * nh), dtype=complex)
    for jj, J in enumerate(model.hub_atoms):
        for iq, q in enumerate(model.qpts):
            col = columns[(iq, J)]
            for l in range(ncell):
                for lp in range(ncell):
                    ph = np.exp(2j * np.pi * np.dot(q, R[l] - R[lp]))
                    chi[l * nh:(l + 1) * nh, lp * nh + jj] += ph * col / nq
    return chi


def hubbard_matrix(chi0, chi):
    """(chi_0^-1 - chi^-1) in eV, from real FP64 matrices."""
    return (np.linalg.inv(chi0) - np.linalg.inv(chi)) * HA_TO_EV


def neighbours(model, s_index, dist_thr=6e-4):
    """Neighbours (l', s') of Hubbard atom s (index into hub_atoms) of a different species, at the
    shortest minimum-image distance within dist_thr, in the supercell of the q mesh."""
    R = model.supercell_R()
    nh = len(model.hub_atoms)
    n = np.array(model.qmesh, dtype=float)
    sc = model.cell * n[:, None]
    ia = model.hub_atoms[s_index]
    sp = model.atom_species[ia]
    dists = []
    for l in range(len(R)):
        for jj, ja in enumerate(model.hub_atoms):
            if model.atom_species[ja] == sp:
                continue
            d = (model.frac[ja] + R[l] - model.frac[ia]) / n
            d -= np.round(d)
            dists.append((float(np.linalg.norm(d @ sc)), l * nh + jj))
    if not dists:
        return []
    dmin = min(d for d, _ in dists)
    return sorted(j for d, j in dists if d <= dmin + dist_thr)


def neighbour_pairs(model, s_index, dist_thr=6e-4):
    """The neighbours of ``neighbours`` as (chi index, Hubbard index j, lattice vector R of the
    neighbour in primitive cells): atom j displaced by R sits at the shortest distance from atom s."""
    R = model.supercell_R()
    nh = len(model.hub_atoms)
    n = np.array(model.qmesh, dtype=float)
    ia = model.hub_atoms[s_index]
    out = []
    for jchi in neighbours(model, s_index, dist_thr):
        l, jj = divmod(jchi, nh)
        ja = model.hub_atoms[jj]
        d = (model.frac[ja] + R[l] - model.frac[ia]) / n
        w = np.round(d)
        out.append((jchi, jj, tuple(int(x) for x in (R[l] - w * n))))
    return out


def cycle_step(model_factory, U_in, pairs_in, solve):
    """One step of the self-consistent U/V cycle (Sec. 2.1 with Sec. 5.2's workflow): the ground
    state with the Hubbard potential of (U_in, pairs_in), every (q, J) response, chi_0 and chi,
    then U_out (per Hubbard atom) and the nearest-neighbour pairs with V_out.  ``model_factory``
    maps (U, pairs) to a Model; ``solve(model)`` returns (chi0, chi) assembled as assemble_chi does."""
    m = model_factory(U_in, pairs_in)
    chi0, chi = solve(m)
    hub = hubbard_matrix(chi0, chi)
    nh = len(m.hub_atoms)
    U_out = [float(hub[s, s]) for s in range(nh)]
    pairs_out = [(s, jj, Rv, float(hub[s, jchi])) for s in range(nh) for jchi, jj, Rv in neighbour_pairs(m, s)]
    return U_out, pairs_out, hub
