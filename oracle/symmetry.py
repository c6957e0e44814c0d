"""Oracle symmetry reductions of the response calculation: which Hubbard atoms are perturbed, how the
columns of the atoms that are not perturbed are rebuilt, and which q points are computed (Sec. 2.4
"Symmetry"; Sec. 3.2, the linear-response step and its post-processing; the hp.x input table of
Appendix B: find_atpert, docc_thr, dist_thr, skip_equivalence_q).

Test infrastructure only (see the package docstring).

Perturbed atoms (find_atpert):
  1  Hubbard atoms of one species whose ground-state occupations Tr n^I (summed over spin, Eq.
     occ_matrix_0) differ by less than docc_thr (5e-5) form a class, whatever the sign of their
     moments; one atom per class, the first in atom order, is perturbed.
  2  one atom per species.
  3  the orbits of the Hubbard atoms under the crystal's space group (below); one atom per orbit, the
     first in atom order.
  4  every Hubbard atom.

Space group: the operations x -> W x + t on fractional coordinates, W an integer matrix with entries
in {-1, 0, 1} and determinant +-1 that keeps the lattice metric (W^T G W = G, G = A A^T with the
lattice vectors as the rows of A), t such that every atom goes onto an atom of its species (within
1e-5 in fractional coordinates), and the spin orientations of the Hubbard atoms kept up to one global
sign.  For find_atpert 3 the columns are rebuilt with the operations themselves: an operation g that
takes J' (cell 0) to J in cell L_J gives chi_{a,(0,J)} = chi_{g^-1(a + L_J),(0,J')}, used when g keeps
the q-mesh supercell's lattice (W diag(n) = diag(n) M with M integer); the atom of g^-1(a + L_J) and its
cell follow from its position.

Column reconstruction (post-processing): the real-space response column of a Hubbard atom J that was
not perturbed, chi_{(l,s),(0,J)} = (1/N_q) sum_q exp(i q.R_l) Delta^J_q n^s (Eqs. chi and
occ_matrix_response_lp_1), is taken from its class representative J': the entry for (l, s) is the
entry (l', s') of J' with the species of s and the spin orientation of s relative to J whose
separation from J' matches that of (l, s) from J within dist_thr (6e-4 bohr): first as a vector
modulo the supercell of the q mesh (exact for atoms that are images under a lattice translation,
whatever the shape of the supercell), else, where no atom matches the vector, as the minimum-image
distance.  The orientation of an atom is the sign of Tr n^up - Tr n^down where that difference
exceeds docc_thr, else 0.  The first matching (l', s') in index order is taken.  The full matrix then
follows from the lattice periodicity of the supercell: chi_{(l,s),(l'',J)} = chi_{(l - l'' mod n,
s),(0,J)}.

Time reversal (the +-q of the small group of q): for a ground state with real potentials and real
Hubbard orbitals the response to exp(-i q.R) is the complex conjugate of the response to exp(i q.R),
Delta_{-q} n = conj(Delta_q n); of each pair {q, -q + G} of the q mesh the first in mesh order is
computed.

Star of q (with the space group): an operation of the q-mesh supercell relates the trace columns of
chi at q and q' = W^-T q (below), so that only one (q, J) pair of each orbit is computed.
"""

from __future__ import annotations

import numpy as np


def spin_traces(model, gs):
    """{atom: [Tr n^{I sigma} for sigma]} of the ground state (nspin = 1: one channel)."""
    return {ia: [float(np.trace(n[s]).real) for s in range(n.shape[0])] for ia, n in gs.occupations().items()}


def total_traces(model, gs):
    """{atom: Tr n^I summed over spin (twice the channel for nspin = 1)}."""
    f = 2.0 if model.nspin == 1 else 1.0
    return {ia: f * sum(t) for ia, t in spin_traces(model, gs).items()}


def space_group(model, orient=None, tol=1e-5):
    """[(W, t, perm)]: the crystal's operations x -> W x + t (fractional coordinates, column vectors)
    and the atom each atom goes to; with orient ({Hubbard atom: +1/-1/0}) only the operations that keep
    the orientations up to one global sign."""
    import itertools

    A = np.array(model.cell, dtype=float)
    G = A @ A.T
    frac = np.array(model.frac, dtype=float)
    spec = list(model.atom_species)
    nat = len(frac)
    ops = []
    for entries in itertools.product((-1, 0, 1), repeat=9):
        Wm = np.array(entries, dtype=float).reshape(3, 3)
        if abs(abs(np.linalg.det(Wm)) - 1.0) > 1e-9:
            continue
        if np.abs(Wm.T @ G @ Wm - G).max() > 1e-8 * np.abs(G).max():
            continue
        y0 = Wm @ frac[0]
        for j in range(nat):
            if spec[j] != spec[0]:
                continue
            t = frac[j] - y0
            perm = []
            for a in range(nat):
                y = Wm @ frac[a] + t
                hit = [b for b in range(nat) if spec[b] == spec[a]
                       and np.abs((y - frac[b]) - np.round(y - frac[b])).max() < tol]
                if len(hit) != 1:
                    break
                perm.append(hit[0])
            if len(perm) != nat or len(set(perm)) != nat:
                continue
            if orient is not None:
                if not any(all(orient[perm[a]] == sg * orient[a] for a in model.hub_atoms) for sg in (1, -1)):
                    continue
            ops.append((Wm.astype(int), t - np.floor(t), perm))
    return ops


def perturbed_atoms(model, gs, find_atpert=1, docc_thr=5e-5):
    """(atoms to perturb in atom order, {Hubbard atom: its class representative})."""
    if find_atpert not in (1, 2, 3, 4):
        raise ValueError("find_atpert must be 1, 2, 3 or 4")
    if find_atpert == 3:
        ops = space_group(model, orientations(model, gs, docc_thr))
        rep = {}
        for ia in model.hub_atoms:  # the first atom of the orbit (the identity is among the operations)
            rep[ia] = min(perm[ia] for _, _, perm in ops)
        return [ia for ia in model.hub_atoms if rep[ia] == ia], rep
    tr = total_traces(model, gs)
    rep = {}
    for ia in model.hub_atoms:
        sp = model.atom_species[ia]
        r = ia
        for ja in model.hub_atoms:
            if ja >= ia:
                break
            if rep[ja] != ja or model.atom_species[ja] != sp:
                continue
            if find_atpert == 4:
                continue
            if find_atpert == 2 or (find_atpert == 1 and abs(tr[ja] - tr[ia]) < docc_thr):
                r = ja
                break
        rep[ia] = r
    return [ia for ia in model.hub_atoms if rep[ia] == ia], rep


def orientations(model, gs, docc_thr=5e-5):
    """{atom: +1 / -1 / 0}: sign of the Hubbard manifold's moment where it exceeds docc_thr."""
    out = {}
    for ia, t in spin_traces(model, gs).items():
        d = t[0] - t[1] if len(t) == 2 else 0.0
        out[ia] = 0 if abs(d) <= docc_thr else (1 if d > 0 else -1)
    return out


def realspace_column(model, qcols):
    """qcols[iq] = trace vector over Hubbard atoms of one perturbed atom J.  Returns the column
    (0, J) of the supercell matrix, index l * N_H + s, as assemble_chi orders it."""
    R = model.supercell_R()
    nh = len(model.hub_atoms)
    nq = len(model.qpts)
    col = np.zeros(len(R) * nh, dtype=complex)
    for iq, q in enumerate(model.qpts):
        for l in range(len(R)):
            col[l * nh:(l + 1) * nh] += np.exp(2j * np.pi * np.dot(q, R[l])) * qcols[iq] / nq
    return col


def _separation(model, ia, ja, Rl):
    """Separation of atom ja of cell Rl from atom ia of cell 0, in supercell fractional coordinates."""
    return (model.frac[ja] + np.asarray(Rl, dtype=float) - model.frac[ia]) / np.array(model.qmesh, dtype=float)


def _length(model, f):
    """Length (bohr) of the supercell fractional vector f taken to its minimum image."""
    n = np.array(model.qmesh, dtype=float)
    f = f - np.round(f)
    return float(np.linalg.norm(f @ (model.cell * n[:, None])))


def _supercell_ops(model, ops):
    """The operations that keep the q-mesh supercell's lattice: W diag(n) = diag(n) M, M integer."""
    n = np.array(model.qmesh, dtype=float)
    out = []
    for Wm, t, perm in ops:
        M = np.diag(1.0 / n) @ Wm @ np.diag(n)
        if np.abs(M - np.round(M)).max() < 1e-9:
            out.append((Wm, t, perm))
    return out


def _rebuild_by_operation(model, src, J, Jp, op):
    """Column (0, J) from column (0, J') through an operation g with g(J' at cell 0) = J at cell L_J."""
    Wm, t, _ = op
    R = model.supercell_R()
    nh = len(model.hub_atoms)
    n = np.array(model.qmesh, dtype=int)
    index = {tuple(int(x) for x in r): l for l, r in enumerate(R)}
    frac = np.array(model.frac, dtype=float)
    L_J = np.round(Wm @ frac[Jp] + t - frac[J])
    Winv = np.linalg.inv(Wm)
    col = np.zeros_like(src)
    for l in range(len(R)):
        for s, ia in enumerate(model.hub_atoms):
            y = Winv @ (frac[ia] + np.asarray(R[l], dtype=float) + L_J - t)
            hit = None
            for sp, ib in enumerate(model.hub_atoms):
                d = y - frac[ib]
                if model.atom_species[ib] == model.atom_species[ia] and np.abs(d - np.round(d)).max() < 1e-5:
                    hit = (sp, np.round(d).astype(int))
                    break
            if hit is None:
                raise ValueError("the operation does not map atom %d of cell %d onto a Hubbard atom" % (ia, l))
            sp, cell = hit
            col[l * nh + s] = src[index[tuple(int(x) for x in np.mod(cell, n))] * nh + sp]
    return col


def reconstruct_columns(model, cols, rep, orient, dist_thr=6e-4, ops=None):
    """cols = {J: real-space column} for the perturbed atoms; returns the columns of every Hubbard
    atom, those of the others rebuilt from their representatives.  With ops (space_group's, for
    find_atpert 3) an operation of the supercell that takes the representative onto the atom rebuilds
    its column; otherwise (or where none does) the separation rule does."""
    R = model.supercell_R()
    nh = len(model.hub_atoms)
    out = dict(cols)
    sops = _supercell_ops(model, ops) if ops is not None else []
    for J in model.hub_atoms:
        if J in out:
            continue
        Jp = rep[J]
        src = cols[Jp]
        op = next((o for o in sops if o[2][Jp] == J), None)
        if op is not None:
            out[J] = _rebuild_by_operation(model, src, J, Jp, op)
            continue
        col = np.zeros_like(src)
        for l in range(len(R)):
            for s, ia in enumerate(model.hub_atoms):
                v = _separation(model, J, ia, R[l])
                d = _length(model, v)
                o = orient[ia] * orient[J]
                cands = [(lp * nh + sp, _separation(model, Jp, ib, R[lp]))
                         for lp in range(len(R)) for sp, ib in enumerate(model.hub_atoms)
                         if model.atom_species[ib] == model.atom_species[ia] and orient[ib] * orient[Jp] == o]
                hit = next((i for i, vp in cands if _length(model, vp - v) <= dist_thr), None)
                if hit is None:
                    hit = next((i for i, vp in cands if abs(_length(model, vp) - d) <= dist_thr), None)
                if hit is None:
                    raise ValueError("no atom of the representative's column matches (%d, %d) of atom %d" % (l, s, J))
                col[l * nh + s] = src[hit]
        out[J] = col
    return out


def chi_from_columns(model, cols):
    """The supercell matrix from the real-space columns (0, J) of every Hubbard atom, by the lattice
    periodicity of the supercell."""
    R = model.supercell_R()
    nh = len(model.hub_atoms)
    n = np.array(model.qmesh, dtype=int)
    index = {tuple(int(x) for x in r): l for l, r in enumerate(R)}
    chi = np.zeros((len(R) * nh, len(R) * nh), dtype=complex)
    for jj, J in enumerate(model.hub_atoms):
        for lp, rp in enumerate(R):
            for l, r in enumerate(R):
                d = index[tuple(int(x) for x in np.mod(np.array(r, dtype=int) - np.array(rp, dtype=int), n))]
                chi[l * nh:(l + 1) * nh, lp * nh + jj] = cols[J][d * nh:(d + 1) * nh]
    return chi


def minus_q(model, iq):
    """Index of -q (mod G) in the q mesh."""
    n = np.array(model.qmesh, dtype=int)
    i = np.rint(np.array(model.qpts[iq]) * n).astype(int)
    j = np.mod(-i, n)
    for jq, q in enumerate(model.qpts):
        if np.array_equal(np.rint(np.array(q) * n).astype(int), j):
            return jq
    raise ValueError("-q is not on the mesh")


def irreducible_q(model):
    """(q indices to compute, partner[iq] = the computed q whose response gives iq: itself, or the
    first of the pair {q, -q} whose conjugate it is)."""
    partner = []
    for iq in range(len(model.qpts)):
        jq = minus_q(model, iq)
        partner.append(min(iq, jq))
    return sorted(set(partner)), partner


# ---- star of q: the (q, J) responses that the space group relates ------------------------------
#
# For an operation g: x -> W x + t of the q-mesh supercell, atom a goes to pi(a) with
# W x_a + t = x_pi(a) + L_a (L_a integer).  The per-q trace columns x_q[J][s] =
# sum_R exp(-2 pi i q.R) chi_{(s, R), (J, 0)} then obey
#     x_{q'}[pi(J)][pi(s)] = exp(2 pi i q'.(L_J - L_s)) x_q[J][s],   q' = W^-T q,
# and time reversal gives x_{-q}[J] = conj(x_q[J]).  A (q, J) pair reached from a computed one by these
# relations need not be computed.

def _q_index(model, qfrac):
    n = np.array(model.qmesh, dtype=int)
    i = np.mod(np.rint(np.asarray(qfrac, dtype=float) * n).astype(int), n)
    return int((i[0] * n[1] + i[1]) * n[2] + i[2])


def _lattice_shifts(model, op):
    Wm, t, perm = op
    frac = np.array(model.frac, dtype=float)
    return {a: np.rint(Wm @ frac[a] + t - frac[perm[a]]) for a in range(len(frac))}


def pair_image(model, op, iq, J):
    """(iq', J') = the image of the pair (q, J) under the operation."""
    Wm, _, perm = op
    qp = np.linalg.inv(Wm).T @ np.asarray(model.qpts[iq], dtype=float)
    return _q_index(model, qp), perm[J]


def irreducible_pairs(model, ops, atoms=None, time_reversal=True):
    """The (iq, J) pairs to compute: the first pair of each orbit under the supercell's operations
    (and q -> -q), the pairs taken J-major (the Hubbard atoms in order), then q in mesh order."""
    atoms = list(model.hub_atoms) if atoms is None else atoms
    sops = _supercell_ops(model, ops)
    seen, out = set(), []
    for J in atoms:
        for iq in range(len(model.qpts)):
            if (iq, J) in seen:
                continue
            out.append((iq, J))
            stack = [(iq, J)]
            seen.add((iq, J))
            while stack:
                p = stack.pop()
                imgs = [pair_image(model, op, p[0], p[1]) for op in sops]
                if time_reversal:
                    imgs.append((minus_q(model, p[0]), p[1]))
                for im in imgs:
                    if im not in seen:
                        seen.add(im)
                        stack.append(im)
    return out


def fill_pairs(model, cols, ops, time_reversal=True):
    """cols = {(iq, J): trace vector over the Hubbard atoms} for the computed pairs; returns the trace
    vectors of every pair reached from them through the supercell's operations and time reversal."""
    sops = _supercell_ops(model, ops)
    hub = list(model.hub_atoms)
    pos = {a: i for i, a in enumerate(hub)}
    out = dict(cols)
    stack = list(cols)
    while stack:
        iq, J = stack.pop()
        x = out[(iq, J)]
        derived = []
        for op in sops:
            iqp, Jp = pair_image(model, op, iq, J)
            if (iqp, Jp) in out:
                continue
            L = _lattice_shifts(model, op)
            qp = np.asarray(model.qpts[iqp], dtype=float)
            y = np.zeros_like(x)
            for s, a in enumerate(hub):
                y[pos[op[2][a]]] = np.exp(2j * np.pi * np.dot(qp, L[J] - L[a])) * x[s]
            derived.append(((iqp, Jp), y))
        if time_reversal:
            mq = minus_q(model, iq)
            if (mq, J) not in out:
                derived.append(((mq, J), x.conj()))
        for key, y in derived:
            if key not in out:
                out[key] = y
                stack.append(key)
    return out
