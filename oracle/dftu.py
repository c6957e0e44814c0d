"""Oracle Hubbard-corrected ground state (DFT+U+V, Sec. 2.1): generalised occupation matrices
(Eq. occ_matrix_0 with the generalised projector of Eq. Pm1m2), the corrective energy (Eq. Edftu)
and the Hubbard potential (Eq. Hub_pot_0) in the plane-wave basis.

Test infrastructure only (see the package docstring).

Parameters come from the workload: ``hubbard_U`` = [(atom, U_eV), ...] for Hubbard atoms I, and
``hubbard_V`` = [(i, j, (R1, R2, R3), V_eV), ...] for the inter-site pairs: atom j displaced by the
lattice vector R (crystal units) is a neighbour of atom i.  The star sum of Eq. Hub_pot_0 runs over
every listed pair, so a pair and its reverse (j, i, -R) are both listed.

Bloch sums of the (atomic or ortho-atomic) orbitals at k have plane-wave coefficients phi_a(k+G)
(the rows of KData.phi).  With A_k[a][v] = <phi_a,k|u_vk>:
  on site       n^{I s}_{m1 m2}        = (1/N_k) sum_k sum_v A[I m1][v] conj(A[I m2][v])
  pair (i,j,R)  n^{ij(R) s}_{m1 m2}    = (1/N_k) sum_k exp(-i k.R) sum_v A[i m1][v] conj(A[j m2][v])
(the lattice sum of |phi^j_{R'+R}><phi^i_{R'}| has the k-space form exp(-i k.R) |phi^j_k><phi^i_k|).
The potential at k acts as V_Hub,s = sum_ab |phi_a,k> W_ks[a][b] <phi_b,k| with
  W[I m1][I m2]  = U^I (delta_m1m2 / 2 - n^{I s}_{m1 m2})
  W[i m1][j m2] += -V^{ij} n^{ij(R) s}_{m1 m2} exp(+i k.R)   for every pair (i, j, R),
Hermitian because the reverse pair carries the conjugate block.  U and V in eV on input, Ha inside.
"""

from __future__ import annotations

import numpy as np

from .model import HA_TO_EV


def parameters(model):
    """(U per Hubbard atom in Ha (dict atom -> U), pairs [(i, j, R (int array), V in Ha)])."""
    U = {int(a): float(u) / HA_TO_EV for a, u in model.w.get("hubbard_U", [])}
    pairs = [(int(i), int(j), np.array(R, dtype=int), float(v) / HA_TO_EV)
             for i, j, R, v in model.w.get("hubbard_V", [])]
    for a in U:
        if a not in model.hub_slice:
            raise ValueError("hubbard_U names an atom without Hubbard orbitals")
    for i, j, _, _ in pairs:
        if i not in model.hub_slice or j not in model.hub_slice:
            raise ValueError("hubbard_V names an atom without Hubbard orbitals")
    return U, pairs


def active(model):
    U, pairs = parameters(model)
    return bool(U) or bool(pairs)


def occupations(model, C, kds):
    """Occupation matrices of the occupied states: (onsite {atom: (nspin, m, m)},
    pairs [(nspin, m_i, m_j) per listed pair, in order])."""
    U, pairs = parameters(model)
    nk = len(kds)
    onsite = {a: np.zeros((model.nspin,) + (model.hub_slice[a].stop - model.hub_slice[a].start,) * 2, dtype=complex)
              for a in model.hub_atoms}
    pocc = [np.zeros((model.nspin, model.hub_slice[i].stop - model.hub_slice[i].start,
                      model.hub_slice[j].stop - model.hub_slice[j].start), dtype=complex) for i, j, _, _ in pairs]
    for s in range(model.nspin):
        for ik, kd in enumerate(kds):
            A = kd.phi.conj() @ C[s][ik][:, : model.nocc]          # (nhub, nocc)
            for a in model.hub_atoms:
                sl = model.hub_slice[a]
                onsite[a][s] += A[sl] @ A[sl].conj().T
            for p, (i, j, R, _) in enumerate(pairs):
                ph = np.exp(-2j * np.pi * np.dot(kd.kfrac, R))
                pocc[p][s] += ph * (A[model.hub_slice[i]] @ A[model.hub_slice[j]].conj().T)
    for a in onsite:
        onsite[a] /= nk
    for p in range(len(pocc)):
        pocc[p] /= nk
    return onsite, pocc


def w_matrix(model, kd, occ, s):
    """W_ks (nhub x nhub) of the Hubbard potential at k point ``kd`` for spin s."""
    U, pairs = parameters(model)
    onsite, pocc = occ
    W = np.zeros((model.nhub, model.nhub), dtype=complex)
    for a, u in U.items():
        sl = model.hub_slice[a]
        m = sl.stop - sl.start
        W[sl, sl] += u * (0.5 * np.eye(m) - onsite[a][s])
    for p, (i, j, R, v) in enumerate(pairs):
        ph = np.exp(2j * np.pi * np.dot(kd.kfrac, R))
        W[model.hub_slice[i], model.hub_slice[j]] += -v * pocc[p][s] * ph
    return W


def dense(model, kd, W):
    """The Hubbard potential at k as a dense (npw, npw) matrix: phi^T W phi^*."""
    return kd.phi.T @ W @ kd.phi.conj()


def apply(model, kd, W, X):
    """V_Hub X for the columns of X (npw, nb)."""
    return kd.phi.T @ (W @ (kd.phi.conj() @ X))


def energy(model, occ):
    """E_{U+V} per cell (Eq. Edftu), Ha; the spin sum runs over both channels (nspin = 2) or is
    twice the single channel (nspin = 1)."""
    U, pairs = parameters(model)
    onsite, pocc = occ
    f = 2.0 if model.nspin == 1 else 1.0
    e = 0.0
    for a, u in U.items():
        for s in range(model.nspin):
            n = onsite[a][s]
            e += f * 0.5 * u * np.trace((np.eye(len(n)) - n) @ n).real
    # pair (i, j, R) and its reverse pair carry n^{ij} and n^{ji} = n^{ij, H}
    for p, (i, j, R, v) in enumerate(pairs):
        for s in range(model.nspin):
            n = pocc[p][s]
            e -= f * 0.5 * v * np.trace(n @ n.conj().T).real
    return e
