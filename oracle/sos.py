"""Oracle pin: bare response by a sum over states from full diagonalisation.

Test infrastructure only (see the package docstring).

In a complete (finite) plane-wave basis the solution of the projected Sternheimer problem
(Eq. LRKSeq_lp with Delta V_Hxc = 0) is Delta u_v = sum_c |c><c|V_pert|u_v> / (eps_v - eps_c) over
all empty states c at k+q, so the trace of Eq. occ_matrix_response_lp_2 becomes

  sum_m Delta_q n^{s sigma}_mm = (2/N_k) sum_k sum_v sum_c sum_m
        <u_vk|phi^s_m,k><phi^s_m,k+q|c_k+q><c_k+q|V^J_pert|u_vk> / (eps_vk - eps_c,k+q)

This route never solves a linear system and never touches the occupied k+q states' projector, so it
checks the Sternheimer solver, the projectors P_c / O, the shift alpha and the TRS factor at once.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg

from .groundstate import kq_states
from .hamiltonian import dense_h


def bare_column(model, gs, iq, J):
    """Trace vector over Hubbard atoms (spin-summed) of the bare response to atom J at q."""
    no = model.nocc
    f = 2.0 if model.nspin == 1 else 1.0
    slJ = model.hub_slice[J]
    out = np.zeros(len(model.hub_atoms), dtype=complex)
    for s in range(model.nspin):
        for ik in range(len(model.kpts)):
            kd = gs.kds[ik]
            kdq, _, _ = kq_states(model, gs, ik, iq)
            H = dense_h(model, kdq, gs.vr(s))
            hub = gs.hub_dense(kdq, s)  # DFT+U+V ground state: its Hubbard potential is part of H
            if hub is not None:
                H = H + hub
            e_all, v_all = scipy.linalg.eigh(H)
            ec, Vc = e_all[no:], v_all[:, no:]
            U = gs.C[s][ik][:, :no]
            ev = gs.eps[s, ik, :no]
            # <c|V_pert|u_v> = sum_m <c|phi_m,k+q><phi_m,k|u_v>
            cV = (Vc.conj().T @ kdq.phi[slJ].T) @ (kd.phi[slJ].conj() @ U)       # (nc, nv)
            denom = ev[None, :] - ec[:, None]
            W = cV / denom
            for si, sa in enumerate(model.hub_atoms):
                sl = model.hub_slice[sa]
                left = (U.conj().T @ kd.phi[sl].T)                               # <u_v|phi_m,k>  (nv, m)
                right = kdq.phi[sl].conj() @ Vc                                  # <phi_m,k+q|c>  (m, nc)
                out[si] += 2.0 * np.einsum("vm,mc,cv->", left, right, W)
    return f * out / len(model.kpts)
