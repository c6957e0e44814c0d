"""Oracle self-consistent q-specific Sternheimer solve (Sec. 2.3).

Test infrastructure only (see the package docstring).

For a perturbed Hubbard atom J (s') and a wavevector q, iterate until self-consistency:

  1. right-hand side (Eq. LRKSeq_lp):
        b_v = - P_c,k+q ( Delta V_Hxc,q u_vk + V_pert,k+q,k u_vk )
     with V_pert = sum_m |phi^J_m,k+q><phi^J_m,k|                                    (Eq. vpert)
     and  P_c = 1 - sum_v' |u_v'k+q><u_v'k+q|                                        (Eq. proj_c)
  2. solve (H_k+q + alpha O_k+q - eps_vk) Delta u_v = b_v by preconditioned conjugate gradients,
     O = sum_v' |u_v'k+q><u_v'k+q| (Eq. proj_v), alpha = 2 (max eps_v - min eps_v) over the
     occupied bands (the text after Eq. proj_c);
  3. response density (time reversal gives the factor 2; f = 2 for nspin = 1, 1 per channel):
        Delta rho_sigma(r) = (2 f / (N_k Omega)) sum_k sum_v conj(u_vk(r)) Delta u_vk(r)
  4. response occupations (Eq. occ_matrix_response_lp_2):
        Delta n^{s sigma}_{m1 m2} = (1/N_k) sum_k sum_v [ <u|phi^s_m2,k><phi^s_m1,k+q|Delta u>
                                                        + <u|phi^s_m1,k><phi^s_m2,k+q|Delta u> ]
  5. Delta V_Hxc,sigma = 4 pi Delta rho_tot(q+G) / |q+G|^2 (q+G = 0 dropped) + sum_sigma' f_xc
     Delta rho_sigma', then modified Broyden mixing of Delta V_Hxc (alpha_mix, nmix).
The first iteration (Delta V_Hxc = 0) gives the bare response chi_0 (Sec. 3.2).

Readings: CG stops per band when ||r_v||_2 <= tol_cg; preconditioner 1 / (1 + |k+q+G|^2 / 2);
the SCF stops when the rms of Delta V_out - Delta V_in is below ``scf_tol`` and the change of every
response trace between iterations is below ``conv_chi``.
"""

from __future__ import annotations

import math

import numpy as np

from . import dftu, xc
from .groundstate import kq_states
from .hamiltonian import apply_h, from_grid, hartree_r, to_grid
from .mixing import Broyden


def sternheimer_operator(model, kdq, vr, Cq, alpha, eps_v, X, W=None):
    """Left-hand side of Eq. LRKSeq_lp on the columns of X (npw_k+q, nb):
    (H_k+q + alpha O_k+q - eps_v) X with O_k+q = Cq Cq^H the projector on the occupied states at
    k+q (Eq. proj_v, Cq (npw_k+q, nocc)), ``vr`` the spin's local potential on the grid and eps_v
    one shift per column.  W: the ground state's Hubbard potential at k+q (DFT+U+V, Eq. Hub_pot_0),
    part of H_k+q; its response is not (Sec. 2.3)."""
    HX = apply_h(model, kdq, vr, X)
    if W is not None:
        HX = HX + dftu.apply(model, kdq, W, X)
    return HX + alpha * (Cq @ (Cq.conj().T @ X)) - X * np.asarray(eps_v)[None, :]


class ResponseContext:
    """Everything a (q, J) solve needs that does not depend on J: k+q states, real-space u_k,
    f_xc, alpha."""

    def __init__(self, model, gs, iq):
        self.model, self.gs, self.iq = model, gs, iq
        self.qfrac = model.qpts[iq]
        no = model.nocc
        self.kq = []
        for ik in range(len(model.kpts)):
            kdq, Cq, eq = kq_states(model, gs, ik, iq)
            self.kq.append((kdq, Cq, eq))
        self.ur = [[to_grid(model, gs.kds[ik], gs.C[s][ik][:, :no]) for ik in range(len(model.kpts))]
                   for s in range(model.nspin)]
        e = gs.eps[:, :, :no]
        self.alpha = 2.0 * float(e.max() - e.min())
        rho = gs.rho
        if model.nspin == 1:
            self.fxc = {(0, 0): xc.fxc_unpolarized(rho[0])}
        else:
            fuu, fud, fdd = xc.fxc_polarized(rho[0], rho[1])
            self.fxc = {(0, 0): fuu, (0, 1): fud, (1, 0): fud, (1, 1): fdd}

    def apply_A(self, s, ik, X, eps_v):
        """(H_k+q + alpha O_k+q - eps_v) X for the columns of X (per-column eps_v)."""
        kdq, Cq, _ = self.kq[ik]
        return sternheimer_operator(self.model, kdq, self.gs.vr(s), Cq[s], self.alpha, eps_v, X,
                                    self.gs.hub_w(kdq, s))

    def dv_times_u(self, s, ik, dv):
        """Delta V_Hxc,q(r) u_k(r), taken to the k+q sphere."""
        kdq = self.kq[ik][0]
        return from_grid(self.model, kdq, dv[None, :] * self.ur[s][ik])

    def hxc_response(self, drho):
        """Delta V_Hxc,sigma from Delta rho_sigma (complex lattice-periodic parts at q)."""
        m = self.model
        tot = drho.sum(axis=0)
        vh = hartree_r(m, tot, self.qfrac)
        out = np.empty_like(drho)
        for s in range(m.nspin):
            out[s] = vh + sum(self.fxc[(s, t)] * drho[t] for t in range(m.nspin))
        return out


def cg_solve(apply_A, b, x0, precond, tol, maxiter=2000):
    """Preconditioned conjugate gradients, one independent system per column; a column stops once
    its residual 2-norm is <= tol.  Returns (x, iterations)."""
    x = x0.copy()
    r = b - apply_A(x, np.arange(b.shape[1]))
    z = precond[:, None] * r
    p = z.copy()
    rz = np.real(np.sum(r.conj() * z, axis=0))
    it = 0
    for it in range(1, maxiter + 1):
        act = np.where(np.linalg.norm(r, axis=0) > tol)[0]
        if len(act) == 0:
            return x, it - 1
        Ap = apply_A(p[:, act], act)
        pAp = np.real(np.sum(p[:, act].conj() * Ap, axis=0))
        a = rz[act] / pAp
        x[:, act] += a[None, :] * p[:, act]
        r[:, act] -= a[None, :] * Ap
        z_act = precond[:, None] * r[:, act]
        rz_new = np.real(np.sum(r[:, act].conj() * z_act, axis=0))
        beta = rz_new / rz[act]
        p[:, act] = z_act + beta[None, :] * p[:, act]
        rz[act] = rz_new
    raise RuntimeError("CG did not converge")


def solve_column(model, gs, iq, J, ctx=None, tol_cg=1e-12, scf_tol=1e-11, conv_chi=1e-12, niter_max=100,
                 alpha_mix=0.3, nmix=4, hxc=True, verbose=False):
    """One (q, J) response.  Returns dict with 'dn0', 'dn' ({atom s: complex (nspin, m, m)}),
    'iterations', 'cg_iterations'."""
    if ctx is None:
        ctx = ResponseContext(model, gs, iq)
    nk = len(model.kpts)
    no = model.nocc
    f = 2.0 if model.nspin == 1 else 1.0
    slJ = model.hub_slice[J]
    x_prev = {}
    dv_in = np.zeros((model.nspin, model.nr), dtype=complex)
    mixer = Broyden(alpha=alpha_mix, nmix=nmix)
    dn0 = None
    prev_tr = None
    cg_total = 0
    # V_pert u_k is fixed across iterations
    vpu = {}
    for s in range(model.nspin):
        for ik in range(nk):
            kd = gs.kds[ik]
            kdq = ctx.kq[ik][0]
            U = gs.C[s][ik][:, :no]
            vpu[(s, ik)] = kdq.phi[slJ].T @ (kd.phi[slJ].conj() @ U)
    for it in range(1, niter_max + 1):
        drho = np.zeros((model.nspin, model.nr), dtype=complex)
        M = np.zeros((model.nspin, model.nhub, model.nhub), dtype=complex)
        for s in range(model.nspin):
            for ik in range(nk):
                kd = gs.kds[ik]
                kdq, Cq, _ = ctx.kq[ik]
                U = gs.C[s][ik][:, :no]
                eps_v = gs.eps[s, ik, :no]
                b = -vpu[(s, ik)]
                if it > 1:
                    b = b - ctx.dv_times_u(s, ik, dv_in[s])
                b = b - Cq[s] @ (Cq[s].conj().T @ b)
                prec = 1.0 / (1.0 + 0.5 * kdq.g2)
                x0 = x_prev.get((s, ik), np.zeros_like(b))
                x, nit = cg_solve(lambda X, cols: ctx.apply_A(s, ik, X, eps_v[cols]), b, x0, prec, tol_cg)
                cg_total += nit
                x_prev[(s, ik)] = x
                drho[s] += (ctx.ur[s][ik].conj() * to_grid(model, kdq, x)).sum(axis=0)
                A = kd.phi.conj() @ U
                B = kdq.phi.conj() @ x
                M[s] += B @ A.conj().T
        drho *= 2.0 * f / (nk * model.omega)
        M /= nk
        dn = {}
        for sa in model.hub_atoms:
            sl = model.hub_slice[sa]
            blk = M[:, sl, sl]
            dn[sa] = blk + np.transpose(blk, (0, 2, 1))
        tr = np.array([np.trace(dn[sa], axis1=1, axis2=2).sum() for sa in model.hub_atoms])
        if it == 1:
            dn0 = {k: v.copy() for k, v in dn.items()}
            if not hxc:
                return dict(dn0=dn0, dn=dn, iterations=1, cg_iterations=cg_total, ctx=ctx)
        dv_out = ctx.hxc_response(drho)
        F = dv_out - dv_in
        res = math.sqrt(float(np.mean(np.abs(F) ** 2)))
        dchi = np.inf if prev_tr is None else float(np.max(np.abs(tr - prev_tr)))
        prev_tr = tr
        if verbose:
            print("resp it", it, "res %.3e dchi %.3e cg %d" % (res, dchi, cg_total))
        if it > 1 and res < scf_tol and dchi < conv_chi:
            return dict(dn0=dn0, dn=dn, iterations=it, cg_iterations=cg_total, ctx=ctx)
        dv_in = mixer.step(dv_in.reshape(-1), F.reshape(-1)).reshape(dv_in.shape)
    raise RuntimeError("response SCF did not converge")
