"""Oracle ground state: fixed-occupation Kohn-Sham SCF (LDA / LSDA), Hubbard occupation matrices
(Eq. occ_matrix_0) and the non-self-consistent bands at k+q (Sec. 2.3, the k+q states of
Eqs. proj_v / proj_c).

Test infrastructure only (see the package docstring).

Readings (the paper's ground state comes from pw.x and is not specified further):
  * occupations are fixed: ``nocc = nelec/2`` bands per spin channel (tot_magnetization = 0 for
    nspin = 2, as in the paper's second SCF step for magnetic insulators, Sec. 5.2);
  * density rho_sigma(r) = (f / (N_k Omega)) sum_k sum_v |u_vk(r)|^2 with f = 2 for nspin = 1 and
    f = 1 per channel for nspin = 2;
  * starting density: uniform rho0 = nelec / Omega; for nspin = 2 it is split as
    rho0/2 (1 +- s(r)) with s(r) = clip(sum_I m_I 0.9 exp(-|r - tau_I|^2 / 2), -0.9, 0.9) over the
    starting moments m_I = +1/-1/0 (minimum image);
  * the SCF mixes V_Hxc with the modified Broyden scheme and stops when the rms residual of
    V_Hxc is below ``tol``.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import dftu, xc
from .hamiltonian import apply_h, dense_h, hartree_r, to_grid
from .mixing import Broyden


def initial_density(model):
    rho0 = model.nelec / model.omega
    if model.nspin == 1:
        return np.full((1, model.nr), rho0)
    N = model.grid
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    s = np.zeros(model.nr)
    mom = model.moments or [0] * model.nat
    for ia in range(model.nat):
        if mom[ia] == 0:
            continue
        d = j - model.frac[ia][None, :]
        d -= np.round(d)
        r = d @ model.cell
        s += mom[ia] * 0.9 * np.exp(-0.5 * np.einsum("ij,ij->i", r, r))
    s = np.clip(s, -0.9, 0.9)
    return np.stack([0.5 * rho0 * (1 + s), 0.5 * rho0 * (1 - s)])


def hxc_potential(model, rho):
    """V_H[rho_total] + V_xc,sigma[rho] on the grid, shape (nspin, nr), real."""
    tot = rho.sum(axis=0)
    vh = hartree_r(model, tot).real
    if model.nspin == 1:
        return (vh + xc.vxc_unpolarized(rho[0]))[None, :]
    vu, vd = xc.vxc_polarized(rho[0], rho[1])
    return np.stack([vh + vu, vh + vd])


def eigensolve(model, kd, vr, nbnd, extra=None):
    """Lowest ``nbnd`` eigenpairs of H (dense Hermitian eigensolver).  ``extra`` is an optional
    dense (npw, npw) operator added to H (used by the finite-difference pins)."""
    H = dense_h(model, kd, vr)
    if extra is not None:
        H = H + extra
    e, v = scipy.linalg.eigh(H, subset_by_index=(0, nbnd - 1))
    return e, v


class GroundState:
    """Converged ground state: eigenpairs at the k mesh, densities and potentials; with a Hubbard
    correction (DFT+U+V) also the occupation matrices its Hubbard potential is built from."""

    def __init__(self, model, vloc, vhxc, rho, eps, C, kds, iterations, residual, hub_occ=None):
        self.model = model
        self.vloc = vloc
        self.vhxc = vhxc
        self.rho = rho
        self.eps = eps            # (nspin, nk, nbnd)
        self.C = C                # C[s][ik] (npw_k, nbnd)
        self.kds = kds
        self.iterations = iterations
        self.residual = residual
        self.hub_occ = hub_occ    # occupations of V_Hub (dftu.occupations), None without a correction

    def vr(self, s):
        return self.vloc + self.vhxc[s]

    def hub_w(self, kd, s):
        """W of the ground state's Hubbard potential at k point ``kd`` (None without a correction)."""
        if self.hub_occ is None:
            return None
        return dftu.w_matrix(self.model, kd, self.hub_occ, s)

    def hub_dense(self, kd, s):
        W = self.hub_w(kd, s)
        return None if W is None else dftu.dense(self.model, kd, W)

    @property
    def nocc(self):
        return self.model.nocc

    def gap(self):
        """min over spin of (lowest empty - highest occupied) over all k (Ha)."""
        no = self.nocc
        return float(min(self.eps[s, :, no].min() - self.eps[s, :, no - 1].max() for s in range(self.eps.shape[0])))

    def occupations(self):
        """n^{I sigma}_{m1 m2} = (1/N_k) sum_k sum_v <u|phi_m2><phi_m1|u>  (Eq. occ_matrix_0 with the
        per-cell 1/N_k normalisation).  Returns {atom: array (nspin, m, m)}."""
        m = self.model
        out = {}
        for ia in m.hub_atoms:
            sl = m.hub_slice[ia]
            nm = sl.stop - sl.start
            n = np.zeros((m.nspin, nm, nm), dtype=complex)
            for s in range(m.nspin):
                for ik, kd in enumerate(self.kds):
                    A = kd.phi[sl].conj() @ self.C[s][ik][:, : m.nocc]
                    n[s] += A @ A.conj().T
            out[ia] = (n / len(self.kds)).real
        return out

    def traces(self):
        """n^I = sum_sigma sum_m n^{I sigma}_{mm} (spin-summed; x2 for nspin = 1)."""
        f = 2.0 if self.model.nspin == 1 else 1.0
        return {ia: f * float(np.trace(n, axis1=1, axis2=2).sum()) for ia, n in self.occupations().items()}


def density(model, C_all, kds):
    f = 2.0 if model.nspin == 1 else 1.0
    rho = np.zeros((model.nspin, model.nr))
    for s in range(model.nspin):
        for ik, kd in enumerate(kds):
            U = to_grid(model, kd, C_all[s][ik][:, : model.nocc])
            rho[s] += (np.abs(U) ** 2).sum(axis=0)
    return rho * f / (len(kds) * model.omega)


def _pack(occ):
    onsite, pocc = occ
    parts = [onsite[a].reshape(-1) for a in sorted(onsite)] + [p.reshape(-1) for p in pocc]
    z = np.concatenate(parts) if parts else np.zeros(0, dtype=complex)
    return np.concatenate([z.real, z.imag])


def _unpack(x, like):
    onsite, pocc = like
    n = len(x) // 2
    z = x[:n] + 1j * x[n:]
    out_on, out_p, o = {}, [], 0
    for a in sorted(onsite):
        sz = onsite[a].size
        out_on[a] = z[o:o + sz].reshape(onsite[a].shape)
        o += sz
    for p in pocc:
        out_p.append(z[o:o + p.size].reshape(p.shape))
        o += p.size
    return out_on, out_p


def scf(model, tol=1e-11, maxiter=300, nextra=4, alpha=0.3, nmix=6, perturb=None, frozen_vhxc=None,
        vstart=None, frozen_hub=None, verbose=False):
    """Fixed-occupation SCF.

    perturb: optional (atom J, lambda): adds lambda sum_m |phi^J_m><phi^J_m| to H (Sec. 2.3, the
    perturbing potential of Eq. chi).  frozen_vhxc: if given, V_Hxc is held at this value and one
    non-self-consistent diagonalisation is done (bare response, chi_0).  vstart: optional starting
    V_Hxc (nspin, nr) instead of the one of the starting density.

    With Hubbard parameters in the workload (DFT+U+V, Sec. 2.1) H carries the Hubbard potential of
    Eq. Hub_pot_0 built from the occupation matrices, which are mixed together with V_Hxc (one
    modified Broyden vector) and converged to ``tol`` as well.  frozen_hub: occupation matrices to
    hold the Hubbard potential at (the response of the Hubbard potential is not part of the
    linear-response problem, Sec. 2.3)."""
    kds = [model.kdata(k) for k in model.kpts]
    vloc = model.vloc_r()
    nbnd = model.nocc + nextra
    extras = [None] * len(kds)
    if perturb is not None:
        J, lam = perturb
        sl = model.hub_slice[J]
        for ik, kd in enumerate(kds):
            ph = kd.phi[sl]
            extras[ik] = lam * (ph.T @ ph.conj())
    hub = dftu.active(model)
    if frozen_vhxc is not None:
        vin = frozen_vhxc.copy()
    elif vstart is not None:
        vin = vstart.copy()
    else:
        vin = hxc_potential(model, initial_density(model))
    occ_in = None
    if hub:
        occ_in = frozen_hub if frozen_hub is not None else dftu.occupations(
            model, [[np.zeros((kd.npw, model.nocc)) for kd in kds] for _ in range(model.nspin)], kds)
    mixer = Broyden(alpha=alpha, nmix=nmix)
    res = np.inf
    it = 0
    for it in range(1, maxiter + 1):
        eps = np.zeros((model.nspin, len(kds), nbnd))
        C = [[None] * len(kds) for _ in range(model.nspin)]
        for s in range(model.nspin):
            for ik, kd in enumerate(kds):
                extra = extras[ik]
                if hub:
                    h = dftu.dense(model, kd, dftu.w_matrix(model, kd, occ_in, s))
                    extra = h if extra is None else extra + h
                e, v = eigensolve(model, kd, vloc + vin[s], nbnd, extra)
                eps[s, ik] = e
                C[s][ik] = v
        rho = density(model, C, kds)
        if frozen_vhxc is not None:
            return GroundState(model, vloc, vin, rho, eps, C, kds, it, 0.0, occ_in)
        vout = hxc_potential(model, rho)
        F = vout - vin
        res = math.sqrt(float(np.mean(F * F)))
        x, f = vin.reshape(-1), F.reshape(-1)
        res_n = 0.0
        if hub and frozen_hub is None:
            occ_out = dftu.occupations(model, C, kds)
            xn, fn = _pack(occ_in), _pack(occ_out) - _pack(occ_in)
            res_n = float(np.abs(fn).max()) if len(fn) else 0.0
            x, f = np.concatenate([x, xn]), np.concatenate([f, fn])
        if verbose:
            print("scf", it, res, res_n)
        if res < tol and res_n < tol:
            return GroundState(model, vloc, vin, rho, eps, C, kds, it, res, occ_in)
        x = mixer.step(x, f)
        vin = x[: vin.size].reshape(vin.shape)
        if hub and frozen_hub is None:
            occ_in = _unpack(x[vin.size:], occ_in)
    raise RuntimeError("ground-state SCF did not converge (residual %.3e)" % res)


def kq_states(model, gs, ik, iq):
    """Occupied states and energies at k+q, as (KData(k+q), C (npw, nocc), eps (nspin, nocc) per
    spin).  On-mesh k+q = k' + G0: c_{k+q}(G) = c_{k'}(G + G0).  Off-mesh: a non-self-consistent
    diagonalisation with the ground-state potential."""
    kq = model.kpts[ik] + model.qpts[iq]
    kdq = model.kdata(kq)
    kp, g0 = model.kq_map(ik, iq)
    Cs, es = [], []
    for s in range(model.nspin):
        if kp is not None:
            src = gs.kds[kp]
            lut = {tuple(m): i for i, m in enumerate(src.miller)}
            rows = [lut[tuple(m + g0)] for m in kdq.miller]
            Cs.append(gs.C[s][kp][rows, : model.nocc])
            es.append(gs.eps[s, kp, : model.nocc])
        else:
            e, v = eigensolve(model, kdq, gs.vr(s), model.nocc, gs.hub_dense(kdq, s))
            Cs.append(v)
            es.append(e)
    return kdq, Cs, np.array(es)
