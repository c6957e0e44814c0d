"""Oracle Kohn-Sham operator on the plane-wave sphere.

Test infrastructure only (see the package docstring).

H u = (1/2)|k+G|^2 u  +  P_sphere FFT[ V(r) * FFT^-1[u] ]  +  sum_p |beta_p> D_p <beta_p|u>

with V(r) = V_loc(r) + V_H(r) + V_xc,sigma(r) on the real-space grid.  The same operator as a dense
matrix has the local part V~((G - G') mod N), the grid transform of V(r) (the FFT grid may be
smaller than alias-free, so the difference G - G' is folded onto the grid exactly like the FFT
route does).
"""

from __future__ import annotations

import math

import numpy as np


def to_grid(model, kd, C):
    """u(r_j) = sum_G c(G) exp(iG.r_j) for each column of C (npw, nb) -> (nb, nr)."""
    nb = C.shape[1]
    X = np.zeros((nb, model.nr), dtype=complex)
    X[:, kd.idx] = C.T
    U = np.fft.ifftn(X.reshape((nb,) + model.grid), axes=(1, 2, 3)) * model.nr
    return U.reshape(nb, model.nr)


def from_grid(model, kd, F):
    """c(G) = (1/N) sum_j f(r_j) exp(-iG.r_j) on the sphere of ``kd``; F (nb, nr) -> (npw, nb)."""
    nb = F.shape[0]
    Fg = np.fft.fftn(F.reshape((nb,) + model.grid), axes=(1, 2, 3)).reshape(nb, model.nr) / model.nr
    return Fg[:, kd.idx].T.copy()


def apply_local(model, kd, vr, C):
    return from_grid(model, kd, vr[None, :] * to_grid(model, kd, C))


def apply_nonlocal(model, kd, C):
    return kd.beta.T @ (model.proj_D[:, None] * (kd.beta.conj() @ C))


def apply_h(model, kd, vr, C):
    """H u for the columns of C (npw, nb); ``vr`` the real local potential on the grid."""
    return 0.5 * kd.g2[:, None] * C + apply_local(model, kd, vr, C) + apply_nonlocal(model, kd, C)


def dense_h(model, kd, vr):
    """The same operator as a dense (npw, npw) Hermitian matrix."""
    vg = np.fft.fftn(vr.reshape(model.grid)) / model.nr
    m = kd.miller
    N = model.grid
    d = m[:, None, :] - m[None, :, :]
    idx = ((d[..., 0] % N[0]) * N[1] + (d[..., 1] % N[1])) * N[2] + (d[..., 2] % N[2])
    H = vg.reshape(-1)[idx]
    H = H + np.diag(0.5 * kd.g2)
    H = H + (kd.beta.T * model.proj_D[None, :]) @ kd.beta.conj()
    return 0.5 * (H + H.conj().T)


def hartree_g(model, rho_g, qfrac=(0.0, 0.0, 0.0)):
    """V_H(q+G) = 4 pi rho(q+G) / |q+G|^2 on the grid mask; q+G = 0 dropped (neutralising
    background)."""
    _, g2, mask = model.grid_gvectors(qfrac)
    out = np.zeros_like(rho_g)
    ok = mask & (g2 > 1e-12)
    out[ok] = 4.0 * math.pi * rho_g[ok] / g2[ok]
    return out


def hartree_r(model, rho_r, qfrac=(0.0, 0.0, 0.0)):
    """V_H(r) for a (lattice-periodic part of a) density on the grid."""
    rg = np.fft.fftn(rho_r.reshape(model.grid)).reshape(-1) / model.nr
    vg = hartree_g(model, rg, qfrac)
    return np.fft.ifftn(vg.reshape(model.grid)).reshape(-1) * model.nr
