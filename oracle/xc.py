"""Oracle LDA: Slater exchange + Perdew-Zunger (1981) correlation, spin-interpolated with the von
Barth-Hedin function f(zeta).  Energies per electron eps(rs, zeta), potentials v_sigma and the
response kernel f_xc = d v_sigma / d rho_sigma' that enters Delta V_Hxc (Sec. 2.3, the response Hxc
potential of Eq. LRKSeq_lp).

Test infrastructure only (see the package docstring).

Closed forms written out from the definitions (rho = rho_up + rho_dn, zeta = (rho_up - rho_dn)/rho,
rs = (3 / (4 pi rho))^(1/3), s_sigma = +1 / -1, e = rho * eps):
  v_sigma       = eps - (rs/3) eps_rs + (s_sigma - zeta) eps_zeta
  f_sigma,sigma' = [(2/3) eps_rs - (rs/3) eps_rsrs + (s_sigma - zeta) eps_rszeta] * (-rs / (3 rho))
                 + [-(rs/3) eps_rszeta + (s_sigma - zeta) eps_zetazeta] * (s_sigma' - zeta) / rho
Points with rho < 1e-10 get v = f = 0.
"""

from __future__ import annotations

import math

import numpy as np

RHO_MIN = 1e-10

# Perdew & Zunger, PRB 23, 5048 (1981), Table XII: unpolarised (U) and fully polarised (P)
PZ_U = dict(gamma=-0.1423, beta1=1.0529, beta2=0.3334, A=0.0311, B=-0.048, C=0.0020, D=-0.0116)
PZ_P = dict(gamma=-0.0843, beta1=1.3981, beta2=0.2611, A=0.01555, B=-0.0269, C=0.0007, D=-0.0048)

EX0 = -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0)  # eps_x(rs, 0) = EX0 / rs
FDEN = 2.0 ** (4.0 / 3.0) - 2.0


def _pz(rs, p):
    """eps_c(rs) and its first two rs-derivatives for one PZ81 parameter set."""
    rs = np.asarray(rs, dtype=float)
    hi = rs >= 1.0
    e = np.empty_like(rs)
    d1 = np.empty_like(rs)
    d2 = np.empty_like(rs)
    r = rs[hi]
    sq = np.sqrt(r)
    den = 1.0 + p["beta1"] * sq + p["beta2"] * r
    dden = p["beta1"] / (2.0 * sq) + p["beta2"]
    ddden = -p["beta1"] / (4.0 * r * sq)
    e[hi] = p["gamma"] / den
    d1[hi] = -p["gamma"] * dden / den ** 2
    d2[hi] = p["gamma"] * (2.0 * dden ** 2 - den * ddden) / den ** 3
    r = rs[~hi]
    lr = np.log(r)
    e[~hi] = p["A"] * lr + p["B"] + p["C"] * r * lr + p["D"] * r
    d1[~hi] = p["A"] / r + p["C"] * (lr + 1.0) + p["D"]
    d2[~hi] = -p["A"] / (r * r) + p["C"] / r
    return e, d1, d2


def eps_derivs(rs, zeta):
    """eps_xc(rs, zeta) and the derivatives eps_rs, eps_zeta, eps_rsrs, eps_rszeta, eps_zetazeta."""
    rs = np.asarray(rs, dtype=float)
    z = np.clip(np.asarray(zeta, dtype=float), -1.0 + 1e-14, 1.0 - 1e-14)
    up, dn = 1.0 + z, 1.0 - z
    # exchange: eps_x = EX0/rs * phi(zeta), phi = ((1+z)^(4/3) + (1-z)^(4/3)) / 2
    phi = 0.5 * (up ** (4 / 3) + dn ** (4 / 3))
    dphi = (2.0 / 3.0) * (up ** (1 / 3) - dn ** (1 / 3))
    ddphi = (2.0 / 9.0) * (up ** (-2 / 3) + dn ** (-2 / 3))
    ex = EX0 / rs * phi
    ex_r = -EX0 / rs ** 2 * phi
    ex_rr = 2.0 * EX0 / rs ** 3 * phi
    ex_z = EX0 / rs * dphi
    ex_zz = EX0 / rs * ddphi
    ex_rz = -EX0 / rs ** 2 * dphi
    # correlation: eps_c = eU + f(z) (eP - eU)
    eU, eU1, eU2 = _pz(rs, PZ_U)
    eP, eP1, eP2 = _pz(rs, PZ_P)
    f = (up ** (4 / 3) + dn ** (4 / 3) - 2.0) / FDEN
    df = (4.0 / 3.0) * (up ** (1 / 3) - dn ** (1 / 3)) / FDEN
    ddf = (4.0 / 9.0) * (up ** (-2 / 3) + dn ** (-2 / 3)) / FDEN
    ec = eU + f * (eP - eU)
    ec_r = eU1 + f * (eP1 - eU1)
    ec_rr = eU2 + f * (eP2 - eU2)
    ec_z = df * (eP - eU)
    ec_zz = ddf * (eP - eU)
    ec_rz = df * (eP1 - eU1)
    return (ex + ec, ex_r + ec_r, ex_z + ec_z, ex_rr + ec_rr, ex_rz + ec_rz, ex_zz + ec_zz)


def _rs(rho):
    return (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)


def exc_density(rho_up, rho_dn):
    """Energy density e = rho * eps_xc (used by the tests to check v = de/drho)."""
    rho = rho_up + rho_dn
    out = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    r = rho[ok]
    e = eps_derivs(_rs(r), (rho_up[ok] - rho_dn[ok]) / r)[0]
    out[ok] = r * e
    return out


def vxc_polarized(rho_up, rho_dn):
    """(v_up, v_dn) on the grid."""
    rho = rho_up + rho_dn
    vu = np.zeros_like(rho)
    vd = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    r = rho[ok]
    z = (rho_up[ok] - rho_dn[ok]) / r
    rs = _rs(r)
    e, e_r, e_z, _, _, _ = eps_derivs(rs, z)
    base = e - rs / 3.0 * e_r
    vu[ok] = base + (1.0 - z) * e_z
    vd[ok] = base + (-1.0 - z) * e_z
    return vu, vd


def fxc_polarized(rho_up, rho_dn):
    """(f_uu, f_ud, f_dd) on the grid; f_du = f_ud."""
    rho = rho_up + rho_dn
    out = [np.zeros_like(rho) for _ in range(3)]
    ok = rho >= RHO_MIN
    r = rho[ok]
    z = np.clip((rho_up[ok] - rho_dn[ok]) / r, -1.0 + 1e-14, 1.0 - 1e-14)
    rs = _rs(r)
    e, e_r, e_z, e_rr, e_rz, e_zz = eps_derivs(rs, z)

    def f(s1, s2):
        dv_drs = (2.0 / 3.0) * e_r - rs / 3.0 * e_rr + (s1 - z) * e_rz
        dv_dz = -rs / 3.0 * e_rz + (s1 - z) * e_zz
        return dv_drs * (-rs / (3.0 * r)) + dv_dz * (s2 - z) / r

    out[0][ok] = f(1.0, 1.0)
    out[1][ok] = f(1.0, -1.0)
    out[2][ok] = f(-1.0, -1.0)
    return tuple(out)


def vxc_unpolarized(rho):
    """v_xc(rho) for a spin-unpolarised density."""
    out = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    r = rho[ok]
    rs = _rs(r)
    e, e_r, _, _, _, _ = eps_derivs(rs, np.zeros_like(r))
    out[ok] = e - rs / 3.0 * e_r
    return out


def fxc_unpolarized(rho):
    """f_xc = d v_xc / d rho for a spin-unpolarised density."""
    out = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    r = rho[ok]
    rs = _rs(r)
    _, e_r, _, e_rr, _, _ = eps_derivs(rs, np.zeros_like(r))
    out[ok] = ((2.0 / 3.0) * e_r - rs / 3.0 * e_rr) * (-rs / (3.0 * r))
    return out
