"""Spin-polarised (LSDA) branches at zeta != 0, on the GPU against the oracle.

1. The LDA kernel of the library (V_xc,sigma and the response kernel f_xc,sigma sigma', the cross
   term f_up,down and the (s - zeta) terms of the von Barth-Hedin interpolation included) on seeded
   spin densities with r_s from 0.1 to 20 (both Perdew-Zunger branches) and |zeta| up to 0.95, plus
   points below the 1e-10 density floor, against oracle/xc.py: FP64 on both sides, 1e-11 relative
   (different cbrt/log implementations, same formulas).
2. A full response on a strongly polarised input: the rocksalt cell (nspin = 2) with the
   antiferromagnetic starting density itself (|zeta| up to 0.9 around the H sites) as rho, its
   Hxc potential as V_Hxc and the occupied states of one diagonalisation at that potential, imported
   identically into both sides.  The response kernel is then evaluated where the spin channels
   differ strongly, and Delta n_up differs from Delta n_down.  FP64 at 1e-8 and the mixed form at
   1e-5 of max |Delta n| (the parity bars of the two forms)."""

import numpy as np
import pytest

import workloads as W
from oracle import groundstate as G, response as R, xc
from oracle.model import Model
from tests.bridge import import_ground_state, oracle_dn_padded

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")


def _densities(n, seed):
    rng = np.random.default_rng(seed)
    rs = np.exp(rng.uniform(np.log(0.1), np.log(20.0), n))
    rho = 3.0 / (4.0 * np.pi * rs ** 3)
    zeta = rng.uniform(-0.95, 0.95, n)
    zeta[:8] = [0.0, 0.5, -0.5, 0.9, -0.9, 0.95, -0.95, 0.0]
    up, dn = 0.5 * rho * (1 + zeta), 0.5 * rho * (1 - zeta)
    up[-4:] = dn[-4:] = 1e-12          # below the floor: v = f = 0
    return up, dn


def test_lsda_kernel_matches_oracle():
    up, dn = _densities(4096, 9)
    v, f = P.selftest_xc(np.stack([up, dn]))
    vu, vd = xc.vxc_polarized(up, dn)
    fuu, fud, fdd = xc.fxc_polarized(up, dn)
    for got, ref in ((v[0], vu), (v[1], vd), (f[0], fuu), (f[1], fud), (f[2], fdd)):
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
    assert np.all(v[:, -4:] == 0) and np.all(f[:, -4:] == 0)
    # the spin channels really differ: f_up,up != f_down,down and f_up,down != f_up,up
    assert np.abs(fuu - fdd).max() > 1e-2 * np.abs(fuu).max()


def test_lda_unpolarised_kernel_matches_oracle():
    up, dn = _densities(2048, 10)
    rho = up + dn
    v, f = P.selftest_xc(rho[None, :])
    assert np.allclose(v[0], xc.vxc_unpolarized(rho), rtol=1e-11, atol=1e-14)
    assert np.allclose(f[0], xc.fxc_unpolarized(rho), rtol=1e-11, atol=1e-14 * np.abs(f[0]).max())


@pytest.fixture(scope="module")
def polarised():
    w = W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 1, 1), qmesh=(2, 1, 1))
    m = Model(w)
    rho0 = G.initial_density(m)
    gs = G.scf(m, frozen_vhxc=G.hxc_potential(m, rho0))
    gs.rho = rho0                       # f_xc at the strongly polarised density
    zeta = (rho0[0] - rho0[1]) / rho0.sum(0)
    assert np.abs(zeta).max() > 0.85
    refs = {}
    for iq, J in ((0, m.hub_atoms[0]), (1, m.hub_atoms[5])):
        refs[(iq, J)] = R.solve_column(m, gs, iq, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
    return w, m, gs, refs


@pytest.mark.parametrize("precision", [0, 1])
def test_polarised_response_matches_oracle(polarised, precision):
    w, m, gs, refs = polarised
    kw = dict(cg_tol=1e-12, scf_tol=1e-11, conv_thr_chi=1e-11) if precision == 0 else {}
    ctx = P.Context.from_workload(w, precision=precision, **kw)
    import_ground_state(ctx, m, gs)
    tol = 1e-8 if precision == 0 else 1e-5
    for (iq, J), ref in refs.items():
        dn0, dn, _ = ctx.response(iq, J)
        r0, r1 = oracle_dn_padded(m, ref["dn0"]), oracle_dn_padded(m, ref["dn"])
        assert np.abs(dn0 - r0).max() < tol * np.abs(r0).max()
        assert np.abs(dn - r1).max() < tol * np.abs(r1).max()
        # the two spin channels of the perturbed atom respond differently
        jj = m.hub_atoms.index(J)
        t_up, t_dn = np.trace(r1[jj, 0]).real, np.trace(r1[jj, 1]).real
        assert abs(t_up - t_dn) > 1e-3 * abs(t_up)
