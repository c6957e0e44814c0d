"""Pins of the oracle's building blocks against closed forms, brute force and independent routes.

Each test is chosen so that a plausible slip in the oracle (a dropped factor, a wrong sign, a
transposed operand, a wrong FFT normalisation) fails it."""

import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import workloads as W
from oracle import xc
from oracle.hamiltonian import apply_h, dense_h, from_grid, hartree_r, to_grid
from oracle.mixing import Broyden
from oracle.model import Model, radial_norm, radial_transform, real_ylm

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ------------------------------------------------------------------ angular / radial parts

def _sphere_quadrature(n=24):
    """Gauss-Legendre in cos(theta) x uniform phi: exact for polynomials of degree < 2n."""
    x, wx = np.polynomial.legendre.leggauss(n)
    phi = np.arange(2 * n) * (math.pi / n)
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    w = (wx[:, None] * np.full(2 * n, math.pi / n)[None, :]).reshape(-1)
    return pts, w


@pytest.mark.parametrize("l", [0, 1, 2])
def test_real_ylm_orthonormal(l):
    pts, w = _sphere_quadrature()
    Y = real_ylm(l, pts)
    G = (Y * w[None, :]) @ Y.T
    assert np.allclose(G, np.eye(2 * l + 1), atol=1e-13)


def test_real_ylm_l_mixing_zero():
    pts, w = _sphere_quadrature()
    for a in range(3):
        for b in range(a + 1, 3):
            assert np.abs((real_ylm(a, pts) * w) @ real_ylm(b, pts).T).max() < 1e-13


@pytest.mark.parametrize("l,s", [(0, 0.8), (1, 1.0), (2, 0.9), (1, 1.2)])
def test_radial_norm_and_transform_vs_quadrature(l, s):
    N = radial_norm(l, s)
    R = lambda r: N * r ** l * np.exp(-r * r / (2 * s * s))
    norm = scipy.integrate.quad(lambda r: r * r * R(r) ** 2, 0, 40 * s)[0]
    assert abs(norm - 1.0) < 1e-12
    for g in [0.0, 0.3, 1.1, 2.7, 5.0]:
        ref = scipy.integrate.quad(lambda r: r * r * R(r) * scipy.special.spherical_jn(l, g * r), 0, 40 * s,
                                   limit=400)[0]
        assert abs(radial_transform(l, s, g) - ref) < 1e-11


def test_plane_wave_expansion_of_projector():
    """<k+G|beta> from the closed form equals a brute-force real-space integral over the cell of
    the Bloch sum (isolated Gaussian in a large box)."""
    w = W.free_electron(a=14.0, ecut=1.2, grid=(28, 28, 28))
    w["species"][0].update(l_proj=2, proj_width=0.9)
    w["atoms"] = [(0, (0.31, 0.27, 0.55))]
    m = Model(w)
    kd = m.kdata((0.5, 0.0, 0.25))
    N = m.grid
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    r = j @ m.cell
    d = r - m.tau[0]
    d -= np.round(d / 14.0) * 14.0        # minimum image: the function is negligible beyond a/2
    dist = np.linalg.norm(d, axis=1)
    sp = m.species[0]
    Rr = radial_norm(2, 0.9) * dist ** 2 * np.exp(-dist ** 2 / (2 * 0.81))
    f = Rr[None, :] * real_ylm(2, d)               # beta_m(r - tau), (5, nr)
    # <k+G|beta> = (1/sqrt(Omega)) int exp(-i(k+G).r) beta(r - tau) d^3r  (quadrature on the grid)
    K = kd.K
    ph = np.exp(-1j * (K @ (m.tau[0] + d).T))      # (npw, nr), r = tau + d
    brute = (f @ ph.T) * (m.omega / m.nr) / math.sqrt(m.omega)
    assert np.abs(brute - kd.beta).max() < 2e-6 * np.abs(kd.beta).max()


# ------------------------------------------------------------------ grids and the operator

@pytest.fixture(scope="module")
def small_model():
    return Model(W.tiny_lowcut(ecut=6.0, grid=(10, 10, 10)))


def test_fft_conventions_vs_direct_sum(small_model):
    m = small_model
    kd = m.kdata(m.kpts[3])
    rng = np.random.default_rng(1)
    C = rng.standard_normal((kd.npw, 2)) + 1j * rng.standard_normal((kd.npw, 2))
    N = m.grid
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    E = np.exp(2j * math.pi * (j @ kd.miller.T))       # exp(i G . r_j), (nr, npw)
    assert np.allclose(to_grid(m, kd, C).T, E @ C, atol=1e-11)
    F = rng.standard_normal((2, m.nr)) + 1j * rng.standard_normal((2, m.nr))
    assert np.allclose(from_grid(m, kd, F), (E.conj().T @ F.T) / m.nr, atol=1e-12)


def test_h_fft_equals_dense_and_hermitian(small_model):
    m = small_model
    kd = m.kdata(m.kpts[5])
    rng = np.random.default_rng(2)
    vr = rng.standard_normal(m.nr)
    C = rng.standard_normal((kd.npw, 3)) + 1j * rng.standard_normal((kd.npw, 3))
    H = dense_h(m, kd, vr)
    assert np.abs(H - H.conj().T).max() < 1e-12
    assert np.allclose(apply_h(m, kd, vr, C), H @ C, atol=1e-10)
    a, b = C[:, :1], C[:, 1:2]
    lhs = np.vdot(a, apply_h(m, kd, vr, b))
    rhs = np.conj(np.vdot(b, apply_h(m, kd, vr, a)))
    assert abs(lhs - rhs) < 1e-10


def test_local_potential_matches_real_space_gaussians():
    """V_loc(r) from the G-space closed form equals the periodic sum of the Gaussian wells in real
    space (high cutoff, so that the truncation of the G set is negligible)."""
    w = W.tiny_lowcut(ecut=40.0, grid=(40, 40, 40))
    m = Model(w)
    vr = m.vloc_r()
    N = m.grid
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    ref = np.zeros(m.nr)
    for ia, s in enumerate(m.atom_species):
        sp = m.species[s]
        for n1 in (-1, 0, 1):
            for n2 in (-1, 0, 1):
                for n3 in (-1, 0, 1):
                    d = (j - m.frac[ia] + np.array([n1, n2, n3])) @ m.cell
                    ref += sp["amp"] * np.exp(-np.einsum("ij,ij->i", d, d) / (2 * sp["width"] ** 2))
    assert np.abs(vr - ref).max() < 1e-6


def test_free_electron_eigenvalues():
    m = Model(W.free_electron())
    for k in m.kpts:
        kd = m.kdata(k)
        e = np.linalg.eigvalsh(dense_h(m, kd, np.zeros(m.nr)))
        assert np.allclose(np.sort(e), np.sort(0.5 * kd.g2), atol=1e-12)


def test_hartree_of_gaussian_charge():
    """Neutralised Gaussian charge in a big cube: V(r) - V(0) = erf(r/(sqrt2 s))/r - sqrt(2/pi)/s
    + (2 pi / (3 Omega)) r^2 + O(r^4 / a^5): the uniform compensating charge -1/Omega solves
    lap V = 4 pi / Omega, and the cubic array of images adds only a constant and r^4 terms."""
    a, s = 20.0, 0.5
    w = W.free_electron(a=a, ecut=30.0, grid=(72, 72, 72))
    m = Model(w)
    N = m.grid
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    d = (j - np.round(j)) @ m.cell
    r = np.linalg.norm(d, axis=1)
    rho = np.exp(-r * r / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    rho -= rho.sum() / m.nr              # neutralising background (drops G = 0 exactly)
    v = hartree_r(m, rho).real
    i0 = int(np.argmin(r))
    for rr in (1.0, 1.5, 2.0):
        i = int(np.argmin(np.abs(r - rr) + 10 * (np.abs(d[:, 1]) + np.abs(d[:, 2]))))
        x = r[i]
        ref = math.erf(x / (math.sqrt(2) * s)) / x - math.sqrt(2 / math.pi) / s + 2 * math.pi / (3 * m.omega) * x * x
        assert abs((v[i] - v[i0]) - ref) < 2e-5


def test_grid_mask_rule_supercell_consistent():
    """The potential G-set of the cell at q = 0 and q = b1/2 is exactly the supercell's set."""
    w = W.tiny_q(ecut=8.0, grid=(12, 12, 12), qmesh=(2, 1, 1))
    m = Model(w)
    ms = Model(W.supercell(w, (2, 1, 1)))
    QGs, g2s, masks = ms.grid_gvectors()
    sc = set(map(tuple, np.round(QGs[masks], 9)))
    cell = set()
    for q in m.qpts:
        QG, g2, mask = m.grid_gvectors(q)
        cell |= set(map(tuple, np.round(QG[mask], 9)))
    assert cell == sc


# ------------------------------------------------------------------ LDA

def _vc_pz81_published(rs, p):
    """PZ81 correlation potential in the closed form printed by Perdew & Zunger (1981)."""
    if rs >= 1:
        sq = math.sqrt(rs)
        return p["gamma"] * (1 + 7 / 6 * p["beta1"] * sq + 4 / 3 * p["beta2"] * rs) / (1 + p["beta1"] * sq + p["beta2"] * rs) ** 2
    return (p["A"] * math.log(rs) + (p["B"] - p["A"] / 3) + 2 / 3 * p["C"] * rs * math.log(rs)
            + (2 * p["D"] - p["C"]) / 3 * rs)


@pytest.mark.parametrize("rho", [1e-4, 3e-3, 0.02, 0.1, 0.6, 3.0])
def test_lda_unpolarised_vs_published_forms(rho):
    rs = (3 / (4 * math.pi * rho)) ** (1 / 3)
    vx = -(3 / math.pi) ** (1 / 3) * rho ** (1 / 3)
    ref = vx + _vc_pz81_published(rs, xc.PZ_U)
    assert abs(xc.vxc_unpolarized(np.array([rho]))[0] - ref) < 1e-13 * max(1, abs(ref))


def test_lda_fully_polarised_exchange_and_pz_p():
    rho = 0.05
    rs = (3 / (4 * math.pi * rho)) ** (1 / 3)
    vu, _ = xc.vxc_polarized(np.array([rho * (1 - 1e-13)]), np.array([rho * 1e-13]))
    ref = -(6 / math.pi) ** (1 / 3) * rho ** (1 / 3) + _vc_pz81_published(rs, xc.PZ_P)
    assert abs(vu[0] - ref) < 1e-6


def test_pz81_continuity_at_rs1():
    e_lo = xc.eps_derivs(np.array([1 - 1e-9]), np.array([0.0]))[0][0]
    e_hi = xc.eps_derivs(np.array([1 + 1e-9]), np.array([0.0]))[0][0]
    assert abs(e_lo - e_hi) < 1e-4  # PZ81 is continuous to the digits of its parameters


def test_vxc_is_derivative_of_energy_and_fxc_of_vxc():
    rng = np.random.default_rng(3)
    ru = rng.uniform(0.002, 0.4, 20)
    rd = rng.uniform(0.002, 0.4, 20)
    h = 1e-6
    vu, vd = xc.vxc_polarized(ru, rd)
    e = lambda a, b: xc.exc_density(a, b)
    assert np.allclose(vu, (e(ru * (1 + h), rd) - e(ru * (1 - h), rd)) / (2 * h * ru), rtol=1e-7, atol=1e-9)
    assert np.allclose(vd, (e(ru, rd * (1 + h)) - e(ru, rd * (1 - h))) / (2 * h * rd), rtol=1e-7, atol=1e-9)
    fuu, fud, fdd = xc.fxc_polarized(ru, rd)
    vp = xc.vxc_polarized(ru * (1 + h), rd)
    vm = xc.vxc_polarized(ru * (1 - h), rd)
    assert np.allclose(fuu, (vp[0] - vm[0]) / (2 * h * ru), rtol=1e-6)
    assert np.allclose(fud, (vp[1] - vm[1]) / (2 * h * ru), rtol=1e-6)
    vp = xc.vxc_polarized(ru, rd * (1 + h))
    vm = xc.vxc_polarized(ru, rd * (1 - h))
    assert np.allclose(fdd, (vp[1] - vm[1]) / (2 * h * rd), rtol=1e-6)
    assert np.allclose(fud, (vp[0] - vm[0]) / (2 * h * rd), rtol=1e-6)
    r = rng.uniform(0.002, 0.8, 20)
    f = xc.fxc_unpolarized(r)
    assert np.allclose(f, (xc.vxc_unpolarized(r * (1 + h)) - xc.vxc_unpolarized(r * (1 - h))) / (2 * h * r), rtol=1e-6)
    # the spin-resolved kernel reduces to the unpolarised one for equal spin densities
    fuu, fud, _ = xc.fxc_polarized(r / 2, r / 2)
    assert np.allclose(0.5 * (fuu + fud), f, rtol=1e-10)
    vu, _ = xc.vxc_polarized(r / 2, r / 2)
    assert np.allclose(vu, xc.vxc_unpolarized(r), rtol=1e-12)


# ------------------------------------------------------------------ mixing

def test_broyden_reaches_fixed_point_of_linear_map():
    rng = np.random.default_rng(4)
    n = 30
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    M = Q @ np.diag(rng.uniform(-0.9, 0.9, n)) @ Q.T
    c = rng.standard_normal(n)
    exact = np.linalg.solve(np.eye(n) - M, c)
    mix = Broyden(alpha=0.3, nmix=4)
    x = np.zeros(n)
    for _ in range(200):
        f = M @ x + c - x
        if np.linalg.norm(f) < 1e-13:
            break
        x = mix.step(x, f)
    assert np.linalg.norm(x - exact) < 1e-11
