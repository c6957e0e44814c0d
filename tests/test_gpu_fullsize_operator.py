"""The Sternheimer operator of the response (Eq. LRKSeq_lp, left-hand side) at the benchmark's full
sizes, through exactly the kernels and launch configuration hp_response uses (the fused column /
plane transforms instantiated for 36^3, 45^3 and 72 x 45 x 36, the combined beta / P_v projection
and expansion, FP32 vectors in the mixed form), against the oracle element by element.

Inputs: each workload's own cell, cutoff, meshes and species; a seeded random Hxc potential and
density and seeded random orthonormal occupied states imported through hp_set_ground_state (the
operator does not need a self-consistent state), occupied energies seeded in [-1, -0.3] Ha (alpha =
2 (max - min) of them); 40 random vectors at one k+q point (several band tiles and a ragged tail)
with one shift each.  The olivine-shaped cell runs with nspin = 1 to halve the imported states; its
112 occupied bands with 92 projector rows exceed one projection's 128 rows, so beta and P_v run as
the two-pass projection the benchmark's olivine launches use.

Tolerances: FP64, 1e-11 of the largest element (two FP64 routes, different summation order).
Mixed form: 2e-5 of the largest element.  The FP32 route rounds the inputs to FP32 (u = 2^-24 =
6e-8), adds at most about u per butterfly stage over the 2 log2 N ~ 34 stages of the forward and
inverse transforms, and sums each projection over at most 256 plane waves in FP32 before the FP64
partial sums (<= 256 u): (34 + 256) u ~ 1.7e-5 in the worst case."""

import numpy as np
import pytest

import workloads as W
from oracle.model import Model
from oracle.response import sternheimer_operator

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")

CASES = {
    # workload, nspin used, q index (on the k mesh), k index
    "medium_36": (W.medium, 2, 4, 5),
    "precision_45": (W.precision, 2, 4, 22),
    "olivine_72x45x36": (W.olivine, 1, 1, 7),
}

_built = {}


def _context(name, precision):
    key = (name, precision)
    if key in _built:
        return _built[key]
    make, nspin, iq, ik = CASES[name]
    w = make()
    m = Model(w)
    ctx = P.Context.from_workload(w, precision=precision)
    s = ctx.query_sizes()
    rng = np.random.default_rng(2203)
    nr, nk, no = s["nr"], s["nk"], int(w["nelec"] // 2)
    vhxc = 0.3 * rng.standard_normal((nspin, nr))
    rho = 0.05 * np.abs(rng.standard_normal((nspin, nr)))
    eps = np.sort(rng.uniform(-1.0, -0.3, size=(nspin, nk, no)), axis=2)
    psi = [[np.linalg.qr(W.random_coefficients(1000 * sp + k, (len(ctx.sphere(k)), no)))[0] for k in range(nk)]
           for sp in range(nspin)]
    ctx.set_ground_state(nspin, 2 * no, vhxc, rho, eps, psi)
    _built.clear()
    _built[key] = (w, m, ctx, vhxc, eps, psi)
    return _built[key]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_sternheimer_operator_full_size(name, precision):
    w, m, ctx, vhxc, eps, psi = _context(name, precision)
    _, nspin, iq, ik = CASES[name]
    kp, g0 = m.kq_map(ik, iq)
    assert kp is not None
    kdq = m.kdata(m.kpts[ik] + m.qpts[iq])
    mil = ctx.sphere_kq(iq, ik)
    lut = {tuple(x): i for i, x in enumerate(kdq.miller)}
    perm = np.array([lut[tuple(x)] for x in mil])           # library k+q order -> oracle order
    assert len(perm) == kdq.npw and np.all(np.sort(perm) == np.arange(kdq.npw))
    alpha = 2.0 * (eps.max() - eps.min())
    vloc = m.vloc_r()
    for sp in range(nspin):
        X = W.random_coefficients(77 + sp, (40, kdq.npw))   # rows in the library's k+q order
        shift = np.linspace(-0.9, -0.35, 40)
        got = ctx.apply_sternheimer(iq, ik, sp, shift, X)
        Cq = np.zeros((kdq.npw, psi[sp][kp].shape[1]), dtype=complex)
        Cq[perm] = psi[sp][kp]                               # c_k+q(G) = c_k'(G + G0)
        Xo = np.zeros((kdq.npw, 40), dtype=complex)
        Xo[perm] = X.T
        ref = sternheimer_operator(m, kdq, vloc + vhxc[sp], Cq, alpha, shift, Xo)[perm].T
        tol = 1e-11 if precision == 0 else 2e-5
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < tol, (name, precision, sp, err)
