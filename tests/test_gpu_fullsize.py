"""The full medium workload (8.4 bohr rocksalt cube, 4 H + 4 L, nspin = 2, 35 Ry, FFT 36^3, k 4x4x4,
q 2x2x2: 2560 band systems per (q, J)) in the launch configuration the benchmark times, checked
through properties that hold at any size: the full chi_0 and chi from all 64 (q, J) responses of the
mixed form are symmetric (chi_IJ = chi_JI) and negative definite, |chi_II| < |chi_0,II|,
equivalent H sites have equal U, and one (q, J) column agrees with the FP64 form to the mixed
form's bar."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")


def test_medium_full_chi_properties():
    w = W.medium()
    ctx = P.Context.from_workload(w, precision=1)
    ctx.ground_state(w["nelec"], w["nspin"], w["moments"])
    atoms, _ = ctx.hubbard_atoms()
    nq = ctx.query_sizes()["nq"]
    for J in atoms:
        for iq in range(nq):
            ctx.response(iq, int(J))
    chi0, chi, hub = ctx.hubbard()
    for X in (chi0, chi):
        assert np.abs(X - X.T).max() < 1e-5 * np.abs(X).max()
        assert np.linalg.eigvalsh(0.5 * (X + X.T)).max() < 0
    assert np.all(np.abs(np.diag(chi)) < np.abs(np.diag(chi0)))
    # the four H sites of the rocksalt cell are equivalent (antiferromagnetic start relaxes to the
    # same non-magnetic state on each): equal U within the mixed form's 1 meV
    nh = len(atoms)
    u = [hub[s, s] for s in range(nh) if w["atoms"][int(atoms[s])][0] == 0]
    assert len(u) == 4 and max(u) - min(u) < 1e-3
    # one column in FP64 on the same ground state
    _, dn32, _ = ctx.response(1, int(atoms[0]))
    ctx.set_precision(0)
    _, dn64, _ = ctx.response(1, int(atoms[0]))
    assert np.abs(dn32 - dn64).max() < 1e-5 * np.abs(dn64).max()
