"""Writes the stored expected values used by the GPU tests.  Calls only the oracle.

    python tests/golden/make_golden.py

tiny_full.json: the two-atom cube at its full size (20 Ry, FFT 20^3, k 2x2x2, q 1x1x1):
oracle ground state (gap, eigenvalues at k = Gamma), chi_0, chi and U of the H atom.

medium_column.json (``python tests/golden/make_golden.py medium``, a few CPU hours): the
medium rocksalt workload at its full size (35 Ry, FFT 36^3, k 4x4x4, q 2x2x2, nspin = 2): the
oracle's ground state (every occupied eigenvalue, the gap, the Hubbard occupations) and one
declared (q, J) column, q = (1/2, 0, 0) and J = the first H atom: Delta_q n^0 and Delta_q n of every
Hubbard atom, both spins, element by element.
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import groundstate as G, hubbard as HB, response as R  # noqa: E402
from oracle.model import Model  # noqa: E402


def tiny_full():
    w = W.tiny()
    m = Model(w)
    gs = G.scf(m, tol=1e-12)
    J = m.hub_atoms[0]
    r = R.solve_column(m, gs, 0, J, tol_cg=1e-13, scf_tol=1e-12, conv_chi=1e-13)
    c0 = HB.trace_column(m, r["dn0"]).real
    c = HB.trace_column(m, r["dn"]).real
    hub = HB.hubbard_matrix(np.array([[c0[0]]]), np.array([[c[0]]]))
    return dict(workload="tiny", gap=gs.gap(), eps_gamma=gs.eps[0, 0, : m.nocc + 1].tolist(),
                chi0=[[float(c0[0])]], chi=[[float(c[0])]], U=float(hub[0, 0]),
                note="oracle: SCF tol 1e-12, CG 1e-13, response SCF 1e-12")


def _cplx(a):
    a = np.asarray(a)
    return [a.real.tolist(), a.imag.tolist()]


def medium_column(iq=4, J=0):
    w = W.medium()
    m = Model(w)
    gs = G.scf(m, tol=1e-12, verbose=True)
    r = R.solve_column(m, gs, iq, J, tol_cg=1e-12, scf_tol=1e-11, conv_chi=1e-12, verbose=True)
    occ = gs.occupations()
    return dict(workload="medium", iq=iq, qfrac=m.qpts[iq].tolist(), J=J, hub_atoms=list(m.hub_atoms),
                gap=gs.gap(), eps=gs.eps[:, :, : m.nocc].tolist(), gs_iterations=gs.iterations,
                gs_residual=gs.residual, occupations={str(a): occ[a].tolist() for a in m.hub_atoms},
                dn0={str(a): _cplx(r["dn0"][a]) for a in m.hub_atoms},
                dn={str(a): _cplx(r["dn"][a]) for a in m.hub_atoms},
                response_iterations=r["iterations"], cg_iterations=r["cg_iterations"],
                note="oracle: ground-state SCF tol 1e-12; response CG 1e-12 per band, SCF 1e-11, "
                     "response traces 1e-12")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "medium":
        name, out = "medium_column.json", medium_column()
    else:
        name, out = "tiny_full.json", tiny_full()
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", name)
