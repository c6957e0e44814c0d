"""Writes the stored expected values used by the GPU tests.  Calls only the oracle.

    python tests/golden/make_golden.py

tiny_config0.json: the two-atom cube at its full size (20 Ry, FFT 20^3, k 2x2x2, q 1x1x1):
oracle ground state (gap, eigenvalues at k = Gamma), chi_0, chi and U of the H atom.
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


def tiny_config0():
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


if __name__ == "__main__":
    out = tiny_config0()
    with open(os.path.join(HERE, "tiny_config0.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)
