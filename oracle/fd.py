"""Oracle pin: response of SCF Hubbard occupations by central finite differences (the supercell
linear-response cDFT definition the paper's DFPT reproduces, Sec. 2.3, Eq. chi).

Test infrastructure only (see the package docstring).

chi_IJ  = d n^I / d lambda^J with the SCF re-converged under lambda^J sum_m |phi^J_m><phi^J_m|;
chi0_IJ = the same with V_Hxc frozen at its unperturbed value (one non-self-consistent step).
Central differences at +-lambda and +-lambda/2, combined by Richardson extrapolation
(4 d(lambda/2) - d(lambda)) / 3, which removes the O(lambda^2) error.
"""

from __future__ import annotations

import numpy as np

from .groundstate import scf


def _traces(gs):
    t = gs.traces()
    return np.array([t[ia] for ia in gs.model.hub_atoms])


def fd_column(model, J, lam=2e-3, gs0=None, tol=1e-12, bare=False):
    """Column J of chi (or chi_0 with bare=True) by Richardson-extrapolated central differences."""
    if gs0 is None:
        gs0 = scf(model, tol=tol)
    frozen = gs0.vhxc if bare else None

    # a Hubbard-corrected ground state keeps its Hubbard potential fixed: the linear-response problem
    # has no response of the Hubbard potential (Sec. 2.3)
    hub = gs0.hub_occ

    def d(h):
        plus = scf(model, tol=tol, perturb=(J, +h), frozen_vhxc=frozen, vstart=gs0.vhxc, frozen_hub=hub)
        minus = scf(model, tol=tol, perturb=(J, -h), frozen_vhxc=frozen, vstart=gs0.vhxc, frozen_hub=hub)
        return (_traces(plus) - _traces(minus)) / (2.0 * h)

    return (4.0 * d(lam / 2.0) - d(lam)) / 3.0
