"""Test helpers that move data between the oracle's and the library's layouts (coefficient order
of the wavefunction spheres, padded Delta n arrays).  No arithmetic of the method lives here."""

import numpy as np


def order_map(ctx, model, ik, kfrac=None):
    """perm such that gpu_coeffs = oracle_coeffs[perm] at mesh point ik."""
    mg = ctx.sphere(ik)
    kd = model.kdata(model.kpts[ik] if kfrac is None else kfrac)
    lut = {tuple(m): i for i, m in enumerate(kd.miller)}
    perm = np.array([lut[tuple(m)] for m in mg])
    return perm, kd


def import_ground_state(ctx, model, gs):
    """Loads the oracle's ground state (occupied bands only) into the library."""
    no = model.nocc
    psi = []
    for s in range(model.nspin):
        row = []
        for ik in range(len(model.kpts)):
            perm, _ = order_map(ctx, model, ik)
            row.append(gs.C[s][ik][perm, :no])
        psi.append(row)
    eps = gs.eps[:, :, :no]
    ctx.set_ground_state(model.nspin, model.nelec, gs.vhxc, gs.rho, eps, psi)


def oracle_dn_padded(model, dn, mmax=5):
    """{atom: (nspin, m, m)} -> [nhub_atoms][nspin][mmax][mmax] complex."""
    out = np.zeros((len(model.hub_atoms), model.nspin, mmax, mmax), dtype=complex)
    for i, a in enumerate(model.hub_atoms):
        m = dn[a].shape[-1]
        out[i, :, :m, :m] = dn[a]
    return out
