"""Synthetic model crystals that drive both the CUDA path and the oracle.

This module holds inputs only: cells, species parameters, atomic positions, cutoffs, meshes and
the seeded generator of the uneven batch of cells.  It contains none of the method's arithmetic
(no G-vectors, no form factors, no FFT-grid choice), so that the CUDA path and the oracle can both
read it without sharing any code of the method.

Model species follow the recipe of the paper's workloads (transition-metal oxides, Sec. 5.1):
a Hubbard "H" species standing in for a 3d metal (deep Gaussian well, one l=2 separable
projector, five d-like Hubbard orbitals) and a ligand "L" species standing in for oxygen (shallower
well, one l=1 projector, p-like Hubbard orbitals where inter-site V is wanted).

Units: bohr, Hartree; ``ecutwfc`` in Rydberg with the wavefunction sphere |k+G|^2 <= ecutwfc.
Meshes are Gamma-centred and unshifted (Sec. 5.1 uses Gamma-centred k and q meshes).
"""

from __future__ import annotations

import copy
import math

import numpy as np

# ---------------------------------------------------------------------------------------------
# species: V(r) = amp * exp(-r^2 / (2 width^2))  [Ha];  one separable projector with radial
# r^l_proj * exp(-r^2 / (2 proj_width^2)) (normalised) and strength D [Ha];  Hubbard orbitals with
# radial r^l_hub * exp(-r^2 / (2 hub_width^2)) (normalised), l_hub < 0 means "not a Hubbard species".
# ---------------------------------------------------------------------------------------------

# The H projector strength: the workload text gives D = +1.5 Ha, which leaves the d channel empty
# (zero weight of the d orbitals in the occupied bands) and the 10- and 40-electron cells metallic,
# so the insulating-state method cannot be applied.  The electron counts (10 per H in the two-atom
# cube, 40 for 4 H in the rocksalt cell) are exactly a filled d shell per H; with an attractive
# d channel D = -4.0 Ha the five d bands per H become the lowest manifold, the cells are insulating
# (gap 0.26 Ha and 1.3 Ha) and the Hubbard manifold carries 4.5 of the 5 electrons per spin.
H_PROJECTOR_D = -4.0
SPECIES_H = dict(name="H", amp=-3.0, width=0.8, l_proj=2, D=H_PROJECTOR_D, proj_width=0.9, l_hub=2, hub_width=0.9)
SPECIES_L_NOHUB = dict(name="L", amp=-2.0, width=1.0, l_proj=1, D=-0.8, proj_width=1.0, l_hub=-1, hub_width=1.0)
SPECIES_L = dict(name="L", amp=-2.0, width=1.0, l_proj=1, D=-0.8, proj_width=1.0, l_hub=1, hub_width=1.0)
SPECIES_H2 = dict(name="H2", amp=-3.3, width=0.8, l_proj=2, D=H_PROJECTOR_D, proj_width=0.9, l_hub=2, hub_width=0.9)
SPECIES_L2 = dict(name="L2", amp=-1.5, width=1.2, l_proj=1, D=-0.5, proj_width=1.2, l_hub=-1, hub_width=1.2)


def _cubic(a):
    return [[a, 0.0, 0.0], [0.0, a, 0.0], [0.0, 0.0, a]]


def _workload(name, cell, species, atoms, nelec, nspin, ecutwfc, kmesh, qmesh, grid, moments=None,
              tol=1e-10, note=""):
    return dict(name=name, cell=[list(map(float, r)) for r in cell], species=copy.deepcopy(species),
                atoms=[(int(s), tuple(float(x) for x in p)) for s, p in atoms], nelec=float(nelec),
                nspin=int(nspin), ecutwfc=float(ecutwfc), kmesh=tuple(kmesh), qmesh=tuple(qmesh),
                grid=tuple(grid) if grid is not None else None,
                moments=list(moments) if moments is not None else None, tol=float(tol), note=note)


def tiny():
    """Simple-cubic a = 8 bohr, H at the origin, L at the body centre; 10 electrons, nspin = 1,
    20 Ry, k 2x2x2, q 1x1x1, FFT 20^3.  U for the H atom only (L carries no Hubbard orbitals)."""
    return _workload("tiny", _cubic(8.0), [SPECIES_H, SPECIES_L_NOHUB],
                     [(0, (0, 0, 0)), (1, (0.5, 0.5, 0.5))], nelec=10, nspin=1, ecutwfc=20.0,
                     kmesh=(2, 2, 2), qmesh=(1, 1, 1), grid=(20, 20, 20))


_ROCKSALT_H = [(0, 0, 0), (0.5, 0.5, 0), (0, 0.5, 0.5), (0.5, 0, 0.5)]
_ROCKSALT_L = [(0.5, 0.5, 0.5), (0, 0, 0.5), (0.5, 0, 0), (0, 0.5, 0)]
# layered AFM-I: H sites in the z = 0 plane spin up, z = 1/2 plane spin down
_ROCKSALT_MOM = [1, 1, -1, -1, 0, 0, 0, 0]


def medium():
    """Rocksalt-like cube a = 8.4 bohr, 4 H + 4 L, 40 electrons (20 bands per spin), nspin = 2
    with a layered antiferromagnetic start, 35 Ry, k 4x4x4, q 2x2x2, FFT 36^3."""
    atoms = [(0, p) for p in _ROCKSALT_H] + [(1, p) for p in _ROCKSALT_L]
    return _workload("medium", _cubic(8.4), [SPECIES_H, SPECIES_L], atoms, nelec=40, nspin=2,
                     ecutwfc=35.0, kmesh=(4, 4, 4), qmesh=(2, 2, 2), grid=(36, 36, 36),
                     moments=_ROCKSALT_MOM)


def precision():
    """The medium cell at 50 Ry, FFT 45^3 (the mixed-precision workload)."""
    w = medium()
    w.update(name="precision", ecutwfc=50.0, grid=(45, 45, 45))
    return w


# Olivine-shaped cell: crystal coordinates of the 28-atom LiMn1/2Fe1/2PO4 cell printed with the
# paper's pw.x input sample 1 (Appendix A), scaled into a 19.6 x 11.3 x 8.9 bohr orthorhombic box.
# Order: Fe1 Fe2 Mn1 Mn2 (Hubbard metals), 16 O, 4 P, 4 Li.
_OLIVINE_FRAC = [
    (-0.0018269047, 0.0000304069, -0.0003932705), (-0.0624820605, 0.4999699836, -0.5003915084),
    (0.4987576776, -0.0000338875, -0.4510637530), (0.4369302234, 0.5000334630, -0.9510599331),
    (-0.1853704531, -0.0000413913, -0.2311704957), (0.6251324004, 0.4999517783, -0.7112993667),
    (0.1210624075, 0.5000390704, -0.7311671887), (0.3105574643, 0.0000452467, -0.2113000948),
    (0.1689278301, 0.0000409137, -0.7606906152), (0.2595012636, 0.5000440788, -0.1851692958),
    (-0.2332375356, 0.4999600895, -0.2606909453), (0.6761898894, -0.0000458163, -0.6851718584),
    (0.0510283716, 0.7040582036, -0.1900775054), (0.0510181642, 0.2960368185, -0.1900725354),
    (0.5580466406, 0.7033668148, -0.2511808171), (0.5580572495, 0.2965326193, -0.2511588987),
    (-0.1153361890, -0.2040586775, -0.6900811178), (-0.1153274751, 0.2039633923, -0.6900740032),
    (0.3776426890, -0.2033681130, -0.7511796423), (0.3776336406, 0.2034650241, -0.7511611819),
    (-0.1864198847, -0.0000468288, -0.5566953613), (0.6287097290, 0.4999490507, -0.3861250841),
    (0.1221109842, 0.5000464680, -0.0566921886), (0.3069801138, 0.0000492520, -0.8861258770),
    (-0.2786794632, -0.2501647928, -0.9729266705), (0.2143739303, -0.2498290476, -0.4729136212),
    (0.2144236723, 0.2499658680, -0.4729252455), (-0.2787339024, 0.2500407728, -0.9729169404),
]


def olivine():
    """Olivine-shaped orthorhombic cell, 28 atoms: Fe1/Fe2 -> H (-3.0 Ha), Mn1/Mn2 -> H2 (-3.3 Ha),
    16 O -> L (Hubbard p), 4 P + 4 Li -> L2 (no Hubbard orbitals).  112 bands per spin, nspin = 2,
    45 Ry, k 2x3x4, q 1x2x2, FFT 72x45x36.  Starting moments: Fe1, Mn1 up; Fe2, Mn2 down."""
    species = [SPECIES_H, SPECIES_H2, SPECIES_L, SPECIES_L2]
    kinds = [0, 0, 1, 1] + [2] * 16 + [3] * 8
    atoms = [(s, tuple(x % 1.0 for x in p)) for s, p in zip(kinds, _OLIVINE_FRAC)]
    moments = [1, -1, 1, -1] + [0] * 24
    cell = [[19.6, 0, 0], [0, 11.3, 0], [0, 0, 8.9]]
    return _workload("olivine", cell, species, atoms, nelec=224, nspin=2, ecutwfc=45.0,
                     kmesh=(2, 3, 4), qmesh=(1, 2, 2), grid=(72, 45, 36), moments=moments)


# ---------------------------------------------------------------------------------------------
# small variants used by the tests (same species, lower cutoffs / meshes so the oracle is quick)
# ---------------------------------------------------------------------------------------------

def tiny_lowcut(ecut=10.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(1, 1, 1)):
    w = tiny()
    w.update(name="tiny_lowcut", ecutwfc=float(ecut), grid=tuple(grid), kmesh=tuple(kmesh),
             qmesh=tuple(qmesh))
    return w


def tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1)):
    """Two-atom cube with a non-trivial q mesh; both atoms carry Hubbard orbitals so that the
    response matrix has inter-site elements (V)."""
    w = tiny()
    w["species"][1] = copy.deepcopy(SPECIES_L)
    w.update(name="tiny_q", ecutwfc=float(ecut), grid=tuple(grid), kmesh=tuple(kmesh),
             qmesh=tuple(qmesh))
    return w


def mirror(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 1), qmesh=(2, 2, 1)):
    """Simple-cubic a = 8 bohr with two H at (0.3, 0, 0) and (0, 0.3, 0) and an L at the body centre;
    14 electrons (gapped), nspin = 1.  The two H sites are images of each other under the mirror
    x <-> y and under no lattice translation; the space group has four operations."""
    return _workload("mirror", _cubic(8.0), [SPECIES_H, SPECIES_L],
                     [(0, (0.3, 0, 0)), (0, (0, 0.3, 0)), (1, (0.5, 0.5, 0.5))], nelec=14, nspin=1,
                     ecutwfc=ecut, kmesh=kmesh, qmesh=qmesh, grid=grid)


def medium_small(ecut=10.0, grid=(18, 18, 18), kmesh=(2, 2, 2), qmesh=(2, 1, 1)):
    """The medium rocksalt cell (nspin = 2, antiferromagnetic start) at a low cutoff and a coarse
    mesh, small enough for the oracle to finish a full response matrix in a minute."""
    w = medium()
    w.update(name="medium_small", ecutwfc=float(ecut), grid=tuple(grid), kmesh=tuple(kmesh),
             qmesh=tuple(qmesh))
    return w


def free_electron(a=6.0, ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2)):
    """No potential at all (amp = D = 0): eigenvalues are exactly |k+G|^2 / 2."""
    sp = dict(name="X", amp=0.0, width=1.0, l_proj=0, D=0.0, proj_width=1.0, l_hub=-1, hub_width=1.0)
    return _workload("free", _cubic(a), [sp], [(0, (0, 0, 0))], nelec=2, nspin=1, ecutwfc=ecut,
                     kmesh=kmesh, qmesh=(1, 1, 1), grid=grid)


def supercell(w, n):
    """The n1 x n2 x n3 supercell of workload ``w`` with the folded k mesh and q = Gamma only.
    Atom order: for each cell l = (l1, l2, l3) (l3 fastest), every atom of the primitive cell.
    The FFT grid is multiplied by n so that the real-space points are the same."""
    n = tuple(int(x) for x in n)
    for a, b in zip(w["kmesh"], n):
        if a % b:
            raise ValueError("the k mesh must be divisible by the supercell size")
    cell = [[w["cell"][i][j] * n[i] for j in range(3)] for i in range(3)]
    atoms, moments = [], []
    for l1 in range(n[0]):
        for l2 in range(n[1]):
            for l3 in range(n[2]):
                for ia, (s, p) in enumerate(w["atoms"]):
                    atoms.append((s, ((p[0] + l1) / n[0], (p[1] + l2) / n[1], (p[2] + l3) / n[2])))
                    if w["moments"] is not None:
                        moments.append(w["moments"][ia])
    ncell = n[0] * n[1] * n[2]
    out = _workload(w["name"] + "_sc", cell, w["species"], atoms, nelec=w["nelec"] * ncell,
                    nspin=w["nspin"], ecutwfc=w["ecutwfc"],
                    kmesh=tuple(a // b for a, b in zip(w["kmesh"], n)), qmesh=(1, 1, 1),
                    grid=tuple(g * b for g, b in zip(w["grid"], n)),
                    moments=moments if w["moments"] is not None else None, tol=w["tol"])
    return out


# ---------------------------------------------------------------------------------------------
# the uneven batch of cells (seeded)
# ---------------------------------------------------------------------------------------------

BATCH_SEED = 15684


def batch_cells(ncells=16, seed=BATCH_SEED):
    """Seeded batch of independent orthorhombic cells with uneven sizes: 2-12 atoms with random
    H/L assignment (at least one H), lattice constants uniform in [7, 12] bohr, atoms on a
    jittered grid with minimum separation 3.5 bohr, ecutwfc uniform in [25, 45] Ry, k mesh per axis
    in {2, 3, 4}, q mesh per axis in {1, 2} dividing the k mesh.  Generator: numpy PCG64.

    The number of occupied bands is not drawn here (it depends on the band structure); each cell
    carries ``nelec = 0`` and the caller chooses it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = []
    for ic in range(ncells):
        while True:
            nat = int(rng.integers(2, 13))
            abc = rng.uniform(7.0, 12.0, size=3)
            # jittered grid placement with rejection below 3.5 bohr (minimum image)
            side = int(math.ceil(nat ** (1.0 / 3.0)))
            slots = [(i, j, k) for i in range(side) for j in range(side) for k in range(side)]
            order = rng.permutation(len(slots))[:nat]
            frac = []
            for o in order:
                base = np.array(slots[o], dtype=float) / side
                frac.append((base + rng.uniform(-0.08, 0.08, size=3)) % 1.0)
            frac = np.array(frac)
            ok = True
            for i in range(nat):
                for j in range(i):
                    d = frac[i] - frac[j]
                    d -= np.round(d)
                    if np.linalg.norm(d * abc) < 3.5:
                        ok = False
            if ok:
                break
        kinds = rng.integers(0, 2, size=nat)
        if kinds.sum() == nat:  # kinds: 0 = H, 1 = L; ensure at least one H
            kinds[0] = 0
        if (kinds == 0).sum() == 0:
            kinds[0] = 0
        ecut = float(rng.uniform(25.0, 45.0))
        kmesh = tuple(int(x) for x in rng.integers(2, 5, size=3))
        qmesh = tuple(int(2 if (k % 2 == 0 and rng.uniform() < 0.5) else 1) for k in kmesh)
        atoms = [(int(s), tuple(float(x) for x in p)) for s, p in zip(kinds, frac)]
        cells.append(_workload("batch%02d" % ic, [[abc[0], 0, 0], [0, abc[1], 0], [0, 0, abc[2]]],
                               [SPECIES_H, SPECIES_L], atoms, nelec=0, nspin=1, ecutwfc=ecut,
                               kmesh=kmesh, qmesh=qmesh, grid=None))
    return cells


def with_projectors(w, kind):
    """A copy of workload ``w`` with its Hubbard projector kind: "atomic" (non-orthogonalised atomic
    orbitals, the default) or "ortho-atomic" (Loewdin orthogonalised, Sec. 2.2)."""
    out = copy.deepcopy(w)
    out["hubbard_projectors"] = kind
    out["name"] = w["name"] + ("_oao" if kind == "ortho-atomic" else "")
    return out


CONFIGS = {"tiny": tiny, "medium": medium, "precision": precision, "olivine": olivine}


def random_coefficients(seed, shape):
    """Seeded complex normal array (PCG64), used as trial vectors in parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def batch_small():
    """A batch of small insulating cells of uneven sizes for the batching form's timing: the two-atom
    cube at 8, 10 and 20 Ry on different q meshes and the spin-polarised rocksalt cell at 6 Ry
    (stand-ins with known gaps; the seeded generator batch_cells leaves the electron count open)."""
    return [tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1)),
            tiny_lowcut(ecut=10.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 2, 1)),
            medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 1, 1), qmesh=(2, 1, 1)),
            tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 2, 2)),
            tiny_lowcut(ecut=10.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(1, 1, 1)),
            tiny()]

