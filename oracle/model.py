"""Oracle model: cell, reciprocal lattice, G-spheres, FFT-grid maps and closed-form form factors.

Test infrastructure only (see the package docstring).

Conventions (Hartree atomic units; the paper uses Hartree units, Sec. 1):
  * lattice vectors are the rows of ``cell``; b_i . a_j = 2 pi delta_ij;
  * the wavefunction sphere at k is {G : |k+G|^2 <= ecutwfc[Ry]};
  * a lattice-periodic function u(r) = sum_G c(G) exp(iG.r), normalised sum |c|^2 = 1 so that
    u_{nk}(r) has unit norm per cell (the 1/sqrt(Omega) is kept out of the coefficients and put
    into the density normalisation);
  * grid point j = (j1, j2, j3) sits at r_j = sum_i (j_i / N_i) a_i and is stored row-major,
    flat index (j1 * N2 + j2) * N3 + j3.
"""

from __future__ import annotations

import math

import numpy as np

HA_TO_EV = 27.211386245988  # CODATA 2018


def real_ylm(l, vec):
    """Real spherical harmonics Y_lm(vec/|vec|), m in a fixed order, for l = 0, 1, 2.

    Returns an array (2l+1, n).  At vec = 0 the l > 0 harmonics are set to 0 (the radial factor
    g^l vanishes there anyway)."""
    vec = np.atleast_2d(np.asarray(vec, dtype=float))
    r = np.linalg.norm(vec, axis=1)
    safe = np.where(r > 0, r, 1.0)
    x, y, z = vec[:, 0] / safe, vec[:, 1] / safe, vec[:, 2] / safe
    zero = r == 0
    if l == 0:
        return np.full((1, len(r)), 0.5 / math.sqrt(math.pi))
    if l == 1:
        c = math.sqrt(3.0 / (4.0 * math.pi))
        out = c * np.stack([x, y, z])
    elif l == 2:
        c1 = math.sqrt(15.0 / (4.0 * math.pi))
        c0 = math.sqrt(5.0 / (16.0 * math.pi))
        c2 = math.sqrt(15.0 / (16.0 * math.pi))
        out = np.stack([c1 * x * y, c1 * y * z, c0 * (3 * z * z - 1.0), c1 * x * z, c2 * (x * x - y * y)])
    else:
        raise ValueError("l > 2 not supported")
    out[:, zero] = 0.0
    return out


def radial_norm(l, s):
    """N such that int_0^inf r^2 [N r^l exp(-r^2/(2 s^2))]^2 dr = 1."""
    return math.sqrt(2.0 / (math.gamma(l + 1.5) * s ** (2 * l + 3)))


def radial_transform(l, s, g):
    """F_l(g) = int_0^inf r^2 R(r) j_l(g r) dr for the normalised R(r) = N r^l exp(-r^2/(2 s^2)).

    Closed form: N sqrt(pi/2) s^(2l+3) g^l exp(-g^2 s^2 / 2)."""
    g = np.asarray(g, dtype=float)
    return radial_norm(l, s) * math.sqrt(math.pi / 2.0) * s ** (2 * l + 3) * g ** l * np.exp(-0.5 * g * g * s * s)


def good_fft_size(n):
    """Smallest m >= n whose prime factors are 2, 3 and 5."""
    m = max(1, int(n))
    while True:
        k = m
        for p in (2, 3, 5):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 1


def lowdin_orthonormalize(phi):
    """Loewdin ortho-atomic orbitals (Sec. 2.2, Eq. OAO_def) from the rows of ``phi`` (orbitals x plane
    waves at one k): O_ab = <phi_a|phi_b>, phi~_b = sum_a phi_a (O^-1/2)_ab, with O^-1/2 from the
    eigen-decomposition of the Hermitian O.  Every orbital of every atom in the set takes part."""
    O = phi.conj() @ phi.T
    w, V = np.linalg.eigh(O)
    Sinv = (V * (w ** -0.5)[None, :]) @ V.conj().T
    return Sinv.T @ phi


class KData:
    """Per-k (or per-(k+q)) basis data: sphere, kinetic energies, grid map, projectors."""

    def __init__(self, model, kfrac):
        self.kfrac = np.asarray(kfrac, dtype=float)
        self.kcart = self.kfrac @ model.bvec
        self.miller = model.sphere_miller(self.kfrac)
        self.K = self.kcart[None, :] + self.miller @ model.bvec
        self.g2 = np.einsum("ij,ij->i", self.K, self.K)
        self.npw = len(self.g2)
        N = model.grid
        m = self.miller
        self.idx = ((m[:, 0] % N[0]) * N[1] + (m[:, 1] % N[1])) * N[2] + (m[:, 2] % N[2])
        if len(np.unique(self.idx)) != self.npw:
            raise ValueError("FFT grid too small to hold the wavefunction sphere")
        self.beta = model.projectors(self.K)          # (nproj, npw)
        self.phi = model.hubbard_orbitals(self.K)     # (nhub, npw)
        if model.ortho_atomic:
            self.phi = lowdin_orthonormalize(self.phi)


class Model:
    """A periodic model crystal built from a workload dictionary (see ``workloads``)."""

    def __init__(self, w):
        self.w = w
        self.cell = np.array(w["cell"], dtype=float)
        self.omega = abs(np.linalg.det(self.cell))
        self.bvec = 2.0 * math.pi * np.linalg.inv(self.cell).T
        self.species = w["species"]
        self.atom_species = [s for s, _ in w["atoms"]]
        self.frac = np.array([p for _, p in w["atoms"]], dtype=float)
        self.tau = self.frac @ self.cell
        self.nat = len(self.atom_species)
        self.ecut = float(w["ecutwfc"])
        self.nspin = int(w["nspin"])
        self.nelec = float(w["nelec"])
        self.nocc = int(round(self.nelec / 2.0))  # bands per spin channel (tot_mag = 0)
        self.kmesh = tuple(w["kmesh"])
        self.qmesh = tuple(w["qmesh"])
        self.grid = tuple(w["grid"]) if w.get("grid") else self.auto_grid()
        self.nr = int(np.prod(self.grid))
        self.kpts = self.mesh_points(self.kmesh)
        self.qpts = self.mesh_points(self.qmesh)
        self.moments = w.get("moments")
        # Hubbard projectors (Sec. 2.2): non-orthogonalised atomic orbitals, or Loewdin ortho-atomic
        # orbitals orthogonalised over every orbital of every atom that carries one (Eq. OAO_def)
        proj = w.get("hubbard_projectors", "atomic")
        if proj not in ("atomic", "ortho-atomic"):
            raise ValueError("hubbard_projectors must be 'atomic' or 'ortho-atomic'")
        self.ortho_atomic = proj == "ortho-atomic"
        # separable projectors: one (l_proj) channel per atom, 2l+1 components
        self.proj_atom, self.proj_l, self.proj_m, self.proj_D = [], [], [], []
        for ia, s in enumerate(self.atom_species):
            sp = self.species[s]
            for m in range(2 * sp["l_proj"] + 1):
                self.proj_atom.append(ia)
                self.proj_l.append(sp["l_proj"])
                self.proj_m.append(m)
                self.proj_D.append(sp["D"])
        self.proj_D = np.array(self.proj_D)
        # Hubbard atoms and their orbital slices
        self.hub_atoms = [ia for ia, s in enumerate(self.atom_species) if self.species[s]["l_hub"] >= 0]
        self.hub_slice = {}
        off = 0
        for ia in self.hub_atoms:
            nm = 2 * self.species[self.atom_species[ia]]["l_hub"] + 1
            self.hub_slice[ia] = slice(off, off + nm)
            off += nm
        self.nhub = off
        self.gvec_cache = {}

    # ------------------------------------------------------------------ meshes and spheres
    @staticmethod
    def mesh_points(n):
        """Gamma-centred unshifted mesh, index (i1 * n2 + i2) * n3 + i3, k = i / n (crystal)."""
        pts = []
        for i1 in range(n[0]):
            for i2 in range(n[1]):
                for i3 in range(n[2]):
                    pts.append((i1 / n[0], i2 / n[1], i3 / n[2]))
        return np.array(pts, dtype=float)

    def sphere_miller(self, kfrac):
        """All Miller triples m with |k + m.B|^2 <= ecut, sorted by (|k+G|^2, m) for determinism."""
        kc = np.asarray(kfrac) @ self.bvec
        gmax = math.sqrt(self.ecut) + np.linalg.norm(kc)
        # bound on |m_i|: |m_i| <= gmax * |a_i| / (2 pi)
        lim = [int(math.ceil(gmax * np.linalg.norm(self.cell[i]) / (2 * math.pi))) + 1 for i in range(3)]
        r = [np.arange(-L, L + 1) for L in lim]
        m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
        K = kc[None, :] + m @ self.bvec
        g2 = np.einsum("ij,ij->i", K, K)
        keep = g2 <= self.ecut
        m, g2 = m[keep], g2[keep]
        order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], np.round(g2, 12)))
        return m[order]

    def auto_grid(self):
        """Alias-free grid: N_i >= 4 max|m_i| + 1 with max|m_i| the largest Miller index along i of
        the density sphere |G|^2 <= 4 ecut, rounded up to a 2-3-5 size."""
        out = []
        for i in range(3):
            mmax = int(math.floor(2.0 * math.sqrt(self.ecut) * np.linalg.norm(self.cell[i]) / (2 * math.pi)))
            out.append(good_fft_size(2 * mmax + 1))
        return tuple(out)

    def kdata(self, kfrac):
        return KData(self, kfrac)

    # ------------------------------------------------------------------ grid G-vectors
    def grid_gvectors(self, qfrac=(0.0, 0.0, 0.0)):
        """For every grid index: the cartesian vector q+G of its representative Miller index and a
        mask of the vectors kept in potentials.

        The representative m_i of grid index j_i is the one with m_i + q_i in the open interval
        (-N_i/2, N_i/2); grid indices with no such representative (the Nyquist plane at q_i = 0 on
        even grids) are masked out, as is every vector with |q+G|^2 > 4 ecutwfc.  The same rule
        applied to an n-fold supercell with grid n*N selects exactly the union of the cell's
        q+G sets, and at q = 0 it is inversion symmetric, so potentials stay real."""
        key = tuple(np.round(np.asarray(qfrac, dtype=float), 14))
        if key in self.gvec_cache:
            return self.gvec_cache[key]
        reps, oks = [], []
        for i in range(3):
            N = self.grid[i]
            j = np.arange(N)
            qi = float(qfrac[i])
            # candidate representative: j or j - N, choose m with m + q in (-N/2, N/2)
            m = np.where(j + qi < N / 2.0, j, j - N).astype(float)
            ok = (m + qi > -N / 2.0) & (m + qi < N / 2.0)
            reps.append(m)
            oks.append(ok)
        M = np.stack(np.meshgrid(*reps, indexing="ij"), axis=-1).reshape(-1, 3)
        OK = (oks[0][:, None, None] & oks[1][None, :, None] & oks[2][None, None, :]).reshape(-1)
        QG = (M + np.asarray(qfrac, dtype=float)[None, :]) @ self.bvec
        g2 = np.einsum("ij,ij->i", QG, QG)
        mask = OK & (g2 <= 4.0 * self.ecut)
        self.gvec_cache[key] = (QG, g2, mask)
        return QG, g2, mask

    # ------------------------------------------------------------------ form factors
    def vloc_g(self):
        """V_loc(G) on the grid (flat), Sec. 2 model: each atom contributes a Gaussian well
        A exp(-r^2/(2 w^2)) whose Fourier coefficient per cell is
        (1/Omega) A (2 pi w^2)^(3/2) exp(-G^2 w^2 / 2) exp(-i G.tau); zero outside the mask."""
        G, g2, mask = self.grid_gvectors()
        out = np.zeros(self.nr, dtype=complex)
        for ia, s in enumerate(self.atom_species):
            sp = self.species[s]
            A, w = sp["amp"], sp["width"]
            out += (A * (2 * math.pi * w * w) ** 1.5 / self.omega) * np.exp(-0.5 * g2 * w * w) * np.exp(-1j * (G @ self.tau[ia]))
        out[~mask] = 0.0
        return out

    def vloc_r(self):
        """V_loc(r) on the grid: sum_G V(G) exp(iG.r) (real by construction)."""
        vg = self.vloc_g().reshape(self.grid)
        vr = np.fft.ifftn(vg) * self.nr
        return vr.real.reshape(-1).copy()

    def _atomic_ft(self, K, ia, l, s):
        """PW coefficients <k+G|f> of f(r) = R(|r - tau|) Y_lm(r - tau) with the normalised radial
        R = N r^l exp(-r^2/(2 s^2)), using exp(-iK.r) = 4 pi sum_lm (-i)^l j_l(Kr) Y_lm(K) Y_lm(r):
        (4 pi / sqrt(Omega)) (-i)^l Y_lm(K) F_l(|K|) exp(-i K.tau)."""
        g = np.sqrt(np.einsum("ij,ij->i", K, K))
        Y = real_ylm(l, K)
        F = radial_transform(l, s, g)
        ph = np.exp(-1j * (K @ self.tau[ia]))
        return (4 * math.pi / math.sqrt(self.omega)) * ((-1j) ** l) * Y * (F * ph)[None, :]

    def projectors(self, K):
        rows = []
        for ia, s in enumerate(self.atom_species):
            sp = self.species[s]
            rows.append(self._atomic_ft(K, ia, sp["l_proj"], sp["proj_width"]))
        return np.concatenate(rows, axis=0) if rows else np.zeros((0, len(K)), dtype=complex)

    def hubbard_orbitals(self, K):
        rows = []
        for ia in self.hub_atoms:
            sp = self.species[self.atom_species[ia]]
            rows.append(self._atomic_ft(K, ia, sp["l_hub"], sp["hub_width"]))
        return np.concatenate(rows, axis=0) if rows else np.zeros((0, len(K)), dtype=complex)

    # ------------------------------------------------------------------ k + q bookkeeping
    def kq_map(self, ik, iq):
        """k + q = k' + G0 for Gamma-centred meshes with q mesh dividing k mesh.  Returns (k', G0)
        or (None, None) when k + q is off the k mesh."""
        k = self.kpts[ik]
        q = self.qpts[iq]
        kq = k + q
        idx, g0 = [], []
        for i in range(3):
            x = kq[i] * self.kmesh[i]
            xi = int(round(x))
            if abs(x - xi) > 1e-9:
                return None, None
            idx.append(xi % self.kmesh[i])
            g0.append((xi - idx[-1]) // self.kmesh[i])
        kp = (idx[0] * self.kmesh[1] + idx[1]) * self.kmesh[2] + idx[2]
        return kp, np.array(g0, dtype=int)

    def supercell_R(self):
        """Lattice vectors R_l (crystal units) of the cells of the supercell matching the q mesh,
        l = (l1 * n2 + l2) * n3 + l3."""
        n = self.qmesh
        return np.array([(l1, l2, l3) for l1 in range(n[0]) for l2 in range(n[1]) for l3 in range(n[2])],
                        dtype=float)
