/*
 * hp.h -- C ABI of the GB300 DFPT Hubbard-parameter engine (arXiv:2203.15684, the "HP" method).
 *
 * The library computes the bare and self-consistent occupation-response matrices chi_0 and chi of
 * the Hubbard manifolds of a periodic crystal by density-functional perturbation theory, and from
 * them the Hubbard U and V (Sec. 2.3, Eqs. chi, U_def, V_def).  For every perturbed Hubbard atom J
 * and wavevector q of a Gamma-centred q mesh it solves the self-consistent q-specific static
 * Sternheimer problem (Eq. LRKSeq_lp) over all occupied bands of all k points, accumulates the
 * response occupations (Eq. occ_matrix_response_lp_2) and sums the q components with phases
 * (Eq. occ_matrix_response_lp_1).  All of it runs in CUDA kernels on one GPU (sm_103a).
 *
 * Model: norm-conserving-like model species (a Gaussian local well, one separable projector of
 * angular momentum l_proj, optional Hubbard orbitals of angular momentum l_hub), plane waves
 * |k+G|^2 <= ecutwfc [Ry], LDA (Slater + Perdew-Zunger 1981), fixed occupations (insulators),
 * nspin = 1 or collinear nspin = 2 with tot_magnetization = 0.
 *
 * Conventions
 *   - Every function returns hp_status; nothing throws or exits across the ABI.  The message of
 *     the last failure is kept in the context (hp_last_error).
 *   - Host buffers are owned by the caller; the library copies what it reads before returning and
 *     writes outputs only on HP_OK (HP_ENOTCONV also fills the partial result).  The library owns
 *     every device allocation it makes and frees it in hp_destroy.
 *   - Complex arrays are interleaved (re, im) FP64.  Units: bohr, Hartree; ecutwfc in Ry; chi in
 *     electrons per Ha; U and V in eV (1 Ha = 27.211386245988 eV).
 *   - Meshes: Gamma-centred, unshifted; point index (i1*n2 + i2)*n3 + i3, crystal coordinate i/n.
 *   - Real-space grid: point (j1, j2, j3) at sum_i (j_i/N_i) a_i, flat index (j1*N2 + j2)*N3 + j3.
 *   - A lattice-periodic function u(r) = sum_G c(G) exp(iG.r) with sum |c|^2 = 1.
 *   - Work is issued on the stream given in hp_options.cuda_stream (0 = legacy default stream);
 *     every call synchronises that stream before returning host results.
 *
 * Environment (read at hp_setup unless noted; for tests and diagnostics, results are the same
 * within the stated tolerances):
 *   HP_NO_FUSED     use the batched 3D FFT with scatter/gather instead of the fused column/plane
 *                   transforms (the fallback taken anyway for grids the fused kernels do not cover)
 *   HP_FUSED_SMEM   fused transforms with shared-memory line FFTs instead of register-resident ones
 *   HP_PROJ_ROWS    at most this many rows (<= 128) in one combined beta / P_v projection
 *   HP_PROF_LOG     file receiving one line per timed launch while profiling (hp_profile_begin)
 *   HP_VERBOSE      progress of the ground state, the k+q eigensolver and the response on stderr
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hp_ctx hp_ctx;

typedef enum {
    HP_OK = 0,
    HP_EINVAL = 1,      /* an argument is out of range or inconsistent */
    HP_ENOMEM = 2,      /* a device or host allocation failed */
    HP_ESTATE = 3,      /* called out of order (e.g. hp_response before a ground state) */
    HP_ENOTCONV = 4,    /* an iteration hit its cap; partial results are filled in */
    HP_ENUMERIC = 5,    /* NaN/Inf met in an FP64 scalar */
    HP_ECUDA = 6,       /* a CUDA runtime call failed (message in hp_last_error) */
    HP_ETIMEOUT = 7,    /* a bounded device-side wait ran out (hp_options.wait_timeout_s) */
    HP_ESINGULAR = 8,   /* chi_0 or chi is singular or its 1-norm condition number exceeds 1e10 */
    HP_ENOGAP = 9,      /* the ground state has no gap (<= 1e-4 Ha) at the fixed band count */
    HP_ENOTIMPL = 10    /* the requested form is not available */
} hp_status;

/* One model species.  V_loc(r) = amp * exp(-r^2 / (2 width^2)) [Ha, bohr]; one separable projector
 * |beta_lm> D <beta_lm| with radial r^l_proj exp(-r^2 / (2 proj_width^2)) normalised to
 * int r^2 R^2 dr = 1 (D in Ha; D = 0 switches it off); Hubbard orbitals phi_lm with radial
 * r^l_hub exp(-r^2 / (2 hub_width^2)), normalised the same way, l_hub < 0: not a Hubbard species.
 * 0 <= l_proj, l_hub <= 2. */
typedef struct {
    double amp, width;
    int l_proj;
    double D, proj_width;
    int l_hub;
    double hub_width;
} hp_species;

#define HP_PRECISION_FP64 0
#define HP_PRECISION_MIXED 1

typedef struct {
    int precision;          /* HP_PRECISION_FP64, or HP_PRECISION_MIXED: FFTs, grid work and the
                               projections in FP32, band vectors, CG scalars, mixing and chi in FP64;
                               CG and SCF stop at 1e-7 of the FP32 noise floor (U, V to < 1 meV) */
    double cg_tol;          /* Sternheimer CG: stop a band when ||r_v||_2 <= cg_tol (1e-11) */
    int cg_maxiter;         /* per outer iteration (default 400) */
    double scf_tol;         /* response SCF: rms of dV_out - dV_in below this (1e-10) ...      */
    double conv_thr_chi;    /* ... and every response trace changed by less than this (1e-10) */
    int niter_max;          /* outer iterations (default 100, as the paper's niter_max) */
    int nmix;               /* modified Broyden history (default 4) */
    double alpha_mix;       /* mixing parameter (default 0.3) */
    double gs_tol;          /* ground-state SCF: rms residual of V_Hxc (default 1e-11) */
    int gs_maxiter;         /* ground-state SCF iterations (default 200) */
    int fft_grid[3];        /* FFT grid; 0 = smallest alias-free 2-3-5 grid */
    int band_batch;         /* bands per FFT batch (0 = automatic) */
    void* cuda_stream;      /* cudaStream_t to issue work on; NULL = legacy default stream */
    double cg_adapt;        /* outer iterations after the first stop each band's CG at
                             * ||r|| <= max(cg_tol, theta ||b||), theta = min(1e-2, cg_adapt x the
                             * previous iteration's relative Hxc residual); 0 = always cg_tol
                             * (default 0.001).  The first iteration (chi_0) always uses cg_tol. */
    double mixed_floor;     /* mixed form only: the response SCF also stops once the residual and the
                             * change of the traces are below mixed_floor x the response potential and
                             * x the largest trace (the FP32 noise floor; default 3e-7) */
    double wait_timeout_s;  /* bound on every device-side wait of the library's kernels (mbarrier polls
                             * of the tensor-core contractions): a wait that runs this long (about; it
                             * is counted in polls) makes the kernel record an error flag and return,
                             * and the call fails with HP_ETIMEOUT.  Default 2 s. */
    /* Device memory.  When dev_alloc is set every device buffer of the context comes from
     * dev_alloc(bytes, alloc_user) (NULL = out of memory) and goes back through
     * dev_free(ptr, alloc_user); the Python binding registers PyTorch's caching allocator here.
     * Both NULL: cudaMalloc / cudaFree.  The library frees a buffer only after the work that uses
     * it has finished on the context's stream. */
    void* (*dev_alloc)(size_t bytes, void* user);
    void (*dev_free)(void* ptr, void* user);
    void* alloc_user;
    int hub_ortho;          /* Hubbard projectors (Sec. 2.2): 0 = non-orthogonalised atomic orbitals
                             * (default); 1 = Loewdin ortho-atomic orbitals (Eq. OAO_def): at every k
                             * (and k+q) phi~_b = sum_a phi_a (O^-1/2)_ab with O_ab = <phi_a|phi_b> over
                             * every Hubbard orbital of every atom that carries one */
} hp_options;

/* Fills *opt with the defaults listed above. */
void hp_default_options(hp_options* opt);

typedef struct {
    int nk, nq, nspin, nocc, nbnd;  /* nbnd: bands kept per k by the ground state (nocc + extra) */
    int grid[3], nr;
    int nat, nhub_atoms, nhub_orb, nproj, mmax; /* mmax: padded m dimension of Delta n (5) */
    int npw_max;                    /* largest wavefunction sphere over the k mesh */
    int ncell;                      /* N_q: cells of the supercell imaged by the q mesh */
    int nchi;                       /* N_H * N_q, the dimension of chi */
} hp_sizes;

typedef struct {
    int iterations;         /* SCF iterations */
    double residual;        /* final rms residual of V_Hxc */
    double gap;             /* min over spins of (lowest empty - highest occupied) [Ha] */
    double homo, lumo;
    double seconds;
} hp_gs_info;

typedef struct {
    int iterations;         /* outer (self-consistency) iterations */
    long long cg_iterations;/* summed over bands */
    long long hpsi;         /* single-band applications of the Sternheimer operator */
    double residual;        /* final rms of dV_out - dV_in */
    double dchi;            /* final change of the response traces */
    double seconds;
    int stagnated;          /* mixed form: 1 when the SCF stopped on the FP32 noise floor rather than on
                             * the mixed_floor test: the residual is below 1e-5 of the response
                             * potential and its last three iterations came no lower than 0.8 of the
                             * best one before them; 0 otherwise */
} hp_resp_info;

/* One inter-site pair of hp_hubbard's V list: Hubbard atom s of the primitive cell (index into the
 * Hubbard-atom list) and its neighbour (l', s') of the q-mesh supercell (chi index l' * nhub_atoms
 * + s'), their distance in bohr and V in eV. */
typedef struct {
    int s, jchi;
    double dist;
    double V;
    int j;                  /* the neighbour's Hubbard-atom index (primitive cell) ... */
    int R[3];               /* ... displaced by the lattice vector R (crystal units) */
} hp_pairV;

/* ------------------------------------------------------------------------------------------ */
/* Set-up (a1 of the hot path: the cell, spheres, grid maps, closed-form form factors).  The paper's
 * method starts from the cell, the pseudopotentials (here the model species), the cutoff and the
 * k and q meshes of the ground-state and linear-response runs (Sec. 3.1-3.2; the q mesh images the
 * supercell of Eq. occ_matrix_response_lp_1).
 * cell: lattice vectors as rows (bohr), 9 doubles.  sp: nspecies species.  species_of: natoms
 * indices into sp.  frac_pos: natoms x 3 crystal coordinates.  kmesh, qmesh: Gamma-centred mesh
 * sizes.  Where k+q lies on the k mesh (k+q = k' + G0) the response reuses the states of k'; where
 * it does not, hp_response computes the occupied states at k+q non-self-consistently at the
 * ground-state potential (once per q) and evaluates the projector and Hubbard rows there.
 * opt may be NULL (defaults).  *out receives a new context owned by the caller (hp_destroy).
 * Errors: HP_EINVAL (bad sizes, a grid too small for the sphere, l out of range), HP_ECUDA,
 * HP_ENOMEM.  On error *out is NULL. */
hp_status hp_setup(const double cell[9], int nspecies, const hp_species* sp, int natoms,
                   const int* species_of, const double* frac_pos, double ecutwfc_ry,
                   const int kmesh[3], const int qmesh[3], const hp_options* opt, hp_ctx** out);

/* Sizes of the context: meshes, bands, grid, Hubbard atoms, and the dimension N_H N_q of chi and
 * chi_0 (Sec. 3.2: the response matrices are N_H^sc x N_H^sc with N_H^sc = N_H N_q).  Output
 * buffers of hp_response / hp_hubbard are sized from it.  Errors: HP_EINVAL (NULL pointer). */
hp_status hp_query_sizes(const hp_ctx* ctx, hp_sizes* out);

/* Switches the precision form of later hp_response calls (HP_PRECISION_FP64 or _MIXED) without
 * touching the ground state; response columns computed so far are discarded.  Errors: HP_EINVAL. */
hp_status hp_set_precision(hp_ctx* ctx, int precision);

/* Wavefunction sphere at k point ik of the mesh: *npw receives its size; if miller != NULL it
 * receives npw x 3 Miller indices (int) in the library's coefficient order. */
hp_status hp_sphere(const hp_ctx* ctx, int ik, int* npw, int* miller);

/* Hubbard atoms: atom index (0-based, into the set-up atom list) and m dimension, for each of the
 * nhub_atoms Hubbard atoms in order.  Either pointer may be NULL. */
hp_status hp_hubbard_atoms(const hp_ctx* ctx, int* atom_index, int* mdim);

/* Ground state by the library (the unperturbed state the response starts from, Sec. 3.1: occupied
 * u_vk, eps_vk, the spin densities and the Hubbard occupations of Eq. occ_matrix_0): fixed-occupation
 * SCF on the GPU (LDA/LSDA), nelec electrons, nspin 1 or 2; init_moment: natoms signs (+1, -1, 0)
 * of the starting magnetisation, NULL for none.  tot_mag: the fixed total magnetisation (occupied
 * bands per spin (nelec +- tot_mag) / 2, the paper's tot_magnetization of a magnetic insulator,
 * Sec. 5.2); only tot_mag = 0 (equal band counts) is built, any other value returns HP_ENOTIMPL.
 * Starting density: uniform nelec/Omega, for nspin = 2 split as rho0/2 (1 +- s(r)),
 * s(r) = clip(sum_I m_I 0.9 exp(-|r - tau_I|^2 / 2), -0.9, 0.9).
 * Errors: HP_EINVAL, HP_ENOTIMPL, HP_ENOTCONV, HP_ENOGAP (the state is kept; hp_response refuses
 * it). */
hp_status hp_ground_state(hp_ctx* ctx, double nelec, int nspin, const int* init_moment, double tot_mag,
                          hp_gs_info* info);

/* Imports a ground state (so that the response can be checked on identical inputs).
 * vhxc, rho: nspin x nr (real, V_H + V_xc and the spin densities).  eps: nspin x nk x nocc.
 * psi: for each spin, for each k, nocc vectors of npw_k complex coefficients in hp_sphere order,
 * packed without padding.  The band count per spin is nocc = nelec / 2 (fixed occupations).
 * Errors: HP_EINVAL. */
hp_status hp_set_ground_state(hp_ctx* ctx, int nspin, double nelec, const double* vhxc,
                              const double* rho, const double* eps, const double* psi);

/* Lowest nlev (1 .. 100) eigenvalues (Ha, ascending) of the bare Hamiltonian T + V_loc + V_NL (no
 * Hxc potential, no Hubbard term) at point ik of the k mesh (ik = 0: k = 0 for the Gamma-centred
 * meshes).  No counterpart in the paper: it serves the electron-count rule of the batch of
 * synthetic cells (the occupied band count is chosen at the largest gap of this spectrum over the
 * k mesh).  Errors: HP_EINVAL (ik outside the mesh, nlev outside 1 .. 100 or above the plane-wave
 * count less 6), HP_ENOTCONV, HP_ECUDA. */
hp_status hp_bare_levels(hp_ctx* ctx, int ik, int nlev, double* eps);

/* Reads back the ground state: any pointer may be NULL.  eps: nspin x nk x nocc; rho, vhxc:
 * nspin x nr.  Errors: HP_ESTATE before a ground state. */
hp_status hp_get_ground_state(const hp_ctx* ctx, double* eps, double* rho, double* vhxc);

/* H psi without allocating: the same operator and kernels as hp_apply_h, for callers that cannot
 * call cudaMalloc while they compute -- applications whose own pool allocator holds all free
 * device memory, and loops that must not call cudaMalloc/cudaFree because those calls can
 * synchronise the device.  The paper has no counterpart; it is a calling convention of this library.
 * psi_dev, out_dev: caller-owned device arrays of nb rows of npw_max complex numbers (interleaved
 * FP64; npw_max from hp_query_sizes; row b holds band b in hp_sphere(ik) order, entries beyond
 * npw_k zero on input and written as zero on output).  stream: a cudaStream_t, or NULL for the
 * context's stream; the call waits for its work on that stream before returning.
 * Scratch: one fixed 64 MiB file-scope device array, which every GPU that loads the library holds
 * until the process exits.  The first call on a device looks up that array's device address with
 * that device current (cudaGetSymbolAddress) and caches it.  Every call reuses the same array and
 * leaves its contents behind; the call clears what it needs cleared.  Calls whose work overlaps on
 * the GPU (other streams, other host threads) race on the array and must be serialised by the
 * caller.  The current device must be the context's device (the one current at hp_setup) and the
 * stream must belong to it.  Errors: HP_EINVAL (bad arguments, another device current, or nb too
 * large for the fixed scratch on this grid: call it on fewer bands), HP_ESTATE (no ground state),
 * HP_ENOTIMPL (a Hubbard-corrected ground state, hp_set_hubbard), HP_ECUDA. */
hp_status hp_apply_h_noalloc(hp_ctx* ctx, int ik, int spin, int nb, const double* psi_dev, double* out_dev,
                             void* stream);

/* Reads back the occupied ground-state wavefunctions in the layout hp_set_ground_state takes: for
 * each spin, each k, nocc vectors of npw_k complex coefficients (hp_sphere order), packed.
 * Errors: HP_ESTATE before a ground state. */
hp_status hp_get_wavefunctions(const hp_ctx* ctx, double* psi);

/* Kohn-Sham operator at mesh point ik and spin s applied to nb host vectors (npw_k complex each,
 * hp_sphere order): out = H psi with H = T + V_loc + V_Hxc,s + V_NL, plus the Hubbard potential of a
 * DFT+U+V ground state (hp_set_hubbard); needs a ground state. */
hp_status hp_apply_h(hp_ctx* ctx, int ik, int spin, int nb, const double* psi, double* out);

/* Wavefunction sphere at k+q for mesh point ik and q point iq, in the coefficient order the
 * response (hp_response, hp_apply_sternheimer) uses for vectors at k+q: *npw receives its size; if
 * miller != NULL it receives npw x 3 Miller indices G with |k+q+G|^2 <= ecutwfc.  Where k+q = k' + G0
 * lies on the k mesh this is the sphere of k' shifted by -G0 in the order of k'.  Errors: HP_EINVAL. */
hp_status hp_sphere_kq(const hp_ctx* ctx, int iq, int ik, int* npw, int* miller);

/* The operator of the q-specific Sternheimer equation (Eq. LRKSeq_lp, left-hand side),
 * out_b = (H_k+q,spin + alpha O_k+q,spin - eps_b) psi_b, with O the projector on the occupied states
 * at k+q (Eq. proj_v) and alpha = 2 (max - min) of the occupied ground-state energies, applied to
 * nb host vectors of hp_sphere_kq(iq, ik) size (complex, packed) through exactly the kernels and
 * the precision form hp_response uses (fused column/plane transforms where the grid allows them,
 * FP32 vectors and projections in the mixed form).  eps: nb shifts (Ha).  Needs a ground state.
 * Allocates its device buffers per call.  Errors: HP_EINVAL, HP_ESTATE, HP_ECUDA. */
hp_status hp_apply_sternheimer(hp_ctx* ctx, int iq, int ik, int spin, int nb, const double* eps,
                               const double* psi, double* out);

/* One (q, J) response (hot path a1-a10): iq indexes the q mesh, atom is the index of the
 * perturbed Hubbard atom in the set-up atom list.  dn0 / dn (may be NULL) receive the bare and
 * self-consistent Delta_q n^{s sigma}_{m1 m2} as complex [nhub_atoms][nspin][mmax][mmax]
 * (m1 slowest of the two, rows beyond the atom's m dimension zero).  The columns are also kept in
 * the context for hp_hubbard.  Errors: HP_ESTATE (no ground state), HP_ENOGAP, HP_EINVAL,
 * HP_ENOTCONV (partial data written), HP_ENUMERIC. */
hp_status hp_response(hp_ctx* ctx, int iq, int atom, double* dn0, double* dn, hp_resp_info* info);

/* Hubbard-corrected ground state (DFT+U+V, Sec. 2.1; the self-consistent U/V cycle of Sec. 5.2
 * runs ground state -> response -> hp_hubbard -> hp_set_hubbard -> ground state ...).  U: on-site
 * U per Hubbard atom in eV (nhub_atoms entries, NULL for none); V[0 .. nV): inter-site pairs
 * (s = atom, j = neighbour, R = its lattice vector, V in eV; s, j index the Hubbard atoms; jchi and
 * dist are ignored), as hp_hubbard returns them.  The Hubbard potential of Eq. Hub_pot_0,
 *   V_Hub = sum_I U^I sum (delta/2 - n^I) |phi^I_m1><phi^I_m2|
 *         - sum_(s,j,R) V sum n^{s j(R)}_m1m2 |phi^s_m1><phi^j_m2 shifted by R|,
 * with the occupation matrices of Eq. occ_matrix_0 (1/N_k per cell) and the star sum over the
 * listed pairs (list a pair in both directions), is added to H in hp_ground_state (its occupation
 * matrices converged together with V_Hxc), in the states at k+q and in the Sternheimer operator;
 * its response is not part of the linear response (Sec. 2.3).  hp_set_ground_state takes the
 * occupation matrices from the imported occupied states.  All zero or nV = 0 with U = NULL: no
 * correction.  Takes effect at the next hp_ground_state or hp_set_ground_state; discards the
 * current ground state.  Errors: HP_EINVAL (an index out of range). */
hp_status hp_set_hubbard(hp_ctx* ctx, const double* U, int nV, const hp_pairV* V);

/* Post-processing (a11): the q-sum with phases (Eq. occ_matrix_response_lp_1) into chi_0 and chi
 * (Eq. chi), their inverses and U, V (Eqs. U_def, V_def).
 * chi0, chi: real nchi x nchi (row-major, index (l, s) -> l*nhub_atoms+s, l the supercell cell
 * (l1*n2 + l2)*n3 + l3); hub: (chi0^-1 - chi^-1) in eV (U on the diagonal, V off it).
 * U: nhub_atoms on-site values U^s = hub[s][s] in eV.  V, nV: the inter-site V of every Hubbard atom
 * s of the primitive cell to its nearest Hubbard neighbours of another species in the q-mesh
 * supercell: every (l', s') at the shortest minimum-image distance d_min of that species class or
 * within d_min + 6e-4 bohr of it (the paper's dist_thr default, Appendix B); *nV is the capacity
 * of V on input and the number of pairs on output (all pairs are counted even when they do not fit;
 * HP_EINVAL then).  Any output pointer may be NULL (nV with V).  Needs every (q, J) column
 * (HP_ESTATE otherwise), where a missing (q, J) is taken from (-q, J) by conjugation, with
 * find_atpert 3 from the star of q (hp_irreducible_pairs), and the columns of an atom that was not
 * perturbed are rebuilt from its class (hp_perturbed_atoms).  chi0 and chi are written even when one of them is singular or has a
 * 1-norm condition number above 1e10; U, V and hub are then not written and the call returns
 * HP_ESINGULAR. */
hp_status hp_hubbard(hp_ctx* ctx, double* chi0, double* chi, double* hub, double* U, hp_pairV* V, int* nV);

/* Symmetry reductions (Sec. 2.4 "Symmetry"; Sec. 3.2, the linear-response step and its
 * post-processing; the hp.x inputs find_atpert, docc_thr, dist_thr and skip_equivalence_q).
 *
 * hp_perturbed_atoms: after a ground state, sorts the Hubbard atoms into classes and keeps them in
 * the context.  find_atpert 1: atoms of one species whose spin-summed occupations Tr n^I (Eq.
 * occ_matrix_0 with the active Hubbard projectors; twice the channel for nspin = 1) differ by less
 * than docc_thr (the paper's default 5e-5) form a class, whatever the sign of their moments;
 * 2: one class per species; 3: the orbits under the crystal's space group (the operations
 * x -> W x + t on fractional coordinates with W an integer matrix of entries -1, 0, 1 and determinant
 * +-1 that keeps the lattice metric, every atom going onto an atom of its species within 1e-5, and the
 * Hubbard atoms' spin orientations kept up to one global sign); 4: every atom alone (this clears the
 * classes).  The first atom of each class in atom order represents it.  Writes *npert and atoms[0 .. *npert) (the representatives,
 * atom indices; capacity nhub_atoms), rep[i] (the representative of the i-th Hubbard atom in
 * hp_hubbard_atoms order; may be NULL) and trace[2 i + s] (Tr n^{I s}, s < nspin; may be NULL).
 * With classes kept, hp_hubbard rebuilds the columns of every atom that does not represent its class
 * (whether or not its responses were computed): the entry
 * of cell l, atom s of the real-space column (0, J), chi_{(l,s),(0,J)} = (1/N_q) sum_q
 * exp(i q.R_l) Delta^J_q n^s, is the entry (l', s') of the representative's column with the species
 * of s and the spin orientation of s relative to J (orientation: the sign of Tr n^up - Tr n^down
 * where that exceeds docc_thr, else 0) whose separation from J' matches that of (l, s) from J within
 * dist_thr bohr (the paper's default 6e-4): as a vector modulo the q-mesh supercell, else, where no
 * atom matches the vector, as the minimum-image distance; the first such (l', s') in index order.
 * With find_atpert 3 an operation g of the space group that keeps the q-mesh supercell's lattice and
 * takes J' (cell 0) to J in cell L_J rebuilds the column exactly: chi_{a,(0,J)} =
 * chi_{g^-1(a + L_J),(0,J')} (the separation rule where no such operation exists).
 * Errors: HP_ESTATE without a ground state; HP_EINVAL for find_atpert outside 1 .. 4, docc_thr <= 0,
 * dist_thr < 0 or a NULL npert/atoms.  A new ground state clears the classes. */
hp_status hp_perturbed_atoms(hp_ctx* ctx, int find_atpert, double docc_thr, double dist_thr, int* npert, int* atoms,
                             int* rep, double* trace);

/* hp_irreducible_q: the q points to compute under time reversal (of the small group of q only the
 * +-q pairs; the ground states here have real potentials and real Hubbard orbitals, so
 * Delta_{-q} n = conj(Delta_q n)): of each pair {q, -q + G} of the q mesh the first in mesh order.
 * Writes *nirr and iq[0 .. *nirr) (capacity nq), and partner[iq] for every q of the mesh (itself, or
 * the computed q whose conjugate response it takes; may be NULL).  hp_hubbard fills a missing (q, J)
 * column from (-q, J) this way.  Errors: HP_EINVAL for a NULL ctx, nirr or iq. */
hp_status hp_irreducible_q(const hp_ctx* ctx, int* nirr, int* iq, int* partner);

/* hp_irreducible_pairs: the (q, J) responses to compute under the kept classes (hp_perturbed_atoms)
 * and, with find_atpert 3, the star of q: an operation x -> W x + t of the space group that keeps the
 * q-mesh supercell relates the trace columns of chi at q and q' = W^-T q,
 *   x_{q'}[pi(J)][pi(s)] = exp(2 pi i q'.(L_J - L_s)) x_q[J][s],   W x_a + t = x_pi(a) + L_a,
 * and time reversal relates q and -q (x_{-q}[J] = conj(x_q[J])).  The first pair of each orbit is
 * listed, J-major (representative atoms in atom order), then q in mesh order.  Writes *npairs,
 * iq[0 .. *npairs) and atom[0 .. *npairs) (capacity nq x nhub_atoms).  hp_hubbard derives the other
 * pairs with these relations.  Errors: HP_EINVAL for a NULL argument. */
hp_status hp_irreducible_pairs(const hp_ctx* ctx, int* npairs, int* iq, int* atom);

/* Several independent cells at once (the batching form; the paper's code runs one system per job,
 * so there is no counterpart there).  For every context cells[0 .. ncells-1], each set up with its
 * own CUDA stream (hp_options.cuda_stream) and holding a ground state, runs every (q, J) response
 * (hp_response) and then hp_hubbard, one host thread per cell, so that the cells' kernels overlap
 * on the GPU; returns when all cells are done.  chi0[i], chi[i], hub[i]: cell i's outputs as for
 * hp_hubbard (the arrays of pointers, or any entry, may be NULL).  status[i] receives cell i's
 * result (caller-owned, ncells entries).  Returns HP_OK when every cell succeeded, else the first
 * failing status in cell order.  Errors: HP_EINVAL (ncells < 1, a NULL or repeated context).
 * While it runs, no other thread may use these contexts; contexts on the same stream serialise. */
hp_status hp_batch_run(int ncells, hp_ctx* const* cells, double* const* chi0, double* const* chi, double* const* hub,
                       hp_status* status);

/* Message of the last failure on this context ("" if none).  Valid until the next call. */
const char* hp_last_error(const hp_ctx* ctx);

/* Frees the context and all device memory it owns.  NULL is ignored. */
void hp_destroy(hp_ctx* ctx);

/* Live timing of the hot kernel families.  Between hp_profile_begin and hp_profile_end every
 * launch of a timed family is bracketed by CUDA events recorded on its own launch stream and adds
 * its algorithmic flops and bytes (counted on the host from the sizes the launch processes):
 *   HP_KF_FFT_PASS  one pass of the batched 3D FFT: every grid point read and written once;
 *                   5 n log2 n flops per line of n points.
 *   HP_KF_COLUMN    fused column transform (z-FFT between the wavefunction sphere and the compact
 *                   column buffer): sphere coefficients read or written in FP64 (plus the input
 *                   vector for the kinetic term, and the zeroed padding), column buffer once.
 *   HP_KF_PLANE     fused plane transform (x/y-FFTs of one z-plane of one band in shared memory and
 *                   the real-space product): column buffer in and out, real-space grids read or
 *                   written once per band, the potential once per spin.
 *   HP_KF_PROJECT   <beta|psi> projections: band vectors and projector rows read once, partial sums
 *                   and results written; 8 flops per complex multiply-add.
 *   HP_KF_EXPAND    psi += beta P: projector rows and coefficients read, band vectors read and written.
 * hp_profile_end waits for the events and fills stats[0 .. HP_KF_COUNT-1] with the summed kernel
 * time (ms), launches, flops and bytes of each family.  Process-wide (one host thread), not per
 * context.  With the environment variable HP_PROF_LOG naming a file, every timed launch also
 * appends one line "family kernel bytes flops" to it.  Errors: HP_ECUDA if an event could not be
 * read. */
enum {
    HP_KF_FFT_PASS = 0,
    HP_KF_COLUMN = 1,
    HP_KF_PLANE = 2,
    HP_KF_PROJECT = 3,
    HP_KF_EXPAND = 4,
    HP_KF_COUNT = 5
};
typedef struct {
    double ms;
    long long launches;
    double flops;
    double bytes;
} hp_kernel_stats;
void hp_profile_begin(void);
hp_status hp_profile_end(hp_kernel_stats* stats);

/* Number of CUDA kernels this library has launched in this process (monotonic counter). */
long long hp_launch_count(void);

/* Number of device allocations this library has made in this process, through cudaMalloc or a
 * registered dev_alloc (monotonic counter; no counterpart in the paper). */
long long hp_alloc_count(void);

/* Host-only self-test of the FFT engine's stage logic (runs the same Stockham code on the CPU).
 * in/out: nlines x n complex; sign -1 forward exp(-2 pi i jk/n), +1 backward (unnormalised). */
hp_status hp_selftest_fft_host(int n, int nlines, int sign, const double* in, double* out);

/* Device self-test of the batched Hermitian eigensolver used by the ground state (one CTA per
 * matrix, cyclic Jacobi).  A: nbatch complex n x n Hermitian matrices, row-major, interleaved;
 * w: nbatch x n eigenvalues ascending; V: nbatch n x n, eigenvectors in the columns.  n <= 512.
 * Allocates its own device buffers.  Errors: HP_EINVAL, HP_ECUDA. */
hp_status hp_selftest_eigh(int n, int nbatch, const double* A, double* w, double* V);

/* Device self-test of the LDA kernel of the ground state and the response (Slater exchange +
 * Perdew-Zunger 1981 correlation, von Barth-Hedin spin interpolation): for n grid points and spin
 * densities rho (nspin x n), vxc receives nspin x n potentials and fxc the kernel f_xc (n values
 * for nspin = 1; 3 x n for nspin = 2: f_up,up, f_up,down, f_down,down), the same kernel as the
 * response's Delta V_xc = sum_s' f_ss' Delta rho_s' (Sec. 2.3, the response Hxc potential).
 * Allocates its own device buffers.  Errors: HP_EINVAL, HP_ECUDA. */
hp_status hp_selftest_xc(int n, int nspin, const double* rho, double* vxc, double* fxc);

/* Device self-test of the tensor-core building block of the projector contractions (no counterpart
 * in the paper): D[m][n] = sum_k A[m][k] B[n][k] for FP32 row-major A (M x K) and B (N x K) by
 * tcgen05 kind::tf32 MMAs with the three-product TF32 split, FP32 accumulation in TMEM.
 * 1 <= M <= 128, 16 <= N <= 128 with N % 16 == 0, K a multiple of 32.  mode bits: 1 exchanges the
 * leading- and stride-byte-offset fields of the operand descriptors (the data layout is unchanged;
 * every address stays inside the staged tiles), for checking which reading the hardware follows;
 * 2 adds the fourth product a_lo b_lo; 4 drains the TMEM accumulator into FP64 registers after every
 * 32 values of K.  Every device-side wait gives up after timeout_s (HP_ETIMEOUT).  Allocates its own
 * device buffers.  Errors: HP_EINVAL, HP_ECUDA, HP_ETIMEOUT. */
hp_status hp_selftest_tc(int M, int N, int K, const float* A, const float* B, float* D, int mode,
                         double timeout_s);

/* Device self-test of the integer-operation FP64 <-> FP32 conversions used in the FP32 form's hot
 * loops (no counterpart in the paper).  For n host values in[i]: f[i] = FP64 -> FP32 rounded to
 * nearest even (results below the FP32 normal range flushed to signed zero), back[i] = f[i]
 * widened exactly to FP64; f_ref and back_ref are the hardware conversions of the same values.
 * Allocates its own device buffers.  Errors: HP_EINVAL (n < 1 or a NULL pointer), HP_ECUDA. */
hp_status hp_selftest_convert(long long n, const double* in, float* f, double* back, float* f_ref, double* back_ref);

#ifdef __cplusplus
}
#endif

#endif /* HP_H */
