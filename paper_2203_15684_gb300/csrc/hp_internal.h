// Internal declarations of the GB300 DFPT Hubbard engine: device complex arithmetic, the FFT
// plan, the batched operator kernels and the context that owns every device buffer.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "hp.h"

namespace hp {

// ------------------------------------------------------------------------------------------------
// complex FP64 helpers (double2 = (re, im))
// ------------------------------------------------------------------------------------------------
#if defined(__CUDACC__)
#define HD __host__ __device__ __forceinline__
#else
#define HD inline
#endif

HD double2 cmk(double r, double i) { double2 z; z.x = r; z.y = i; return z; }
HD double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
HD double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
HD double2 cmul(double2 a, double2 b) { return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
HD double2 cmulc(double2 a, double2 b) { return cmk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a)*b
HD double2 cscale(double2 a, double s) { return cmk(a.x * s, a.y * s); }
HD double2 cconj(double2 a) { return cmk(a.x, -a.y); }
// a * (s i) for s = +-1
HD double2 cmul_si(double2 a, int s) { return s > 0 ? cmk(-a.y, a.x) : cmk(a.y, -a.x); }

// the same helpers for FP32 complex (float2)
HD float2 cmkf(float r, float i) { float2 z; z.x = r; z.y = i; return z; }
HD float2 cadd(float2 a, float2 b) { return cmkf(a.x + b.x, a.y + b.y); }
HD float2 csub(float2 a, float2 b) { return cmkf(a.x - b.x, a.y - b.y); }
HD float2 cmul(float2 a, float2 b) { return cmkf(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
HD float2 cscale(float2 a, float s) { return cmkf(a.x * s, a.y * s); }
HD float2 cmul_si(float2 a, int s) { return s > 0 ? cmkf(-a.y, a.x) : cmkf(a.y, -a.x); }

template <class V> struct Scalar;
template <> struct Scalar<double2> { using type = double; };
template <> struct Scalar<float2> { using type = float; };
template <class V> HD V cpack(double r, double i);
template <> HD double2 cpack<double2>(double r, double i) { return cmk(r, i); }
template <> HD float2 cpack<float2>(double r, double i) { return cmkf((float)r, (float)i); }

#if defined(__CUDACC__)
// FP64 <-> FP32 conversions with integer operations on the IEEE 754 bit patterns, for hot loops:
// the FP64 pipe that runs the hardware conversions is narrow on this part.
// d2f_bits: round to nearest, ties to even; results below the FP32 normal range flush to a signed
// zero and results above it become infinity (NaN inputs are not expected).
__device__ __forceinline__ float d2f_bits(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int fe = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;  // FP32 biased exponent
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    unsigned f = ((unsigned)fe << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;  // the 29 dropped mantissa bits
    f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
    return __uint_as_float(sign | f);
}
// f2d_bits: exact widening; FP32 subnormals become zero (infinity and NaN are not expected).
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned sign = u & 0x80000000u;
    const unsigned hi = e ? (sign | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)) : sign;
    const unsigned lo = e ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
#endif

// every kernel launch of the library increments this counter (read by hp_launch_count)
extern std::atomic<long long> g_launches;
// every device allocation of the library increments this counter (read by hp_alloc_count)
extern std::atomic<long long> g_allocs;
#define HP_LAUNCHED() (hp::g_launches.fetch_add(1, std::memory_order_relaxed))

// ------------------------------------------------------------------------------------------------
// FFT (batched 3D complex, mixed radix 2/3/4/5 Stockham in shared memory, one pass per axis)
// ------------------------------------------------------------------------------------------------
constexpr int kMaxStages = 12;

struct Radices {
    int n, nst;
    int r[kMaxStages];
};

struct FftAxis {
    Radices rad;
    double2* d_tw = nullptr;   // n twiddles exp(-2 pi i t / n)
    float2* d_tw32 = nullptr;  // the same, rounded to FP32
};

struct FftPlan {
    int N[3] = {0, 0, 0};
    FftAxis ax[3];
};

bool fft_factor(int n, Radices& out);
// twiddle tables are context allocations (freed with the context)
cudaError_t fft_plan_create(hp_ctx* c, FftPlan& p, const int N[3]);
void fft_plan_destroy(FftPlan& p);
// In place, nb grids of N0*N1*N2 complex each, contiguous.  sign +1: sum_G c(G) exp(+iG.r)
// (to real space), sign -1: sum_r f(r) exp(-iG.r).  Unnormalised both ways.
cudaError_t fft3d(const FftPlan& p, double2* data, int nb, int sign, cudaStream_t st);
cudaError_t fft3d(const FftPlan& p, float2* data, int nb, int sign, cudaStream_t st);
// the same Stockham code on the host (self-test of the stage logic)
void fft_host_lines(const Radices& rad, const std::vector<double2>& tw, int nlines, int sign,
                    double2* data);

// ------------------------------------------------------------------------------------------------
// Batched band operations.  A band list names nb vectors: for item c its row (index of a vector
// of ld complex numbers in the matrix it lives in), its sphere k, its spin and a scalar shift.
// Items are sorted into segments of consecutive items with the same (spin, k); a projector matrix
// for a segment sits at element offset spin * a_stride_s + k * a_stride_k of its base pointer.
// ------------------------------------------------------------------------------------------------
struct SphereSet {          // device arrays, nk spheres of at most ld points
    int nk = 0, ld = 0;
    int* d_npw = nullptr;   // [nk]
    int* d_idx = nullptr;   // [nk][ld] flat grid index of each coefficient
    double* d_g2 = nullptr; // [nk][ld] |k+G|^2
    double* d_prec = nullptr;  // [nk][ld] CG preconditioner 1 / (1 + |k+G|^2 / 2), 0 beyond npw
    float* d_prec32 = nullptr; // the same in FP32
    float* d_kin32 = nullptr;  // [nk][ld] |k+G|^2 / 2 in FP32
    std::vector<int> npw;   // host copy
    // column structure (the sphere is stored column by column, z fastest): for each k, ncol
    // columns (x, y) of the grid that hold sphere points, their first point and length, and the
    // z index of every point
    int ncmax = 0;
    int* d_ncol = nullptr;      // [nk]
    int* d_col_start = nullptr; // [nk][ncmax]
    int* d_col_len = nullptr;   // [nk][ncmax]
    int* d_col_xy = nullptr;    // [nk][ncmax] x * N1 + y
    int* d_iz = nullptr;        // [nk][ld]
    std::vector<int> ncol;      // host copy of d_ncol
    // per (k, x): the columns with grid x are columns j0 .. j0 + cnt - 1 with y = y0, y0 + 1, ...
    // (mod N1); [nk][xtab_n0][3] = (j0, cnt, y0); null when some x does not form such a run
    int* d_xtab = nullptr;
    int xtab_n0 = 0;
    bool contig = false;        // every column is one run of consecutive z (mod N2)
    // every sphere point's x, y and z grid indices lie within (N - 1) / 4 of 0 (mod N): the column and
    // plane transforms may prune their lines to those positions
    bool lines_prunable = false;
    bool cols_distinct = true;  // no two columns of one k share an (x, y) (the fused transforms need this)
};

struct BandList {
    int nb = 0, nseg = 0;
    int* d_row = nullptr;
    int* d_k = nullptr;
    int* d_spin = nullptr;
    double* d_shift = nullptr;
    int* d_seg_start = nullptr;     // [nseg + 1]
    int* d_seg_k = nullptr;         // [nseg]
    int* d_seg_s = nullptr;         // [nseg]
    int cap = 0;                    // allocated items
    std::vector<int> row, k, spin, seg_start, seg_k, seg_s;
    std::vector<double> shift;
};

struct ProjMat {            // a family of projector matrices: base + s*stride_s + k*stride_k
    const double2* base;
    long long stride_s, stride_k;
    int nrow;               // rows used (nrow + nrow2 <= 128)
    int row0;               // first row inside each matrix
    const int* kmap;        // optional device map: matrix of list sphere k is kmap[k]
    const float2* base32 = nullptr;     // FP32 copy of the family (same layout), read by the FP32 form
    // optional second family, rows nrow .. nrow + nrow2 - 1 of the projection (same kmap)
    const double2* base2 = nullptr;
    const float2* base2_32 = nullptr;
    long long stride2_s = 0, stride2_k = 0;
    int nrow2 = 0, row02 = 0;
    double scale2 = 1.0;    // expansion weight of the second family's rows
};

// device view of a ProjMat (families in FP64 or in their FP32 copies)
struct ProjDev {
    const void* a0;
    const void* a1;
    long long s0_s, s0_k, s1_s, s1_k;
    int n0, r0, n1, r1;
    const int* kmap;
};

#if defined(__CUDACC__)
template <class AT>
__device__ __forceinline__ const AT* proj_row(const ProjDev& d, int s, int mk, int p, int ld) {
    if (p < d.n0) return (const AT*)d.a0 + s * d.s0_s + mk * d.s0_k + (long long)(d.r0 + p) * ld;
    return (const AT*)d.a1 + s * d.s1_s + mk * d.s1_k + (long long)(d.r1 + p - d.n0) * ld;
}
#endif

// tc.cu: the FP32 projections and expansions on the tensor cores (tcgen05 kind::tf32, three-product
// TF32 split, FP32 accumulation in TMEM); FP32 families and FP32 band vectors only
bool tc_enabled();
void tc_set_timeout(double seconds);
// partial sums part[ks][item][p] of the projection over the ksplit plane-wave splits of each segment
cudaError_t tc_proj(const ProjDev& d, const BandList& L, const SphereSet& S, const float2* X, int ld, int ksplit,
                    double2* part, cudaStream_t st);
cudaError_t tc_expand(const ProjDev& d, const BandList& L, const SphereSet& S, const double2* P, const double* pscale,
                      double alpha, double scale2, float2* Y, int ld, cudaStream_t st);
// 1 when a tensor-core kernel gave up on a bounded wait since the last call (synchronises the stream)
int tc_take_error(cudaStream_t st);

// kernels.cu
cudaError_t k_scatter(const SphereSet& S, const BandList& L, int c0, int nc, const double2* X, int ldx,
                      double2* grid, int nr, cudaStream_t st);
cudaError_t k_gather_h(const SphereSet& S, const BandList& L, int c0, int nc, const double2* grid, int nr,
                       const double2* X, double2* Y, int ld, cudaStream_t st);
cudaError_t k_gather_scaled(const SphereSet& S, const BandList& L, int c0, int nc, const double2* grid,
                            int nr, double scale, double2* Y, int ld, int accumulate, cudaStream_t st);
cudaError_t k_mul_rpot(double2* grid, int nc, int nr, const double* v, const BandList& L, int c0,
                       cudaStream_t st);
cudaError_t k_mul_cpot(double2* grid, const double2* src_rows, const int* src_row_of_item, int nc, int nr,
                       const double2* v, const BandList& L, int c0, cudaStream_t st);
cudaError_t k_proj(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* X, int ld,
                   double2* P, double2* scratch, size_t scratch_elems, cudaStream_t st, bool fp32 = false);
cudaError_t k_proj(const BandList& L, const SphereSet& S, const ProjMat& A, const float2* X, int ld,
                   double2* P, double2* scratch, size_t scratch_elems, cudaStream_t st, bool fp32 = false);
cudaError_t k_expand(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* P,
                     const double* pscale, double alpha, double2* Y, int ld, cudaStream_t st, bool fp32 = false);
cudaError_t k_expand(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* P,
                     const double* pscale, double alpha, float2* Y, int ld, cudaStream_t st, bool fp32 = false);
// FP32 forms (mixed precision)
cudaError_t k_scatter32(const SphereSet& S, const BandList& L, int c0, int nc, const double2* X, float2* grid, int nr,
                        cudaStream_t st);
cudaError_t k_mul_rpot32(float2* grid, int nc, int nr, const float* v, const BandList& L, int c0, cudaStream_t st);
cudaError_t k_gather_h32(const SphereSet& S, const BandList& L, int c0, int nc, const float2* grid, int nr,
                         const double2* X, double2* Y, int ld, cudaStream_t st);
cudaError_t k_gather_scaled32(const SphereSet& S, const BandList& L, int c0, int nc, const float2* grid, int nr,
                              double scale, double2* Y, int ld, cudaStream_t st);
cudaError_t k_mul_cpot32(float2* grid, const float2* src_rows, const int* src_row_of_item, int nc, int nr,
                         const float2* v, const BandList& L, int c0, cudaStream_t st);
cudaError_t k_drho_acc32(const float2* ur, const int* ur_row_of_item, const float2* xr, int nc, int nr,
                         const BandList& L, int c0, double weight, int nspin, double2* drho, double2* part,
                         size_t part_elems, cudaStream_t st);
cudaError_t k_to_f32(const double* a, float* b, long long n, cudaStream_t st);
cudaError_t k_to_c32(const double2* a, float2* b, long long n, cudaStream_t st);
cudaError_t k_to_c64(const float2* a, double2* b, long long n, cudaStream_t st);
cudaError_t k_band_dot(const BandList& L, const SphereSet& S, const double2* X, const double2* Y, int ld,
                       double* out, cudaStream_t st);
cudaError_t k_band_dot(const BandList& L, const SphereSet& S, const float2* X, const float2* Y, int ld,
                       double* out, cudaStream_t st);
cudaError_t k_cg_init(const BandList& L, const SphereSet& S, const double2* r, double2* p, int ld,
                      double* rz, double* rr, cudaStream_t st);
cudaError_t k_cg_init(const BandList& L, const SphereSet& S, const float2* r, float2* p, int ld,
                      double* rz, double* rr, cudaStream_t st);
cudaError_t k_cg_step(const BandList& L, const SphereSet& S, double2* x, double2* r, double2* p, const double2* ap,
                      int ld, double* pap, double* rz, double* rr, cudaStream_t st);
cudaError_t k_cg_step(const BandList& L, const SphereSet& S, float2* x, float2* r, float2* p, const float2* ap,
                      int ld, double* pap, double* rz, double* rr, cudaStream_t st);
cudaError_t k_formfactor(const double* kcart, int nk, const int* miller, const int* npw, int ld,
                         const double* bvec, int nrow, const int* row_atom, const int* row_l, const int* row_m,
                         const double* row_width, const double* row_pref, const double* tau, double2* out,
                         cudaStream_t st);
// drho[s][r] += weight * sum over the nsplit partial sums part[slice][s][r] (fixed order); with a
// mask, only the slices whose bit s of mask[slice] is set hold spin s (the others are skipped)
cudaError_t k_drho_reduce(const double2* part, int nsplit, int nr, int nspin, double weight, double2* drho,
                          cudaStream_t st, const int* mask = nullptr);
cudaError_t k_drho_acc(const double2* ur, const int* ur_row_of_item, const double2* xr, int nc, int nr,
                       const BandList& L, int c0, double weight, int nspin, double2* drho, double2* part,
                         size_t part_elems, cudaStream_t st);
cudaError_t k_density_acc(const double2* ur, int nc, int nr, const BandList& L, int c0, double weight, int nspin,
                          double* rho, cudaStream_t st);
cudaError_t k_hartree_q(double2* rho_g, const int N[3], const double* bvec, const double qfrac[3], double ecut4,
                        double scale, cudaStream_t st);
cudaError_t k_vloc_g(double2* vg, const int N[3], const double* bvec, double ecut4, int nat, const double* tau,
                     const double* amp, const double* width, double omega, cudaStream_t st);
cudaError_t k_real_part(const double2* z, double* out, int n, double scale, cudaStream_t st);
cudaError_t k_xc(const double* rho, int nspin, int nr, double* vxc, double* fxc, cudaStream_t st);
cudaError_t k_hxc_combine(const double2* vh, const double2* drho, const double* fxc, int nspin, int nr,
                          double2* dv, cudaStream_t st);
cudaError_t k_occ_response(const double2* B, const double2* Aphi, int ngroups, int nocc, int nhub, int nk,
                           int nspin, double2* M, cudaStream_t st);
cudaError_t k_dn_blocks(const double2* M, int nspin, int nhub, int nhub_atoms, const int* off, const int* mdim,
                        int mmax, double2* dn, cudaStream_t st);
cudaError_t k_dn_traces(const double2* dn, int nh, int nspin, int mmax, double f, double2* tr, cudaStream_t st);
cudaError_t k_vec_dot(const double2* a, const double2* b, long long n, double* out, double* partial,
                      cudaStream_t st);
// out[p] = Re <A[p] | B[p]> for p < npairs (device pointer arrays), each as k_vec_dot computes it;
// partials: npairs x 256 doubles
cudaError_t k_vec_dots(const double2* const* A, const double2* const* B, int npairs, long long n, double* out,
                       double* partials, cudaStream_t st);
constexpr int kMaxDots = 72;  // nmix (m <= 8) x (m + 1) overlaps of a Broyden step
cudaError_t k_vec_axpy(double2* y, const double2* x, double a, long long n, cudaStream_t st);
cudaError_t k_vec_axpy(float2* y, const float2* x, double a, long long n, cudaStream_t st);
cudaError_t k_vec_sub(double2* out, const double2* a, const double2* b, long long n, cudaStream_t st);
cudaError_t k_vec_sub(float2* out, const float2* a, const float2* b, long long n, cudaStream_t st);
cudaError_t k_vec_scale_copy(double2* out, const double2* a, double s, long long n, cudaStream_t st);
cudaError_t k_vec_scale_copy(float2* out, const float2* a, double s, long long n, cudaStream_t st);
cudaError_t k_broyden_coef(const double* dots, int m, int ld, double w0, double* gamma, cudaStream_t st);
cudaError_t k_broyden_apply(double2* x, const double2* f, const double2* const* dx, const double2* const* df,
                            const double* gamma, int m, double alpha, long long n, cudaStream_t st);
cudaError_t k_chi_assemble(const double2* cols, int nq, int nh, const double* qfrac, const double* Rl, int ncell,
                           double* chi_re, double* chi_im, cudaStream_t st);
cudaError_t k_invert(double* a, double* work, int n, int* singular, cudaStream_t st);
cudaError_t k_hub_matrix(const double* inv0, const double* inv, int n, double scale, double* hub, cudaStream_t st);
// out = max_j sum_i |a_ij| (the matrix 1-norm), one CTA
cudaError_t k_norm1(const double* a, int n, double* out, cudaStream_t st);
cudaError_t k_add_real(const double* a, const double* b, double* out, int n, cudaStream_t st);
cudaError_t k_sum_reduce(const double* partial, int nparts, double* out, cudaStream_t st);

// ------------------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------------------
struct KSphere {
    double kfrac[3], kcart[3];
    int npw = 0;
    std::vector<int> miller;    // npw x 3
    std::vector<int> idx;       // flat grid index
    std::vector<double> g2;
};

struct RespCols {
    std::vector<double> dn0, dn;   // complex [nhub_atoms][nspin][mmax][mmax]
    std::vector<double> tr0, tr;   // spin-summed traces per Hubbard atom
};

// families at k+q for a q with some k+q off the k mesh, materialised once per q: occupied states
// (copied rows of k' where k+q = k' + G0, non-self-consistent states elsewhere) and the projector
// and Hubbard rows evaluated at k+q, in FP64 and FP32
struct QFam {
    bool built = false;
    double2 *psi = nullptr, *beta = nullptr, *phi = nullptr;  // [nspin][nk][nocc][ld], [nk][nproj][ld], [nk][nhub][ld]
    float2 *psi32 = nullptr, *beta32 = nullptr, *phi32 = nullptr;
    double2* hubW = nullptr;       // DFT+U+V: W of the Hubbard potential at each k+q, [nspin][nk][nhub][nhub]
};

// DFT+U+V (hubbard.cu): parameters on the device and the Hubbard potential in the projection basis
struct HubPair {
    int i, j, R[3];                // Hubbard-atom indices and the lattice vector of j
    double V;                      // Ha
};

struct QCache {                    // per-q data: the k+q sphere set and the k map of the families
    int iq = -1;
    bool off = false;              // some k+q of this q is off the k mesh: use the QFam of iq
    SphereSet set;
    int* d_miller = nullptr;       // [nk] family index of each k+q (k' on the mesh, k itself off it)
};

// fused.cu: sphere-sparse column/plane transforms
struct FusedArgs {
    const SphereSet* S = nullptr;
    const BandList* L = nullptr;
    const FftPlan* fft = nullptr;
    int c0 = 0, nc = 0, N0 = 0, N1 = 0, N2 = 0;
    const void* X = nullptr;     // band vectors: double2, or float2 when vec32
    void* Y = nullptr;
    bool vec32 = false;
    int mode = 0;
    double scale = 1.0;
    void* colA = nullptr;        // column buffer written by col_inv, read by plane
    void* colB = nullptr;        // column buffer written by plane, read by col_fwd
    const void* vt = nullptr;    // plane-major real potential [spin][z][y][x]
    const void* vtx = nullptr;   // the same with x-major planes [spin][z][x][y] (register plane kernels)
    const void* ur = nullptr;    // plane-major real-space bands [row][z][y][x]
    const void* dvt = nullptr;   // plane-major complex Delta V [spin][z][y][x]
    void* out = nullptr;         // plane-major real-space output [c][z][y][x]
    double inv_n = 1.0;
    bool reg = true;             // register-resident line FFTs where the sizes allow
    cudaStream_t st = nullptr;
};
// live kernel timing (hp_profile_*): mark before a launch, stop after it with its family and its
// algorithmic flops and bytes; both are no-ops while profiling is off
struct ProfMark {
    cudaEvent_t e0 = nullptr;
};
bool prof_on();
ProfMark prof_start(cudaStream_t st);
// tag: kernel name written with the launch's bytes and flops to the file named by HP_PROF_LOG
// (one line per timed launch), which lets a profiler capture of one launch be matched to its
// algorithmic bytes
void prof_stop(const ProfMark& m, int fam, cudaStream_t st, double flops, double bytes, const char* tag = nullptr);

bool fused_supported(const int N[3]);
cudaError_t fused_col(bool fp32, bool inv, const FusedArgs& a);
cudaError_t fused_plane(bool fp32, int op, const FusedArgs& a);
// out[plane][x][y] = in[plane][y][x] for nplanes planes of N1 x N0 reals (float or double)
cudaError_t k_planes_xmajor(const void* in, void* out, int N0, int N1, long long nplanes, bool fp32, cudaStream_t st);
// Delta rho of the FP32 form with the inverse plane transform fused in: partial sums of groups of
// bands, part[group0 + g][spin][z][y][x] (FP64) for the spins of the group, mask[group0 + g] = those
// spins as bits; the groups are then added by k_drho_reduce
bool fused_drho_supported(const FusedArgs& a);
int fused_drho_groups(int n0, int n1, int nc);
cudaError_t fused_drho(const FusedArgs& a, double2* part, int* mask, int group0);
cudaError_t k_to_planes_real(const double* a, double* b, const int N[3], int nvec, cudaStream_t st);
cudaError_t k_to_planes_c(const double2* a, double2* b, const int N[3], int nvec, cudaStream_t st);
cudaError_t k_from_planes_c(const double2* b, double2* a, const int N[3], int nvec, cudaStream_t st);

// engine.cu helpers shared with the ground-state code
hp_status fail(hp_ctx* c, hp_status s, const std::string& msg);
hp_status cuda_fail(hp_ctx* c, cudaError_t e, const char* what);
void dfree(hp_ctx* c, void* p);
hp_status upload_list(hp_ctx* c, BandList& L);
void list_clear(BandList& L);
void list_add(BandList& L, int row, int k, int spin, double shift);
hp_status ensure_grid(hp_ctx* c, int want);
// sphere sets (engine.cu): spheres of the given k points, Miller indices shifted by -shift[k]
hp_status upload_sphereset(hp_ctx* c, const std::vector<const KSphere*>& sph,
                           const std::vector<std::array<int, 3>>* shift, SphereSet& S);
void free_sphereset(hp_ctx* c, SphereSet& S);
int band_batch(const hp_ctx* c, int nb);
hp_status apply_local(hp_ctx* c, const SphereSet& S, const BandList& L, const double2* X, double2* Y,
                      const double* veff, bool fp32 = false);
hp_status project(hp_ctx* c, const SphereSet& S, const BandList& L, const ProjMat& A, const double2* X, double2* P,
                  bool fp32 = false);
hp_status project(hp_ctx* c, const SphereSet& S, const BandList& L, const ProjMat& A, const float2* X, double2* P,
                  bool fp32 = false);
hp_status apply_nonlocal(hp_ctx* c, const SphereSet& S, const BandList& L, const double2* X, double2* Y, double2* P,
                         const int* kmap, bool fp32 = false);
void invalidate_response(hp_ctx* c);
// Loewdin ortho-atomic Hubbard rows (Eq. OAO_def) in place: for each of the nk spheres of S,
// phi_b <- sum_a phi_a (O^-1/2)_ab with O_ab = <phi_a|phi_b> over the nhub rows (groundstate.cu)
hp_status ortho_hubbard_rows(hp_ctx* c, const SphereSet& S, int nk, double2* phi);
// occupied states at k points off the k mesh with the ground-state potential fixed (groundstate.cu);
// phi / hubW: Hubbard rows and W at those k points (DFT+U+V ground states), else null
hp_status nscf_states(hp_ctx* c, const std::vector<const KSphere*>& sph, const SphereSet& S, const double2* beta,
                      const double2* phi, const double2* hubW, double2* out, std::vector<double>& eps_occ);
// DFT+U+V (hubbard.cu).  The occupation vector holds, as complex numbers, the on-site matrices
// [nspin][nhub][nhub] (blocks of one atom used) then the pair matrices [npairs][nspin][5][5].
int hub_occ_len(const hp_ctx* c, int nspin);
hp_status hub_upload(hp_ctx* c);
// occupation vector from the projections P[item][p] (stride 128) of the occupied states, items in
// (spin, k, band) order with nocc bands per (spin, k); kfrac_dev [nk][3]
hp_status hub_occupations(hp_ctx* c, const double2* P, int nspin, int nk, int nocc, const double* kfrac_dev,
                          double2* occ);
// W [nspin][nkf][nhub][nhub] at nkf k points (fractional coordinates kfrac_dev [nkf][3])
hp_status hub_build_w(hp_ctx* c, const double2* occ, int nspin, int nkf, const double* kfrac_dev, double2* W);
// Y += V_Hub X on the list items: projection on the Hubbard rows phi (family of the list's spheres,
// optional kmap), W of the item's (spin, k) (same kmap), expansion; P: projection scratch (items x 128)
hp_status hub_apply(hp_ctx* c, const SphereSet& S, const BandList& L, const double2* phi, const int* kmap,
                    const double2* W, const void* X, void* Y, bool vec32, bool fp32, double2* P);

}  // namespace hp

struct hp_ctx {
    hp_options opt;
    cudaStream_t st = nullptr;
    int device = 0;                    // CUDA device current at hp_setup
    std::string err;
    // cell
    double cell[9], bvec[9], omega = 0;
    std::vector<hp_species> species;
    std::vector<int> atom_species;
    std::vector<double> frac, tau;     // natoms x 3
    double ecut = 0;
    int kmesh[3], qmesh[3];
    int N[3], nr = 0;
    int nk = 0, nq = 0;
    std::vector<hp::KSphere> ks;       // sphere per mesh k
    std::vector<hp::KSphere> kq_ks;    // [nq][nk] spheres at k+q off the k mesh (npw 0 where on the mesh)
    std::vector<hp::QFam> qfam;        // [nq]
    int ld = 0;                        // padded sphere length (max npw over k and every k+q)
    // projector rows and Hubbard rows
    int nproj = 0, nhub = 0;
    std::vector<int> proj_atom, proj_l, proj_m;
    std::vector<double> proj_D, proj_w, proj_pref;
    std::vector<int> hub_row_atom, hub_row_l, hub_row_m;
    std::vector<double> hub_row_w, hub_row_pref;
    std::vector<int> hub_atoms, hub_off, hub_mdim;
    hp::FftPlan fft;
    hp::SphereSet kset;                // mesh spheres
    // device constants
    double* d_bvec = nullptr;
    double* d_tau = nullptr;
    double* d_vloc = nullptr;          // [nr]
    double* d_projD = nullptr;         // [nproj]
    double2* d_beta_k = nullptr;       // [nk][nproj][ld]
    double2* d_phi_k = nullptr;        // [nk][nhub][ld]
    int* d_proj_int = nullptr;         // row_atom, row_l, row_m for projectors then Hubbard rows
    double* d_proj_dbl = nullptr;      // widths and prefactors
    // ground state
    bool have_gs = false;
    int nspin = 0, nocc = 0, nbnd = 0;
    double nelec = 0;
    double gap = 0;
    std::vector<double> eps;           // [nspin][nk][nbnd]
    double* d_vhxc = nullptr;          // [nspin][nr]
    double* d_rho = nullptr;           // [nspin][nr]
    double* d_veff = nullptr;          // [nspin][nr] V_loc + V_Hxc
    double2* d_psi = nullptr;          // [nspin][nk][nbnd][ld]
    // FP32 copies of the projector families for the mixed form (same layouts), built with the
    // response caches
    float2* d_psi32 = nullptr;
    float2* d_beta32 = nullptr;
    float2* d_phi32 = nullptr;
    // response caches (built on first use after a ground state)
    bool resp_ready = false;
    double2* d_ur = nullptr;           // [nspin][nk][nocc][nr]
    double2* d_aphi = nullptr;         // [nspin][nk][nocc][nhub] <phi_m,k|u_v>
    double* d_fxc = nullptr;           // [3 or 1][nr]
    float2* d_ur32 = nullptr;          // mixed precision: [nspin][nk][nocc][nr] FP32 u_k(r)
    float* d_veff32 = nullptr;         // mixed precision: FP32 copy of V_loc + V_Hxc
    float2* d_dv32 = nullptr;          // mixed precision: FP32 copy of Delta V_Hxc
    // sphere-sparse fused transforms (when the grid sizes are supported)
    bool fused = false;                // the fused transforms serve the current k and k+q sets
    bool fused_grid = false;           // the grid sizes allow the fused transforms
    int proj_rows_max = 128;           // rows of one combined beta / P_v projection
    bool vec32 = false;                // response band vectors stored in FP32 (mixed form, fused path)
    bool fused_reg = true;             // fused transforms with register-resident line FFTs
    bool ur_planes = false;            // the real-space band cache is plane-major (built by the fused path)
    void* d_vt = nullptr;              // plane-major V_eff [nspin][z][y][x] (double or float)
    void* d_vtx = nullptr;             // V_eff with x-major planes [nspin][z][x][y] (double or float)
    void* d_dvt = nullptr;             // plane-major Delta V (double2 or float2)
    double2* d_drho_pm = nullptr;      // plane-major Delta rho accumulation
    void* d_colA = nullptr;
    void* d_colB = nullptr;
    size_t col_cap = 0;                // bytes of each column buffer
    double alpha_pv = 0;
    hp::QCache qc;
    // response work arrays
    int resp_rows = 0;
    double2 *d_x = nullptr, *d_r = nullptr, *d_p = nullptr, *d_ap = nullptr, *d_b = nullptr, *d_vpu = nullptr;
    double *d_rz = nullptr, *d_rzold = nullptr, *d_rr = nullptr, *d_pap = nullptr;
    double2 *d_dv = nullptr, *d_dvout = nullptr, *d_drho = nullptr, *d_dvh = nullptr;
    double2* d_Pbuf = nullptr;         // projections [rows][128]
    double2* d_M = nullptr;            // [nspin][nhub][nhub]
    double2* d_dn = nullptr;           // [nhub_atoms][nspin][mmax][mmax]
    std::vector<double2*> d_hist_dx, d_hist_df;
    double2** d_hist_ptrs = nullptr;
    double* d_small = nullptr;         // small scalars for reductions / Broyden
    double* d_partial = nullptr;
    double* d_partials = nullptr;      // kMaxDots x 256 partial sums of the batched dot products
    // results
    std::map<std::pair<int, int>, hp::RespCols> cols;
    // symmetry classes of the Hubbard atoms (hp_perturbed_atoms; empty: every atom is perturbed)
    std::vector<int> hub_rep;          // per Hubbard atom: index (in hub_atoms) of its representative
    std::vector<int> hub_orient;       // per Hubbard atom: +1 / -1 / 0 spin orientation
    double dist_thr = 6e-4;            // bohr, distance tolerance of the column reconstruction
    // find_atpert 3: the space-group operations x -> W x + t (fractional) and the atom each atom goes to
    struct SymOp {
        int W[9];
        double t[3];
        std::vector<int> perm;
    };
    std::vector<SymOp> sym_ops;
    // scratch (device)
    double2* d_grid = nullptr;         // grid_cap x nr
    int grid_cap = 0;
    double2* d_scratch = nullptr;
    size_t scratch_elems = 0;
    hp::BandList L1, L2, L3;           // reusable band lists
    std::vector<void*> owned;          // device allocations freed in hp_destroy
    // DFT+U+V ground state (hp_set_hubbard)
    std::vector<double> hubU;          // [nhub_atoms] Ha
    std::vector<hp::HubPair> hubV;
    bool hub_on = false;
    double* d_hubU = nullptr;          // [nhub_atoms]
    int* d_hub_pair_int = nullptr;     // [npairs][5] i, j, R
    double* d_hub_pairV = nullptr;     // [npairs]
    int* d_hub_row_atom = nullptr;     // [nhub] Hubbard-atom index of each Hubbard row
    int* d_hub_off = nullptr;          // [nhub_atoms] first row, then [nhub_atoms] m dimension
    double* d_kfrac = nullptr;         // [nk][3] the k mesh, crystal coordinates
    double2* d_hub_occ = nullptr;      // occupation vector of the ground state's Hubbard potential
    double2* d_hubW = nullptr;         // [nspin][nk][nhub][nhub] W at the k mesh
};

namespace hp {

// device memory of a context: the registered allocator (hp_options.dev_alloc) or cudaMalloc
inline cudaError_t dev_malloc(hp_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    if (c->opt.dev_alloc) {
        *p = c->opt.dev_alloc(bytes, c->opt.alloc_user);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

inline void dev_free_raw(hp_ctx* c, void* p) {
    if (!p) return;
    if (c->opt.dev_alloc) {
        if (c->opt.dev_free) c->opt.dev_free(p, c->opt.alloc_user);
    } else {
        cudaFree(p);
    }
}

template <class T>
cudaError_t dalloc(hp_ctx* c, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    void* q = nullptr;
    cudaError_t e = dev_malloc(c, &q, sizeof(T) * n);
    if (e == cudaSuccess) {
        *p = (T*)q;
        c->owned.push_back(q);
    }
    return e;
}

template <class T>
cudaError_t h2d(T* d, const T* h, size_t n, cudaStream_t st) {
    return cudaMemcpyAsync(d, h, sizeof(T) * n, cudaMemcpyHostToDevice, st);
}

template <class T>
cudaError_t d2h(T* h, const T* d, size_t n, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(T) * n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace hp

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return hp::cuda_fail(c, e_, #call); \
    } while (0)
