// Ground state on the GPU: fixed-occupation LDA/LSDA SCF (the unperturbed states that the paper
// takes from pw.x, Sec. 3.1) by Chebyshev-filtered subspace iteration.
//
// Per SCF iteration and per (spin, k): filter the block of nbnd vectors with a degree-m Chebyshev
// polynomial of H that damps [a, b] (a = largest kept Ritz value, b = an upper bound of the
// spectrum), orthonormalise the block (Lowdin, S^-1/2 from a Jacobi eigen-decomposition of the
// overlap), Rayleigh-Ritz (Jacobi on X^H H X), density, V_Hxc, modified Broyden on V_Hxc.
// The small dense eigenproblems run as one CTA per (spin, k) matrix (cyclic Jacobi with
// round-robin pivot pairs); every vector operation uses the engine's batched kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "hp_internal.h"

namespace hp {

static inline int cdiv_(long long a, long long b) { return (int)((a + b - 1) / b); }
constexpr int kPS = 128;  // row stride of projection buffers

// ------------------------------------------------------------------------------------------------
// batched Hermitian Jacobi: A (n x n, row-major, per matrix) -> eigenvalues w (ascending) and
// eigenvectors as the columns of V.  One CTA per matrix; A and V in global memory.
// A plane rotation on (p, q) with a_pq = |a_pq| e:  U = [[c, s], [-s conj(e), c conj(e)]],
// t = tan(theta) = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 |a_pq|).
// Sweeps stop once a whole sweep skips every pair (|a_pq| <= 1e-16 (|a_pp| + |a_qq|)).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) jacobi_kernel(double2* __restrict__ Ab, double2* __restrict__ Vb,
                                                     double* __restrict__ wb, double2* __restrict__ tmpb, int n,
                                                     int max_sweeps) {
    extern __shared__ double shj[];
    const int m = n + (n & 1);  // even number of players (the extra one sits out)
    const int np = m / 2;
    double* cs = shj;            // [np] c
    double* sn = cs + np;        // [np] s
    double* er = sn + np;        // [np] Re e
    double* ei = er + np;        // [np] Im e
    int* pp = (int*)(ei + np);   // [np]
    int* qq = pp + np;           // [np]
    __shared__ int rot_count;
    double2* A = Ab + (long long)blockIdx.x * n * n;
    double2* V = Vb + (long long)blockIdx.x * n * n;
    double* w = wb + (long long)blockIdx.x * n;
    double2* tmp = tmpb + (long long)blockIdx.x * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = cmk((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // a sweep that finds every |a_pq| below 1e-16 (|a_pp| + |a_qq|) ends the iteration; pairs
        // below that threshold are skipped, so the rotation phase a_pq / |a_pq| is never formed
        // from underflowing (denormal) entries, which would make the rotation non-unitary
        if (threadIdx.x == 0) rot_count = 0;
        __syncthreads();
        for (int r = 0; r < m - 1; ++r) {
            // round-robin pairs: position 0 fixed, others rotate
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + r) % (m - 1)) + 1; };
                int p = player(i), q = player(m - 1 - i);
                if (p > q) { const int t = p; p = q; q = t; }
                pp[i] = p;
                qq[i] = q;
                double c = 1.0, s = 0.0, ere = 1.0, eim = 0.0;
                if (q < n) {
                    const double2 apq = A[(long long)p * n + q];
                    const double mag = hypot(apq.x, apq.y);
                    const double app = A[(long long)p * n + p].x, aqq = A[(long long)q * n + q].x;
                    if (mag > 1e-16 * (fabs(app) + fabs(aqq)) + 1e-300) {
                        atomicAdd(&rot_count, 1);
                        const double tau = (aqq - app) / (2.0 * mag);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        ere = apq.x / mag;
                        eim = apq.y / mag;
                    }
                }
                cs[i] = c;
                sn[i] = s;
                er[i] = ere;
                ei[i] = eim;
            }
            __syncthreads();
            // column update of A and V: (a_ip, a_iq) <- (c a_ip - s conj(e) a_iq, s a_ip + c conj(e) a_iq)
            for (int e = threadIdx.x; e < np * n; e += blockDim.x) {
                const int i = e % n, k = e / n;
                const int p = pp[k], q = qq[k];
                if (q >= n || sn[k] == 0.0) continue;
                const double c = cs[k], s = sn[k];
                const double2 ec = cmk(er[k], -ei[k]);
                {
                    const double2 ap = A[(long long)i * n + p], aq = A[(long long)i * n + q];
                    const double2 t = cmul(ec, aq);
                    A[(long long)i * n + p] = cmk(c * ap.x - s * t.x, c * ap.y - s * t.y);
                    A[(long long)i * n + q] = cmk(s * ap.x + c * t.x, s * ap.y + c * t.y);
                }
                {
                    const double2 vp = V[(long long)i * n + p], vq = V[(long long)i * n + q];
                    const double2 t = cmul(ec, vq);
                    V[(long long)i * n + p] = cmk(c * vp.x - s * t.x, c * vp.y - s * t.y);
                    V[(long long)i * n + q] = cmk(s * vp.x + c * t.x, s * vp.y + c * t.y);
                }
            }
            __syncthreads();
            // row update: (a_pj, a_qj) <- (c a_pj - s e a_qj, s a_pj + c e a_qj)
            for (int e = threadIdx.x; e < np * n; e += blockDim.x) {
                const int j = e % n, k = e / n;
                const int p = pp[k], q = qq[k];
                if (q >= n || sn[k] == 0.0) continue;
                const double c = cs[k], s = sn[k];
                const double2 ee = cmk(er[k], ei[k]);
                const double2 ap = A[(long long)p * n + j], aq = A[(long long)q * n + j];
                const double2 t = cmul(ee, aq);
                A[(long long)p * n + j] = cmk(c * ap.x - s * t.x, c * ap.y - s * t.y);
                A[(long long)q * n + j] = cmk(s * ap.x + c * t.x, s * ap.y + c * t.y);
            }
            __syncthreads();
        }
        if (rot_count == 0) break;
        __syncthreads();
    }
    // eigenvalues, ascending order, columns of V permuted accordingly (copy through tmp)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) tmp[e] = V[e];
    __syncthreads();
    if (threadIdx.x == 0) {
        // selection by rank: rank[i] = #{j : d_j < d_i or (d_j == d_i and j < i)}
        for (int i = 0; i < n; ++i) {
            const double di = A[(long long)i * n + i].x;
            int rank = 0;
            for (int j = 0; j < n; ++j) {
                const double dj = A[(long long)j * n + j].x;
                if (dj < di || (dj == di && j < i)) ++rank;
            }
            w[rank] = di;
            for (int row = 0; row < n; ++row) V[(long long)row * n + rank] = tmp[(long long)row * n + i];
        }
    }
}

// pack P rows (item c0 + j of segment g, stride 128) into matrices M[g][p][j] = P[c0 + j][p]
__global__ void pack_seg_kernel(const double2* __restrict__ P, const int* __restrict__ seg_start, int n,
                                double2* __restrict__ M) {
    const int g = blockIdx.x;
    const int c0 = seg_start[g];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int p = e / n, j = e % n;
        M[(long long)g * n * n + e] = P[(long long)(c0 + j) * kPS + p];
    }
}

// Pout[c0 + j][p] = V[g][p][j] * scale_j,  scale_j = 1/sqrt(w_j) (Lowdin) or 1
__global__ void seg_transform_kernel(const double2* __restrict__ V, const double* __restrict__ w, int lowdin,
                                     const int* __restrict__ seg_start, int n, double2* __restrict__ Pout,
                                     int* __restrict__ bad) {
    const int g = blockIdx.x;
    const int c0 = seg_start[g];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int p = e / n, j = e % n;
        double sc = 1.0;
        if (lowdin) {
            const double ww = w[(long long)g * n + j];
            if (!(ww > 1e-28)) {
                if (bad) *bad = 1;
                sc = 0.0;
            } else {
                sc = 1.0 / sqrt(ww);
            }
        }
        Pout[(long long)(c0 + j) * kPS + p] = cscale(V[(long long)g * n * n + e], sc);
    }
}

// y = a x - y
__global__ void vec_axmy_kernel(double2* __restrict__ y, const double2* __restrict__ x, double a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = cmk(a * x[i].x - y[i].x, a * x[i].y - y[i].y);
}

// row[c] *= 1/sqrt(nrm[row[c]])
__global__ void rows_normalize_kernel(const int* __restrict__ row, const double* __restrict__ nrm,
                                      double2* __restrict__ X, int ld) {
    const int c = blockIdx.y;
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= ld) return;
    const double v = nrm[row[c]];
    const double s = v > 0 ? 1.0 / sqrt(v) : 0.0;
    const long long o = (long long)row[c] * ld + G;
    X[o] = cscale(X[o], s);
}

// starting density: rho0 uniform; nspin = 2: rho0/2 (1 +- s(r)), s = clip(sum_I m_I 0.9 exp(-|r - tau_I|^2/2))
__global__ void init_density_kernel(double* __restrict__ rho, int N0, int N1, int N2, const double* __restrict__ cell,
                                    int nat, const double* __restrict__ frac, const int* __restrict__ mom, double rho0,
                                    int nspin) {
    const long long nr = (long long)N0 * N1 * N2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long long)gridDim.x * blockDim.x) {
        if (nspin == 1) {
            rho[e] = rho0;
            continue;
        }
        const int j2 = (int)(e % N2), j1 = (int)((e / N2) % N1), j0 = (int)(e / ((long long)N1 * N2));
        const double f[3] = {(double)j0 / N0, (double)j1 / N1, (double)j2 / N2};
        double s = 0.0;
        for (int a = 0; a < nat; ++a) {
            if (mom[a] == 0) continue;
            double d[3];
            for (int i = 0; i < 3; ++i) {
                d[i] = f[i] - frac[3 * a + i];
                d[i] -= rint(d[i]);
            }
            double r2 = 0.0;
            for (int x = 0; x < 3; ++x) {
                const double rx = d[0] * cell[x] + d[1] * cell[3 + x] + d[2] * cell[6 + x];
                r2 += rx * rx;
            }
            s += mom[a] * 0.9 * exp(-0.5 * r2);
        }
        s = fmin(0.9, fmax(-0.9, s));
        rho[e] = 0.5 * rho0 * (1.0 + s);
        rho[nr + e] = 0.5 * rho0 * (1.0 - s);
    }
}

// V_Hxc (complex storage, imaginary part 0) = V_H[rho_tot] + V_xc,s[rho]
__global__ void hxc_assemble_kernel(const double2* __restrict__ vh, const double* __restrict__ vxc, int nspin, int nr,
                                    double2* __restrict__ v) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x)
        for (int s = 0; s < nspin; ++s) v[(long long)s * nr + r] = cmk(vh[r].x + vxc[(long long)s * nr + r], 0.0);
}

// veff[s][r] = vloc[r] + Re v[s][r];  vhxc[s][r] = Re v[s][r]
__global__ void veff_kernel(const double* __restrict__ vloc, const double2* __restrict__ v, int nspin, int nr,
                            double* __restrict__ veff, double* __restrict__ vhxc) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x)
        for (int s = 0; s < nspin; ++s) {
            const double x = v[(long long)s * nr + r].x;
            veff[(long long)s * nr + r] = vloc[r] + x;
            vhxc[(long long)s * nr + r] = x;
        }
}

__global__ void vec_max_kernel(const double* __restrict__ a, long long n, double* __restrict__ out) {
    __shared__ double sh[32];
    double m = -1e300;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = -1e300;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, sh[i]);
        *out = r;
    }
}

__global__ void to_complex_kernel(const double* __restrict__ a, double2* __restrict__ z, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = cmk(a[i], 0.0);
}

}  // namespace hp

using namespace hp;

namespace {

// the band space an eigensolve works on: spheres, their k count, bands per (spin, k) and the
// projector family at those k (rows of band (s, k, v) are (s * nk + k) * nbnd + v)
struct EigSpace {
    const SphereSet* S;
    int nk, nbnd;
    const double2* beta;  // [nk][nproj][ld]
    const double2* phi = nullptr;   // DFT+U+V: Hubbard rows [nk][nhub][ld] ...
    const double2* hubW = nullptr;  // ... and W [nspin][nk][nhub][nhub]; null without a correction
};

struct GsWork {
    double2 *X = nullptr, *Y0 = nullptr, *Y1 = nullptr, *T = nullptr;
    double2 *Pb = nullptr, *Mb = nullptr, *Vb = nullptr, *Tmp = nullptr;
    double* w = nullptr;
    double* nrm = nullptr;
    int* bad = nullptr;
};

// Y = (H - shift) X for the list (shift taken from the list), including the nonlocal part
hp_status apply_h_shift(hp_ctx* c, const EigSpace& E, const BandList& L, const double2* X, double2* Y, double2* P) {
    hp_status s = apply_local(c, *E.S, L, X, Y, c->d_veff);
    if (s != HP_OK) return s;
    if (c->nproj > 0) {
        ProjMat B{E.beta, 0, (long long)c->nproj * c->ld, c->nproj, 0, nullptr};
        s = project(c, *E.S, L, B, X, P);
        if (s != HP_OK) return s;
        CK(k_expand(L, *E.S, B, P, c->d_projD, 1.0, Y, c->ld, c->st));
    }
    if (E.hubW) return hub_apply(c, *E.S, L, E.phi, nullptr, E.hubW, X, Y, false, false, P);
    return HP_OK;
}

// Rayleigh-Ritz on the block Y (rows of L): X <- orthonormal Ritz vectors, eps <- Ritz values
hp_status rayleigh_ritz(hp_ctx* c, const EigSpace& E, BandList& L, BandList& L0, GsWork& W, double2* Y, double2* X,
                        std::vector<double>& ritz) {
    const int n = E.nbnd, nseg = L.nseg, ld = c->ld;
    const long long nvec = (long long)L.nb * ld;
    const SphereSet& S = *E.S;
    ProjMat fam{nullptr, (long long)E.nk * n * ld, (long long)n * ld, n, 0, nullptr};
    // normalise columns, then overlap S = Y^H Y
    CK(k_band_dot(L, S, Y, Y, ld, W.nrm, c->st));
    {
        dim3 g(cdiv_(ld, 128), L.nb);
        rows_normalize_kernel<<<g, 128, 0, c->st>>>(L.d_row, W.nrm, Y, ld);
        HP_LAUNCHED();
        CK(cudaGetLastError());
    }
    fam.base = Y;
    hp_status s = project(c, S, L, fam, Y, W.Pb);
    if (s != HP_OK) return s;
    pack_seg_kernel<<<nseg, 256, 0, c->st>>>(W.Pb, L.d_seg_start, n, W.Mb);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    const size_t jsh = (size_t)(n / 2 + 1) * (4 * sizeof(double) + 2 * sizeof(int));
    jacobi_kernel<<<nseg, 256, jsh, c->st>>>(W.Mb, W.Vb, W.w, W.Tmp, n, 40);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    if (getenv("HP_VERBOSE")) {
        std::vector<double> ws((size_t)nseg * n);
        CK(d2h(ws.data(), W.w, ws.size(), c->st));
        double worst = 1.0;
        int wg = 0;
        for (int g = 0; g < nseg; ++g) {
            double lo = INFINITY, hi = 0;
            for (int j = 0; j < n; ++j) {
                lo = std::min(lo, ws[(size_t)g * n + j]);
                hi = std::max(hi, ws[(size_t)g * n + j]);
            }
            if (lo / hi < worst) { worst = lo / hi; wg = g; }
        }
        fprintf(stderr, "  overlap conditioning: worst min/max eigenvalue %.3e (segment %d)\n", worst, wg);
    }
    CK(cudaMemsetAsync(W.bad, 0, sizeof(int), c->st));
    seg_transform_kernel<<<nseg, 256, 0, c->st>>>(W.Vb, W.w, 1, L.d_seg_start, n, W.Pb, W.bad);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(X, 0, sizeof(double2) * nvec, c->st));
    CK(k_expand(L, S, fam, W.Pb, nullptr, 1.0, X, ld, c->st));
    // H in the orthonormal block
    s = apply_h_shift(c, E, L0, X, W.T, W.Pb);
    if (s != HP_OK) return s;
    fam.base = X;
    s = project(c, S, L, fam, W.T, W.Pb);
    if (s != HP_OK) return s;
    pack_seg_kernel<<<nseg, 256, 0, c->st>>>(W.Pb, L.d_seg_start, n, W.Mb);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    jacobi_kernel<<<nseg, 256, jsh, c->st>>>(W.Mb, W.Vb, W.w, W.Tmp, n, 40);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    seg_transform_kernel<<<nseg, 256, 0, c->st>>>(W.Vb, W.w, 0, L.d_seg_start, n, W.Pb, nullptr);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(Y, 0, sizeof(double2) * nvec, c->st));
    CK(k_expand(L, S, fam, W.Pb, nullptr, 1.0, Y, ld, c->st));
    CK(cudaMemcpyAsync(X, Y, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
    ritz.resize((size_t)nseg * n);
    CK(d2h(ritz.data(), W.w, ritz.size(), c->st));
    int bad = 0;
    CK(d2h(&bad, W.bad, 1, c->st));
    if (bad) return fail(c, HP_ENUMERIC, "hp_ground_state: the filtered block lost rank");
    return HP_OK;
}

// Chebyshev filter of degree m damping [a, b]: X <- p_m(H) X
hp_status cheb_filter(hp_ctx* c, const EigSpace& E, BandList& L, GsWork& W, double2* X, int m,
                      const std::vector<double>& a_seg, double b, BandList& Lc) {
    const int ld = c->ld;
    const long long nvec = (long long)L.nb * ld;
    // one interval for every segment: [a, b] with a the largest kept Ritz value over all segments
    // (a segment whose own top Ritz value lies below a is filtered a little less sharply)
    double a = -INFINITY;
    for (double x : a_seg) a = std::max(a, x);
    double e = 0.5 * (b - a);
    if (!(e > 0)) e = 1.0;
    const double centre = 0.5 * (b + a);
    Lc.row = L.row;
    Lc.k = L.k;
    Lc.spin = L.spin;
    Lc.shift.assign(L.nb, centre);
    hp_status s = upload_list(c, Lc);
    if (s != HP_OK) return s;
    // Y0 = X ; Y1 = (H - c) X / e
    CK(cudaMemcpyAsync(W.Y0, X, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
    s = apply_h_shift(c, E, Lc, X, W.Y1, W.Pb);
    if (s != HP_OK) return s;
    CK(k_vec_scale_copy(W.Y1, W.Y1, 1.0 / e, nvec, c->st));
    double2* ym1 = W.Y0;
    double2* y = W.Y1;
    for (int k = 2; k <= m; ++k) {
        s = apply_h_shift(c, E, Lc, y, W.T, W.Pb);
        if (s != HP_OK) return s;
        // y_{k} = 2/e (H - c) y_{k-1} - y_{k-2}, written over y_{k-2}
        vec_axmy_kernel<<<std::min(cdiv_(nvec, 256), 4096), 256, 0, c->st>>>(ym1, W.T, 2.0 / e, nvec);
        HP_LAUNCHED();
        CK(cudaGetLastError());
        double2* t = ym1;
        ym1 = y;
        y = t;
    }
    CK(cudaMemcpyAsync(X, y, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
    return HP_OK;
}

}  // namespace

// Pout[c0 + b][a] = sum_j V[g][a][j] w_j^-1/2 conj(V[g][b][j]) = (O^-1/2)_ab for O = V diag(w) V^H
__global__ void lowdin_sym_kernel(const double2* __restrict__ V, const double* __restrict__ w,
                                  const int* __restrict__ seg_start, int n, double2* __restrict__ Pout,
                                  int* __restrict__ bad) {
    const int g = blockIdx.x;
    const int c0 = seg_start[g];
    const double2* Vg = V + (long long)g * n * n;
    const double* wg = w + (long long)g * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int a = e / n, b = e % n;
        double2 s = cmk(0.0, 0.0);
        for (int j = 0; j < n; ++j) {
            const double ww = wg[j];
            if (!(ww > 1e-28)) {
                *bad = 1;
                continue;
            }
            s = cadd(s, cscale(cmulc(Vg[(long long)b * n + j], Vg[(long long)a * n + j]), 1.0 / sqrt(ww)));
        }
        Pout[(long long)(c0 + b) * kPS + a] = s;
    }
}

hp_status hp::ortho_hubbard_rows(hp_ctx* c, const SphereSet& S, int nk, double2* phi) {
    const int n = c->nhub, ld = c->ld;
    if (n == 0 || nk == 0) return HP_OK;
    const int rows = nk * n;
    double2 *Pb = nullptr, *Mb = nullptr, *Vb = nullptr, *Tmp = nullptr, *out = nullptr;
    double* w = nullptr;
    int* bad = nullptr;
    CK(dalloc(c, &Pb, (size_t)rows * kPS));
    CK(dalloc(c, &Mb, (size_t)nk * n * n));
    CK(dalloc(c, &Vb, (size_t)nk * n * n));
    CK(dalloc(c, &Tmp, (size_t)nk * n * n));
    CK(dalloc(c, &w, (size_t)nk * n));
    CK(dalloc(c, &out, (size_t)rows * ld));
    CK(dalloc(c, &bad, 1));
    auto release = [&]() {
        for (void* p : {(void*)Pb, (void*)Mb, (void*)Vb, (void*)Tmp, (void*)w, (void*)out, (void*)bad}) dfree(c, p);
    };
    BandList& L = c->L3;
    list_clear(L);
    for (int k = 0; k < nk; ++k)
        for (int m = 0; m < n; ++m) list_add(L, k * n + m, k, 0, 0.0);
    hp_status st = upload_list(c, L);
    if (st != HP_OK) return st;
    // O_ab = <phi_a|phi_b>: the projection of every row on the family, packed per k as M[k][a][b]
    ProjMat fam{phi, 0, (long long)n * ld, n, 0, nullptr};
    if ((st = project(c, S, L, fam, phi, Pb)) != HP_OK) return st;
    pack_seg_kernel<<<nk, 256, 0, c->st>>>(Pb, L.d_seg_start, n, Mb);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    const size_t jsh = (size_t)(n / 2 + 1) * (4 * sizeof(double) + 2 * sizeof(int));
    jacobi_kernel<<<nk, 256, jsh, c->st>>>(Mb, Vb, w, Tmp, n, 40);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(bad, 0, sizeof(int), c->st));
    lowdin_sym_kernel<<<nk, 256, 0, c->st>>>(Vb, w, L.d_seg_start, n, Pb, bad);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    // phi~_b = sum_a phi_a (O^-1/2)_ab
    CK(cudaMemsetAsync(out, 0, sizeof(double2) * (size_t)rows * ld, c->st));
    CK(k_expand(L, S, fam, Pb, nullptr, 1.0, out, ld, c->st));
    CK(cudaMemcpyAsync(phi, out, sizeof(double2) * (size_t)rows * ld, cudaMemcpyDeviceToDevice, c->st));
    int hbad = 0;
    CK(d2h(&hbad, bad, 1, c->st));
    release();
    if (hbad) return fail(c, HP_ENUMERIC, "ortho-atomic projectors: the Hubbard orbitals are linearly dependent");
    return HP_OK;
}

// Non-self-consistent occupied states at k points off the k mesh (k + q): Chebyshev-filtered
// subspace iteration with the ground-state potential V_eff held fixed, nocc + extra bands, until the
// occupied residuals ||(H - eps) u|| are below 1e-11.  out: [nspin][nkq][nocc][ld]; eps_occ:
// [nspin][nkq][nocc].
hp_status hp::nscf_states(hp_ctx* c, const std::vector<const KSphere*>& sph, const SphereSet& S, const double2* beta,
                          const double2* phi, const double2* hubW, double2* out, std::vector<double>& eps_occ) {
    const int nspin = c->nspin, nocc = c->nocc, ld = c->ld, nr = c->nr;
    const int nkq = (int)sph.size();
    int npw_min = ld;
    for (const KSphere* k : sph) npw_min = std::min(npw_min, k->npw);
    const int nbnd = std::min({kPS, nocc + std::max(6, nocc / 4), npw_min});
    if (nbnd <= nocc) return fail(c, HP_EINVAL, "nscf: fewer plane waves at k+q than occupied bands plus a buffer");
    const int rows = nspin * nkq * nbnd;
    const long long nvec = (long long)rows * ld;
    const long long ndv = (long long)nspin * nr;
    const EigSpace E{&S, nkq, nbnd, beta, phi, hubW};
    GsWork W;
    CK(dalloc(c, &W.X, nvec));
    CK(dalloc(c, &W.Y0, nvec));
    CK(dalloc(c, &W.Y1, nvec));
    CK(dalloc(c, &W.T, nvec));
    CK(dalloc(c, &W.Pb, (size_t)rows * kPS));
    CK(dalloc(c, &W.Mb, (size_t)nspin * nkq * nbnd * nbnd));
    CK(dalloc(c, &W.Vb, (size_t)nspin * nkq * nbnd * nbnd));
    CK(dalloc(c, &W.Tmp, (size_t)nspin * nkq * nbnd * nbnd));
    CK(dalloc(c, &W.w, (size_t)nspin * nkq * nbnd));
    CK(dalloc(c, &W.nrm, rows));
    CK(dalloc(c, &W.bad, 1));
    auto release = [&]() {
        for (void* p : {(void*)W.X, (void*)W.Y0, (void*)W.Y1, (void*)W.T, (void*)W.Pb, (void*)W.Mb, (void*)W.Vb,
                        (void*)W.Tmp, (void*)W.w, (void*)W.nrm, (void*)W.bad})
            dfree(c, p);
    };
    BandList& L = c->L1;
    BandList& L0 = c->L2;
    BandList& Lc = c->L3;
    list_clear(L);
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nkq; ++k)
            for (int v = 0; v < nbnd; ++v) list_add(L, (sp * nkq + k) * nbnd + v, k, sp, 0.0);
    hp_status st = upload_list(c, L);
    if (st != HP_OK) return st;
    L0.row = L.row;
    L0.k = L.k;
    L0.spin = L.spin;
    L0.shift.assign(L.nb, 0.0);
    if ((st = upload_list(c, L0)) != HP_OK) return st;
    {   // random start (64-bit LCG + xorshift output, seed 2204), damped at large |k+G|
        std::vector<double2> h(nvec, cmk(0.0, 0.0));
        uint64_t state = 2204ULL * 6364136223846793005ULL + 1442695040888963407ULL;
        auto next = [&]() {
            state = state * 6364136223846793005ULL + 1442695040888963407ULL;
            uint64_t x = state ^ (state >> 33);
            x *= 0xff51afd7ed558ccdULL;
            x ^= x >> 33;
            return (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        };
        for (int sp = 0; sp < nspin; ++sp)
            for (int k = 0; k < nkq; ++k)
                for (int v = 0; v < nbnd; ++v)
                    for (int i = 0; i < sph[k]->npw; ++i) {
                        const double damp = 1.0 / (1.0 + sph[k]->g2[i]);
                        h[((size_t)(sp * nkq + k) * nbnd + v) * ld + i] = cmk(next() * damp, next() * damp);
                    }
        CK(h2d(W.X, h.data(), h.size(), c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    double dplus = 0.0;
    for (int a = 0; a < (int)c->atom_species.size(); ++a) dplus += std::max(0.0, c->species[c->atom_species[a]].D);
    if (!c->d_small) CK(dalloc(c, &c->d_small, 512));
    vec_max_kernel<<<1, 256, 0, c->st>>>(c->d_veff, ndv, c->d_small + 100);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    double vmax = 0.0;
    CK(d2h(&vmax, c->d_small + 100, 1, c->st));
    const double b = 0.5 * c->ecut + vmax + 2.0 * dplus + 1.0;
    const int nseg = nspin * nkq;
    std::vector<double> ritz, aseg(nseg, 0.0);
    if ((st = rayleigh_ritz(c, E, L, L0, W, W.X, W.Y0, ritz)) != HP_OK) return st;
    CK(cudaMemcpyAsync(W.X, W.Y0, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
    double rmax = INFINITY;
    for (int pass = 0; pass < 120 && !(rmax < 1e-11); ++pass) {
        for (int gi = 0; gi < nseg; ++gi) aseg[gi] = ritz[(size_t)gi * nbnd + nbnd - 1];
        if ((st = cheb_filter(c, E, L, W, W.X, 10, aseg, b, Lc)) != HP_OK) return st;
        if ((st = rayleigh_ritz(c, E, L, L0, W, W.X, W.Y0, ritz)) != HP_OK) return st;
        CK(cudaMemcpyAsync(W.X, W.Y0, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
        if (pass < 2) continue;
        Lc.row = L.row;
        Lc.k = L.k;
        Lc.spin = L.spin;
        Lc.shift.assign(ritz.begin(), ritz.end());
        if ((st = upload_list(c, Lc)) != HP_OK) return st;
        if ((st = apply_h_shift(c, E, Lc, W.X, W.T, W.Pb)) != HP_OK) return st;
        CK(k_band_dot(Lc, S, W.T, W.T, ld, W.nrm, c->st));
        std::vector<double> nr2(rows);
        CK(d2h(nr2.data(), W.nrm, rows, c->st));
        rmax = 0.0;
        for (int sp = 0; sp < nspin; ++sp)
            for (int k = 0; k < nkq; ++k)
                for (int v = 0; v < nocc; ++v) rmax = std::max(rmax, std::sqrt(nr2[(size_t)(sp * nkq + k) * nbnd + v]));
        if (getenv("HP_VERBOSE")) fprintf(stderr, "nscf: pass %d max occupied residual %.3e\n", pass, rmax);
    }
    if (!(rmax < 1e-9)) {
        release();
        return fail(c, HP_ENOTCONV, "nscf: occupied residuals at k+q did not converge");
    }
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nkq; ++k)
            CK(cudaMemcpyAsync(out + (size_t)(sp * nkq + k) * nocc * ld, W.X + (size_t)(sp * nkq + k) * nbnd * ld,
                               sizeof(double2) * (size_t)nocc * ld, cudaMemcpyDeviceToDevice, c->st));
    eps_occ.assign((size_t)nspin * nkq * nocc, 0.0);
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nkq; ++k)
            for (int v = 0; v < nocc; ++v)
                eps_occ[(size_t)(sp * nkq + k) * nocc + v] = ritz[(size_t)(sp * nkq + k) * nbnd + v];
    CK(cudaStreamSynchronize(c->st));
    release();
    return HP_OK;
}

extern "C" hp_status hp_ground_state(hp_ctx* c, double nelec, int nspin, const int* init_moment, double tot_mag,
                                     hp_gs_info* info) {
    if (!c) return HP_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    if (nspin != 1 && nspin != 2) return fail(c, HP_EINVAL, "hp_ground_state: nspin must be 1 or 2");
    if (!std::isfinite(tot_mag) || (nspin == 1 && tot_mag != 0.0))
        return fail(c, HP_EINVAL, "hp_ground_state: tot_mag must be finite, and 0 for nspin = 1");
    if (tot_mag != 0.0)
        return fail(c, HP_ENOTIMPL, "hp_ground_state: only tot_mag = 0 (equal occupied band counts per spin) is built");
    const int nocc = (int)std::lround(nelec / 2.0);
    if (nocc < 1 || std::fabs(nelec - 2.0 * nocc) > 1e-9)
        return fail(c, HP_EINVAL, "hp_ground_state: nelec must be an even positive number");
    const int nextra = std::max(6, nocc / 4);
    const int nbnd = std::min(kPS, nocc + nextra);
    if (nbnd <= nocc) return fail(c, HP_EINVAL, "hp_ground_state: too many bands (at most 127 occupied)");
    for (int k = 0; k < c->nk; ++k)
        if (c->ks[k].npw < nbnd) return fail(c, HP_EINVAL, "hp_ground_state: fewer plane waves than bands");
    invalidate_response(c);
    c->have_gs = false;
    for (void* p : {(void*)c->d_vhxc, (void*)c->d_rho, (void*)c->d_veff, (void*)c->d_psi}) dfree(c, p);
    c->nspin = nspin;
    c->nocc = nocc;
    c->nbnd = nbnd;
    c->nelec = nelec;
    const int nk = c->nk, nr = c->nr, ld = c->ld;
    const int rows = nspin * nk * nbnd;
    const long long nvec = (long long)rows * ld;
    const long long ndv = (long long)nspin * nr;
    CK(dalloc(c, &c->d_vhxc, ndv));
    CK(dalloc(c, &c->d_rho, ndv));
    CK(dalloc(c, &c->d_veff, ndv));
    CK(dalloc(c, &c->d_psi, nvec));
    // DFT+U+V: the occupation matrices of the Hubbard potential ride at the end of the mixed vector
    const bool hub = c->hub_on;
    const long long nho = hub ? hub_occ_len(c, nspin) : 0;
    const long long ndvx = ndv + nho;
    for (void* p : {(void*)c->d_hub_occ, (void*)c->d_hubW}) dfree(c, p);
    c->d_hub_occ = nullptr;
    c->d_hubW = nullptr;
    if (hub) {
        CK(dalloc(c, &c->d_hub_occ, nho));
        CK(dalloc(c, &c->d_hubW, (size_t)nspin * nk * c->nhub * c->nhub));
    }
    const EigSpace E{&c->kset, nk, nbnd, c->d_beta_k, hub ? c->d_phi_k : nullptr, hub ? c->d_hubW : nullptr};
    GsWork W;
    CK(dalloc(c, &W.X, nvec));
    CK(dalloc(c, &W.Y0, nvec));
    CK(dalloc(c, &W.Y1, nvec));
    CK(dalloc(c, &W.T, nvec));
    CK(dalloc(c, &W.Pb, (size_t)rows * kPS));
    CK(dalloc(c, &W.Mb, (size_t)nspin * nk * nbnd * nbnd));
    CK(dalloc(c, &W.Vb, (size_t)nspin * nk * nbnd * nbnd));
    CK(dalloc(c, &W.Tmp, (size_t)nspin * nk * nbnd * nbnd));
    CK(dalloc(c, &W.w, (size_t)nspin * nk * nbnd));
    CK(dalloc(c, &W.nrm, rows));
    CK(dalloc(c, &W.bad, 1));
    // lists: all bands (shift 0) and the same items with shift = Ritz value (residuals)
    BandList& L = c->L1;
    BandList& Lc = c->L3;
    list_clear(L);
    for (int s = 0; s < nspin; ++s)
        for (int k = 0; k < nk; ++k)
            for (int v = 0; v < nbnd; ++v) list_add(L, (s * nk + k) * nbnd + v, k, s, 0.0);
    hp_status st = upload_list(c, L);
    if (st != HP_OK) return st;
    BandList& L0 = c->L2;  // same items, shift 0 (the Rayleigh quotient needs H itself)
    L0.row = L.row;
    L0.k = L.k;
    L0.spin = L.spin;
    L0.shift.assign(L.nb, 0.0);
    if ((st = upload_list(c, L0)) != HP_OK) return st;
    // random start (PCG-style 64-bit LCG + xorshift output, seed 2203), zero padding
    {
        std::vector<double2> h(nvec, cmk(0.0, 0.0));
        uint64_t state = 2203ULL * 6364136223846793005ULL + 1442695040888963407ULL;
        auto next = [&]() {
            state = state * 6364136223846793005ULL + 1442695040888963407ULL;
            uint64_t x = state ^ (state >> 33);
            x *= 0xff51afd7ed558ccdULL;
            x ^= x >> 33;
            return (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        };
        for (int s = 0; s < nspin; ++s)
            for (int k = 0; k < nk; ++k)
                for (int v = 0; v < nbnd; ++v)
                    for (int i = 0; i < c->ks[k].npw; ++i) {
                        const double damp = 1.0 / (1.0 + c->ks[k].g2[i]);
                        h[((size_t)(s * nk + k) * nbnd + v) * ld + i] = cmk(next() * damp, next() * damp);
                    }
        CK(h2d(W.X, h.data(), h.size(), c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    // starting potential from the starting density
    if (!c->d_small) CK(dalloc(c, &c->d_small, 512));
    if (!c->d_partial) CK(dalloc(c, &c->d_partial, 1024));
    double2 *vin, *vout, *dvh, *xprev, *fprev;
    double* vxc;
    CK(dalloc(c, &vin, ndvx));
    CK(dalloc(c, &vout, ndvx));
    CK(dalloc(c, &dvh, nr));
    CK(dalloc(c, &xprev, ndvx));
    CK(dalloc(c, &fprev, ndvx));
    CK(dalloc(c, &vxc, ndv));
    if (hub) CK(cudaMemsetAsync(vin + ndv, 0, sizeof(double2) * nho, c->st));  // start: empty occupations
    const int nmix = 6;
    std::vector<double2*> hdx(nmix), hdf(nmix);
    for (int i = 0; i < nmix; ++i) {
        CK(dalloc(c, &hdx[i], ndvx));
        CK(dalloc(c, &hdf[i], ndvx));
    }
    double2** dptrs;
    CK(dalloc(c, &dptrs, 2 * (nmix + 1)));
    {
        double* d_cell;
        double* d_frac;
        int* d_mom;
        const int nat = (int)c->atom_species.size();
        std::vector<int> mom(nat, 0);
        if (init_moment)
            for (int a = 0; a < nat; ++a) mom[a] = init_moment[a] > 0 ? 1 : (init_moment[a] < 0 ? -1 : 0);
        CK(dalloc(c, &d_cell, 9));
        CK(dalloc(c, &d_frac, 3 * nat));
        CK(dalloc(c, &d_mom, nat));
        CK(h2d(d_cell, c->cell, 9, c->st));
        CK(h2d(d_frac, c->frac.data(), 3 * nat, c->st));
        CK(h2d(d_mom, mom.data(), nat, c->st));
        init_density_kernel<<<cdiv_(nr, 256), 256, 0, c->st>>>(c->d_rho, c->N[0], c->N[1], c->N[2], d_cell, nat, d_frac,
                                                                d_mom, nelec / c->omega, nspin);
        HP_LAUNCHED();
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(c->st));
        dfree(c, d_cell);
        dfree(c, d_frac);
        dfree(c, d_mom);
    }
    const double zq[3] = {0.0, 0.0, 0.0};
    auto hxc = [&](double2* out) -> hp_status {
        // V_H[rho_tot]
        to_complex_kernel<<<cdiv_(nr, 256), 256, 0, c->st>>>(c->d_rho, dvh, nr);
        HP_LAUNCHED();
        CK(cudaGetLastError());
        if (nspin == 2) {
            double2* tmp = out;  // use out as scratch for the second spin
            to_complex_kernel<<<cdiv_(nr, 256), 256, 0, c->st>>>(c->d_rho + nr, tmp, nr);
            HP_LAUNCHED();
            CK(cudaGetLastError());
            CK(k_vec_axpy(dvh, tmp, 1.0, nr, c->st));
        }
        CK(fft3d(c->fft, dvh, 1, -1, c->st));
        CK(k_hartree_q(dvh, c->N, c->d_bvec, zq, 4.0 * c->ecut, 1.0 / nr, c->st));
        CK(fft3d(c->fft, dvh, 1, +1, c->st));
        CK(k_xc(c->d_rho, nspin, nr, vxc, nullptr, c->st));
        hxc_assemble_kernel<<<cdiv_(nr, 256), 256, 0, c->st>>>(dvh, vxc, nspin, nr, out);
        HP_LAUNCHED();
        return cudaGetLastError() == cudaSuccess ? HP_OK : fail(c, HP_ECUDA, "hxc");
    };
    if ((st = hxc(vin)) != HP_OK) return st;
    // upper bound of the spectrum: max kinetic + max V_eff + positive projector strengths
    double dplus = 0.0;
    for (int a = 0; a < (int)c->atom_species.size(); ++a) dplus += std::max(0.0, c->species[c->atom_species[a]].D);
    const double f = nspin == 1 ? 2.0 : 1.0;
    const double wrho = f / (nk * c->omega);
    std::vector<double> ritz;
    int it = 0, nhist = 0;
    double res = INFINITY;
    bool converged = false;
    const int nseg = nspin * nk;
    std::vector<double> aseg(nseg, 0.0);
    const int deg = 10;
    const bool verbose = getenv("HP_VERBOSE") != nullptr;
    for (it = 1; it <= c->opt.gs_maxiter; ++it) {
        veff_kernel<<<cdiv_(nr, 256), 256, 0, c->st>>>(c->d_vloc, vin, nspin, nr, c->d_veff, c->d_vhxc);
        HP_LAUNCHED();
        CK(cudaGetLastError());
        if (hub && (st = hub_build_w(c, vin + ndv, nspin, nk, c->d_kfrac, c->d_hubW)) != HP_OK) return st;
        vec_max_kernel<<<1, 256, 0, c->st>>>(c->d_veff, ndv, c->d_small + 100);
        HP_LAUNCHED();
        CK(cudaGetLastError());
        double vmax = 0.0;
        CK(d2h(&vmax, c->d_small + 100, 1, c->st));
        const double b = 0.5 * c->ecut + vmax + 2.0 * dplus + 1.0;
        // subspace iteration: a few passes on the first SCF steps, one afterwards
        const int passes = it == 1 ? 4 : (it <= 5 ? 2 : 1);
        for (int pass = 0; pass < passes; ++pass) {
            if (!ritz.empty()) {
                for (int g = 0; g < nseg; ++g) aseg[g] = ritz[(size_t)g * nbnd + nbnd - 1];
                if ((st = cheb_filter(c, E, L, W, W.X, deg, aseg, b, Lc)) != HP_OK) return st;
            }
            if ((st = rayleigh_ritz(c, E, L, L0, W, W.X, W.Y0, ritz)) != HP_OK) return st;
            CK(cudaMemcpyAsync(W.X, W.Y0, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
        }
        // density of the occupied Ritz vectors
        CK(cudaMemsetAsync(c->d_rho, 0, sizeof(double) * ndv, c->st));
        {
            BandList& Lo = c->L3;
            list_clear(Lo);
            for (int s = 0; s < nspin; ++s)
                for (int k = 0; k < nk; ++k)
                    for (int v = 0; v < nocc; ++v) list_add(Lo, (s * nk + k) * nbnd + v, k, s, 0.0);
            if ((st = upload_list(c, Lo)) != HP_OK) return st;
            const int gchunk = band_batch(c, Lo.nb);  // fixed by the sizes, not by the buffer's history
            if ((st = ensure_grid(c, gchunk)) != HP_OK) return st;
            for (int c0 = 0; c0 < Lo.nb; c0 += gchunk) {
                const int nc = std::min(gchunk, Lo.nb - c0);
                CK(k_scatter(c->kset, Lo, c0, nc, W.X, ld, c->d_grid, nr, c->st));
                CK(fft3d(c->fft, c->d_grid, nc, +1, c->st));
                CK(k_density_acc(c->d_grid, nc, nr, Lo, c0, wrho, nspin, c->d_rho, c->st));
            }
            if (hub) {  // occupation matrices of the occupied states, at the end of the output vector
                ProjMat F{c->d_phi_k, 0, (long long)c->nhub * ld, c->nhub, 0, nullptr};
                if ((st = project(c, c->kset, Lo, F, W.X, W.Pb)) != HP_OK) return st;
                if ((st = hub_occupations(c, W.Pb, nspin, nk, nocc, c->d_kfrac, vout + ndv)) != HP_OK) return st;
            }
        }
        if ((st = hxc(vout)) != HP_OK) return st;
        CK(k_vec_sub(vout, vout, vin, ndvx, c->st));  // residual F
        double ff = 0.0, fn = 0.0;
        CK(k_vec_dot(vout, vout, ndv, c->d_small, c->d_partial, c->st));
        CK(d2h(&ff, c->d_small, 1, c->st));
        if (hub) {
            CK(k_vec_dot(vout + ndv, vout + ndv, nho, c->d_small, c->d_partial, c->st));
            CK(d2h(&fn, c->d_small, 1, c->st));
        }
        if (!std::isfinite(ff) || !std::isfinite(fn)) return fail(c, HP_ENUMERIC, "hp_ground_state: non-finite residual");
        res = std::max(std::sqrt(ff / (double)ndv), hub ? std::sqrt(fn / (double)nho) : 0.0);
        if (verbose)
            fprintf(stderr, "hp_ground_state: it %d res %.3e vmax %.3f b %.3f top %.4f occ %.6f\n", it, res, vmax, b,
                    aseg.empty() ? 0.0 : *std::max_element(ritz.begin(), ritz.end()), ritz[nocc - 1]);
        if (res < c->opt.gs_tol) {
            converged = true;
            break;
        }
        // modified Broyden on V_Hxc (alpha 0.3, w0 0.01, history nmix)
        if (it > 1) {
            if (nhist == nmix) {
                double2* t0x = hdx[0];
                double2* t0f = hdf[0];
                for (int i = 0; i + 1 < nmix; ++i) {
                    hdx[i] = hdx[i + 1];
                    hdf[i] = hdf[i + 1];
                }
                hdx[nmix - 1] = t0x;
                hdf[nmix - 1] = t0f;
                --nhist;
            }
            CK(k_vec_sub(hdf[nhist], vout, fprev, ndvx, c->st));
            CK(k_vec_sub(hdx[nhist], vin, xprev, ndvx, c->st));
            double nn = 0.0;
            CK(k_vec_dot(hdf[nhist], hdf[nhist], ndvx, c->d_small, c->d_partial, c->st));
            CK(d2h(&nn, c->d_small, 1, c->st));
            if (nn > 0) {
                CK(k_vec_scale_copy(hdf[nhist], hdf[nhist], 1.0 / std::sqrt(nn), ndvx, c->st));
                CK(k_vec_scale_copy(hdx[nhist], hdx[nhist], 1.0 / std::sqrt(nn), ndvx, c->st));
                ++nhist;
            }
        }
        CK(cudaMemcpyAsync(xprev, vin, sizeof(double2) * ndvx, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(fprev, vout, sizeof(double2) * ndvx, cudaMemcpyDeviceToDevice, c->st));
        const int m = nhist;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j <= m; ++j)
                CK(k_vec_dot(hdf[i], j < m ? hdf[j] : vout, ndvx, c->d_small + 16 + i * (m + 1) + j, c->d_partial, c->st));
        CK(k_broyden_coef(c->d_small + 16, m, m + 1, 0.01, c->d_small + 8, c->st));
        std::vector<const double2*> ptrs(2 * (nmix + 1), nullptr);
        for (int i = 0; i < m; ++i) {
            ptrs[i] = hdx[i];
            ptrs[nmix + 1 + i] = hdf[i];
        }
        CK(h2d((const double2**)dptrs, ptrs.data(), ptrs.size(), c->st));
        CK(k_broyden_apply(vin, vout, (const double2* const*)dptrs, (const double2* const*)(dptrs + nmix + 1),
                           c->d_small + 8, m, 0.3, ndvx, c->st));
    }
    // polish: extra filter passes at the final potential until the occupied residuals are small
    veff_kernel<<<cdiv_(nr, 256), 256, 0, c->st>>>(c->d_vloc, vin, nspin, nr, c->d_veff, c->d_vhxc);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    if (hub && (st = hub_build_w(c, vin + ndv, nspin, nk, c->d_kfrac, c->d_hubW)) != HP_OK) return st;
    double rmax = INFINITY;
    for (int pass = 0; pass < 30; ++pass) {
        vec_max_kernel<<<1, 256, 0, c->st>>>(c->d_veff, ndv, c->d_small + 100);
        HP_LAUNCHED();
        double vmax = 0.0;
        CK(d2h(&vmax, c->d_small + 100, 1, c->st));
        const double b = 0.5 * c->ecut + vmax + 2.0 * dplus + 1.0;
        for (int g = 0; g < nseg; ++g) aseg[g] = ritz[(size_t)g * nbnd + nbnd - 1];
        if ((st = cheb_filter(c, E, L, W, W.X, deg, aseg, b, Lc)) != HP_OK) return st;
        if ((st = rayleigh_ritz(c, E, L, L0, W, W.X, W.Y0, ritz)) != HP_OK) return st;
        CK(cudaMemcpyAsync(W.X, W.Y0, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
        // residual norms ||(H - eps) x|| of the occupied bands
        Lc.row = L.row;
        Lc.k = L.k;
        Lc.spin = L.spin;
        Lc.shift.assign(ritz.begin(), ritz.end());
        if ((st = upload_list(c, Lc)) != HP_OK) return st;
        if ((st = apply_h_shift(c, E, Lc, W.X, W.T, W.Pb)) != HP_OK) return st;
        CK(k_band_dot(Lc, c->kset, W.T, W.T, ld, W.nrm, c->st));
        std::vector<double> nr2(rows);
        CK(d2h(nr2.data(), W.nrm, rows, c->st));
        rmax = 0.0;
        int ws = 0, wk = 0, wv = 0;
        for (int s = 0; s < nspin; ++s)
            for (int k = 0; k < nk; ++k)
                for (int v = 0; v < nocc; ++v) {
                    const double r = std::sqrt(nr2[(size_t)(s * nk + k) * nbnd + v]);
                    if (r > rmax) { rmax = r; ws = s; wk = k; wv = v; }
                }
        if (verbose) {
            fprintf(stderr, "  worst s %d k %d v %d ritz:", ws, wk, wv);
            for (int v = 0; v < nbnd; ++v) fprintf(stderr, " %.4f(%.0e)", ritz[(size_t)(ws * nk + wk) * nbnd + v],
                                                   std::sqrt(nr2[(size_t)(ws * nk + wk) * nbnd + v]));
            fprintf(stderr, "\n");
        }
        if (verbose) fprintf(stderr, "hp_ground_state: polish %d max occupied residual %.3e\n", pass, rmax);
        if (rmax < 1e-11) break;
    }
    // the density of the final states (consistent with the eigenpairs kept)
    CK(cudaMemcpyAsync(c->d_psi, W.X, sizeof(double2) * nvec, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemsetAsync(c->d_rho, 0, sizeof(double) * ndv, c->st));
    {
        BandList& Lo = c->L3;
        list_clear(Lo);
        for (int s = 0; s < nspin; ++s)
            for (int k = 0; k < nk; ++k)
                for (int v = 0; v < nocc; ++v) list_add(Lo, (s * nk + k) * nbnd + v, k, s, 0.0);
        if ((st = upload_list(c, Lo)) != HP_OK) return st;
        const int gchunk = band_batch(c, Lo.nb);
        if ((st = ensure_grid(c, gchunk)) != HP_OK) return st;
        for (int c0 = 0; c0 < Lo.nb; c0 += gchunk) {
            const int nc = std::min(gchunk, Lo.nb - c0);
            CK(k_scatter(c->kset, Lo, c0, nc, c->d_psi, ld, c->d_grid, nr, c->st));
            CK(fft3d(c->fft, c->d_grid, nc, +1, c->st));
            CK(k_density_acc(c->d_grid, nc, nr, Lo, c0, wrho, nspin, c->d_rho, c->st));
        }
        if (hub) {  // the occupations (and W) the response's Hamiltonian uses: those of the final states
            ProjMat F{c->d_phi_k, 0, (long long)c->nhub * ld, c->nhub, 0, nullptr};
            if ((st = project(c, c->kset, Lo, F, c->d_psi, W.Pb)) != HP_OK) return st;
            if ((st = hub_occupations(c, W.Pb, nspin, nk, nocc, c->d_kfrac, c->d_hub_occ)) != HP_OK) return st;
            if ((st = hub_build_w(c, c->d_hub_occ, nspin, nk, c->d_kfrac, c->d_hubW)) != HP_OK) return st;
        }
    }
    CK(cudaStreamSynchronize(c->st));
    c->eps = ritz;
    double homo = -INFINITY, lumo = INFINITY, gap = INFINITY;
    for (int s = 0; s < nspin; ++s) {
        double h = -INFINITY, l = INFINITY;
        for (int k = 0; k < nk; ++k) {
            h = std::max(h, ritz[(size_t)(s * nk + k) * nbnd + nocc - 1]);
            l = std::min(l, ritz[(size_t)(s * nk + k) * nbnd + nocc]);
        }
        homo = std::max(homo, h);
        lumo = std::min(lumo, l);
        gap = std::min(gap, l - h);
    }
    c->gap = gap;
    for (void* p : {(void*)W.X, (void*)W.Y0, (void*)W.Y1, (void*)W.T, (void*)W.Pb, (void*)W.Mb, (void*)W.Vb,
                    (void*)W.Tmp, (void*)W.w, (void*)W.nrm, (void*)W.bad, (void*)vin, (void*)vout, (void*)dvh,
                    (void*)xprev, (void*)fprev, (void*)vxc, (void*)dptrs})
        dfree(c, p);
    for (int i = 0; i < nmix; ++i) {
        dfree(c, hdx[i]);
        dfree(c, hdf[i]);
    }
    c->have_gs = true;
    if (info) {
        info->iterations = std::min(it, c->opt.gs_maxiter);
        info->residual = res;
        info->gap = gap;
        info->homo = homo;
        info->lumo = lumo;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged || rmax > 1e-9) return fail(c, HP_ENOTCONV, "hp_ground_state: SCF or eigenvector residual cap reached");
    if (!(gap > 1e-4)) return fail(c, HP_ENOGAP, "hp_ground_state: no gap at the fixed band count");
    return HP_OK;
}

// Lowest levels of the bare Hamiltonian T + V_loc + V_NL (no Hxc, no Hubbard term) at the first k
// point of the mesh (Gamma for the Gamma-centred meshes), by the non-self-consistent eigensolver.
extern "C" hp_status hp_bare_levels(hp_ctx* c, int ik, int nlev, double* eps) {
    if (!c) return HP_EINVAL;
    if (ik < 0 || ik >= c->nk || nlev < 1 || nlev > 100 || !eps)
        return fail(c, HP_EINVAL, "hp_bare_levels: k index in the mesh, 1 <= nlev <= 100 and eps given");
    if (c->ks[ik].npw < nlev + 6) return fail(c, HP_EINVAL, "hp_bare_levels: fewer plane waves than levels");
    const int nspin0 = c->nspin, nocc0 = c->nocc;
    double* veff0 = c->d_veff;
    const bool hub0 = c->hub_on;
    c->nspin = 1;
    c->nocc = nlev;
    c->d_veff = c->d_vloc;
    c->hub_on = false;
    SphereSet S0;
    std::vector<const KSphere*> sph{&c->ks[ik]};
    const bool fused0 = c->fused;
    hp_status st = upload_sphereset(c, sph, nullptr, S0);
    c->fused = fused0;
    double2* psi = nullptr;
    std::vector<double> lev;
    if (st == HP_OK && dalloc(c, &psi, (size_t)nlev * c->ld) != cudaSuccess) st = fail(c, HP_ENOMEM, "hp_bare_levels");
    if (st == HP_OK)
        st = nscf_states(c, sph, S0, c->d_beta_k + (size_t)ik * std::max(1, c->nproj) * c->ld, nullptr, nullptr, psi, lev);
    c->nspin = nspin0;
    c->nocc = nocc0;
    c->d_veff = veff0;
    c->hub_on = hub0;
    dfree(c, psi);
    free_sphereset(c, S0);
    if (st != HP_OK) return st;
    for (int i = 0; i < nlev; ++i) eps[i] = lev[i];
    return HP_OK;
}

extern "C" hp_status hp_selftest_eigh(int n, int nbatch, const double* A, double* w, double* V) {
    if (n < 1 || n > 512 || nbatch < 1 || !A || !w || !V) return HP_EINVAL;
    const size_t nn = (size_t)n * n * nbatch;
    double2 *dA = nullptr, *dV = nullptr, *dT = nullptr;
    double* dw = nullptr;
    hp_status st = HP_OK;
    if (cudaMalloc(&dA, sizeof(double2) * nn) != cudaSuccess || cudaMalloc(&dV, sizeof(double2) * nn) != cudaSuccess ||
        cudaMalloc(&dT, sizeof(double2) * nn) != cudaSuccess || cudaMalloc(&dw, sizeof(double) * n * nbatch) != cudaSuccess)
        st = HP_ECUDA;
    hp::g_allocs.fetch_add(4, std::memory_order_relaxed);
    if (st == HP_OK && cudaMemcpy(dA, A, sizeof(double2) * nn, cudaMemcpyHostToDevice) != cudaSuccess) st = HP_ECUDA;
    if (st == HP_OK) {
        const size_t jsh = (size_t)(n / 2 + 1) * (4 * sizeof(double) + 2 * sizeof(int));
        hp::jacobi_kernel<<<nbatch, 256, jsh>>>(dA, dV, dw, dT, n, 40);
        HP_LAUNCHED();
        if (cudaDeviceSynchronize() != cudaSuccess) st = HP_ECUDA;
    }
    if (st == HP_OK && (cudaMemcpy(V, dV, sizeof(double2) * nn, cudaMemcpyDeviceToHost) != cudaSuccess ||
                        cudaMemcpy(w, dw, sizeof(double) * n * nbatch, cudaMemcpyDeviceToHost) != cudaSuccess))
        st = HP_ECUDA;
    cudaFree(dA);
    cudaFree(dV);
    cudaFree(dT);
    cudaFree(dw);
    return st;
}
