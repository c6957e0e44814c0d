// Orchestration and C ABI of the DFPT Hubbard engine.
//
// hp_setup        a1: cell, reciprocal lattice, wavefunction spheres, FFT grid maps, closed-form
//                 form factors beta and phi at the k mesh, V_loc on the grid.
// hp_response     a3-a10 for one (q, J): V_pert u, Delta V_Hxc u, P_c, the batched Sternheimer CG
//                 over every (spin, k, band), Delta rho, Delta n, Delta V_Hxc, modified Broyden.
// hp_hubbard      a11: q-sum with phases, chi_0 and chi, FP64 inverses, U and V.
// Every arithmetic step runs in the kernels of kernels.cu / fft.cu; host code only builds index
// lists, moves a few scalars for control flow and copies results out.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <thread>
#include <cstring>

#include "hp_internal.h"

using namespace hp;

namespace hp {

std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};

constexpr double kHaToEv = 27.211386245988;
constexpr int kMmax = 5;
constexpr int kPStride = 128;

hp_status fail(hp_ctx* c, hp_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

hp_status cuda_fail(hp_ctx* c, cudaError_t e, const char* what) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    if (c) c->err = buf;
    return e == cudaErrorMemoryAllocation ? HP_ENOMEM : HP_ECUDA;
}


void dfree(hp_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->owned.begin(), c->owned.end(), p);
    if (it != c->owned.end()) c->owned.erase(it);
    dev_free_raw(c, p);
}

int good_fft_size(int n) {
    for (int m = std::max(1, n);; ++m) {
        int k = m;
        for (int p : {2, 3, 5})
            while (k % p == 0) k /= p;
        if (k == 1) return m;
    }
}

void cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// enumerate the sphere |k + m.B|^2 <= ecut, ordered by Miller index (column by column)
void build_sphere(const hp_ctx* c, const double kfrac[3], KSphere& s) {
    for (int i = 0; i < 3; ++i) {
        s.kfrac[i] = kfrac[i];
        s.kcart[i] = kfrac[0] * c->bvec[0 * 3 + i] + kfrac[1] * c->bvec[1 * 3 + i] + kfrac[2] * c->bvec[2 * 3 + i];
    }
    const double kn = std::sqrt(s.kcart[0] * s.kcart[0] + s.kcart[1] * s.kcart[1] + s.kcart[2] * s.kcart[2]);
    const double gmax = std::sqrt(c->ecut) + kn;
    int lim[3];
    for (int i = 0; i < 3; ++i) {
        const double an = std::sqrt(c->cell[3 * i] * c->cell[3 * i] + c->cell[3 * i + 1] * c->cell[3 * i + 1] +
                                    c->cell[3 * i + 2] * c->cell[3 * i + 2]);
        lim[i] = (int)std::ceil(gmax * an / (2.0 * M_PI)) + 1;
    }
    struct E { double g2; int m[3]; };
    std::vector<E> v;
    for (int a = -lim[0]; a <= lim[0]; ++a)
        for (int b = -lim[1]; b <= lim[1]; ++b)
            for (int d = -lim[2]; d <= lim[2]; ++d) {
                double K[3];
                for (int i = 0; i < 3; ++i) K[i] = s.kcart[i] + a * c->bvec[i] + b * c->bvec[3 + i] + d * c->bvec[6 + i];
                const double g2 = K[0] * K[0] + K[1] * K[1] + K[2] * K[2];
                if (g2 <= c->ecut) v.push_back({g2, {a, b, d}});
            }
    // column by column (m0, m1), then m2: the points of one z-column of the FFT grid are contiguous
    std::sort(v.begin(), v.end(), [](const E& x, const E& y) {
        if (x.m[0] != y.m[0]) return x.m[0] < y.m[0];
        if (x.m[1] != y.m[1]) return x.m[1] < y.m[1];
        return x.m[2] < y.m[2];
    });
    s.npw = (int)v.size();
    s.miller.resize(3 * s.npw);
    s.g2.resize(s.npw);
    for (int i = 0; i < s.npw; ++i) {
        for (int j = 0; j < 3; ++j) s.miller[3 * i + j] = v[i].m[j];
        s.g2[i] = v[i].g2;
    }
}

int grid_index(const hp_ctx* c, int m0, int m1, int m2) {
    auto md = [](int m, int n) { return ((m % n) + n) % n; };
    return (md(m0, c->N[0]) * c->N[1] + md(m1, c->N[1])) * c->N[2] + md(m2, c->N[2]);
}

// sphere set upload: npw per k, grid index (Miller shifted by -shift[k]), |k+G|^2
hp_status upload_sphereset(hp_ctx* c, const std::vector<const KSphere*>& sph, const std::vector<std::array<int, 3>>* shift,
                           SphereSet& S) {
    const int nk = (int)sph.size(), ld = c->ld;
    S.nk = nk;
    S.ld = ld;
    S.npw.resize(nk);
    std::vector<int> idx((size_t)nk * ld, 0);
    std::vector<double> g2((size_t)nk * ld, 0.0);
    for (int k = 0; k < nk; ++k) {
        const KSphere& s = *sph[k];
        S.npw[k] = s.npw;
        std::vector<char> seen(c->nr, 0);
        for (int i = 0; i < s.npw; ++i) {
            int m[3];
            for (int j = 0; j < 3; ++j) m[j] = s.miller[3 * i + j] - (shift ? (*shift)[k][j] : 0);
            const int gi = grid_index(c, m[0], m[1], m[2]);
            if (seen[gi]) return fail(c, HP_EINVAL, "FFT grid too small to hold the wavefunction sphere");
            seen[gi] = 1;
            idx[(size_t)k * ld + i] = gi;
            g2[(size_t)k * ld + i] = s.g2[i];
        }
    }
    // columns: runs of points with the same grid (x, y)
    std::vector<std::vector<int>> cs(nk), cl(nk), cxy(nk);
    std::vector<int> iz((size_t)nk * ld, 0), ncol(nk);
    int ncmax = 0;
    for (int k = 0; k < nk; ++k) {
        const int npw = S.npw[k];
        for (int i = 0; i < npw; ++i) {
            const int gi = idx[(size_t)k * ld + i];
            const int xy = gi / c->N[2];
            iz[(size_t)k * ld + i] = gi % c->N[2];
            if (i == 0 || xy != idx[(size_t)k * ld + i - 1] / c->N[2]) {
                cs[k].push_back(i);
                cl[k].push_back(0);
                cxy[k].push_back(xy);
            }
            cl[k].back() += 1;
        }
        ncol[k] = (int)cs[k].size();
        ncmax = std::max(ncmax, ncol[k]);
    }
    std::vector<int> hs((size_t)nk * ncmax, 0), hl((size_t)nk * ncmax, 0), hxy((size_t)nk * ncmax, 0);
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < ncol[k]; ++j) {
            hs[(size_t)k * ncmax + j] = cs[k][j];
            hl[(size_t)k * ncmax + j] = cl[k][j];
            hxy[(size_t)k * ncmax + j] = cxy[k][j];
        }
    if (!S.d_npw) {
        CK(dalloc(c, &S.d_npw, nk));
        CK(dalloc(c, &S.d_idx, (size_t)nk * ld));
        CK(dalloc(c, &S.d_g2, (size_t)nk * ld));
        CK(dalloc(c, &S.d_prec, (size_t)nk * ld));
        CK(dalloc(c, &S.d_prec32, (size_t)nk * ld));
        CK(dalloc(c, &S.d_kin32, (size_t)nk * ld));
        CK(dalloc(c, &S.d_iz, (size_t)nk * ld));
        CK(dalloc(c, &S.d_ncol, nk));
    }
    if (ncmax > S.ncmax) {
        for (void* p : {(void*)S.d_col_start, (void*)S.d_col_len, (void*)S.d_col_xy}) dfree(c, p);
        CK(dalloc(c, &S.d_col_start, (size_t)nk * ncmax));
        CK(dalloc(c, &S.d_col_len, (size_t)nk * ncmax));
        CK(dalloc(c, &S.d_col_xy, (size_t)nk * ncmax));
    }
    S.ncmax = ncmax;
    S.ncol = ncol;
    // whether each column is one run of consecutive z, and the run of columns of each grid x
    const int N0 = c->N[0], N1 = c->N[1], N2 = c->N[2];
    bool contig = true, xruns = true;
    std::vector<int> xt((size_t)nk * N0 * 3, 0);
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < ncol[k]; ++j) {
            const int st = cs[k][j];
            for (int p = 1; p < cl[k][j]; ++p)
                if (iz[(size_t)k * ld + st + p] != (iz[(size_t)k * ld + st] + p) % N2) contig = false;
            const int x = cxy[k][j] / N1, y = cxy[k][j] % N1;
            int* t = &xt[((size_t)k * N0 + x) * 3];
            if (t[1] == 0) {
                t[0] = j;
                t[2] = y;
            } else if (t[0] + t[1] != j || (t[2] + t[1]) % N1 != y) {
                xruns = false;
            }
            t[1] += 1;
        }
    S.contig = contig;
    {
        const int m0 = (N0 - 1) / 4, m1 = (N1 - 1) / 4, m2 = (N2 - 1) / 4;
        bool prun = true;
        for (int k = 0; k < nk && prun; ++k) {
            for (int j = 0; j < ncol[k]; ++j) {
                const int x = cxy[k][j] / N1, y = cxy[k][j] % N1;
                if (!((x <= m0 || x >= N0 - m0) && (y <= m1 || y >= N1 - m1))) {
                    prun = false;
                    break;
                }
            }
            for (int i = 0; i < S.npw[k] && prun; ++i) {
                const int z = iz[(size_t)k * ld + i];
                if (!(z <= m2 || z >= N2 - m2)) prun = false;
            }
        }
        S.lines_prunable = prun;
    }
    if (S.d_xtab && S.xtab_n0 != N0) {
        dfree(c, S.d_xtab);
        S.d_xtab = nullptr;
    }
    if (xruns) {
        if (!S.d_xtab) CK(dalloc(c, &S.d_xtab, xt.size()));
        CK(h2d(S.d_xtab, xt.data(), xt.size(), c->st));
        S.xtab_n0 = N0;
    } else if (S.d_xtab) {
        dfree(c, S.d_xtab);
        S.d_xtab = nullptr;
        S.xtab_n0 = 0;
    }
    S.cols_distinct = true;
    for (int k = 0; k < nk && S.cols_distinct; ++k) {  // the fused transforms need one buffer slot per grid column
        std::vector<int> xs(cxy[k]);
        std::sort(xs.begin(), xs.end());
        if (std::adjacent_find(xs.begin(), xs.end()) != xs.end()) S.cols_distinct = false;
    }
    if (!S.cols_distinct) c->fused = false;
    CK(h2d(S.d_npw, S.npw.data(), nk, c->st));
    CK(h2d(S.d_idx, idx.data(), idx.size(), c->st));
    CK(h2d(S.d_g2, g2.data(), g2.size(), c->st));
    std::vector<double> prec(g2.size(), 0.0);
    for (int k = 0; k < nk; ++k)
        for (int i = 0; i < S.npw[k]; ++i) prec[(size_t)k * ld + i] = 1.0 / (1.0 + 0.5 * g2[(size_t)k * ld + i]);
    CK(h2d(S.d_prec, prec.data(), prec.size(), c->st));
    std::vector<float> prec32(prec.begin(), prec.end()), kin32(g2.size(), 0.0f);
    for (size_t i = 0; i < g2.size(); ++i) kin32[i] = (float)(0.5 * g2[i]);
    CK(h2d(S.d_prec32, prec32.data(), prec32.size(), c->st));
    CK(h2d(S.d_kin32, kin32.data(), kin32.size(), c->st));
    CK(h2d(S.d_iz, iz.data(), iz.size(), c->st));
    CK(h2d(S.d_ncol, ncol.data(), nk, c->st));
    CK(h2d(S.d_col_start, hs.data(), hs.size(), c->st));
    CK(h2d(S.d_col_len, hl.data(), hl.size(), c->st));
    CK(h2d(S.d_col_xy, hxy.data(), hxy.size(), c->st));
    CK(cudaStreamSynchronize(c->st));
    return HP_OK;
}

// upload a band list (host vectors row/k/spin/shift filled by the caller); builds segments
hp_status upload_list(hp_ctx* c, BandList& L) {
    L.nb = (int)L.row.size();
    L.seg_start.clear();
    L.seg_k.clear();
    L.seg_s.clear();
    for (int i = 0; i < L.nb; ++i) {
        if (i == 0 || L.k[i] != L.k[i - 1] || L.spin[i] != L.spin[i - 1]) {
            L.seg_start.push_back(i);
            L.seg_k.push_back(L.k[i]);
            L.seg_s.push_back(L.spin[i]);
        }
    }
    L.seg_start.push_back(L.nb);
    L.nseg = (int)L.seg_k.size();
    if (L.nb + 1 > L.cap) {
        for (void* p : {(void*)L.d_row, (void*)L.d_k, (void*)L.d_spin, (void*)L.d_shift, (void*)L.d_seg_start,
                        (void*)L.d_seg_k, (void*)L.d_seg_s})
            dfree(c, p);
        const int cap = L.nb + 1;
        CK(dalloc(c, &L.d_row, cap));
        CK(dalloc(c, &L.d_k, cap));
        CK(dalloc(c, &L.d_spin, cap));
        CK(dalloc(c, &L.d_shift, cap));
        CK(dalloc(c, &L.d_seg_start, cap + 1));
        CK(dalloc(c, &L.d_seg_k, cap));
        CK(dalloc(c, &L.d_seg_s, cap));
        L.cap = cap;
    }
    if (L.nb == 0) return HP_OK;
    CK(h2d(L.d_row, L.row.data(), L.nb, c->st));
    CK(h2d(L.d_k, L.k.data(), L.nb, c->st));
    CK(h2d(L.d_spin, L.spin.data(), L.nb, c->st));
    CK(h2d(L.d_shift, L.shift.data(), L.nb, c->st));
    CK(h2d(L.d_seg_start, L.seg_start.data(), L.nseg + 1, c->st));
    CK(h2d(L.d_seg_k, L.seg_k.data(), L.nseg, c->st));
    CK(h2d(L.d_seg_s, L.seg_s.data(), L.nseg, c->st));
    return HP_OK;
}

void list_clear(BandList& L) {
    L.row.clear();
    L.k.clear();
    L.spin.clear();
    L.shift.clear();
}

void list_add(BandList& L, int row, int k, int spin, double shift) {
    L.row.push_back(row);
    L.k.push_back(k);
    L.spin.push_back(spin);
    L.shift.push_back(shift);
}

hp_status ensure_grid(hp_ctx* c, int want) {
    if (want <= c->grid_cap) return HP_OK;
    dfree(c, c->d_grid);
    c->d_grid = nullptr;
    CK(dalloc(c, &c->d_grid, (size_t)want * c->nr));
    c->grid_cap = want;
    return HP_OK;
}

int band_batch(const hp_ctx* c, int nb) {
    if (c->opt.band_batch > 0) return std::min(nb, std::min(c->opt.band_batch, 32768));
    const size_t budget = (size_t)768 << 20;  // bytes of grid buffers
    int b = (int)std::min<size_t>(32768, std::max<size_t>(1, budget / (sizeof(double2) * (size_t)c->nr)));
    return std::max(1, std::min(nb, b));
}

hp_status ensure_scratch(hp_ctx* c, size_t elems) {
    if (elems <= c->scratch_elems) return HP_OK;
    dfree(c, c->d_scratch);
    c->d_scratch = nullptr;
    CK(dalloc(c, &c->d_scratch, elems));
    c->scratch_elems = elems;
    return HP_OK;
}

// Y = (T + V_loc + V_Hxc,s - shift) X on the list items (grid part + kinetic, zero padding)
hp_status apply_local(hp_ctx* c, const SphereSet& S, const BandList& L, const double2* X, double2* Y,
                      const double* veff, bool fp32) {
    if (L.nb == 0) return HP_OK;
    // chunks of a size fixed by the sizes alone (not by the buffer's history), so that a result does
    // not depend on what ran before it
    const int chunk = band_batch(c, L.nb);
    hp_status s = ensure_grid(c, chunk);
    if (s != HP_OK) return s;
    if (fp32) {  // FP32 grids: twice as many per batch in the same buffer
        float2* g32 = (float2*)c->d_grid;
        const int cap = 2 * chunk;
        for (int c0 = 0; c0 < L.nb; c0 += cap) {
            const int nc = std::min(cap, L.nb - c0);
            CK(k_scatter32(S, L, c0, nc, X, g32, c->nr, c->st));
            CK(fft3d(c->fft, g32, nc, +1, c->st));
            CK(k_mul_rpot32(g32, nc, c->nr, c->d_veff32, L, c0, c->st));
            CK(fft3d(c->fft, g32, nc, -1, c->st));
            CK(k_gather_h32(S, L, c0, nc, g32, c->nr, X, Y, c->ld, c->st));
        }
        return HP_OK;
    }
    for (int c0 = 0; c0 < L.nb; c0 += chunk) {
        const int nc = std::min(chunk, L.nb - c0);
        CK(k_scatter(S, L, c0, nc, X, c->ld, c->d_grid, c->nr, c->st));
        CK(fft3d(c->fft, c->d_grid, nc, +1, c->st));
        CK(k_mul_rpot(c->d_grid, nc, c->nr, veff, L, c0, c->st));
        CK(fft3d(c->fft, c->d_grid, nc, -1, c->st));
        CK(k_gather_h(S, L, c0, nc, c->d_grid, c->nr, X, Y, c->ld, c->st));
    }
    return HP_OK;
}

hp_status ensure_colbuf(hp_ctx* c, size_t bytes) {
    if (bytes <= c->col_cap) return HP_OK;
    dfree(c, c->d_colA);
    dfree(c, c->d_colB);
    c->d_colA = c->d_colB = nullptr;
    unsigned char *a = nullptr, *b = nullptr;
    CK(dalloc(c, &a, bytes));
    CK(dalloc(c, &b, bytes));
    c->d_colA = a;
    c->d_colB = b;
    c->col_cap = bytes;
    return HP_OK;
}

// bands per batch of the fused transforms: the two column buffers (2 GB each at most), or the
// caller's band_batch option; not bound by the 3D-FFT grid budget, so that one launch covers as many
// bands as the buffers hold
int fused_batch(const hp_ctx* c, const SphereSet& S, int nb) {
    const size_t per = sizeof(double2) * (size_t)c->N[2] * std::max(1, S.ncmax);
    int b = (int)std::min<size_t>(32768, std::max<size_t>(1, ((size_t)2 << 30) / per));
    if (c->opt.band_batch > 0) b = std::min(b, c->opt.band_batch);
    return std::max(1, std::min(nb, b));
}

FusedArgs fused_args(hp_ctx* c, const SphereSet& S, const BandList& L) {
    FusedArgs a;
    a.S = &S;
    a.L = &L;
    a.fft = &c->fft;
    a.N0 = c->N[0];
    a.N1 = c->N[1];
    a.N2 = c->N[2];
    a.colA = c->d_colA;
    a.colB = c->d_colB;
    a.vt = c->d_vt;
    a.vtx = c->d_vtx;
    a.inv_n = 1.0 / c->nr;
    a.reg = c->fused_reg;
    a.st = c->st;
    return a;
}

// Y = (T + V - shift) X through the fused column/plane transforms
hp_status apply_local_fused(hp_ctx* c, const SphereSet& S, const BandList& L, const void* X, void* Y, bool fp32) {
    if (L.nb == 0) return HP_OK;
    const int chunk = fused_batch(c, S, L.nb);
    hp_status s = ensure_colbuf(c, sizeof(double2) * (size_t)chunk * c->N[2] * S.ncmax);
    if (s != HP_OK) return s;
    for (int c0 = 0; c0 < L.nb; c0 += chunk) {
        FusedArgs a = fused_args(c, S, L);
        a.c0 = c0;
        a.nc = std::min(chunk, L.nb - c0);
        a.X = X;
        a.Y = Y;
        a.vec32 = c->vec32;
        a.mode = 0;
        CK(fused_col(fp32, true, a));
        CK(fused_plane(fp32, 0, a));
        CK(fused_col(fp32, false, a));
    }
    return HP_OK;
}

hp_status project(hp_ctx* c, const SphereSet& S, const BandList& L, const ProjMat& A, const double2* X, double2* P,
                  bool fp32) {
    hp_status s = ensure_scratch(c, (size_t)16 * std::max(1, L.nb) * kPStride);
    if (s != HP_OK) return s;
    CK(k_proj(L, S, A, X, c->ld, P, c->d_scratch, c->scratch_elems, c->st, fp32));
    return HP_OK;
}

hp_status project(hp_ctx* c, const SphereSet& S, const BandList& L, const ProjMat& A, const float2* X, double2* P,
                  bool fp32) {
    hp_status s = ensure_scratch(c, (size_t)16 * std::max(1, L.nb) * kPStride);
    if (s != HP_OK) return s;
    CK(k_proj(L, S, A, X, c->ld, P, c->d_scratch, c->scratch_elems, c->st, fp32));
    return HP_OK;
}

ProjMat beta_family(const hp_ctx* c, const int* kmap) {
    return ProjMat{c->d_beta_k, 0, (long long)c->nproj * c->ld, c->nproj, 0, kmap};
}

// Y += V_NL X  (beta D beta^H, beta at the list's spheres)
hp_status apply_nonlocal(hp_ctx* c, const SphereSet& S, const BandList& L, const double2* X, double2* Y, double2* P,
                         const int* kmap, bool fp32) {
    if (c->nproj == 0) return HP_OK;
    ProjMat B = beta_family(c, kmap);
    hp_status s = project(c, S, L, B, X, P, fp32);
    if (s != HP_OK) return s;
    CK(k_expand(L, S, B, P, c->d_projD, 1.0, Y, c->ld, c->st, fp32));
    return HP_OK;
}

}  // namespace hp

namespace {
hp_status resp_alloc(hp_ctx* c);
}  // namespace

// ================================================================================================
// C ABI
// ================================================================================================
extern "C" void hp_default_options(hp_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = HP_PRECISION_FP64;
    o->cg_tol = 1e-11;
    o->cg_maxiter = 400;
    o->scf_tol = 1e-10;
    o->cg_adapt = 0.001;
    o->conv_thr_chi = 1e-10;
    o->niter_max = 100;
    o->nmix = 4;
    o->alpha_mix = 0.3;
    o->gs_tol = 1e-11;
    o->gs_maxiter = 200;
    o->band_batch = 0;
    o->cuda_stream = nullptr;
    o->mixed_floor = 3e-7;
    o->wait_timeout_s = 2.0;
    o->dev_alloc = nullptr;
    o->dev_free = nullptr;
    o->alloc_user = nullptr;
    o->hub_ortho = 0;
}

extern "C" const char* hp_last_error(const hp_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" void hp_destroy(hp_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);  // nothing of this context may still run on its buffers
    else cudaDeviceSynchronize();
    for (void* p : c->owned) dev_free_raw(c, p);
    c->owned.clear();
    fft_plan_destroy(c->fft);
    delete c;
}

static hp_status setup_impl(hp_ctx* c, const double cell[9], int nspecies, const hp_species* sp, int natoms,
                            const int* species_of, const double* frac_pos, double ecut, const int kmesh[3],
                            const int qmesh[3]) {
    if (!cell || nspecies < 1 || !sp || natoms < 1 || !species_of || !frac_pos || !(ecut > 0) || !kmesh || !qmesh)
        return fail(c, HP_EINVAL, "hp_setup: missing or non-positive argument");
    for (int i = 0; i < 3; ++i) {
        if (kmesh[i] < 1 || qmesh[i] < 1) return fail(c, HP_EINVAL, "hp_setup: mesh sizes must be >= 1");
    }
    if (c->opt.hub_ortho != 0 && c->opt.hub_ortho != 1)
        return fail(c, HP_EINVAL, "hp_setup: hub_ortho must be 0 (atomic) or 1 (ortho-atomic)");
    if (c->opt.nmix < 0 || c->opt.nmix > 8 || !(c->opt.cg_tol > 0) || c->opt.niter_max < 1 || c->opt.cg_maxiter < 1 ||
        !(c->opt.mixed_floor >= 0) || !(c->opt.wait_timeout_s > 0))
        return fail(c, HP_EINVAL, "hp_setup: options out of range (0 <= nmix <= 8, tolerances > 0, wait_timeout_s > 0)");
    if ((c->opt.dev_alloc == nullptr) != (c->opt.dev_free == nullptr))
        return fail(c, HP_EINVAL, "hp_setup: dev_alloc and dev_free must be given together");
    for (int s = 0; s < nspecies; ++s) {
        if (sp[s].l_proj < 0 || sp[s].l_proj > 2 || sp[s].l_hub > 2 || !(sp[s].width > 0) || !(sp[s].proj_width > 0) ||
            (sp[s].l_hub >= 0 && !(sp[s].hub_width > 0)))
            return fail(c, HP_EINVAL, "hp_setup: species parameters out of range (0 <= l <= 2, widths > 0)");
    }
    memcpy(c->cell, cell, sizeof(double) * 9);
    // reciprocal vectors: b_i = 2 pi (a_j x a_k) / Omega
    double cr[3][3];
    cross(cell + 3, cell + 6, cr[0]);
    cross(cell + 6, cell + 0, cr[1]);
    cross(cell + 0, cell + 3, cr[2]);
    const double vol = cell[0] * cr[0][0] + cell[1] * cr[0][1] + cell[2] * cr[0][2];
    if (std::fabs(vol) < 1e-12) return fail(c, HP_EINVAL, "hp_setup: degenerate cell");
    c->omega = std::fabs(vol);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c->bvec[3 * i + j] = 2.0 * M_PI * cr[i][j] / vol;
    c->species.assign(sp, sp + nspecies);
    c->atom_species.assign(species_of, species_of + natoms);
    c->frac.assign(frac_pos, frac_pos + 3 * natoms);
    c->tau.resize(3 * natoms);
    for (int a = 0; a < natoms; ++a) {
        if (species_of[a] < 0 || species_of[a] >= nspecies) return fail(c, HP_EINVAL, "hp_setup: bad species index");
        for (int j = 0; j < 3; ++j)
            c->tau[3 * a + j] = frac_pos[3 * a] * cell[j] + frac_pos[3 * a + 1] * cell[3 + j] + frac_pos[3 * a + 2] * cell[6 + j];
    }
    c->ecut = ecut;
    for (int i = 0; i < 3; ++i) {
        c->kmesh[i] = kmesh[i];
        c->qmesh[i] = qmesh[i];
    }
    c->nk = kmesh[0] * kmesh[1] * kmesh[2];
    c->nq = qmesh[0] * qmesh[1] * qmesh[2];
    // FFT grid
    for (int i = 0; i < 3; ++i) {
        if (c->opt.fft_grid[i] > 0) {
            c->N[i] = c->opt.fft_grid[i];
        } else {
            const double an = std::sqrt(cell[3 * i] * cell[3 * i] + cell[3 * i + 1] * cell[3 * i + 1] + cell[3 * i + 2] * cell[3 * i + 2]);
            const int mmax = (int)std::floor(2.0 * std::sqrt(ecut) * an / (2.0 * M_PI));
            c->N[i] = good_fft_size(2 * mmax + 1);
        }
        Radices r;
        if (!fft_factor(c->N[i], r)) return fail(c, HP_EINVAL, "hp_setup: FFT grid sizes must factor into 2, 3 and 5");
    }
    c->nr = c->N[0] * c->N[1] * c->N[2];
    // spheres at the k mesh
    c->ks.resize(c->nk);
    c->ld = 0;
    for (int i1 = 0, ik = 0; i1 < kmesh[0]; ++i1)
        for (int i2 = 0; i2 < kmesh[1]; ++i2)
            for (int i3 = 0; i3 < kmesh[2]; ++i3, ++ik) {
                const double kf[3] = {(double)i1 / kmesh[0], (double)i2 / kmesh[1], (double)i3 / kmesh[2]};
                build_sphere(c, kf, c->ks[ik]);
                c->ld = std::max(c->ld, c->ks[ik].npw);
            }
    // spheres at k+q where k+q is off the k mesh (Gamma-centred meshes: (k+q)_d kmesh_d is an
    // integer for every d exactly when k+q is on the mesh)
    c->kq_ks.assign((size_t)c->nq * c->nk, KSphere());
    c->qfam.assign(c->nq, QFam());
    for (int iq = 0; iq < c->nq; ++iq)
        for (int ik = 0; ik < c->nk; ++ik) {
            const int qi[3] = {iq / (qmesh[1] * qmesh[2]), (iq / qmesh[2]) % qmesh[1], iq % qmesh[2]};
            const int ki[3] = {ik / (kmesh[1] * kmesh[2]), (ik / kmesh[2]) % kmesh[1], ik % kmesh[2]};
            bool on = true;
            for (int d = 0; d < 3; ++d) on = on && ((ki[d] * qmesh[d] + qi[d] * kmesh[d]) % qmesh[d] == 0);
            if (on) continue;
            double kf[3];
            for (int d = 0; d < 3; ++d) kf[d] = (double)ki[d] / kmesh[d] + (double)qi[d] / qmesh[d];
            KSphere& ks = c->kq_ks[(size_t)iq * c->nk + ik];
            build_sphere(c, kf, ks);
            c->ld = std::max(c->ld, ks.npw);
        }
    // projector and Hubbard rows, with the K-independent prefactor
    //   (4 pi / sqrt(Omega)) N_R sqrt(pi/2) s^(2l+3),  N_R = sqrt(2 / (Gamma(l + 3/2) s^(2l+3)))
    auto pref = [&](int l, double s) {
        const double s2l3 = std::pow(s, 2 * l + 3);
        const double NR = std::sqrt(2.0 / (std::tgamma(l + 1.5) * s2l3));
        return 4.0 * M_PI / std::sqrt(c->omega) * NR * std::sqrt(M_PI / 2.0) * s2l3;
    };
    for (int a = 0; a < natoms; ++a) {
        const hp_species& s = sp[species_of[a]];
        for (int m = 0; m < 2 * s.l_proj + 1; ++m) {
            c->proj_atom.push_back(a);
            c->proj_l.push_back(s.l_proj);
            c->proj_m.push_back(m);
            c->proj_D.push_back(s.D);
            c->proj_w.push_back(s.proj_width);
            c->proj_pref.push_back(pref(s.l_proj, s.proj_width));
        }
        if (s.l_hub >= 0) {
            c->hub_atoms.push_back(a);
            c->hub_off.push_back((int)c->hub_row_atom.size());
            c->hub_mdim.push_back(2 * s.l_hub + 1);
            for (int m = 0; m < 2 * s.l_hub + 1; ++m) {
                c->hub_row_atom.push_back(a);
                c->hub_row_l.push_back(s.l_hub);
                c->hub_row_m.push_back(m);
                c->hub_row_w.push_back(s.hub_width);
                c->hub_row_pref.push_back(pref(s.l_hub, s.hub_width));
            }
        }
    }
    c->nproj = (int)c->proj_atom.size();
    c->nhub = (int)c->hub_row_atom.size();
    if (c->nproj > kPStride || c->nhub > kPStride) return fail(c, HP_EINVAL, "hp_setup: more than 128 projector rows");
    if (c->hub_atoms.empty()) return fail(c, HP_EINVAL, "hp_setup: no Hubbard species");
    // device data
    tc_set_timeout(c->opt.wait_timeout_s);
    c->fused_grid = fused_supported(c->N) && !getenv("HP_NO_FUSED");
    c->fused = c->fused_grid;
    c->fused_reg = !getenv("HP_FUSED_SMEM");  // HP_FUSED_SMEM: shared-memory line FFTs instead
    // rows of one combined projection (at most the buffer's 128; HP_PROJ_ROWS lowers it)
    c->proj_rows_max = kPStride;
    if (const char* r = getenv("HP_PROJ_ROWS")) c->proj_rows_max = std::max(1, std::min(kPStride, atoi(r)));
    CK(fft_plan_create(c, c->fft, c->N));
    CK(dalloc(c, &c->d_bvec, 9));
    CK(h2d(c->d_bvec, c->bvec, 9, c->st));
    CK(dalloc(c, &c->d_tau, 3 * natoms));
    CK(h2d(c->d_tau, c->tau.data(), 3 * natoms, c->st));
    std::vector<const KSphere*> sph;
    for (auto& s : c->ks) sph.push_back(&s);
    hp_status st = upload_sphereset(c, sph, nullptr, c->kset);
    if (st != HP_OK) return st;
    // V_loc(r): closed-form V(G) on the grid, then to real space
    {
        std::vector<double> amp(natoms), wid(natoms);
        for (int a = 0; a < natoms; ++a) {
            amp[a] = sp[species_of[a]].amp;
            wid[a] = sp[species_of[a]].width;
        }
        double *d_amp, *d_wid;
        double2* d_vg;
        CK(dalloc(c, &d_amp, natoms));
        CK(dalloc(c, &d_wid, natoms));
        CK(dalloc(c, &d_vg, c->nr));
        CK(h2d(d_amp, amp.data(), natoms, c->st));
        CK(h2d(d_wid, wid.data(), natoms, c->st));
        CK(k_vloc_g(d_vg, c->N, c->d_bvec, 4.0 * ecut, natoms, c->d_tau, d_amp, d_wid, c->omega, c->st));
        CK(fft3d(c->fft, d_vg, 1, +1, c->st));
        CK(dalloc(c, &c->d_vloc, c->nr));
        CK(k_real_part(d_vg, c->d_vloc, c->nr, 1.0, c->st));
        CK(cudaStreamSynchronize(c->st));
        dfree(c, d_amp);
        dfree(c, d_wid);
        dfree(c, d_vg);
    }
    // form factors beta_k, phi_k
    {
        const int nrow_all = c->nproj + c->nhub;
        std::vector<int> ri(3 * nrow_all);
        std::vector<double> rd(2 * nrow_all);
        for (int r = 0; r < c->nproj; ++r) {
            ri[r] = c->proj_atom[r];
            ri[nrow_all + r] = c->proj_l[r];
            ri[2 * nrow_all + r] = c->proj_m[r];
            rd[r] = c->proj_w[r];
            rd[nrow_all + r] = c->proj_pref[r];
        }
        for (int r = 0; r < c->nhub; ++r) {
            const int o = c->nproj + r;
            ri[o] = c->hub_row_atom[r];
            ri[nrow_all + o] = c->hub_row_l[r];
            ri[2 * nrow_all + o] = c->hub_row_m[r];
            rd[o] = c->hub_row_w[r];
            rd[nrow_all + o] = c->hub_row_pref[r];
        }
        CK(dalloc(c, &c->d_proj_int, ri.size()));
        CK(dalloc(c, &c->d_proj_dbl, rd.size()));
        CK(h2d(c->d_proj_int, ri.data(), ri.size(), c->st));
        CK(h2d(c->d_proj_dbl, rd.data(), rd.size(), c->st));
        std::vector<int> mil((size_t)c->nk * c->ld * 3, 0);
        std::vector<double> kc(3 * c->nk);
        for (int k = 0; k < c->nk; ++k) {
            for (int i = 0; i < c->ks[k].npw * 3; ++i) mil[(size_t)k * c->ld * 3 + i] = c->ks[k].miller[i];
            for (int j = 0; j < 3; ++j) kc[3 * k + j] = c->ks[k].kcart[j];
        }
        int* d_mil;
        double* d_kc;
        CK(dalloc(c, &d_mil, mil.size()));
        CK(dalloc(c, &d_kc, kc.size()));
        CK(h2d(d_mil, mil.data(), mil.size(), c->st));
        CK(h2d(d_kc, kc.data(), kc.size(), c->st));
        CK(dalloc(c, &c->d_beta_k, (size_t)c->nk * std::max(1, c->nproj) * c->ld));
        CK(dalloc(c, &c->d_phi_k, (size_t)c->nk * c->nhub * c->ld));
        CK(k_formfactor(d_kc, c->nk, d_mil, c->kset.d_npw, c->ld, c->d_bvec, c->nproj, c->d_proj_int,
                        c->d_proj_int + nrow_all, c->d_proj_int + 2 * nrow_all, c->d_proj_dbl,
                        c->d_proj_dbl + nrow_all, c->d_tau, c->d_beta_k, c->st));
        CK(k_formfactor(d_kc, c->nk, d_mil, c->kset.d_npw, c->ld, c->d_bvec, c->nhub, c->d_proj_int + c->nproj,
                        c->d_proj_int + nrow_all + c->nproj, c->d_proj_int + 2 * nrow_all + c->nproj,
                        c->d_proj_dbl + c->nproj, c->d_proj_dbl + nrow_all + c->nproj, c->d_tau, c->d_phi_k, c->st));
        CK(dalloc(c, &c->d_projD, std::max(1, c->nproj)));
        if (c->nproj) CK(h2d(c->d_projD, c->proj_D.data(), c->nproj, c->st));
        CK(cudaStreamSynchronize(c->st));
        dfree(c, d_mil);
        dfree(c, d_kc);
    }
    if (c->opt.hub_ortho) {  // Loewdin ortho-atomic Hubbard projectors at every k of the mesh
        st = ortho_hubbard_rows(c, c->kset, c->nk, c->d_phi_k);
        if (st != HP_OK) return st;
    }
    return HP_OK;
}

extern "C" hp_status hp_setup(const double cell[9], int nspecies, const hp_species* sp, int natoms,
                              const int* species_of, const double* frac_pos, double ecutwfc_ry, const int kmesh[3],
                              const int qmesh[3], const hp_options* opt, hp_ctx** out) {
    if (!out) return HP_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HP_ECUDA;
    hp_ctx* c = new hp_ctx();
    if (opt) c->opt = *opt;
    else hp_default_options(&c->opt);
    c->st = (cudaStream_t)c->opt.cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) c->device = 0;
    hp_status s = setup_impl(c, cell, nspecies, sp, natoms, species_of, frac_pos, ecutwfc_ry, kmesh, qmesh);
    if (s != HP_OK) {
        fprintf(stderr, "hp_setup: %s\n", c->err.c_str());
        hp_destroy(c);
        return s;
    }
    *out = c;
    return HP_OK;
}

extern "C" hp_status hp_set_precision(hp_ctx* c, int precision) {
    if (!c) return HP_EINVAL;
    if (precision != HP_PRECISION_FP64 && precision != HP_PRECISION_MIXED)
        return fail(c, HP_EINVAL, "hp_set_precision: unknown precision");
    if (precision != c->opt.precision) {
        c->opt.precision = precision;
        c->resp_ready = false;  // caches are precision-specific; the ground state is kept
        c->cols.clear();
    }
    return HP_OK;
}

extern "C" hp_status hp_query_sizes(const hp_ctx* c, hp_sizes* o) {
    if (!c || !o) return HP_EINVAL;
    o->nk = c->nk;
    o->nq = c->nq;
    o->nspin = c->nspin;
    o->nocc = c->nocc;
    o->nbnd = c->nbnd;
    for (int i = 0; i < 3; ++i) o->grid[i] = c->N[i];
    o->nr = c->nr;
    o->nat = (int)c->atom_species.size();
    o->nhub_atoms = (int)c->hub_atoms.size();
    o->nhub_orb = c->nhub;
    o->nproj = c->nproj;
    o->mmax = kMmax;
    o->npw_max = c->ld;
    o->ncell = c->nq;
    o->nchi = c->nq * (int)c->hub_atoms.size();
    return HP_OK;
}

extern "C" hp_status hp_sphere(const hp_ctx* c, int ik, int* npw, int* miller) {
    if (!c || !npw || ik < 0 || ik >= c->nk) return HP_EINVAL;
    *npw = c->ks[ik].npw;
    if (miller) memcpy(miller, c->ks[ik].miller.data(), sizeof(int) * 3 * c->ks[ik].npw);
    return HP_OK;
}

extern "C" hp_status hp_hubbard_atoms(const hp_ctx* c, int* atom_index, int* mdim) {
    if (!c) return HP_EINVAL;
    for (size_t i = 0; i < c->hub_atoms.size(); ++i) {
        if (atom_index) atom_index[i] = c->hub_atoms[i];
        if (mdim) mdim[i] = c->hub_mdim[i];
    }
    return HP_OK;
}

// ------------------------------------------------------------------------------------------------
// ground state import / export
// ------------------------------------------------------------------------------------------------
static hp_status gs_alloc(hp_ctx* c, int nspin, int nbnd) {
    for (void* p : {(void*)c->d_vhxc, (void*)c->d_rho, (void*)c->d_veff, (void*)c->d_psi}) dfree(c, p);
    c->d_vhxc = c->d_rho = c->d_veff = nullptr;
    c->d_psi = nullptr;
    CK(dalloc(c, &c->d_vhxc, (size_t)nspin * c->nr));
    CK(dalloc(c, &c->d_rho, (size_t)nspin * c->nr));
    CK(dalloc(c, &c->d_veff, (size_t)nspin * c->nr));
    CK(dalloc(c, &c->d_psi, (size_t)nspin * c->nk * nbnd * c->ld));
    CK(cudaMemsetAsync(c->d_psi, 0, sizeof(double2) * (size_t)nspin * c->nk * nbnd * c->ld, c->st));
    return HP_OK;
}

void hp::invalidate_response(hp_ctx* c) {
    c->resp_ready = false;
    c->qc.iq = -1;
    c->cols.clear();
    c->hub_rep.clear();  // the classes follow the ground state's occupations
    c->hub_orient.clear();
    c->sym_ops.clear();
    for (QFam& F : c->qfam) F.built = false;  // the states at k+q follow the ground state
}

extern "C" hp_status hp_set_ground_state(hp_ctx* c, int nspin, double nelec, const double* vhxc, const double* rho,
                                         const double* eps, const double* psi) {
    if (!c) return HP_EINVAL;
    if ((nspin != 1 && nspin != 2) || !vhxc || !rho || !eps || !psi)
        return fail(c, HP_EINVAL, "hp_set_ground_state: nspin must be 1 or 2 and every array given");
    const int nocc = (int)std::lround(nelec / 2.0);
    if (nocc < 1 || std::fabs(nelec - 2.0 * nocc) > 1e-9)
        return fail(c, HP_EINVAL, "hp_set_ground_state: nelec must be an even positive number");
    for (int k = 0; k < c->nk; ++k)
        if (c->ks[k].npw < nocc) return fail(c, HP_EINVAL, "hp_set_ground_state: fewer plane waves than bands");
    invalidate_response(c);
    c->have_gs = false;
    hp_status s = gs_alloc(c, nspin, nocc);
    if (s != HP_OK) return s;
    c->nspin = nspin;
    c->nelec = nelec;
    c->nocc = c->nbnd = nocc;
    c->gap = INFINITY;
    c->eps.assign(eps, eps + (size_t)nspin * c->nk * nocc);
    CK(h2d(c->d_vhxc, vhxc, (size_t)nspin * c->nr, c->st));
    CK(h2d(c->d_rho, rho, (size_t)nspin * c->nr, c->st));
    for (int sp = 0; sp < nspin; ++sp) CK(k_add_real(c->d_vloc, c->d_vhxc + (size_t)sp * c->nr, c->d_veff + (size_t)sp * c->nr, c->nr, c->st));
    size_t off = 0;
    std::vector<double2> row(c->ld);
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < c->nk; ++k)
            for (int v = 0; v < nocc; ++v) {
                const int npw = c->ks[k].npw;
                std::fill(row.begin(), row.end(), cmk(0.0, 0.0));
                for (int i = 0; i < npw; ++i) row[i] = cmk(psi[2 * (off + i)], psi[2 * (off + i) + 1]);
                off += npw;
                CK(cudaMemcpy(c->d_psi + ((size_t)(sp * c->nk + k) * nocc + v) * c->ld, row.data(), sizeof(double2) * c->ld,
                              cudaMemcpyHostToDevice));
            }
    CK(cudaStreamSynchronize(c->st));
    if (c->hub_on) {  // DFT+U+V: the Hubbard potential from the occupation matrices of the imported states
        for (void* p : {(void*)c->d_hub_occ, (void*)c->d_hubW}) dfree(c, p);
        CK(dalloc(c, &c->d_hub_occ, hub_occ_len(c, nspin)));
        CK(dalloc(c, &c->d_hubW, (size_t)nspin * c->nk * c->nhub * c->nhub));
        BandList& L = c->L3;
        list_clear(L);
        for (int sp = 0; sp < nspin; ++sp)
            for (int k = 0; k < c->nk; ++k)
                for (int v = 0; v < nocc; ++v) list_add(L, (sp * c->nk + k) * nocc + v, k, sp, 0.0);
        if ((s = upload_list(c, L)) != HP_OK) return s;
        double2* P;
        CK(dalloc(c, &P, (size_t)L.nb * kPStride));
        ProjMat F{c->d_phi_k, 0, (long long)c->nhub * c->ld, c->nhub, 0, nullptr};
        if ((s = project(c, c->kset, L, F, c->d_psi, P)) != HP_OK) return s;
        if ((s = hub_occupations(c, P, nspin, c->nk, nocc, c->d_kfrac, c->d_hub_occ)) != HP_OK) return s;
        if ((s = hub_build_w(c, c->d_hub_occ, nspin, c->nk, c->d_kfrac, c->d_hubW)) != HP_OK) return s;
        CK(cudaStreamSynchronize(c->st));
        dfree(c, P);
    }
    c->have_gs = true;
    return HP_OK;
}

extern "C" hp_status hp_get_ground_state(const hp_ctx* cc, double* eps, double* rho, double* vhxc) {
    hp_ctx* c = const_cast<hp_ctx*>(cc);
    if (!c) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "no ground state");
    if (eps) {
        for (int s = 0; s < c->nspin; ++s)
            for (int k = 0; k < c->nk; ++k)
                for (int v = 0; v < c->nocc; ++v) eps[((size_t)s * c->nk + k) * c->nocc + v] = c->eps[((size_t)s * c->nk + k) * c->nbnd + v];
    }
    if (rho) CK(d2h(rho, c->d_rho, (size_t)c->nspin * c->nr, c->st));
    if (vhxc) CK(d2h(vhxc, c->d_vhxc, (size_t)c->nspin * c->nr, c->st));
    return HP_OK;
}

extern "C" hp_status hp_get_wavefunctions(const hp_ctx* cc, double* psi) {
    hp_ctx* c = const_cast<hp_ctx*>(cc);
    if (!c || !psi) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "no ground state");
    std::vector<double2> row(c->ld);
    size_t off = 0;
    for (int sp = 0; sp < c->nspin; ++sp)
        for (int k = 0; k < c->nk; ++k)
            for (int v = 0; v < c->nocc; ++v) {
                CK(cudaMemcpy(row.data(), c->d_psi + ((size_t)(sp * c->nk + k) * c->nbnd + v) * c->ld,
                              sizeof(double2) * c->ld, cudaMemcpyDeviceToHost));
                for (int i = 0; i < c->ks[k].npw; ++i) {
                    psi[2 * (off + i)] = row[i].x;
                    psi[2 * (off + i) + 1] = row[i].y;
                }
                off += c->ks[k].npw;
            }
    return HP_OK;
}

extern "C" hp_status hp_apply_h(hp_ctx* c, int ik, int spin, int nb, const double* psi, double* out) {
    if (!c) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "hp_apply_h: no ground state (potential) yet");
    if (ik < 0 || ik >= c->nk || spin < 0 || spin >= c->nspin || nb < 1 || !psi || !out)
        return fail(c, HP_EINVAL, "hp_apply_h: bad arguments");
    const int npw = c->ks[ik].npw, ld = c->ld;
    std::vector<double2> h((size_t)nb * ld, cmk(0.0, 0.0));
    for (int b = 0; b < nb; ++b)
        for (int i = 0; i < npw; ++i) h[(size_t)b * ld + i] = cmk(psi[2 * ((size_t)b * npw + i)], psi[2 * ((size_t)b * npw + i) + 1]);
    double2 *dX, *dY, *dP;
    CK(dalloc(c, &dX, (size_t)nb * ld));
    CK(dalloc(c, &dY, (size_t)nb * ld));
    CK(dalloc(c, &dP, (size_t)nb * kPStride));
    CK(h2d(dX, h.data(), h.size(), c->st));
    BandList& L = c->L1;
    list_clear(L);
    for (int b = 0; b < nb; ++b) list_add(L, b, ik, spin, 0.0);
    hp_status s = upload_list(c, L);
    if (s == HP_OK) s = apply_local(c, c->kset, L, dX, dY, c->d_veff);
    if (s == HP_OK) s = apply_nonlocal(c, c->kset, L, dX, dY, dP, nullptr);
    if (s == HP_OK && c->hub_on && c->d_hubW) s = hub_apply(c, c->kset, L, c->d_phi_k, nullptr, c->d_hubW, dX, dY, false, false, dP);
    if (s == HP_OK) {
        cudaError_t e = d2h(h.data(), dY, h.size(), c->st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "hp_apply_h copy-out");
    }
    dfree(c, dX);
    dfree(c, dY);
    dfree(c, dP);
    if (s != HP_OK) return s;
    for (int b = 0; b < nb; ++b)
        for (int i = 0; i < npw; ++i) {
            out[2 * ((size_t)b * npw + i)] = h[(size_t)b * ld + i].x;
            out[2 * ((size_t)b * npw + i) + 1] = h[(size_t)b * ld + i].y;
        }
    return HP_OK;
}

// ------------------------------------------------------------------------------------------------
// response
// ------------------------------------------------------------------------------------------------
namespace {

hp_status resp_alloc(hp_ctx* c) {
    const int rows = c->nspin * c->nk * c->nocc;
    if (rows == c->resp_rows && c->d_x) return HP_OK;
    for (void* p : {(void*)c->d_x, (void*)c->d_r, (void*)c->d_p, (void*)c->d_ap, (void*)c->d_b, (void*)c->d_vpu,
                    (void*)c->d_rz, (void*)c->d_rzold, (void*)c->d_rr, (void*)c->d_pap, (void*)c->d_Pbuf})
        dfree(c, p);
    const size_t n = (size_t)rows * c->ld;
    CK(dalloc(c, &c->d_x, n));
    CK(dalloc(c, &c->d_r, n));
    CK(dalloc(c, &c->d_p, n));
    CK(dalloc(c, &c->d_ap, n));
    CK(dalloc(c, &c->d_b, n));
    CK(dalloc(c, &c->d_vpu, n));
    CK(dalloc(c, &c->d_rz, rows));
    CK(dalloc(c, &c->d_rzold, rows));
    CK(dalloc(c, &c->d_rr, rows));
    CK(dalloc(c, &c->d_pap, rows));
    CK(dalloc(c, &c->d_Pbuf, (size_t)rows * kPStride));
    c->resp_rows = rows;
    return HP_OK;
}

// per ground state: real-space occupied u_k, <phi_k|u_k>, f_xc, alpha
hp_status prepare_resp(hp_ctx* c) {
    if (c->resp_ready) return HP_OK;
    const int nspin = c->nspin, nk = c->nk, nocc = c->nocc, nr = c->nr;
    const int rows = nspin * nk * nocc;
    hp_status s = resp_alloc(c);
    if (s != HP_OK) return s;
    const bool mixed = c->opt.precision == HP_PRECISION_MIXED;
    dfree(c, c->d_ur);
    dfree(c, c->d_ur32);
    dfree(c, c->d_veff32);
    dfree(c, c->d_dv32);
    c->d_ur = nullptr;
    c->d_ur32 = nullptr;
    dfree(c, c->d_aphi);
    dfree(c, c->d_fxc);
    for (float2** p : {&c->d_psi32, &c->d_beta32, &c->d_phi32}) {
        dfree(c, *p);
        *p = nullptr;
    }
    if (mixed) {
        CK(dalloc(c, &c->d_ur32, (size_t)rows * nr));
        CK(dalloc(c, &c->d_veff32, (size_t)nspin * nr));
        CK(dalloc(c, &c->d_dv32, (size_t)nspin * nr));
        CK(k_to_f32(c->d_veff, c->d_veff32, (long long)nspin * nr, c->st));
        const size_t npsi = (size_t)nspin * nk * c->nbnd * c->ld, nbeta = (size_t)nk * c->nproj * c->ld,
                     nphi = (size_t)nk * c->nhub * c->ld;
        CK(dalloc(c, &c->d_psi32, npsi));
        CK(k_to_c32(c->d_psi, c->d_psi32, (long long)npsi, c->st));
        if (nbeta) {
            CK(dalloc(c, &c->d_beta32, nbeta));
            CK(k_to_c32(c->d_beta_k, c->d_beta32, (long long)nbeta, c->st));
        }
        if (nphi) {
            CK(dalloc(c, &c->d_phi32, nphi));
            CK(k_to_c32(c->d_phi_k, c->d_phi32, (long long)nphi, c->st));
        }
    } else {
        CK(dalloc(c, &c->d_ur, (size_t)rows * nr));
    }
    CK(dalloc(c, &c->d_aphi, (size_t)rows * kPStride));
    CK(dalloc(c, &c->d_fxc, (size_t)(nspin == 1 ? 1 : 3) * nr));
    // list of occupied ground-state rows (psi rows), items ordered (s, k, v)
    BandList& L = c->L2;
    list_clear(L);
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nk; ++k)
            for (int v = 0; v < nocc; ++v) list_add(L, (sp * nk + k) * c->nbnd + v, k, sp, 0.0);
    s = upload_list(c, L);
    if (s != HP_OK) return s;
    // u_k(r): scatter straight into the cache and transform in place
    if (c->fused) {
        // plane-major V_eff (FP64 or FP32) and the real-space occupied bands through the fused path
        dfree(c, c->d_vt);
        dfree(c, c->d_vtx);
        dfree(c, c->d_dvt);
        dfree(c, c->d_drho_pm);
        c->d_vt = c->d_vtx = c->d_dvt = nullptr;
        double* tmp;
        CK(dalloc(c, &tmp, (size_t)nspin * nr));
        CK(k_to_planes_real(c->d_veff, tmp, c->N, nspin, c->st));
        if (mixed) {
            float* v32;
            float2* dv32;
            CK(dalloc(c, &v32, (size_t)nspin * nr));
            CK(k_to_f32(tmp, v32, (long long)nspin * nr, c->st));
            CK(dalloc(c, &dv32, (size_t)nspin * nr));
            c->d_vt = v32;
            c->d_dvt = dv32;
            CK(cudaStreamSynchronize(c->st));
            dfree(c, tmp);
        } else {
            double2* dv64;
            CK(dalloc(c, &dv64, (size_t)nspin * nr));
            c->d_vt = tmp;
            c->d_dvt = dv64;
        }
        // x-major copy: the register plane kernels read it with consecutive threads on consecutive y
        void* vx;
        if (mixed) {
            float* v;
            CK(dalloc(c, &v, (size_t)nspin * nr));
            vx = v;
        } else {
            double* v;
            CK(dalloc(c, &v, (size_t)nspin * nr));
            vx = v;
        }
        c->d_vtx = vx;
        CK(k_planes_xmajor(c->d_vt, c->d_vtx, c->N[0], c->N[1], (long long)nspin * c->N[2], mixed, c->st));
        CK(dalloc(c, &c->d_drho_pm, (size_t)nspin * nr));
        const int chunk = fused_batch(c, c->kset, rows);
        s = ensure_colbuf(c, sizeof(double2) * (size_t)chunk * c->N[2] * c->kset.ncmax);
        if (s != HP_OK) return s;
        for (int c0 = 0; c0 < rows; c0 += chunk) {
            FusedArgs a = fused_args(c, c->kset, L);
            a.c0 = c0;
            a.nc = std::min(chunk, rows - c0);
            a.X = c->d_psi;
            a.out = mixed ? (void*)(c->d_ur32 + (size_t)c0 * nr) : (void*)(c->d_ur + (size_t)c0 * nr);
            CK(fused_col(mixed, true, a));
            CK(fused_plane(mixed, 1, a));
        }
    }
    c->ur_planes = c->fused;
    const int chunk = std::max(1, band_batch(c, rows));
    for (int c0 = 0; c0 < rows && !c->fused; c0 += chunk) {
        const int nc = std::min(chunk, rows - c0);
        if (mixed) {
            CK(k_scatter32(c->kset, L, c0, nc, c->d_psi, c->d_ur32 + (size_t)c0 * nr, nr, c->st));
            CK(fft3d(c->fft, c->d_ur32 + (size_t)c0 * nr, nc, +1, c->st));
        } else {
            CK(k_scatter(c->kset, L, c0, nc, c->d_psi, c->ld, c->d_ur + (size_t)c0 * nr, nr, c->st));
            CK(fft3d(c->fft, c->d_ur + (size_t)c0 * nr, nc, +1, c->st));
        }
    }
    // <phi_m,k|u_vk>
    ProjMat phi{c->d_phi_k, 0, (long long)c->nhub * c->ld, c->nhub, 0, nullptr};
    s = project(c, c->kset, L, phi, c->d_psi, c->d_aphi);
    if (s != HP_OK) return s;
    // f_xc
    double* d_vtmp;
    CK(dalloc(c, &d_vtmp, (size_t)nspin * nr));
    CK(k_xc(c->d_rho, nspin, nr, d_vtmp, c->d_fxc, c->st));
    CK(cudaStreamSynchronize(c->st));
    dfree(c, d_vtmp);
    double emax = -INFINITY, emin = INFINITY;
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nk; ++k)
            for (int v = 0; v < nocc; ++v) {
                const double e = c->eps[((size_t)sp * nk + k) * c->nbnd + v];
                emax = std::max(emax, e);
                emin = std::min(emin, e);
            }
    c->alpha_pv = 2.0 * (emax - emin);
    if (c->alpha_pv <= 0) c->alpha_pv = 1.0;
    // small work buffers
    if (!c->d_small) CK(dalloc(c, &c->d_small, 512));
    if (!c->d_partial) CK(dalloc(c, &c->d_partial, 1024));
    dfree(c, c->d_dv);
    dfree(c, c->d_dvout);
    dfree(c, c->d_drho);
    dfree(c, c->d_dvh);
    CK(dalloc(c, &c->d_dv, (size_t)nspin * nr));
    CK(dalloc(c, &c->d_dvout, (size_t)nspin * nr));
    CK(dalloc(c, &c->d_drho, (size_t)nspin * nr));
    CK(dalloc(c, &c->d_dvh, (size_t)nr));
    dfree(c, c->d_M);
    dfree(c, c->d_dn);
    CK(dalloc(c, &c->d_M, (size_t)nspin * c->nhub * c->nhub));
    CK(dalloc(c, &c->d_dn, (size_t)c->hub_atoms.size() * nspin * kMmax * kMmax + c->hub_atoms.size()));
    for (auto p : c->d_hist_dx) dfree(c, p);
    for (auto p : c->d_hist_df) dfree(c, p);
    c->d_hist_dx.assign(c->opt.nmix + 2, nullptr);
    c->d_hist_df.assign(c->opt.nmix + 2, nullptr);
    for (int i = 0; i < c->opt.nmix + 2; ++i) {
        CK(dalloc(c, &c->d_hist_dx[i], (size_t)nspin * nr));
        CK(dalloc(c, &c->d_hist_df[i], (size_t)nspin * nr));
    }
    if (!c->d_hist_ptrs) CK(dalloc(c, &c->d_hist_ptrs, 32 + 2 * kMaxDots));
    if (!c->d_partials) CK(dalloc(c, &c->d_partials, (size_t)kMaxDots * 256));
    c->resp_ready = true;
    return HP_OK;
}


}  // namespace

void hp::free_sphereset(hp_ctx* c, SphereSet& S) {
    for (void* p : {(void*)S.d_npw, (void*)S.d_idx, (void*)S.d_g2, (void*)S.d_prec, (void*)S.d_prec32, (void*)S.d_kin32,
                    (void*)S.d_iz, (void*)S.d_ncol, (void*)S.d_col_start, (void*)S.d_col_len, (void*)S.d_col_xy,
                    (void*)S.d_xtab})
        dfree(c, p);
    S = SphereSet();
}

namespace {

// projector (nrow0 = nproj) or Hubbard rows (nhub) at the given k points: kc [nk][3] Cartesian,
// Miller indices [nk][ld][3] of the sphere set S
hp_status family_rows(hp_ctx* c, const std::vector<double>& kc, const std::vector<int>& mil, const SphereSet& S,
                      bool hub, double2* out) {
    const int nk = (int)kc.size() / 3;
    const int nrow_all = c->nproj + c->nhub;
    const int nrow = hub ? c->nhub : c->nproj;
    if (nrow == 0) return HP_OK;
    const int o = hub ? c->nproj : 0;
    int* d_mil;
    double* d_kc;
    CK(dalloc(c, &d_mil, mil.size()));
    CK(dalloc(c, &d_kc, kc.size()));
    CK(h2d(d_mil, mil.data(), mil.size(), c->st));
    CK(h2d(d_kc, kc.data(), kc.size(), c->st));
    CK(k_formfactor(d_kc, nk, d_mil, S.d_npw, c->ld, c->d_bvec, nrow, c->d_proj_int + o, c->d_proj_int + nrow_all + o,
                    c->d_proj_int + 2 * nrow_all + o, c->d_proj_dbl + o, c->d_proj_dbl + nrow_all + o, c->d_tau, out,
                    c->st));
    CK(cudaStreamSynchronize(c->st));
    dfree(c, d_mil);
    dfree(c, d_kc);
    return HP_OK;
}

// the families at k+q for a q with off-mesh points (QFam of iq)
hp_status build_qfam(hp_ctx* c, int iq, const std::vector<const KSphere*>& sph, const std::vector<std::array<int, 3>>& g0,
                     const std::vector<int>& kprime) {
    QFam& F = c->qfam[iq];
    const int nk = c->nk, ld = c->ld, nspin = c->nspin, nocc = c->nocc;
    const size_t npsi = (size_t)nspin * nk * nocc * ld, nbeta = (size_t)nk * std::max(1, c->nproj) * ld,
                 nphi = (size_t)nk * c->nhub * ld;
    if (!F.beta) {
        CK(dalloc(c, &F.beta, nbeta));
        CK(dalloc(c, &F.phi, nphi));
        CK(dalloc(c, &F.beta32, nbeta));
        CK(dalloc(c, &F.phi32, nphi));
    }
    dfree(c, F.psi);
    dfree(c, F.psi32);
    CK(dalloc(c, &F.psi, npsi));
    CK(dalloc(c, &F.psi32, npsi));
    // Miller indices and Cartesian k+q of every k of this q (the q sphere set's order)
    std::vector<int> mil((size_t)nk * ld * 3, 0);
    std::vector<double> kc(3 * nk);
    const int qi[3] = {iq / (c->qmesh[1] * c->qmesh[2]), (iq / c->qmesh[2]) % c->qmesh[1], iq % c->qmesh[2]};
    for (int ik = 0; ik < nk; ++ik) {
        const KSphere& s = *sph[ik];
        for (int i = 0; i < s.npw; ++i)
            for (int d = 0; d < 3; ++d) mil[((size_t)ik * ld + i) * 3 + d] = s.miller[3 * i + d] - g0[ik][d];
        const int ki[3] = {ik / (c->kmesh[1] * c->kmesh[2]), (ik / c->kmesh[2]) % c->kmesh[1], ik % c->kmesh[2]};
        double kf[3];
        for (int d = 0; d < 3; ++d) kf[d] = (double)ki[d] / c->kmesh[d] + (double)qi[d] / c->qmesh[d];
        for (int d = 0; d < 3; ++d)
            kc[3 * ik + d] = kf[0] * c->bvec[0 * 3 + d] + kf[1] * c->bvec[1 * 3 + d] + kf[2] * c->bvec[2 * 3 + d];
    }
    hp_status s = family_rows(c, kc, mil, c->qc.set, false, F.beta);
    if (s == HP_OK) s = family_rows(c, kc, mil, c->qc.set, true, F.phi);
    if (s == HP_OK && c->opt.hub_ortho) s = ortho_hubbard_rows(c, c->qc.set, nk, F.phi);
    if (s != HP_OK) return s;
    if (c->hub_on) {  // W of the ground state's Hubbard potential at every k+q of this q
        std::vector<double> kf(3 * nk);
        for (int ik = 0; ik < nk; ++ik) {
            const int ki[3] = {ik / (c->kmesh[1] * c->kmesh[2]), (ik / c->kmesh[2]) % c->kmesh[1], ik % c->kmesh[2]};
            for (int d = 0; d < 3; ++d) kf[3 * ik + d] = (double)ki[d] / c->kmesh[d] + (double)qi[d] / c->qmesh[d];
        }
        double* d_kf;
        CK(dalloc(c, &d_kf, kf.size()));
        CK(h2d(d_kf, kf.data(), kf.size(), c->st));
        dfree(c, F.hubW);
        CK(dalloc(c, &F.hubW, (size_t)nspin * nk * c->nhub * c->nhub));
        if ((s = hub_build_w(c, c->d_hub_occ, nspin, nk, d_kf, F.hubW)) != HP_OK) return s;
        CK(cudaStreamSynchronize(c->st));
        dfree(c, d_kf);
    }
    // occupied states: rows of k' on the mesh, non-self-consistent states off it
    std::vector<int> off;
    for (int ik = 0; ik < nk; ++ik) {
        if (kprime[ik] >= 0) {
            for (int sp = 0; sp < nspin; ++sp)
                CK(cudaMemcpyAsync(F.psi + ((size_t)sp * nk + ik) * nocc * ld,
                                   c->d_psi + ((size_t)sp * nk + kprime[ik]) * c->nbnd * ld,
                                   sizeof(double2) * (size_t)nocc * ld, cudaMemcpyDeviceToDevice, c->st));
        } else {
            off.push_back(ik);
        }
    }
    if (!off.empty()) {
        const int noff = (int)off.size();
        std::vector<const KSphere*> so(noff);
        std::vector<double> kco(3 * noff);
        std::vector<int> milo((size_t)noff * ld * 3, 0);
        for (int j = 0; j < noff; ++j) {
            so[j] = sph[off[j]];
            for (int d = 0; d < 3; ++d) kco[3 * j + d] = kc[3 * off[j] + d];
            std::copy(mil.begin() + (size_t)off[j] * ld * 3, mil.begin() + (size_t)(off[j] + 1) * ld * 3,
                      milo.begin() + (size_t)j * ld * 3);
        }
        SphereSet So;
        const bool fused_before = c->fused;
        s = upload_sphereset(c, so, nullptr, So);
        c->fused = fused_before;  // the off-mesh set is not used by the fused transforms
        if (s != HP_OK) return s;
        double2 *beta_o = nullptr, *psi_o = nullptr, *phi_o = nullptr, *w_o = nullptr;
        CK(dalloc(c, &beta_o, (size_t)noff * std::max(1, c->nproj) * ld));
        CK(dalloc(c, &psi_o, (size_t)nspin * noff * nocc * ld));
        s = family_rows(c, kco, milo, So, false, beta_o);
        if (s == HP_OK && c->hub_on) {  // Hubbard rows and W of the off-mesh points, packed like beta_o
            const size_t nn = (size_t)c->nhub * c->nhub;
            CK(dalloc(c, &phi_o, (size_t)noff * c->nhub * ld));
            CK(dalloc(c, &w_o, (size_t)nspin * noff * nn));
            for (int j = 0; j < noff; ++j) {
                CK(cudaMemcpyAsync(phi_o + (size_t)j * c->nhub * ld, F.phi + (size_t)off[j] * c->nhub * ld,
                                   sizeof(double2) * c->nhub * ld, cudaMemcpyDeviceToDevice, c->st));
                for (int sp = 0; sp < nspin; ++sp)
                    CK(cudaMemcpyAsync(w_o + ((size_t)sp * noff + j) * nn, F.hubW + ((size_t)sp * nk + off[j]) * nn,
                                       sizeof(double2) * nn, cudaMemcpyDeviceToDevice, c->st));
            }
        }
        std::vector<double> eps_o;
        if (s == HP_OK) s = nscf_states(c, so, So, beta_o, phi_o, w_o, psi_o, eps_o);
        if (s != HP_OK) return s;
        dfree(c, phi_o);
        dfree(c, w_o);
        for (int j = 0; j < noff; ++j)
            for (int sp = 0; sp < nspin; ++sp)
                CK(cudaMemcpyAsync(F.psi + ((size_t)sp * nk + off[j]) * nocc * ld,
                                   psi_o + ((size_t)sp * noff + j) * nocc * ld, sizeof(double2) * (size_t)nocc * ld,
                                   cudaMemcpyDeviceToDevice, c->st));
        CK(cudaStreamSynchronize(c->st));
        dfree(c, beta_o);
        dfree(c, psi_o);
        free_sphereset(c, So);
    }
    CK(k_to_c32(F.psi, F.psi32, (long long)npsi, c->st));
    CK(k_to_c32(F.beta, F.beta32, (long long)nbeta, c->st));
    if (nphi) CK(k_to_c32(F.phi, F.phi32, (long long)nphi, c->st));
    CK(cudaStreamSynchronize(c->st));
    F.built = true;
    return HP_OK;
}

// per q: spheres at k+q = k' + G0 (the k' sphere with Miller indices shifted by -G0) and kmap k -> k';
// where k+q is off the mesh, its own sphere and the families materialised at k+q (QFam)
hp_status prepare_q(hp_ctx* c, int iq, std::vector<int>& kprime) {
    const int qi[3] = {iq / (c->qmesh[1] * c->qmesh[2]), (iq / c->qmesh[2]) % c->qmesh[1], iq % c->qmesh[2]};
    kprime.assign(c->nk, 0);
    std::vector<std::array<int, 3>> g0(c->nk);
    std::vector<const KSphere*> sph(c->nk);
    bool off = false;
    for (int ik = 0; ik < c->nk; ++ik) {
        const int ki[3] = {ik / (c->kmesh[1] * c->kmesh[2]), (ik / c->kmesh[2]) % c->kmesh[1], ik % c->kmesh[2]};
        const KSphere& kq = c->kq_ks[(size_t)iq * c->nk + ik];
        if (kq.npw > 0) {  // off the mesh
            off = true;
            kprime[ik] = -1;
            g0[ik] = {0, 0, 0};
            sph[ik] = &kq;
            continue;
        }
        int j[3];
        for (int d = 0; d < 3; ++d) {
            const int x = (ki[d] * c->qmesh[d] + qi[d] * c->kmesh[d]) / c->qmesh[d];  // (k+q) in units of 1/kmesh
            j[d] = x % c->kmesh[d];
            g0[ik][d] = x / c->kmesh[d];
        }
        kprime[ik] = (j[0] * c->kmesh[1] + j[1]) * c->kmesh[2] + j[2];
        sph[ik] = &c->ks[kprime[ik]];
    }
    // the route of this q: fused where the grid, the k set and the k+q set allow it, whatever earlier
    // q points chose (so that a response does not depend on the calls before it)
    if (c->qc.iq == iq) {
        c->fused = c->fused_grid && c->kset.cols_distinct && c->qc.set.cols_distinct;
        return HP_OK;
    }
    hp_status s = upload_sphereset(c, sph, &g0, c->qc.set);
    c->fused = c->fused_grid && c->kset.cols_distinct && c->qc.set.cols_distinct;
    if (s != HP_OK) return s;
    std::vector<int> kmap(c->nk);
    for (int ik = 0; ik < c->nk; ++ik) kmap[ik] = off ? ik : kprime[ik];
    if (!c->qc.d_miller) CK(dalloc(c, &c->qc.d_miller, c->nk));  // holds the k map of the families
    CK(h2d(c->qc.d_miller, kmap.data(), c->nk, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->qc.off = off;
    if (off && !c->qfam[iq].built) {
        s = build_qfam(c, iq, sph, g0, kprime);
        if (s != HP_OK) return s;
    }
    c->qc.iq = iq;
    return HP_OK;
}

// projector, Hubbard and occupied-state families at k+q for the current q (through the k map on
// the mesh, or the materialised QFam)
ProjMat fam_beta_kq(const hp_ctx* c) {
    if (c->qc.off) {
        const QFam& F = c->qfam[c->qc.iq];
        return ProjMat{F.beta, 0, (long long)c->nproj * c->ld, c->nproj, 0, nullptr, F.beta32};
    }
    ProjMat A = beta_family(c, c->qc.d_miller);
    A.base32 = c->d_beta32;
    return A;
}

ProjMat fam_phi_kq(const hp_ctx* c, int nrow, int row0) {
    if (c->qc.off) {
        const QFam& F = c->qfam[c->qc.iq];
        return ProjMat{F.phi, 0, (long long)c->nhub * c->ld, nrow, row0, nullptr, F.phi32};
    }
    return ProjMat{c->d_phi_k, 0, (long long)c->nhub * c->ld, nrow, row0, c->qc.d_miller, c->d_phi32};
}

// occupied states at k+q as a family: base, strides, FP32 copy
void fam_psi_kq(const hp_ctx* c, const double2** base, const float2** base32, long long* ss, long long* sk) {
    if (c->qc.off) {
        const QFam& F = c->qfam[c->qc.iq];
        *base = F.psi;
        *base32 = F.psi32;
        *ss = (long long)c->nk * c->nocc * c->ld;
        *sk = (long long)c->nocc * c->ld;
    } else {
        *base = c->d_psi;
        *base32 = c->d_psi32;
        *ss = (long long)c->nk * c->nbnd * c->ld;
        *sk = (long long)c->nbnd * c->ld;
    }
}

// Y += V_Hub X at k+q (DFT+U+V ground states; the Hubbard potential is fixed in the response)
hp_status hub_term_kq(hp_ctx* c, const BandList& L, const double2* X, double2* Y) {
    if (!c->hub_on || !c->d_hubW) return HP_OK;
    const bool fp32 = c->opt.precision == HP_PRECISION_MIXED;
    const ProjMat F = fam_phi_kq(c, c->nhub, 0);
    const double2* W = c->qc.off ? c->qfam[c->qc.iq].hubW : c->d_hubW;
    return hub_apply(c, c->qc.set, L, F.base, F.kmap, W, X, Y, c->vec32, fp32, c->d_Pbuf);
}

// Y = A X = (H_k+q + alpha O_k+q - eps_v) X on the items of L
hp_status apply_sternheimer(hp_ctx* c, const BandList& L, const double2* X, double2* Y) {
    const SphereSet& S = c->qc.set;
    const bool fp32 = c->opt.precision == HP_PRECISION_MIXED;
    hp_status s = (c->fused && c->d_vt) ? apply_local_fused(c, S, L, X, Y, fp32) : apply_local(c, S, L, X, Y, c->d_veff, fp32);
    // (FP32 band vectors are used only together with the fused transforms)
    if (s != HP_OK) return s;
    // V_NL and alpha P_v in one projection and one expansion: rows 0 .. nproj-1 are beta (weights
    // D), rows nproj .. nproj+nocc-1 the occupied states at k+q (weight alpha)
    ProjMat A = fam_beta_kq(c);
    fam_psi_kq(c, &A.base2, &A.base2_32, &A.stride2_s, &A.stride2_k);
    A.nrow2 = c->nocc;
    A.scale2 = c->alpha_pv;
    if (A.nrow + A.nrow2 > c->proj_rows_max) {  // more rows than one projection holds: beta, then P_v
        ProjMat U{A.base2, A.stride2_s, A.stride2_k, c->nocc, 0, A.kmap, A.base2_32};
        A.base2 = nullptr;
        A.base2_32 = nullptr;
        A.nrow2 = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const ProjMat& F = pass == 0 ? A : U;
            const double* w = pass == 0 ? c->d_projD : nullptr;
            const double al = pass == 0 ? 1.0 : c->alpha_pv;
            if (F.nrow == 0) continue;
            if (c->vec32) {
                if ((s = project(c, S, L, F, (const float2*)X, c->d_Pbuf, fp32)) != HP_OK) return s;
                CK(k_expand(L, S, F, c->d_Pbuf, w, al, (float2*)Y, c->ld, c->st, fp32));
            } else {
                if ((s = project(c, S, L, F, X, c->d_Pbuf, fp32)) != HP_OK) return s;
                CK(k_expand(L, S, F, c->d_Pbuf, w, al, Y, c->ld, c->st, fp32));
            }
        }
        return hub_term_kq(c, L, X, Y);
    }
    if (c->vec32) {
        s = project(c, S, L, A, (const float2*)X, c->d_Pbuf, fp32);
        if (s != HP_OK) return s;
        CK(k_expand(L, S, A, c->d_Pbuf, c->d_projD, 1.0, (float2*)Y, c->ld, c->st, fp32));
    } else {
        s = project(c, S, L, A, X, c->d_Pbuf, fp32);
        if (s != HP_OK) return s;
        CK(k_expand(L, S, A, c->d_Pbuf, c->d_projD, 1.0, Y, c->ld, c->st, fp32));
    }
    return hub_term_kq(c, L, X, Y);
}

double dev_dot(hp_ctx* c, const double2* a, const double2* b, long long n, cudaError_t* err) {
    double v = 0.0;
    cudaError_t e = k_vec_dot(a, b, n, c->d_small, c->d_partial, c->st);
    if (e == cudaSuccess) e = d2h(&v, c->d_small, 1, c->st);
    *err = e;
    return v;
}

}  // namespace

// k+q for mesh point ik and q point iq: on the k mesh k+q = k' + G0 (kp >= 0), else kp = -1
static void kq_point(const hp_ctx* c, int iq, int ik, int* kp, int g0[3]) {
    const int qi[3] = {iq / (c->qmesh[1] * c->qmesh[2]), (iq / c->qmesh[2]) % c->qmesh[1], iq % c->qmesh[2]};
    const int ki[3] = {ik / (c->kmesh[1] * c->kmesh[2]), (ik / c->kmesh[2]) % c->kmesh[1], ik % c->kmesh[2]};
    if (c->kq_ks[(size_t)iq * c->nk + ik].npw > 0) {
        *kp = -1;
        g0[0] = g0[1] = g0[2] = 0;
        return;
    }
    int j[3];
    for (int d = 0; d < 3; ++d) {
        const int x = (ki[d] * c->qmesh[d] + qi[d] * c->kmesh[d]) / c->qmesh[d];
        j[d] = x % c->kmesh[d];
        g0[d] = x / c->kmesh[d];
    }
    *kp = (j[0] * c->kmesh[1] + j[1]) * c->kmesh[2] + j[2];
}

extern "C" hp_status hp_sphere_kq(const hp_ctx* c, int iq, int ik, int* npw, int* miller) {
    if (!c || !npw || iq < 0 || iq >= c->nq || ik < 0 || ik >= c->nk) return HP_EINVAL;
    int kp, g0[3];
    kq_point(c, iq, ik, &kp, g0);
    const KSphere& s = kp >= 0 ? c->ks[kp] : c->kq_ks[(size_t)iq * c->nk + ik];
    *npw = s.npw;
    if (miller)
        for (int i = 0; i < s.npw; ++i)
            for (int d = 0; d < 3; ++d) miller[3 * i + d] = s.miller[3 * i + d] - g0[d];
    return HP_OK;
}

extern "C" hp_status hp_apply_sternheimer(hp_ctx* c, int iq, int ik, int spin, int nb, const double* eps,
                                          const double* psi, double* out) {
    if (!c) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "hp_apply_sternheimer: no ground state");
    if (iq < 0 || iq >= c->nq || ik < 0 || ik >= c->nk || spin < 0 || spin >= c->nspin || nb < 1 || !eps || !psi || !out)
        return fail(c, HP_EINVAL, "hp_apply_sternheimer: bad arguments");
    const bool mixed = c->opt.precision == HP_PRECISION_MIXED;
    hp_status s = prepare_resp(c);
    if (s != HP_OK) return s;
    std::vector<int> kprime;
    if ((s = prepare_q(c, iq, kprime)) != HP_OK) return s;
    if (c->ur_planes != c->fused) {
        c->resp_ready = false;
        if ((s = prepare_resp(c)) != HP_OK) return s;
    }
    const bool v32 = mixed && c->fused;
    c->vec32 = v32;
    const int ld = c->ld, npw = c->qc.set.npw[ik];
    const int chunk = std::min(nb, c->resp_rows);
    double2 *dX64, *dX, *dY;
    CK(dalloc(c, &dX64, (size_t)chunk * ld));
    CK(dalloc(c, &dX, (size_t)chunk * ld));
    CK(dalloc(c, &dY, (size_t)chunk * ld));
    std::vector<double2> h((size_t)chunk * ld);
    for (int b0 = 0; b0 < nb && s == HP_OK; b0 += chunk) {
        const int nc = std::min(chunk, nb - b0);
        std::fill(h.begin(), h.end(), cmk(0.0, 0.0));
        for (int b = 0; b < nc; ++b)
            for (int i = 0; i < npw; ++i)
                h[(size_t)b * ld + i] = cmk(psi[2 * ((size_t)(b0 + b) * npw + i)], psi[2 * ((size_t)(b0 + b) * npw + i) + 1]);
        CK(h2d(dX64, h.data(), (size_t)nc * ld, c->st));
        CK(cudaMemsetAsync(dY, 0, sizeof(double2) * (size_t)chunk * ld, c->st));
        if (v32) CK(k_to_c32(dX64, reinterpret_cast<float2*>(dX), (long long)nc * ld, c->st));
        else CK(cudaMemcpyAsync(dX, dX64, sizeof(double2) * (size_t)nc * ld, cudaMemcpyDeviceToDevice, c->st));
        BandList& L = c->L3;
        list_clear(L);
        for (int b = 0; b < nc; ++b) list_add(L, b, ik, spin, eps[b0 + b]);
        if ((s = upload_list(c, L)) != HP_OK) break;
        if ((s = apply_sternheimer(c, L, dX, dY)) != HP_OK) break;
        if (v32) CK(k_to_c64(reinterpret_cast<const float2*>(dY), dX64, (long long)nc * ld, c->st));
        else CK(cudaMemcpyAsync(dX64, dY, sizeof(double2) * (size_t)nc * ld, cudaMemcpyDeviceToDevice, c->st));
        CK(d2h(h.data(), dX64, (size_t)nc * ld, c->st));
        for (int b = 0; b < nc; ++b)
            for (int i = 0; i < npw; ++i) {
                out[2 * ((size_t)(b0 + b) * npw + i)] = h[(size_t)b * ld + i].x;
                out[2 * ((size_t)(b0 + b) * npw + i) + 1] = h[(size_t)b * ld + i].y;
            }
    }
    dfree(c, dX64);
    dfree(c, dX);
    dfree(c, dY);
    if (s == HP_OK && tc_enabled() && tc_take_error(c->st))
        return fail(c, HP_ETIMEOUT, "hp_apply_sternheimer: a tensor-core contraction gave up on a bounded wait");
    return s;
}

extern "C" hp_status hp_response(hp_ctx* c, int iq, int atom, double* dn0_out, double* dn_out, hp_resp_info* info) {
    if (!c) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "hp_response: no ground state");
    if (!(c->gap > 1e-4)) return fail(c, HP_ENOGAP, "hp_response: the ground state has no gap at the fixed band count");
    if (iq < 0 || iq >= c->nq) return fail(c, HP_EINVAL, "hp_response: q index out of range");
    int jj = -1;
    for (size_t i = 0; i < c->hub_atoms.size(); ++i)
        if (c->hub_atoms[i] == atom) jj = (int)i;
    if (jj < 0) return fail(c, HP_EINVAL, "hp_response: atom is not a Hubbard atom");
    if (c->opt.precision != HP_PRECISION_FP64 && c->opt.precision != HP_PRECISION_MIXED)
        return fail(c, HP_EINVAL, "hp_response: unknown precision");
    const bool mixed = c->opt.precision == HP_PRECISION_MIXED;
    auto t0 = std::chrono::steady_clock::now();
    hp_status s = prepare_resp(c);
    if (s != HP_OK) return s;
    std::vector<int> kprime;
    s = prepare_q(c, iq, kprime);
    if (s != HP_OK) return s;
    if (c->ur_planes != c->fused) {  // the route changed with q: rebuild the caches
        c->resp_ready = false;
        if ((s = prepare_resp(c)) != HP_OK) return s;
    }
    // Band vectors of the response (x, r, p, Ap, b, V_pert u) are FP32 in the mixed form with the
    // fused transforms (step lengths, residual norms and every sum stay FP64), FP64 otherwise.
    const bool v32 = mixed && c->fused;
    c->vec32 = v32;
    auto F32 = [](double2* p) { return reinterpret_cast<float2*>(p); };
    const int nspin = c->nspin, nk = c->nk, nocc = c->nocc, nr = c->nr, ld = c->ld;
    const int rows = nspin * nk * nocc;
    const int nh = (int)c->hub_atoms.size();
    const long long nvec = (long long)rows * ld;
    const long long ndv = (long long)nspin * nr;
    const SphereSet& Sq = c->qc.set;
    // lists: Lall over response rows, Lpsi over the same (s, k, v) items with psi rows
    BandList& Lall = c->L1;
    BandList& Lpsi = c->L2;
    list_clear(Lall);
    list_clear(Lpsi);
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nk; ++k)
            for (int v = 0; v < nocc; ++v) {
                const int item = (sp * nk + k) * nocc + v;
                list_add(Lall, item, k, sp, c->eps[((size_t)sp * nk + k) * c->nbnd + v]);
                list_add(Lpsi, (sp * nk + k) * c->nbnd + v, k, sp, 0.0);
            }
    if ((s = upload_list(c, Lall)) != HP_OK) return s;
    if ((s = upload_list(c, Lpsi)) != HP_OK) return s;
    // V_pert u_k = sum_m phi^J_m,k+q <phi^J_m,k|u_k>
    const int mJ = c->hub_mdim[jj], oJ = c->hub_off[jj];
    ProjMat phiJk{c->d_phi_k, 0, (long long)c->nhub * ld, mJ, oJ, nullptr, c->d_phi32};
    ProjMat phiJkq = fam_phi_kq(c, mJ, oJ);
    ProjMat phikq = fam_phi_kq(c, c->nhub, 0);
    ProjMat Ukq{nullptr, 0, 0, nocc, 0, nullptr};
    {
        const double2* b64;
        const float2* b32;
        long long ss, sk;
        fam_psi_kq(c, &b64, &b32, &ss, &sk);
        Ukq = ProjMat{b64, ss, sk, nocc, 0, c->qc.off ? nullptr : c->qc.d_miller, b32};
    }
    if ((s = project(c, c->kset, Lpsi, phiJk, c->d_psi, c->d_Pbuf, mixed)) != HP_OK) return s;
    CK(cudaMemsetAsync(c->d_vpu, 0, sizeof(double2) * nvec, c->st));
    if (v32) CK(k_expand(Lall, Sq, phiJkq, c->d_Pbuf, nullptr, 1.0, F32(c->d_vpu), ld, c->st, mixed));
    else CK(k_expand(Lall, Sq, phiJkq, c->d_Pbuf, nullptr, 1.0, c->d_vpu, ld, c->st, mixed));
    CK(cudaMemsetAsync(c->d_x, 0, sizeof(double2) * nvec, c->st));
    CK(cudaMemsetAsync(c->d_dv, 0, sizeof(double2) * ndv, c->st));
    const double f = nspin == 1 ? 2.0 : 1.0;
    const double wrho = 2.0 * f / (nk * c->omega);
    const double tol2 = c->opt.cg_tol * c->opt.cg_tol;
    std::vector<double> rr(rows);
    std::vector<double> dn0, dn((size_t)nh * nspin * kMmax * kMmax * 2);
    std::vector<double> tr0, tr((size_t)2 * nh), tr_prev;
    long long cg_total = 0, hpsi = 0;
    int nhist = 0;
    double res = INFINITY, dchi = INFINITY, res_rel = 1.0;
    bool converged = false, cg_ok = true, stagnated = false;
    int it = 0;
    std::vector<double> res_hist;
    const bool verbose = getenv("HP_VERBOSE") != nullptr;
    for (it = 1; it <= c->opt.niter_max; ++it) {
        // ---- right-hand side b = -P_c (dV u + V_pert u)
        if (it == 1) {
            if (v32) CK(k_vec_scale_copy(F32(c->d_b), F32(c->d_vpu), -1.0, nvec, c->st));
            else CK(k_vec_scale_copy(c->d_b, c->d_vpu, -1.0, nvec, c->st));
        } else {
            s = ensure_grid(c, band_batch(c, rows));
            if (s != HP_OK) return s;
            if (c->fused) {
                // plane-major Delta V, then u_k(r) Delta V(r) -> forward transform onto the k+q sphere
                CK(k_to_planes_c(c->d_dv, c->d_drho_pm, c->N, nspin, c->st));
                if (mixed) CK(k_to_c32(c->d_drho_pm, (float2*)c->d_dvt, ndv, c->st));
                else CK(cudaMemcpyAsync(c->d_dvt, c->d_drho_pm, sizeof(double2) * ndv, cudaMemcpyDeviceToDevice, c->st));
                const int chunk = fused_batch(c, Sq, rows);
                if ((s = ensure_colbuf(c, sizeof(double2) * (size_t)chunk * c->N[2] * Sq.ncmax)) != HP_OK) return s;
                for (int c0 = 0; c0 < rows; c0 += chunk) {
                    FusedArgs a = fused_args(c, Sq, Lall);
                    a.c0 = c0;
                    a.nc = std::min(chunk, rows - c0);
                    a.ur = mixed ? (const void*)c->d_ur32 : (const void*)c->d_ur;
                    a.dvt = c->d_dvt;
                    a.Y = c->d_b;
                    a.vec32 = v32;
                    a.mode = 1;
                    a.scale = -1.0;
                    CK(fused_plane(mixed, 2, a));
                    CK(fused_col(mixed, false, a));
                }
            } else if (mixed) {
                float2* g32 = (float2*)c->d_grid;
                const int cap = 2 * band_batch(c, rows);
                CK(k_to_c32(c->d_dv, c->d_dv32, ndv, c->st));
                for (int c0 = 0; c0 < rows; c0 += cap) {
                    const int nc = std::min(cap, rows - c0);
                    CK(k_mul_cpot32(g32, c->d_ur32, Lall.d_row, nc, nr, c->d_dv32, Lall, c0, c->st));
                    CK(fft3d(c->fft, g32, nc, -1, c->st));
                    CK(k_gather_scaled32(Sq, Lall, c0, nc, g32, nr, -1.0 / nr, c->d_b, ld, c->st));
                }
            } else {
                const int chunk = band_batch(c, rows);
                for (int c0 = 0; c0 < rows; c0 += chunk) {
                    const int nc = std::min(chunk, rows - c0);
                    CK(k_mul_cpot(c->d_grid, c->d_ur, Lall.d_row, nc, nr, c->d_dv, Lall, c0, c->st));
                    CK(fft3d(c->fft, c->d_grid, nc, -1, c->st));
                    CK(k_gather_scaled(Sq, Lall, c0, nc, c->d_grid, nr, -1.0 / nr, c->d_b, ld, 0, c->st));
                }
            }
            if (v32) CK(k_vec_axpy(F32(c->d_b), F32(c->d_vpu), -1.0, nvec, c->st));
            else CK(k_vec_axpy(c->d_b, c->d_vpu, -1.0, nvec, c->st));
        }
        if (v32) {
            if ((s = project(c, Sq, Lall, Ukq, F32(c->d_b), c->d_Pbuf, mixed)) != HP_OK) return s;
            CK(k_expand(Lall, Sq, Ukq, c->d_Pbuf, nullptr, -1.0, F32(c->d_b), ld, c->st, mixed));
        } else {
            if ((s = project(c, Sq, Lall, Ukq, c->d_b, c->d_Pbuf, mixed)) != HP_OK) return s;
            CK(k_expand(Lall, Sq, Ukq, c->d_Pbuf, nullptr, -1.0, c->d_b, ld, c->st, mixed));
        }
        // per-band stopping rule: ||r|| <= cg_tol, and in the mixed form also <= 1e-7 ||b|| (the FP32
        // operator is accurate to about 1e-7 relative; iterating below that buys nothing)
        // Outer iterations after the first solve only as far as the response potential is known:
        // theta = min(1e-2, cg_adapt x the previous relative Hxc residual) of ||b|| (the first
        // iteration gives chi_0 and is solved to cg_tol).
        std::vector<double> tolb(rows, tol2);
        const double theta = (it > 1 && c->opt.cg_adapt > 0) ? std::min(1e-2, c->opt.cg_adapt * res_rel) : 0.0;
        if (mixed || theta > 0) {
            if (v32) CK(k_band_dot(Lall, Sq, F32(c->d_b), F32(c->d_b), ld, c->d_pap, c->st));
            else CK(k_band_dot(Lall, Sq, c->d_b, c->d_b, ld, c->d_pap, c->st));
            CK(d2h(rr.data(), c->d_pap, rows, c->st));
            const double f2 = std::max(mixed ? 1e-14 : 0.0, theta * theta);
            for (int i = 0; i < rows; ++i) tolb[i] = std::max(tol2, f2 * rr[i]);
        }
        // ---- CG on every band, warm start from the previous x
        if ((s = apply_sternheimer(c, Lall, c->d_x, c->d_ap)) != HP_OK) return s;
        hpsi += rows;
        if (v32) {
            CK(k_vec_sub(F32(c->d_r), F32(c->d_b), F32(c->d_ap), nvec, c->st));
            CK(k_cg_init(Lall, Sq, F32(c->d_r), F32(c->d_p), ld, c->d_rz, c->d_rr, c->st));
        } else {
            CK(k_vec_sub(c->d_r, c->d_b, c->d_ap, nvec, c->st));
            CK(k_cg_init(Lall, Sq, c->d_r, c->d_p, ld, c->d_rz, c->d_rr, c->st));
        }
        int cgit = 0;
        BandList& La = c->L3;  // active (not yet converged) bands
        for (;;) {
            CK(d2h(rr.data(), c->d_rr, rows, c->st));
            list_clear(La);
            for (int i = 0; i < rows; ++i) {
                if (!std::isfinite(rr[i])) {
                    if (tc_enabled() && tc_take_error(c->st))
                        return fail(c, HP_ETIMEOUT, "hp_response: a tensor-core contraction gave up on a bounded wait");
                    return fail(c, HP_ENUMERIC, "hp_response: non-finite CG residual");
                }
                if (rr[i] > tolb[i]) list_add(La, Lall.row[i], Lall.k[i], Lall.spin[i], Lall.shift[i]);
            }
            if (La.row.empty()) break;
            if (cgit >= c->opt.cg_maxiter) {
                cg_ok = false;
                break;
            }
            if ((s = upload_list(c, La)) != HP_OK) return s;
            if ((s = apply_sternheimer(c, La, c->d_p, c->d_ap)) != HP_OK) return s;
            hpsi += La.nb;
            if (v32)
                CK(k_cg_step(La, Sq, F32(c->d_x), F32(c->d_r), F32(c->d_p), F32(c->d_ap), ld, c->d_pap, c->d_rz,
                             c->d_rr, c->st));
            else
                CK(k_cg_step(La, Sq, c->d_x, c->d_r, c->d_p, c->d_ap, ld, c->d_pap, c->d_rz, c->d_rr, c->st));
            cg_total += La.nb;
            ++cgit;
        }
        // ---- response density
        CK(cudaMemsetAsync(c->d_drho, 0, sizeof(double2) * ndv, c->st));
        s = ensure_grid(c, band_batch(c, rows));
        if (s != HP_OK) return s;
        if ((s = ensure_scratch(c, (size_t)64 * nr)) != HP_OK) return s;  // band-slice partial sums
        if (c->fused) {
            // x -> real space (plane-major) through the fused path, then conj(u) x accumulated per spin
            CK(cudaMemsetAsync(c->d_drho_pm, 0, sizeof(double2) * ndv, c->st));
            const int chunk = fused_batch(c, Sq, rows);
            if ((s = ensure_colbuf(c, sizeof(double2) * (size_t)chunk * c->N[2] * Sq.ncmax)) != HP_OK) return s;
            FusedArgs probe = fused_args(c, Sq, Lall);
            const bool fdrho = v32 && fused_drho_supported(probe);
            if (fdrho) {
                // FP32 form: Delta u(r) stays on chip; group sums of conj(u) Delta u, then the groups in order
                int ng = 0;
                for (int c0 = 0; c0 < rows; c0 += chunk) ng += fused_drho_groups(c->N[0], c->N[1], std::min(chunk, rows - c0));
                // the groups' sums, then their spin masks (ints) in the scratch's last elements
                const size_t nmask = ((size_t)ng + 3) / 4;
                if ((s = ensure_scratch(c, (size_t)ng * 2 * nr + nmask)) != HP_OK) return s;
                int* gmask = reinterpret_cast<int*>(c->d_scratch + (size_t)ng * 2 * nr);
                int g0 = 0;
                for (int c0 = 0; c0 < rows; c0 += chunk) {
                    FusedArgs a = fused_args(c, Sq, Lall);
                    a.c0 = c0;
                    a.nc = std::min(chunk, rows - c0);
                    a.X = c->d_x;
                    a.vec32 = true;
                    a.ur = c->d_ur32;
                    CK(fused_col(true, true, a));
                    CK(fused_drho(a, c->d_scratch, gmask, g0));
                    g0 += fused_drho_groups(c->N[0], c->N[1], a.nc);
                }
                CK(k_drho_reduce(c->d_scratch, ng, nr, nspin, wrho, c->d_drho_pm, c->st, gmask));
            }
            const int gchunk = std::min(chunk, band_batch(c, rows));  // real-space bands in the grid buffer
            for (int c0 = 0; c0 < rows && !fdrho; c0 += gchunk) {
                FusedArgs a = fused_args(c, Sq, Lall);
                a.c0 = c0;
                a.nc = std::min(gchunk, rows - c0);
                a.X = c->d_x;
                a.vec32 = v32;
                a.out = c->d_grid;
                CK(fused_col(mixed, true, a));
                CK(fused_plane(mixed, 1, a));
                if (mixed)
                    CK(k_drho_acc32(c->d_ur32, Lall.d_row, (const float2*)c->d_grid, a.nc, nr, Lall, c0, wrho, nspin,
                                    c->d_drho_pm, c->d_scratch, c->scratch_elems, c->st));
                else
                    CK(k_drho_acc(c->d_ur, Lall.d_row, c->d_grid, a.nc, nr, Lall, c0, wrho, nspin, c->d_drho_pm, c->d_scratch, c->scratch_elems, c->st));
            }
            CK(k_from_planes_c(c->d_drho_pm, c->d_drho, c->N, nspin, c->st));
        } else if (mixed) {
            float2* g32 = (float2*)c->d_grid;
            const int cap = 2 * band_batch(c, rows);
            for (int c0 = 0; c0 < rows; c0 += cap) {
                const int nc = std::min(cap, rows - c0);
                CK(k_scatter32(Sq, Lall, c0, nc, c->d_x, g32, nr, c->st));
                CK(fft3d(c->fft, g32, nc, +1, c->st));
                CK(k_drho_acc32(c->d_ur32, Lall.d_row, g32, nc, nr, Lall, c0, wrho, nspin, c->d_drho, c->d_scratch,
                                   c->scratch_elems, c->st));
            }
        } else {
            const int chunk = band_batch(c, rows);
            for (int c0 = 0; c0 < rows; c0 += chunk) {
                const int nc = std::min(chunk, rows - c0);
                CK(k_scatter(Sq, Lall, c0, nc, c->d_x, ld, c->d_grid, nr, c->st));
                CK(fft3d(c->fft, c->d_grid, nc, +1, c->st));
                CK(k_drho_acc(c->d_ur, Lall.d_row, c->d_grid, nc, nr, Lall, c0, wrho, nspin, c->d_drho, c->d_scratch,
                                   c->scratch_elems, c->st));
            }
        }
        // ---- response occupations
        if (v32) s = project(c, Sq, Lall, phikq, F32(c->d_x), c->d_Pbuf, mixed);
        else s = project(c, Sq, Lall, phikq, c->d_x, c->d_Pbuf, mixed);
        if (s != HP_OK) return s;
        CK(k_occ_response(c->d_Pbuf, c->d_aphi, nspin * nk, nocc, c->nhub, nk, nspin, c->d_M, c->st));
        {
            std::vector<int> off(c->hub_off), md(c->hub_mdim);
            int* d_int;
            CK(dalloc(c, &d_int, 2 * nh));
            CK(h2d(d_int, off.data(), nh, c->st));
            CK(h2d(d_int + nh, md.data(), nh, c->st));
            CK(k_dn_blocks(c->d_M, nspin, c->nhub, nh, d_int, d_int + nh, kMmax, c->d_dn, c->st));
            double2* d_tr = c->d_dn + (size_t)nh * nspin * kMmax * kMmax;
            CK(k_dn_traces(c->d_dn, nh, nspin, kMmax, f, d_tr, c->st));
            CK(d2h((double2*)dn.data(), c->d_dn, (size_t)nh * nspin * kMmax * kMmax, c->st));
            CK(d2h((double2*)tr.data(), d_tr, nh, c->st));
            dfree(c, d_int);
        }
        if (it == 1) {
            dn0 = dn;
            tr0 = tr;
        }
        // ---- Delta V_Hxc from Delta rho
        CK(cudaMemcpyAsync(c->d_dvh, c->d_drho, sizeof(double2) * nr, cudaMemcpyDeviceToDevice, c->st));
        if (nspin == 2) CK(k_vec_axpy(c->d_dvh, c->d_drho + nr, 1.0, nr, c->st));
        CK(fft3d(c->fft, c->d_dvh, 1, -1, c->st));
        const int qi[3] = {iq / (c->qmesh[1] * c->qmesh[2]), (iq / c->qmesh[2]) % c->qmesh[1], iq % c->qmesh[2]};
        const double qf[3] = {(double)qi[0] / c->qmesh[0], (double)qi[1] / c->qmesh[1], (double)qi[2] / c->qmesh[2]};
        CK(k_hartree_q(c->d_dvh, c->N, c->d_bvec, qf, 4.0 * c->ecut, 1.0 / nr, c->st));
        CK(fft3d(c->fft, c->d_dvh, 1, +1, c->st));
        CK(k_hxc_combine(c->d_dvh, c->d_drho, c->d_fxc, nspin, nr, c->d_dvout, c->st));
        cudaError_t e;
        double scf_tol = c->opt.scf_tol, chi_tol = c->opt.conv_thr_chi;
        const double vv = dev_dot(c, c->d_dvout, c->d_dvout, ndv, &e);
        if (e != cudaSuccess) return cuda_fail(c, e, "response norm");
        const double vrms = std::sqrt(vv / (double)ndv);
        double tmax = 0.0;
        for (int a = 0; a < 2 * nh; ++a) tmax = std::max(tmax, std::fabs(tr[a]));
        if (mixed) {  // FP32 noise floor: mixed_floor (3e-7) of the response potential and of the traces
            scf_tol = std::max(scf_tol, c->opt.mixed_floor * vrms);
            chi_tol = std::max(chi_tol, c->opt.mixed_floor * tmax);
        }
        // residual F = dV_out - dV_in (kept in d_dvout)
        CK(k_vec_sub(c->d_dvout, c->d_dvout, c->d_dv, ndv, c->st));
        const double ff = dev_dot(c, c->d_dvout, c->d_dvout, ndv, &e);
        if (e != cudaSuccess) return cuda_fail(c, e, "residual");
        if (!std::isfinite(ff)) return fail(c, HP_ENUMERIC, "hp_response: non-finite Hxc residual");
        res = std::sqrt(ff / (double)ndv);
        res_rel = vrms > 0 ? res / vrms : 1.0;
        dchi = INFINITY;
        if (!tr_prev.empty()) {
            dchi = 0.0;
            for (int a = 0; a < 2 * nh; ++a) dchi = std::max(dchi, std::fabs(tr[a] - tr_prev[a]));
        }
        tr_prev = tr;
        res_hist.push_back(res);
        if (verbose)
            fprintf(stderr, "hp_response: it %d res %.3e (tol %.3e) dchi %.3e (tol %.3e) cg %d bands-iterations %lld\n",
                    it, res, scf_tol, dchi, chi_tol, cgit, cg_total);
        if (it > 1 && res < scf_tol && dchi < chi_tol) {
            converged = true;
            break;
        }
        // mixed form: a residual below 1e-5 of the response potential whose last three iterations
        // came no lower than 0.8 of the best one before them sits on the FP32 noise floor; the
        // iteration has done what it can
        if (mixed && it >= 6 && res < 1e-5 * vrms) {
            const size_t n = res_hist.size();
            const double lo = std::min(res_hist[n - 1], std::min(res_hist[n - 2], res_hist[n - 3]));
            const double best = *std::min_element(res_hist.begin(), res_hist.end() - 3);
            if (lo > 0.8 * best && dchi < 1e-5 * tmax) {
                converged = true;
                stagnated = true;
                break;
            }
        }
        // ---- modified Broyden step on dV (history in a ring of nmix pairs)
        const int nmix = c->opt.nmix;
        double2* xprev = c->d_hist_dx[nmix];
        double2* fprev = c->d_hist_df[nmix];
        if (it > 1 && nmix > 0) {
            // new pair: dF = F - F_prev, dX = X - X_prev, both / |dF|
            if (nhist == nmix) {  // drop the oldest
                double2* t0x = c->d_hist_dx[0];
                double2* t0f = c->d_hist_df[0];
                for (int i = 0; i + 1 < nmix; ++i) {
                    c->d_hist_dx[i] = c->d_hist_dx[i + 1];
                    c->d_hist_df[i] = c->d_hist_df[i + 1];
                }
                c->d_hist_dx[nmix - 1] = t0x;
                c->d_hist_df[nmix - 1] = t0f;
                --nhist;
            }
            double2* ndf = c->d_hist_df[nhist];
            double2* ndx = c->d_hist_dx[nhist];
            CK(k_vec_sub(ndf, c->d_dvout, fprev, ndv, c->st));
            CK(k_vec_sub(ndx, c->d_dv, xprev, ndv, c->st));
            const double nn = dev_dot(c, ndf, ndf, ndv, &e);
            if (e != cudaSuccess) return cuda_fail(c, e, "broyden norm");
            if (nn > 0) {
                const double inv = 1.0 / std::sqrt(nn);
                CK(k_vec_scale_copy(ndf, ndf, inv, ndv, c->st));
                CK(k_vec_scale_copy(ndx, ndx, inv, ndv, c->st));
                ++nhist;
            }
        }
        CK(cudaMemcpyAsync(xprev, c->d_dv, sizeof(double2) * ndv, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(fprev, c->d_dvout, sizeof(double2) * ndv, cudaMemcpyDeviceToDevice, c->st));
        const int m = nhist;
        // overlaps <dF_i|dF_j> and <dF_k|F> into d_small[16 + i*(m+1) + j], in one batched launch;
        // pointer table: [0, nmix] dX, [nmix + 1, 2 nmix + 1] dF, from 32 the dot operands
        std::vector<const double2*> ptrs(32 + 2 * kMaxDots, nullptr);
        for (int i = 0; i < m; ++i) {
            ptrs[i] = c->d_hist_dx[i];
            ptrs[nmix + 1 + i] = c->d_hist_df[i];
            for (int j = 0; j <= m; ++j) {
                ptrs[32 + i * (m + 1) + j] = c->d_hist_df[i];
                ptrs[32 + kMaxDots + i * (m + 1) + j] = (j < m) ? c->d_hist_df[j] : c->d_dvout;
            }
        }
        CK(h2d((const double2**)c->d_hist_ptrs, ptrs.data(), ptrs.size(), c->st));
        CK(k_vec_dots((const double2* const*)(c->d_hist_ptrs + 32), (const double2* const*)(c->d_hist_ptrs + 32 + kMaxDots),
                      m * (m + 1), ndv, c->d_small + 16, c->d_partials, c->st));
        CK(k_broyden_coef(c->d_small + 16, m, m + 1, 0.01, c->d_small + 8, c->st));
        CK(k_broyden_apply(c->d_dv, c->d_dvout, (const double2* const*)c->d_hist_ptrs,
                           (const double2* const*)(c->d_hist_ptrs + nmix + 1), c->d_small + 8, m, c->opt.alpha_mix, ndv,
                           c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    if (tc_enabled() && tc_take_error(c->st))
        return fail(c, HP_ETIMEOUT, "hp_response: a tensor-core contraction gave up on a bounded wait");
    RespCols& rc = c->cols[{iq, atom}];
    rc.dn0 = dn0;
    rc.dn = dn;
    rc.tr0 = tr0;
    rc.tr = tr;
    if (dn0_out) memcpy(dn0_out, dn0.data(), sizeof(double) * dn0.size());
    if (dn_out) memcpy(dn_out, dn.data(), sizeof(double) * dn.size());
    if (info) {
        info->iterations = std::min(it, c->opt.niter_max);
        info->cg_iterations = cg_total;
        info->hpsi = hpsi;
        info->residual = res;
        info->dchi = dchi;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->stagnated = stagnated ? 1 : 0;
    }
    if (!converged || !cg_ok) {
        c->cols.erase({iq, atom});
        char msg[200];
        snprintf(msg, sizeof(msg), "hp_response: %s cap reached (residual %.3e, dchi %.3e)",
                 cg_ok ? "self-consistency" : "CG", res, dchi);
        return fail(c, HP_ENOTCONV, msg);
    }
    return HP_OK;
}

// Nearest Hubbard neighbours of another species for the V list: for Hubbard atom s of cell 0, every
// (l', s') of the q-mesh supercell with a minimum-image distance within d_min + dist_thr of the
// shortest one (dist_thr = 6e-4 bohr, the paper's default, Appendix B); (chi index, distance) pairs
struct Neighbour {
    int jchi, j;
    double dist;
    int R[3];
};

static std::vector<Neighbour> nearest_hubbard(const hp_ctx* c, int s) {
    const int nh = (int)c->hub_atoms.size();
    const double n[3] = {(double)c->qmesh[0], (double)c->qmesh[1], (double)c->qmesh[2]};
    const int ia = c->hub_atoms[s];
    std::vector<Neighbour> all;
    for (int l1 = 0, l = 0; l1 < c->qmesh[0]; ++l1)
        for (int l2 = 0; l2 < c->qmesh[1]; ++l2)
            for (int l3 = 0; l3 < c->qmesh[2]; ++l3, ++l) {
                const int R[3] = {l1, l2, l3};
                for (int jj = 0; jj < nh; ++jj) {
                    const int ja = c->hub_atoms[jj];
                    if (c->atom_species[ja] == c->atom_species[ia]) continue;
                    double d[3], x[3] = {0, 0, 0};
                    Neighbour nb{l * nh + jj, jj, 0.0, {0, 0, 0}};
                    for (int i = 0; i < 3; ++i) {
                        d[i] = (c->frac[3 * ja + i] + R[i] - c->frac[3 * ia + i]) / n[i];
                        const double w = std::nearbyint(d[i]);
                        d[i] -= w;
                        nb.R[i] = R[i] - (int)w * c->qmesh[i];  // the neighbour's lattice vector, primitive cells
                    }
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) x[j] += d[i] * n[i] * c->cell[3 * i + j];
                    nb.dist = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                    all.push_back(nb);
                }
            }
    std::vector<Neighbour> out;
    if (all.empty()) return out;
    double dmin = INFINITY;
    for (auto& p : all) dmin = std::min(dmin, p.dist);
    for (auto& p : all)
        if (p.dist <= dmin + 6e-4) out.push_back(p);
    std::sort(out.begin(), out.end(), [](const Neighbour& a, const Neighbour& b) { return a.jchi < b.jchi; });
    return out;
}

// ------------------------------------------------------------------------------------------------
// symmetry reductions: classes of Hubbard atoms, time-reversal q pairs, rebuilt columns
// ------------------------------------------------------------------------------------------------
// index of -q (mod G) in the q mesh
static int minus_q(const hp_ctx* c, int iq) {
    const int n0 = c->qmesh[0], n1 = c->qmesh[1], n2 = c->qmesh[2];
    const int i0 = iq / (n1 * n2), i1 = (iq / n2) % n1, i2 = iq % n2;
    return (((n0 - i0) % n0) * n1 + (n1 - i1) % n1) * n2 + (n2 - i2) % n2;
}

extern "C" hp_status hp_irreducible_q(const hp_ctx* c, int* nirr, int* iq_out, int* partner) {
    if (!c || !nirr || !iq_out) return HP_EINVAL;
    int m = 0;
    for (int iq = 0; iq < c->nq; ++iq) {
        const int p = std::min(iq, minus_q(c, iq));
        if (partner) partner[iq] = p;
        if (p == iq) iq_out[m++] = iq;
    }
    *nirr = m;
    return HP_OK;
}

// separation of Hubbard atom b of cell (l1, l2, l3) from Hubbard atom a of cell 0, in fractional
// coordinates of the q-mesh supercell
static void supercell_separation(const hp_ctx* c, int a, int b, const int R[3], double f[3]) {
    const int ia = c->hub_atoms[a], ja = c->hub_atoms[b];
    for (int i = 0; i < 3; ++i) f[i] = (c->frac[3 * ja + i] + R[i] - c->frac[3 * ia + i]) / c->qmesh[i];
}

// length (bohr) of a supercell fractional vector taken to its minimum image
static double supercell_length(const hp_ctx* c, const double f[3]) {
    double x[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        const double d = f[i] - std::nearbyint(f[i]);
        for (int j = 0; j < 3; ++j) x[j] += d * c->qmesh[i] * c->cell[3 * i + j];
    }
    return std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
}

// The crystal's space group: operations x -> W x + t on fractional coordinates (column vectors), W with
// entries in {-1, 0, 1} and determinant +-1 keeping the lattice metric (W^T G W = G, G = A A^T, the
// lattice vectors the rows of A), t taking every atom onto an atom of its species (1e-5 in fractional
// coordinates), the Hubbard atoms' spin orientations kept up to one global sign.
static std::vector<hp_ctx::SymOp> space_group(const hp_ctx* c, const std::vector<int>& orient) {
    const int nat = (int)c->atom_species.size();
    double G[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            G[3 * i + j] = 0.0;
            for (int k = 0; k < 3; ++k) G[3 * i + j] += c->cell[3 * i + k] * c->cell[3 * j + k];
        }
    double gmax = 0.0;
    for (double g : G) gmax = std::max(gmax, std::fabs(g));
    auto frac_close = [](double d) { return std::fabs(d - std::nearbyint(d)) < 1e-5; };
    std::vector<hp_ctx::SymOp> ops;
    int W[9];
    for (int code = 0; code < 19683; ++code) {  // 3^9 matrices with entries in {-1, 0, 1}
        int r = code;
        for (int i = 0; i < 9; ++i) {
            W[i] = r % 3 - 1;
            r /= 3;
        }
        const int det = W[0] * (W[4] * W[8] - W[5] * W[7]) - W[1] * (W[3] * W[8] - W[5] * W[6]) +
                        W[2] * (W[3] * W[7] - W[4] * W[6]);
        if (det != 1 && det != -1) continue;
        bool metric = true;  // (W^T G W)_ij = sum_kl W_ki G_kl W_lj
        for (int i = 0; i < 3 && metric; ++i)
            for (int j = 0; j < 3 && metric; ++j) {
                double v = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) v += W[3 * k + i] * G[3 * k + l] * W[3 * l + j];
                metric = std::fabs(v - G[3 * i + j]) <= 1e-8 * gmax;
            }
        if (!metric) continue;
        auto image = [&](int a, const double t[3], double y[3]) {
            for (int i = 0; i < 3; ++i) {
                y[i] = t[i];
                for (int k = 0; k < 3; ++k) y[i] += W[3 * i + k] * c->frac[3 * a + k];
            }
        };
        const double zero[3] = {0, 0, 0};
        double y0[3];
        image(0, zero, y0);
        for (int j = 0; j < nat; ++j) {
            if (c->atom_species[j] != c->atom_species[0]) continue;
            hp_ctx::SymOp op;
            for (int i = 0; i < 9; ++i) op.W[i] = W[i];
            for (int i = 0; i < 3; ++i) op.t[i] = c->frac[3 * j + i] - y0[i];
            bool ok = true;
            std::vector<char> used(nat, 0);
            for (int a = 0; a < nat && ok; ++a) {
                double y[3];
                image(a, op.t, y);
                int hit = -1, nhit = 0;
                for (int b = 0; b < nat; ++b)
                    if (c->atom_species[b] == c->atom_species[a] && frac_close(y[0] - c->frac[3 * b]) &&
                        frac_close(y[1] - c->frac[3 * b + 1]) && frac_close(y[2] - c->frac[3 * b + 2])) {
                        hit = b;
                        ++nhit;
                    }
                ok = nhit == 1 && !used[hit];
                if (ok) {
                    used[hit] = 1;
                    op.perm.push_back(hit);
                }
            }
            if (!ok) continue;
            bool spin = false;
            for (int sg = 1; sg >= -1 && !spin; sg -= 2) {
                spin = true;
                for (size_t h = 0; h < c->hub_atoms.size() && spin; ++h) {
                    const int img = op.perm[c->hub_atoms[h]];
                    int hi = -1;
                    for (size_t g = 0; g < c->hub_atoms.size(); ++g)
                        if (c->hub_atoms[g] == img) hi = (int)g;
                    spin = hi >= 0 && orient[hi] == sg * orient[h];
                }
            }
            if (!spin) continue;
            for (int i = 0; i < 3; ++i) op.t[i] -= std::floor(op.t[i]);
            ops.push_back(op);
        }
    }
    return ops;
}

extern "C" hp_status hp_perturbed_atoms(hp_ctx* c, int find_atpert, double docc_thr, double dist_thr, int* npert,
                                        int* atoms, int* rep, double* trace) {
    if (!c) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "hp_perturbed_atoms: no ground state");
    if (find_atpert < 1 || find_atpert > 4 || !(docc_thr > 0) || !(dist_thr >= 0) || !npert || !atoms)
        return fail(c, HP_EINVAL, "hp_perturbed_atoms: find_atpert 1 to 4, docc_thr > 0, dist_thr >= 0, outputs given");
    const int nh = (int)c->hub_atoms.size(), nspin = c->nspin, nk = c->nk, nocc = c->nocc;
    // Tr n^{I s} = (1/N_k) sum_k sum_v sum_m |<phi^I_m,k|u_vk>|^2 (Eq. occ_matrix_0)
    BandList& L = c->L3;
    list_clear(L);
    for (int sp = 0; sp < nspin; ++sp)
        for (int k = 0; k < nk; ++k)
            for (int v = 0; v < nocc; ++v) list_add(L, (sp * nk + k) * c->nbnd + v, k, sp, 0.0);
    hp_status s = upload_list(c, L);
    if (s != HP_OK) return s;
    double2* P;
    CK(dalloc(c, &P, (size_t)L.nb * kPStride));
    ProjMat F{c->d_phi_k, 0, (long long)c->nhub * c->ld, c->nhub, 0, nullptr};
    s = project(c, c->kset, L, F, c->d_psi, P);
    std::vector<double2> h((size_t)L.nb * kPStride);
    if (s == HP_OK) {
        cudaError_t e = d2h(h.data(), P, h.size(), c->st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "hp_perturbed_atoms");
    }
    dfree(c, P);
    if (s != HP_OK) return s;
    std::vector<double> tr((size_t)nh * 2, 0.0);
    for (int b = 0; b < L.nb; ++b)
        for (int a = 0; a < nh; ++a)
            for (int m = 0; m < c->hub_mdim[a]; ++m) {
                const double2 p = h[(size_t)b * kPStride + c->hub_off[a] + m];
                tr[2 * a + L.spin[b]] += (p.x * p.x + p.y * p.y) / nk;
            }
    const double f = nspin == 1 ? 2.0 : 1.0;
    std::vector<int> orient(nh, 0);
    for (int a = 0; a < nh; ++a) {
        const double d = nspin == 2 ? tr[2 * a] - tr[2 * a + 1] : 0.0;
        orient[a] = std::fabs(d) <= docc_thr ? 0 : (d > 0 ? 1 : -1);
    }
    std::vector<hp_ctx::SymOp> ops;
    if (find_atpert == 3) ops = space_group(c, orient);
    std::vector<int> rp(nh);
    for (int a = 0; a < nh; ++a) {
        rp[a] = a;
        if (find_atpert == 4) continue;
        if (find_atpert == 3) {  // the first atom of the orbit (the identity is among the operations)
            for (const auto& op : ops)
                for (int b = 0; b < nh; ++b)
                    if (c->hub_atoms[b] == op.perm[c->hub_atoms[a]]) rp[a] = std::min(rp[a], b);
            continue;
        }
        const double ta = f * (tr[2 * a] + tr[2 * a + 1]);
        for (int b = 0; b < a; ++b) {
            if (rp[b] != b || c->atom_species[c->hub_atoms[b]] != c->atom_species[c->hub_atoms[a]]) continue;
            const double tb = f * (tr[2 * b] + tr[2 * b + 1]);
            if (find_atpert == 2 || std::fabs(ta - tb) < docc_thr) {
                rp[a] = b;
                break;
            }
        }
    }
    int m = 0;
    for (int a = 0; a < nh; ++a) {
        if (rp[a] == a) atoms[m++] = c->hub_atoms[a];
        if (rep) rep[a] = c->hub_atoms[rp[a]];
        if (trace)
            for (int sp = 0; sp < nspin; ++sp) trace[2 * a + sp] = tr[2 * a + sp];
    }
    *npert = m;
    c->hub_rep.clear();
    c->hub_orient.clear();
    c->sym_ops.clear();
    if (find_atpert != 4) {
        c->hub_rep = rp;
        c->hub_orient = orient;
        c->dist_thr = dist_thr;
        if (find_atpert == 3) c->sym_ops = ops;
    }
    return HP_OK;
}

// cell l of the q-mesh supercell as integer coordinates
static void cell_of(const hp_ctx* c, int l, int R[3]) {
    R[0] = l / (c->qmesh[1] * c->qmesh[2]);
    R[1] = (l / c->qmesh[2]) % c->qmesh[1];
    R[2] = l % c->qmesh[2];
}

// the operation keeps the q-mesh supercell's lattice: W diag(n) = diag(n) M with M integer
static bool keeps_supercell(const hp_ctx* c, const hp_ctx::SymOp& op) {
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            if ((op.W[3 * i + k] * c->qmesh[k]) % c->qmesh[i] != 0) return false;
    return true;
}

// inverse of a unimodular integer matrix: the adjugate times the determinant (+-1)
static void int_inverse(const int W[9], int Wi[9]) {
    const int det = W[0] * (W[4] * W[8] - W[5] * W[7]) - W[1] * (W[3] * W[8] - W[5] * W[6]) +
                    W[2] * (W[3] * W[7] - W[4] * W[6]);
    Wi[0] = (W[4] * W[8] - W[5] * W[7]) * det;
    Wi[1] = (W[2] * W[7] - W[1] * W[8]) * det;
    Wi[2] = (W[1] * W[5] - W[2] * W[4]) * det;
    Wi[3] = (W[5] * W[6] - W[3] * W[8]) * det;
    Wi[4] = (W[0] * W[8] - W[2] * W[6]) * det;
    Wi[5] = (W[2] * W[3] - W[0] * W[5]) * det;
    Wi[6] = (W[3] * W[7] - W[4] * W[6]) * det;
    Wi[7] = (W[1] * W[6] - W[0] * W[7]) * det;
    Wi[8] = (W[0] * W[4] - W[1] * W[3]) * det;
}

// q' = W^-T q on the q mesh (q = i / n per axis); returns its index
static int q_image(const hp_ctx* c, const int Wi[9], int iq) {
    int Q[3];
    cell_of(c, iq, Q);
    int out = 0;
    for (int i = 0; i < 3; ++i) {
        double v = 0.0;  // (W^-T q)_i = sum_k (W^-1)_ki q_k
        for (int k = 0; k < 3; ++k) v += Wi[3 * k + i] * (double)Q[k] / c->qmesh[k];
        const int m = (int)std::nearbyint(v * c->qmesh[i]);
        out = out * c->qmesh[i] + ((m % c->qmesh[i]) + c->qmesh[i]) % c->qmesh[i];
    }
    return out;
}

// index of a Hubbard atom (atom index) in hub_atoms
static int hub_index(const hp_ctx* c, int atom) {
    for (size_t h = 0; h < c->hub_atoms.size(); ++h)
        if (c->hub_atoms[h] == atom) return (int)h;
    return -1;
}

// Star of q: from the known (q, J) trace columns of chi0 and chi, every pair reached through the
// operations that keep the supercell, x_{q'}[pi(J)][pi(s)] = exp(2 pi i q'.(L_J - L_s)) x_q[J][s] with
// q' = W^-T q and W x_a + t = x_pi(a) + L_a, and through time reversal, x_{-q}[J] = conj(x_q[J]).
// cols0, cols: [q][J][s]; have: [q][J].
static void fill_star(const hp_ctx* c, std::vector<double2>& cols0, std::vector<double2>& cols,
                      std::vector<char>& have) {
    const int nh = (int)c->hub_atoms.size(), nq = c->nq;
    const double PI2 = 6.28318530717958647692;
    struct Prep {
        int Wi[9];
        std::vector<std::array<int, 3>> L;  // per atom
        std::vector<int> hperm;             // per Hubbard index: the image's Hubbard index
    };
    std::vector<Prep> ops;
    for (const auto& op : c->sym_ops) {
        if (!keeps_supercell(c, op)) continue;
        Prep p;
        int_inverse(op.W, p.Wi);
        const int nat = (int)op.perm.size();
        p.L.resize(nat);
        for (int a = 0; a < nat; ++a)
            for (int i = 0; i < 3; ++i) {
                double v = op.t[i] - c->frac[3 * op.perm[a] + i];
                for (int k = 0; k < 3; ++k) v += op.W[3 * i + k] * c->frac[3 * a + k];
                p.L[a][i] = (int)std::nearbyint(v);
            }
        p.hperm.resize(nh);
        for (int h = 0; h < nh; ++h) p.hperm[h] = hub_index(c, op.perm[c->hub_atoms[h]]);
        ops.push_back(std::move(p));
    }
    std::vector<int> stack;
    for (int i = 0; i < nq * nh; ++i)
        if (have[i]) stack.push_back(i);
    auto put = [&](int iqp, int Jp, const std::vector<double2>& y0, const std::vector<double2>& y) {
        const size_t k = (size_t)iqp * nh + Jp;
        if (have[k]) return;
        have[k] = 1;
        for (int s = 0; s < nh; ++s) {
            cols0[k * nh + s] = y0[s];
            cols[k * nh + s] = y[s];
        }
        stack.push_back((int)k);
    };
    std::vector<double2> y0(nh), y(nh);
    while (!stack.empty()) {
        const int key = stack.back();
        stack.pop_back();
        const int iq = key / nh, J = key % nh;
        const double2* x0 = &cols0[(size_t)key * nh];
        const double2* x = &cols[(size_t)key * nh];
        for (const Prep& p : ops) {
            const int iqp = q_image(c, p.Wi, iq), Jp = p.hperm[J];
            if (Jp < 0 || have[(size_t)iqp * nh + Jp]) continue;
            int Qp[3];
            cell_of(c, iqp, Qp);
            bool ok = true;
            for (int s = 0; s < nh && ok; ++s) {
                const int sp = p.hperm[s];
                ok = sp >= 0;
                if (!ok) break;
                double a = 0.0;
                for (int i = 0; i < 3; ++i)
                    a += (double)Qp[i] / c->qmesh[i] * (p.L[c->hub_atoms[J]][i] - p.L[c->hub_atoms[s]][i]);
                const double cs = std::cos(PI2 * a), sn = std::sin(PI2 * a);
                y0[sp] = cmk(cs * x0[s].x - sn * x0[s].y, cs * x0[s].y + sn * x0[s].x);
                y[sp] = cmk(cs * x[s].x - sn * x[s].y, cs * x[s].y + sn * x[s].x);
            }
            if (ok) put(iqp, Jp, y0, y);
        }
        const int mq = minus_q(c, iq);
        for (int s = 0; s < nh; ++s) {
            y0[s] = cmk(x0[s].x, -x0[s].y);
            y[s] = cmk(x[s].x, -x[s].y);
        }
        put(mq, J, y0, y);
    }
}

extern "C" hp_status hp_irreducible_pairs(const hp_ctx* c, int* npairs, int* iq_out, int* atom_out) {
    if (!c || !npairs || !iq_out || !atom_out) return HP_EINVAL;
    const int nh = (int)c->hub_atoms.size(), nq = c->nq;
    std::vector<int> Wis;
    std::vector<std::vector<int>> hperm;
    for (const auto& op : c->sym_ops) {
        if (!keeps_supercell(c, op)) continue;
        int Wi[9];
        int_inverse(op.W, Wi);
        Wis.insert(Wis.end(), Wi, Wi + 9);
        std::vector<int> hp(nh);
        for (int h = 0; h < nh; ++h) hp[h] = hub_index(c, op.perm[c->hub_atoms[h]]);
        hperm.push_back(hp);
    }
    std::vector<char> seen((size_t)nq * nh, 0);
    int n = 0;
    for (int J = 0; J < nh; ++J) {
        if (!c->hub_rep.empty() && c->hub_rep[J] != J) continue;
        for (int iq = 0; iq < nq; ++iq) {
            if (seen[(size_t)iq * nh + J]) continue;
            iq_out[n] = iq;
            atom_out[n] = c->hub_atoms[J];
            ++n;
            std::vector<int> stack{iq * nh + J};
            seen[(size_t)iq * nh + J] = 1;
            while (!stack.empty()) {
                const int key = stack.back();
                stack.pop_back();
                const int q0 = key / nh, j0 = key % nh;
                std::vector<int> imgs{minus_q(c, q0) * nh + j0};
                for (size_t o = 0; o < hperm.size(); ++o)
                    if (hperm[o][j0] >= 0) imgs.push_back(q_image(c, &Wis[9 * o], q0) * nh + hperm[o][j0]);
                for (int im : imgs)
                    if (!seen[im]) {
                        seen[im] = 1;
                        stack.push_back(im);
                    }
            }
        }
    }
    *npairs = n;
    return HP_OK;
}

// Column (q, J) traces of every q for Hubbard atom jj, rebuilt from its class representative: the
// representative's real-space column chi_{(l,s),(0,J')} = (1/N_q) sum_q exp(2 pi i q.R_l) x_q[s],
// the distance rule, and back to q: x_q[s] = sum_l exp(-2 pi i q.R_l) chi_{(l,s),(0,J)}.
// cols: [q][J][s] complex, the representative's entries filled.
static hp_status rebuild_atom(hp_ctx* c, int jj, std::vector<double2>& cols) {
    const int nh = (int)c->hub_atoms.size(), nq = c->nq;
    const int jr = c->hub_rep[jj];
    const double PI2 = 6.28318530717958647692;
    auto phase = [&](int iq, int l) {
        int Q[3], R[3];
        cell_of(c, iq, Q);
        cell_of(c, l, R);
        double d = 0.0;
        for (int i = 0; i < 3; ++i) d += (double)Q[i] / c->qmesh[i] * R[i];
        return PI2 * d;
    };
    std::vector<double2> rs((size_t)nq * nh, cmk(0.0, 0.0));  // representative, real space [l][s]
    for (int l = 0; l < nq; ++l)
        for (int s = 0; s < nh; ++s) {
            double re = 0.0, im = 0.0;
            for (int iq = 0; iq < nq; ++iq) {
                const double2 x = cols[((size_t)iq * nh + jr) * nh + s];
                const double a = phase(iq, l);
                re += std::cos(a) * x.x - std::sin(a) * x.y;
                im += std::cos(a) * x.y + std::sin(a) * x.x;
            }
            rs[(size_t)l * nh + s] = cmk(re / nq, im / nq);
        }
    std::vector<double2> rj((size_t)nq * nh);
    // find_atpert 3: an operation g of the q-mesh supercell (W diag(n) = diag(n) M, M integer) that
    // takes J' (cell 0) to J in cell L_J gives chi_{a,(0,J)} = chi_{g^-1(a + L_J),(0,J')}
    const hp_ctx::SymOp* use = nullptr;
    for (const auto& op : c->sym_ops)
        if (op.perm[c->hub_atoms[jr]] == c->hub_atoms[jj] && keeps_supercell(c, op)) {
            use = &op;
            break;
        }
    if (use) {
        const int* W = use->W;
        int Wi[9];
        int_inverse(W, Wi);
        const int ir = c->hub_atoms[jr], ij = c->hub_atoms[jj];
        double LJ[3];
        for (int i = 0; i < 3; ++i) {
            double v = use->t[i] - c->frac[3 * ij + i];
            for (int k = 0; k < 3; ++k) v += W[3 * i + k] * c->frac[3 * ir + k];
            LJ[i] = std::nearbyint(v);
        }
        for (int l = 0; l < nq; ++l)
            for (int s = 0; s < nh; ++s) {
                int R[3];
                cell_of(c, l, R);
                const int ia = c->hub_atoms[s];
                double X[3], y[3];
                for (int i = 0; i < 3; ++i) X[i] = c->frac[3 * ia + i] + R[i] + LJ[i] - use->t[i];
                for (int i = 0; i < 3; ++i) y[i] = Wi[3 * i] * X[0] + Wi[3 * i + 1] * X[1] + Wi[3 * i + 2] * X[2];
                int hit = -1;
                for (int sp = 0; sp < nh && hit < 0; ++sp) {
                    const int ib = c->hub_atoms[sp];
                    if (c->atom_species[ib] != c->atom_species[ia]) continue;
                    bool on = true;
                    int cell[3];
                    for (int i = 0; i < 3 && on; ++i) {
                        const double d = y[i] - c->frac[3 * ib + i];
                        cell[i] = (int)std::nearbyint(d);
                        on = std::fabs(d - cell[i]) < 1e-5;
                    }
                    if (!on) continue;
                    int lp = 0;
                    for (int i = 0; i < 3; ++i) lp = lp * c->qmesh[i] + ((cell[i] % c->qmesh[i]) + c->qmesh[i]) % c->qmesh[i];
                    hit = lp * nh + sp;
                }
                if (hit < 0) return fail(c, HP_ESTATE, "hp_hubbard: a symmetry operation does not map a Hubbard atom onto one");
                rj[(size_t)l * nh + s] = rs[hit];
            }
    }
    // otherwise the entry of (l, s) is that of the first (l', s') of the species of s and the
    // orientation of s relative to J whose separation from J' matches: as a vector modulo the supercell
    // (translation images), else as a minimum-image distance
    for (int l = 0; l < nq && !use; ++l)
        for (int s = 0; s < nh; ++s) {
            int R[3];
            cell_of(c, l, R);
            double v[3];
            supercell_separation(c, jj, s, R, v);
            const double d = supercell_length(c, v);
            const int o = c->hub_orient[s] * c->hub_orient[jj];
            int hit = -1;
            for (int pass = 0; pass < 2 && hit < 0; ++pass)
                for (int lp = 0; lp < nq && hit < 0; ++lp) {
                    int Rp[3];
                    cell_of(c, lp, Rp);
                    for (int sp = 0; sp < nh; ++sp) {
                        if (c->atom_species[c->hub_atoms[sp]] != c->atom_species[c->hub_atoms[s]]) continue;
                        if (c->hub_orient[sp] * c->hub_orient[jr] != o) continue;
                        double vp[3];
                        supercell_separation(c, jr, sp, Rp, vp);
                        const double dv[3] = {vp[0] - v[0], vp[1] - v[1], vp[2] - v[2]};
                        const bool match = pass == 0 ? supercell_length(c, dv) <= c->dist_thr
                                                     : std::fabs(supercell_length(c, vp) - d) <= c->dist_thr;
                        if (match) {
                            hit = lp * nh + sp;
                            break;
                        }
                    }
                }
            if (hit < 0) {
                char msg[200];
                snprintf(msg, sizeof(msg), "hp_hubbard: no entry of atom %d's column matches cell %d, atom %d of atom %d's",
                         c->hub_atoms[jr], l, c->hub_atoms[s], c->hub_atoms[jj]);
                return fail(c, HP_ESTATE, msg);
            }
            rj[(size_t)l * nh + s] = rs[hit];
        }
    for (int iq = 0; iq < nq; ++iq)
        for (int s = 0; s < nh; ++s) {
            double re = 0.0, im = 0.0;
            for (int l = 0; l < nq; ++l) {
                const double2 x = rj[(size_t)l * nh + s];
                const double a = -phase(iq, l);
                re += std::cos(a) * x.x - std::sin(a) * x.y;
                im += std::cos(a) * x.y + std::sin(a) * x.x;
            }
            cols[((size_t)iq * nh + jj) * nh + s] = cmk(re, im);
        }
    return HP_OK;
}

extern "C" hp_status hp_hubbard(hp_ctx* c, double* chi0_out, double* chi_out, double* hub_out, double* U_out,
                                hp_pairV* V_out, int* nV) {
    if (!c) return HP_EINVAL;
    if (V_out && !nV) return fail(c, HP_EINVAL, "hp_hubbard: V needs its capacity nV");
    const int nh = (int)c->hub_atoms.size(), nq = c->nq;
    const int n = nh * nq;
    std::vector<double2> cols0((size_t)nq * nh * nh), cols((size_t)nq * nh * nh);
    std::vector<char> have((size_t)nq * nh, 0);
    for (int iq = 0; iq < nq; ++iq)
        for (int jj = 0; jj < nh; ++jj) {
            // with classes kept only the representatives' columns are taken as computed
            if (!c->hub_rep.empty() && c->hub_rep[jj] != jj) continue;
            // the column itself, else the conjugate of (-q, J) (time reversal)
            auto it = c->cols.find({iq, c->hub_atoms[jj]});
            double cj = 1.0;
            if (it == c->cols.end()) {
                it = c->cols.find({minus_q(c, iq), c->hub_atoms[jj]});
                cj = -1.0;
            }
            if (it == c->cols.end()) continue;
            have[(size_t)iq * nh + jj] = 1;
            for (int s = 0; s < nh; ++s) {
                cols0[((size_t)iq * nh + jj) * nh + s] = cmk(it->second.tr0[2 * s], cj * it->second.tr0[2 * s + 1]);
                cols[((size_t)iq * nh + jj) * nh + s] = cmk(it->second.tr[2 * s], cj * it->second.tr[2 * s + 1]);
            }
        }
    auto complete = [&](int jj) {
        for (int iq = 0; iq < nq; ++iq)
            if (!have[(size_t)iq * nh + jj]) return false;
        return true;
    };
    // find_atpert 3: every pair the space group and time reversal reach from the computed ones
    if (!c->sym_ops.empty()) fill_star(c, cols0, cols, have);
    // with classes kept, every atom that does not represent its class (and that the star of q has not
    // completed) takes the rebuilt columns
    for (int jj = 0; jj < nh; ++jj) {
        const bool rebuilt = !c->hub_rep.empty() && c->hub_rep[jj] != jj;
        if (complete(jj)) continue;
        if (!rebuilt || !complete(c->hub_rep[jj])) return fail(c, HP_ESTATE, "hp_hubbard: a (q, J) response is missing");
        hp_status s = rebuild_atom(c, jj, cols0);
        if (s == HP_OK) s = rebuild_atom(c, jj, cols);
        if (s != HP_OK) return s;
    }
    std::vector<double> qf(3 * nq), Rl(3 * nq);
    for (int i1 = 0, i = 0; i1 < c->qmesh[0]; ++i1)
        for (int i2 = 0; i2 < c->qmesh[1]; ++i2)
            for (int i3 = 0; i3 < c->qmesh[2]; ++i3, ++i) {
                qf[3 * i] = (double)i1 / c->qmesh[0];
                qf[3 * i + 1] = (double)i2 / c->qmesh[1];
                qf[3 * i + 2] = (double)i3 / c->qmesh[2];
                Rl[3 * i] = i1;
                Rl[3 * i + 1] = i2;
                Rl[3 * i + 2] = i3;
            }
    double2* d_cols;
    double *d_q, *d_R, *d_mats, *d_work, *d_norms;
    int* d_sing;
    CK(dalloc(c, &d_cols, 2 * cols.size()));
    CK(dalloc(c, &d_q, 3 * nq));
    CK(dalloc(c, &d_R, 3 * nq));
    CK(dalloc(c, &d_mats, (size_t)7 * n * n));
    CK(dalloc(c, &d_work, n));
    CK(dalloc(c, &d_norms, 4));
    CK(dalloc(c, &d_sing, 2));
    CK(h2d(d_cols, cols0.data(), cols0.size(), c->st));
    CK(h2d(d_cols + cols0.size(), cols.data(), cols.size(), c->st));
    CK(h2d(d_q, qf.data(), qf.size(), c->st));
    CK(h2d(d_R, Rl.data(), Rl.size(), c->st));
    double* chi0 = d_mats;
    double* chi0i = d_mats + (size_t)n * n;
    double* chi = d_mats + (size_t)2 * n * n;
    double* chii = d_mats + (size_t)3 * n * n;
    double* inv0 = d_mats + (size_t)4 * n * n;
    double* inv = d_mats + (size_t)5 * n * n;
    double* hub = d_mats + (size_t)6 * n * n;
    CK(k_chi_assemble(d_cols, nq, nh, d_q, d_R, nq, chi0, chi0i, c->st));
    CK(k_chi_assemble(d_cols + cols0.size(), nq, nh, d_q, d_R, nq, chi, chii, c->st));
    CK(cudaMemcpyAsync(inv0, chi0, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(inv, chi, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->st));
    CK(k_invert(inv0, d_work, n, d_sing, c->st));
    CK(k_invert(inv, d_work, n, d_sing + 1, c->st));
    // 1-norm condition numbers ||A||_1 ||A^-1||_1 of chi_0 and chi
    CK(k_norm1(chi0, n, d_norms + 0, c->st));
    CK(k_norm1(inv0, n, d_norms + 1, c->st));
    CK(k_norm1(chi, n, d_norms + 2, c->st));
    CK(k_norm1(inv, n, d_norms + 3, c->st));
    CK(k_hub_matrix(inv0, inv, n, kHaToEv, hub, c->st));
    std::vector<double> h((size_t)7 * n * n);
    int sing[2];
    double nrm[4];
    CK(d2h(h.data(), d_mats, h.size(), c->st));
    CK(d2h(sing, d_sing, 2, c->st));
    CK(d2h(nrm, d_norms, 4, c->st));
    for (void* p : {(void*)d_cols, (void*)d_q, (void*)d_R, (void*)d_mats, (void*)d_work, (void*)d_norms, (void*)d_sing})
        dfree(c, p);
    if (chi0_out) memcpy(chi0_out, h.data(), sizeof(double) * n * n);
    if (chi_out) memcpy(chi_out, h.data() + (size_t)2 * n * n, sizeof(double) * n * n);
    const double cond0 = nrm[0] * nrm[1], cond = nrm[2] * nrm[3];
    if (sing[0] || sing[1] || !(cond0 <= 1e10) || !(cond <= 1e10)) {
        char msg[200];
        snprintf(msg, sizeof(msg), "hp_hubbard: chi0 or chi is singular or ill-conditioned (1-norm condition numbers "
                 "%.3e, %.3e; bound 1e10)", cond0, cond);
        return fail(c, HP_ESINGULAR, msg);
    }
    const double* hubh = h.data() + (size_t)6 * n * n;
    if (hub_out) memcpy(hub_out, hubh, sizeof(double) * n * n);
    if (U_out)
        for (int s = 0; s < nh; ++s) U_out[s] = hubh[(size_t)s * n + s];
    if (V_out || nV) {
        int cnt = 0;
        const int cap = nV ? *nV : 0;
        for (int s = 0; s < nh; ++s)
            for (auto& p : nearest_hubbard(c, s)) {
                if (V_out && cnt < cap)
                    V_out[cnt] = hp_pairV{s, p.jchi, p.dist, hubh[(size_t)s * n + p.jchi], p.j, {p.R[0], p.R[1], p.R[2]}};
                ++cnt;
            }
        if (nV) *nV = cnt;
        if (V_out && cnt > cap) return fail(c, HP_EINVAL, "hp_hubbard: V holds fewer entries than the neighbour pairs");
    }
    return HP_OK;
}

// ------------------------------------------------------------------------------------------------
// several independent cells at once: one host thread per cell, each on its context's stream
// ------------------------------------------------------------------------------------------------
extern "C" hp_status hp_batch_run(int ncells, hp_ctx* const* cells, double* const* chi0, double* const* chi,
                                  double* const* hub, hp_status* status) {
    if (ncells < 1 || !cells || !status) return HP_EINVAL;
    for (int i = 0; i < ncells; ++i) {
        if (!cells[i]) return HP_EINVAL;
        for (int j = 0; j < i; ++j)
            if (cells[j] == cells[i]) return HP_EINVAL;  // a context serves one thread
    }
    auto run = [&](int i) {
        hp_ctx* c = cells[i];
        if (cudaSetDevice(c->device) != cudaSuccess) {
            status[i] = fail(c, HP_ECUDA, "hp_batch_run: cannot select the context's device");
            return;
        }
        hp_status s = HP_OK;
        for (size_t a = 0; a < c->hub_atoms.size() && s == HP_OK; ++a)
            for (int iq = 0; iq < c->nq && s == HP_OK; ++iq) s = hp_response(c, iq, c->hub_atoms[a], nullptr, nullptr, nullptr);
        if (s == HP_OK)
            s = hp_hubbard(c, chi0 ? chi0[i] : nullptr, chi ? chi[i] : nullptr, hub ? hub[i] : nullptr, nullptr, nullptr,
                           nullptr);
        status[i] = s;
    };
    std::vector<std::thread> th;
    th.reserve(ncells);
    for (int i = 0; i < ncells; ++i) th.emplace_back(run, i);
    for (auto& t : th) t.join();
    for (int i = 0; i < ncells; ++i)
        if (status[i] != HP_OK) return status[i];
    return HP_OK;
}
