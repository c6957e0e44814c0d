// Hubbard-corrected ground state (DFT+U+V, Sec. 2.1): occupation matrices (Eq. occ_matrix_0 with
// the generalised projector of Eq. Pm1m2, 1/N_k per cell) and the Hubbard potential of
// Eq. Hub_pot_0 in the basis of the Hubbard rows phi_a,k:
//     V_Hub,s(k) = sum_ab |phi_a,k> W_ks[a][b] <phi_b,k|
//     W[I m1][I m2]  = U^I (delta_m1m2 / 2 - n^{I s}_m1m2)
//     W[i m1][j m2] += -V^{ij} n^{ij(R) s}_m1m2 exp(+2 pi i k.R)       for each listed pair (i, j, R)
// with A_k[a][v] = <phi_a,k|u_vk> and
//     n^{I s}_m1m2       = (1/N_k) sum_k sum_v A[I m1][v] conj(A[I m2][v])
//     n^{ij(R) s}_m1m2   = (1/N_k) sum_k exp(-2 pi i k.R) sum_v A[i m1][v] conj(A[j m2][v]),
// k in crystal coordinates.  The lattice sum of |phi^i_R'><phi^j_R'+R| has the k-space form
// exp(+i k.R) |phi^i_k><phi^j_k|, which gives the phases.  Applying V_Hub is a projection on the
// Hubbard rows, a small per-(spin, k) matrix product and an expansion.
#include <cmath>
#include <cstring>

#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kPS = 128;
constexpr int kMm = 5;  // padded m dimension of the pair matrices
constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ double2 phase(const double* kf, const int* R, double sign) {
    const double a = sign * kTwoPi * (kf[0] * R[0] + kf[1] * R[1] + kf[2] * R[2]);
    double sn, cs;
    sincos(a, &sn, &cs);
    return cmk(cs, sn);
}

// M[s][k][a][b] = sum_v P[(s k v)][a] conj(P[(s k v)][b]); one CTA per (s, k)
__global__ void hub_mk_kernel(const double2* __restrict__ P, int nocc, int nhub, double2* __restrict__ M) {
    const int g = blockIdx.x;
    const double2* Pg = P + (long long)g * nocc * kPS;
    for (int e = threadIdx.x; e < nhub * nhub; e += blockDim.x) {
        const int a = e / nhub, b = e % nhub;
        double2 acc = cmk(0.0, 0.0);
        for (int v = 0; v < nocc; ++v) acc = cadd(acc, cmulc(Pg[(long long)v * kPS + b], Pg[(long long)v * kPS + a]));
        M[(long long)g * nhub * nhub + e] = acc;
    }
}

// occupation vector from M: on-site [s][a][b], then pairs [p][s][m1][m2]
__global__ void hub_occ_kernel(const double2* __restrict__ M, int nspin, int nk, int nhub, int npairs,
                               const int* __restrict__ pint, const int* __restrict__ off, int nh,
                               const double* __restrict__ kfrac, double2* __restrict__ occ) {
    const long long n_on = (long long)nspin * nhub * nhub;
    const long long n_all = n_on + (long long)npairs * nspin * kMm * kMm;
    const double inv = 1.0 / nk;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_all; e += (long long)gridDim.x * blockDim.x) {
        double2 acc = cmk(0.0, 0.0);
        if (e < n_on) {
            const int s = (int)(e / ((long long)nhub * nhub)), ab = (int)(e % ((long long)nhub * nhub));
            for (int k = 0; k < nk; ++k) acc = cadd(acc, M[((long long)s * nk + k) * nhub * nhub + ab]);
        } else {
            const long long r = e - n_on;
            const int p = (int)(r / (nspin * kMm * kMm));
            const int s = (int)(r / (kMm * kMm)) % nspin;
            const int m1 = (int)(r / kMm) % kMm, m2 = (int)(r % kMm);
            const int* q = pint + 5 * p;
            const int i = q[0], j = q[1];
            if (m1 < off[nh + i] && m2 < off[nh + j]) {
                const int a = off[i] + m1, b = off[j] + m2;
                for (int k = 0; k < nk; ++k)
                    acc = cadd(acc, cmul(phase(kfrac + 3 * k, q + 2, -1.0), M[((long long)s * nk + k) * nhub * nhub + a * nhub + b]));
            }
        }
        occ[e] = cscale(acc, inv);
    }
}

// W[s][k][a][b] at nkf k points
__global__ void hub_w_kernel(const double2* __restrict__ occ, int nspin, int nkf, int nhub, int npairs,
                             const int* __restrict__ pint, const double* __restrict__ pV, const double* __restrict__ U,
                             const int* __restrict__ row_atom, const int* __restrict__ off, int nh,
                             const double* __restrict__ kfrac, double2* __restrict__ W) {
    const long long n = (long long)nspin * nkf * nhub * nhub;
    const long long n_on = (long long)nspin * nhub * nhub;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int ab = (int)(e % ((long long)nhub * nhub));
        const int k = (int)((e / ((long long)nhub * nhub)) % nkf);
        const int s = (int)(e / ((long long)nkf * nhub * nhub));
        const int a = ab / nhub, b = ab % nhub;
        const int ia = row_atom[a], ib = row_atom[b];
        double2 w = cmk(0.0, 0.0);
        if (ia == ib) {
            const double2 n_ab = occ[(long long)s * nhub * nhub + ab];
            w = cmk(U[ia] * ((a == b ? 0.5 : 0.0) - n_ab.x), -U[ia] * n_ab.y);
        }
        const int m1 = a - off[ia], m2 = b - off[ib];
        for (int p = 0; p < npairs; ++p) {
            const int* q = pint + 5 * p;
            if (q[0] != ia || q[1] != ib) continue;
            const double2 n = occ[n_on + (((long long)p * nspin + s) * kMm + m1) * kMm + m2];
            w = csub(w, cscale(cmul(n, phase(kfrac + 3 * k, q + 2, +1.0)), pV[p]));
        }
        W[e] = w;
    }
}

// P[c][a] <- sum_b W[s(c)][k(c)][a][b] P[c][b] for the list items, in place (one CTA per item)
__global__ void hub_apply_kernel(double2* __restrict__ P, const double2* __restrict__ W, const int* __restrict__ kk,
                                 const int* __restrict__ spin, const int* __restrict__ kmap, int nkf, int nhub) {
    __shared__ double2 p[kPS];
    const int c = blockIdx.x;
    for (int a = threadIdx.x; a < nhub; a += blockDim.x) p[a] = P[(long long)c * kPS + a];
    __syncthreads();
    const int k = kmap ? kmap[kk[c]] : kk[c];
    const double2* Wc = W + ((long long)spin[c] * nkf + k) * nhub * nhub;
    for (int a = threadIdx.x; a < nhub; a += blockDim.x) {
        double2 acc = cmk(0.0, 0.0);
        for (int b = 0; b < nhub; ++b) acc = cadd(acc, cmul(Wc[(long long)a * nhub + b], p[b]));
        P[(long long)c * kPS + a] = acc;
    }
}

}  // namespace

int hub_occ_len(const hp_ctx* c, int nspin) {
    return nspin * c->nhub * c->nhub + (int)c->hubV.size() * nspin * kMm * kMm;
}

// parameters, the Hubbard-row map and the k mesh on the device (after hp_set_hubbard)
hp_status hub_upload(hp_ctx* c) {
    const int nh = (int)c->hub_atoms.size();
    for (void* p : {(void*)c->d_hubU, (void*)c->d_hub_pair_int, (void*)c->d_hub_pairV, (void*)c->d_hub_row_atom,
                    (void*)c->d_hub_off, (void*)c->d_kfrac})
        dfree(c, p);
    c->d_hubU = nullptr;
    c->d_hub_pair_int = nullptr;
    c->d_hub_pairV = nullptr;
    c->d_hub_row_atom = nullptr;
    c->d_hub_off = nullptr;
    c->d_kfrac = nullptr;
    if (!c->hub_on) return HP_OK;
    const int np = (int)c->hubV.size();
    std::vector<int> pint(5 * std::max(1, np), 0), row_atom(c->nhub), off(2 * nh);
    std::vector<double> pv(std::max(1, np), 0.0), kf(3 * c->nk);
    for (int p = 0; p < np; ++p) {
        const HubPair& q = c->hubV[p];
        pint[5 * p] = q.i;
        pint[5 * p + 1] = q.j;
        for (int d = 0; d < 3; ++d) pint[5 * p + 2 + d] = q.R[d];
        pv[p] = q.V;
    }
    for (int i = 0; i < nh; ++i) {
        off[i] = c->hub_off[i];
        off[nh + i] = c->hub_mdim[i];
        for (int m = 0; m < c->hub_mdim[i]; ++m) row_atom[c->hub_off[i] + m] = i;
    }
    for (int k = 0; k < c->nk; ++k)
        for (int d = 0; d < 3; ++d) kf[3 * k + d] = c->ks[k].kfrac[d];
    CK(dalloc(c, &c->d_hubU, nh));
    CK(dalloc(c, &c->d_hub_pair_int, pint.size()));
    CK(dalloc(c, &c->d_hub_pairV, pv.size()));
    CK(dalloc(c, &c->d_hub_row_atom, c->nhub));
    CK(dalloc(c, &c->d_hub_off, 2 * nh));
    CK(dalloc(c, &c->d_kfrac, kf.size()));
    CK(h2d(c->d_hubU, c->hubU.data(), nh, c->st));
    CK(h2d(c->d_hub_pair_int, pint.data(), pint.size(), c->st));
    CK(h2d(c->d_hub_pairV, pv.data(), pv.size(), c->st));
    CK(h2d(c->d_hub_row_atom, row_atom.data(), c->nhub, c->st));
    CK(h2d(c->d_hub_off, off.data(), off.size(), c->st));
    CK(h2d(c->d_kfrac, kf.data(), kf.size(), c->st));
    CK(cudaStreamSynchronize(c->st));
    return HP_OK;
}

hp_status hub_occupations(hp_ctx* c, const double2* P, int nspin, int nk, int nocc, const double* kfrac_dev,
                          double2* occ) {
    const int nhub = c->nhub, nh = (int)c->hub_atoms.size();
    double2* M;
    CK(dalloc(c, &M, (size_t)nspin * nk * nhub * nhub));
    hub_mk_kernel<<<nspin * nk, 256, 0, c->st>>>(P, nocc, nhub, M);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    const long long n = hub_occ_len(c, nspin);
    hub_occ_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, c->st>>>(
        M, nspin, nk, nhub, (int)c->hubV.size(), c->d_hub_pair_int, c->d_hub_off, nh, kfrac_dev, occ);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    dfree(c, M);
    return HP_OK;
}

hp_status hub_build_w(hp_ctx* c, const double2* occ, int nspin, int nkf, const double* kfrac_dev, double2* W) {
    const long long n = (long long)nspin * nkf * c->nhub * c->nhub;
    hub_w_kernel<<<(int)std::min<long long>((n + 255) / 256, 8192), 256, 0, c->st>>>(
        occ, nspin, nkf, c->nhub, (int)c->hubV.size(), c->d_hub_pair_int, c->d_hub_pairV, c->d_hubU,
        c->d_hub_row_atom, c->d_hub_off, (int)c->hub_atoms.size(), kfrac_dev, W);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    return HP_OK;
}

hp_status hub_apply(hp_ctx* c, const SphereSet& S, const BandList& L, const double2* phi, const int* kmap,
                    const double2* W, const void* X, void* Y, bool vec32, bool fp32, double2* P) {
    if (L.nb == 0) return HP_OK;
    ProjMat F{phi, 0, (long long)c->nhub * c->ld, c->nhub, 0, kmap};
    hp_status s = vec32 ? project(c, S, L, F, (const float2*)X, P, fp32) : project(c, S, L, F, (const double2*)X, P, fp32);
    if (s != HP_OK) return s;
    hub_apply_kernel<<<L.nb, 128, 0, c->st>>>(P, W, L.d_k, L.d_spin, kmap, S.nk, c->nhub);
    HP_LAUNCHED();
    CK(cudaGetLastError());
    if (vec32) CK(k_expand(L, S, F, P, nullptr, 1.0, (float2*)Y, c->ld, c->st, fp32));
    else CK(k_expand(L, S, F, P, nullptr, 1.0, (double2*)Y, c->ld, c->st, fp32));
    return HP_OK;
}

}  // namespace hp

extern "C" hp_status hp_set_hubbard(hp_ctx* c, const double* U, int nV, const hp_pairV* V) {
    using namespace hp;
    if (!c) return HP_EINVAL;
    const int nh = (int)c->hub_atoms.size();
    if (nV < 0 || (nV > 0 && !V)) return fail(c, HP_EINVAL, "hp_set_hubbard: nV < 0 or V missing");
    constexpr double kHaToEv = 27.211386245988;
    std::vector<double> u(nh, 0.0);
    if (U)
        for (int i = 0; i < nh; ++i) u[i] = U[i] / kHaToEv;
    std::vector<HubPair> pairs;
    for (int p = 0; p < nV; ++p) {
        if (V[p].s < 0 || V[p].s >= nh || V[p].j < 0 || V[p].j >= nh)
            return fail(c, HP_EINVAL, "hp_set_hubbard: a pair names a Hubbard atom out of range");
        if (V[p].V == 0.0) continue;
        pairs.push_back(HubPair{V[p].s, V[p].j, {V[p].R[0], V[p].R[1], V[p].R[2]}, V[p].V / kHaToEv});
    }
    bool any = !pairs.empty();
    for (double x : u) any = any || x != 0.0;
    invalidate_response(c);
    c->have_gs = false;
    c->hubU = u;
    c->hubV = pairs;
    c->hub_on = any;
    for (void* p : {(void*)c->d_hub_occ, (void*)c->d_hubW}) dfree(c, p);
    c->d_hub_occ = nullptr;
    c->d_hubW = nullptr;
    for (QFam& F : c->qfam) {
        dfree(c, F.hubW);
        F.hubW = nullptr;
    }
    return hub_upload(c);
}
