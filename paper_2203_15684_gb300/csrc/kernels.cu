// Operator kernels of the FP64 Sternheimer path: sphere <-> grid maps, local potentials, the
// segmented projector contractions (nonlocal beta D beta^H, the valence projector alpha O and P_c,
// Hubbard projections), CG vector updates, response densities, the Hartree and LDA response
// kernels, and the small dense algebra of the mixing and of chi.
#include <cmath>
#include <type_traits>

#include "hp_internal.h"

namespace hp {

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of one double (blockDim.x multiple of 32, <= 1024); result valid in thread 0
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// the same sum, returned to every thread of the block (sh holds at least 33 doubles)
__device__ double block_allsum(double v, double* sh) {
    v = block_sum(v, sh);
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    v = sh[32];
    __syncthreads();
    return v;
}

// ------------------------------------------------------------------------------------------------
// sphere <-> grid
// ------------------------------------------------------------------------------------------------
__global__ void scatter_kernel(const int* __restrict__ npw, const int* __restrict__ idx, int ld,
                               const int* __restrict__ row, const int* __restrict__ kk, int c0,
                               const double2* __restrict__ X, double2* __restrict__ grid, int nr) {
    const int c = c0 + blockIdx.y;
    const int k = kk[c];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G < npw[k]) grid[(long long)blockIdx.y * nr + idx[(long long)k * ld + G]] = X[(long long)row[c] * ld + G];
}

cudaError_t k_scatter(const SphereSet& S, const BandList& L, int c0, int nc, const double2* X, int ldx,
                      double2* grid, int nr, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(grid, 0, sizeof(double2) * (size_t)nc * nr, st);
    if (e != cudaSuccess) return e;
    dim3 g(cdiv(S.ld, 128), nc);
    scatter_kernel<<<g, 128, 0, st>>>(S.d_npw, S.d_idx, S.ld, L.d_row, L.d_k, c0, X, grid, nr);
    HP_LAUNCHED();
    (void)ldx;
    return cudaGetLastError();
}

// Y = grid[idx] / nr + (|k+G|^2/2 - shift) X   (local + kinetic - shift), zero beyond npw
__global__ void gather_h_kernel(const int* __restrict__ npw, const int* __restrict__ idx,
                                const double* __restrict__ g2, int ld, const int* __restrict__ row,
                                const int* __restrict__ kk, const double* __restrict__ shift, int c0,
                                const double2* __restrict__ grid, int nr, const double2* __restrict__ X,
                                double2* __restrict__ Y) {
    const int c = c0 + blockIdx.y;
    const int k = kk[c];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= ld) return;
    const long long o = (long long)row[c] * ld + G;
    if (G < npw[k]) {
        const double inv = 1.0 / (double)nr;
        const double2 v = grid[(long long)blockIdx.y * nr + idx[(long long)k * ld + G]];
        const double d = 0.5 * g2[(long long)k * ld + G] - shift[c];
        const double2 x = X[o];
        Y[o] = cmk(v.x * inv + d * x.x, v.y * inv + d * x.y);
    } else {
        Y[o] = cmk(0.0, 0.0);
    }
}

cudaError_t k_gather_h(const SphereSet& S, const BandList& L, int c0, int nc, const double2* grid, int nr,
                       const double2* X, double2* Y, int ld, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(ld, 128), nc);
    gather_h_kernel<<<g, 128, 0, st>>>(S.d_npw, S.d_idx, S.d_g2, ld, L.d_row, L.d_k, L.d_shift, c0, grid, nr, X, Y);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void gather_scaled_kernel(const int* __restrict__ npw, const int* __restrict__ idx, int ld,
                                     const int* __restrict__ row, const int* __restrict__ kk, int c0,
                                     const double2* __restrict__ grid, int nr, double scale,
                                     double2* __restrict__ Y, int accumulate) {
    const int c = c0 + blockIdx.y;
    const int k = kk[c];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= ld) return;
    const long long o = (long long)row[c] * ld + G;
    double2 v = cmk(0.0, 0.0);
    if (G < npw[k]) v = cscale(grid[(long long)blockIdx.y * nr + idx[(long long)k * ld + G]], scale);
    Y[o] = accumulate ? cadd(Y[o], v) : v;
}

cudaError_t k_gather_scaled(const SphereSet& S, const BandList& L, int c0, int nc, const double2* grid, int nr,
                            double scale, double2* Y, int ld, int accumulate, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(ld, 128), nc);
    gather_scaled_kernel<<<g, 128, 0, st>>>(S.d_npw, S.d_idx, ld, L.d_row, L.d_k, c0, grid, nr, scale, Y, accumulate);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void mul_rpot_kernel(double2* __restrict__ grid, int nr, const double* __restrict__ v,
                                const int* __restrict__ spin, int c0) {
    const int c = blockIdx.y;
    const double* vs = v + (long long)spin[c0 + c] * nr;
    double2* g = grid + (long long)c * nr;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const double s = vs[r];
        const double2 z = g[r];
        g[r] = cmk(z.x * s, z.y * s);
    }
}

cudaError_t k_mul_rpot(double2* grid, int nc, int nr, const double* v, const BandList& L, int c0, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(nr, 256 * 4), nc);
    mul_rpot_kernel<<<g, 256, 0, st>>>(grid, nr, v, L.d_spin, c0);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// grid[c] = v[spin] * src_rows[src_row_of_item[c]]   (complex potential times a cached real-space u)
__global__ void mul_cpot_kernel(double2* __restrict__ grid, const double2* __restrict__ src,
                                const int* __restrict__ src_row, int nr, const double2* __restrict__ v,
                                const int* __restrict__ spin, int c0) {
    const int c = blockIdx.y;
    const double2* vs = v + (long long)spin[c0 + c] * nr;
    const double2* u = src + (long long)src_row[c0 + c] * nr;
    double2* g = grid + (long long)c * nr;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) g[r] = cmul(vs[r], u[r]);
}

cudaError_t k_mul_cpot(double2* grid, const double2* src_rows, const int* src_row_of_item, int nc, int nr,
                       const double2* v, const BandList& L, int c0, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(nr, 256 * 4), nc);
    mul_cpot_kernel<<<g, 256, 0, st>>>(grid, src_rows, src_row_of_item, nr, v, L.d_spin, c0);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// FP32 forms of the grid kernels (mixed precision: FP64 band vectors, FP32 grids and potentials)
// ------------------------------------------------------------------------------------------------
__global__ void scatter32_kernel(const int* __restrict__ npw, const int* __restrict__ idx, int ld,
                                 const int* __restrict__ row, const int* __restrict__ kk, int c0,
                                 const double2* __restrict__ X, float2* __restrict__ grid, int nr) {
    const int c = c0 + blockIdx.y;
    const int k = kk[c];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G < npw[k]) {
        const double2 x = X[(long long)row[c] * ld + G];
        grid[(long long)blockIdx.y * nr + idx[(long long)k * ld + G]] = cmkf((float)x.x, (float)x.y);
    }
}

cudaError_t k_scatter32(const SphereSet& S, const BandList& L, int c0, int nc, const double2* X, float2* grid, int nr,
                        cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)nc * nr, st);
    if (e != cudaSuccess) return e;
    dim3 g(cdiv(S.ld, 128), nc);
    scatter32_kernel<<<g, 128, 0, st>>>(S.d_npw, S.d_idx, S.ld, L.d_row, L.d_k, c0, X, grid, nr);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void mul_rpot32_kernel(float2* __restrict__ grid, int nr, const float* __restrict__ v,
                                  const int* __restrict__ spin, int c0) {
    const int c = blockIdx.y;
    const float* vs = v + (long long)spin[c0 + c] * nr;
    float2* g = grid + (long long)c * nr;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const float s = vs[r];
        const float2 z = g[r];
        g[r] = cmkf(z.x * s, z.y * s);
    }
}

cudaError_t k_mul_rpot32(float2* grid, int nc, int nr, const float* v, const BandList& L, int c0, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(nr, 256 * 4), nc);
    mul_rpot32_kernel<<<g, 256, 0, st>>>(grid, nr, v, L.d_spin, c0);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// Y = grid[idx] / nr + (|k+G|^2/2 - shift) X, the grid part in FP32, the rest in FP64
__global__ void gather_h32_kernel(const int* __restrict__ npw, const int* __restrict__ idx,
                                  const double* __restrict__ g2, int ld, const int* __restrict__ row,
                                  const int* __restrict__ kk, const double* __restrict__ shift, int c0,
                                  const float2* __restrict__ grid, int nr, const double2* __restrict__ X,
                                  double2* __restrict__ Y) {
    const int c = c0 + blockIdx.y;
    const int k = kk[c];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= ld) return;
    const long long o = (long long)row[c] * ld + G;
    if (G < npw[k]) {
        const double inv = 1.0 / (double)nr;
        const float2 v = grid[(long long)blockIdx.y * nr + idx[(long long)k * ld + G]];
        const double d = 0.5 * g2[(long long)k * ld + G] - shift[c];
        const double2 x = X[o];
        Y[o] = cmk((double)v.x * inv + d * x.x, (double)v.y * inv + d * x.y);
    } else {
        Y[o] = cmk(0.0, 0.0);
    }
}

cudaError_t k_gather_h32(const SphereSet& S, const BandList& L, int c0, int nc, const float2* grid, int nr,
                         const double2* X, double2* Y, int ld, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(ld, 128), nc);
    gather_h32_kernel<<<g, 128, 0, st>>>(S.d_npw, S.d_idx, S.d_g2, ld, L.d_row, L.d_k, L.d_shift, c0, grid, nr, X, Y);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void gather_scaled32_kernel(const int* __restrict__ npw, const int* __restrict__ idx, int ld,
                                       const int* __restrict__ row, const int* __restrict__ kk, int c0,
                                       const float2* __restrict__ grid, int nr, double scale, double2* __restrict__ Y) {
    const int c = c0 + blockIdx.y;
    const int k = kk[c];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= ld) return;
    double2 v = cmk(0.0, 0.0);
    if (G < npw[k]) {
        const float2 z = grid[(long long)blockIdx.y * nr + idx[(long long)k * ld + G]];
        v = cmk((double)z.x * scale, (double)z.y * scale);
    }
    Y[(long long)row[c] * ld + G] = v;
}

cudaError_t k_gather_scaled32(const SphereSet& S, const BandList& L, int c0, int nc, const float2* grid, int nr,
                              double scale, double2* Y, int ld, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(ld, 128), nc);
    gather_scaled32_kernel<<<g, 128, 0, st>>>(S.d_npw, S.d_idx, ld, L.d_row, L.d_k, c0, grid, nr, scale, Y);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void mul_cpot32_kernel(float2* __restrict__ grid, const float2* __restrict__ src,
                                  const int* __restrict__ src_row, int nr, const float2* __restrict__ v,
                                  const int* __restrict__ spin, int c0) {
    const int c = blockIdx.y;
    const float2* vs = v + (long long)spin[c0 + c] * nr;
    const float2* u = src + (long long)src_row[c0 + c] * nr;
    float2* g = grid + (long long)c * nr;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) g[r] = cmul(vs[r], u[r]);
}

cudaError_t k_mul_cpot32(float2* grid, const float2* src_rows, const int* src_row_of_item, int nc, int nr,
                         const float2* v, const BandList& L, int c0, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    dim3 g(cdiv(nr, 256 * 4), nc);
    mul_cpot32_kernel<<<g, 256, 0, st>>>(grid, src_rows, src_row_of_item, nr, v, L.d_spin, c0);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// drho[s][r] += weight * sum_c conj(ur[ur_row[c]][r]) xr[c][r]  (FP32 inputs, FP64 accumulation)
__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

cudaError_t k_to_f32(const double* a, float* b, long long n, cudaStream_t st) {
    to_f32_kernel<<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(a, b, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_to_c32(const double2* a, float2* b, long long n, cudaStream_t st) {
    to_f32_kernel<<<std::min(cdiv(2 * n, 256), 4096), 256, 0, st>>>((const double*)a, (float*)b, 2 * n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

cudaError_t k_to_c64(const float2* a, double2* b, long long n, cudaStream_t st) {
    to_f64_kernel<<<std::min(cdiv(2 * n, 256), 4096), 256, 0, st>>>((const float*)a, (double*)b, 2 * n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// segmented projector contractions over one or two projector families (rows 0 .. n0-1 from the
// first, n0 .. n0+n1-1 from the second):
//   proj:   P[c][p]  = sum_G conj(A_seg[p][G]) X[row[c]][G]
//   expand: Y[row[c]][G] += alpha sum_p A_seg[p][G] w_p P[c][p],  w_p = pscale[p] (first family)
//           or scale2 (second family)
// P is indexed by list item c with a row stride of 128.  In the FP32 form the families are read
// from their FP32 copies when present, and FP64 band data is rounded with integer operations.
// ------------------------------------------------------------------------------------------------
constexpr int kPStride = 128;
constexpr int TG = 32;


template <class V>
__device__ __forceinline__ V load_as(const double2& x) {
    if constexpr (sizeof(V) == 8) return cmkf(d2f_bits(x.x), d2f_bits(x.y));
    else return x;
}
template <class V>
__device__ __forceinline__ V load_as(const float2& x) {
    if constexpr (sizeof(V) == 8) return x;
    else return cmk((double)x.x, (double)x.y);
}

template <class V>
__device__ __forceinline__ double2 widen(const V& x) {
    if constexpr (sizeof(V) == 8) return cmk(f2d_bits(x.x), f2d_bits(x.y));
    else return x;
}

// CTA (segment, G split): rows in NPT tiles of 32 (lane = row), bands in tiles of 8 NBI (NBI per
// warp, sized to the largest segment of the list).  G tiles (32 points FP32, 16 FP64) go through
// shared memory with the next tile's global loads issued before the current tile is used; each
// tile is summed in the compute precision, eight tiles in the compute precision, then FP64.
template <class S, class AT, class XT, int NPT, int NBI>
__global__ void __launch_bounds__(256) proj_kernel(ProjDev d, int ld, const XT* __restrict__ X,
                                                   const int* __restrict__ row, const int* __restrict__ seg_start,
                                                   const int* __restrict__ seg_k, const int* __restrict__ seg_s,
                                                   const int* __restrict__ npw_of_k, int ksplit,
                                                   double2* __restrict__ part, int nb) {
    using V = typename std::conditional<std::is_same<S, float>::value, float2, double2>::type;
    constexpr int TP = 32 * NPT;
    constexpr int TGV = sizeof(V) == 16 ? 16 : 32;  // G tile (keeps static shared memory under 48 KB)
    constexpr int TCB = 8 * NBI;                    // bands per tile
    constexpr int RS = 256 / TGV;                   // rows (or bands) advanced per load step
    constexpr int AE = TP / RS;                     // A elements per thread per tile
    constexpr int XE = (TCB + RS - 1) / RS;         // X elements per thread per tile
    __shared__ V As[TGV][TP + 1];
    __shared__ V Xs[TGV][TCB + 1];
    const int seg = blockIdx.x, ks = blockIdx.y;
    const int cbeg = seg_start[seg], cend = seg_start[seg + 1];
    const int k = seg_k[seg], sp = seg_s[seg];
    const int npw = npw_of_k[k];
    const int chunk = ((npw + ksplit - 1) / ksplit + TGV - 1) / TGV * TGV;
    const int g0 = ks * chunk;
    const int g1 = min(npw, g0 + chunk);
    if (g0 >= g1) {
        // empty split: its partial sums are zero
        const int nrow = d.n0 + d.n1;
        for (int e = threadIdx.x; e < (cend - cbeg) * nrow; e += 256)
            part[((long long)ks * nb + cbeg + e / nrow) * kPStride + e % nrow] = cmk(0.0, 0.0);
        return;
    }
    const int mk = d.kmap ? d.kmap[k] : k;
    const int nrow = d.n0 + d.n1;
    const int tid = threadIdx.x;
    const int tp = tid & 31, tc = tid >> 5;  // compute mapping: lane = row, warp = band
    const int lg = tid % TGV, lr = tid / TGV;  // load mapping: G within the tile, first row / band
    const AT* arow[AE];
#pragma unroll
    for (int j = 0; j < AE; ++j) {
        const int p = lr + j * RS;
        arow[j] = p < nrow ? proj_row<AT>(d, sp, mk, p, ld) : nullptr;
    }
    for (int ct = cbeg; ct < cend; ct += TCB) {
        const XT* xrow[XE];
#pragma unroll
        for (int j = 0; j < XE; ++j) {
            const int cc = lr + j * RS;
            xrow[j] = (cc < TCB && ct + cc < cend) ? X + (long long)row[ct + cc] * ld : nullptr;
        }
        V ra[AE], rx[XE];
        auto fetch = [&](int gt) {
            const int G = gt + lg;
#pragma unroll
            for (int j = 0; j < AE; ++j) ra[j] = (arow[j] && G < g1) ? load_as<V>(arow[j][G]) : cpack<V>(0.0, 0.0);
#pragma unroll
            for (int j = 0; j < XE; ++j) rx[j] = (xrow[j] && G < g1) ? load_as<V>(xrow[j][G]) : cpack<V>(0.0, 0.0);
        };
        double2 acc[NPT][NBI];
        V macc[NPT][NBI];
#pragma unroll
        for (int r = 0; r < NPT; ++r)
#pragma unroll
            for (int i = 0; i < NBI; ++i) {
                acc[r][i] = cmk(0.0, 0.0);
                macc[r][i] = cpack<V>(0.0, 0.0);
            }
        int ntile = 0;
        fetch(g0);
        for (int gt = g0; gt < g1; gt += TGV) {
#pragma unroll
            for (int j = 0; j < AE; ++j) As[lg][lr + j * RS] = ra[j];
#pragma unroll
            for (int j = 0; j < XE; ++j)
                if (lr + j * RS < TCB) Xs[lg][lr + j * RS] = rx[j];
            __syncthreads();
            if (gt + TGV < g1) fetch(gt + TGV);  // next tile's loads overlap this tile's arithmetic
            V tacc[NPT][NBI];
#pragma unroll
            for (int r = 0; r < NPT; ++r)
#pragma unroll
                for (int i = 0; i < NBI; ++i) tacc[r][i] = cpack<V>(0.0, 0.0);
#pragma unroll 8
            for (int gg = 0; gg < TGV; ++gg) {
                V x[NBI];
#pragma unroll
                for (int i = 0; i < NBI; ++i) x[i] = Xs[gg][tc + 8 * i];
#pragma unroll
                for (int r = 0; r < NPT; ++r) {
                    const V a = As[gg][tp + 32 * r];
#pragma unroll
                    for (int i = 0; i < NBI; ++i) {
                        tacc[r][i].x += a.x * x[i].x + a.y * x[i].y;
                        tacc[r][i].y += a.x * x[i].y - a.y * x[i].x;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NPT; ++r)
#pragma unroll
                for (int i = 0; i < NBI; ++i) macc[r][i] = cadd(macc[r][i], tacc[r][i]);
            if (++ntile == 8) {
                ntile = 0;
#pragma unroll
                for (int r = 0; r < NPT; ++r)
#pragma unroll
                    for (int i = 0; i < NBI; ++i) {
                        acc[r][i] = cadd(acc[r][i], widen<V>(macc[r][i]));
                        macc[r][i] = cpack<V>(0.0, 0.0);
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < NPT; ++r)
#pragma unroll
            for (int i = 0; i < NBI; ++i) {
                acc[r][i] = cadd(acc[r][i], widen<V>(macc[r][i]));
                const int p = tp + 32 * r;
                const int c = ct + tc + 8 * i;
                if (p < nrow && c < cend) part[((long long)ks * nb + c) * kPStride + p] = acc[r][i];
            }
    }
}

__global__ void proj_reduce_kernel(const double2* __restrict__ part, int ksplit, int nb, int nrow,
                                   double2* __restrict__ P) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nb * nrow) return;
    const int c = (int)(e / nrow), p = (int)(e % nrow);
    double2 s = cmk(0.0, 0.0);
    for (int ks = 0; ks < ksplit; ++ks) s = cadd(s, part[((long long)ks * nb + c) * kPStride + p]);
    P[(long long)c * kPStride + p] = s;
}

static bool fam32(const ProjMat& A) {
    return (A.nrow == 0 || A.base32) && (A.nrow2 == 0 || !A.base2 || A.base2_32);
}

static ProjDev proj_dev(const ProjMat& A, bool use32) {
    ProjDev d;
    d.a0 = use32 ? (const void*)A.base32 : (const void*)A.base;
    d.a1 = use32 ? (const void*)A.base2_32 : (const void*)A.base2;
    d.s0_s = A.stride_s;
    d.s0_k = A.stride_k;
    d.s1_s = A.stride2_s;
    d.s1_k = A.stride2_k;
    d.n0 = A.nrow;
    d.r0 = A.row0;
    d.n1 = A.base2 ? A.nrow2 : 0;
    d.r1 = A.row02;
    d.kmap = A.kmap;
    return d;
}

template <class S, class AT, class XT, int NBI>
static void proj_launch_b(int npt, dim3 g, cudaStream_t st, const ProjDev& d, int ld, const XT* X,
                          const BandList& L, const SphereSet& Sp, int ksplit, double2* scratch) {
    if (npt == 1)
        proj_kernel<S, AT, XT, 1, NBI><<<g, 256, 0, st>>>(d, ld, X, L.d_row, L.d_seg_start, L.d_seg_k, L.d_seg_s,
                                                      Sp.d_npw, ksplit, scratch, L.nb);
    else if (npt == 2)
        proj_kernel<S, AT, XT, 2, NBI><<<g, 256, 0, st>>>(d, ld, X, L.d_row, L.d_seg_start, L.d_seg_k, L.d_seg_s,
                                                      Sp.d_npw, ksplit, scratch, L.nb);
    else
        proj_kernel<S, AT, XT, 4, NBI><<<g, 256, 0, st>>>(d, ld, X, L.d_row, L.d_seg_start, L.d_seg_k, L.d_seg_s,
                                                      Sp.d_npw, ksplit, scratch, L.nb);
}

template <class S, class AT, class XT>
static void proj_launch(int npt, int nbi, dim3 g, cudaStream_t st, const ProjDev& d, int ld, const XT* X,
                        const BandList& L, const SphereSet& Sp, int ksplit, double2* scratch) {
    if (nbi == 1) proj_launch_b<S, AT, XT, 1>(npt, g, st, d, ld, X, L, Sp, ksplit, scratch);
    else if (nbi == 2) proj_launch_b<S, AT, XT, 2>(npt, g, st, d, ld, X, L, Sp, ksplit, scratch);
    else if (nbi == 3) proj_launch_b<S, AT, XT, 3>(npt, g, st, d, ld, X, L, Sp, ksplit, scratch);
    else proj_launch_b<S, AT, XT, 4>(npt, g, st, d, ld, X, L, Sp, ksplit, scratch);
}

// largest number of list items in one (k, spin) segment
static int max_seg(const BandList& L) {
    int m = 0;
    for (int i = 0; i + 1 < (int)L.seg_start.size(); ++i) m = std::max(m, L.seg_start[i + 1] - L.seg_start[i]);
    return L.seg_start.size() < 2 ? L.nb : m;
}

template <class XT>
static cudaError_t proj_t(const BandList& L, const SphereSet& S, const ProjMat& A, const XT* X, int ld, double2* P,
                         double2* scratch, size_t scratch_elems, cudaStream_t st, bool fp32) {
    const int nrow = A.nrow + (A.base2 ? A.nrow2 : 0);
    if (L.nb <= 0 || nrow <= 0) return cudaSuccess;
    if (nrow > kPStride) return cudaErrorInvalidValue;
    // about one wave of 8 resident CTAs per SM, at least two 32-point tiles per split
    int ksplit = std::max(1, cdiv(152 * 8, std::max(1, L.nseg)));
    ksplit = std::min(ksplit, std::max(1, S.ld / (2 * TG)));
    // at most 16 splits, which the callers' scratch holds: the split, and with it the order of the sums,
    // is then fixed by the sizes alone and not by how large the scratch has grown
    ksplit = std::min(ksplit, 16);
    while (ksplit > 1 && (size_t)ksplit * L.nb * kPStride > scratch_elems) --ksplit;
    if ((size_t)ksplit * L.nb * kPStride > scratch_elems) return cudaErrorMemoryAllocation;
    const int npt = nrow <= 32 ? 1 : nrow <= 64 ? 2 : 4;
    const int ms = max_seg(L);
    const int nbi = ms <= 8 ? 1 : ms <= 16 ? 2 : ms <= 24 ? 3 : 4;
    dim3 g(L.nseg, ksplit);
    const bool use32 = fp32 && fam32(A);
    const ProjDev d = proj_dev(A, use32);
    const ProfMark pm = prof_start(st);
    const bool tc = use32 && std::is_same<XT, float2>::value && tc_enabled();
    cudaError_t e = cudaSuccess;
    if (tc) {
        e = tc_proj(d, L, S, reinterpret_cast<const float2*>(X), ld, ksplit, scratch, st);
    } else {
        if (!fp32)
            proj_launch<double, double2, XT>(npt, nbi, g, st, d, ld, X, L, S, ksplit, scratch);
        else if (use32)
            proj_launch<float, float2, XT>(npt, nbi, g, st, d, ld, X, L, S, ksplit, scratch);
        else
            proj_launch<float, double2, XT>(npt, nbi, g, st, d, ld, X, L, S, ksplit, scratch);
        HP_LAUNCHED();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    proj_reduce_kernel<<<cdiv((long long)L.nb * nrow, 256), 256, 0, st>>>(scratch, ksplit, L.nb, nrow, P);
    HP_LAUNCHED();
    if (prof_on() && L.k.size() >= (size_t)L.nb && L.seg_k.size() >= (size_t)L.nseg) {
        // band vectors once, projector rows once per (k, spin) segment, partial sums written and
        // read, results written; 8 flops per complex multiply-add
        const double ab = use32 ? 8.0 : 16.0;
        double bytes = 2.0 * 16.0 * ksplit * L.nb * nrow + 16.0 * L.nb * nrow, flops = 0.0;
        for (int b = 0; b < L.nb; ++b) {
            bytes += (double)sizeof(XT) * S.npw[L.k[b]];
            flops += 8.0 * nrow * S.npw[L.k[b]];
        }
        for (int sg = 0; sg < L.nseg; ++sg) bytes += ab * nrow * S.npw[L.seg_k[sg]];
        prof_stop(pm, HP_KF_PROJECT, st, flops, bytes, "proj");
    }
    return cudaGetLastError();
}

cudaError_t k_proj(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* X, int ld, double2* P,
                   double2* scratch, size_t scratch_elems, cudaStream_t st, bool fp32) {
    return proj_t<double2>(L, S, A, X, ld, P, scratch, scratch_elems, st, fp32);
}

cudaError_t k_proj(const BandList& L, const SphereSet& S, const ProjMat& A, const float2* X, int ld, double2* P,
                   double2* scratch, size_t scratch_elems, cudaStream_t st, bool fp32) {
    return proj_t<float2>(L, S, A, X, ld, P, scratch, scratch_elems, st, fp32);
}

// y += a for a band-vector element of either storage type
__device__ __forceinline__ void acc_into(double2& y, const double2& a) { y = cadd(y, a); }
__device__ __forceinline__ void acc_into(double2& y, const float2& a) { y = cadd(y, widen<float2>(a)); }
__device__ __forceinline__ void acc_into(float2& y, const float2& a) { y = cadd(y, a); }
__device__ __forceinline__ void acc_into(float2& y, const double2& a) { y = cadd(y, cmkf(d2f_bits(a.x), d2f_bits(a.y))); }

// bands per pass kExpC (4 to 24), sized to the largest segment of the list
template <class S, class AT, class YT, int kExpC>
__global__ void __launch_bounds__(128) expand_kernel(ProjDev d, int ld, const double2* __restrict__ P,
                                                     const double* __restrict__ pscale, double alpha, double scale2,
                                                     YT* __restrict__ Y, const int* __restrict__ row,
                                                     const int* __restrict__ seg_start, const int* __restrict__ seg_k,
                                                     const int* __restrict__ seg_s, const int* __restrict__ npw_of_k) {
    using V = typename std::conditional<std::is_same<S, float>::value, float2, double2>::type;
    __shared__ __align__(16) V Ps[kPStride][kExpC];  // [row][band]: two FP32 bands per 16-byte read
    const int seg = blockIdx.y;
    const int cbeg = seg_start[seg], cend = seg_start[seg + 1];
    const int k = seg_k[seg], sp = seg_s[seg];
    const int npw = npw_of_k[k];
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    const int mk = d.kmap ? d.kmap[k] : k;
    const int nrow = d.n0 + d.n1;
    // row p of the first family at G is a0[p * ld], of the second a1[(p - n0) * ld]
    const AT* a0 = (const AT*)d.a0 + sp * d.s0_s + mk * d.s0_k + (long long)d.r0 * ld + G;
    const AT* a1 = d.n1 > 0 ? (const AT*)d.a1 + sp * d.s1_s + mk * d.s1_k + (long long)d.r1 * ld + G : nullptr;
    for (int ct = cbeg; ct < cend; ct += kExpC) {
        for (int e = threadIdx.x; e < kExpC * nrow; e += blockDim.x) {
            const int cc = e / nrow, p = e % nrow;
            const int c = ct + cc;
            double2 v = cmk(0.0, 0.0);
            if (c < cend) {
                const double w = p < d.n0 ? (pscale ? pscale[p] : 1.0) : scale2;
                v = cscale(P[(long long)c * kPStride + p], alpha * w);
            }
            Ps[p][cc] = load_as<V>(v);
        }
        __syncthreads();
        if (G < npw) {
            V acc[kExpC];
#pragma unroll
            for (int i = 0; i < kExpC; ++i) acc[i] = cpack<V>(0.0, 0.0);
            auto mac = [&](const V a, int p) {
                if constexpr (sizeof(V) == 8 && kExpC % 2 == 0) {
                    const float4* q4 = reinterpret_cast<const float4*>(&Ps[p][0]);
#pragma unroll
                    for (int i = 0; i < kExpC / 2; ++i) {
                        const float4 q = q4[i];
                        acc[2 * i].x += a.x * q.x - a.y * q.y;
                        acc[2 * i].y += a.x * q.y + a.y * q.x;
                        acc[2 * i + 1].x += a.x * q.z - a.y * q.w;
                        acc[2 * i + 1].y += a.x * q.w + a.y * q.z;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < kExpC; ++i) {
                        const V q = Ps[p][i];
                        acc[i].x += a.x * q.x - a.y * q.y;
                        acc[i].y += a.x * q.y + a.y * q.x;
                    }
                }
            };
            int p = 0;
            for (; p + 1 < d.n0; p += 2) {  // first family, two rows at a time (both loads in flight)
                const V x0 = load_as<V>(a0[(long long)p * ld]);
                const V x1 = load_as<V>(a0[(long long)(p + 1) * ld]);
                mac(x0, p);
                mac(x1, p + 1);
            }
            for (; p < d.n0; ++p) mac(load_as<V>(a0[(long long)p * ld]), p);
            for (; p + 1 < nrow; p += 2) {
                const V x0 = load_as<V>(a1[(long long)(p - d.n0) * ld]);
                const V x1 = load_as<V>(a1[(long long)(p + 1 - d.n0) * ld]);
                mac(x0, p);
                mac(x1, p + 1);
            }
            for (; p < nrow; ++p) mac(load_as<V>(a1[(long long)(p - d.n0) * ld]), p);
#pragma unroll
            for (int i = 0; i < kExpC; ++i) {
                const int c = ct + i;
                if (c < cend) {
                    const long long o = (long long)row[c] * ld + G;
                    acc_into(Y[o], acc[i]);
                }
            }
        }
        __syncthreads();
    }
}

template <int KC, class YT>
static void expand_launch(bool fp32, bool use32, dim3 g, cudaStream_t st, const ProjDev& d, int ld, const double2* P,
                          const double* pscale, double alpha, double scale2, YT* Y, const BandList& L,
                          const SphereSet& S) {
    if (!fp32)
        expand_kernel<double, double2, YT, KC><<<g, 128, 0, st>>>(d, ld, P, pscale, alpha, scale2, Y, L.d_row,
                                                                  L.d_seg_start, L.d_seg_k, L.d_seg_s, S.d_npw);
    else if (use32)
        expand_kernel<float, float2, YT, KC><<<g, 128, 0, st>>>(d, ld, P, pscale, alpha, scale2, Y, L.d_row,
                                                                L.d_seg_start, L.d_seg_k, L.d_seg_s, S.d_npw);
    else
        expand_kernel<float, double2, YT, KC><<<g, 128, 0, st>>>(d, ld, P, pscale, alpha, scale2, Y, L.d_row,
                                                                 L.d_seg_start, L.d_seg_k, L.d_seg_s, S.d_npw);
}

template <class YT>
static cudaError_t expand_t(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* P,
                           const double* pscale, double alpha, YT* Y, int ld, cudaStream_t st, bool fp32) {
    const int nrow = A.nrow + (A.base2 ? A.nrow2 : 0);
    if (L.nb <= 0 || nrow <= 0) return cudaSuccess;
    if (nrow > kPStride) return cudaErrorInvalidValue;
    dim3 g(cdiv(ld, 128), L.nseg);
    const bool use32 = fp32 && fam32(A);
    const ProjDev d = proj_dev(A, use32);
    const ProfMark pm = prof_start(st);
    const int ms = max_seg(L);
    if (use32 && std::is_same<YT, float2>::value && tc_enabled()) {
        const cudaError_t e = tc_expand(d, L, S, P, pscale, alpha, A.scale2, reinterpret_cast<float2*>(Y), ld, st);
        if (e != cudaSuccess) return e;
    } else {
        if (ms <= 4) expand_launch<4>(fp32, use32, g, st, d, ld, P, pscale, alpha, A.scale2, Y, L, S);
        else if (ms <= 8) expand_launch<8>(fp32, use32, g, st, d, ld, P, pscale, alpha, A.scale2, Y, L, S);
        else if (ms <= 12) expand_launch<12>(fp32, use32, g, st, d, ld, P, pscale, alpha, A.scale2, Y, L, S);
        else if (ms <= 16 || !fp32) expand_launch<16>(fp32, use32, g, st, d, ld, P, pscale, alpha, A.scale2, Y, L, S);
        else if (ms <= 20) expand_launch<20>(fp32, use32, g, st, d, ld, P, pscale, alpha, A.scale2, Y, L, S);
        else expand_launch<24>(fp32, use32, g, st, d, ld, P, pscale, alpha, A.scale2, Y, L, S);
        HP_LAUNCHED();
    }
    if (prof_on() && L.k.size() >= (size_t)L.nb && L.seg_k.size() >= (size_t)L.nseg) {
        // band vectors read and written, coefficients read, projector rows once per segment
        const double ab = use32 ? 8.0 : 16.0;
        double bytes = 16.0 * L.nb * nrow, flops = 0.0;
        for (int b = 0; b < L.nb; ++b) {
            bytes += 2.0 * (double)sizeof(YT) * S.npw[L.k[b]];
            flops += 8.0 * nrow * S.npw[L.k[b]];
        }
        for (int sg = 0; sg < L.nseg; ++sg) bytes += ab * nrow * S.npw[L.seg_k[sg]];
        prof_stop(pm, HP_KF_EXPAND, st, flops, bytes, "expand");
    }
    return cudaGetLastError();
}

cudaError_t k_expand(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* P, const double* pscale,
                     double alpha, double2* Y, int ld, cudaStream_t st, bool fp32) {
    return expand_t<double2>(L, S, A, P, pscale, alpha, Y, ld, st, fp32);
}

cudaError_t k_expand(const BandList& L, const SphereSet& S, const ProjMat& A, const double2* P, const double* pscale,
                     double alpha, float2* Y, int ld, cudaStream_t st, bool fp32) {
    return expand_t<float2>(L, S, A, P, pscale, alpha, Y, ld, st, fp32);
}

// ------------------------------------------------------------------------------------------------
// per-band reductions and CG updates (one CTA per list item, fixed reduction order)
// preconditioner M^-1 = 1 / (1 + |k+G|^2 / 2)
// ------------------------------------------------------------------------------------------------
// Band vectors are FP64 (double2) or, in the mixed form with the fused transforms, FP32 (float2).
// With FP32 vectors the per-thread partial sums are FP32 (a few terms each) and the block sums FP64.
template <class VT>
__device__ __forceinline__ typename Scalar<VT>::type prec_at(const double* p64, const float* p32, long long i);
template <>
__device__ __forceinline__ double prec_at<double2>(const double* p64, const float*, long long i) { return p64[i]; }
template <>
__device__ __forceinline__ float prec_at<float2>(const double*, const float* p32, long long i) { return p32[i]; }

template <class VT>
__global__ void band_dot_kernel(const int* __restrict__ row, const int* __restrict__ kk, const int* __restrict__ npw,
                                const VT* __restrict__ X, const VT* __restrict__ Y, int ld, double* __restrict__ out) {
    using T = typename Scalar<VT>::type;
    __shared__ double sh[32];
    const int c = blockIdx.x;
    const int n = npw[kk[c]];
    const long long o = (long long)row[c] * ld;
    T s = 0;
    for (int G = threadIdx.x; G < n; G += blockDim.x) {
        const VT a = X[o + G], b = Y[o + G];
        s += a.x * b.x + a.y * b.y;
    }
    const double t = block_sum((double)s, sh);
    if (threadIdx.x == 0) out[row[c]] = t;
}

cudaError_t k_band_dot(const BandList& L, const SphereSet& S, const double2* X, const double2* Y, int ld, double* out,
                       cudaStream_t st) {
    if (L.nb <= 0) return cudaSuccess;
    band_dot_kernel<double2><<<L.nb, 256, 0, st>>>(L.d_row, L.d_k, S.d_npw, X, Y, ld, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_band_dot(const BandList& L, const SphereSet& S, const float2* X, const float2* Y, int ld, double* out,
                       cudaStream_t st) {
    if (L.nb <= 0) return cudaSuccess;
    band_dot_kernel<float2><<<L.nb, 256, 0, st>>>(L.d_row, L.d_k, S.d_npw, X, Y, ld, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// p = M r; rz = <r, M r>; rr = <r, r>   (M^-1 = 1 + |k+G|^2 / 2, precomputed per point)
template <class VT>
__global__ void cg_init_kernel(const int* __restrict__ row, const int* __restrict__ kk, const int* __restrict__ npw,
                               const double* __restrict__ prec, const float* __restrict__ prec32,
                               const VT* __restrict__ r, VT* __restrict__ p, int ld, double* __restrict__ rz,
                               double* __restrict__ rr) {
    using T = typename Scalar<VT>::type;
    __shared__ double sh[32];
    const int c = blockIdx.x, k = kk[c];
    const int n = npw[k];
    const long long o = (long long)row[c] * ld;
    T s1 = 0, s2 = 0;
    for (int G = threadIdx.x; G < n; G += blockDim.x) {
        const T m = prec_at<VT>(prec, prec32, (long long)k * ld + G);
        const VT x = r[o + G];
        const T q = x.x * x.x + x.y * x.y;
        p[o + G] = cscale(x, m);
        s1 += m * q;
        s2 += q;
    }
    const double t1 = block_sum((double)s1, sh);
    const double t2 = block_sum((double)s2, sh);
    if (threadIdx.x == 0) {
        rz[row[c]] = t1;
        rr[row[c]] = t2;
    }
}

cudaError_t k_cg_init(const BandList& L, const SphereSet& S, const double2* r, double2* p, int ld, double* rz,
                      double* rr, cudaStream_t st) {
    if (L.nb <= 0) return cudaSuccess;
    cg_init_kernel<double2><<<L.nb, 256, 0, st>>>(L.d_row, L.d_k, S.d_npw, S.d_prec, S.d_prec32, r, p, ld, rz, rr);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_cg_init(const BandList& L, const SphereSet& S, const float2* r, float2* p, int ld, double* rz,
                      double* rr, cudaStream_t st) {
    if (L.nb <= 0) return cudaSuccess;
    cg_init_kernel<float2><<<L.nb, 256, 0, st>>>(L.d_row, L.d_k, S.d_npw, S.d_prec, S.d_prec32, r, p, ld, rz, rr);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// One CG step per band, fused: pAp = <p, Ap>; a = rz / pAp; x += a p; r -= a Ap;
// rz' = <r, M r>, rr = <r, r>; p = M r + (rz' / rz) p.  One CTA per band; with E > 0 the band's p
// and Ap (then r) stay in registers (E elements per thread, npw <= 256 E), with E = 0 they are
// read again.  Reductions in a fixed order; step lengths in FP64.
template <class VT, int E>
__global__ void __launch_bounds__(256) cg_step_kernel(const int* __restrict__ row, const int* __restrict__ kk,
                                                      const int* __restrict__ npw, const double* __restrict__ prec,
                                                      const float* __restrict__ prec32, VT* __restrict__ x,
                                                      VT* __restrict__ r, VT* __restrict__ p,
                                                      const VT* __restrict__ ap, int ld, double* __restrict__ pap,
                                                      double* __restrict__ rz, double* __restrict__ rr) {
    using T = typename Scalar<VT>::type;
    __shared__ double sh[33];
    const int c = blockIdx.x, k = kk[c];
    const int b = row[c];
    const int n = npw[k];
    const long long o = (long long)b * ld;
    const long long mo = (long long)k * ld;
    const double rz0 = rz[b];
    constexpr int EC = E > 0 ? E : 1;
    VT pv[EC], av[EC];
    T s = 0;
    if (E > 0) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const int G = threadIdx.x + 256 * e;
            if (G < n) {
                pv[e] = p[o + G];
                av[e] = ap[o + G];
                s += pv[e].x * av[e].x + pv[e].y * av[e].y;
            }
        }
    } else {
        for (int G = threadIdx.x; G < n; G += 256) {
            const VT a = p[o + G], q = ap[o + G];
            s += a.x * q.x + a.y * q.y;
        }
    }
    const double pAp = block_allsum((double)s, sh);
    const T alpha = (T)(rz0 / pAp);
    T s1 = 0, s2 = 0;
    auto upd = [&](int G, const VT& pg, const VT& ag) {
        VT xv = x[o + G], rv = r[o + G];
        xv.x += alpha * pg.x;
        xv.y += alpha * pg.y;
        rv.x -= alpha * ag.x;
        rv.y -= alpha * ag.y;
        x[o + G] = xv;
        r[o + G] = rv;
        const T q = rv.x * rv.x + rv.y * rv.y;
        s1 += prec_at<VT>(prec, prec32, mo + G) * q;
        s2 += q;
        return rv;
    };
    if (E > 0) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const int G = threadIdx.x + 256 * e;
            if (G < n) av[e] = upd(G, pv[e], av[e]);
        }
    } else {
        for (int G = threadIdx.x; G < n; G += 256) upd(G, p[o + G], ap[o + G]);
    }
    const double t1 = block_allsum((double)s1, sh);
    const double t2 = block_allsum((double)s2, sh);
    const T beta = (T)(t1 / rz0);
    if (E > 0) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const int G = threadIdx.x + 256 * e;
            if (G < n) {
                const T mm = prec_at<VT>(prec, prec32, mo + G);
                VT q;
                q.x = mm * av[e].x + beta * pv[e].x;
                q.y = mm * av[e].y + beta * pv[e].y;
                p[o + G] = q;
            }
        }
    } else {
        for (int G = threadIdx.x; G < n; G += 256) {
            const T mm = prec_at<VT>(prec, prec32, mo + G);
            const VT rv = r[o + G], q0 = p[o + G];
            VT q;
            q.x = mm * rv.x + beta * q0.x;
            q.y = mm * rv.y + beta * q0.y;
            p[o + G] = q;
        }
    }
    if (threadIdx.x == 0) {
        pap[b] = pAp;
        rz[b] = t1;
        rr[b] = t2;
    }
}

template <class VT>
static cudaError_t cg_step_launch(const BandList& L, const SphereSet& S, VT* x, VT* r, VT* p, const VT* ap, int ld,
                                  double* pap, double* rz, double* rr, cudaStream_t st) {
    if (L.nb <= 0) return cudaSuccess;
    int nmax = 0;
    for (int v : S.npw) nmax = std::max(nmax, v);
    const int e = (nmax + 255) / 256;
#define HP_CGS(EE)                                                                                                  \
    cg_step_kernel<VT, EE><<<L.nb, 256, 0, st>>>(L.d_row, L.d_k, S.d_npw, S.d_prec, S.d_prec32, x, r, p, ap, ld, pap, \
                                                 rz, rr)
    if (e <= 3) HP_CGS(3);
    else if (e <= 6) HP_CGS(6);
    else if (e <= 9) HP_CGS(9);
    else if (e <= 12) HP_CGS(12);
    else if (sizeof(VT) == 8 && e <= 18) HP_CGS(18);
    else HP_CGS(0);
#undef HP_CGS
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_cg_step(const BandList& L, const SphereSet& S, double2* x, double2* r, double2* p, const double2* ap,
                      int ld, double* pap, double* rz, double* rr, cudaStream_t st) {
    return cg_step_launch<double2>(L, S, x, r, p, ap, ld, pap, rz, rr, st);
}

cudaError_t k_cg_step(const BandList& L, const SphereSet& S, float2* x, float2* r, float2* p, const float2* ap, int ld,
                      double* pap, double* rz, double* rr, cudaStream_t st) {
    return cg_step_launch<float2>(L, S, x, r, p, ap, ld, pap, rz, rr, st);
}



// ------------------------------------------------------------------------------------------------
// closed-form atomic form factors <k+G|f_lm>:
//   (4 pi / sqrt(Omega)) (-i)^l Y_lm(K) N_R sqrt(pi/2) s^(2l+3) |K|^l exp(-|K|^2 s^2 / 2) exp(-i K.tau)
// with the prefactor (all but the K dependence) computed on the host per row.
// Real harmonics: l=1 (x, y, z); l=2 (xy, yz, 3z^2-r^2, xz, x^2-y^2) in that order.
// ------------------------------------------------------------------------------------------------
__device__ double real_harmonic(int l, int m, double x, double y, double z, double r) {
    const double PI = 3.14159265358979323846;
    if (l == 0) return 0.5 / sqrt(PI);
    if (r <= 0.0) return 0.0;
    const double ir = 1.0 / r;
    x *= ir;
    y *= ir;
    z *= ir;
    if (l == 1) {
        const double c = sqrt(3.0 / (4.0 * PI));
        return c * (m == 0 ? x : (m == 1 ? y : z));
    }
    const double c1 = sqrt(15.0 / (4.0 * PI));
    switch (m) {
        case 0: return c1 * x * y;
        case 1: return c1 * y * z;
        case 2: return sqrt(5.0 / (16.0 * PI)) * (3.0 * z * z - 1.0);
        case 3: return c1 * x * z;
        default: return sqrt(15.0 / (16.0 * PI)) * (x * x - y * y);
    }
}

__global__ void formfactor_kernel(const double* __restrict__ kcart, const int* __restrict__ miller,
                                  const int* __restrict__ npw, int ld, const double* __restrict__ bvec, int nrow,
                                  const int* __restrict__ row_atom, const int* __restrict__ row_l,
                                  const int* __restrict__ row_m, const double* __restrict__ row_width,
                                  const double* __restrict__ row_pref, const double* __restrict__ tau,
                                  double2* __restrict__ out) {
    const int k = blockIdx.z;
    const int rw = blockIdx.y;
    const int G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= ld) return;
    const long long o = ((long long)k * nrow + rw) * ld + G;
    if (G >= npw[k]) {
        out[o] = cmk(0.0, 0.0);
        return;
    }
    const int* m = miller + ((long long)k * ld + G) * 3;
    double K[3];
    for (int i = 0; i < 3; ++i)
        K[i] = kcart[3 * k + i] + m[0] * bvec[0 * 3 + i] + m[1] * bvec[1 * 3 + i] + m[2] * bvec[2 * 3 + i];
    const double g = sqrt(K[0] * K[0] + K[1] * K[1] + K[2] * K[2]);
    const int l = row_l[rw], a = row_atom[rw];
    const double s = row_width[rw];
    const double Y = real_harmonic(l, row_m[rw], K[0], K[1], K[2], g);
    double gl = 1.0;
    for (int i = 0; i < l; ++i) gl *= g;
    const double mag = row_pref[rw] * Y * gl * exp(-0.5 * g * g * s * s);
    const double ph = -(K[0] * tau[3 * a] + K[1] * tau[3 * a + 1] + K[2] * tau[3 * a + 2]);
    double sp, cp;
    sincos(ph, &sp, &cp);
    double2 z = cmk(mag * cp, mag * sp);
    // (-i)^l
    if (l == 1) z = cmk(z.y, -z.x);
    else if (l == 2) z = cmk(-z.x, -z.y);
    out[o] = z;
}

cudaError_t k_formfactor(const double* kcart, int nk, const int* miller, const int* npw, int ld, const double* bvec,
                         int nrow, const int* row_atom, const int* row_l, const int* row_m, const double* row_width,
                         const double* row_pref, const double* tau, double2* out, cudaStream_t st) {
    if (nrow <= 0 || nk <= 0) return cudaSuccess;
    dim3 g(cdiv(ld, 128), nrow, nk);
    formfactor_kernel<<<g, 128, 0, st>>>(kcart, miller, npw, ld, bvec, nrow, row_atom, row_l, row_m, row_width, row_pref,
                                         tau, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// densities
// ------------------------------------------------------------------------------------------------
// drho[s][r] += weight * sum_c conj(ur[ur_row[c]][r]) xr[c][r]   (items of spin s), fixed order
// Delta rho[s][r] += weight * sum_c conj(ur[row(c)][r]) xr[c][r], split over band slices: each CTA
// sums one slice of bands for 256 points (tiles of 16 bands in the compute precision, FP64 across
// tiles) into part[slice][spin][r]; the slices are then added in fixed order.
constexpr int kDrhoTile = 16;

template <class V>
__global__ void __launch_bounds__(256) drho_part_kernel(const V* __restrict__ ur, const int* __restrict__ ur_row,
                                                        const V* __restrict__ xr, int nc, int nr,
                                                        const int* __restrict__ spin, int c0, int slice,
                                                        double2* __restrict__ part) {
    using T = typename Scalar<V>::type;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = blockIdx.y;
    const int cb = sl * slice, ce = min(nc, cb + slice);
    if (r >= nr) return;
    double a0r = 0.0, a0i = 0.0, a1r = 0.0, a1i = 0.0;
    for (int t = cb; t < ce; t += kDrhoTile) {
        const int te = min(ce, t + kDrhoTile);
        T t0r = 0, t0i = 0, t1r = 0, t1i = 0;
#pragma unroll 4
        for (int c = t; c < te; ++c) {
            const V u = ur[(long long)ur_row[c0 + c] * nr + r];
            const V x = xr[(long long)c * nr + r];
            const T tr = u.x * x.x + u.y * x.y;
            const T ti = u.x * x.y - u.y * x.x;
            if (spin[c0 + c] == 0) {
                t0r += tr;
                t0i += ti;
            } else {
                t1r += tr;
                t1i += ti;
            }
        }
        a0r += (double)t0r;
        a0i += (double)t0i;
        a1r += (double)t1r;
        a1i += (double)t1i;
    }
    part[((long long)sl * 2) * nr + r] = cmk(a0r, a0i);
    part[((long long)sl * 2 + 1) * nr + r] = cmk(a1r, a1i);
}

__global__ void drho_reduce_kernel(const double2* __restrict__ part, int nsplit, int nr, int nspin, double weight,
                                   double2* __restrict__ drho, const int* __restrict__ mask) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nspin * nr) return;
    const int s = (int)(e / nr), r = (int)(e % nr);
    double2 acc = cmk(0.0, 0.0);
    for (int sl = 0; sl < nsplit; ++sl)
        if (!mask || ((mask[sl] >> s) & 1)) acc = cadd(acc, part[((long long)sl * 2 + s) * nr + r]);
    drho[e] = cadd(drho[e], cscale(acc, weight));
}

template <class V>
static cudaError_t drho_acc_launch(const V* ur, const int* ur_row, const V* xr, int nc, int nr, const BandList& L,
                                   int c0, double weight, int nspin, double2* drho, double2* part, size_t part_elems,
                                   cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    const int bx = cdiv(nr, 256);
    // about two waves of 8 resident CTAs per SM, slices of at least one tile, partials within the scratch
    int nsplit = std::max(1, std::min(cdiv(2 * 152 * 8, bx), cdiv(nc, kDrhoTile)));
    nsplit = std::min(nsplit, 32);  // what the callers' scratch (64 grids) holds, whatever its current size
    while (nsplit > 1 && (size_t)nsplit * 2 * nr > part_elems) --nsplit;
    if ((size_t)nsplit * 2 * nr > part_elems) return cudaErrorMemoryAllocation;
    const int slice = cdiv(nc, nsplit);
    nsplit = cdiv(nc, slice);
    drho_part_kernel<V><<<dim3(bx, nsplit), 256, 0, st>>>(ur, ur_row, xr, nc, nr, L.d_spin, c0, slice, part);
    HP_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    drho_reduce_kernel<<<cdiv((long long)nspin * nr, 256), 256, 0, st>>>(part, nsplit, nr, nspin, weight, drho,
                                                                          nullptr);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_drho_reduce(const double2* part, int nsplit, int nr, int nspin, double weight, double2* drho,
                          cudaStream_t st, const int* mask) {
    drho_reduce_kernel<<<cdiv((long long)nspin * nr, 256), 256, 0, st>>>(part, nsplit, nr, nspin, weight, drho, mask);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_drho_acc(const double2* ur, const int* ur_row_of_item, const double2* xr, int nc, int nr,
                       const BandList& L, int c0, double weight, int nspin, double2* drho, double2* part,
                       size_t part_elems, cudaStream_t st) {
    return drho_acc_launch<double2>(ur, ur_row_of_item, xr, nc, nr, L, c0, weight, nspin, drho, part, part_elems, st);
}

cudaError_t k_drho_acc32(const float2* ur, const int* ur_row_of_item, const float2* xr, int nc, int nr,
                         const BandList& L, int c0, double weight, int nspin, double2* drho, double2* part,
                         size_t part_elems, cudaStream_t st) {
    return drho_acc_launch<float2>(ur, ur_row_of_item, xr, nc, nr, L, c0, weight, nspin, drho, part, part_elems, st);
}

// rho[s][r] += weight * sum_c |ur[c][r]|^2
__global__ void density_acc_kernel(const double2* __restrict__ ur, int nc, int nr, const int* __restrict__ spin, int c0,
                                   double weight, int nspin, double* __restrict__ rho) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        double a0 = 0.0, a1 = 0.0;
        for (int c = 0; c < nc; ++c) {
            const double2 u = ur[(long long)c * nr + r];
            const double q = u.x * u.x + u.y * u.y;
            if (spin[c0 + c] == 0) a0 += q;
            else a1 += q;
        }
        rho[r] += weight * a0;
        if (nspin == 2) rho[(long long)nr + r] += weight * a1;
    }
}

cudaError_t k_density_acc(const double2* ur, int nc, int nr, const BandList& L, int c0, double weight, int nspin,
                          double* rho, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    density_acc_kernel<<<cdiv(nr, 256), 256, 0, st>>>(ur, nc, nr, L.d_spin, c0, weight, nspin, rho);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// reciprocal-space potentials
// For grid index j_i the representative Miller index m_i satisfies m_i + q_i in (-N_i/2, N_i/2); an
// index without one (the Nyquist plane of an even grid at q_i = 0) and every |q+G|^2 > ecut4 are
// dropped.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool qg_vector(long long flat, const int* N, const double* q, const double* b, double* v) {
    int j[3];
    j[2] = (int)(flat % N[2]);
    j[1] = (int)((flat / N[2]) % N[1]);
    j[0] = (int)(flat / ((long long)N[1] * N[2]));
    double f[3];
    bool ok = true;
    for (int i = 0; i < 3; ++i) {
        double m = (j[i] + q[i] < 0.5 * N[i]) ? (double)j[i] : (double)(j[i] - N[i]);
        const double x = m + q[i];
        if (!(x > -0.5 * N[i] && x < 0.5 * N[i])) ok = false;
        f[i] = x;
    }
    for (int i = 0; i < 3; ++i) v[i] = f[0] * b[0 * 3 + i] + f[1] * b[1 * 3 + i] + f[2] * b[2 * 3 + i];
    return ok;
}

struct Int3 { int v[3]; };
struct Dbl3 { double v[3]; };

__global__ void hartree_q_kernel(double2* __restrict__ rg, Int3 N, const double* __restrict__ bvec, Dbl3 q,
                                 double ecut4, double scale) {
    const long long nr = (long long)N.v[0] * N.v[1] * N.v[2];
    const double FOURPI = 12.566370614359172954;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long long)gridDim.x * blockDim.x) {
        double v[3];
        const bool ok = qg_vector(e, N.v, q.v, bvec, v);
        const double g2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double f = 0.0;
        if (ok && g2 <= ecut4 && g2 > 1e-12) f = scale * FOURPI / g2;
        rg[e] = cscale(rg[e], f);
    }
}

cudaError_t k_hartree_q(double2* rho_g, const int N[3], const double* bvec, const double qfrac[3], double ecut4,
                        double scale, cudaStream_t st) {
    Int3 n = {{N[0], N[1], N[2]}};
    Dbl3 q = {{qfrac[0], qfrac[1], qfrac[2]}};
    const long long nr = (long long)N[0] * N[1] * N[2];
    hartree_q_kernel<<<cdiv(nr, 256), 256, 0, st>>>(rho_g, n, bvec, q, ecut4, scale);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void vloc_g_kernel(double2* __restrict__ vg, Int3 N, const double* __restrict__ bvec, double ecut4, int nat,
                              const double* __restrict__ tau, const double* __restrict__ amp,
                              const double* __restrict__ width, double omega) {
    const long long nr = (long long)N.v[0] * N.v[1] * N.v[2];
    const double PI = 3.14159265358979323846;
    const double zq[3] = {0.0, 0.0, 0.0};
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long long)gridDim.x * blockDim.x) {
        double G[3];
        const bool ok = qg_vector(e, N.v, zq, bvec, G);
        const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        double2 acc = cmk(0.0, 0.0);
        if (ok && g2 <= ecut4) {
            for (int a = 0; a < nat; ++a) {
                const double w = width[a];
                const double mag = amp[a] * pow(2.0 * PI * w * w, 1.5) / omega * exp(-0.5 * g2 * w * w);
                const double ph = -(G[0] * tau[3 * a] + G[1] * tau[3 * a + 1] + G[2] * tau[3 * a + 2]);
                double sp, cp;
                sincos(ph, &sp, &cp);
                acc = cadd(acc, cmk(mag * cp, mag * sp));
            }
        }
        vg[e] = acc;
    }
}

cudaError_t k_vloc_g(double2* vg, const int N[3], const double* bvec, double ecut4, int nat, const double* tau,
                     const double* amp, const double* width, double omega, cudaStream_t st) {
    Int3 n = {{N[0], N[1], N[2]}};
    const long long nr = (long long)N[0] * N[1] * N[2];
    vloc_g_kernel<<<cdiv(nr, 256), 256, 0, st>>>(vg, n, bvec, ecut4, nat, tau, amp, width, omega);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void real_part_kernel(const double2* __restrict__ z, double* __restrict__ out, int n, double scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = z[i].x * scale;
}

cudaError_t k_real_part(const double2* z, double* out, int n, double scale, cudaStream_t st) {
    real_part_kernel<<<cdiv(n, 256), 256, 0, st>>>(z, out, n, scale);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// LDA: Slater exchange + Perdew-Zunger 1981 correlation (parameters from Table XII of that paper),
// spin interpolation f(z) = ((1+z)^(4/3) + (1-z)^(4/3) - 2) / (2^(4/3) - 2).
// eps(rs, z) and its derivatives d/drs, d/dz, d2/drs2, d2/drsdz, d2/dz2; then
// v_s = eps - rs/3 eps_r + (s - z) eps_z and f_ss' = dv_s/drho_s'.
// ------------------------------------------------------------------------------------------------
struct PZ { double g, b1, b2, A, B, C, D; };

__device__ void pz_corr(double rs, const PZ& p, double& e, double& e1, double& e2) {
    if (rs >= 1.0) {
        const double sq = sqrt(rs);
        const double den = 1.0 + p.b1 * sq + p.b2 * rs;
        const double d1 = 0.5 * p.b1 / sq + p.b2;
        const double d2 = -0.25 * p.b1 / (rs * sq);
        e = p.g / den;
        e1 = -p.g * d1 / (den * den);
        e2 = p.g * (2.0 * d1 * d1 - den * d2) / (den * den * den);
    } else {
        const double lr = log(rs);
        e = p.A * lr + p.B + p.C * rs * lr + p.D * rs;
        e1 = p.A / rs + p.C * (lr + 1.0) + p.D;
        e2 = -p.A / (rs * rs) + p.C / rs;
    }
}

struct XcD { double e, er, ez, err, erz, ezz; };

__device__ XcD lda_derivs(double rs, double z) {
    const double PI = 3.14159265358979323846;
    const PZ U = {-0.1423, 1.0529, 0.3334, 0.0311, -0.048, 0.0020, -0.0116};
    const PZ P = {-0.0843, 1.3981, 0.2611, 0.01555, -0.0269, 0.0007, -0.0048};
    const double X0 = -(3.0 / (4.0 * PI)) * cbrt(9.0 * PI / 4.0);
    const double up = 1.0 + z, dn = 1.0 - z;
    const double cu = cbrt(up), cd = cbrt(dn);
    const double phi = 0.5 * (up * cu + dn * cd);                 // ((1+z)^(4/3) + (1-z)^(4/3)) / 2
    const double dphi = (2.0 / 3.0) * (cu - cd);
    const double ddphi = (2.0 / 9.0) * (1.0 / (cu * cu) + 1.0 / (cd * cd));
    const double fden = 2.0 * cbrt(2.0) - 2.0;
    const double f = (up * cu + dn * cd - 2.0) / fden;
    const double df = (4.0 / 3.0) * (cu - cd) / fden;
    const double ddf = (4.0 / 9.0) * (1.0 / (cu * cu) + 1.0 / (cd * cd)) / fden;
    double eU, eU1, eU2, eP, eP1, eP2;
    pz_corr(rs, U, eU, eU1, eU2);
    pz_corr(rs, P, eP, eP1, eP2);
    XcD o;
    const double irs = 1.0 / rs;
    o.e = X0 * irs * phi + eU + f * (eP - eU);
    o.er = -X0 * irs * irs * phi + eU1 + f * (eP1 - eU1);
    o.err = 2.0 * X0 * irs * irs * irs * phi + eU2 + f * (eP2 - eU2);
    o.ez = X0 * irs * dphi + df * (eP - eU);
    o.ezz = X0 * irs * ddphi + ddf * (eP - eU);
    o.erz = -X0 * irs * irs * dphi + df * (eP1 - eU1);
    return o;
}

__global__ void xc_kernel(const double* __restrict__ rho, int nspin, int nr, double* __restrict__ vxc,
                          double* __restrict__ fxc) {
    const double PI = 3.14159265358979323846;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const double ru = nspin == 1 ? 0.5 * rho[r] : rho[r];
        const double rd = nspin == 1 ? 0.5 * rho[r] : rho[nr + r];
        const double n = ru + rd;
        if (!(n >= 1e-10)) {
            for (int s = 0; s < nspin; ++s) vxc[(long long)s * nr + r] = 0.0;
            if (fxc) for (int s = 0; s < (nspin == 1 ? 1 : 3); ++s) fxc[(long long)s * nr + r] = 0.0;
            continue;
        }
        const double rs = cbrt(3.0 / (4.0 * PI * n));
        double z = (ru - rd) / n;
        z = fmin(fmax(z, -1.0 + 1e-14), 1.0 - 1e-14);
        const XcD d = lda_derivs(rs, z);
        const double base = d.e - rs / 3.0 * d.er;
        auto fss = [&](double s1, double s2) {
            const double dvdrs = (2.0 / 3.0) * d.er - rs / 3.0 * d.err + (s1 - z) * d.erz;
            const double dvdz = -rs / 3.0 * d.erz + (s1 - z) * d.ezz;
            return dvdrs * (-rs / (3.0 * n)) + dvdz * (s2 - z) / n;
        };
        if (nspin == 1) {
            vxc[r] = base;  // z = 0
            if (fxc) fxc[r] = 0.5 * (fss(1.0, 1.0) + fss(1.0, -1.0));
        } else {
            vxc[r] = base + (1.0 - z) * d.ez;
            vxc[(long long)nr + r] = base + (-1.0 - z) * d.ez;
            if (fxc) {
                fxc[r] = fss(1.0, 1.0);
                fxc[(long long)nr + r] = fss(1.0, -1.0);
                fxc[2LL * nr + r] = fss(-1.0, -1.0);
            }
        }
    }
}

cudaError_t k_xc(const double* rho, int nspin, int nr, double* vxc, double* fxc, cudaStream_t st) {
    xc_kernel<<<cdiv(nr, 256), 256, 0, st>>>(rho, nspin, nr, vxc, fxc);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// dv[s] = vh + sum_t f_st drho[t]
__global__ void hxc_combine_kernel(const double2* __restrict__ vh, const double2* __restrict__ drho,
                                   const double* __restrict__ fxc, int nspin, int nr, double2* __restrict__ dv) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const double2 h = vh[r];
        if (nspin == 1) {
            dv[r] = cadd(h, cscale(drho[r], fxc[r]));
        } else {
            const double2 a = drho[r], b = drho[(long long)nr + r];
            const double fuu = fxc[r], fud = fxc[(long long)nr + r], fdd = fxc[2LL * nr + r];
            dv[r] = cadd(h, cadd(cscale(a, fuu), cscale(b, fud)));
            dv[(long long)nr + r] = cadd(h, cadd(cscale(a, fud), cscale(b, fdd)));
        }
    }
}

cudaError_t k_hxc_combine(const double2* vh, const double2* drho, const double* fxc, int nspin, int nr, double2* dv,
                          cudaStream_t st) {
    hxc_combine_kernel<<<cdiv(nr, 256), 256, 0, st>>>(vh, drho, fxc, nspin, nr, dv);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// response occupations: M[s][m1][m2] = (1/N_k) sum_k sum_v B[(s,k,v)][m1] conj(Aphi[(s,k,v)][m2])
// B: projections <phi_m1,k+q|Delta u_v>, Aphi: <phi_m2,k|u_v>, both with row stride 128
// ------------------------------------------------------------------------------------------------
__global__ void occ_response_kernel(const double2* __restrict__ B, const double2* __restrict__ Aphi, int nk, int nocc,
                                    int nhub, double2* __restrict__ M) {
    __shared__ double sh[32];
    const int m1 = blockIdx.x, m2 = blockIdx.y, s = blockIdx.z;
    const int nit = nk * nocc;
    double sr = 0.0, si = 0.0;
    for (int i = threadIdx.x; i < nit; i += blockDim.x) {
        const long long item = (long long)s * nit + i;
        const double2 b = B[item * kPStride + m1];
        const double2 a = Aphi[item * kPStride + m2];
        sr += b.x * a.x + b.y * a.y;
        si += b.y * a.x - b.x * a.y;
    }
    sr = block_sum(sr, sh);
    si = block_sum(si, sh);
    if (threadIdx.x == 0) M[((long long)s * nhub + m1) * nhub + m2] = cmk(sr / nk, si / nk);
}

cudaError_t k_occ_response(const double2* B, const double2* Aphi, int ngroups, int nocc, int nhub, int nk, int nspin,
                           double2* M, cudaStream_t st) {
    (void)ngroups;
    dim3 g(nhub, nhub, nspin);
    occ_response_kernel<<<g, 128, 0, st>>>(B, Aphi, nk, nocc, nhub, M);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// dn[a][s][m1][m2] = M[s][o+m1][o+m2] + M[s][o+m2][o+m1]   (Eq. occ_matrix_response_lp_2, both terms)
__global__ void dn_blocks_kernel(const double2* __restrict__ M, int nspin, int nhub, const int* __restrict__ off,
                                 const int* __restrict__ mdim, int mmax, double2* __restrict__ dn) {
    const int a = blockIdx.x;
    const int s = blockIdx.y;
    const int o = off[a], md = mdim[a];
    for (int e = threadIdx.x; e < mmax * mmax; e += blockDim.x) {
        const int m1 = e / mmax, m2 = e % mmax;
        double2 v = cmk(0.0, 0.0);
        if (m1 < md && m2 < md) {
            v = cadd(M[((long long)s * nhub + o + m1) * nhub + o + m2], M[((long long)s * nhub + o + m2) * nhub + o + m1]);
        }
        dn[(((long long)a * nspin + s) * mmax + m1) * mmax + m2] = v;
    }
}

// tr[a] = f sum_s sum_m dn[a][s][m][m]  (spin-summed trace; f = 2 for nspin = 1)
__global__ void dn_traces_kernel(const double2* __restrict__ dn, int nh, int nspin, int mmax, double f,
                                 double2* __restrict__ tr) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nh) return;
    double2 t = cmk(0.0, 0.0);
    for (int s = 0; s < nspin; ++s)
        for (int m = 0; m < mmax; ++m) t = cadd(t, dn[(((long long)a * nspin + s) * mmax + m) * mmax + m]);
    tr[a] = cscale(t, f);
}

cudaError_t k_dn_traces(const double2* dn, int nh, int nspin, int mmax, double f, double2* tr, cudaStream_t st) {
    dn_traces_kernel<<<cdiv(nh, 64), 64, 0, st>>>(dn, nh, nspin, mmax, f, tr);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_dn_blocks(const double2* M, int nspin, int nhub, int nhub_atoms, const int* off, const int* mdim, int mmax,
                        double2* dn, cudaStream_t st) {
    dim3 g(nhub_atoms, nspin);
    dn_blocks_kernel<<<g, 64, 0, st>>>(M, nspin, nhub, off, mdim, mmax, dn);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// long-vector algebra for the mixing (deterministic two-stage reductions)
// ------------------------------------------------------------------------------------------------
constexpr int kRedBlocks = 256;

__global__ void vec_dot_kernel(const double2* __restrict__ a, const double2* __restrict__ b, long long n,
                               double* __restrict__ partial) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 x = a[i], y = b[i];
        s += x.x * y.x + x.y * y.y;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void sum_reduce_kernel(const double* __restrict__ partial, int nparts, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

cudaError_t k_vec_dot(const double2* a, const double2* b, long long n, double* out, double* partial, cudaStream_t st) {
    vec_dot_kernel<<<kRedBlocks, 256, 0, st>>>(a, b, n, partial);
    HP_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_reduce_kernel<<<1, 256, 0, st>>>(partial, kRedBlocks, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// npairs dot products Re<A_p|B_p> at once, each with the partition and reduction order of k_vec_dot
// (so each result equals k_vec_dot's bit for bit): block (b, p) sums the slice b of pair p.
__global__ void vec_dots_kernel(const double2* const* __restrict__ A, const double2* const* __restrict__ B, long long n,
                                double* __restrict__ partial) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    const double2* __restrict__ a = A[p];
    const double2* __restrict__ b = B[p];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 x = a[i], y = b[i];
        s += x.x * y.x + x.y * y.y;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(long long)p * gridDim.x + blockIdx.x] = s;
}

__global__ void sums_reduce_kernel(const double* __restrict__ partial, int nparts, double* __restrict__ out) {
    __shared__ double sh[32];
    const double* part = partial + (long long)blockIdx.x * nparts;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

cudaError_t k_vec_dots(const double2* const* A, const double2* const* B, int npairs, long long n, double* out,
                       double* partials, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    vec_dots_kernel<<<dim3(kRedBlocks, npairs), 256, 0, st>>>(A, B, n, partials);
    HP_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sums_reduce_kernel<<<npairs, 256, 0, st>>>(partials, kRedBlocks, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_sum_reduce(const double* partial, int nparts, double* out, cudaStream_t st) {
    sum_reduce_kernel<<<1, 256, 0, st>>>(partial, nparts, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

template <class VT>
__global__ void vec_axpy_kernel(VT* __restrict__ y, const VT* __restrict__ x, typename Scalar<VT>::type a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        VT v = y[i];
        v.x += a * x[i].x;
        v.y += a * x[i].y;
        y[i] = v;
    }
}

template <class VT>
__global__ void vec_sub_kernel(VT* __restrict__ out, const VT* __restrict__ a, const VT* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = csub(a[i], b[i]);
}

template <class VT>
__global__ void vec_scale_copy_kernel(VT* __restrict__ out, const VT* __restrict__ a, typename Scalar<VT>::type s,
                                      long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = cscale(a[i], s);
}

cudaError_t k_vec_axpy(double2* y, const double2* x, double a, long long n, cudaStream_t st) {
    vec_axpy_kernel<double2><<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(y, x, a, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_vec_axpy(float2* y, const float2* x, double a, long long n, cudaStream_t st) {
    vec_axpy_kernel<float2><<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(y, x, (float)a, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_vec_sub(double2* out, const double2* a, const double2* b, long long n, cudaStream_t st) {
    vec_sub_kernel<double2><<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(out, a, b, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_vec_sub(float2* out, const float2* a, const float2* b, long long n, cudaStream_t st) {
    vec_sub_kernel<float2><<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(out, a, b, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_vec_scale_copy(double2* out, const double2* a, double s, long long n, cudaStream_t st) {
    vec_scale_copy_kernel<double2><<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(out, a, s, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_vec_scale_copy(float2* out, const float2* a, double s, long long n, cudaStream_t st) {
    vec_scale_copy_kernel<float2><<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(out, a, (float)s, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// Johnson's modified Broyden coefficients: dots = [m x m overlaps <dF_i|dF_j> | m projections
// <dF_k|F>] (row stride ld); a = w0^2 I + overlaps; gamma = c^T a^-1 (Gauss-Jordan, m <= 8).
__global__ void broyden_coef_kernel(const double* __restrict__ dots, int m, int ld, double w0, double* __restrict__ gamma) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[8][9];
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) a[i][j] = dots[i * ld + j] + (i == j ? w0 * w0 : 0.0);
        a[i][m] = dots[i * ld + m];  // c_i ; a symmetric, so gamma = a^-1 c
    }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int i = col + 1; i < m; ++i)
            if (fabs(a[i][col]) > fabs(a[piv][col])) piv = i;
        if (piv != col)
            for (int j = 0; j <= m; ++j) {
                const double t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        const double d = a[col][col];
        for (int j = col; j <= m; ++j) a[col][j] /= d;
        for (int i = 0; i < m; ++i) {
            if (i == col) continue;
            const double f = a[i][col];
            for (int j = col; j <= m; ++j) a[i][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < m; ++i) gamma[i] = a[i][m];
}

cudaError_t k_broyden_coef(const double* dots, int m, int ld, double w0, double* gamma, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (m > 8) return cudaErrorInvalidValue;
    broyden_coef_kernel<<<1, 32, 0, st>>>(dots, m, ld, w0, gamma);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// x += alpha f - sum_l gamma_l (dx_l + alpha df_l)
__global__ void broyden_apply_kernel(double2* __restrict__ x, const double2* __restrict__ f,
                                     const double2* const* __restrict__ dx, const double2* const* __restrict__ df,
                                     const double* __restrict__ gamma, int m, double alpha, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 v = cadd(x[i], cscale(f[i], alpha));
        for (int l = 0; l < m; ++l) {
            const double2 t = cadd(dx[l][i], cscale(df[l][i], alpha));
            v = csub(v, cscale(t, gamma[l]));
        }
        x[i] = v;
    }
}

cudaError_t k_broyden_apply(double2* x, const double2* f, const double2* const* dx, const double2* const* df,
                            const double* gamma, int m, double alpha, long long n, cudaStream_t st) {
    broyden_apply_kernel<<<std::min(cdiv(n, 256), 4096), 256, 0, st>>>(x, f, dx, df, gamma, m, alpha, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// chi assembly (Eq. occ_matrix_response_lp_1) and FP64 inversion
//   chi[(l,s)][(l',s')] = (1/N_q) sum_q exp(2 pi i q.(R_l - R_l')) col[q][s'][s]
// cols: [nq][nh (perturbed s')][nh (responding s)] complex
// ------------------------------------------------------------------------------------------------
__global__ void chi_assemble_kernel(const double2* __restrict__ cols, int nq, int nh, const double* __restrict__ qfrac,
                                    const double* __restrict__ Rl, int ncell, double* __restrict__ chi_re,
                                    double* __restrict__ chi_im) {
    const int n = ncell * nh;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int I = e / n, J = e % n;
    const int l = I / nh, s = I % nh, lp = J / nh, sp = J % nh;
    const double PI2 = 6.28318530717958647692;
    double re = 0.0, im = 0.0;
    for (int iq = 0; iq < nq; ++iq) {
        const double d = qfrac[3 * iq] * (Rl[3 * l] - Rl[3 * lp]) + qfrac[3 * iq + 1] * (Rl[3 * l + 1] - Rl[3 * lp + 1]) +
                         qfrac[3 * iq + 2] * (Rl[3 * l + 2] - Rl[3 * lp + 2]);
        double sp_, cp;
        sincos(PI2 * d, &sp_, &cp);
        const double2 c = cols[((long long)iq * nh + sp) * nh + s];
        re += cp * c.x - sp_ * c.y;
        im += cp * c.y + sp_ * c.x;
    }
    chi_re[e] = re / nq;
    chi_im[e] = im / nq;
}

cudaError_t k_chi_assemble(const double2* cols, int nq, int nh, const double* qfrac, const double* Rl, int ncell,
                           double* chi_re, double* chi_im, cudaStream_t st) {
    const int n = ncell * nh;
    chi_assemble_kernel<<<cdiv((long long)n * n, 128), 128, 0, st>>>(cols, nq, nh, qfrac, Rl, ncell, chi_re, chi_im);
    HP_LAUNCHED();
    return cudaGetLastError();
}

// in-place Gauss-Jordan inverse with partial pivoting, one CTA (n <= 512); work: n doubles
__global__ void invert_kernel(double* __restrict__ a, double* __restrict__ work, int n, int* __restrict__ singular) {
    __shared__ int piv_s;
    __shared__ double pv_s;
    extern __shared__ int perm[];
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
    if (threadIdx.x == 0) *singular = 0;
    __syncthreads();
    double amax = 0.0;
    for (int col = 0; col < n; ++col) {
        if (threadIdx.x == 0) {
            int p = col;
            double best = fabs(a[(long long)col * n + col]);
            for (int i = col + 1; i < n; ++i) {
                const double v = fabs(a[(long long)i * n + col]);
                if (v > best) { best = v; p = i; }
            }
            piv_s = p;
            if (col == 0) amax = best;
            if (best <= 1e-300) *singular = 1;
        }
        __syncthreads();
        const int p = piv_s;
        if (p != col) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const double t = a[(long long)col * n + j];
                a[(long long)col * n + j] = a[(long long)p * n + j];
                a[(long long)p * n + j] = t;
            }
            if (threadIdx.x == 0) {
                const int t = perm[col];
                perm[col] = perm[p];
                perm[p] = t;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) pv_s = a[(long long)col * n + col];
        __syncthreads();
        const double pv = pv_s;
        // scale the pivot row (the pivot element becomes 1/pv)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            if (j == col) continue;
            a[(long long)col * n + j] /= pv;
        }
        __syncthreads();
        if (threadIdx.x == 0) a[(long long)col * n + col] = 1.0 / pv;
        for (int i = threadIdx.x; i < n; i += blockDim.x) work[i] = (i == col) ? 0.0 : a[(long long)i * n + col];
        __syncthreads();
        // eliminate
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
            const int i = (int)(e / n), j = (int)(e % n);
            if (i == col) continue;
            const double f = work[i];
            if (j == col) a[e] = -f * a[(long long)col * n + col];
            else a[e] -= f * a[(long long)col * n + j];
        }
        __syncthreads();
    }
    (void)amax;
    // undo the row permutation: the sweep inverted P A, and A^-1 = (P A)^-1 P
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) work[j] = a[(long long)i * n + j];
            for (int j = 0; j < n; ++j) a[(long long)i * n + perm[j]] = work[j];
        }
    }
}

cudaError_t k_invert(double* a, double* work, int n, int* singular, cudaStream_t st) {
    invert_kernel<<<1, 256, sizeof(int) * n, st>>>(a, work, n, singular);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void hub_matrix_kernel(const double* __restrict__ inv0, const double* __restrict__ inv, int n, double scale,
                                  double* __restrict__ hub) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * n) hub[e] = (inv0[e] - inv[e]) * scale;
}

cudaError_t k_hub_matrix(const double* inv0, const double* inv, int n, double scale, double* hub, cudaStream_t st) {
    hub_matrix_kernel<<<cdiv((long long)n * n, 128), 128, 0, st>>>(inv0, inv, n, scale, hub);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void norm1_kernel(const double* __restrict__ a, int n, double* __restrict__ out) {
    __shared__ double red[256];
    double best = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double col = 0.0;
        for (int i = 0; i < n; ++i) col += fabs(a[(long long)i * n + j]);
        best = fmax(best, col);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t k_norm1(const double* a, int n, double* out, cudaStream_t st) {
    norm1_kernel<<<1, 256, 0, st>>>(a, n, out);
    HP_LAUNCHED();
    return cudaGetLastError();
}

__global__ void add_real_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}

cudaError_t k_add_real(const double* a, const double* b, double* out, int n, cudaStream_t st) {
    add_real_kernel<<<cdiv(n, 256), 256, 0, st>>>(a, b, out, n);
    HP_LAUNCHED();
    return cudaGetLastError();
}

}  // namespace hp

namespace {
__global__ void convert_selftest_kernel(const double* __restrict__ in, long long n, float* __restrict__ f,
                                        double* __restrict__ back, float* __restrict__ f_ref,
                                        double* __restrict__ back_ref) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float a = hp::d2f_bits(in[i]);
        f[i] = a;
        back[i] = hp::f2d_bits(a);
        const float r = __double2float_rn(in[i]);
        f_ref[i] = r;
        back_ref[i] = (double)r;
    }
}
}  // namespace

extern "C" hp_status hp_selftest_xc(int n, int nspin, const double* rho, double* vxc, double* fxc) {
    if (n < 1 || (nspin != 1 && nspin != 2) || !rho || !vxc || !fxc) return HP_EINVAL;
    const int nf = nspin == 1 ? 1 : 3;
    double *d_rho = nullptr, *d_v = nullptr, *d_f = nullptr;
    cudaError_t e = cudaMalloc(&d_rho, sizeof(double) * (size_t)nspin * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_v, sizeof(double) * (size_t)nspin * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_f, sizeof(double) * (size_t)nf * n);
    if (e == cudaSuccess) hp::g_allocs.fetch_add(3, std::memory_order_relaxed);
    if (e == cudaSuccess) e = cudaMemcpy(d_rho, rho, sizeof(double) * (size_t)nspin * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = hp::k_xc(d_rho, nspin, n, d_v, d_f, 0);
    if (e == cudaSuccess) e = cudaMemcpy(vxc, d_v, sizeof(double) * (size_t)nspin * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fxc, d_f, sizeof(double) * (size_t)nf * n, cudaMemcpyDeviceToHost);
    cudaFree(d_rho);
    cudaFree(d_v);
    cudaFree(d_f);
    return e == cudaSuccess ? HP_OK : HP_ECUDA;
}

extern "C" hp_status hp_selftest_convert(long long n, const double* in, float* f, double* back, float* f_ref,
                                         double* back_ref) {
    if (n < 1 || !in || !f || !back || !f_ref || !back_ref) return HP_EINVAL;
    double *d_in = nullptr, *d_back = nullptr, *d_back_ref = nullptr;
    float *d_f = nullptr, *d_f_ref = nullptr;
    const size_t n8 = sizeof(double) * (size_t)n, n4 = sizeof(float) * (size_t)n;
    cudaError_t e = cudaMalloc(&d_in, n8);
    if (e == cudaSuccess) e = cudaMalloc(&d_back, n8);
    if (e == cudaSuccess) e = cudaMalloc(&d_back_ref, n8);
    if (e == cudaSuccess) e = cudaMalloc(&d_f, n4);
    if (e == cudaSuccess) e = cudaMalloc(&d_f_ref, n4);
    if (e == cudaSuccess) hp::g_allocs.fetch_add(5, std::memory_order_relaxed);
    if (e == cudaSuccess) e = cudaMemcpy(d_in, in, n8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        convert_selftest_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256>>>(d_in, n, d_f, d_back, d_f_ref,
                                                                                       d_back_ref);
        hp::g_launches.fetch_add(1, std::memory_order_relaxed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(f, d_f, n4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(back, d_back, n8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(f_ref, d_f_ref, n4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(back_ref, d_back_ref, n8, cudaMemcpyDeviceToHost);
    cudaFree(d_in);
    cudaFree(d_back);
    cudaFree(d_back_ref);
    cudaFree(d_f);
    cudaFree(d_f_ref);
    return e == cudaSuccess ? HP_OK : HP_ECUDA;
}
