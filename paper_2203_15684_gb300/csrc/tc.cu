// Tensor-core (tcgen05, kind::tf32 with a three-product TF32 split) contractions of the response: the
// projections <beta|psi>, <u_v|psi> and the expansions psi += beta P of the Sternheimer operator and
// the right-hand side (Sec. 2.3: the nonlocal term of H_k+q and the projectors of Eqs. proj_v and
// proj_c), and the self-test of the MMA building block.  The building blocks are in tc.cuh.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "hp_internal.h"
#include "tc.cuh"

namespace hp {
namespace {

constexpr int kSelfKF = 32;  // FP32 values along K per staged tile

// D[m][n] = sum_k A[m][k] B[n][k] for m < M <= 128, n < N (N a multiple of 16, <= 128), K a multiple
// of 32, one CTA: tiles staged by the threads (TF32 split on the way), MMAs issued by thread 0,
// completion on an mbarrier, D read back from TMEM with 32x32b loads (warp w holds rows 32w..32w+31).
// lbo_swap = 1 exchanges the descriptor's LBO and SBO fields (the data layout stays the same), so
// that a test can tell the two readings of the descriptor apart; every address stays in the tiles.
// mode bits: 1 = exchange LBO and SBO; 2 = add the fourth product a_lo b_lo; 4 = drain the TMEM
// accumulator into FP64 registers after every staged chunk (the accumulator then restarts)
__global__ void __launch_bounds__(128) tc_selftest_kernel(const float* __restrict__ A, int M, const float* __restrict__ B,
                                                          int N, int K, float* __restrict__ D, int mode,
                                                          unsigned long long timeout_ns, int* __restrict__ err) {
    const int lbo_swap = mode & 1;
    const bool four = (mode & 2) != 0, drain = (mode & 4) != 0;
    double acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.0;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    constexpr int KF = kSelfKF;
    constexpr uint32_t kTile = 128 * KF * 4;
    unsigned char* Ahi = sm;
    unsigned char* Alo = sm + kTile;
    unsigned char* Bhi = sm + 2 * kTile;
    unsigned char* Blo = sm + 3 * kTile;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = 128;
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&bar), 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_slot), ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t lbo = lbo_swap ? 32 * KF : 128, sbo = lbo_swap ? 128 : 32 * KF;
    const uint32_t idesc = tc::idesc_tf32(128, N);
    uint32_t phase = 0;
    int failed = 0;
    for (int k0 = 0; k0 < K && !failed; k0 += KF) {
        for (int e = tid; e < 128 * KF; e += 128) {
            const int r = e / KF, k = e % KF;
            const float a = r < M ? A[(long long)r * K + k0 + k] : 0.0f;
            float hi, lo;
            tc::tf32_split(a, hi, lo);
            const uint32_t o = tc::kmajor_offset(r, k, KF);
            *reinterpret_cast<float*>(Ahi + o) = hi;
            *reinterpret_cast<float*>(Alo + o) = lo;
        }
        for (int e = tid; e < N * KF; e += 128) {
            const int r = e / KF, k = e % KF;
            float hi, lo;
            tc::tf32_split(B[(long long)r * K + k0 + k], hi, lo);
            const uint32_t o = tc::kmajor_offset(r, k, KF);
            *reinterpret_cast<float*>(Bhi + o) = hi;
            *reinterpret_cast<float*>(Blo + o) = lo;
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_addr(Ahi), a1 = tc::smem_addr(Alo), b0 = tc::smem_addr(Bhi),
                           b1 = tc::smem_addr(Blo);
            for (int j = 0; j < KF / 8; ++j) {
                const uint32_t step = (uint32_t)j * 256;  // two core matrices along K per MMA
                tc::mma_tf32(tmem, tc::smem_desc(a0 + step, lbo, sbo), tc::smem_desc(b0 + step, lbo, sbo), idesc,
                             ((k0 > 0 && !drain) || j > 0) ? 1u : 0u);
                tc::mma_tf32(tmem, tc::smem_desc(a0 + step, lbo, sbo), tc::smem_desc(b1 + step, lbo, sbo), idesc, 1u);
                tc::mma_tf32(tmem, tc::smem_desc(a1 + step, lbo, sbo), tc::smem_desc(b0 + step, lbo, sbo), idesc, 1u);
                if (four)
                    tc::mma_tf32(tmem, tc::smem_desc(a1 + step, lbo, sbo), tc::smem_desc(b1 + step, lbo, sbo), idesc, 1u);
            }
            tc::mma_commit(tc::smem_addr(&bar));
        }
        const bool ok = tc::mbar_wait(tc::smem_addr(&bar), phase, timeout_ns);
        phase ^= 1;
        failed = __syncthreads_or(!ok);
        if (drain && !failed) {
            tc::tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < 128; c0 += 8) {
                if (c0 < N) {
                    float v[8];
                    tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[c0 + i] += (double)v[i];
                }
            }
            tc::tc_fence_before();
            __syncthreads();
        }
    }
    tc::tc_fence_after();
    if (!failed) {
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 8) {
            if (c0 < N) {
                float v[8];
                if (!drain) tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
                const int row = warp * 32 + lane;
                if (row < M)
                    for (int i = 0; i < 8; ++i)
                        if (c0 + i < N) D[(long long)row * N + c0 + i] = drain ? (float)acc[c0 + i] : v[i];
            }
        }
    } else {
        // gave up: wait once more (bounded) for the MMAs in flight before the accumulator is freed
        if (tid == 0) *err = 1;
        tc::mbar_wait(tc::smem_addr(&bar), phase ^ 1, timeout_ns);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------------------------------
// Projection on the tensor cores: for each (k, spin) segment of the band list and each of ksplit
// plane-wave ranges, part[ks][c][p] = sum_G conj(A_p(G)) X_c(G) over the range, as the real product
//     D[p][n] = sum_k A'[p][k] B'[n][k],  k = 2G + (0: re, 1: im),
// A' the family rows as stored (re, im interleaved), B' rows 2c = X_c (re, im) and 2c+1 = (im, -re)
// of band c, so that D[p][2c] = Re P and D[p][2c+1] = Im P.  M = 128 rows (zero beyond nrow),
// N = 2 x bands of a tile (at most 32 bands), K in chunks of 16 plane waves.
//
// Pipeline: two shared-memory stages and two TMEM accumulators.  Chunk i is staged into stage i % 2
// and multiplied into accumulator i % 2 while chunk i-1's MMAs run; before stage i % 2 is refilled,
// chunk i-2's MMAs must have completed (mbarrier of that stage) and their accumulator is drained
// into FP32 registers.  Draining every chunk keeps each tensor-core accumulation to 32 values of K:
// the tensor core's accumulator does not round to nearest, and over hundreds of terms its error
// grows with K; the FP32 registers add the chunk sums with rounding to nearest.
// ------------------------------------------------------------------------------------------------
constexpr int kKF = 32;                            // FP32 values along K per staged chunk
constexpr int kBandTile = 32;                      // bands per tile (N <= 64)
constexpr int kNMax = 2 * kBandTile;
constexpr uint32_t kATile = 128u * kKF * 4u;       // 16 KB: one A operand (hi or lo)
constexpr uint32_t kBTile = (uint32_t)kNMax * kKF * 4u;  // 8 KB: one B operand
constexpr uint32_t kStage = 2 * kATile + 2 * kBTile;
constexpr int kTcSmem = 2 * (int)kStage;           // 96 KB: two CTAs per SM
constexpr uint32_t kTcCols = 128;                  // TMEM columns: accumulators at 0 and 64

__device__ int g_tc_err = 0;

__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
    float h, l;
    tc::tf32_split(v, h, l);
    *reinterpret_cast<float*>(hi + off) = h;
    *reinterpret_cast<float*>(lo + off) = l;
}

struct Stage {
    unsigned char *Ahi, *Alo, *Bhi, *Blo;
};
__device__ __forceinline__ Stage stage_of(unsigned char* sm, int s) {
    unsigned char* b = sm + (uint32_t)s * kStage;
    return Stage{b, b + kATile, b + 2 * kATile, b + 2 * kATile + kBTile};
}

// thread 0: the three TF32 products of one staged chunk (4 MMAs of K = 8 each) into a fresh accumulator
__device__ __forceinline__ void issue_chunk(uint32_t tmem, const Stage& st, uint32_t idesc) {
    const uint32_t a0 = tc::smem_addr(st.Ahi), a1 = tc::smem_addr(st.Alo), b0 = tc::smem_addr(st.Bhi),
                   b1 = tc::smem_addr(st.Blo);
    constexpr uint32_t lbo = 128, sbo = 32 * kKF;
#pragma unroll
    for (int j = 0; j < kKF / 8; ++j) {
        const uint32_t step = (uint32_t)j * 256;
        tc::mma_tf32(tmem, tc::smem_desc(a0 + step, lbo, sbo), tc::smem_desc(b0 + step, lbo, sbo), idesc,
                     j == 0 ? 0u : 1u);
        tc::mma_tf32(tmem, tc::smem_desc(a0 + step, lbo, sbo), tc::smem_desc(b1 + step, lbo, sbo), idesc, 1u);
        tc::mma_tf32(tmem, tc::smem_desc(a1 + step, lbo, sbo), tc::smem_desc(b0 + step, lbo, sbo), idesc, 1u);
    }
}

// acc[0 .. N-1] += the accumulator at TMEM column col0 (this thread's lane), N a multiple of 16
__device__ __forceinline__ void drain(uint32_t taddr, int N, float (&acc)[kNMax]) {
    tc::tc_fence_after();
#pragma unroll
    for (int c0 = 0; c0 < kNMax; c0 += 8) {
        if (c0 < N) {
            float v[8];
            tc::tmem_ld8(taddr + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[c0 + i] += v[i];
        }
    }
    tc::tc_fence_before();
}

// zero rows r0 .. r1-1 of a K-major tile (both split halves)
__device__ __forceinline__ void zero_rows(unsigned char* hi, unsigned char* lo, int r0, int r1) {
    for (int e = threadIdx.x; e < (r1 - r0) * kKF; e += 128) {
        const uint32_t o = tc::kmajor_offset(r0 + e / kKF, e % kKF, kKF);
        *reinterpret_cast<float*>(hi + o) = 0.0f;
        *reinterpret_cast<float*>(lo + o) = 0.0f;
    }
}

__global__ void __launch_bounds__(128, 2) proj_tc_kernel(ProjDev d, int ld, const float2* __restrict__ X,
                                                         const int* __restrict__ row, const int* __restrict__ seg_start,
                                                         const int* __restrict__ seg_k, const int* __restrict__ seg_s,
                                                         const int* __restrict__ npw_of_k, int ksplit,
                                                         double2* __restrict__ part, int nb,
                                                         unsigned long long timeout_ns) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    const int seg = blockIdx.x, ks = blockIdx.y;
    const int cbeg = seg_start[seg], cend = seg_start[seg + 1];
    const int k = seg_k[seg], sp = seg_s[seg];
    const int npw = npw_of_k[k];
    const int nrow = d.n0 + d.n1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = ((npw + ksplit - 1) / ksplit + 15) / 16 * 16;
    const int g0 = ks * chunk;
    const int g1 = min(npw, g0 + chunk);
    if (g0 >= g1) {  // empty split: its partial sums are zero
        for (int e = tid; e < (cend - cbeg) * nrow; e += 128)
            part[((long long)ks * nb + cbeg + e / nrow) * 128 + e % nrow] = make_double2(0.0, 0.0);
        return;
    }
    const int mk = d.kmap ? d.kmap[k] : k;
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&bar[0]), 1);
        tc::mbar_init(tc::smem_addr(&bar[1]), 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_slot), kTcCols);
    for (int s = 0; s < 2; ++s) {  // rows nrow .. 127 of both A stages stay zero
        const Stage st = stage_of(sm, s);
        zero_rows(st.Ahi, st.Alo, nrow, 128);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    const int gg = tid & 15;      // the plane wave of the chunk this thread loads
    const int pa = tid >> 4;      // A rows pa + 8 i
    const int nchunk = (g1 - g0 + 15) / 16;
    uint32_t phase[2] = {0, 0};
    int failed = 0;
    for (int ct0 = cbeg; ct0 < cend && !failed; ct0 += kBandTile) {
        const int nbt = min(kBandTile, cend - ct0);
        const int N = 2 * ((nbt + 7) / 8 * 8);
        const uint32_t idesc = tc::idesc_tf32(128, N);
        for (int s = 0; s < 2; ++s) {  // B rows 2 nbt .. N-1 stay zero for this tile
            const Stage st = stage_of(sm, s);
            zero_rows(st.Bhi, st.Blo, 2 * nbt, N);
        }
        // X loads: element e = tid + 128 i -> band c = e / 16 (at most 4 per thread)
        const float2* xrow[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = (tid + 128 * i) >> 4;
            xrow[i] = c < nbt ? X + (long long)row[ct0 + c] * ld : nullptr;
        }
        float acc[kNMax];
#pragma unroll
        for (int i = 0; i < kNMax; ++i) acc[i] = 0.0f;
        float2 ra[16], rx[4];
        auto fetch = [&](int gt) {
            const int G = gt + gg;
            const bool in = G < g1;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int p = pa + 8 * i;
                ra[i] = (p < nrow && in) ? proj_row<float2>(d, sp, mk, p, ld)[G] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) rx[i] = (xrow[i] && in) ? xrow[i][G] : make_float2(0.f, 0.f);
        };
        fetch(g0);
        for (int ci = 0; ci < nchunk; ++ci) {
            const int s = ci & 1;
            const Stage st = stage_of(sm, s);
            if (ci >= 2) {  // chunk ci-2 used this stage and accumulator: wait for it, drain it
                const bool ok = tc::mbar_wait(tc::smem_addr(&bar[s]), phase[s], timeout_ns);
                phase[s] ^= 1;
                if (__syncthreads_or(!ok)) {
                    failed = 1;
                    break;
                }
                drain(lane_addr + (uint32_t)s * 64, N, acc);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int p = pa + 8 * i;
                if (p < nrow) {
                    put_split(st.Ahi, st.Alo, tc::kmajor_offset(p, 2 * gg, kKF), ra[i].x);
                    put_split(st.Ahi, st.Alo, tc::kmajor_offset(p, 2 * gg + 1, kKF), ra[i].y);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = (tid + 128 * i) >> 4;
                if (c < nbt) {
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c, 2 * gg, kKF), rx[i].x);
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c, 2 * gg + 1, kKF), rx[i].y);
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c + 1, 2 * gg, kKF), rx[i].y);
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c + 1, 2 * gg + 1, kKF), -rx[i].x);
                }
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                issue_chunk(tmem + (uint32_t)s * 64, st, idesc);
                tc::mma_commit(tc::smem_addr(&bar[s]));
            }
            if (ci + 1 < nchunk) fetch(g0 + 16 * (ci + 1));
        }
        // the last one or two chunks are still in flight
        for (int ci = max(0, nchunk - 2); ci < nchunk && !failed; ++ci) {
            const int s = ci & 1;
            const bool ok = tc::mbar_wait(tc::smem_addr(&bar[s]), phase[s], timeout_ns);
            phase[s] ^= 1;
            if (__syncthreads_or(!ok)) {
                failed = 1;
                break;
            }
            drain(lane_addr + (uint32_t)s * 64, N, acc);
        }
        if (failed) break;
        const int p = warp * 32 + lane;
#pragma unroll
        for (int i = 0; i < kBandTile; ++i)
            if (p < nrow && i < nbt)
                part[((long long)ks * nb + ct0 + i) * 128 + p] = make_double2((double)acc[2 * i], (double)acc[2 * i + 1]);
        __syncthreads();  // every TMEM read of this tile done before the next tile's MMAs
    }
    if (failed) {
        if (tid == 0) atomicExch(&g_tc_err, 1);
        // MMAs possibly still in flight on either stage: one more bounded wait each
        tc::mbar_wait(tc::smem_addr(&bar[0]), phase[0], timeout_ns);
        tc::mbar_wait(tc::smem_addr(&bar[1]), phase[1], timeout_ns);
        const double nan = __longlong_as_double(0x7FF8000000000000LL);
        for (int e = tid; e < (cend - cbeg) * nrow; e += 128)
            part[((long long)ks * nb + cbeg + e / nrow) * 128 + e % nrow] = make_double2(nan, nan);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

// ------------------------------------------------------------------------------------------------
// Expansion on the tensor cores: Y_c(G) += alpha sum_p A_p(G) w_p P[c][p] for the bands c of each
// segment and a tile of 128 plane waves, as the real product
//     D[G][n] = sum_k A'[G][k] B'[n][k],  k = 2p + (0: re, 1: im),
// A' the family rows transposed onto the plane-wave tile, B' rows 2c = (Re Q, -Im Q) and
// 2c+1 = (Im Q, Re Q) of Q_c = alpha w P_c, so that D[G][2c] = Re dY and D[G][2c+1] = Im dY.
// M = 128 plane waves, N = 2 x bands of a tile, K in chunks of 16 rows p; the same two-stage
// pipeline and per-chunk draining as the projection.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 2) expand_tc_kernel(ProjDev d, int ld, const double2* __restrict__ P,
                                                           const double* __restrict__ pscale, double alpha, double scale2,
                                                           float2* __restrict__ Y, const int* __restrict__ row,
                                                           const int* __restrict__ seg_start,
                                                           const int* __restrict__ seg_k, const int* __restrict__ seg_s,
                                                           const int* __restrict__ npw_of_k,
                                                           unsigned long long timeout_ns) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    const int seg = blockIdx.y;
    const int cbeg = seg_start[seg], cend = seg_start[seg + 1];
    const int k = seg_k[seg], sp = seg_s[seg];
    const int npw = npw_of_k[k];
    const int G0 = blockIdx.x * 128;
    if (G0 >= npw) return;
    const int nrow = d.n0 + d.n1;
    const int nkc = (nrow + 15) / 16;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = G0 + tid;
    const int mk = d.kmap ? d.kmap[k] : k;
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&bar[0]), 1);
        tc::mbar_init(tc::smem_addr(&bar[1]), 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_slot), kTcCols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase[2] = {0, 0};
    int failed = 0;
    for (int ct0 = cbeg; ct0 < cend && !failed; ct0 += kBandTile) {
        const int nbt = min(kBandTile, cend - ct0);
        const int N = 2 * ((nbt + 7) / 8 * 8);
        const uint32_t idesc = tc::idesc_tf32(128, N);
        for (int s = 0; s < 2; ++s) {
            const Stage st = stage_of(sm, s);
            zero_rows(st.Bhi, st.Blo, 2 * nbt, N);
        }
        float acc[kNMax];
#pragma unroll
        for (int i = 0; i < kNMax; ++i) acc[i] = 0.0f;
        float2 ra[16];
        double2 rq[4];
        auto fetch = [&](int j) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int p = 16 * j + i;
                ra[i] = (p < nrow && G < npw) ? proj_row<float2>(d, sp, mk, p, ld)[G] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = tid + 128 * i, c = e >> 4, p = 16 * j + (e & 15);
                double2 q = make_double2(0.0, 0.0);
                if (c < nbt && p < nrow) {
                    const double w = alpha * (p < d.n0 ? (pscale ? pscale[p] : 1.0) : scale2);
                    const double2 v = P[(long long)(ct0 + c) * 128 + p];
                    q = make_double2(v.x * w, v.y * w);
                }
                rq[i] = q;
            }
        };
        fetch(0);
        for (int j = 0; j < nkc; ++j) {
            const int s = j & 1;
            const Stage st = stage_of(sm, s);
            if (j >= 2) {
                const bool ok = tc::mbar_wait(tc::smem_addr(&bar[s]), phase[s], timeout_ns);
                phase[s] ^= 1;
                if (__syncthreads_or(!ok)) {
                    failed = 1;
                    break;
                }
                drain(lane_addr + (uint32_t)s * 64, N, acc);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                put_split(st.Ahi, st.Alo, tc::kmajor_offset(tid, 2 * i, kKF), ra[i].x);
                put_split(st.Ahi, st.Alo, tc::kmajor_offset(tid, 2 * i + 1, kKF), ra[i].y);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = tid + 128 * i, c = e >> 4, pl = e & 15;
                if (c < nbt) {
                    const float qr = (float)rq[i].x, qi = (float)rq[i].y;
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c, 2 * pl, kKF), qr);
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c, 2 * pl + 1, kKF), -qi);
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c + 1, 2 * pl, kKF), qi);
                    put_split(st.Bhi, st.Blo, tc::kmajor_offset(2 * c + 1, 2 * pl + 1, kKF), qr);
                }
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                issue_chunk(tmem + (uint32_t)s * 64, st, idesc);
                tc::mma_commit(tc::smem_addr(&bar[s]));
            }
            if (j + 1 < nkc) fetch(j + 1);
        }
        for (int j = max(0, nkc - 2); j < nkc && !failed; ++j) {
            const int s = j & 1;
            const bool ok = tc::mbar_wait(tc::smem_addr(&bar[s]), phase[s], timeout_ns);
            phase[s] ^= 1;
            if (__syncthreads_or(!ok)) {
                failed = 1;
                break;
            }
            drain(lane_addr + (uint32_t)s * 64, N, acc);
        }
        if (failed) break;
        const int Gw = G0 + warp * 32 + lane;  // TMEM lane of this thread = plane wave
#pragma unroll
        for (int i = 0; i < kBandTile; ++i) {
            if (i < nbt && Gw < npw) {
                float2* y = Y + (long long)row[ct0 + i] * ld + Gw;
                float2 t = *y;
                t.x += acc[2 * i];
                t.y += acc[2 * i + 1];
                *y = t;
            }
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicExch(&g_tc_err, 1);
        tc::mbar_wait(tc::smem_addr(&bar[0]), phase[0], timeout_ns);
        tc::mbar_wait(tc::smem_addr(&bar[1]), phase[1], timeout_ns);
        const float nan = __int_as_float(0x7FC00000);
        if (G < npw)
            for (int c = cbeg; c < cend; ++c) Y[(long long)row[c] * ld + G] = make_float2(nan, nan);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

unsigned long long g_timeout_ns = 2000000000ULL;

}  // namespace

bool tc_enabled() {  // opt-in while the tensor-core path is being validated (HP_TC=1)
    static const bool on = getenv("HP_TC") != nullptr && getenv("HP_NO_TC") == nullptr;
    return on;
}

void tc_set_timeout(double seconds) { g_timeout_ns = (unsigned long long)(seconds * 1e9); }

cudaError_t tc_proj(const ProjDev& d, const BandList& L, const SphereSet& S, const float2* X, int ld, int ksplit,
                    double2* part, cudaStream_t st) {
    static bool attr = [] {
        return cudaFuncSetAttribute(proj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) == cudaSuccess;
    }();
    if (!attr) return cudaErrorInvalidConfiguration;
    dim3 g(L.nseg, ksplit);
    proj_tc_kernel<<<g, 128, kTcSmem, st>>>(d, ld, X, L.d_row, L.d_seg_start, L.d_seg_k, L.d_seg_s, S.d_npw, ksplit,
                                            part, L.nb, g_timeout_ns);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t tc_expand(const ProjDev& d, const BandList& L, const SphereSet& S, const double2* P, const double* pscale,
                      double alpha, double scale2, float2* Y, int ld, cudaStream_t st) {
    static bool attr = [] {
        return cudaFuncSetAttribute(expand_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) ==
               cudaSuccess;
    }();
    if (!attr) return cudaErrorInvalidConfiguration;
    dim3 g((ld + 127) / 128, L.nseg);
    expand_tc_kernel<<<g, 128, kTcSmem, st>>>(d, ld, P, pscale, alpha, scale2, Y, L.d_row, L.d_seg_start, L.d_seg_k,
                                              L.d_seg_s, S.d_npw, g_timeout_ns);
    HP_LAUNCHED();
    return cudaGetLastError();
}

int tc_take_error(cudaStream_t st) {
    int v = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(int)) != cudaSuccess) return 0;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(int));
    }
    return v;
}

}  // namespace hp

extern "C" hp_status hp_selftest_tc(int M, int N, int K, const float* A, const float* B, float* D, int mode,
                                    double timeout_s) {
    if (M < 1 || M > 128 || N < 16 || N > 128 || N % 16 || K < 32 || K % 32 || !A || !B || !D || !(timeout_s > 0))
        return HP_EINVAL;
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int* dErr = nullptr;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * (size_t)M * K);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(float) * (size_t)N * K);
    if (e == cudaSuccess) e = cudaMalloc(&dD, sizeof(float) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&dErr, sizeof(int));
    if (e == cudaSuccess) hp::g_allocs.fetch_add(4, std::memory_order_relaxed);
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, sizeof(float) * (size_t)M * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, sizeof(float) * (size_t)N * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dD, 0, sizeof(float) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMemset(dErr, 0, sizeof(int));
    const int smem = 4 * 128 * hp::kSelfKF * 4;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hp::tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        hp::tc_selftest_kernel<<<1, 128, smem>>>(dA, M, dB, N, K, dD, mode,
                                                 (unsigned long long)(timeout_s * 1e9), dErr);
        HP_LAUNCHED();
        e = cudaGetLastError();
    }
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, dErr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dErr);
    if (e != cudaSuccess) return HP_ECUDA;
    return err ? HP_ETIMEOUT : HP_OK;
}
