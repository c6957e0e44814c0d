// Sphere-sparse fused transforms for H.psi, Delta V u and Delta rho ("column -> plane -> column").
//
// The wavefunction sphere is stored column by column (z fastest), so the points of one z-column of
// the FFT grid are contiguous in a band vector.  A transform to real space and back then runs as
//   col_inv   : inverse z-FFT of the columns that hold sphere points (about 15 % of the grid's
//               columns) into a compact column buffer [band][z][column];
//   plane     : per (band, z-plane) in shared memory: inverse y- and x-FFTs, the real-space work
//               (multiply by V, or by u_k(r) Delta V(r), or write the real-space function), forward
//               x- and y-FFTs, and the gather of the column positions;
//   col_fwd   : forward z-FFT of the columns and the gather onto the sphere, with the kinetic term.
// Real-space band grids use the plane-major layout [z][y][x] so that a plane is contiguous.
// HBM traffic per band drops from ~6 full-grid round trips to two compact column buffers.
#include <type_traits>

#include "hp_internal.h"

namespace hp {

static inline int cdivf(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---- compile-time Stockham stages on a shared-memory array with element stride ES and line
// stride LS (NL lines of N points); returns the buffer holding the result.
template <int... R>
struct Radices_ {};
template <int N> struct FactorF;
template <> struct FactorF<10> { using type = Radices_<2, 5>; };
template <> struct FactorF<12> { using type = Radices_<4, 3>; };
template <> struct FactorF<15> { using type = Radices_<3, 5>; };
template <> struct FactorF<16> { using type = Radices_<4, 4>; };
template <> struct FactorF<18> { using type = Radices_<2, 3, 3>; };
template <> struct FactorF<20> { using type = Radices_<4, 5>; };
template <> struct FactorF<24> { using type = Radices_<4, 2, 3>; };
template <> struct FactorF<36> { using type = Radices_<4, 3, 3>; };
template <> struct FactorF<45> { using type = Radices_<3, 3, 5>; };
template <> struct FactorF<72> { using type = Radices_<4, 2, 3, 3>; };

template <class V>
__device__ __forceinline__ void bfly(V* v, int R, int s) {
    if (R == 2) {
        V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        V t2 = cadd(v[1], v[3]), t3 = cmul_si(csub(v[1], v[3]), s);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if (R == 3) {
        using T = typename Scalar<V>::type;
        const T h = (T)0.86602540378443864676;
        V t1 = cadd(v[1], v[2]);
        V t2 = csub(v[0], cscale(t1, (T)0.5));
        V t3 = cmul_si(cscale(csub(v[1], v[2]), h), s);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if (R == 5) {
        using T = typename Scalar<V>::type;
        const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
        const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
        V t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        V t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        V a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
        V a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
        V b1 = cmul_si(cadd(cscale(t3, s1), cscale(t4, s2)), s);
        V b2 = cmul_si(csub(cscale(t3, s2), cscale(t4, s1)), s);
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
}

template <class V, int N, int SIGN, int NL, int ES, int LS, int NT, int NS, int R, int... Rest>
__device__ __forceinline__ V* fst(V* src, V* dst, const V* __restrict__ tw) {
    constexpr int NR = N / R;
    constexpr int ITEMS = NL * NR;
    constexpr int TSTEP = N / (NS * R);
#pragma unroll
    for (int w0 = 0; w0 < ITEMS; w0 += NT) {
        const int w = w0 + (int)threadIdx.x;
        if ((ITEMS % NT) == 0 || w < ITEMS) {
            const int l = w % NL;
            const int j = w / NL;
            const int k = j % NS;
            V v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                V x = src[(j + r * NR) * ES + l * LS];
                if (NS > 1 && r > 0) {
                    V t = tw[r * k * TSTEP];
                    if (SIGN > 0) t.y = -t.y;
                    x = cmul(x, t);
                }
                v[r] = x;
            }
            bfly(v, R, SIGN);
            const int idxD = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[(idxD + r * NS) * ES + l * LS] = v[r];
        }
    }
    __syncthreads();
    if constexpr (sizeof...(Rest) == 0) {
        return dst;
    } else {
        return fst<V, N, SIGN, NL, ES, LS, NT, NS * R, Rest...>(dst, src, tw);
    }
}

template <class V, int N, int SIGN, int NL, int ES, int LS, int NT, int... R>
__device__ __forceinline__ V* fft_lines(Radices_<R...>, V* src, V* dst, const V* __restrict__ tw) {
    return fst<V, N, SIGN, NL, ES, LS, NT, 1, R...>(src, dst, tw);
}

template <class V, int N, int SIGN, int NL, int ES, int LS, int NT>
__device__ __forceinline__ V* lines(V* src, V* dst, const V* __restrict__ tw) {
    return fft_lines<V, N, SIGN, NL, ES, LS, NT>(typename FactorF<N>::type{}, src, dst, tw);
}

template <class V>
__device__ __forceinline__ V from64(double2 x) {
    return cpack<V>(x.x, x.y);
}

// ------------------------------------------------------------------------------------------------
// col_inv: band vectors (FP64 rows, sphere in column order) -> column buffer [c][z][ncmax],
// inverse z-FFT.  16 columns per CTA.
// ------------------------------------------------------------------------------------------------
constexpr int kCT = 16, kCLD = kCT + 1, kColThreads = 128;

template <class V, int N2>
__global__ void __launch_bounds__(kColThreads) col_inv_kernel(const double2* __restrict__ X, int ld,
                                                              const int* __restrict__ row, const int* __restrict__ kk,
                                                              int c0, const int* __restrict__ ncol,
                                                              const int* __restrict__ col_start,
                                                              const int* __restrict__ col_len,
                                                              const int* __restrict__ iz, int ncmax,
                                                              V* __restrict__ colbuf, const V* __restrict__ tw) {
    __shared__ V s0[N2 * kCLD];
    __shared__ V s1[N2 * kCLD];
    const int c = blockIdx.y;
    const int k = kk[c0 + c];
    const int nc = ncol[k];
    const int cb = blockIdx.x * kCT;
    if (cb >= nc) return;
    for (int e = threadIdx.x; e < N2 * kCLD; e += kColThreads) s0[e] = cpack<V>(0.0, 0.0);
    __syncthreads();
    const double2* x = X + (long long)row[c0 + c] * ld;
    for (int t = 0; t < kCT; ++t) {
        const int col = cb + t;
        if (col >= nc) break;
        const int st = col_start[(long long)k * ncmax + col], len = col_len[(long long)k * ncmax + col];
        for (int p = threadIdx.x; p < len; p += kColThreads) {
            const int g = st + p;
            s0[iz[(long long)k * ld + g] * kCLD + t] = from64<V>(x[g]);
        }
    }
    __syncthreads();
    V* out = lines<V, N2, +1, kCT, kCLD, 1, kColThreads>(s0, s1, tw);
    V* dst = colbuf + (long long)c * N2 * ncmax;
    for (int e = threadIdx.x; e < N2 * kCT; e += kColThreads) {
        const int t = e % kCT, z = e / kCT;
        if (cb + t < nc) dst[(long long)z * ncmax + cb + t] = out[z * kCLD + t];
    }
}

// ------------------------------------------------------------------------------------------------
// col_fwd: column buffer -> forward z-FFT -> sphere.  mode 0: Y = col + (|k+G|^2/2 - shift) X;
// mode 1: Y = scale * col.  Padding beyond npw is written as zero.
// ------------------------------------------------------------------------------------------------
template <class V, int N2>
__global__ void __launch_bounds__(kColThreads) col_fwd_kernel(const V* __restrict__ colbuf, int ncmax,
                                                              const int* __restrict__ row, const int* __restrict__ kk,
                                                              int c0, const int* __restrict__ npw,
                                                              const int* __restrict__ ncol,
                                                              const int* __restrict__ col_start,
                                                              const int* __restrict__ col_len,
                                                              const int* __restrict__ iz, const double* __restrict__ g2,
                                                              const double* __restrict__ shift,
                                                              const double2* __restrict__ X, double2* __restrict__ Y,
                                                              int ld, int mode, double scale, const V* __restrict__ tw) {
    __shared__ V s0[N2 * kCLD];
    __shared__ V s1[N2 * kCLD];
    const int c = blockIdx.y;
    const int k = kk[c0 + c];
    const int nc = ncol[k];
    const int cb = blockIdx.x * kCT;
    const long long ro = (long long)row[c0 + c] * ld;
    if (blockIdx.x == 0)
        for (int g = npw[k] + threadIdx.x; g < ld; g += kColThreads) Y[ro + g] = cmk(0.0, 0.0);
    if (cb >= nc) return;
    const V* src = colbuf + (long long)c * N2 * ncmax;
    for (int e = threadIdx.x; e < N2 * kCT; e += kColThreads) {
        const int t = e % kCT, z = e / kCT;
        s0[z * kCLD + t] = (cb + t < nc) ? src[(long long)z * ncmax + cb + t] : cpack<V>(0.0, 0.0);
    }
    __syncthreads();
    V* out = lines<V, N2, -1, kCT, kCLD, 1, kColThreads>(s0, s1, tw);
    const double sh = mode == 0 ? shift[c0 + c] : 0.0;
    for (int t = 0; t < kCT; ++t) {
        const int col = cb + t;
        if (col >= nc) break;
        const int st = col_start[(long long)k * ncmax + col], len = col_len[(long long)k * ncmax + col];
        for (int p = threadIdx.x; p < len; p += kColThreads) {
            const int g = st + p;
            const V v = out[iz[(long long)k * ld + g] * kCLD + t];
            double2 y;
            if (mode == 0) {
                const double d = 0.5 * g2[(long long)k * ld + g] - sh;
                const double2 xv = X[ro + g];
                y = cmk((double)v.x + d * xv.x, (double)v.y + d * xv.y);
            } else {
                y = cmk((double)v.x * scale, (double)v.y * scale);
            }
            Y[ro + g] = y;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// plane kernels, one CTA per (z-plane, band); plane in shared memory as [y][x] with row stride
// N0 + 1.  op 0: H.psi local part (colbuf in -> y,x inverse FFT -> * V -> x,y forward FFT ->
// colbuf out, scaled 1/N);  op 1: inverse only, real-space plane written to out grid [c][z][y][x];
// op 2: forward only from u(r) dV(r) (plane-major inputs) -> colbuf out, scaled 1/N.
// ------------------------------------------------------------------------------------------------
constexpr int kPlaneThreads = 256;

template <class V, int N0, int N1, int OP>
__global__ void __launch_bounds__(kPlaneThreads) plane_kernel(
    const V* __restrict__ colin, V* __restrict__ colout, int ncmax, const int* __restrict__ kk,
    const int* __restrict__ spin, int c0, const int* __restrict__ ncol, const int* __restrict__ col_xy, int N2,
    const typename Scalar<V>::type* __restrict__ vt,  // op 0: V [spin][z][y][x] (real)
    const V* __restrict__ ur, const int* __restrict__ ur_row, const V* __restrict__ dvt,  // op 2
    V* __restrict__ out, double inv_n, const V* __restrict__ tw0, const V* __restrict__ tw1) {
    using T = typename Scalar<V>::type;
    constexpr int LD = N0 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* A = (V*)smraw;
    V* B = A + N1 * LD;
    const int z = blockIdx.x;
    const int c = blockIdx.y;
    const int k = kk[c0 + c];
    const int nc = ncol[k];
    const long long nplane = (long long)N0 * N1;
    if (OP == 2) {
        const int s = spin[c0 + c];
        const V* u = ur + ((long long)ur_row[c0 + c] * N2 + z) * nplane;
        const V* d = dvt + ((long long)s * N2 + z) * nplane;
        for (int e = threadIdx.x; e < N0 * N1; e += kPlaneThreads) {
            const int x = e % N0, y = e / N0;
            A[y * LD + x] = cmul(u[e], d[e]);
        }
    } else {
        for (int e = threadIdx.x; e < N1 * LD; e += kPlaneThreads) A[e] = cpack<V>(0.0, 0.0);
        __syncthreads();
        const V* src = colin + ((long long)c * N2 + z) * ncmax;
        for (int j = threadIdx.x; j < nc; j += kPlaneThreads) {
            const int xy = col_xy[(long long)k * ncmax + j];
            const int x = xy / N1, y = xy % N1;
            A[y * LD + x] = src[j];
        }
    }
    __syncthreads();
    V* P = A;
    V* Q = B;
    if (OP != 2) {
        // inverse: along y (N0 lines x, element stride LD), then along x (N1 lines y, element stride 1)
        P = lines<V, N1, +1, N0, LD, 1, kPlaneThreads>(P, Q, tw1);
        Q = (P == A) ? B : A;
        P = lines<V, N0, +1, N1, 1, LD, kPlaneThreads>(P, Q, tw0);
        Q = (P == A) ? B : A;
    }
    if (OP == 1) {
        V* o = out + ((long long)c * N2 + z) * nplane;
        for (int e = threadIdx.x; e < N0 * N1; e += kPlaneThreads) {
            const int x = e % N0, y = e / N0;
            o[e] = P[y * LD + x];
        }
        return;
    }
    if (OP == 0) {
        const int s = spin[c0 + c];
        const T* v = vt + ((long long)s * N2 + z) * nplane;
        for (int e = threadIdx.x; e < N0 * N1; e += kPlaneThreads) {
            const int x = e % N0, y = e / N0;
            P[y * LD + x] = cscale(P[y * LD + x], v[e]);
        }
        __syncthreads();
    }
    // forward: along x, then along y
    P = lines<V, N0, -1, N1, 1, LD, kPlaneThreads>(P, Q, tw0);
    Q = (P == A) ? B : A;
    P = lines<V, N1, -1, N0, LD, 1, kPlaneThreads>(P, Q, tw1);
    V* dst = colout + ((long long)c * N2 + z) * ncmax;
    const T sc = (T)inv_n;
    for (int j = threadIdx.x; j < nc; j += kPlaneThreads) {
        const int xy = col_xy[(long long)k * ncmax + j];
        const int x = xy / N1, y = xy % N1;
        dst[j] = cscale(P[y * LD + x], sc);
    }
}

// ------------------------------------------------------------------------------------------------
// dispatch
// ------------------------------------------------------------------------------------------------
template <class V>
static const V* tw_of(const FftAxis& a);
template <>
const double2* tw_of<double2>(const FftAxis& a) { return a.d_tw; }
template <>
const float2* tw_of<float2>(const FftAxis& a) { return a.d_tw32; }

template <class V, int N2>
static cudaError_t col_launch(bool inv, const FusedArgs& a) {
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    dim3 g(cdivf(S.ncmax, kCT), a.nc);
    if (inv) {
        col_inv_kernel<V, N2><<<g, kColThreads, 0, a.st>>>(a.X, S.ld, L.d_row, L.d_k, a.c0, S.d_ncol, S.d_col_start,
                                                           S.d_col_len, S.d_iz, S.ncmax, (V*)a.colA,
                                                           tw_of<V>(a.fft->ax[2]));
    } else {
        col_fwd_kernel<V, N2><<<g, kColThreads, 0, a.st>>>((const V*)a.colB, S.ncmax, L.d_row, L.d_k, a.c0, S.d_npw,
                                                           S.d_ncol, S.d_col_start, S.d_col_len, S.d_iz, S.d_g2,
                                                           L.d_shift, a.X, a.Y, S.ld, a.mode, a.scale,
                                                           tw_of<V>(a.fft->ax[2]));
    }
    HP_LAUNCHED();
    return cudaGetLastError();
}

template <class V, int N0, int N1, int OP>
static cudaError_t plane_launch(const FusedArgs& a) {
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    const size_t smem = 2 * sizeof(V) * N1 * (N0 + 1);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(plane_kernel<V, N0, N1, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g(a.N2, a.nc);
    using T = typename Scalar<V>::type;
    plane_kernel<V, N0, N1, OP><<<g, kPlaneThreads, smem, a.st>>>(
        (const V*)a.colA, (V*)a.colB, S.ncmax, L.d_k, L.d_spin, a.c0, S.d_ncol, S.d_col_xy, a.N2, (const T*)a.vt,
        (const V*)a.ur, L.d_row, (const V*)a.dvt, (V*)a.out, a.inv_n, tw_of<V>(a.fft->ax[0]), tw_of<V>(a.fft->ax[1]));
    HP_LAUNCHED();
    return cudaGetLastError();
}

template <class V>
static cudaError_t col_dispatch(int n2, bool inv, const FusedArgs& a) {
    switch (n2) {
        case 10: return col_launch<V, 10>(inv, a);
        case 12: return col_launch<V, 12>(inv, a);
        case 15: return col_launch<V, 15>(inv, a);
        case 16: return col_launch<V, 16>(inv, a);
        case 18: return col_launch<V, 18>(inv, a);
        case 20: return col_launch<V, 20>(inv, a);
        case 24: return col_launch<V, 24>(inv, a);
        case 36: return col_launch<V, 36>(inv, a);
        case 45: return col_launch<V, 45>(inv, a);
        default: return cudaErrorInvalidValue;
    }
}

template <class V, int OP>
static cudaError_t plane_dispatch(int n0, int n1, const FusedArgs& a) {
#define HP_PL(A0, A1) \
    if (n0 == A0 && n1 == A1) return plane_launch<V, A0, A1, OP>(a);
    HP_PL(10, 10) HP_PL(12, 12) HP_PL(15, 15) HP_PL(16, 16) HP_PL(18, 18) HP_PL(20, 20) HP_PL(24, 24)
    HP_PL(36, 36) HP_PL(45, 45) HP_PL(72, 45)
#undef HP_PL
    return cudaErrorInvalidValue;
}

bool fused_supported(const int N[3]) {
    auto colok = [](int n) { return n == 10 || n == 12 || n == 15 || n == 16 || n == 18 || n == 20 || n == 24 || n == 36 || n == 45; };
    auto plok = [](int a, int b) {
        return (a == b && (a == 10 || a == 12 || a == 15 || a == 16 || a == 18 || a == 20 || a == 24 || a == 36 || a == 45)) ||
               (a == 72 && b == 45);
    };
    return colok(N[2]) && plok(N[0], N[1]);
}

cudaError_t fused_col(bool fp32, bool inv, const FusedArgs& a) {
    return fp32 ? col_dispatch<float2>(a.N2, inv, a) : col_dispatch<double2>(a.N2, inv, a);
}

cudaError_t fused_plane(bool fp32, int op, const FusedArgs& a) {
    if (fp32) {
        if (op == 0) return plane_dispatch<float2, 0>(a.N0, a.N1, a);
        if (op == 1) return plane_dispatch<float2, 1>(a.N0, a.N1, a);
        return plane_dispatch<float2, 2>(a.N0, a.N1, a);
    }
    if (op == 0) return plane_dispatch<double2, 0>(a.N0, a.N1, a);
    if (op == 1) return plane_dispatch<double2, 1>(a.N0, a.N1, a);
    return plane_dispatch<double2, 2>(a.N0, a.N1, a);
}

// transposes between the standard grid layout [x][y][z] and the plane-major layout [z][y][x]
template <class T>
__global__ void to_planes_kernel(const T* __restrict__ a, T* __restrict__ b, int N0, int N1, int N2, int nvec) {
    const long long nr = (long long)N0 * N1 * N2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr * nvec; e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / nr, r = e % nr;  // r in plane-major order
        const int x = (int)(r % N0), y = (int)((r / N0) % N1), z = (int)(r / ((long long)N0 * N1));
        b[e] = a[v * nr + ((long long)x * N1 + y) * N2 + z];
    }
}

template <class T>
__global__ void from_planes_kernel(const T* __restrict__ b, T* __restrict__ a, int N0, int N1, int N2, int nvec) {
    const long long nr = (long long)N0 * N1 * N2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr * nvec; e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / nr, r = e % nr;  // r in standard order
        const int z = (int)(r % N2), y = (int)((r / N2) % N1), x = (int)(r / ((long long)N1 * N2));
        a[e] = b[v * nr + ((long long)z * N1 + y) * N0 + x];
    }
}

cudaError_t k_to_planes_real(const double* a, double* b, const int N[3], int nvec, cudaStream_t st) {
    const long long n = (long long)N[0] * N[1] * N[2] * nvec;
    to_planes_kernel<double><<<std::min(cdivf(n, 256), 8192), 256, 0, st>>>(a, b, N[0], N[1], N[2], nvec);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_to_planes_c(const double2* a, double2* b, const int N[3], int nvec, cudaStream_t st) {
    const long long n = (long long)N[0] * N[1] * N[2] * nvec;
    to_planes_kernel<double2><<<std::min(cdivf(n, 256), 8192), 256, 0, st>>>(a, b, N[0], N[1], N[2], nvec);
    HP_LAUNCHED();
    return cudaGetLastError();
}

cudaError_t k_from_planes_c(const double2* b, double2* a, const int N[3], int nvec, cudaStream_t st) {
    const long long n = (long long)N[0] * N[1] * N[2] * nvec;
    from_planes_kernel<double2><<<std::min(cdivf(n, 256), 8192), 256, 0, st>>>(b, a, N[0], N[1], N[2], nvec);
    HP_LAUNCHED();
    return cudaGetLastError();
}

}  // namespace hp
