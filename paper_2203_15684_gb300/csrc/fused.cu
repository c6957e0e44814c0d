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
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <type_traits>
#include <vector>

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
// factors of the prime-factor (Good-Thomas) register FFTs below
template <> struct FactorF<4> { using type = Radices_<4>; };
template <> struct FactorF<5> { using type = Radices_<5>; };
template <> struct FactorF<8> { using type = Radices_<4, 2>; };
template <> struct FactorF<9> { using type = Radices_<3, 3>; };

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
    if constexpr (sizeof(V) == 8) return cmkf(d2f_bits(x.x), d2f_bits(x.y));
    else return x;
}

template <class V>
__device__ __forceinline__ double2 to64(V x) {
    if constexpr (sizeof(V) == 8) return cmk(f2d_bits(x.x), f2d_bits(x.y));
    else return x;
}

// band-vector element (FP64 or FP32 storage) to the compute type
template <class V>
__device__ __forceinline__ V from_vec(const double2& x) {
    return from64<V>(x);
}
template <class V>
__device__ __forceinline__ V from_vec(const float2& x) {
    if constexpr (sizeof(V) == 8) return x;
    else return cmk(f2d_bits(x.x), f2d_bits(x.y));
}

// Y[g] of the forward column transform: mode 0 adds the kinetic term (|k+G|^2/2 - shift) X[g], mode 1
// scales.  FP64 storage forms the sum in FP64; FP32 storage (mixed form) in FP32.
template <class V>
__device__ __forceinline__ void fwd_store(double2* __restrict__ Y, const double2* __restrict__ X, long long g, V a,
                                          int mode, double g2, float, double sh, float, double scale) {
    const double2 v = to64<V>(a);
    if (mode == 0) {
        const double d = 0.5 * g2 - sh;
        const double2 xv = X[g];
        Y[g] = cmk(v.x + d * xv.x, v.y + d * xv.y);
    } else {
        Y[g] = cscale(v, scale);
    }
}
template <class V>
__device__ __forceinline__ void fwd_store(float2* __restrict__ Y, const float2* __restrict__ X, long long g, V a,
                                          int mode, double, float kin, double, float sh32, double scale) {
    const float2 v = sizeof(V) == 8 ? *reinterpret_cast<const float2*>(&a) : from64<float2>(*reinterpret_cast<const double2*>(&a));
    if (mode == 0) {
        const float d = kin - sh32;
        const float2 xv = X[g];
        Y[g] = cmkf(v.x + d * xv.x, v.y + d * xv.y);
    } else {
        Y[g] = cscale(v, (float)scale);
    }
}
__device__ __forceinline__ void zero_el(double2& y) { y = cmk(0.0, 0.0); }
__device__ __forceinline__ void zero_el(float2& y) { y = cmkf(0.f, 0.f); }

// ------------------------------------------------------------------------------------------------
// register-resident FFTs: one thread holds a whole line of N points in registers and runs the
// Stockham stages with every index and twiddle position known at compile time; twiddles
// W_N^e = exp(-2 pi i e / N) come from constant memory.
// ------------------------------------------------------------------------------------------------
template <int N> struct TwOff;
template <> struct TwOff<10> { static constexpr int v = 0; };
template <> struct TwOff<12> { static constexpr int v = 10; };
template <> struct TwOff<15> { static constexpr int v = 22; };
template <> struct TwOff<16> { static constexpr int v = 37; };
template <> struct TwOff<18> { static constexpr int v = 53; };
template <> struct TwOff<20> { static constexpr int v = 71; };
template <> struct TwOff<24> { static constexpr int v = 91; };
template <> struct TwOff<36> { static constexpr int v = 115; };
template <> struct TwOff<45> { static constexpr int v = 151; };
template <> struct TwOff<72> { static constexpr int v = 196; };
template <> struct TwOff<4> { static constexpr int v = 268; };
template <> struct TwOff<5> { static constexpr int v = 272; };
template <> struct TwOff<8> { static constexpr int v = 277; };
template <> struct TwOff<9> { static constexpr int v = 285; };
constexpr int kTwTotal = 294;
constexpr int kTwSizes[] = {10, 12, 15, 16, 18, 20, 24, 36, 45, 72, 4, 5, 8, 9};
__constant__ float2 c_tw32[kTwTotal];
__constant__ double2 c_tw64[kTwTotal];

template <class V>
__device__ __forceinline__ V ctw(int i);
template <>
__device__ __forceinline__ float2 ctw<float2>(int i) { return c_tw32[i]; }
template <>
__device__ __forceinline__ double2 ctw<double2>(int i) { return c_tw64[i]; }

template <class V, int N, int SIGN, int NS, int R, int... Rest>
__device__ __forceinline__ void rstages(V (&a)[N]) {
    constexpr int NR = N / R;
    constexpr int TSTEP = N / (NS * R);
    V b[N];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int k = j % NS;
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            V x = a[j + r * NR];
            if (r > 0 && k > 0) {
                V t = ctw<V>(TwOff<N>::v + r * k * TSTEP);
                if (SIGN > 0) t.y = -t.y;
                x = cmul(x, t);
            }
            v[r] = x;
        }
        bfly(v, R, SIGN);
        const int d = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) b[d + r * NS] = v[r];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = b[i];
    if constexpr (sizeof...(Rest) > 0) rstages<V, N, SIGN, NS * R, Rest...>(a);
}

template <class V, int N, int SIGN, int... R>
__device__ __forceinline__ void rfft_(Radices_<R...>, V (&a)[N]) {
    rstages<V, N, SIGN, 1, R...>(a);
}

// Lengths N = N1 N2 with coprime N1, N2 run as a prime-factor (Good-Thomas) FFT: input n =
// (N2 n1 + N1 n2) mod N, N2 transforms of length N1 over n1, N1 transforms of length N2 over n2, and
// output k = (N2 [N2^-1 mod N1] k1 + N1 [N1^-1 mod N2] k2) mod N, with no twiddle factors between
// the two sets of transforms (W_N^(nk) = W_N1^(n1 k1) W_N2^(n2 k2) for these index maps).
template <int N>
struct PfaF {
    static constexpr int n1 = 0, n2 = 0;
};
template <> struct PfaF<36> { static constexpr int n1 = 4, n2 = 9; };
template <> struct PfaF<45> { static constexpr int n1 = 9, n2 = 5; };
template <> struct PfaF<72> { static constexpr int n1 = 8, n2 = 9; };

__host__ __device__ constexpr int inv_mod(int a, int m) {
    for (int x = 1; x < m; ++x)
        if ((a * x) % m == 1) return x;
    return 1;
}

template <class V, int N, int SIGN>
__device__ __forceinline__ void rfft(V (&a)[N]);

template <class V, int N1, int N2, int SIGN>
__device__ __forceinline__ void rfft_pfa(V (&a)[N1 * N2]) {
    constexpr int N = N1 * N2;
    constexpr int A = inv_mod(N2 % N1, N1), B = inv_mod(N1 % N2, N2);
    V y[N];  // y[k1 N2 + n2]
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
        V t[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) t[n1] = a[(N2 * n1 + N1 * n2) % N];
        rfft<V, N1, SIGN>(t);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) y[k1 * N2 + n2] = t[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        V t[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) t[n2] = y[k1 * N2 + n2];
        rfft<V, N2, SIGN>(t);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a[(N2 * A * k1 + N1 * B * k2) % N] = t[k2];
    }
}

template <class V, int N, int SIGN>
__device__ __forceinline__ void rfft(V (&a)[N]) {
    if constexpr (PfaF<N>::n1 > 0) rfft_pfa<V, PfaF<N>::n1, PfaF<N>::n2, SIGN>(a);
    else rfft_<V, N, SIGN>(typename FactorF<N>::type{}, a);
}

// line lengths a thread can hold: 72 complex FP32 or 36 complex FP64 values
template <class V>
constexpr int reg_nmax() { return sizeof(V) == 8 ? 72 : 36; }

static cudaError_t regfft_init() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        std::vector<float2> t32(kTwTotal);
        std::vector<double2> t64(kTwTotal);
        int off = 0;
        for (int n : kTwSizes) {
            for (int e = 0; e < n; ++e) {
                const double a = -2.0 * M_PI * (double)e / (double)n;
                t64[off + e] = cmk(std::cos(a), std::sin(a));
                t32[off + e] = cmkf((float)std::cos(a), (float)std::sin(a));
            }
            off += n;
        }
        err = cudaMemcpyToSymbol(c_tw32, t32.data(), sizeof(float2) * kTwTotal);
        if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_tw64, t64.data(), sizeof(double2) * kTwTotal);
    });
    return err;
}

// PR (pruned lines): every sphere point has x, y and z grid indices within m of 0 (mod N) with
// m = (N - 1) / 4 (the sphere of an alias-free grid), so the lines along x, y and z carry their nonzero
// inputs, and need their outputs, only there.  The other positions enter the register FFTs as literal
// zeros or are never stored, and the compiler drops the arithmetic that feeds nothing.
template <int N, bool PR>
__device__ __forceinline__ constexpr bool live(int i) {
    return !PR || i <= (N - 1) / 4 || i >= N - (N - 1) / 4;
}

// The x-lines that a plane's y-transforms run on: all N0, or with pruned lines only the live ones,
// numbered 0 .. n-1 so that consecutive threads take consecutive live lines and no warp issues for
// lines that are never computed.
template <int N0, bool PR>
struct YLines {
    static constexpr int m = (N0 - 1) / 4;
    static constexpr int n = PR ? 2 * m + 1 : N0;
    __device__ __forceinline__ static int x(int i) { return (!PR || i <= m) ? i : i + N0 - n; }
};

// column transforms with one thread per (band, column): the column's sphere points are one run of
// consecutive z (wrapping at N2), so every register index is a compile-time z.
constexpr int kColRegThreads = 128;

template <class V, int N2, class VT, bool PR>
__global__ void __launch_bounds__(kColRegThreads) col_inv_reg_kernel(
    const VT* __restrict__ X, int ld, const int* __restrict__ row, const int* __restrict__ kk, int c0,
    const int* __restrict__ ncol, const int* __restrict__ col_start, const int* __restrict__ col_len,
    const int* __restrict__ iz, int ncmax, int nc, V* __restrict__ colbuf) {
    // thread t: band c = t / ncmax of the chunk, column j = t % ncmax (the bands' columns packed, so
    // that no warp is mostly past the last column of its band)
    const long long t = (long long)blockIdx.x * kColRegThreads + threadIdx.x;
    const int c = (int)(t / ncmax);
    if (c >= nc) return;
    const int j = (int)(t - (long long)c * ncmax);
    const int k = kk[c0 + c];
    if (j >= ncol[k]) return;
    const int st = col_start[(long long)k * ncmax + j], len = col_len[(long long)k * ncmax + j];
    const int z0 = iz[(long long)k * ld + st];
    const VT* x = X + (long long)row[c0 + c] * ld + st;
    V a[N2];
#pragma unroll
    for (int z = 0; z < N2; ++z) {
        int p = z - z0;
        if (p < 0) p += N2;
        a[z] = (live<N2, PR>(z) && p < len) ? from_vec<V>(x[p]) : cpack<V>(0.0, 0.0);
    }
    rfft<V, N2, +1>(a);
    V* dst = colbuf + (long long)c * N2 * ncmax + j;
#pragma unroll
    for (int z = 0; z < N2; ++z) dst[(long long)z * ncmax] = a[z];
}

template <class V, int N2, class VT, bool PR>
__global__ void __launch_bounds__(kColRegThreads) col_fwd_reg_kernel(
    const V* __restrict__ colbuf, int ncmax, const int* __restrict__ row, const int* __restrict__ kk, int c0,
    const int* __restrict__ npw, const int* __restrict__ ncol, const int* __restrict__ col_start,
    const int* __restrict__ col_len, const int* __restrict__ iz, const double* __restrict__ g2,
    const float* __restrict__ kin32, const double* __restrict__ shift, const VT* __restrict__ X,
    VT* __restrict__ Y, int ld, int mode, double scale, int nc) {
    // thread t: band c = t / ncmax of the chunk, column j = t % ncmax (as in col_inv_reg_kernel); the
    // band's threads also zero its padding beyond npw
    const long long t = (long long)blockIdx.x * kColRegThreads + threadIdx.x;
    const int c = (int)(t / ncmax);
    if (c >= nc) return;
    const int j = (int)(t - (long long)c * ncmax);
    const int k = kk[c0 + c];
    const long long ro = (long long)row[c0 + c] * ld;
    for (int g = npw[k] + j; g < ld; g += ncmax) zero_el(Y[ro + g]);
    if (j >= ncol[k]) return;
    const int st = col_start[(long long)k * ncmax + j], len = col_len[(long long)k * ncmax + j];
    const int z0 = iz[(long long)k * ld + st];
    const V* src = colbuf + (long long)c * N2 * ncmax + j;
    V a[N2];
#pragma unroll
    for (int z = 0; z < N2; ++z) a[z] = src[(long long)z * ncmax];
    rfft<V, N2, -1>(a);
    const double sh = mode == 0 ? shift[c0 + c] : 0.0;
    const float sh32 = (float)sh;
    const long long ko = (long long)k * ld + st;
#pragma unroll
    for (int z = 0; z < N2; ++z) {
        int p = z - z0;
        if (p < 0) p += N2;
        if (live<N2, PR>(z) && p < len) {
            const bool k32 = sizeof(VT) == 8;
            fwd_store<V>(Y, X, ro + st + p, a[z], mode, (mode == 0 && !k32) ? g2[ko + p] : 0.0,
                         (mode == 0 && k32) ? kin32[ko + p] : 0.f, sh, sh32, scale);
        }
    }
}

// plane transforms with one thread per line: P (band, z) planes per CTA, each [y][x] in shared
// memory with an odd row stride (N0, or N0 + 1 for even N0: 8-byte rows of different y then fall in
// different bank pairs).  The columns with one grid x form one run of consecutive column
// indices and consecutive y (mod N1), given per (k, x) by xtab = (first column, count, first y), so
// the y-line threads read and write their column values straight from and to the column buffers:
//   op 0: y-inverse (columns -> smem) | x: inverse, * V, forward | y-forward (smem -> columns)
//   op 1: y-inverse | x-inverse | coalesced copy of the real-space planes
//   op 2: x-forward of u(r) Delta V(r) read row by row | y-forward
template <class V, int N0, int N1>
struct PlaneCfg {
    static constexpr int L = N0 > N1 ? N0 : N1;
    static constexpr int LD = (N0 % 2) ? N0 : N0 + 1;
    static constexpr int kSmemMax = 227 * 1024;
    static constexpr int per_plane = N1 * LD * (int)sizeof(V);
    static constexpr int P0 = 256 / L > 0 ? 256 / L : 1;
    static constexpr int P = P0 * per_plane <= kSmemMax ? P0 : (kSmemMax / per_plane > 0 ? kSmemMax / per_plane : 1);
    static constexpr int NT = ((P * L + 31) / 32) * 32;
    static constexpr bool ok = N0 <= reg_nmax<V>() && N1 <= reg_nmax<V>() && P * per_plane <= kSmemMax;
    // resident CTAs per SM asked of the compiler (register budget 65536 / (NT * MINB) per thread):
    // three for the inverse-only form of FP32 lines up to 36 points, which fits 80 registers
    // without spilling, two for the other FP32 forms up to 45 points (128 registers, no spills)
    template <int OP>
    static constexpr int minb() {
        return (sizeof(V) == 8 && L <= 45) ? (OP == 1 && L <= 36 && 3 * P * per_plane <= 228 * 1024 ? 3 : 2) : 1;
    }
};

// row of N real or complex values from global memory into registers, 16-byte loads where aligned
template <class E, int N>
__device__ __forceinline__ void load_row(const E* __restrict__ p, E (&a)[N]) {
    constexpr int W = 16 / (int)sizeof(E);
    if constexpr (W > 1 && N % W == 0) {
        if ((reinterpret_cast<size_t>(p) & 15) == 0) {
            const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
            for (int i = 0; i < N / W; ++i) {
                const float4 v = __ldg(q + i);
                const E* e = reinterpret_cast<const E*>(&v);
#pragma unroll
                for (int w = 0; w < W; ++w) a[i * W + w] = e[w];
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = p[i];
}

// a[x] *= row[x] for a row of N real or complex values in global memory, read in 16-byte pieces
// where aligned (multiplied as they arrive, so no second row is held in registers)
template <class V, class E, int N>
__device__ __forceinline__ void mul_row(const E* __restrict__ p, V (&a)[N]) {
    constexpr int W = 16 / (int)sizeof(E);
    if constexpr (W > 1 && N % W == 0) {
        if ((reinterpret_cast<size_t>(p) & 15) == 0) {
            const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
            for (int i = 0; i < N / W; ++i) {
                const float4 v = __ldg(q + i);
                const E* e = reinterpret_cast<const E*>(&v);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if constexpr (sizeof(E) == sizeof(V)) a[i * W + w] = cmul(a[i * W + w], e[w]);
                    else a[i * W + w] = cscale(a[i * W + w], e[w]);
                }
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if constexpr (sizeof(E) == sizeof(V)) a[i] = cmul(a[i], p[i]);
        else a[i] = cscale(a[i], p[i]);
    }
}

template <class V, int N0, int N1, int OP, bool PR>
__global__ void __launch_bounds__(PlaneCfg<V, N0, N1>::NT, PlaneCfg<V, N0, N1>::template minb<OP>()) plane_reg_kernel(
    const V* __restrict__ colin, V* __restrict__ colout, int ncmax, const int* __restrict__ kk,
    const int* __restrict__ spin, int c0, int nc, const int* __restrict__ xtab, int N2,
    const typename Scalar<V>::type* __restrict__ vtx, const V* __restrict__ ur, const int* __restrict__ ur_row,
    const V* __restrict__ dvt, V* __restrict__ out, double inv_n) {
    using Cfg = PlaneCfg<V, N0, N1>;
    using T = typename Scalar<V>::type;
    constexpr int P = Cfg::P, NT = Cfg::NT, LD = Cfg::LD, NP = N0 * N1, PS = N1 * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* S = (V*)smraw;  // [P][N1][LD]
    const long long q0 = (long long)blockIdx.x * P;
    const long long npairs = (long long)nc * N2;
    const int tid = threadIdx.x;
    if constexpr (OP == 2) {
        // ---- u(r) Delta V(r) of each plane into shared memory, consecutive threads on consecutive points
        constexpr int EPT = (NP + NT - 1) / NT;
        __shared__ long long u_of[P], d_of[P];
        if (tid < P) {
            const long long q = q0 + tid;
            if (q < npairs) {
                const int c = (int)(q / N2), z = (int)(q % N2);
                u_of[tid] = ((long long)ur_row[c0 + c] * N2 + z) * NP;
                d_of[tid] = ((long long)spin[c0 + c] * N2 + z) * NP;
            }
        }
        __syncthreads();
        // plane by plane, every load of the plane issued before the first product
        const int np = (int)min((long long)P, npairs - q0);
        for (int p = 0; p < np; ++p) {
            const V* u = ur + u_of[p];
            const V* d = dvt + d_of[p];
            V uv[EPT], dv[EPT];
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const int e = tid + j * NT;
                if (e < NP) {
                    uv[j] = __ldcs(u + e);
                    dv[j] = __ldg(d + e);
                }
            }
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const int e = tid + j * NT;
                if (e < NP) S[p * PS + (e / N0) * LD + e % N0] = cmul(uv[j], dv[j]);
            }
        }
        __syncthreads();
    } else {
        // ---- y-inverse: line x of plane p from its run of columns (zero where x has none)
        if (tid < P * YLines<N0, PR>::n) {
            const int p = tid / YLines<N0, PR>::n, x = YLines<N0, PR>::x(tid % YLines<N0, PR>::n);
            const long long q = q0 + p;
            if (q < npairs && (!PR || live<N0, PR>(x))) {
                const int k = kk[c0 + (int)(q / N2)];
                const int* t = xtab + ((long long)k * N0 + x) * 3;
                const int j0 = t[0], cnt = t[1], y0 = t[2];
                V a[N1];
                const V* src = colin + q * ncmax + j0;  // pair q = c * N2 + z: plane z of chunk band c
#pragma unroll
                for (int y = 0; y < N1; ++y) {
                    int i = y - y0;
                    if (i < 0) i += N1;
                    a[y] = (live<N1, PR>(y) && i < cnt) ? src[i] : cpack<V>(0.0, 0.0);
                }
                if (cnt > 0) rfft<V, N1, +1>(a);
                V* col = S + p * PS + x;
#pragma unroll
                for (int y = 0; y < N1; ++y) col[y * LD] = a[y];
            }
        }
        __syncthreads();
    }
    // ---- along x
    if (tid < P * N1) {
        const int p = tid / N1, y = tid % N1;
        const long long q = q0 + p;
        if (q < npairs) {
            const int c = (int)(q / N2), z = (int)(q % N2);
            V* rowp = S + p * PS + y * LD;
            V a[N0];
            if (OP == 2) {
#pragma unroll
                for (int x = 0; x < N0; ++x) a[x] = rowp[x];
            } else {
#pragma unroll
                for (int x = 0; x < N0; ++x) a[x] = live<N0, PR>(x) ? rowp[x] : cpack<V>(0.0, 0.0);
                rfft<V, N0, +1>(a);
            }
            if (OP == 0) {  // V(r) from the x-major planes: consecutive threads (y) on consecutive words
                const T* vx = vtx + ((long long)spin[c0 + c] * N2 + z) * NP + y;
#pragma unroll
                for (int x = 0; x < N0; ++x) a[x] = cscale(a[x], __ldg(vx + x * N1));
            }
            if (OP != 1) rfft<V, N0, -1>(a);
#pragma unroll
            for (int x = 0; x < N0; ++x)
                if (OP == 1 || live<N0, PR>(x)) rowp[x] = a[x];
        }
    }
    __syncthreads();
    if (OP == 1) {
        for (int p = 0; p < P; ++p) {
            const long long q = q0 + p;
            if (q >= npairs) break;
            V* o = out + q * NP;
            for (int e = tid; e < NP; e += NT) o[e] = S[p * PS + (e / N0) * LD + e % N0];
        }
        return;
    }
    // ---- y-forward on the x-lines that hold columns, written straight to the column buffer
    if (tid < P * YLines<N0, PR>::n) {
        const int p = tid / YLines<N0, PR>::n, x = YLines<N0, PR>::x(tid % YLines<N0, PR>::n);
        const long long q = q0 + p;
        if (q < npairs) {
            const int k = kk[c0 + (int)(q / N2)];
            const int* t = xtab + ((long long)k * N0 + x) * 3;
            const int j0 = t[0], cnt = t[1], y0 = t[2];
            if (cnt > 0) {
                const V* col = S + p * PS + x;
                V a[N1];
#pragma unroll
                for (int y = 0; y < N1; ++y) a[y] = col[y * LD];
                rfft<V, N1, -1>(a);
                const T sc = (T)inv_n;
                V* dst = colout + q * ncmax + j0;
#pragma unroll
                for (int y = 0; y < N1; ++y) {
                    int i = y - y0;
                    if (i < 0) i += N1;
                    if (live<N1, PR>(y) && i < cnt) dst[i] = cscale(a[y], sc);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// col_inv: band vectors (FP64 rows, sphere in column order) -> column buffer [c][z][ncmax],
// inverse z-FFT.  16 columns per CTA.
// ------------------------------------------------------------------------------------------------
constexpr int kCT = 16, kCLD = kCT + 1, kColThreads = 128;

template <class V, int N2, class VT>
__global__ void __launch_bounds__(kColThreads) col_inv_kernel(const VT* __restrict__ X, int ld,
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
    const VT* x = X + (long long)row[c0 + c] * ld;
    for (int t = 0; t < kCT; ++t) {
        const int col = cb + t;
        if (col >= nc) break;
        const int st = col_start[(long long)k * ncmax + col], len = col_len[(long long)k * ncmax + col];
        for (int p = threadIdx.x; p < len; p += kColThreads) {
            const int g = st + p;
            s0[iz[(long long)k * ld + g] * kCLD + t] = from_vec<V>(x[g]);
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
template <class V, int N2, class VT>
__global__ void __launch_bounds__(kColThreads) col_fwd_kernel(const V* __restrict__ colbuf, int ncmax,
                                                              const int* __restrict__ row, const int* __restrict__ kk,
                                                              int c0, const int* __restrict__ npw,
                                                              const int* __restrict__ ncol,
                                                              const int* __restrict__ col_start,
                                                              const int* __restrict__ col_len,
                                                              const int* __restrict__ iz, const double* __restrict__ g2,
                                                              const float* __restrict__ kin32,
                                                              const double* __restrict__ shift,
                                                              const VT* __restrict__ X, VT* __restrict__ Y,
                                                              int ld, int mode, double scale, const V* __restrict__ tw) {
    __shared__ V s0[N2 * kCLD];
    __shared__ V s1[N2 * kCLD];
    const int c = blockIdx.y;
    const int k = kk[c0 + c];
    const int nc = ncol[k];
    const int cb = blockIdx.x * kCT;
    const long long ro = (long long)row[c0 + c] * ld;
    if (blockIdx.x == 0)
        for (int g = npw[k] + threadIdx.x; g < ld; g += kColThreads) zero_el(Y[ro + g]);
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
            const bool k32 = sizeof(VT) == 8;
            fwd_store<V>(Y, X, ro + g, v, mode, (mode == 0 && !k32) ? g2[(long long)k * ld + g] : 0.0,
                         (mode == 0 && k32) ? kin32[(long long)k * ld + g] : 0.f, sh, (float)sh, scale);
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

template <class V, int N2, class VT>
static void col_kernels(bool inv, bool reg, dim3 g, const FusedArgs& a) {
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    const VT* X = (const VT*)a.X;
    VT* Y = (VT*)a.Y;
    // pruned z lines for the FP32 production grids (36 and more points) when the spheres allow them
    constexpr bool kPrunable = sizeof(V) == 8 && N2 >= 36;
    const bool pr = kPrunable && S.lines_prunable && !getenv("HP_NO_PRUNE");
    const dim3 gr(cdivf((long long)a.nc * S.ncmax, kColRegThreads));  // register kernels: packed (band, column)
    if (reg && inv) {
        if (pr)
            col_inv_reg_kernel<V, N2, VT, kPrunable><<<gr, kColRegThreads, 0, a.st>>>(
                X, S.ld, L.d_row, L.d_k, a.c0, S.d_ncol, S.d_col_start, S.d_col_len, S.d_iz, S.ncmax, a.nc,
                (V*)a.colA);
        else
            col_inv_reg_kernel<V, N2, VT, false><<<gr, kColRegThreads, 0, a.st>>>(
                X, S.ld, L.d_row, L.d_k, a.c0, S.d_ncol, S.d_col_start, S.d_col_len, S.d_iz, S.ncmax, a.nc,
                (V*)a.colA);
    } else if (reg) {
        if (pr)
            col_fwd_reg_kernel<V, N2, VT, kPrunable><<<gr, kColRegThreads, 0, a.st>>>(
                (const V*)a.colB, S.ncmax, L.d_row, L.d_k, a.c0, S.d_npw, S.d_ncol, S.d_col_start, S.d_col_len,
                S.d_iz, S.d_g2, S.d_kin32, L.d_shift, X, Y, S.ld, a.mode, a.scale, a.nc);
        else
            col_fwd_reg_kernel<V, N2, VT, false><<<gr, kColRegThreads, 0, a.st>>>(
                (const V*)a.colB, S.ncmax, L.d_row, L.d_k, a.c0, S.d_npw, S.d_ncol, S.d_col_start, S.d_col_len,
                S.d_iz, S.d_g2, S.d_kin32, L.d_shift, X, Y, S.ld, a.mode, a.scale, a.nc);
    } else if (inv) {
        col_inv_kernel<V, N2, VT><<<g, kColThreads, 0, a.st>>>(X, S.ld, L.d_row, L.d_k, a.c0, S.d_ncol, S.d_col_start,
                                                               S.d_col_len, S.d_iz, S.ncmax, (V*)a.colA,
                                                               tw_of<V>(a.fft->ax[2]));
    } else {
        col_fwd_kernel<V, N2, VT><<<g, kColThreads, 0, a.st>>>((const V*)a.colB, S.ncmax, L.d_row, L.d_k, a.c0,
                                                               S.d_npw, S.d_ncol, S.d_col_start, S.d_col_len, S.d_iz,
                                                               S.d_g2, S.d_kin32, L.d_shift, X, Y, S.ld, a.mode,
                                                               a.scale, tw_of<V>(a.fft->ax[2]));
    }
}

template <class V, int N2>
static cudaError_t col_launch(bool inv, const FusedArgs& a) {
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    const bool reg = a.reg && S.contig && N2 <= reg_nmax<V>();
    if (reg) {
        cudaError_t e = regfft_init();
        if (e != cudaSuccess) return e;
    }
    // FP32 band vectors only with FP32 transforms
    if (a.vec32 && sizeof(V) != 8) return cudaErrorInvalidValue;
    dim3 g(cdivf(S.ncmax, reg ? kColRegThreads : kCT), a.nc);
    const ProfMark pm = prof_start(a.st);
    if (a.vec32) col_kernels<V, N2, float2>(inv, reg, g, a);
    else col_kernels<V, N2, double2>(inv, reg, g, a);
    HP_LAUNCHED();
    if (prof_on() && L.k.size() >= (size_t)(a.c0 + a.nc) && !S.ncol.empty()) {
        // sphere coefficients (FP64) once, column buffer once; forward: input vector for the kinetic
        // term and the zeroed padding as well
        double bytes = 0.0, flops = 0.0;
        for (int b = a.c0; b < a.c0 + a.nc; ++b) {
            const int k = L.k[b];
            const double col = (double)sizeof(V) * N2 * S.ncol[k];
            const double vb = a.vec32 ? 8.0 : 16.0;  // band-vector element
            bytes += col + vb * S.npw[k];
            if (!inv) bytes += vb * (S.ld - S.npw[k]) + (a.mode == 0 ? vb * S.npw[k] : 0.0);
            flops += 5.0 * N2 * std::log2((double)N2) * S.ncol[k];
        }
        prof_stop(pm, HP_KF_COLUMN, a.st, flops, bytes, inv ? (reg ? "col_inv_reg" : "col_inv") : (reg ? "col_fwd_reg" : "col_fwd"));
    }
    return cudaGetLastError();
}

template <class V, int N0, int N1, int OP, bool PR>
static cudaError_t plane_reg_go(const FusedArgs& a, size_t smem, int grid) {
    using Cfg = PlaneCfg<V, N0, N1>;
    using T = typename Scalar<V>::type;
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    // set once per kernel (a function-local static is initialised once, also with several host threads)
    static const cudaError_t attr = cudaFuncSetAttribute(plane_reg_kernel<V, N0, N1, OP, PR>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    plane_reg_kernel<V, N0, N1, OP, PR><<<grid, Cfg::NT, smem, a.st>>>(
        (const V*)a.colA, (V*)a.colB, S.ncmax, L.d_k, L.d_spin, a.c0, a.nc, S.d_xtab, a.N2, (const T*)a.vtx,
        (const V*)a.ur, L.d_row, (const V*)a.dvt, (V*)a.out, a.inv_n);
    return cudaSuccess;
}

template <class V, int N0, int N1, int OP>
static cudaError_t plane_reg_launch(const FusedArgs& a) {
    using Cfg = PlaneCfg<V, N0, N1>;
    using T = typename Scalar<V>::type;
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    cudaError_t e = regfft_init();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)Cfg::P * Cfg::per_plane;
    const long long npairs = (long long)a.nc * a.N2;
    const int grid = cdivf(npairs, Cfg::P);
    const ProfMark pm = prof_start(a.st);
    // pruned lines for the FP32 production grids (36 and more points) when the spheres allow them
    constexpr bool kPrunable = sizeof(V) == 8 && N0 >= 36 && N1 >= 36;
    if constexpr (kPrunable) {
        if (S.lines_prunable && !getenv("HP_NO_PRUNE")) e = plane_reg_go<V, N0, N1, OP, true>(a, smem, grid);
        else e = plane_reg_go<V, N0, N1, OP, false>(a, smem, grid);
    } else {
        e = plane_reg_go<V, N0, N1, OP, false>(a, smem, grid);
    }
    if (e != cudaSuccess) return e;
    HP_LAUNCHED();
    if (prof_on() && L.k.size() >= (size_t)(a.c0 + a.nc) && L.spin.size() >= (size_t)(a.c0 + a.nc) && !S.ncol.empty()) {
        const double nr = (double)N0 * N1 * a.N2;
        double bytes = 0.0;
        bool spin_seen[2] = {false, false};
        for (int b = a.c0; b < a.c0 + a.nc; ++b) {
            const double col = (double)sizeof(V) * a.N2 * S.ncol[L.k[b]];
            bytes += OP == 0 ? 2.0 * col : col + (double)sizeof(V) * nr;
            spin_seen[L.spin[b] & 1] = true;
        }
        const double pot = OP == 0 ? (double)sizeof(T) * nr : OP == 2 ? (double)sizeof(V) * nr : 0.0;
        bytes += pot * ((int)spin_seen[0] + (int)spin_seen[1]);
        const double flops = (OP == 0 ? 2.0 : 1.0) * 5.0 * nr * std::log2((double)N0 * N1) * a.nc;
        prof_stop(pm, HP_KF_PLANE, a.st, flops, bytes, OP == 0 ? "plane_reg_op0" : OP == 1 ? "plane_reg_op1" : "plane_reg_op2");
    }
    return cudaGetLastError();
}

template <class V, int N0, int N1, int OP>
static cudaError_t plane_launch(const FusedArgs& a) {
    if constexpr (PlaneCfg<V, N0, N1>::ok) {
        if (a.reg && a.S->d_xtab && a.S->xtab_n0 == N0) return plane_reg_launch<V, N0, N1, OP>(a);
    }
    const SphereSet& S = *a.S;
    const BandList& L = *a.L;
    const size_t smem = 2 * sizeof(V) * N1 * (N0 + 1);
    static const cudaError_t attr =
        cudaFuncSetAttribute(plane_kernel<V, N0, N1, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    dim3 g(a.N2, a.nc);
    using T = typename Scalar<V>::type;
    const ProfMark pm = prof_start(a.st);
    plane_kernel<V, N0, N1, OP><<<g, kPlaneThreads, smem, a.st>>>(
        (const V*)a.colA, (V*)a.colB, S.ncmax, L.d_k, L.d_spin, a.c0, S.d_ncol, S.d_col_xy, a.N2, (const T*)a.vt,
        (const V*)a.ur, L.d_row, (const V*)a.dvt, (V*)a.out, a.inv_n, tw_of<V>(a.fft->ax[0]), tw_of<V>(a.fft->ax[1]));
    HP_LAUNCHED();
    if (prof_on() && L.k.size() >= (size_t)(a.c0 + a.nc) && L.spin.size() >= (size_t)(a.c0 + a.nc) && !S.ncol.empty()) {
        // column buffer in and/or out per band, real-space grids once per band, potential once per spin
        const double nr = (double)N0 * N1 * a.N2;
        double bytes = 0.0;
        bool spin_seen[2] = {false, false};
        for (int b = a.c0; b < a.c0 + a.nc; ++b) {
            const double col = (double)sizeof(V) * a.N2 * S.ncol[L.k[b]];
            bytes += OP == 0 ? 2.0 * col : col + (double)sizeof(V) * nr;
            spin_seen[L.spin[b] & 1] = true;
        }
        const double pot = OP == 0 ? (double)sizeof(T) * nr : OP == 2 ? (double)sizeof(V) * nr : 0.0;
        bytes += pot * ((int)spin_seen[0] + (int)spin_seen[1]);
        const double flops = (OP == 0 ? 2.0 : 1.0) * 5.0 * nr * std::log2((double)N0 * N1) * a.nc;
        prof_stop(pm, HP_KF_PLANE, a.st, flops, bytes, OP == 0 ? "plane_op0" : OP == 1 ? "plane_op1" : "plane_op2");
    }
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

// ------------------------------------------------------------------------------------------------
// Delta rho with the inverse transform of Delta u fused in (FP32 form): CTA (z-plane, group of G
// bands, G the multiple of P nearest above 32).  Rounds of P bands: y- and x-inverse transforms of the
// bands' z-plane as in op 1, left in shared memory; then, point by point with coalesced reads of
// u(r), conj(u(r)) Delta u(r) added to the group's sum of its spin (FP32, shared memory).  The sums
// are written as FP64 to part[group][spin][z][y][x] for the spins the group holds (bit s of
// mask[group]); the groups are added in a fixed order afterwards.  Delta u(r) never goes to HBM.
// ------------------------------------------------------------------------------------------------
template <int N0, int N1>
__host__ __device__ constexpr int drho_group() {
    constexpr int P = PlaneCfg<float2, N0, N1>::P;
    return ((32 + P - 1) / P) * P;
}

// two resident CTAs per SM asked of the compiler for lines up to 45 points
template <int N0, int N1>
constexpr int drho_minb() { return (N0 <= 45 && N1 <= 45) ? 2 : 1; }

template <int N0, int N1, bool PR>
__global__ void __launch_bounds__(PlaneCfg<float2, N0, N1>::NT, drho_minb<N0, N1>()) drho_plane_kernel(
    const float2* __restrict__ colin, int ncmax, const int* __restrict__ kk, const int* __restrict__ spin,
    const int* __restrict__ ur_row, int c0, int nc, const int* __restrict__ xtab, int N2,
    const float2* __restrict__ ur, double2* __restrict__ part, int* __restrict__ mask, int group0) {
    using V = float2;
    using Cfg = PlaneCfg<V, N0, N1>;
    constexpr int P = Cfg::P, NT = Cfg::NT, LD = Cfg::LD, NP = N0 * N1, PS = N1 * LD, G = drho_group<N0, N1>();
    constexpr int EPT = (NP + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* S = (V*)smraw;          // [P][N1][LD]
    V* A = S + P * PS;         // [2][NP] the group's sums per spin (each point owned by one thread)
    __shared__ int sp_of[P];
    __shared__ long long u_of[P];  // offset of the band's plane z in ur
    __shared__ int seen;           // bit s: the group holds a band of spin s
    const int z = blockIdx.x, grp = blockIdx.y;
    const int b0 = grp * G, b1 = min(nc, b0 + G);
    const int tid = threadIdx.x;
    int myseen = 0;
    if (tid == 0) seen = 0;
    for (int e = tid; e < 2 * NP; e += NT) A[e] = cmkf(0.f, 0.f);
    for (int r0 = b0; r0 < b1; r0 += P) {
        if (tid < P) {
            const bool in = r0 + tid < b1;
            sp_of[tid] = in ? spin[c0 + r0 + tid] : -1;
            u_of[tid] = in ? ((long long)ur_row[c0 + r0 + tid] * N2 + z) * NP : 0;
            if (in) myseen |= 1 << sp_of[tid];
        }
        // y-inverse on the x-lines of each band's column runs (zero elsewhere)
        if (tid < P * YLines<N0, PR>::n) {
            const int p = tid / YLines<N0, PR>::n, x = YLines<N0, PR>::x(tid % YLines<N0, PR>::n);
            const int c = r0 + p;
            if (c < b1 && live<N0, PR>(x)) {
                const int k = kk[c0 + c];
                const int* t = xtab + ((long long)k * N0 + x) * 3;
                const int j0 = t[0], cnt = t[1], y0 = t[2];
                const V* src = colin + ((long long)c * N2 + z) * ncmax + j0;
                V a[N1];
#pragma unroll
                for (int y = 0; y < N1; ++y) {
                    int i = y - y0;
                    if (i < 0) i += N1;
                    a[y] = (live<N1, PR>(y) && i < cnt) ? src[i] : cmkf(0.f, 0.f);
                }
                if (cnt > 0) rfft<V, N1, +1>(a);
                V* col = S + p * PS + x;
#pragma unroll
                for (int y = 0; y < N1; ++y) col[y * LD] = a[y];
            }
        }
        __syncthreads();
        // x-inverse in place
        if (tid < P * N1) {
            const int p = tid / N1, y = tid % N1;
            if (r0 + p < b1) {
                V* rowp = S + p * PS + y * LD;
                V a[N0];
#pragma unroll
                for (int x = 0; x < N0; ++x) a[x] = live<N0, PR>(x) ? rowp[x] : cmkf(0.f, 0.f);
                rfft<V, N0, +1>(a);
#pragma unroll
                for (int x = 0; x < N0; ++x) rowp[x] = a[x];
            }
        }
        __syncthreads();
        // conj(u(r)) Delta u(r) of the round's bands into the per-spin sums, in band order; u(r) read
        // with consecutive threads on consecutive points, every load of a band issued before its sums
        const int np = min(P, b1 - r0);
        for (int p = 0; p < np; ++p) {
            const V* up = ur + u_of[p];
            V* Ap = A + sp_of[p] * NP;
            V u[EPT];
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const int e = tid + j * NT;
                if (e < NP) u[j] = __ldcs(up + e);
            }
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const int e = tid + j * NT;
                if (e < NP) {
                    const V d = S[p * PS + (e / N0) * LD + e % N0];
                    Ap[e] = cadd(Ap[e], cmkf(u[j].x * d.x + u[j].y * d.y, u[j].x * d.y - u[j].y * d.x));
                }
            }
        }
        __syncthreads();
    }
    if (myseen) atomicOr(&seen, myseen);
    __syncthreads();
    const int bits = seen;
    const long long nr = (long long)NP * N2;
    for (int sp = 0; sp < 2; ++sp) {
        if (!((bits >> sp) & 1)) continue;
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const int e = tid + j * NT;
            if (e < NP) {
                const V v = A[sp * NP + e];
                part[((long long)(group0 + grp) * 2 + sp) * nr + (long long)z * NP + e] = cmk((double)v.x, (double)v.y);
            }
        }
    }
    if (z == 0 && tid == 0) mask[group0 + grp] = bits;
}

template <int N0, int N1>
static cudaError_t drho_plane_launch(const FusedArgs& a, double2* part, int* mask, int group0) {
    using Cfg = PlaneCfg<float2, N0, N1>;
    if constexpr (!Cfg::ok) {
        return cudaErrorInvalidValue;
    } else {
        const SphereSet& S = *a.S;
        const BandList& L = *a.L;
        cudaError_t e = regfft_init();
        if (e != cudaSuccess) return e;
        const size_t smem = ((size_t)Cfg::P * N1 * Cfg::LD + 2 * (size_t)N0 * N1) * sizeof(float2);
        static const cudaError_t attr =
            cudaFuncSetAttribute(drho_plane_kernel<N0, N1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (attr != cudaSuccess) return attr;
        constexpr int G = drho_group<N0, N1>();
        dim3 g(a.N2, (a.nc + G - 1) / G);
        if constexpr (N0 >= 36 && N1 >= 36) {
            if (S.lines_prunable && !getenv("HP_NO_PRUNE")) {
                static const cudaError_t attr_p = cudaFuncSetAttribute(
                    drho_plane_kernel<N0, N1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (attr_p != cudaSuccess) return attr_p;
                drho_plane_kernel<N0, N1, true><<<g, Cfg::NT, smem, a.st>>>(
                    (const float2*)a.colA, S.ncmax, L.d_k, L.d_spin, L.d_row, a.c0, a.nc, S.d_xtab, a.N2,
                    (const float2*)a.ur, part, mask, group0);
                HP_LAUNCHED();
                return cudaGetLastError();
            }
        }
        drho_plane_kernel<N0, N1, false><<<g, Cfg::NT, smem, a.st>>>((const float2*)a.colA, S.ncmax, L.d_k, L.d_spin,
                                                                      L.d_row, a.c0, a.nc, S.d_xtab, a.N2,
                                                                      (const float2*)a.ur, part, mask, group0);
        HP_LAUNCHED();
        return cudaGetLastError();
    }
}

#define HP_DRHO_SIZES(M) M(10, 10) M(12, 12) M(15, 15) M(16, 16) M(18, 18) M(20, 20) M(24, 24) M(36, 36) M(45, 45) M(72, 45)

int fused_drho_groups(int n0, int n1, int nc) {
#define HP_DG(A0, A1) \
    if (n0 == A0 && n1 == A1) return (nc + drho_group<A0, A1>() - 1) / drho_group<A0, A1>();
    HP_DRHO_SIZES(HP_DG)
#undef HP_DG
    return 0;
}

bool fused_drho_supported(const FusedArgs& a) {
    const int n0 = a.N0, n1 = a.N1;
    const bool sizes = (n0 == n1 && (n0 == 10 || n0 == 12 || n0 == 15 || n0 == 16 || n0 == 18 || n0 == 20 ||
                                     n0 == 24 || n0 == 36 || n0 == 45)) ||
                       (n0 == 72 && n1 == 45);
    return sizes && a.reg && a.S->d_xtab && a.S->xtab_n0 == n0;
}

cudaError_t fused_drho(const FusedArgs& a, double2* part, int* mask, int group0) {
#define HP_DR(A0, A1) \
    if (a.N0 == A0 && a.N1 == A1) return drho_plane_launch<A0, A1>(a, part, mask, group0);
    HP_DRHO_SIZES(HP_DR)
#undef HP_DR
    return cudaErrorInvalidValue;
}

template <class T>
__global__ void planes_xmajor_kernel(const T* __restrict__ in, T* __restrict__ out, int N0, int N1, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long np = (long long)N0 * N1;
    const long long pl = i / np;
    const int r = (int)(i % np), x = r / N1, y = r % N1;
    out[i] = in[pl * np + (long long)y * N0 + x];
}

cudaError_t k_planes_xmajor(const void* in, void* out, int N0, int N1, long long nplanes, bool fp32, cudaStream_t st) {
    const long long n = nplanes * N0 * N1;
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256);
    if (fp32) planes_xmajor_kernel<float><<<blocks, 256, 0, st>>>((const float*)in, (float*)out, N0, N1, n);
    else planes_xmajor_kernel<double><<<blocks, 256, 0, st>>>((const double*)in, (double*)out, N0, N1, n);
    HP_LAUNCHED();
    return cudaGetLastError();
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
