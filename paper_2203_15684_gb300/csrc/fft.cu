// Batched 3D complex FFT for the plane-wave <-> real-space transforms of H.psi (the "FFT to real
// space, multiply by V_loc + V_Hxc, FFT back" step of every Sternheimer iteration, Sec. 2.3).
//
// Design: one kernel launch per axis.  A grid is viewed as [A][n][B] with the transformed axis of
// length n in the middle; a CTA stages a tile of LT lines (TA consecutive a's x TB consecutive b's)
// in shared memory with the line index fastest (conflict-free butterfly reads), runs every mixed-
// radix Stockham stage (radix 4, 2, 3, 5) in shared memory, and writes the tile back in place.
// Reads and writes of a tile are runs of TB contiguous complex numbers (whole lines when B = 1).
#include <cmath>
#include <cstdio>

#include "hp_internal.h"

namespace hp {

bool fft_factor(int n, Radices& out) {
    out.n = n;
    out.nst = 0;
    int m = n;
    while (m % 4 == 0 && out.nst < kMaxStages) { out.r[out.nst++] = 4; m /= 4; }
    while (m % 2 == 0 && out.nst < kMaxStages) { out.r[out.nst++] = 2; m /= 2; }
    while (m % 3 == 0 && out.nst < kMaxStages) { out.r[out.nst++] = 3; m /= 3; }
    while (m % 5 == 0 && out.nst < kMaxStages) { out.r[out.nst++] = 5; m /= 5; }
    return m == 1 && n >= 1;
}

// ---- one work item of one Stockham stage: butterfly j of line l (shared by host and device) ----
// src/dst: [n][LT] (line fastest).  Ns: product of the radices of the earlier stages.  V is double2
// (FP64 form) or float2 (FP32 form); the constants are rounded to the working precision.
template <class V>
HD void radix_butterfly(V* v, int R, int s) {
    using T = typename Scalar<V>::type;
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
        const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
        V t1 = cadd(v[1], v[2]);
        V t2 = csub(v[0], cscale(t1, (T)0.5));
        V t3 = cmul_si(cscale(csub(v[1], v[2]), h), s);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if (R == 5) {
        const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
        const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
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

template <class V>
HD void stockham_item(const V* src, V* dst, const V* tw, int n, int LT, int R, int Ns, int sign, int w) {
    const int l = w % LT;
    const int j = w / LT;
    const int nR = n / R;
    V v[5];
    const int k = j % Ns;
    const int tstep = k * (n / (Ns * R));
    for (int r = 0; r < R; ++r) {
        V x = src[(j + r * nR) * LT + l];
        if (r > 0 && tstep != 0) {
            V t = tw[(r * tstep) % n];
            if (sign > 0) t.y = -t.y;
            x = cmul(x, t);
        }
        v[r] = x;
    }
    radix_butterfly(v, R, sign);
    const int idxD = (j / Ns) * Ns * R + k;
    for (int r = 0; r < R; ++r) dst[(idxD + r * Ns) * LT + l] = v[r];
}

// ---- device kernel: one pass along the middle axis of [batch][A][n][B] ----
template <int LT, class V>
__global__ void __launch_bounds__(256) fft_axis_kernel(V* __restrict__ data, int A, int B, Radices rad,
                                                        const V* __restrict__ tw, int sign, int TA,
                                                        int TB, int tilesA, int tilesB) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V* sm = (V*)sm_raw;
    const int n = rad.n;
    V* buf0 = sm;
    V* buf1 = sm + n * LT;
    const int tile = blockIdx.x;
    const long long g = blockIdx.y;
    const int ta = tile / tilesB, tb = tile % tilesB;
    const int a0 = ta * TA, b0 = tb * TB;
    const long long gbase = g * (long long)A * n * B;
    const int nel = n * TA * TB;
    // load
    if (B == 1) {
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int i = e % n, la = e / n;
            const int a = a0 + la;
            V x = cpack<V>(0.0, 0.0);
            if (a < A) x = data[gbase + (long long)a * n + i];
            buf0[i * LT + la] = x;
        }
    } else {
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int lb = e % TB, rest = e / TB;
            const int la = rest % TA, i = rest / TA;
            const int a = a0 + la, b = b0 + lb;
            V x = cpack<V>(0.0, 0.0);
            if (a < A && b < B) x = data[gbase + ((long long)a * n + i) * B + b];
            buf0[i * LT + la * TB + lb] = x;
        }
    }
    __syncthreads();
    V* src = buf0;
    V* dst = buf1;
    int Ns = 1;
    for (int st = 0; st < rad.nst; ++st) {
        const int R = rad.r[st];
        const int items = LT * (n / R);
        for (int w = threadIdx.x; w < items; w += blockDim.x) stockham_item(src, dst, tw, n, LT, R, Ns, sign, w);
        __syncthreads();
        Ns *= R;
        V* t = src;
        src = dst;
        dst = t;
    }
    // store from src
    if (B == 1) {
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int i = e % n, la = e / n;
            const int a = a0 + la;
            if (a < A) data[gbase + (long long)a * n + i] = src[i * LT + la];
        }
    } else {
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int lb = e % TB, rest = e / TB;
            const int la = rest % TA, i = rest / TA;
            const int a = a0 + la, b = b0 + lb;
            if (a < A && b < B) data[gbase + ((long long)a * n + i) * B + b] = src[i * LT + la * TB + lb];
        }
    }
}


// ---- compile-time form of the pass: sizes, radices, strides and the sign are template constants,
// so every index division and modulo folds into multiplies and shifts and the stage loops unroll.
// Shared-memory rows are padded by one element (LDS = LT + 1) against bank conflicts when a warp
// loads consecutive points of one line.
template <int... R>
struct RadixList {};

template <int N> struct Factor;
template <> struct Factor<8> { using type = RadixList<4, 2>; };
template <> struct Factor<9> { using type = RadixList<3, 3>; };
template <> struct Factor<10> { using type = RadixList<2, 5>; };
template <> struct Factor<12> { using type = RadixList<4, 3>; };
template <> struct Factor<15> { using type = RadixList<3, 5>; };
template <> struct Factor<16> { using type = RadixList<4, 4>; };
template <> struct Factor<18> { using type = RadixList<2, 3, 3>; };
template <> struct Factor<20> { using type = RadixList<4, 5>; };
template <> struct Factor<24> { using type = RadixList<4, 2, 3>; };
template <> struct Factor<25> { using type = RadixList<5, 5>; };
template <> struct Factor<27> { using type = RadixList<3, 3, 3>; };
template <> struct Factor<30> { using type = RadixList<2, 3, 5>; };
template <> struct Factor<32> { using type = RadixList<4, 4, 2>; };
template <> struct Factor<36> { using type = RadixList<4, 3, 3>; };
template <> struct Factor<40> { using type = RadixList<4, 2, 5>; };
template <> struct Factor<45> { using type = RadixList<3, 3, 5>; };
template <> struct Factor<48> { using type = RadixList<4, 4, 3>; };
template <> struct Factor<50> { using type = RadixList<2, 5, 5>; };
template <> struct Factor<54> { using type = RadixList<2, 3, 3, 3>; };
template <> struct Factor<60> { using type = RadixList<4, 3, 5>; };
template <> struct Factor<64> { using type = RadixList<4, 4, 4>; };
template <> struct Factor<72> { using type = RadixList<4, 2, 3, 3>; };
template <> struct Factor<75> { using type = RadixList<3, 5, 5>; };
template <> struct Factor<80> { using type = RadixList<4, 4, 5>; };
template <> struct Factor<90> { using type = RadixList<2, 3, 3, 5>; };
template <> struct Factor<96> { using type = RadixList<4, 4, 2, 3>; };

constexpr int kFixedThreads = 128;
constexpr int kFixedLT = 16;
constexpr int kFixedLDS = kFixedLT + 1;

template <class V, int N, int SIGN, int NS, int R, int... Rest>
__device__ __forceinline__ V* fixed_stages(V* src, V* dst, const V* __restrict__ tw) {
    constexpr int NR = N / R;
    constexpr int ITEMS = kFixedLT * NR;
    constexpr int TSTEP = N / (NS * R);
#pragma unroll
    for (int w0 = 0; w0 < ITEMS; w0 += kFixedThreads) {
        const int w = w0 + (int)threadIdx.x;
        if ((ITEMS % kFixedThreads) == 0 || w < ITEMS) {
            const int l = w % kFixedLT;
            const int j = w / kFixedLT;
            const int k = j % NS;
            V v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                V x = src[(j + r * NR) * kFixedLDS + l];
                if (NS > 1 && r > 0) {
                    V t = tw[r * k * TSTEP];  // r k TSTEP < N: no wrap needed
                    if (SIGN > 0) t.y = -t.y;
                    x = cmul(x, t);
                }
                v[r] = x;
            }
            radix_butterfly(v, R, SIGN);
            const int idxD = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[(idxD + r * NS) * kFixedLDS + l] = v[r];
        }
    }
    __syncthreads();
    if constexpr (sizeof...(Rest) == 0) {
        return dst;
    } else {
        return fixed_stages<V, N, SIGN, NS * R, Rest...>(dst, src, tw);
    }
}

template <class V, int N, int SIGN, int... R>
__device__ __forceinline__ V* fixed_all(RadixList<R...>, V* src, V* dst, const V* __restrict__ tw) {
    return fixed_stages<V, N, SIGN, 1, R...>(src, dst, tw);
}

template <class V, int N, int SIGN, bool CONTIG>
__global__ void __launch_bounds__(kFixedThreads) fft_fixed_kernel(V* __restrict__ data, int A, int B,
                                                                  const V* __restrict__ tw, int TA, int TB, int tilesB) {
    __shared__ V sm[2 * N * kFixedLDS];
    V* buf0 = sm;
    V* buf1 = sm + N * kFixedLDS;
    const int tile = blockIdx.x;
    const long long gbase = (long long)blockIdx.y * A * N * B;
    const int ta = tile / tilesB, tb = tile % tilesB;
    const int a0 = ta * TA, b0 = tb * TB;
    if (CONTIG) {  // B == 1: TA = LT whole lines, contiguous
        constexpr int NEL = N * kFixedLT;
#pragma unroll 4
        for (int e = threadIdx.x; e < NEL; e += kFixedThreads) {
            const int i = e % N, la = e / N;
            const int a = a0 + la;
            V x = cpack<V>(0.0, 0.0);
            if (a < A) x = data[gbase + (long long)a * N + i];
            buf0[i * kFixedLDS + la] = x;
        }
    } else {
        const int nel = N * TA * TB;
        for (int e = threadIdx.x; e < nel; e += kFixedThreads) {
            const int lb = e % TB, rest = e / TB;
            const int la = rest % TA, i = rest / TA;
            const int a = a0 + la, b = b0 + lb;
            V x = cpack<V>(0.0, 0.0);
            if (a < A && b < B) x = data[gbase + ((long long)a * N + i) * B + b];
            buf0[i * kFixedLDS + la * TB + lb] = x;
        }
    }
    __syncthreads();
    V* out = fixed_all<V, N, SIGN>(typename Factor<N>::type{}, buf0, buf1, tw);
    if (CONTIG) {
        constexpr int NEL = N * kFixedLT;
#pragma unroll 4
        for (int e = threadIdx.x; e < NEL; e += kFixedThreads) {
            const int i = e % N, la = e / N;
            const int a = a0 + la;
            if (a < A) data[gbase + (long long)a * N + i] = out[i * kFixedLDS + la];
        }
    } else {
        const int nel = N * TA * TB;
        for (int e = threadIdx.x; e < nel; e += kFixedThreads) {
            const int lb = e % TB, rest = e / TB;
            const int la = rest % TA, i = rest / TA;
            const int a = a0 + la, b = b0 + lb;
            if (a < A && b < B) data[gbase + ((long long)a * N + i) * B + b] = out[i * kFixedLDS + la * TB + lb];
        }
    }
}

// launches the compile-time pass for size n if it is one of the listed sizes; returns false otherwise
template <class V, int N>
static bool launch_fixed_n(V* data, int A, int B, const V* tw, int sign, int nb, cudaStream_t st) {
    if constexpr (sizeof(V) * 2 * N * kFixedLDS > 48 * 1024) {
        return false;  // beyond static shared memory: the runtime-size pass takes it
    }
    int TB = B < kFixedLT ? B : kFixedLT;
    int TA = kFixedLT / TB;
    if (TA < 1) TA = 1;
    const int tilesA = (A + TA - 1) / TA, tilesB = (B + TB - 1) / TB;
    dim3 grid(tilesA * tilesB, nb);
    if (B == 1) {
        if (sign > 0) fft_fixed_kernel<V, N, 1, true><<<grid, kFixedThreads, 0, st>>>(data, A, B, tw, TA, TB, tilesB);
        else fft_fixed_kernel<V, N, -1, true><<<grid, kFixedThreads, 0, st>>>(data, A, B, tw, TA, TB, tilesB);
    } else {
        if (sign > 0) fft_fixed_kernel<V, N, 1, false><<<grid, kFixedThreads, 0, st>>>(data, A, B, tw, TA, TB, tilesB);
        else fft_fixed_kernel<V, N, -1, false><<<grid, kFixedThreads, 0, st>>>(data, A, B, tw, TA, TB, tilesB);
    }
    return true;
}

template <class V>
static bool launch_fixed(int n, V* data, int A, int B, const V* tw, int sign, int nb, cudaStream_t st) {
    switch (n) {
#define HP_FIXED(NN) \
    case NN: return launch_fixed_n<V, NN>(data, A, B, tw, sign, nb, st);
        HP_FIXED(8) HP_FIXED(9) HP_FIXED(10) HP_FIXED(12) HP_FIXED(15) HP_FIXED(16) HP_FIXED(18) HP_FIXED(20)
        HP_FIXED(24) HP_FIXED(25) HP_FIXED(27) HP_FIXED(30) HP_FIXED(32) HP_FIXED(36) HP_FIXED(40) HP_FIXED(45)
        HP_FIXED(48) HP_FIXED(50) HP_FIXED(54) HP_FIXED(60) HP_FIXED(64) HP_FIXED(72) HP_FIXED(75) HP_FIXED(80)
        HP_FIXED(90) HP_FIXED(96)
#undef HP_FIXED
        default: return false;
    }
}

cudaError_t fft_plan_create(hp_ctx* c, FftPlan& p, const int N[3]) {
    for (int d = 0; d < 3; ++d) {
        p.N[d] = N[d];
        if (!fft_factor(N[d], p.ax[d].rad)) return cudaErrorInvalidValue;
        std::vector<double2> tw(N[d]);
        for (int t = 0; t < N[d]; ++t) {
            const double a = -2.0 * M_PI * (double)t / (double)N[d];
            tw[t] = cmk(std::cos(a), std::sin(a));
        }
        cudaError_t e = dalloc(c, &p.ax[d].d_tw, N[d]);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(p.ax[d].d_tw, tw.data(), sizeof(double2) * N[d], cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        std::vector<float2> tw32(N[d]);
        for (int t = 0; t < N[d]; ++t) tw32[t] = cmkf((float)tw[t].x, (float)tw[t].y);
        e = dalloc(c, &p.ax[d].d_tw32, N[d]);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(p.ax[d].d_tw32, tw32.data(), sizeof(float2) * N[d], cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void fft_plan_destroy(FftPlan& p) {  // the tables themselves are freed with the context's allocations
    for (int d = 0; d < 3; ++d) {
        p.ax[d].d_tw = nullptr;
        p.ax[d].d_tw32 = nullptr;
    }
}

static constexpr int kLT = 16;

template <class V>
static const V* twiddles(const FftAxis& a);
template <>
const double2* twiddles<double2>(const FftAxis& a) { return a.d_tw; }
template <>
const float2* twiddles<float2>(const FftAxis& a) { return a.d_tw32; }

template <class V>
static cudaError_t fft3d_impl(const FftPlan& p, V* data, int nb, int sign, cudaStream_t st) {
    const int N0 = p.N[0], N1 = p.N[1], N2 = p.N[2];
    // axis d: A = prod of earlier dims, B = prod of later dims
    const int As[3] = {1, N0, N0 * N1};
    const int Bs[3] = {N1 * N2, N2, 1};
    // order: contiguous axis first for the forward-to-real (any order gives the same result)
    const int order[3] = {2, 1, 0};
    for (int oi = 0; oi < 3; ++oi) {
        const int d = order[oi];
        const int A = As[d], B = Bs[d], n = p.N[d];
        int TB = B < kLT ? B : kLT;
        int TA = kLT / TB;
        if (TA < 1) TA = 1;
        const int tilesA = (A + TA - 1) / TA, tilesB = (B + TB - 1) / TB;
        const size_t smem = 2 * sizeof(V) * n * kLT;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(fft_axis_kernel<kLT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        dim3 grid(tilesA * tilesB, nb);
        const ProfMark pm = prof_start(st);
        if (!launch_fixed<V>(n, data, A, B, twiddles<V>(p.ax[d]), sign, nb, st))
            fft_axis_kernel<kLT, V><<<grid, 128, smem, st>>>(data, A, B, p.ax[d].rad, twiddles<V>(p.ax[d]), sign, TA, TB,
                                                             tilesA, tilesB);
        HP_LAUNCHED();
        if (prof_on()) {
            const double nrg = (double)N0 * N1 * N2 * nb;
            // 5 n log2 n flops per line of n points; every point read and written once
            prof_stop(pm, HP_KF_FFT_PASS, st, nrg * 5.0 * std::log2((double)n), nrg * 2.0 * sizeof(V));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t fft3d(const FftPlan& p, double2* data, int nb, int sign, cudaStream_t st) {
    return fft3d_impl(p, data, nb, sign, st);
}

cudaError_t fft3d(const FftPlan& p, float2* data, int nb, int sign, cudaStream_t st) {
    return fft3d_impl(p, data, nb, sign, st);
}

void fft_host_lines(const Radices& rad, const std::vector<double2>& tw, int nlines, int sign, double2* data) {
    const int n = rad.n;
    std::vector<double2> b0(n * nlines), b1(n * nlines);
    for (int l = 0; l < nlines; ++l)
        for (int i = 0; i < n; ++i) b0[i * nlines + l] = data[l * n + i];
    double2* src = b0.data();
    double2* dst = b1.data();
    int Ns = 1;
    for (int s = 0; s < rad.nst; ++s) {
        const int R = rad.r[s];
        for (int w = 0; w < nlines * (n / R); ++w) stockham_item(src, dst, tw.data(), n, nlines, R, Ns, sign, w);
        Ns *= R;
        double2* t = src;
        src = dst;
        dst = t;
    }
    for (int l = 0; l < nlines; ++l)
        for (int i = 0; i < n; ++i) data[l * n + i] = src[i * nlines + l];
}

}  // namespace hp

extern "C" long long hp_launch_count(void) { return hp::g_launches.load(); }

extern "C" long long hp_alloc_count(void) { return hp::g_allocs.load(); }

extern "C" hp_status hp_selftest_fft_host(int n, int nlines, int sign, const double* in, double* out) {
    if (n < 1 || nlines < 1 || !in || !out || (sign != 1 && sign != -1)) return HP_EINVAL;
    hp::Radices rad;
    if (!hp::fft_factor(n, rad)) return HP_EINVAL;
    std::vector<double2> tw(n);
    for (int t = 0; t < n; ++t) {
        const double a = -2.0 * M_PI * (double)t / (double)n;
        tw[t] = hp::cmk(std::cos(a), std::sin(a));
    }
    std::vector<double2> d(n * nlines);
    for (int i = 0; i < n * nlines; ++i) d[i] = hp::cmk(in[2 * i], in[2 * i + 1]);
    hp::fft_host_lines(rad, tw, nlines, sign, d.data());
    for (int i = 0; i < n * nlines; ++i) {
        out[2 * i] = d[i].x;
        out[2 * i + 1] = d[i].y;
    }
    return HP_OK;
}
