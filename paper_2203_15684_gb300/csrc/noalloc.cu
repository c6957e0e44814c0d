// H.psi without any device allocation at call time.
//
// Some callers cannot call cudaMalloc while they compute: applications that hand all free device
// memory to their own pool allocator at start-up, and loops that must not call cudaMalloc/cudaFree
// because those calls can synchronise the whole device.  hp_apply_h_noalloc serves them: it runs
// the same kernels as hp_apply_h (scatter, FFT passes, local potential, gather with the kinetic
// term, nonlocal projections) on caller-owned device input and output, and keeps every piece of
// scratch (band list, FFT grids, projections, split-K partial sums) in one fixed file-scope device
// array instead of allocating it.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "hp_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;  // 64 MiB, held by every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The name of a __device__ array in
// host code is only a host-side stand-in, so the address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
hp_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HP_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HP_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" hp_status hp_apply_h_noalloc(hp_ctx* c, int ik, int spin, int nb, const double* psi_dev, double* out_dev,
                                        void* stream) {
    using namespace hp;
    if (!c) return HP_EINVAL;
    if (!c->have_gs) return fail(c, HP_ESTATE, "hp_apply_h_noalloc: no ground state (potential) yet");
    if (c->hub_on) return fail(c, HP_ENOTIMPL, "hp_apply_h_noalloc: no Hubbard-corrected (DFT+U+V) operator");
    if (ik < 0 || ik >= c->nk || spin < 0 || spin >= c->nspin || nb < 1 || !psi_dev || !out_dev)
        return fail(c, HP_EINVAL, "hp_apply_h_noalloc: bad arguments");
    // the context's buffers (potential, projectors, sphere tables) live on the device current at
    // hp_setup; the scratch array is looked up on the current device, so both must be the same
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(c, HP_ECUDA, "hp_apply_h_noalloc: cudaGetDevice failed");
    if (dev != c->device) {
        char msg[160];
        snprintf(msg, sizeof(msg), "hp_apply_h_noalloc: current device %d is not the context's device %d", dev,
                 c->device);
        return fail(c, HP_EINVAL, msg);
    }
    cudaStream_t st = stream ? (cudaStream_t)stream : c->st;
    const int ld = c->ld, nr = c->nr;
    constexpr int kPS = 128;
    // layout of the fixed scratch: band list | projections | split-K partials | FFT grids
    const size_t b_ints = align256(sizeof(int) * (size_t)(3 * nb + 4));
    const size_t b_shift = align256(sizeof(double) * (size_t)nb);
    const size_t b_proj = align256(sizeof(double2) * (size_t)nb * kPS);
    const size_t b_part = b_proj;  // one split at least
    const size_t b_grid1 = sizeof(double2) * (size_t)nr;
    const size_t fixed = b_ints + b_shift + b_proj + b_part;
    if (fixed + b_grid1 > kNoallocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "hp_apply_h_noalloc: %d bands on a %d-point grid need more than the fixed %zu MiB scratch; "
                 "call it on fewer bands",
                 nb, nr, kNoallocScratchBytes >> 20);
        return fail(c, HP_EINVAL, msg);
    }
    void* base = nullptr;
    hp_status s = scratch_address(&base);
    if (s != HP_OK) return fail(c, s, "hp_apply_h_noalloc: cudaGetSymbolAddress of the scratch array failed");
    unsigned char* p = (unsigned char*)base;
    int* d_ints = (int*)p;
    double* d_shift = (double*)(p + b_ints);
    double2* d_P = (double2*)(p + b_ints + b_shift);
    double2* d_part = (double2*)(p + b_ints + b_shift + b_proj);
    double2* d_grid = (double2*)(p + fixed);
    const int chunk = (int)std::min<size_t>((size_t)nb, (kNoallocScratchBytes - fixed) / b_grid1);
    // the band list lives in the scratch; its host copy is uploaded with plain copies
    BandList L;
    L.nb = nb;
    L.nseg = 1;
    L.row.resize(nb);
    L.k.assign(nb, ik);
    L.spin.assign(nb, spin);
    L.shift.assign(nb, 0.0);
    for (int b = 0; b < nb; ++b) L.row[b] = b;
    L.seg_start = {0, nb};
    L.seg_k = {ik};
    L.seg_s = {spin};
    std::vector<int> ints(3 * nb + 4);
    memcpy(ints.data(), L.row.data(), sizeof(int) * nb);
    memcpy(ints.data() + nb, L.k.data(), sizeof(int) * nb);
    memcpy(ints.data() + 2 * nb, L.spin.data(), sizeof(int) * nb);
    ints[3 * nb] = 0;
    ints[3 * nb + 1] = nb;
    ints[3 * nb + 2] = ik;
    ints[3 * nb + 3] = spin;
    L.d_row = d_ints;
    L.d_k = d_ints + nb;
    L.d_spin = d_ints + 2 * nb;
    L.d_seg_start = d_ints + 3 * nb;
    L.d_seg_k = d_ints + 3 * nb + 2;
    L.d_seg_s = d_ints + 3 * nb + 3;
    L.d_shift = d_shift;
    CK(cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_shift, L.shift.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    const double2* X = (const double2*)psi_dev;
    double2* Y = (double2*)out_dev;
    // local part and kinetic energy, chunk by chunk through the FFT grids (zeroed by the scatter)
    for (int c0 = 0; c0 < nb; c0 += chunk) {
        const int nc = std::min(chunk, nb - c0);
        CK(k_scatter(c->kset, L, c0, nc, X, ld, d_grid, nr, st));
        CK(fft3d(c->fft, d_grid, nc, +1, st));
        CK(k_mul_rpot(d_grid, nc, nr, c->d_veff, L, c0, st));
        CK(fft3d(c->fft, d_grid, nc, -1, st));
        CK(k_gather_h(c->kset, L, c0, nc, d_grid, nr, X, Y, ld, st));
    }
    // nonlocal part: every projection and partial sum is written before it is read
    if (c->nproj > 0) {
        ProjMat B{c->d_beta_k, 0, (long long)c->nproj * ld, c->nproj, 0, nullptr};
        CK(k_proj(L, c->kset, B, X, ld, d_P, d_part, b_part / sizeof(double2), st));
        CK(k_expand(L, c->kset, B, d_P, c->d_projD, 1.0, Y, ld, st));
    }
    CK(cudaStreamSynchronize(st));
    return HP_OK;
}
