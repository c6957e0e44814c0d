// Live timing of the hot kernel families with CUDA events recorded on each launch's own stream.
//
// Between hp_profile_begin and hp_profile_end every launch of a timed family (FFT passes, fused
// column transforms, fused plane transforms, projections, expansions) is bracketed by a pair of
// events; each launch also adds its algorithmic flops and bytes, counted on the host from the sizes
// it processes.  hp_profile_end waits for the events and returns per-family sums.  The profiler is
// process-wide and meant for one host thread driving the library.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hp_internal.h"

namespace hp {

namespace {

struct Rec {
    int fam;
    cudaEvent_t e0, e1;
};

struct Prof {
    bool on = false;
    std::vector<Rec> rec;
    std::vector<cudaEvent_t> pool;  // events kept across profiles
    size_t used = 0;
    long long launches[HP_KF_COUNT] = {};
    double flops[HP_KF_COUNT] = {}, bytes[HP_KF_COUNT] = {};
};

Prof g_prof;

cudaEvent_t take_event() {
    if (g_prof.used == g_prof.pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_prof.pool.push_back(e);
    }
    return g_prof.pool[g_prof.used++];
}

}  // namespace

bool prof_on() { return g_prof.on; }

ProfMark prof_start(cudaStream_t st) {
    ProfMark m;
    if (!g_prof.on) return m;
    m.e0 = take_event();
    if (m.e0) cudaEventRecord(m.e0, st);
    return m;
}

void prof_stop(const ProfMark& m, int fam, cudaStream_t st, double flops, double bytes, const char* tag) {
    if (!g_prof.on || !m.e0 || fam < 0 || fam >= HP_KF_COUNT) return;
    static FILE* log = [] {
        const char* path = getenv("HP_PROF_LOG");
        return path ? fopen(path, "a") : nullptr;
    }();
    if (log) {
        fprintf(log, "%d %s %.0f %.0f\n", fam, tag ? tag : "-", bytes, flops);
        fflush(log);
    }
    cudaEvent_t e1 = take_event();
    if (!e1) return;
    cudaEventRecord(e1, st);
    g_prof.rec.push_back(Rec{fam, m.e0, e1});
    g_prof.launches[fam] += 1;
    g_prof.flops[fam] += flops;
    g_prof.bytes[fam] += bytes;
}

}  // namespace hp

extern "C" void hp_profile_begin(void) {
    using hp::g_prof;
    std::vector<cudaEvent_t> pool;
    pool.swap(g_prof.pool);
    g_prof = hp::Prof();
    g_prof.pool.swap(pool);
    g_prof.on = true;
}

extern "C" hp_status hp_profile_end(hp_kernel_stats* stats) {
    using hp::g_prof;
    cudaError_t err = cudaSuccess;
    double ms[HP_KF_COUNT] = {};
    for (const auto& r : g_prof.rec) {
        cudaError_t e = cudaEventSynchronize(r.e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.e0, r.e1);
        if (e != cudaSuccess) err = e;
        ms[r.fam] += t;
    }
    if (stats)
        for (int f = 0; f < HP_KF_COUNT; ++f) {
            stats[f].ms = ms[f];
            stats[f].launches = g_prof.launches[f];
            stats[f].flops = g_prof.flops[f];
            stats[f].bytes = g_prof.bytes[f];
        }
    std::vector<cudaEvent_t> pool;
    pool.swap(g_prof.pool);
    g_prof = hp::Prof();
    g_prof.pool.swap(pool);
    return err == cudaSuccess ? HP_OK : HP_ECUDA;
}
