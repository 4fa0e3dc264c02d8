// Opt-in per-kernel-group timing (KLST_TIMING=1).  Events are recorded on the launching stream
// and resolved when klst_eigs reports; the library's normal path never touches this code.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace klst {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_recs;
static std::map<std::string, cudaEvent_t> g_open;
static std::map<std::string, std::pair<double, long>> g_sum;

bool prof_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("KLST_TIMING");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on == 1;
}

void prof_begin(const char* name, cudaStream_t s) {
    if (!prof_enabled()) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    g_open[name] = e;
}

void prof_end(const char* name, cudaStream_t s) {
    if (!prof_enabled()) return;
    auto it = g_open.find(name);
    if (it == g_open.end()) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    g_recs.push_back({name, it->second, e});
    g_open.erase(it);
    if (g_recs.size() > 20000) {
        cudaStreamSynchronize(s);
        for (auto& r : g_recs) {
            float ms = 0;
            cudaEventElapsedTime(&ms, r.a, r.b);
            auto& acc = g_sum[r.name];
            acc.first += ms;
            acc.second += 1;
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        g_recs.clear();
    }
}

void prof_report(cudaStream_t s) {
    if (!prof_enabled()) return;
    cudaStreamSynchronize(s);
    for (auto& r : g_recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto& acc = g_sum[r.name];
        acc.first += ms;
        acc.second += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
    fprintf(stderr, "[klst timing] %-22s %12s %8s %10s\n", "group", "total ms", "calls", "ms/call");
    for (auto& kv : g_sum)
        fprintf(stderr, "[klst timing] %-22s %12.3f %8ld %10.4f\n", kv.first.c_str(), kv.second.first, kv.second.second,
                kv.second.first / (kv.second.second ? kv.second.second : 1));
    g_sum.clear();
}

}  // namespace klst

extern "C" unsigned long long klst_launch_count(void) { return klst::g_launches.load(std::memory_order_relaxed); }
