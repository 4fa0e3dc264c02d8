// Opt-in per-kernel-group timing, switched on by KLST_TIMING=1 in the environment (totals are
// printed to stderr after every klst_eigs) or by klst_prof_enable(1) (totals accumulate until
// klst_prof_reset and are read with klst_prof_entry).  Events are recorded on the launching
// stream around each group of launches; with timing off the library never touches this code
// beyond one flag test.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace klst {

static std::atomic<unsigned long long> g_launches{0};
// While a thread captures a CUDA graph its launches are recorded, not run: they are counted when
// the graph is launched (note_launches with the graph's kernel-node count).
static thread_local bool t_capturing = false;
void set_capturing(bool on) { t_capturing = on; }
std::mutex& attr_mutex() {
    static std::mutex m;
    return m;
}

void note_launch() {
    if (!t_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void note_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_recs;
static std::map<std::string, cudaEvent_t> g_open;
static std::map<std::string, std::pair<double, long>> g_sum;
static std::atomic<int> g_prof_api{0};

static bool env_timing() {
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("KLST_TIMING");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on == 1;
}

bool prof_enabled() { return g_prof_api.load(std::memory_order_relaxed) || env_timing(); }

// caller holds g_prof_mu; waits for every pending record and folds it into the totals
static void resolve_locked() {
    for (auto& r : g_recs) {
        float ms = 0;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto& acc = g_sum[r.name];
        acc.first += ms;
        acc.second += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
}

void prof_begin(const char* name, cudaStream_t s) {
    if (!prof_enabled()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    g_open[name] = e;
}

void prof_end(const char* name, cudaStream_t s) {
    if (!prof_enabled()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto it = g_open.find(name);
    if (it == g_open.end()) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    g_recs.push_back({name, it->second, e});
    g_open.erase(it);
    if (g_recs.size() > 200000) resolve_locked();
}

void prof_report(cudaStream_t s) {
    if (!env_timing()) return;
    cudaStreamSynchronize(s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_locked();
    fprintf(stderr, "[klst timing] %-22s %12s %8s %10s\n", "group", "total ms", "calls", "ms/call");
    for (auto& kv : g_sum)
        fprintf(stderr, "[klst timing] %-22s %12.3f %8ld %10.4f\n", kv.first.c_str(), kv.second.first, kv.second.second,
                kv.second.first / (kv.second.second ? kv.second.second : 1));
    if (!g_prof_api.load()) g_sum.clear();
}

}  // namespace klst

using namespace klst;

extern "C" void klst_debug_fail_alloc_after(int64_t n) { klst::fail_alloc_after(n); }

extern "C" unsigned long long klst_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" void klst_prof_enable(int32_t on) { g_prof_api.store(on ? 1 : 0); }

extern "C" void klst_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_locked();
    g_sum.clear();
    g_open.clear();
}

extern "C" int32_t klst_prof_entry(int32_t i, char* name, int32_t name_cap, double* total_ms, int64_t* calls) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_locked();
    const int32_t count = (int32_t)g_sum.size();
    if (i < 0 || i >= count) return count;
    auto it = g_sum.begin();
    std::advance(it, i);
    if (name && name_cap > 0) {
        strncpy(name, it->first.c_str(), (size_t)name_cap - 1);
        name[name_cap - 1] = '\0';
    }
    if (total_ms) *total_ms = it->second.first;
    if (calls) *calls = it->second.second;
    return count;
}
