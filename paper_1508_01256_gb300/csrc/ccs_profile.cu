// ccs_profile.cu -- launch counting and optional per-kernel event timing.
#include <atomic>
#include <mutex>
#include <vector>

#include "ccs_internal.cuh"

namespace ccs {

namespace {
struct Pending {
    int kind;
    cudaEvent_t start, stop;
};
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
ccs_kernel_time g_times[CCS_K_COUNT];

cudaEvent_t take_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

bool profiling() { return g_on; }

int prof_start(int kind, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return -1;
    Pending p{kind, take_event(), take_event()};
    if (!p.start || !p.stop) return -1;
    cudaEventRecord(p.start, s);
    g_pending.push_back(p);
    return (int)g_pending.size() - 1;
}

void prof_stop(int slot, cudaStream_t s) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].stop, s);
}

// Call after the stream has been synchronised: folds finished pairs into the
// per-kind totals.
void prof_collect() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            g_times[p.kind].launches += 1;
            g_times[p.kind].total_ms += ms;
        }
        g_free.push_back(p.start);
        g_free.push_back(p.stop);
    }
    g_pending.clear();
}

void prof_add(int kind, double ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    g_times[kind].launches += 1;
    g_times[kind].total_ms += ms;
}

}  // namespace ccs

using namespace ccs;

extern "C" int ccs_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &t : g_times) t = ccs_kernel_time{0, 0.0};
    g_pending.clear();
    g_on = true;
    return CCS_OK;
}

extern "C" int ccs_profile_end(ccs_kernel_time *times) {
    prof_collect();
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = false;
    if (times)
        for (int k = 0; k < CCS_K_COUNT; ++k) times[k] = g_times[k];
    return CCS_OK;
}

extern "C" int64_t ccs_launch_count(void) { return g_launches.load(); }
