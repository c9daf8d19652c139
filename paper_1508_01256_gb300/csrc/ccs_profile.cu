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
std::vector<unsigned long long> g_stamps;  // last persistent launch, device ns
int g_sub_base = 0;

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

void prof_keep_stamps(const unsigned long long *st, int count, int sub_base) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stamps.assign(st, st + count);
    g_sub_base = sub_base;
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

extern "C" int ccs_profile_phases(int32_t iteration, double *phase_us) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!phase_us || iteration < 0) return CCS_EINVAL;
    const size_t b0 = 2 * (size_t)iteration, b1 = b0 + 1, b2 = b0 + 2;
    const size_t s0 = (size_t)g_sub_base + 3 * (size_t)iteration;
    if (g_stamps.empty() || s0 + 2 >= g_stamps.size() || b2 >= (size_t)g_sub_base) return CCS_EINVAL;
    const unsigned long long t0 = g_stamps[b0], t1 = g_stamps[b1], t2 = g_stamps[b2];
    const unsigned long long f = g_stamps[s0], st = g_stamps[s0 + 1], q = g_stamps[s0 + 2];
    if (!t0 || !t1 || !t2 || t1 < t0 || t2 < t1) return CCS_EINVAL;
    phase_us[0] = (t1 - t0) * 1e-3;
    phase_us[1] = (t2 - t1) * 1e-3;
    phase_us[2] = (f >= t0 && f) ? (f - t0) * 1e-3 : -1.0;
    phase_us[3] = (st >= f && f) ? (st - f) * 1e-3 : -1.0;
    phase_us[4] = (q >= st && st) ? (q - st) * 1e-3 : -1.0;
    return CCS_OK;
}
