// profile.cu -- opt-in per-kernel event timing and the launch counter (benchmarking aid).
#include <atomic>
#include <mutex>
#include <vector>

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

struct Rec {
    int kind;
    cudaEvent_t a, b;
};

std::atomic<long long> g_launches{0};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;

cudaEvent_t take_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

ProfScope::ProfScope(int kind, cudaStream_t s) : kind_(kind), s_(s), a_(nullptr) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s_);
    g_recs.push_back(Rec{kind_, static_cast<cudaEvent_t>(a_), b});
}

}  // namespace dvgo

extern "C" {

int dvgo_profile_enable(int on) {
    dvgo::g_on.store(on != 0);
    return DVGO_OK;
}

int dvgo_profile_read(int kind, double *total_ms, long long *launches) {
    using namespace dvgo;
    if (kind < 0 || kind >= DVGO_K_COUNT || !total_ms || !launches) return DVGO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    double tot = 0.0;
    long long n = 0;
    std::vector<Rec> keep;
    for (const Rec &r : g_recs) {
        if (r.kind != kind) {
            keep.push_back(r);
            continue;
        }
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            return DVGO_ERR_CUDA;
        tot += ms;
        ++n;
        g_free.push_back(r.a);
        g_free.push_back(r.b);
    }
    g_recs.swap(keep);
    *total_ms = tot;
    *launches = n;
    return DVGO_OK;
}

int dvgo_profile_trace(int max_records, int *kinds, double *start_ms, double *end_ms, int *n_out) {
    using namespace dvgo;
    if (max_records < 0 || !n_out || (max_records > 0 && (!kinds || !start_ms || !end_ms)))
        return DVGO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    const int n = (int)g_recs.size() < max_records ? (int)g_recs.size() : max_records;
    int st = DVGO_OK;
    if (!g_recs.empty() && cudaEventSynchronize(g_recs.back().b) != cudaSuccess) st = DVGO_ERR_CUDA;
    for (int i = 0; i < n && st == DVGO_OK; ++i) {
        const Rec &r = g_recs[i];
        float a = 0.0f, b = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess ||
            cudaEventElapsedTime(&a, g_recs[0].a, r.a) != cudaSuccess ||
            cudaEventElapsedTime(&b, g_recs[0].a, r.b) != cudaSuccess) {
            st = DVGO_ERR_CUDA;
            break;
        }
        kinds[i] = r.kind;
        start_ms[i] = a;
        end_ms[i] = b;
    }
    for (const Rec &r : g_recs) {
        g_free.push_back(r.a);
        g_free.push_back(r.b);
    }
    g_recs.clear();
    *n_out = st == DVGO_OK ? n : 0;
    return st;
}

long long dvgo_launch_counter(void) { return dvgo::g_launches.load(); }

}  // extern "C"
