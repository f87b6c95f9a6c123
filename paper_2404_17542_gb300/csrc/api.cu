// Error reporting, version and kernel instrumentation of the C ABI.
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "krylov_common.cuh"

namespace mcd {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

// ---- instrumentation --------------------------------------------------
static std::atomic<long long> g_launches{0};

struct EventPair {
    cudaEvent_t a, b;
    int kind;
};

struct Timing {
    std::mutex mu;
    int sample_every = 0;
    long long seen[MCD_K_COUNT] = {0};
    std::vector<EventPair> used;
    std::vector<EventPair> pool;
};
static Timing g_timing;
static const size_t kMaxPairs = 1 << 16;

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

KTimer::KTimer(int kind, cudaStream_t s, int nlaunch) : kind_(kind), stream_(s), active_(false) {
    g_launches.fetch_add(nlaunch, std::memory_order_relaxed);
    if (g_timing.sample_every <= 0) return;
    std::lock_guard<std::mutex> lk(g_timing.mu);
    if (g_timing.seen[kind]++ % g_timing.sample_every != 0) return;
    if (g_timing.used.size() >= kMaxPairs) return;
    EventPair ep;
    if (!g_timing.pool.empty()) {
        ep = g_timing.pool.back();
        g_timing.pool.pop_back();
    } else if (cudaEventCreate(&ep.a) != cudaSuccess || cudaEventCreate(&ep.b) != cudaSuccess) {
        return;
    }
    ep.kind = kind;
    if (cudaEventRecord(ep.a, s) != cudaSuccess) return;
    a_ = ep.a;
    b_ = ep.b;
    g_timing.used.push_back(ep);
    active_ = true;
}

KTimer::~KTimer() {
    if (active_) cudaEventRecord(b_, stream_);
}

// Probe of the grid barriers' bounded wait: thread 0 polls `word` for
// `expect` with wait_eq and records 1 if it saw it, 0 if the wait gave up.
__global__ void wait_probe_kernel(const unsigned *word, unsigned expect, long long polls, int *seen) {
    if (threadIdx.x == 0) *seen = wait_eq(word, expect, polls) ? 1 : 0;
}

}  // namespace mcd

using namespace mcd;

extern "C" mcd_status mcd_selftest_bounded_wait(int set_flag, int64_t polls, mcd_stream_t stream) {
    MCD_CHECK_ARG(polls >= 1 && polls <= (int64_t(1) << 20), "polls must be in [1, 2^20]");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *buf = nullptr;   // [0] the polled word, [1] the result
    if (cudaMalloc(&buf, 2 * sizeof(unsigned)) != cudaSuccess) {
        set_error("bounded-wait self-test: cudaMalloc failed");
        return MCD_ECUDA;
    }
    int seen = -1;
    cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess && set_flag) e = cudaMemsetAsync(buf, 0x01, 1, s);   // word = 1 (little endian)
    if (e == cudaSuccess) {
        wait_probe_kernel<<<1, 32, 0, s>>>(buf, 1u, (long long)polls, reinterpret_cast<int *>(buf + 1));
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&seen, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_error(std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
        return MCD_ECUDA;
    }
    if (seen != 1) {
        set_error("bounded-wait self-test: the wait gave up after " + std::to_string(polls) + " polls");
        return MCD_ETIMEOUT;
    }
    return MCD_OK;
}

extern "C" const char *mcd_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *mcd_version(void) { return "mcd-gb300 0.1 (sm_103a)"; }

extern "C" int64_t mcd_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" mcd_status mcd_timing_enable(int sample_every) {
    MCD_CHECK_ARG(sample_every >= 0, "sample_every must be >= 0");
    std::lock_guard<std::mutex> lk(g_timing.mu);
    for (auto &ep : g_timing.used) g_timing.pool.push_back(ep);
    g_timing.used.clear();
    for (int k = 0; k < MCD_K_COUNT; ++k) g_timing.seen[k] = 0;
    g_timing.sample_every = sample_every;
    return MCD_OK;
}

extern "C" mcd_status mcd_timing_read(int kernel, int64_t *sampled, double *total_ms) {
    MCD_CHECK_ARG(kernel >= 0 && kernel < MCD_K_COUNT && sampled && total_ms, "bad argument");
    std::lock_guard<std::mutex> lk(g_timing.mu);
    int64_t n = 0;
    double tot = 0.0;
    for (auto &ep : g_timing.used) {
        if (ep.kind != kernel) continue;
        MCD_CUDA_TRY(cudaEventSynchronize(ep.b));
        float ms = 0.0f;
        MCD_CUDA_TRY(cudaEventElapsedTime(&ms, ep.a, ep.b));
        tot += ms;
        ++n;
    }
    *sampled = n;
    *total_ms = tot;
    return MCD_OK;
}
