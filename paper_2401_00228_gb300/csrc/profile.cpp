// Launch counting and kernel-class timing (CUDA events), see mk_internal.h.
#include <atomic>
#include <mutex>

#include "mk_internal.h"

namespace mk {

static std::atomic<int64_t> g_launches{0};
static thread_local int64_t *t_capture_counter = nullptr;

void count_launch(int n) {
    if (t_capture_counter) *t_capture_counter += n;
    else g_launches.fetch_add(n, std::memory_order_relaxed);
}
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(); }
void set_capture_counter(int64_t *c) { t_capture_counter = c; }

struct Acc {
    double ms = 0.0, bytes = 0.0;
    int64_t n = 0;
};

static std::atomic<bool> g_prof{false};
static std::mutex g_mu;
static Acc g_acc[PROF_NCLASS][MK_MAX_LEVELS + 1];
static std::vector<cudaEvent_t> g_pool;
static std::vector<ProfPair> g_transient;
static thread_local std::vector<ProfPair> *t_sink = nullptr;
static thread_local int t_level = 0, t_j = -1;
static thread_local double t_alg_n = 0.0;
static thread_local cudaEvent_t t_pending = nullptr;

static cudaEvent_t take_event() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_pool.empty()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) break;
            g_pool.push_back(e);
        }
        if (g_pool.empty()) return nullptr;
    }
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
}

void release_pairs(std::vector<ProfPair> &pairs) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : pairs) {
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    pairs.clear();
}

bool prof_enabled() { return g_prof.load(); }

void prof_set_context(int level, int j, double alg_n) {
    t_level = level;
    t_j = j;
    t_alg_n = alg_n;
}

double prof_alg_n() { return t_alg_n; }

void prof_set_sink(std::vector<ProfPair> *sink) { t_sink = sink; }

// Inside a stream capture a plain record only orders work; the External flag makes it an
// event-record node of the graph, so the event is recorded on every replay.
static void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
}

void prof_begin(cudaStream_t s) {
    if (!prof_enabled()) return;
    t_pending = take_event();
    if (t_pending) record(t_pending, s);
}

void prof_end(cudaStream_t s, int cls, double bytes) {
    if (!prof_enabled() || !t_pending) return;
    cudaEvent_t b = take_event();
    if (!b) return;
    record(b, s);
    ProfPair p{t_pending, b, cls, t_level, t_j, bytes};
    t_pending = nullptr;
    if (t_sink) t_sink->push_back(p);
    else {
        std::lock_guard<std::mutex> lk(g_mu);
        g_transient.push_back(p);
    }
}

void prof_accumulate(const std::vector<ProfPair> &pairs, int j_limit) {
    for (const auto &p : pairs) {
        if (p.j >= 0 && p.j >= j_limit) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int lv = p.level < 0 ? 0 : (p.level > MK_MAX_LEVELS ? MK_MAX_LEVELS : p.level);
        std::lock_guard<std::mutex> lk(g_mu);
        Acc &a = g_acc[p.cls][lv];
        a.ms += ms;
        a.bytes += p.bytes;
        a.n += 1;
    }
}

void prof_accumulate_transient() {
    std::vector<ProfPair> mine;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        mine.swap(g_transient);
    }
    prof_accumulate(mine, 1 << 30);
    release_pairs(mine);
}

void prof_set_enabled(bool on) { g_prof.store(on); }

void prof_reset() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &row : g_acc)
        for (auto &a : row) a = Acc();
}

bool prof_read(int cls, int level, double &ms, double &bytes, int64_t &n) {
    if (cls < 0 || cls >= PROF_NCLASS || level < 0 || level > MK_MAX_LEVELS) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    ms = g_acc[cls][level].ms;
    bytes = g_acc[cls][level].bytes;
    n = g_acc[cls][level].n;
    return true;
}

}  // namespace mk
