// profile.cu -- launch counting and optional per-kernel CUDA-event timing of
// the library's own launches (events are recorded on the stream each kernel
// is launched on, so the times are device times of exactly those kernels).
#include <atomic>
#include <mutex>
#include <vector>

#include "sph_internal.cuh"
#include "profile.cuh"

namespace sph {

static std::atomic<long long> g_launches{0};
static thread_local bool t_capturing = false;  // this thread is recording a CUDA graph
static std::atomic<int> g_enabled{0};
static std::mutex g_mu;

struct Pair {
    int tag;
    cudaEvent_t a, b;
};
static std::vector<Pair> g_pending;
static std::vector<cudaEvent_t> g_free;
static double g_ms[TAG_COUNT_] = {0};
static long long g_calls[TAG_COUNT_] = {0};

static const char *const g_names[TAG_COUNT_] = {"bounds", "hash",  "scan",    "scatter", "sort",
                                                "convert", "count", "fill",    "density", "canon",
                                                "fused",   "batch", "step"};

const char *tag_name(int tag) { return (tag >= 0 && tag < TAG_COUNT_) ? g_names[tag] : ""; }

void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

long long launch_count() { return g_launches.load(); }

static cudaEvent_t take_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(int tag, cudaStream_t s) : tag_(tag), s_(s), a_(nullptr) {
    if (t_capturing || !((g_enabled.load(std::memory_order_relaxed) >> tag) & 1)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s_);
    g_pending.push_back({tag_, (cudaEvent_t)a_, b});
}

static void drain_locked() {
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.tag] += ms;
            g_calls[p.tag] += 1;
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.clear();
    cudaGetLastError();
}

void prof_set_capturing(bool on) { t_capturing = on; }

void prof_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_enabled.store(on ? (1 << TAG_COUNT_) - 1 : 0);
}

int prof_select(const char *names) {
    if (names == nullptr) {
        prof_enable(1);
        return 0;
    }
    int mask = 0;
    const char *p = names;
    while (*p) {
        const char *e = strchr(p, ',');
        const size_t len = e ? (size_t)(e - p) : strlen(p);
        int found = -1;
        for (int t = 0; t < TAG_COUNT_; ++t)
            if (strlen(g_names[t]) == len && strncmp(p, g_names[t], len) == 0) found = t;
        if (found < 0) return -1;
        mask |= 1 << found;
        p += len;
        if (*p == ',') ++p;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_enabled.store(mask);
    return 0;
}

void prof_reset() {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    for (int t = 0; t < TAG_COUNT_; ++t) {
        g_ms[t] = 0;
        g_calls[t] = 0;
    }
}

int prof_read(const char *name, double *ms, long long *calls) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    for (int t = 0; t < TAG_COUNT_; ++t) {
        if (strcmp(name, g_names[t]) == 0) {
            if (ms) *ms = g_ms[t];
            if (calls) *calls = g_calls[t];
            return 0;
        }
    }
    return -1;
}

}  // namespace sph

// ---- FP64 FMA throughput of the device ---------------------------------------
// Eight independent FMA chains per thread keep the FP64 pipe busy; the result
// is stored so that nothing is optimised away.
namespace sph {
namespace {
constexpr int FP64_CHAINS = 8;
constexpr int FP64_ITERS = 2048;

__global__ void k_fp64_fma(double *out, double a, double b) {
    double v[FP64_CHAINS];
#pragma unroll
    for (int c = 0; c < FP64_CHAINS; ++c) v[c] = (double)(threadIdx.x + c);
    for (int it = 0; it < FP64_ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < FP64_CHAINS; ++c) v[c] = __fma_rn(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < FP64_CHAINS; ++c) s += v[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

int fp64_fma_rate(double *flops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int nt = 256, blocks = sms * 8;
    double *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * nt * sizeof(double)) != cudaSuccess) return -1;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    note_launch(1);
    k_fp64_fma<<<blocks, nt>>>(out, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(a);
    const int reps = 5;
    note_launch(reps);
    for (int r = 0; r < reps; ++r) k_fp64_fma<<<blocks, nt>>>(out, 0.999999, 1e-7);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return -1;
    *flops = 2.0 * (double)reps * blocks * nt * FP64_CHAINS * FP64_ITERS / (ms * 1e-3);
    return 0;
}
}  // namespace sph
