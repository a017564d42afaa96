// admission.h -- admission policy of the request server (no CUDA; the server in
// server.cu applies it under its lock, and a host-only test builds it alone).
//
// Requests wait in submission order.  A request is admitted when its
// estimated device footprint fits the remaining budget.  A request that does
// not fit blocks only the requests behind it that have waited less than
// max_wait_ns: younger ones that fit may pass it (so small requests are not
// stuck behind a large one), but once it has waited max_wait_ns nothing
// passes it any more and it takes the next memory that is freed.  An admitted
// small request (n <= small_n) takes the later small requests of the same
// dimension that also fit along, up to max_batch requests and batch_max_n
// particles, and they run as one batch (continuous batching).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <deque>
#include <vector>

namespace sph {

struct QItem {
    uint64_t ticket;
    int64_t n;
    int dim;
    int64_t est_bytes;
    int64_t t_submit_ns;
};

struct SchedCfg {
    int64_t budget_bytes;
    int64_t small_n;       // requests with n <= small_n may be batched
    int64_t batch_max_n;   // particles per batch
    int max_batch;         // requests per batch
    int64_t max_wait_ns;   // a blocked request older than this is not passed
    int64_t large_n = 262144;    // requests above it run on a low-priority stream on part of the GPU
    int large_sm_percent = 75;   // the share of the GPU's resident thread blocks they take
};

// Device bytes held for a request of n particles: working arrays, the
// coordinates, and the result (row pointers, density, permutation, and the
// column array sized for nbr_max neighbours per particle).
inline int64_t request_bytes(int64_t n, int dim, int64_t nbr_max) {
    const int64_t work = 72 + 8 * dim;  // binning arrays and the device copy of the coordinates
    const int64_t result = 8 + 4 + 4;   // row_ptr, rho, orig_id
    return n * (work + result + 4 * nbr_max) + 8 + 4096;
}

// Indices into q of the requests to start now (ascending), given the bytes
// currently held and the clock.  Empty when nothing can start.
inline std::vector<size_t> sched_pick(const std::deque<QItem> &q, int64_t held, const SchedCfg &c, int64_t now_ns) {
    std::vector<size_t> out;
    size_t first = q.size();
    for (size_t k = 0; k < q.size(); ++k) {
        if (held + q[k].est_bytes <= c.budget_bytes) {
            first = k;
            break;
        }
        // q[k] does not fit: an old enough request is not passed
        if (now_ns - q[k].t_submit_ns >= c.max_wait_ns) return out;
    }
    if (first == q.size()) return out;
    out.push_back(first);
    const QItem &a = q[first];
    if (a.n > c.small_n) return out;
    int64_t bytes = held + a.est_bytes, parts = a.n;
    for (size_t k = first + 1; k < q.size() && (int)out.size() < c.max_batch; ++k) {
        const QItem &b = q[k];
        if (b.n > c.small_n || b.dim != a.dim) continue;
        if (parts + b.n > c.batch_max_n || bytes + b.est_bytes > c.budget_bytes) continue;
        out.push_back(k);
        bytes += b.est_bytes;
        parts += b.n;
    }
    return out;
}

}  // namespace sph
