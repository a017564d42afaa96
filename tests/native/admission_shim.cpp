// Host-only test shim: the request server's admission policy
// (paper_2401_08586_gb300/csrc/admission.h) behind a C interface, built by
// tests/test_admission.py with the host compiler.  No CUDA.
#include <stdint.h>

#include <deque>

#include "../../paper_2401_08586_gb300/csrc/admission.h"

extern "C" int adm_pick(const int64_t *n, const int32_t *dim, const int64_t *est, const int64_t *t_submit, int nq,
                        int64_t held, int64_t budget, int64_t small_n, int64_t batch_max_n, int32_t max_batch,
                        int64_t max_wait_ns, int64_t now_ns, int32_t *out) {
    std::deque<sph::QItem> q;
    for (int i = 0; i < nq; ++i) {
        sph::QItem it;
        it.ticket = (uint64_t)i;
        it.n = n[i];
        it.dim = dim[i];
        it.est_bytes = est[i];
        it.t_submit_ns = t_submit[i];
        q.push_back(it);
    }
    sph::SchedCfg c;
    c.budget_bytes = budget;
    c.small_n = small_n;
    c.batch_max_n = batch_max_n;
    c.max_batch = max_batch;
    c.max_wait_ns = max_wait_ns;
    const std::vector<size_t> v = sph::sched_pick(q, held, c, now_ns);
    for (size_t k = 0; k < v.size(); ++k) out[k] = (int32_t)v[k];
    return (int)v.size();
}

extern "C" int64_t adm_request_bytes(int64_t n, int32_t dim, int64_t nbr_max) {
    return sph::request_bytes(n, dim, nbr_max);
}
