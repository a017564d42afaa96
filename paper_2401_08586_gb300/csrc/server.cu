// server.cu -- request server over the search (include/sph.h, "Serving").
//
// Clients submit particle systems and poll for results; worker threads, each
// with its own CUDA stream, grid and batch workspace, take admitted requests
// off the queue (admission policy in admission.h), run binning + search + fused
// density, and leave row pointers, columns, densities and the permutation in
// device buffers owned by the request until the client releases it.  Small
// requests that are waiting together run as one batched search (continuous
// batching); their results are split into per-request buffers afterwards.
// Every request is isolated: a batch that fails is re-run one request at a
// time so that only the offending request reports the error.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "host.cuh"
#include "profile.cuh"
#include "admission.h"
#include "sph_internal.cuh"

namespace sph {
namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

__global__ void k_rebase_i64(const long long *__restrict__ in, long long *__restrict__ out, long long n,
                             long long base) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] - base;
}

__global__ void k_rebase_i32(const int *__restrict__ in, int *__restrict__ out, long long n, int base) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] - base;
}

unsigned blocks_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 2048) b = 2048;
    return (unsigned)(b < 1 ? 1 : b);
}

enum ReqState { RQ_QUEUED, RQ_RUNNING, RQ_DONE };

struct Req {
    uint64_t ticket = 0;
    sph_request r;
    ReqState state = RQ_QUEUED;
    int status = SPH_OK;
    std::string msg;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int64_t est = 0;   // bytes reserved at admission
    int64_t held = 0;  // bytes held once done (the result buffers)
    DevBuf rp, col, rho, orig;
    int64_t nnz = 0;
};

}  // namespace

struct ServerWorker;

}  // namespace sph

using namespace sph;

struct sph_server_s {
    sph_server_cfg cfg;
    SchedCfg sc;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<QItem> q;
    std::map<uint64_t, Req *> reqs;
    std::vector<std::thread> threads;
    std::vector<ServerWorker *> workers;
    int64_t held = 0, peak_held = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    cudaStream_t release_stream = nullptr;
    int device = 0;
    sph_server_stats stats;
};

namespace sph {
namespace {

int64_t nbr_max_for(int dim) { return dim == 3 ? 128 : 40; }

// Free a request's result buffers (stream-ordered on the server's release stream).
void free_result(sph_server_s *S, Req *q) {
    release(q->rp, S->release_stream);
    release(q->col, S->release_stream);
    release(q->rho, S->release_stream);
    release(q->orig, S->release_stream);
}

}  // namespace

struct ServerWorker {
    sph_server_s *S;
    cudaStream_t s = nullptr;     // stream of the current request
    cudaStream_t s_hi = nullptr;  // high priority: requests of up to large_n particles, batches
    cudaStream_t s_lo = nullptr;  // low priority: larger requests
    long long *rp_idx = nullptr, *rp_val = nullptr;  // pinned: a batch's row offsets, read by a kernel
    int rp_cap = 0;
    sph_grid_t grid = nullptr;
    sph_batch_t batch = nullptr;
    DevBuf xyz, brp, bcol, brho, borig;

    // One request on its own.  Returns SPH_OK or the request's error.
    int run_one(Req *q) {
        const sph_request &r = q->r;
        const int dim = r.params.dim;
        const double *x = r.xyz;
        const bool large = r.n > S->sc.large_n;
        s = large ? s_lo : s_hi;
        if (r.n > 0 && !r.xyz_on_device) {
            SPH_TRY(ensure(xyz, (size_t)r.n * dim * sizeof(double), s));
            SPH_CUDA(cudaMemcpyAsync(xyz.p, r.xyz, (size_t)r.n * dim * sizeof(double), cudaMemcpyHostToDevice, s));
            x = P<double>(xyz);
        }
        SPH_TRY(sph_bin_cells(&r.params, x, r.n, s, &grid));
        SPH_TRY(sph_grid_set_option(grid, SPH_OPT_SM_SHARE, large ? S->sc.large_sm_percent : 100));
        SPH_TRY(ensure(q->rp, (size_t)(r.n + 1) * sizeof(int64_t), s));
        if (r.want_density) SPH_TRY(ensure(q->rho, (size_t)(r.n > 0 ? r.n : 1) * sizeof(float), s));
        // the search writes straight into the request's column buffer, sized
        // from the grid's neighbour estimate (particles per cell times the
        // search sphere's volume in cells, 30 % to spare); a miss re-runs the
        // search with the exact size
        sph_grid_info info;
        SPH_TRY(sph_grid_info_get(grid, &info));
        const double ppc = info.ncell > 0 ? (double)r.n / (double)info.ncell : 0.0;
        const double rk = r.params.kh / info.cell_size;
        const double nbr = dim == 3 ? ppc * 4.18879 * rk * rk * rk : ppc * 3.14159 * rk * rk;
        int64_t cap = (int64_t)((double)r.n * nbr * 1.3) + 1024, nnz = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            SPH_TRY(ensure(q->col, (size_t)cap * sizeof(int32_t), s));
            const int rc = sph_nnps_query(grid, P<int64_t>(q->rp), P<int32_t>(q->col), cap, &nnz,
                                          r.want_density ? P<float>(q->rho) : nullptr, s);
            if (rc == SPH_OK) break;
            if (rc != SPH_ERR_CAPACITY || attempt == 1) return rc;
            release(q->col, s);
            cap = nnz;
        }
        q->nnz = nnz;
        SPH_TRY(ensure(q->orig, (size_t)(r.n > 0 ? r.n : 1) * sizeof(int32_t), s));
        if (r.n > 0 && r.params.order == SPH_ORDER_CELL)
            SPH_TRY(sph_grid_export(grid, P<int32_t>(q->orig), nullptr, nullptr, s));
        SPH_CUDA(cudaStreamSynchronize(s));
        return SPH_OK;
    }

    // Several small cell-order requests of one dimension as one batched run.
    int run_batch(std::vector<Req *> &qs) {
        s = s_hi;
        const int k = (int)qs.size();
        const int dim = qs[0]->r.params.dim;
        int64_t ntot = 0;
        std::vector<int64_t> off(k + 1, 0);
        for (int i = 0; i < k; ++i) {
            off[i] = ntot;
            ntot += qs[i]->r.n;
        }
        off[k] = ntot;
        SPH_TRY(ensure(xyz, (size_t)(ntot > 0 ? ntot : 1) * dim * sizeof(double), s));
        std::vector<const double *> xs(k);
        std::vector<int64_t> ns(k);
        std::vector<sph_params> ps(k);
        for (int i = 0; i < k; ++i) {
            const sph_request &r = qs[i]->r;
            ps[i] = r.params;
            ns[i] = r.n;
            if (r.xyz_on_device || r.n == 0) {
                xs[i] = r.xyz;
            } else {
                double *dst = P<double>(xyz) + off[i] * dim;
                SPH_CUDA(cudaMemcpyAsync(dst, r.xyz, (size_t)r.n * dim * sizeof(double), cudaMemcpyHostToDevice, s));
                xs[i] = dst;
            }
        }
        SPH_TRY(ensure(brp, (size_t)(ntot + 1) * sizeof(int64_t), s));
        SPH_TRY(ensure(brho, (size_t)(ntot > 0 ? ntot : 1) * sizeof(float), s));
        SPH_TRY(ensure(borig, (size_t)(ntot > 0 ? ntot : 1) * sizeof(int32_t), s));
        std::vector<int64_t> first(k + 1, 0);
        int64_t cap = ntot * nbr_max_for(dim);
        sph_batch_out out;
        for (int attempt = 0; attempt < 2; ++attempt) {
            SPH_TRY(ensure(bcol, (size_t)(cap > 0 ? cap : 1) * sizeof(int32_t), s));
            memset(&out, 0, sizeof(out));
            out.row_ptr = P<int64_t>(brp);
            out.col = P<int32_t>(bcol);
            out.col_capacity = cap;
            out.rho = P<float>(brho);
            out.orig_id = P<int32_t>(borig);
            out.sys_first = first.data();
            const int rc = sph_batch_run(&batch, ps.data(), xs.data(), ns.data(), k, &out, s);
            if (rc == SPH_OK) break;
            if (rc != SPH_ERR_CAPACITY || attempt == 1) return rc;
            cap = out.nnz;
        }
        // split into per-request buffers: each request's first and last row
        // offsets, gathered by a kernel into pinned memory
        if (k + 1 > rp_cap) return fail(SPH_ERR_INVALID, "batch of %d requests exceeds the worker's tables", k);
        for (int i = 0; i <= k; ++i) rp_idx[i] = first[i];
        SPH_CUDA(gather_i64_to_host(rp_val, P<long long>(brp), rp_idx, k + 1, s));
        SPH_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> rp_host(2 * k);
        for (int i = 0; i < k; ++i) {
            rp_host[2 * i] = rp_val[i];
            rp_host[2 * i + 1] = rp_val[i + 1];
        }
        for (int i = 0; i < k; ++i) {
            Req *q = qs[i];
            const int64_t n = q->r.n, a = first[i], c0 = rp_host[2 * i], c1 = rp_host[2 * i + 1];
            q->nnz = c1 - c0;
            SPH_TRY(ensure(q->rp, (size_t)(n + 1) * sizeof(int64_t), s));
            SPH_TRY(ensure(q->col, (size_t)(q->nnz > 0 ? q->nnz : 1) * sizeof(int32_t), s));
            SPH_TRY(ensure(q->orig, (size_t)(n > 0 ? n : 1) * sizeof(int32_t), s));
            if (q->r.want_density) SPH_TRY(ensure(q->rho, (size_t)(n > 0 ? n : 1) * sizeof(float), s));
            note_launch(q->nnz > 0 ? 2 : 1);
            k_rebase_i64<<<blocks_for(n + 1), 256, 0, s>>>(P<long long>(brp) + a, P<long long>(q->rp), n + 1, c0);
            if (q->nnz > 0)
                k_rebase_i32<<<blocks_for(q->nnz), 256, 0, s>>>(P<int>(bcol) + c0, P<int>(q->col), q->nnz, (int)a);
            SPH_CUDA(cudaGetLastError());
            if (n > 0) {
                SPH_CUDA(copy_d2d_kernel(q->orig.p, P<int32_t>(borig) + a, (size_t)n * sizeof(int32_t), s));
                if (q->r.want_density)
                    SPH_CUDA(copy_d2d_kernel(q->rho.p, P<float>(brho) + a, (size_t)n * sizeof(float), s));
            }
        }
        SPH_CUDA(cudaStreamSynchronize(s));
        return SPH_OK;
    }

    void finish(Req *q, int rc) {
        q->status = rc;
        if (rc != SPH_OK) {
            q->msg = last_error();
            free_result(S, q);
        }
        q->held = (int64_t)(q->rp.cap + q->col.cap + q->rho.cap + q->orig.cap);
    }

    void loop() {  // one worker thread
        cudaSetDevice(S->device);
        while (true) {
            std::vector<Req *> picked;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                while (true) {
                    if (S->stop) return;
                    if (!S->q.empty()) {
                        const std::vector<size_t> idx = sched_pick(S->q, S->held, S->sc, now_ns());
                        if (!idx.empty()) {
                            const int64_t t = now_ns();
                            for (size_t i : idx) {
                                Req *q = S->reqs[S->q[i].ticket];
                                q->state = RQ_RUNNING;
                                q->t_admit = t;
                                S->held += q->est;
                                picked.push_back(q);
                            }
                            for (size_t j = idx.size(); j-- > 0;) S->q.erase(S->q.begin() + (long)idx[j]);
                            if (S->held > S->peak_held) S->peak_held = S->held;
                            break;
                        }
                        // blocked by the budget: wake on a release or to re-check ages
                        S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
                    } else {
                        S->cv_work.wait(lk);
                    }
                }
            }
            std::vector<int> rcs(picked.size(), SPH_OK);
            bool batched = picked.size() > 1;
            if (batched) {
                const int rc = run_batch(picked);
                if (rc != SPH_OK) {
                    // isolate: run each request alone
                    cudaGetLastError();
                    batched = false;
                    for (size_t i = 0; i < picked.size(); ++i) rcs[i] = run_one(picked[i]);
                }
            } else {
                rcs[0] = run_one(picked[0]);
            }
            std::lock_guard<std::mutex> lk(S->mu);
            const int64_t t = now_ns();
            for (size_t i = 0; i < picked.size(); ++i) {
                Req *q = picked[i];
                finish(q, rcs[i]);
                S->held += q->held - q->est;
                if (S->held > S->peak_held) S->peak_held = S->held;
                q->t_done = t;
                q->state = RQ_DONE;
                S->stats.completed++;
                if (rcs[i] != SPH_OK) S->stats.failed++;
            }
            if (batched) {
                S->stats.batches++;
                S->stats.batched_requests += (int64_t)picked.size();
            }
            S->cv_done.notify_all();
            S->cv_work.notify_all();
        }
    }
};

}  // namespace sph

extern "C" int sph_server_create(const sph_server_cfg *cfg, sph_server_t *server) {
    if (!cfg || !server) return fail(SPH_ERR_INVALID, "NULL argument");
    if (cfg->hbm_budget_bytes <= 0) return fail(SPH_ERR_INVALID, "hbm_budget_bytes must be > 0");
    if (cfg->streams < 0 || cfg->streams > 16) return fail(SPH_ERR_INVALID, "streams must be in [0, 16]");
    if (cfg->max_batch < 0 || cfg->small_n < 0 || cfg->max_wait_ns < 0)
        return fail(SPH_ERR_INVALID, "negative batching parameter");
    sph_server_s *S = new (std::nothrow) sph_server_s();
    if (!S) return fail(SPH_ERR_NOMEM, "host allocation failed");
    S->cfg = *cfg;
    memset(&S->stats, 0, sizeof(S->stats));
    S->sc.budget_bytes = cfg->hbm_budget_bytes;
    S->sc.small_n = cfg->small_n > 0 ? cfg->small_n : 32768;
    S->sc.max_batch = cfg->max_batch > 0 ? cfg->max_batch : 64;
    S->sc.batch_max_n = 8 * S->sc.small_n;
    S->sc.max_wait_ns = cfg->max_wait_ns > 0 ? cfg->max_wait_ns : 20000000;
    S->sc.large_n = cfg->large_n > 0 ? cfg->large_n : 262144;
    S->sc.large_sm_percent = cfg->large_sm_percent > 0 && cfg->large_sm_percent <= 100 ? cfg->large_sm_percent : 75;
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->release_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(SPH_ERR_CUDA, "CUDA initialisation failed");
    }
    // keep freed result memory in the stream-ordered pool up to the budget,
    // and grow the pool to it now (halving on failure down to 256 MiB): a
    // request whose allocation has to grow the pool waits for the mapping,
    // and every worker's allocations wait with it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
        uint64_t thr = (uint64_t)cfg->hbm_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        if (cfg->reserve_pool != -1) {
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            size_t want = (size_t)cfg->hbm_budget_bytes;
            if (want > free_b / 10 * 9) want = free_b / 10 * 9;
            for (; want >= ((size_t)256 << 20); want /= 2) {
                void *p = nullptr;
                if (cudaMallocAsync(&p, want, S->release_stream) == cudaSuccess) {
                    cudaFreeAsync(p, S->release_stream);
                    cudaStreamSynchronize(S->release_stream);
                    break;
                }
                cudaGetLastError();
            }
        }
    }
    cudaGetLastError();
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaGetLastError();
    const int nw = cfg->streams > 0 ? cfg->streams : 2;
    for (int i = 0; i < nw; ++i) {
        ServerWorker *w = new ServerWorker();
        w->S = S;
        if (cudaStreamCreateWithPriority(&w->s_hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&w->s_lo, cudaStreamNonBlocking, prio_lo) != cudaSuccess) {
            cudaGetLastError();
            if (w->s_hi) cudaStreamDestroy(w->s_hi);
            delete w;
            break;
        }
        w->s = w->s_hi;
        w->rp_cap = S->sc.max_batch + 1;
        if (cudaMallocHost((void **)&w->rp_idx, (size_t)w->rp_cap * sizeof(long long)) != cudaSuccess ||
            cudaMallocHost((void **)&w->rp_val, (size_t)w->rp_cap * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            if (w->rp_idx) cudaFreeHost(w->rp_idx);
            cudaStreamDestroy(w->s_hi);
            cudaStreamDestroy(w->s_lo);
            delete w;
            break;
        }
        // batches of waiting requests change shape every time: no graph
        // recording, staging sized from the density estimate (no timing runs)
        if (sph_batch_create(&w->batch) == SPH_OK) {
            sph_batch_set_option(w->batch, SPH_BATCH_OPT_GRAPH, 0);
            sph_batch_set_option(w->batch, SPH_BATCH_OPT_STAGING, -2);
        }
        S->workers.push_back(w);
    }
    if (S->workers.empty()) {
        cudaStreamDestroy(S->release_stream);
        delete S;
        return fail(SPH_ERR_CUDA, "stream creation failed");
    }
    for (ServerWorker *w : S->workers) S->threads.emplace_back([w] { w->loop(); });
    *server = S;
    return SPH_OK;
}

extern "C" int sph_serve_submit(sph_server_t S, const sph_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return fail(SPH_ERR_INVALID, "NULL argument");
    SPH_TRY(validate_params(&r->params, r->n, r->xyz));
    const int64_t est = request_bytes(r->n, r->params.dim, nbr_max_for(r->params.dim));
    if (est > S->cfg.hbm_budget_bytes)
        return fail(SPH_ERR_BUDGET, "request of %lld particles needs ~%lld bytes, over the budget of %lld",
                    (long long)r->n, (long long)est, (long long)S->cfg.hbm_budget_bytes);
    Req *q = new (std::nothrow) Req();
    if (!q) return fail(SPH_ERR_NOMEM, "host allocation failed");
    q->r = *r;
    q->est = est;
    q->t_submit = now_ns();
    // only cell-order FP16 requests can share a batched run
    const bool batchable = r->params.order == SPH_ORDER_CELL && r->params.precision == SPH_PREC_FP16_RCLL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete q;
            return fail(SPH_ERR_INVALID, "server is shutting down");
        }
        q->ticket = S->next_ticket++;
        S->reqs[q->ticket] = q;
        QItem it;
        it.ticket = q->ticket;
        it.n = batchable ? r->n : S->sc.small_n + 1 + r->n;  // non-batchable requests never join a batch
        it.dim = r->params.dim;
        it.est_bytes = est;
        it.t_submit_ns = q->t_submit;
        S->q.push_back(it);
        S->stats.submitted++;
        *ticket = q->ticket;
    }
    S->cv_work.notify_one();
    return SPH_OK;
}

static void fill_result(const Req *q, sph_result *res) {
    memset(res, 0, sizeof(*res));
    res->status = q->status;
    res->n = q->r.n;
    res->nnz = q->status == SPH_OK ? q->nnz : 0;
    if (q->status == SPH_OK) {
        res->row_ptr = reinterpret_cast<const int64_t *>(q->rp.p);
        res->col = reinterpret_cast<const int32_t *>(q->col.p);
        res->rho = q->r.want_density ? reinterpret_cast<const float *>(q->rho.p) : nullptr;
        res->orig_id = q->r.params.order == SPH_ORDER_CELL ? reinterpret_cast<const int32_t *>(q->orig.p) : nullptr;
    }
    res->t_submit_ns = q->t_submit;
    res->t_admit_ns = q->t_admit;
    res->t_done_ns = q->t_done;
}

extern "C" int sph_serve_poll(sph_server_t S, uint64_t ticket, sph_result *res) {
    if (!S || !res) return fail(SPH_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(SPH_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->state != RQ_DONE) return SPH_PENDING;
    fill_result(it->second, res);
    if (res->status != SPH_OK) fail(res->status, "%s", it->second->msg.c_str());
    return SPH_OK;
}

extern "C" int sph_serve_wait(sph_server_t S, uint64_t ticket, int64_t timeout_ns, sph_result *res) {
    if (!S || !res) return fail(SPH_ERR_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
    while (true) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(SPH_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
        if (it->second->state == RQ_DONE) {
            fill_result(it->second, res);
            if (res->status != SPH_OK) fail(res->status, "%s", it->second->msg.c_str());
            return SPH_OK;
        }
        if (timeout_ns >= 0 && S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = S->reqs.find(ticket);
            if (it != S->reqs.end() && it->second->state == RQ_DONE) continue;
            return SPH_PENDING;
        }
        if (timeout_ns < 0) S->cv_done.wait(lk);
    }
}

extern "C" int sph_result_copy(sph_server_t S, uint64_t ticket, int64_t *row_ptr, int32_t *col, float *rho,
                               int32_t *orig_id, void *stream) {
    if (!S) return fail(SPH_ERR_INVALID, "NULL argument");
    sph_result res;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(SPH_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
        if (it->second->state != RQ_DONE) return fail(SPH_ERR_INVALID, "request %llu has not finished",
                                                      (unsigned long long)ticket);
        fill_result(it->second, &res);
    }
    if (res.status != SPH_OK) return fail(res.status, "request %llu failed", (unsigned long long)ticket);
    cudaStream_t s = (cudaStream_t)stream;
    if (row_ptr) SPH_CUDA(cudaMemcpyAsync(row_ptr, res.row_ptr, (size_t)(res.n + 1) * 8, cudaMemcpyDefault, s));
    if (col && res.nnz > 0) SPH_CUDA(cudaMemcpyAsync(col, res.col, (size_t)res.nnz * 4, cudaMemcpyDefault, s));
    if (rho && res.rho && res.n > 0) SPH_CUDA(cudaMemcpyAsync(rho, res.rho, (size_t)res.n * 4, cudaMemcpyDefault, s));
    if (orig_id && res.orig_id && res.n > 0)
        SPH_CUDA(cudaMemcpyAsync(orig_id, res.orig_id, (size_t)res.n * 4, cudaMemcpyDefault, s));
    return SPH_OK;
}

extern "C" int sph_result_release(sph_server_t S, uint64_t ticket) {
    if (!S) return fail(SPH_ERR_INVALID, "NULL argument");
    Req *q = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(SPH_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
        if (it->second->state != RQ_DONE) return fail(SPH_ERR_INVALID, "request %llu has not finished",
                                                      (unsigned long long)ticket);
        q = it->second;
        S->reqs.erase(it);
        S->held -= q->held;
    }
    free_result(S, q);
    delete q;
    S->cv_work.notify_all();
    return SPH_OK;
}

extern "C" int sph_server_get_stats(sph_server_t S, sph_server_stats *st) {
    if (!S || !st) return fail(SPH_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->stats;
    st->held_bytes = S->held;
    st->peak_held_bytes = S->peak_held;
    st->queued = (int64_t)S->q.size();
    return SPH_OK;
}

extern "C" int sph_server_destroy(sph_server_t S) {
    if (!S) return SPH_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->threads) t.join();
    for (ServerWorker *w : S->workers) {
        cudaStreamSynchronize(w->s_hi);
        cudaStreamSynchronize(w->s_lo);
        if (w->grid) sph_grid_free(w->grid);
        if (w->batch) sph_batch_free(w->batch);
        DevBuf *bufs[] = {&w->xyz, &w->brp, &w->bcol, &w->brho, &w->borig};
        for (DevBuf *b : bufs) release(*b, w->s);
        cudaStreamSynchronize(w->s);
        cudaStreamDestroy(w->s_hi);
        cudaStreamDestroy(w->s_lo);
        cudaFreeHost(w->rp_idx);
        cudaFreeHost(w->rp_val);
        delete w;
    }
    for (auto &kv : S->reqs) {
        free_result(S, kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(S->release_stream);
    cudaStreamDestroy(S->release_stream);
    cudaGetLastError();
    delete S;
    return SPH_OK;
}
