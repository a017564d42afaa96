// batch.cu -- sph_batch_run: the binning, search and density of many
// independent particle systems in one pass (include/sph.h).
//
// The systems are concatenated: particle I of the batch is particle
// I - off[s] of system s, system s owns cells [cell_base[s], cell_base[s+1])
// and rows of cells [row_base[s], row_base[s+1]) of one global cell space, so
// the cell-sorted arrays of all systems form one array in which system s
// occupies positions [off[s], off[s+1]).  One launch of each binning kernel
// covers every system; one launch of the single-pass tile search processes
// the tiles of all systems (each tile carries its system, whose GridDev the
// kernel reads from a device table), so the output is one block-diagonal
// CSR over the concatenation.
//
// After the bounds (one device->host read for all systems), the launches of
// the binning, tile-list and search steps depend only on the batch's shapes,
// buffers and the chosen tile shape: they are recorded once as a CUDA graph
// (the persistent search included) and replayed while those stay the same.
// The tile shape and staging are tuned by timing the candidates on the first
// run of each density class; that run launches directly and records the
// graph with its choice.
#include <math.h>
#include <string.h>

#include <map>
#include <new>
#include <vector>

#include "host.cuh"
#include "cellcount.cuh"
#include "launch.cuh"
#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr int BATCH_MAX_SYS = 1 << 16;

// What the binning kernels need of one system (device table).
struct BinSys {
    const double *xyz;
    double lo[3];
    double two_over_hc;
    int nk[3];
    int n;
    int check_box;
    int cell_base;
};

__device__ __forceinline__ int find_sys(const long long *first, int nsys, long long i) {
    // last s with first[s] <= i
    int a = 0, b = nsys - 1;
    while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (first[m] <= i) a = m;
        else b = m - 1;
    }
    return a;
}

__device__ __forceinline__ void key_minmax(unsigned long long b, unsigned long long &mn, unsigned long long &mx,
                                           bool &bad) {
    bad |= ((b >> 52) & 0x7ffull) == 0x7ffull;
    const unsigned long long k = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    mn = k < mn ? k : mn;
    mx = k > mx ? k : mx;
}

// Per-system bounds: blockIdx.y is the system; keys[s*6 + a] min, +3 max.
__global__ void k_batch_bounds(const BinSys *__restrict__ sys, int dim, unsigned long long *__restrict__ keys,
                               DevStatus *st) {
    const BinSys &S = sys[blockIdx.y];
    const long long total = (long long)S.n * dim;
    const unsigned long long *bits = reinterpret_cast<const unsigned long long *>(S.xyz);
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    // stride: a multiple of dim, so each thread stays on one axis
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ax = (int)(t % dim);
    for (long long f = t; f < total; f += stride) key_minmax(__ldg(bits + f), mn[ax], mx[ax], bad);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->flags, ST_NONFINITE);
    for (int a = 0; a < dim; ++a) {
        unsigned long long vmn = mn[a], vmx = mx[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long pm = __shfl_xor_sync(0xffffffffu, vmn, o);
            const unsigned long long px = __shfl_xor_sync(0xffffffffu, vmx, o);
            vmn = pm < vmn ? pm : vmn;
            vmx = px > vmx ? px : vmx;
        }
        if ((threadIdx.x & 31) == 0 && vmn <= vmx) {
            atomicMin(&keys[(long long)blockIdx.y * 6 + a], vmn);
            atomicMax(&keys[(long long)blockIdx.y * 6 + 3 + a], vmx);
        }
    }
}

// Cell, relative coordinates and warp-aggregated cell histogram of every
// particle of the batch (as k_hash of a single grid).
template <int DIM>
__global__ void k_batch_hash(const BinSys *__restrict__ sys, const long long *__restrict__ first, int nsys,
                             long long ntot, int *__restrict__ cnt, int *__restrict__ cid,
                             int *__restrict__ slot, uint2 *__restrict__ rel16u, float4 *__restrict__ rel32u,
                             DevStatus *st) {
    for (long long base = (long long)blockIdx.x * blockDim.x; base < ntot; base += (long long)gridDim.x * blockDim.x) {
        const long long I = base + threadIdx.x;
        const bool live = I < ntot;
        int c = -1;
        if (live) {
            const int s = find_sys(first, nsys, I);
            const BinSys &S = sys[s];
            const long long i = I - first[s];
            int cc[3] = {0, 0, 0};
            double a[3] = {0.0, 0.0, 0.0};
            float fr[3] = {0.f, 0.f, 0.f};
            bool out = false;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const double sk = __dmul_rn(__dsub_rn(S.xyz[i * DIM + k], S.lo[k]), S.two_over_hc);
                // without a box check the FP64 relative coordinate itself is not needed
                if (!S.check_box && rel_axis_bits(sk, S.nk[k], cc[k], fr[k])) continue;
                cc[k] = rel_axis_s(sk, S.nk[k], a[k]);
                out |= fabs(a[k]) > 1.0 + 1e-6;
                fr[k] = __double2float_rn(a[k]);
            }
            if (out && S.check_box) atomicOr(&st->flags, ST_OUT_OF_BOX);
            c = S.cell_base + (cc[2] * S.nk[1] + cc[1]) * S.nk[0] + cc[0];
            uint2 q;
            float4 f;
            round_rel_f(fr[0], fr[1], fr[2], cc[0], q, f);
            rel16u[I] = q;
            rel32u[I] = f;
        }
        const int sl = cell_run_slot(c, live, cnt);
        if (live) {
            cid[I] = c;
            slot[I] = sl;
        }
    }
}

// Cell order: rank, cell x within the system, system-local input index and
// the relative coordinates of every sorted position.
__global__ void k_batch_convert(const BinSys *__restrict__ sys, const long long *__restrict__ first, int nsys,
                                long long ntot, const int *__restrict__ orig_global, const int *__restrict__ cid,
                                const uint2 *__restrict__ rel16u, const float4 *__restrict__ rel32u,
                                int *__restrict__ rank, int *__restrict__ orig_local, int *__restrict__ scell_x,
                                uint2 *__restrict__ rel16, float4 *__restrict__ rel32) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < ntot;
         p += (long long)gridDim.x * blockDim.x) {
        const int I = orig_global[p];
        const int s = find_sys(first, nsys, p);  // sorted positions of system s: [first[s], first[s+1])
        const BinSys &S = sys[s];
        rank[I] = (int)p;
        orig_local[p] = (int)(I - first[s]);
        scell_x[p] = (cid[I] - S.cell_base) % S.nk[0];
        rel16[p] = rel16u[I];
        rel32[p] = rel32u[I];
    }
}

// Row tiles (row_tile_end) over the rows of all systems.
__global__ void k_batch_rows_count(const BinSys *__restrict__ sys, const long long *__restrict__ row_first, int nsys,
                                   long long nrow, const int *__restrict__ cell_start, int *__restrict__ tcount) {
    for (long long R = (long long)blockIdx.x * blockDim.x + threadIdx.x; R < nrow;
         R += (long long)gridDim.x * blockDim.x) {
        const int s = find_sys(row_first, nsys, R);
        const BinSys &S = sys[s];
        const int *cs = cell_start + S.cell_base + (R - row_first[s]) * S.nk[0];
        int count = 0, c = 0;
        for (int p = cs[0]; p < cs[S.nk[0]]; ++count) p = row_tile_end(cs, S.nk[0], p, c);
        tcount[R] = count;
    }
}

__global__ void k_batch_rows_write(const BinSys *__restrict__ sys, const long long *__restrict__ row_first, int nsys,
                                   long long nrow, const int *__restrict__ cell_start,
                                   const long long *__restrict__ toff, int4 *__restrict__ tiles) {
    for (long long R = (long long)blockIdx.x * blockDim.x + threadIdx.x; R < nrow;
         R += (long long)gridDim.x * blockDim.x) {
        const int s = find_sys(row_first, nsys, R);
        const BinSys &S = sys[s];
        const long long r = R - row_first[s];
        const int *cs = cell_start + S.cell_base + r * S.nk[0];
        long long o = toff[R];
        int c = 0;
        for (int p = cs[0]; p < cs[S.nk[0]];) {
            const int e = row_tile_end(cs, S.nk[0], p, c);
            tiles[o++] = make_int4(p, e - p, (int)r, s);
            p = e;
        }
    }
}

unsigned grid_blocks(long long n, int nt, int sm_count, int per_sm) {
    long long b = (n + nt - 1) / nt;
    if (b > (long long)sm_count * per_sm) b = (long long)sm_count * per_sm;
    return (unsigned)(b < 1 ? 1 : b);
}

// Everything the recorded launch sequence depends on besides table contents.
struct GraphKey {
    long long ntot, ncell, nrow, ntiles_max, cap;
    int nsys, dim;
    int shape, extra;  // the search's tile shape and staging
    const void *ptrs[32];
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

}  // namespace
}  // namespace sph

using namespace sph;

struct sph_batch_s {
    int device = 0, sm_count = 0;
    DevBuf bsys, gsys, first, row_first, keys, status;
    DevBuf cnt, cid, slot, cell_start, orig_g, orig_l, rank, scell_x, rel16u, rel32u, rel16, rel32, scan_tmp,
        big_list, tcount, toff, tiles, tstate;
    // pinned host staging of the tables
    BinSys *h_bsys = nullptr;
    GridDev *h_gsys = nullptr;
    long long *h_first = nullptr, *h_row_first = nullptr;
    unsigned long long *h_keys = nullptr;
    DevStatus *h_status = nullptr;
    long long *h_nnz = nullptr;
    int host_cap = 0;
    cudaStream_t cap_stream = nullptr;  // stream the graph is recorded on
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    long long graph_launches = 0;  // kernels per replay
    bool use_graph = true;
    int staging = -1;  // -1: autotune, -2: size from the density estimate without timing
    std::map<int, TileLaunch> tuned;  // density class -> tile shape and staging bytes
    sph_batch_stats stats;
};

static void batch_host_free(sph_batch_s *b) {
    cudaFreeHost(b->h_bsys);
    cudaFreeHost(b->h_gsys);
    cudaFreeHost(b->h_first);
    cudaFreeHost(b->h_row_first);
    cudaFreeHost(b->h_keys);
    b->h_bsys = nullptr;
    b->h_gsys = nullptr;
    b->h_first = b->h_row_first = nullptr;
    b->h_keys = nullptr;
    b->host_cap = 0;
}

static int batch_host_tables(sph_batch_s *b, int nsys) {
    if (nsys <= b->host_cap) return SPH_OK;
    batch_host_free(b);
    if (cudaMallocHost((void **)&b->h_bsys, nsys * sizeof(BinSys)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_gsys, nsys * sizeof(GridDev)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_first, (nsys + 1) * sizeof(long long)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_row_first, (nsys + 1) * sizeof(long long)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_keys, (size_t)nsys * 6 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        batch_host_free(b);
        return fail(SPH_ERR_NOMEM, "pinned host allocation failed");
    }
    b->host_cap = nsys;
    return SPH_OK;
}

static int batch_create(sph_batch_s **out) {
    sph_batch_s *b = new (std::nothrow) sph_batch_s();
    if (!b) return fail(SPH_ERR_NOMEM, "host allocation failed");
    memset(&b->key, 0, sizeof(b->key));
    memset(&b->stats, 0, sizeof(b->stats));
    b->stats.tuned_staging = -1;
    b->stats.tuned_shape = -1;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_nnz, sizeof(long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (b->h_status) cudaFreeHost(b->h_status);
        if (b->h_nnz) cudaFreeHost(b->h_nnz);
        delete b;
        return fail(SPH_ERR_CUDA, "CUDA initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return SPH_OK;
}

// Launches after the bounds up to the search: binning of all systems and the
// tile list (the part recorded as a CUDA graph).
static cudaError_t batch_prep(sph_batch_s *b, int nsys, int dim, long long ntot, long long ncell, long long nrow,
                              const sph_batch_out *out, cudaStream_t s) {
    const int nt = 256;
    const BinSys *bsys = P<BinSys>(b->bsys);
    const long long *first = P<long long>(b->first), *row_first = P<long long>(b->row_first);
    DevStatus *st = P<DevStatus>(b->status);
    cudaError_t e = launch_status_reset_counters(st, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->cnt.p, 0, (size_t)ncell * sizeof(int), s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(TAG_HASH, s);
        note_launch(1);
        (dim == 2 ? k_batch_hash<2> : k_batch_hash<3>)<<<grid_blocks(ntot, nt, b->sm_count, 16), nt, 0, s>>>(
            bsys, first, nsys, ntot, P<int>(b->cnt), P<int>(b->cid), P<int>(b->slot), P<uint2>(b->rel16u),
            P<float4>(b->rel32u), st);
    }
    if ((e = exclusive_scan_i32(P<int>(b->cnt), P<int>(b->cell_start), ncell, b->scan_tmp.p, s)) != cudaSuccess)
        return e;
    if ((e = launch_scatter((int)ntot, P<int>(b->cell_start), P<int>(b->cid), P<int>(b->slot), P<int>(b->orig_g),
                            b->sm_count, s)) != cudaSuccess)
        return e;
    if ((e = segmented_sort_i32(P<int>(b->orig_g), P<int>(b->cell_start), ncell, P<int>(b->big_list),
                                &st->big_cells, b->sm_count, s)) != cudaSuccess)
        return e;
    {
        ProfScope ps(TAG_CONVERT, s);
        note_launch(1);
        k_batch_convert<<<grid_blocks(ntot, nt, b->sm_count, 16), nt, 0, s>>>(
            bsys, first, nsys, ntot, P<int>(b->orig_g), P<int>(b->cid), P<uint2>(b->rel16u), P<float4>(b->rel32u),
            P<int>(b->rank), out->orig_id ? out->orig_id : P<int>(b->orig_l), P<int>(b->scell_x), P<uint2>(b->rel16),
            P<float4>(b->rel32));
    }
    {
        ProfScope ps(TAG_SCAN, s);
        note_launch(2);
        const unsigned rb = grid_blocks(nrow, nt, b->sm_count, 8);
        k_batch_rows_count<<<rb, nt, 0, s>>>(bsys, row_first, nsys, nrow, P<int>(b->cell_start), P<int>(b->tcount));
        if ((e = exclusive_scan_i64(P<int>(b->tcount), P<long long>(b->toff), nrow, b->scan_tmp.p, s)) != cudaSuccess)
            return e;
        k_batch_rows_write<<<rb, nt, 0, s>>>(bsys, row_first, nsys, nrow, P<int>(b->cell_start),
                                             P<long long>(b->toff), P<int4>(b->tiles));
    }
    return cudaGetLastError();
}

// The tile search over all systems' tiles (one persistent launch).
static cudaError_t batch_search(sph_batch_s *b, int dim, long long ntot, long long nrow, long long ntiles_max,
                                const sph_batch_out *out, TileLaunch tv, cudaStream_t s) {
    GridDev g0;
    memset(&g0, 0, sizeof(g0));
    g0.dim = dim;
    g0.n = (int)ntot;
    g0.status = P<DevStatus>(b->status);
    return launch_nnps_tile(g0, P<GridDev>(b->gsys), P<int4>(b->tiles), P<long long>(b->toff) + nrow, ntiles_max,
                            reinterpret_cast<long long *>(out->row_ptr), out->col, out->col ? out->col_capacity : 0,
                            out->rho, P<unsigned long long>(b->tstate), tv, false, b->sm_count, s);
}

// Time one launch of the tile search (after a full sequence has prepared its
// inputs) with shape and staging tv.
static float time_search(sph_batch_s *b, int dim, long long ntot, long long nrow, long long ntiles_max,
                         const sph_batch_out *out, TileLaunch tv, cudaStream_t s) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a candidate whose counters could not be reset is not timed (a stale
    // tile ticket would make its search skip tiles)
    cudaError_t err = launch_status_reset_counters(P<DevStatus>(b->status), s);
    if (err == cudaSuccess) {
        cudaEventRecord(e0, s);
        err = batch_search(b, dim, ntot, nrow, ntiles_max, out, tv, s);
        cudaEventRecord(e1, s);
    }
    float ms = INFINITY;
    if (err == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

extern "C" int sph_batch_run(sph_batch_t *batch, const sph_params *per_system, const double *const *xyz,
                             const int64_t *n, int nsys, sph_batch_out *out, void *stream) {
    if (!batch || !per_system || !xyz || !n || !out) return fail(SPH_ERR_INVALID, "NULL argument");
    if (nsys < 1 || nsys > BATCH_MAX_SYS) return fail(SPH_ERR_INVALID, "nsys must be in [1, %d]", BATCH_MAX_SYS);
    if (!out->row_ptr) return fail(SPH_ERR_INVALID, "row_ptr is NULL");
    if (out->rho && !out->col) return fail(SPH_ERR_INVALID, "rho needs col");
    if (out->col && out->col_capacity < 0) return fail(SPH_ERR_INVALID, "negative col_capacity");
    const int dim = per_system[0].dim;
    long long ntot = 0;
    for (int s = 0; s < nsys; ++s) {
        SPH_TRY(validate_params(&per_system[s], n[s], xyz[s]));
        if (per_system[s].dim != dim) return fail(SPH_ERR_INVALID, "all systems of a batch must have one dim");
        if (per_system[s].precision != SPH_PREC_FP16_RCLL)
            return fail(SPH_ERR_INVALID, "batched runs use the FP16-RCLL search");
        if (per_system[s].order != SPH_ORDER_CELL) return fail(SPH_ERR_INVALID, "batched runs are in cell order");
        ntot += n[s];
    }
    if (ntot >= 0x7fffffffLL) return fail(SPH_ERR_INVALID, "batch of %lld particles exceeds 2^31 - 1", ntot);
    if (*batch == nullptr) SPH_TRY(batch_create(batch));
    sph_batch_s *b = *batch;
    cudaStream_t s = (cudaStream_t)stream;
    SPH_TRY(batch_host_tables(b, nsys));

    const long long launches_before = launch_count();
    // ---- per-system bounds (one read for all systems) -------------------------
    long long nn = ntot > 0 ? ntot : 1;
    SPH_TRY(ensure(b->status, sizeof(DevStatus), s));
    SPH_TRY(ensure(b->bsys, nsys * sizeof(BinSys), s));
    SPH_TRY(ensure(b->gsys, nsys * sizeof(GridDev), s));
    SPH_TRY(ensure(b->first, (nsys + 1) * sizeof(long long), s));
    SPH_TRY(ensure(b->row_first, (nsys + 1) * sizeof(long long), s));
    SPH_TRY(ensure(b->keys, (size_t)nsys * 6 * sizeof(unsigned long long), s));
    SPH_CUDA(launch_status_init(P<DevStatus>(b->status), s));
    bool need_bounds = false;
    long long nmax = 0;
    for (int k = 0; k < nsys; ++k) {
        BinSys &S = b->h_bsys[k];
        memset(&S, 0, sizeof(S));
        S.xyz = xyz[k];
        S.n = (int)n[k];
        S.check_box = per_system[k].have_box;
        need_bounds |= !per_system[k].have_box && n[k] > 0;
        if (n[k] > nmax) nmax = n[k];
    }
    if (need_bounds) {
        SPH_CUDA(cudaMemcpyAsync(b->bsys.p, b->h_bsys, nsys * sizeof(BinSys), cudaMemcpyHostToDevice, s));
        // min keys all ones, max keys zero
        for (int k = 0; k < nsys; ++k)
            for (int a = 0; a < 6; ++a) b->h_keys[k * 6 + a] = a < 3 ? ~0ull : 0ull;
        SPH_CUDA(cudaMemcpyAsync(b->keys.p, b->h_keys, (size_t)nsys * 6 * 8, cudaMemcpyHostToDevice, s));
        const int nt = 96 * 2;  // multiple of 2 and 3
        long long bx = (nmax * dim + nt * 4 - 1) / (nt * 4);
        if (bx > 64) bx = 64;
        if (bx < 1) bx = 1;
        {
            ProfScope ps(TAG_BOUNDS, s);
            note_launch(1);
            k_batch_bounds<<<dim3((unsigned)bx, (unsigned)nsys), nt, 0, s>>>(P<BinSys>(b->bsys), dim,
                                                                              P<unsigned long long>(b->keys),
                                                                              P<DevStatus>(b->status));
        }
        SPH_CUDA(cudaGetLastError());
        SPH_CUDA(copy_small_to_host(b->h_keys, b->keys.p, (size_t)nsys * 6 * 8, s));
        SPH_CUDA(status_to_host(b->h_status, P<DevStatus>(b->status), nullptr, s));
        SPH_CUDA(cudaStreamSynchronize(s));
        if (b->h_status->flags & ST_NONFINITE) return fail(SPH_ERR_INVALID, "non-finite particle coordinate");
    }

    // ---- geometry and tables ----------------------------------------------------
    long long ncell = 0, nrow = 0, off = 0;
    double nbr_w = 0.0;
    for (int k = 0; k < nsys; ++k) {
        const sph_params &p = per_system[k];
        BinSys &S = b->h_bsys[k];
        const double hc = p.cell_size != 0 ? p.cell_size : p.kh * (1.0 + 0x1p-30);
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            if (p.have_box) {
                lo[a] = p.box_lo[a];
                hi[a] = p.box_hi[a];
            } else if (n[k] > 0) {
                lo[a] = dkey_inv(b->h_keys[k * 6 + a]);
                hi[a] = dkey_inv(b->h_keys[k * 6 + 3 + a]);
            }
        }
        long long nc = 1;
        int nk[3] = {1, 1, 1};
        for (int a = 0; a < dim; ++a) {
            const double span = ceil((hi[a] - lo[a]) / hc);
            if (!(span <= (double)(1 << 20))) return fail(SPH_ERR_INVALID, "system %d: more than 2^20 cells", k);
            nk[a] = span < 1.0 ? 1 : (int)span;
            nc *= nk[a];
        }
        if (nc > (1LL << 28)) return fail(SPH_ERR_INVALID, "system %d: more than 2^28 cells", k);
        for (int a = 0; a < 3; ++a) {
            S.lo[a] = lo[a];
            S.nk[a] = nk[a];
        }
        S.two_over_hc = 2.0 / hc;
        if (ncell + nc >= 0x7fffffffLL) return fail(SPH_ERR_INVALID, "batch exceeds 2^31 cells");
        S.cell_base = (int)ncell;
        b->h_first[k] = off;
        b->h_row_first[k] = nrow;
        GridDev &d = b->h_gsys[k];
        memset(&d, 0, sizeof(d));
        d.dim = dim;
        d.n = (int)ntot;
        for (int a = 0; a < 3; ++a) {
            d.nk[a] = nk[a];
            d.lo[a] = lo[a];
        }
        d.ncell = nc;
        set_divisors(d);
        d.hc = hc;
        d.two_over_hc = 2.0 / hc;
        d.xyz = xyz[k];
        set_constants(d, p, hc);
        const double r = p.kh / hc, ppc = (double)n[k] / (double)nc;
        nbr_w += (double)n[k] * (dim == 3 ? ppc * 4.18879 * r * r * r : ppc * 3.14159 * r * r);
        ncell += nc;
        nrow += (long long)nk[1] * nk[2];
        off += n[k];
    }
    b->h_first[nsys] = off;
    b->h_row_first[nsys] = nrow;
    const long long ntiles_max = tiles_max(ntot, ncell, nrow);
    if ((int)ensure(b->cnt, ncell * sizeof(int), s) || ensure(b->cell_start, (ncell + 1) * sizeof(int), s) ||
        ensure(b->cid, nn * sizeof(int), s) || ensure(b->slot, nn * sizeof(int), s) ||
        ensure(b->orig_g, nn * sizeof(int), s) || ensure(b->orig_l, nn * sizeof(int), s) ||
        ensure(b->rank, nn * sizeof(int), s) || ensure(b->scell_x, nn * sizeof(int), s) ||
        ensure(b->rel16u, nn * sizeof(uint2), s) || ensure(b->rel32u, nn * sizeof(float4), s) ||
        ensure(b->rel16, nn * sizeof(uint2), s) || ensure(b->rel32, nn * sizeof(float4), s) ||
        ensure(b->scan_tmp, scan_tmp_bytes((ncell > nrow ? ncell : nrow) + 1), s) ||
        ensure(b->big_list, ncell * sizeof(int), s) || ensure(b->tcount, nrow * sizeof(int), s) ||
        ensure(b->toff, (nrow + 1) * sizeof(long long), s) || ensure(b->tiles, ntiles_max * sizeof(int4), s) ||
        ensure(b->tstate, ntiles_max * sizeof(unsigned long long), s))
        return SPH_ERR_NOMEM;
    const int *orig_local = out->orig_id ? out->orig_id : P<int>(b->orig_l);
    for (int k = 0; k < nsys; ++k) {
        GridDev &d = b->h_gsys[k];
        d.cell_start = P<int>(b->cell_start) + b->h_bsys[k].cell_base;
        d.rel16 = P<uint2>(b->rel16);
        d.rel32 = P<float4>(b->rel32);
        d.orig_id = orig_local;
        d.scell_x = P<int>(b->scell_x);
        d.status = P<DevStatus>(b->status);
    }
    SPH_CUDA(cudaMemcpyAsync(b->bsys.p, b->h_bsys, nsys * sizeof(BinSys), cudaMemcpyHostToDevice, s));
    SPH_CUDA(cudaMemcpyAsync(b->gsys.p, b->h_gsys, nsys * sizeof(GridDev), cudaMemcpyHostToDevice, s));
    SPH_CUDA(cudaMemcpyAsync(b->first.p, b->h_first, (nsys + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
    SPH_CUDA(cudaMemcpyAsync(b->row_first.p, b->h_row_first, (nsys + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                             s));
    if (out->sys_first)
        for (int k = 0; k <= nsys; ++k) out->sys_first[k] = b->h_first[k];

    // ---- staging size: fixed, tuned earlier for this density class, or tuned now
    const double nbr = ntot > 0 ? nbr_w / (double)ntot : 0.0;
    const int dclass = dim * 1000 + (nbr > 0 ? (int)floor(4.0 * log2(nbr)) : -999);
    TileLaunch tv = tile_choose(nbr, -1);
    bool tune = false;
    if (b->staging >= 0) {
        tv.extra = b->staging;
    } else if (b->staging == -1) {
        auto it = b->tuned.find(dclass);
        if (it != b->tuned.end()) tv = it->second;
        else tune = ntot > 0 && out->col != nullptr;
    }

    // ---- the launch sequence: replayed graph, recorded graph or direct -----------
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.ntot = ntot;
    key.ncell = ncell;
    key.nrow = nrow;
    key.ntiles_max = ntiles_max;
    key.cap = out->col ? out->col_capacity : 0;
    key.nsys = nsys;
    key.dim = dim;
    const void *ptrs[] = {out->row_ptr, out->col, out->rho, out->orig_id, b->bsys.p, b->gsys.p, b->first.p,
                          b->row_first.p, b->status.p, b->cnt.p, b->cid.p, b->slot.p, b->cell_start.p,
                          b->orig_g.p, b->orig_l.p, b->rank.p, b->scell_x.p, b->rel16u.p, b->rel32u.p,
                          b->rel16.p, b->rel32.p, b->scan_tmp.p, b->big_list.p, b->tcount.p, b->toff.p,
                          b->tiles.p, b->tstate.p};
    static_assert(sizeof(ptrs) / sizeof(ptrs[0]) <= sizeof(key.ptrs) / sizeof(key.ptrs[0]), "GraphKey slots");
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) key.ptrs[k] = ptrs[k];

    key.shape = tv.shape;
    key.extra = tv.extra;

    b->stats.runs++;
    b->stats.graph_launched = 0;
    long long graph_kernels = 0;  // kernels of a replayed graph (counted as launches too)
    if (ntot == 0) {
        SPH_CUDA(cudaMemsetAsync(out->row_ptr, 0, sizeof(int64_t), s));
    } else if (!tune && b->use_graph && b->exec && b->key == key) {
        // binning, tile list and search: one graph launch
        SPH_CUDA(cudaGraphLaunch(b->exec, s));
        note_launch((int)b->graph_launches);
        graph_kernels = b->graph_launches;
        b->stats.graph_replays++;
        b->stats.graph_launched = 1;
    } else {
        cudaError_t e = batch_prep(b, nsys, dim, ntot, ncell, nrow, out, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SPH_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
        }
        // the search: tuned candidates are timed here (each run leaves the
        // same result), then one launch with the chosen staging
        if (tune) {
            const TileLaunch cand[] = {{TILE_SPARSE, 0}, {TILE_SPARSE, 2048}, {TILE_DENSE, 0}, {TILE_DENSE, 2048},
                                       {TILE_DENSE, 4096}};
            float best_ms = INFINITY;
            TileLaunch best = tv;
            for (const TileLaunch &c : cand) {
                const float ms = time_search(b, dim, ntot, nrow, ntiles_max, out, c, s);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            b->tuned[dclass] = best;
            b->stats.tuned_staging = best.extra;
            b->stats.tuned_shape = best.shape;
            b->stats.tuned_candidates = (int)(sizeof(cand) / sizeof(cand[0]));
            tv = best;
            key.shape = tv.shape;
            key.extra = tv.extra;
        }
        SPH_CUDA(launch_status_reset_counters(P<DevStatus>(b->status), s));
        SPH_CUDA(batch_search(b, dim, ntot, nrow, ntiles_max, out, tv, s));
        // record the whole sequence for the next run with these shapes
        if (b->use_graph) {
            if (b->exec) {
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            const long long l0 = launch_count();
            prof_set_capturing(true);
            cudaError_t ce = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
            if (ce == cudaSuccess) {
                ce = batch_prep(b, nsys, dim, ntot, ncell, nrow, out, b->cap_stream);
                if (ce == cudaSuccess) ce = launch_status_reset_counters(P<DevStatus>(b->status), b->cap_stream);
                if (ce == cudaSuccess) ce = batch_search(b, dim, ntot, nrow, ntiles_max, out, tv, b->cap_stream);
                cudaError_t ce2 = cudaStreamEndCapture(b->cap_stream, &graph);
                if (ce == cudaSuccess) ce = ce2;
            }
            prof_set_capturing(false);
            // captured work does not run: take the recorded launches back out
            // of the launch count; each replay adds them
            b->graph_launches = launch_count() - l0;
            note_launch(-(int)b->graph_launches);
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                b->exec = nullptr;
            } else {
                b->key = key;
                b->stats.graph_captures++;
            }
        }
    }
    b->stats.direct_launches = launch_count() - launches_before - graph_kernels;

    // ---- nnz, status ------------------------------------------------------------
    SPH_CUDA(status_to_host(b->h_status, P<DevStatus>(b->status), reinterpret_cast<const long long *>(out->row_ptr) + ntot,
                            s));
    SPH_CUDA(cudaStreamSynchronize(s));
    out->nnz = b->h_status->nnz;
    b->stats.fp32_pairs = (int64_t)b->h_status->fp32_pairs;
    b->stats.fp64_pairs = (int64_t)b->h_status->fp64_pairs;
    int rc = status_to_code(b->h_status->flags & ~(unsigned)ST_CAPACITY);
    if (rc != SPH_OK) return rc;
    if (out->col && out->nnz > out->col_capacity)
        return fail(SPH_ERR_CAPACITY, "nnz %lld exceeds col_capacity %lld", (long long)out->nnz,
                    (long long)out->col_capacity);
    return SPH_OK;
}

extern "C" int sph_batch_create(sph_batch_t *batch) {
    if (!batch) return fail(SPH_ERR_INVALID, "NULL argument");
    sph_batch_s *b = nullptr;
    SPH_TRY(batch_create(&b));
    *batch = b;
    return SPH_OK;
}

extern "C" int sph_batch_get_stats(sph_batch_t batch, sph_batch_stats *st) {
    if (!batch || !st) return fail(SPH_ERR_INVALID, "NULL argument");
    *st = batch->stats;
    return SPH_OK;
}

extern "C" int sph_batch_set_option(sph_batch_t batch, int option, int64_t value) {
    if (!batch) return fail(SPH_ERR_INVALID, "batch is NULL");
    if (option == SPH_BATCH_OPT_GRAPH) {
        if (value != 0 && value != 1) return fail(SPH_ERR_INVALID, "SPH_BATCH_OPT_GRAPH takes 0 or 1");
        batch->use_graph = value != 0;
        return SPH_OK;
    }
    if (option == SPH_BATCH_OPT_STAGING) {
        if (value < -2 || value > 65536 || (value > 0 && value % 16 != 0))
            return fail(SPH_ERR_INVALID, "SPH_BATCH_OPT_STAGING takes -1, -2 or a multiple of 16 in [0, 65536]");
        batch->staging = (int)value;
        return SPH_OK;
    }
    return fail(SPH_ERR_INVALID, "unknown option %d", option);
}

extern "C" int sph_batch_free(sph_batch_t batch) {
    if (!batch) return SPH_OK;
    sph_batch_s *b = batch;
    cudaStream_t s = nullptr;
    cudaStreamSynchronize(b->cap_stream);
    DevBuf *bufs[] = {&b->bsys, &b->gsys, &b->first, &b->row_first, &b->keys, &b->status, &b->cnt, &b->cid,
                      &b->slot, &b->cell_start, &b->orig_g, &b->orig_l, &b->rank, &b->scell_x, &b->rel16u,
                      &b->rel32u, &b->rel16, &b->rel32, &b->scan_tmp, &b->big_list, &b->tcount, &b->toff,
                      &b->tiles, &b->tstate};
    cudaDeviceSynchronize();
    for (DevBuf *d : bufs) release(*d, s);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaStreamDestroy(b->cap_stream);
    batch_host_free(b);
    cudaFreeHost(b->h_status);
    cudaFreeHost(b->h_nnz);
    cudaStreamSynchronize(s);
    delete b;
    return SPH_OK;
}
