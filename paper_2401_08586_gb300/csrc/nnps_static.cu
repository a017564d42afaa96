// nnps_static.cu -- sph_nnps_query_static: the single-pass row-tile search
// without any device allocation, for callers that must not allocate at the
// time of the call (see include/sph.h).
//
// The search's working memory (the tile list and its row offsets, the
// look-back state of the tiles, the scan's tile sums) lives in one fixed
// file-scope device array.  Host code must not hand the array's name to a
// kernel (in host code it names a host-side stand-in), so the first call in
// each CUDA context, with its device current, asks the runtime for the
// array's device address and caches it per device, keyed by the context (a
// device reset or another context on the device looks it up again).
#include <cuda.h>

#include <mutex>

#include "launch.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr long long STATIC_MAX_N = 1LL << 20;     // particles
constexpr long long STATIC_MAX_ROWS = 1LL << 16;  // rows of cells (ny * nz)
constexpr long long STATIC_MAX_TILES = STATIC_MAX_N / 32 + STATIC_MAX_ROWS + 1;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the array.
constexpr size_t OFF_TCOUNT = 0;
constexpr size_t OFF_TOFF = align256(OFF_TCOUNT + STATIC_MAX_ROWS * sizeof(int));
constexpr size_t OFF_TILES = align256(OFF_TOFF + (STATIC_MAX_ROWS + 1) * sizeof(long long));
constexpr size_t OFF_TSTATE = align256(OFF_TILES + STATIC_MAX_TILES * sizeof(int4));
constexpr size_t OFF_SCAN = align256(OFF_TSTATE + STATIC_MAX_TILES * sizeof(unsigned long long));
constexpr size_t STATIC_SCRATCH_BYTES = align256(OFF_SCAN + 64 * 1024);

__device__ __align__(256) unsigned char g_query_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_addr_mu;
struct Cached {
    unsigned long long ctx_id = 0;
    void *addr = nullptr;
};
Cached g_addr[MAX_DEVICES];

// Context id of the calling thread's current context (driver entry points
// through the runtime, so the library needs no link against the driver).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
int current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS)
        return set_error(SPH_ERR_CUDA, "cannot identify the current CUDA context");
    return SPH_OK;
}

// Device address of the array in the current context (looked up once per
// context).
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(SPH_ERR_CUDA, "cudaGetDevice failed");
    }
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(SPH_ERR_INVALID, "device index out of range");
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc != SPH_OK) return rc;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    Cached &c = g_addr[dev];
    if (!c.addr || c.ctx_id != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_query_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            c.addr = nullptr;
            return set_error(SPH_ERR_CUDA, "cudaGetSymbolAddress of the static search scratch failed");
        }
        c.addr = p;
        c.ctx_id = ctx;
    }
    *out = c.addr;
    return SPH_OK;
}

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" int sph_nnps_query_static(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity,
                                     float *rho, void *stream) {
    GridView v;
    int rc = grid_view(grid, &v);
    if (rc != SPH_OK) return rc;
    if (!row_ptr || !col || col_capacity < 0) return set_error(SPH_ERR_INVALID, "row_ptr and col are required");
    if (v.precision != SPH_PREC_FP16_RCLL || v.order != SPH_ORDER_CELL)
        return set_error(SPH_ERR_INVALID, "sph_nnps_query_static needs a grid binned with SPH_PREC_FP16_RCLL "
                                          "and SPH_ORDER_CELL");
    if (v.n > STATIC_MAX_N)
        return set_error(SPH_ERR_INVALID, "sph_nnps_query_static handles at most 1048576 particles");
    if (v.nrow > STATIC_MAX_ROWS)
        return set_error(SPH_ERR_INVALID, "sph_nnps_query_static handles at most 65536 rows of cells (ny * nz)");
    cudaStream_t s = (cudaStream_t)stream;
    if (v.n == 0) {
        if (cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s) != cudaSuccess) {
            cudaGetLastError();
            return set_error(SPH_ERR_CUDA, "cudaMemsetAsync failed");
        }
        return SPH_OK;
    }
    void *base = nullptr;
    rc = scratch_address(&base);
    if (rc != SPH_OK) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    int *tcount = reinterpret_cast<int *>(b + OFF_TCOUNT);
    long long *toff = reinterpret_cast<long long *>(b + OFF_TOFF);
    int4 *tiles = reinterpret_cast<int4 *>(b + OFF_TILES);
    unsigned long long *tstate = reinterpret_cast<unsigned long long *>(b + OFF_TSTATE);
    void *scan_tmp = b + OFF_SCAN;
    // plain runs of 32 particles per row: at most n / 32 + nrow + 1 tiles,
    // the bound the array is sized for (span-limited tiles could exceed it)
    const long long ntiles_max = v.n / 32 + v.nrow + 1;
    // the tile ticket counter must start at zero; the look-back state is
    // cleared by the launcher; everything else is fully rewritten
    TileLaunch tv;
    tv.shape = v.tile_shape;
    tv.extra = v.tile_extra;
    cudaError_t e = reset_counters_async(v.d.status, s);
    if (e == cudaSuccess) e = launch_tiles(v.d, false, tcount, toff, scan_tmp, tiles, nullptr, v.sm_count, s);
    if (e == cudaSuccess)
        e = launch_nnps_tile(v.d, nullptr, tiles, toff + v.nrow, ntiles_max, reinterpret_cast<long long *>(row_ptr),
                             col, col_capacity, rho, tstate, tv, false, v.sm_count, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(SPH_ERR_CUDA, cudaGetErrorString(e));
    }
    return SPH_OK;
}
