// api.cu -- C ABI of libsph (declared in include/sph.h): grid objects,
// parameter validation, the launch sequence of the binning and search steps,
// and error reporting.  No exception crosses the ABI.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {
cudaError_t launch_bounds(const double *xyz, long long n, int dim, DevStatus *st, int sm_count,
                          cudaStream_t s);
cudaError_t launch_hash_scatter_convert(const GridDev &g, const double *xyz, int n, int dim, int prec,
                                        int *cnt, int *cid, int *slot, int *cell_start, int *orig_id,
                                        int *rank, int *scell, uint2 *rel16, float4 *rel32, uint2 *rel16u,
                                        float4 *rel32u, double4 *x64,
                                        void *scan_tmp, int *big_list, unsigned int *big_count,
                                        int check_box, int sm_count, cudaStream_t s);
cudaError_t launch_nnps(const GridDev &g, int prec, int mode_fill, int *cnt, const long long *row_ptr,
                        int *col, long long cap, float *rho, int sm_count, cudaStream_t s);
cudaError_t launch_density(const GridDev &g, int prec, const int *rank, const int *scell,
                           const long long *row_ptr, const int *col, int canonical, float *rho,
                           int sm_count, cudaStream_t s);
cudaError_t launch_nnps_fused(const GridDev &g, long long *row_ptr, int *col, long long cap, float *rho,
                              unsigned long long *tstate, int *rowcnt, int sm_count, cudaStream_t s);
cudaError_t launch_tiles(const GridDev &g, const int *scell, int *scell_x, int *tcount, long long *toff,
                         void *scan_tmp, int4 *tiles, int sm_count, cudaStream_t s);
cudaError_t launch_nnps_tile(const GridDev &g, const int4 *tiles, const long long *ntiles_dev, long long ntiles_max,
                             long long *row_ptr, int *col, long long cap, float *rho, unsigned long long *tstate,
                             int sm_count, cudaStream_t s);
cudaError_t launch_canon(int n, const int *rank, const int *orig_id, const long long *rp_cell,
                         const int *col_cell, const float *rho_cell, int *cnt_tmp, void *scan_tmp,
                         long long *rp, int *col, float *rho, int *big_list, unsigned int *big_count,
                         int sm_count, cudaStream_t s);

__global__ void k_status_init(DevStatus *st) {
    st->flags = 0;
    st->big_cells = 0;
    for (int a = 0; a < 3; ++a) {
        st->min_key[a] = ~0ull;
        st->max_key[a] = 0ull;
    }
    st->fp32_pairs = 0;
    st->fp64_pairs = 0;
    st->nnz = 0;
    st->ticket = 0;
}

__global__ void k_status_reset_counters(DevStatus *st) {
    st->fp32_pairs = 0;
    st->fp64_pairs = 0;
    st->ticket = 0;
}
}  // namespace sph

using namespace sph;

// Error band of the FP16 "maybe" test and of the FP32 re-decision, in units
// of u^2 (u = h_c / 2).  Derivation (worst case over all pairs with r < kh,
// |x_rel| <= 1): FP16 rounding of x_rel <= 2^-12, of the pre-shifted
// candidate <= 2^-10, of the difference <= 2^-10, so |d - D| <= 2.5 * 2^-10
// per axis; squaring over three axes with |D| <= 2 adds <= 0.0169 and the
// three rounded FMAs of e = d^2 - T add <= 3 * 2^-10: 0.0199 < 0.03.  FP32:
// |d - D| <= 2 * 2^-25 + 2 * 2^-23 per axis -> <= 3.8e-6, plus three FMA
// roundings <= 7.2e-7 and the FP32 rounding of T: 4.7e-6 < 8e-6.
static const double TAU16 = 0.03;
static const double TAU32 = 8e-6;

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct sph_grid_s {
    sph_params p;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    long long n = 0;
    int nk[3] = {1, 1, 1};
    long long ncell = 1;
    double lo[3] = {0, 0, 0};
    double hc = 0;
    const double *xyz = nullptr;
    DevBuf cell_start, cnt, cid, slot, orig_id, rank, scell, rel16, rel32, rel16u, rel32u, x64, scan_tmp, big_list,
        rowcnt, tmp_rp, tmp_col, tmp_rho, status, own_xyz, own_rp, own_col, own_rho, tstate, scell_x, tcount,
        toff, tiles;
    int fused_enabled = 1;  // search variant for cell-order FP16 queries (SPH_OPT_FUSED)
    long long own_nnz = 0;
    DevStatus *h_status = nullptr;  // pinned host mirror
};

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define SPH_CUDA(x)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(SPH_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_));        \
        }                                                                                  \
    } while (0)

#define SPH_TRY(x)                   \
    do {                             \
        int r_ = (x);                \
        if (r_ != SPH_OK) return r_; \
    } while (0)

static int ensure(DevBuf &b, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return SPH_OK;
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.cap = 0;
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMallocAsync(&b.p, want, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SPH_ERR_NOMEM, "device allocation of %zu bytes failed: %s", want,
                    cudaGetErrorString(e));
    }
    b.cap = want;
    return SPH_OK;
}

static void release(DevBuf &b, cudaStream_t s) {
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.cap = 0;
}

template <typename T>
static T *P(DevBuf &b) {
    return reinterpret_cast<T *>(b.p);
}

static double kernel_alpha(int dim, double h) {
    const double pi = 3.14159265358979323846;
    return dim == 2 ? 15.0 / (7.0 * pi * h * h) : 3.0 / (2.0 * pi * h * h * h);
}

static float f32_down(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}
static float f32_up(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

static unsigned int half2_splat_bits(__half h) {
    __half2 v = __halves2half2(h, h);
    unsigned int u;
    memcpy(&u, &v, 4);
    return u;
}

static GridDev make_dev(sph_grid_s *g) {
    GridDev d;
    memset(&d, 0, sizeof(d));
    d.dim = g->p.dim;
    d.n = (int)g->n;
    for (int k = 0; k < 3; ++k) {
        d.nk[k] = g->nk[k];
        d.lo[k] = g->lo[k];
    }
    d.ncell = g->ncell;
    d.hc = g->hc;
    d.two_over_hc = 2.0 / g->hc;
    d.cell_start = P<int>(g->cell_start);
    d.rel16 = P<uint2>(g->rel16);
    d.rel32 = P<float4>(g->rel32);
    d.x64 = P<double>(g->x64);
    d.orig_id = P<int>(g->orig_id);
    d.scell_x = P<int>(g->scell_x);
    d.xyz = g->xyz;
    const double kh = g->p.kh, h = g->p.h;
    d.kh2 = kh * kh;
    const double u = g->hc * 0.5;
    const double T = d.kh2 / (u * u);
    d.t32_in = f32_down(T - TAU32);
    d.t32_out = f32_up(T + TAU32);
    // FP16 threshold rounded upward so that e = r2 - T16 never exceeds r2 - T.
    __half t16 = __double2half(T);
    if ((double)__half2float(t16) < T) t16 = __float2half_rn(nextafterf(__half2float(t16), INFINITY));
    while ((double)__half2float(t16) < T) {
        unsigned short b;
        memcpy(&b, &t16, 2);
        ++b;
        memcpy(&t16, &b, 2);
    }
    d.neg_t16 = half2_splat_bits(__hneg(t16));
    d.tau16 = half2_splat_bits(__double2half(TAU16));
    const double alpha = kernel_alpha(g->p.dim, h);
    d.r_scale = (float)(u / h);
    d.w_norm = (float)(g->p.mass * alpha);
    d.w_self = (float)(g->p.mass * alpha * (2.0 / 3.0));
    d.r_scale64 = 1.0 / h;
    d.w_norm64 = g->p.mass * alpha;
    d.w_self64 = g->p.mass * alpha * (2.0 / 3.0);
    d.status = P<DevStatus>(g->status);
    return d;
}

static int status_to_code(unsigned int flags) {
    if (flags & ST_NONFINITE) return fail(SPH_ERR_INVALID, "non-finite particle coordinate");
    if (flags & ST_OUT_OF_BOX) return fail(SPH_ERR_INVALID, "particle outside the given box");
    if (flags & ST_TIMEOUT) return fail(SPH_ERR_TIMEOUT, "a bounded device wait ran out");
    if (flags & ST_CAPACITY) return fail(SPH_ERR_CAPACITY, "nnz exceeds col_capacity");
    if (flags & ST_DEVICE_CHECK) return fail(SPH_ERR_DEVICE_CHECK, "device consistency check failed");
    return SPH_OK;
}

// Copy the status record to the host mirror and wait.
static int read_status(sph_grid_s *g) {
    SPH_CUDA(cudaMemcpyAsync(g->h_status, g->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                             g->stream));
    SPH_CUDA(cudaStreamSynchronize(g->stream));
    return SPH_OK;
}

static int validate(const sph_params *p, int64_t n, const double *xyz) {
    if (!p) return fail(SPH_ERR_INVALID, "params is NULL");
    if (p->dim != 2 && p->dim != 3) return fail(SPH_ERR_INVALID, "dim must be 2 or 3 (got %d)", p->dim);
    if (p->order != SPH_ORDER_CELL && p->order != SPH_ORDER_CANONICAL)
        return fail(SPH_ERR_INVALID, "unknown order %d", p->order);
    if (p->precision != SPH_PREC_FP16_RCLL && p->precision != SPH_PREC_FP64_CLL)
        return fail(SPH_ERR_INVALID, "unknown precision %d", p->precision);
    if (!(p->kh > 0) || !isfinite(p->kh)) return fail(SPH_ERR_INVALID, "kh must be finite and > 0");
    if (!(p->h > 0) || !isfinite(p->h)) return fail(SPH_ERR_INVALID, "h must be finite and > 0");
    if (!isfinite(p->mass)) return fail(SPH_ERR_INVALID, "mass must be finite");
    const double hc_min = p->kh * (1.0 + 0x1p-30);
    if (p->cell_size != 0 && !(p->cell_size >= hc_min && isfinite(p->cell_size)))
        return fail(SPH_ERR_INVALID, "cell_size must be 0 or >= kh * (1 + 2^-30)");
    if (n < 0 || n >= 0x7fffffffLL) return fail(SPH_ERR_INVALID, "n out of range: %lld", (long long)n);
    if (n > 0 && xyz == nullptr) return fail(SPH_ERR_INVALID, "xyz is NULL");
    if (p->have_box) {
        for (int k = 0; k < p->dim; ++k)
            if (!isfinite(p->box_lo[k]) || !isfinite(p->box_hi[k]) || !(p->box_hi[k] >= p->box_lo[k]))
                return fail(SPH_ERR_INVALID, "invalid box on axis %d", k);
    }
    return SPH_OK;
}

extern "C" int sph_version(void) { return 100; }

extern "C" int sph_precision_bands(double *tau16, double *tau32) {
    if (tau16) *tau16 = TAU16;
    if (tau32) *tau32 = TAU32;
    return SPH_OK;
}

extern "C" const char *sph_last_error(void) { return g_err.c_str(); }

static int grid_create(sph_grid_s **out) {
    sph_grid_s *g = new (std::nothrow) sph_grid_s();
    if (!g) return fail(SPH_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_status, sizeof(DevStatus));
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return fail(SPH_ERR_CUDA, "CUDA initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = g;
    return SPH_OK;
}

extern "C" int sph_bin_cells(const sph_params *p, const double *xyz, int64_t n, void *stream,
                             sph_grid_t *grid) {
    if (!grid) return fail(SPH_ERR_INVALID, "grid is NULL");
    SPH_TRY(validate(p, n, xyz));
    bool created = false;
    if (*grid == nullptr) {
        SPH_TRY(grid_create(grid));
        created = true;
    }
    sph_grid_s *g = *grid;
    cudaStream_t s = (cudaStream_t)stream;
    g->p = *p;
    g->stream = s;
    g->n = n;
    g->xyz = xyz;
    g->hc = p->cell_size != 0 ? p->cell_size : p->kh * (1.0 + 0x1p-30);
    const int dim = p->dim;
    int rc = SPH_OK;
    do {
        if ((rc = ensure(g->status, sizeof(DevStatus), s)) != SPH_OK) break;
        note_launch(1);
        k_status_init<<<1, 1, 0, s>>>(P<DevStatus>(g->status));
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        if (p->have_box) {
            for (int k = 0; k < dim; ++k) {
                lo[k] = p->box_lo[k];
                hi[k] = p->box_hi[k];
            }
        } else if (n > 0) {
            if (launch_bounds(xyz, n, dim, P<DevStatus>(g->status), g->sm_count, s) != cudaSuccess) {
                rc = fail(SPH_ERR_CUDA, "bounds launch failed");
                break;
            }
            if ((rc = read_status(g)) != SPH_OK) break;
            if (g->h_status->flags & ST_NONFINITE) {
                rc = fail(SPH_ERR_INVALID, "non-finite particle coordinate");
                break;
            }
            for (int k = 0; k < dim; ++k) {
                lo[k] = dkey_inv(g->h_status->min_key[k]);
                hi[k] = dkey_inv(g->h_status->max_key[k]);
            }
        }
        long long ncell = 1;
        for (int k = 0; k < 3; ++k) {
            g->lo[k] = lo[k];
            g->nk[k] = 1;
            if (k < dim) {
                double span = ceil((hi[k] - lo[k]) / g->hc);
                if (!(span <= (double)(1 << 20))) {
                    rc = fail(SPH_ERR_INVALID, "more than 2^20 cells along axis %d", k);
                    break;
                }
                g->nk[k] = span < 1.0 ? 1 : (int)span;
            }
            ncell *= g->nk[k];
        }
        if (rc != SPH_OK) break;
        if (ncell > (1LL << 28)) {
            rc = fail(SPH_ERR_INVALID, "grid of %lld cells exceeds 2^28", ncell);
            break;
        }
        g->ncell = ncell;
        const long long nn = n > 0 ? n : 1;
        const long long big = ncell > nn ? ncell : nn;
        if ((rc = ensure(g->cell_start, (ncell + 1) * sizeof(int), s)) ||
            (rc = ensure(g->cnt, ncell * sizeof(int), s)) || (rc = ensure(g->cid, nn * sizeof(int), s)) ||
            (rc = ensure(g->slot, nn * sizeof(int), s)) || (rc = ensure(g->orig_id, nn * sizeof(int), s)) ||
            (rc = ensure(g->rank, nn * sizeof(int), s)) || (rc = ensure(g->scell, nn * sizeof(int), s)) ||
            (rc = ensure(g->scan_tmp, scan_tmp_bytes(big + 1), s)) ||
            (rc = ensure(g->big_list, big * sizeof(int), s)))
            break;
        if (p->precision == SPH_PREC_FP16_RCLL) {
            if ((rc = ensure(g->rel16, nn * sizeof(uint2), s)) || (rc = ensure(g->rel32, nn * sizeof(float4), s)) ||
                (rc = ensure(g->rel16u, nn * sizeof(uint2), s)) || (rc = ensure(g->rel32u, nn * sizeof(float4), s)))
                break;
        } else {
            if ((rc = ensure(g->x64, nn * sizeof(double4), s))) break;
        }
        if (n == 0) {
            if (cudaMemsetAsync(g->cell_start.p, 0, (ncell + 1) * sizeof(int), s) != cudaSuccess) {
                rc = fail(SPH_ERR_CUDA, "memset failed");
                break;
            }
            break;
        }
        GridDev d = make_dev(g);
        cudaError_t e = launch_hash_scatter_convert(
            d, xyz, (int)n, dim, p->precision, P<int>(g->cnt), P<int>(g->cid), P<int>(g->slot),
            P<int>(g->cell_start), P<int>(g->orig_id), P<int>(g->rank), P<int>(g->scell), P<uint2>(g->rel16),
            P<float4>(g->rel32), P<uint2>(g->rel16u), P<float4>(g->rel32u), P<double4>(g->x64), g->scan_tmp.p, P<int>(g->big_list),
            &P<DevStatus>(g->status)->big_cells, p->have_box, g->sm_count, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(SPH_ERR_CUDA, "binning launch failed: %s", cudaGetErrorString(e));
        }
    } while (0);
    if (rc != SPH_OK && created) {
        sph_grid_free(*grid);
        *grid = nullptr;
    }
    return rc;
}

extern "C" int sph_nnps_query(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity,
                              int64_t *nnz_out, float *rho, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!row_ptr) return fail(SPH_ERR_INVALID, "row_ptr is NULL");
    if (col && col_capacity < 0) return fail(SPH_ERR_INVALID, "negative col_capacity");
    if (rho && !col) return fail(SPH_ERR_INVALID, "rho needs col (the density is fused into the fill)");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    const long long n = g->n;
    if (n == 0) {
        SPH_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
        if (nnz_out) {
            SPH_CUDA(cudaStreamSynchronize(s));
            *nnz_out = 0;
        }
        return SPH_OK;
    }
    GridDev d = make_dev(g);
    note_launch(1);
    k_status_reset_counters<<<1, 1, 0, s>>>(P<DevStatus>(g->status));
    SPH_TRY(ensure(g->rowcnt, n * sizeof(int), s));
    const bool canonical = g->p.order == SPH_ORDER_CANONICAL;
    const int prec = g->p.precision;
    long long *rp_cell = reinterpret_cast<long long *>(row_ptr);
    if (canonical) {
        SPH_TRY(ensure(g->tmp_rp, (n + 1) * sizeof(long long), s));
        rp_cell = P<long long>(g->tmp_rp);
    }
    const bool fused = !canonical && col != nullptr && prec == SPH_PREC_FP16_RCLL && g->fused_enabled;
    if (fused && g->fused_enabled == 2) {
        // single pass, one CTA per cell, row offsets by look-back across cells
        SPH_TRY(ensure(g->tstate, (size_t)g->ncell * sizeof(unsigned long long), s));
        SPH_CUDA(launch_nnps_fused(d, rp_cell, col, col_capacity, rho, P<unsigned long long>(g->tstate),
                                   P<int>(g->rowcnt), g->sm_count, s));
    } else if (fused) {
        // single pass, one warp per 32-particle row tile, look-back across tiles
        const long long nrow = (long long)g->nk[1] * g->nk[2];
        const long long ntiles_max = n / 32 + nrow + 1;
        SPH_TRY(ensure(g->scell_x, n * sizeof(int), s));
        SPH_TRY(ensure(g->tcount, nrow * sizeof(int), s));
        SPH_TRY(ensure(g->toff, (nrow + 1) * sizeof(long long), s));
        SPH_TRY(ensure(g->tiles, ntiles_max * sizeof(int4), s));
        SPH_TRY(ensure(g->tstate, ntiles_max * sizeof(unsigned long long), s));
        d = make_dev(g);
        SPH_CUDA(launch_tiles(d, P<int>(g->scell), P<int>(g->scell_x), P<int>(g->tcount), P<long long>(g->toff),
                              g->scan_tmp.p, P<int4>(g->tiles), g->sm_count, s));
        SPH_CUDA(launch_nnps_tile(d, P<int4>(g->tiles), P<long long>(g->toff) + nrow, ntiles_max, rp_cell, col,
                                  col_capacity, rho, P<unsigned long long>(g->tstate), g->sm_count, s));
    } else {
        SPH_CUDA(launch_nnps(d, prec, 0, P<int>(g->rowcnt), nullptr, nullptr, 0, nullptr, g->sm_count, s));
        SPH_CUDA(exclusive_scan_i64(P<int>(g->rowcnt), rp_cell, n, g->scan_tmp.p, s));
    }
    if (!canonical) {
        if (col && !fused)
            SPH_CUDA(launch_nnps(d, prec, 1, nullptr, rp_cell, col, col_capacity, rho, g->sm_count, s));
        if (nnz_out) {
            SPH_CUDA(cudaMemcpyAsync(&g->h_status->nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            long long nnz_host = 0;
            SPH_CUDA(cudaStreamSynchronize(s));
            nnz_host = g->h_status->nnz;
            SPH_TRY(read_status(g));
            *nnz_out = nnz_host;
            int rc = status_to_code(g->h_status->flags);
            if (rc == SPH_OK && col && nnz_host > col_capacity)
                rc = fail(SPH_ERR_CAPACITY, "nnz %lld exceeds col_capacity %lld", nnz_host,
                          (long long)col_capacity);
            return rc;
        }
        return SPH_OK;
    }
    // Canonical order: learn nnz first (this path always synchronises).
    long long nnz = 0;
    SPH_CUDA(cudaMemcpyAsync(&g->h_status->nnz, rp_cell + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    nnz = g->h_status->nnz;
    if (nnz_out) *nnz_out = nnz;
    if (col && nnz > col_capacity) {
        SPH_TRY(launch_canon((int)n, P<int>(g->rank), P<int>(g->orig_id), rp_cell, nullptr, nullptr,
                             P<int>(g->rowcnt), g->scan_tmp.p, reinterpret_cast<long long *>(row_ptr), nullptr,
                             nullptr, P<int>(g->big_list), &P<DevStatus>(g->status)->big_cells, g->sm_count, s) ==
                        cudaSuccess
                    ? SPH_OK
                    : fail(SPH_ERR_CUDA, "canonical row pointer launch failed"));
        SPH_CUDA(cudaStreamSynchronize(s));
        return fail(SPH_ERR_CAPACITY, "nnz %lld exceeds col_capacity %lld", nnz, (long long)col_capacity);
    }
    if (col) {
        SPH_TRY(ensure(g->tmp_col, (nnz > 0 ? nnz : 1) * sizeof(int), s));
        if (rho) SPH_TRY(ensure(g->tmp_rho, n * sizeof(float), s));
        SPH_CUDA(launch_nnps(d, prec, 1, nullptr, rp_cell, P<int>(g->tmp_col), nnz, rho ? P<float>(g->tmp_rho) : nullptr,
                             g->sm_count, s));
    }
    // row lengths are needed again: rowcnt is reused as scratch by launch_canon
    SPH_CUDA(launch_canon((int)n, P<int>(g->rank), P<int>(g->orig_id), rp_cell, P<int>(g->tmp_col),
                          rho ? P<float>(g->tmp_rho) : nullptr, P<int>(g->rowcnt), g->scan_tmp.p,
                          reinterpret_cast<long long *>(row_ptr), col, rho, P<int>(g->big_list),
                          &P<DevStatus>(g->status)->big_cells, g->sm_count, s));
    SPH_TRY(read_status(g));
    return status_to_code(g->h_status->flags);
}

extern "C" int sph_density_sum(sph_grid_t grid, const int64_t *row_ptr, const int32_t *col, float *rho,
                               void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!row_ptr || !rho || (!col && g->n > 0)) return fail(SPH_ERR_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    if (g->n == 0) return SPH_OK;
    GridDev d = make_dev(g);
    SPH_CUDA(launch_density(d, g->p.precision, P<int>(g->rank), P<int>(g->scell),
                            reinterpret_cast<const long long *>(row_ptr), col,
                            g->p.order == SPH_ORDER_CANONICAL, rho, g->sm_count, s));
    return SPH_OK;
}

extern "C" int sph_grid_info_get(sph_grid_t grid, sph_grid_info *info) {
    sph_grid_s *g = grid;
    if (!g || !info) return fail(SPH_ERR_INVALID, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->ncell = g->ncell;
    info->dim = g->p.dim;
    for (int k = 0; k < 3; ++k) {
        info->nk[k] = g->nk[k];
        info->lo[k] = g->lo[k];
    }
    info->cell_size = g->hc;
    info->cell_start = P<int>(g->cell_start);
    info->orig_id = P<int>(g->orig_id);
    info->rank = P<int>(g->rank);
    if (g->h_status) {
        info->stat_fp32_pairs = (int64_t)g->h_status->fp32_pairs;
        info->stat_fp64_pairs = (int64_t)g->h_status->fp64_pairs;
    }
    return SPH_OK;
}

extern "C" int sph_grid_export(sph_grid_t grid, int32_t *orig_id, int32_t *rank, int32_t *cell_start,
                               void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (orig_id && g->n)
        SPH_CUDA(cudaMemcpyAsync(orig_id, g->orig_id.p, g->n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (rank && g->n)
        SPH_CUDA(cudaMemcpyAsync(rank, g->rank.p, g->n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (cell_start && g->cell_start.p)
        SPH_CUDA(cudaMemcpyAsync(cell_start, g->cell_start.p, (g->ncell + 1) * sizeof(int),
                                 cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

extern "C" int sph_grid_set_option(sph_grid_t grid, int option, int64_t value) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (option == SPH_OPT_FUSED) {
        if (value < 0 || value > 2) return fail(SPH_ERR_INVALID, "SPH_OPT_FUSED takes 0, 1 or 2");
        g->fused_enabled = (int)value;
        return SPH_OK;
    }
    return fail(SPH_ERR_INVALID, "unknown option %d", option);
}

extern "C" int sph_grid_check(sph_grid_t grid, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    g->stream = (cudaStream_t)stream;
    if (!g->status.p) return SPH_OK;
    SPH_TRY(read_status(g));
    return status_to_code(g->h_status->flags);
}

extern "C" int sph_search_host(const sph_params *p, const double *xyz_host, int64_t n, float *rho_host,
                               int64_t *nnz_host, sph_grid_t *grid, void *stream) {
    if (!grid) return fail(SPH_ERR_INVALID, "grid is NULL");
    SPH_TRY(validate(p, n, xyz_host));
    cudaStream_t s = (cudaStream_t)stream;
    if (*grid == nullptr) SPH_TRY(grid_create(grid));
    sph_grid_s *g = *grid;
    g->stream = s;
    const size_t xbytes = (size_t)(n > 0 ? n : 1) * p->dim * sizeof(double);
    SPH_TRY(ensure(g->own_xyz, xbytes, s));
    if (n > 0) SPH_CUDA(cudaMemcpyAsync(g->own_xyz.p, xyz_host, (size_t)n * p->dim * sizeof(double),
                                        cudaMemcpyHostToDevice, s));
    SPH_TRY(sph_bin_cells(p, P<double>(g->own_xyz), n, stream, grid));
    SPH_TRY(ensure(g->own_rp, (size_t)(n + 1) * sizeof(long long), s));
    SPH_TRY(ensure(g->own_rho, (size_t)(n > 0 ? n : 1) * sizeof(float), s));
    int64_t nnz = 0;
    const long long cap = (long long)(g->own_col.cap / sizeof(int));
    int rc = sph_nnps_query(g, P<int64_t>(g->own_rp), g->own_col.p ? P<int32_t>(g->own_col) : nullptr, cap,
                            &nnz, g->own_col.p ? P<float>(g->own_rho) : nullptr, stream);
    if (rc == SPH_ERR_CAPACITY || (rc == SPH_OK && !g->own_col.p)) {
        SPH_TRY(ensure(g->own_col, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int), s));
        rc = sph_nnps_query(g, P<int64_t>(g->own_rp), P<int32_t>(g->own_col),
                            (long long)(g->own_col.cap / sizeof(int)), &nnz, P<float>(g->own_rho), stream);
    }
    if (rc != SPH_OK) return rc;
    g->own_nnz = nnz;
    if (rho_host && n > 0)
        SPH_CUDA(cudaMemcpyAsync(rho_host, g->own_rho.p, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    if (nnz_host) *nnz_host = nnz;
    return SPH_OK;
}

extern "C" int sph_grid_csr(sph_grid_t grid, const int64_t **row_ptr, const int32_t **col, const float **rho,
                            int64_t *nnz) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (row_ptr) *row_ptr = P<int64_t>(g->own_rp);
    if (col) *col = P<int32_t>(g->own_col);
    if (rho) *rho = P<float>(g->own_rho);
    if (nnz) *nnz = g->own_nnz;
    return SPH_OK;
}

extern "C" int sph_profile_enable(int on) {
    prof_enable(on);
    return SPH_OK;
}

extern "C" int sph_profile_select(const char *kernels) {
    if (prof_select(kernels) != 0) return fail(SPH_ERR_INVALID, "unknown kernel tag in \"%s\"", kernels);
    return SPH_OK;
}

extern "C" int sph_device_fp64_rate(double *flops) {
    if (!flops) return fail(SPH_ERR_INVALID, "NULL argument");
    if (fp64_fma_rate(flops) != 0) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "FP64 rate measurement failed");
    }
    return SPH_OK;
}

extern "C" int sph_profile_reset(void) {
    prof_reset();
    return SPH_OK;
}

extern "C" int sph_profile_read(const char *kernel, double *total_ms, int64_t *launches) {
    if (!kernel) return fail(SPH_ERR_INVALID, "kernel name is NULL");
    long long c = 0;
    if (prof_read(kernel, total_ms, &c) != 0) return fail(SPH_ERR_NOT_FOUND, "unknown kernel tag %s", kernel);
    if (launches) *launches = c;
    return SPH_OK;
}

extern "C" int64_t sph_launch_count(void) { return launch_count(); }

namespace sph {

int grid_view(sph_grid_t grid, GridView *v) {
    sph_grid_s *g = grid;
    if (!g || !v) return fail(SPH_ERR_INVALID, "grid is NULL");
    v->d = make_dev(g);
    v->scell = P<int>(g->scell);
    v->sm_count = g->sm_count;
    v->precision = g->p.precision;
    v->order = g->p.order;
    v->n = g->n;
    v->nrow = (long long)g->nk[1] * g->nk[2];
    return SPH_OK;
}

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

void reset_counters_async(DevStatus *st, cudaStream_t s) {
    note_launch(1);
    k_status_reset_counters<<<1, 1, 0, s>>>(st);
}

}  // namespace sph

extern "C" int sph_grid_free(sph_grid_t grid) {
    sph_grid_s *g = grid;
    if (!g) return SPH_OK;
    cudaStream_t s = g->stream;
    DevBuf *bufs[] = {&g->cell_start, &g->cnt, &g->cid, &g->slot, &g->orig_id, &g->rank, &g->scell,
                      &g->rel16, &g->rel32, &g->rel16u, &g->rel32u, &g->x64, &g->scan_tmp, &g->big_list,
                      &g->rowcnt, &g->tmp_rp, &g->tmp_col, &g->tmp_rho, &g->status, &g->own_xyz, &g->own_rp, &g->own_col, &g->own_rho,
                      &g->tstate, &g->scell_x, &g->tcount, &g->toff, &g->tiles};
    for (DevBuf *b : bufs) release(*b, s);
    if (g->h_status) {
        cudaStreamSynchronize(s);
        cudaFreeHost(g->h_status);
    }
    cudaGetLastError();
    delete g;
    return SPH_OK;
}
