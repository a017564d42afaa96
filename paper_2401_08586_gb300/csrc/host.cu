// host.cu -- host-side helpers shared by the C-ABI translation units.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <string>

#include "host.cuh"
#include "profile.cuh"

namespace sph {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

const char *last_error() { return g_err.c_str(); }

int ensure(DevBuf &b, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return SPH_OK;
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.cap = 0;
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMallocAsync(&b.p, want, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SPH_ERR_NOMEM, "device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
    return SPH_OK;
}

void release(DevBuf &b, cudaStream_t s) {
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.cap = 0;
}

int status_to_code(unsigned int flags) {
    if (flags & ST_NONFINITE) return fail(SPH_ERR_INVALID, "non-finite particle coordinate");
    if (flags & ST_OUT_OF_BOX) return fail(SPH_ERR_INVALID, "particle outside the given box");
    if (flags & ST_TIMEOUT) return fail(SPH_ERR_TIMEOUT, "a bounded device wait ran out");
    if (flags & ST_CAPACITY) return fail(SPH_ERR_CAPACITY, "nnz exceeds col_capacity");
    if (flags & ST_DEVICE_CHECK) return fail(SPH_ERR_DEVICE_CHECK, "device consistency check failed");
    return SPH_OK;
}

int validate_params(const sph_params *p, int64_t n, const double *xyz) {
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

void set_divisors(GridDev &d) {
    d.div_nx = fastdiv_make((uint32_t)d.nk[0]);
    d.div_nxy = fastdiv_make((uint32_t)d.nk[0] * (uint32_t)d.nk[1]);
}

void set_constants(GridDev &d, const sph_params &p, double hc) {
    const double kh = p.kh, h = p.h;
    d.kh2 = kh * kh;
    const double u = hc * 0.5;
    const double T = d.kh2 / (u * u);
    d.t32_in = f32_down(T - TAU32);
    d.t32_out = f32_up(T + TAU32);
    // FP16 threshold rounded upward so that e = r2 - T16 never exceeds r2 - T.
    __half t16 = __double2half(T);
    while ((double)__half2float(t16) < T) {
        unsigned short b;
        memcpy(&b, &t16, 2);
        ++b;
        memcpy(&t16, &b, 2);
    }
    d.neg_t16 = half2_splat_bits(__hneg(t16));
    d.tau16 = half2_splat_bits(__double2half(TAU16));
    const double alpha = kernel_alpha(p.dim, h);
    d.r_scale = (float)(u / h);
    d.w_norm = (float)(p.mass * alpha);
    d.w_self = (float)(p.mass * alpha * (2.0 / 3.0));
    d.r_scale64 = 1.0 / h;
    d.w_norm64 = p.mass * alpha;
    d.w_self64 = p.mass * alpha * (2.0 / 3.0);
}

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

// Per-query state: the tier counters, the tile ticket and the flags a query
// raises (capacity, timeout); the binning flags stay.  first_ticket is 0
// except in the bounded-wait test (SPH_OPT_TEST_LOOKBACK), which starts at 1.
__global__ void k_status_reset_counters(DevStatus *st, unsigned long long first_ticket) {
    st->fp32_pairs = 0;
    st->fp64_pairs = 0;
    st->ticket = first_ticket;
    st->flags &= ~(ST_CAPACITY | ST_TIMEOUT);
}

__global__ void k_copy_words(unsigned int *__restrict__ dst, const unsigned int *__restrict__ src, long long words) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void k_status_to_host(DevStatus *host, const DevStatus *st, const long long *nnz_src) {
    const unsigned int *src = reinterpret_cast<const unsigned int *>(st);
    unsigned int *dst = reinterpret_cast<unsigned int *>(host);
    for (int i = threadIdx.x; i < (int)(sizeof(DevStatus) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0 && nnz_src != nullptr) host->nnz = *nnz_src;
}

__global__ void k_status_to_host_flag(DevStatus *host, const DevStatus *st, unsigned int *flag, unsigned int seq) {
    const unsigned int *src = reinterpret_cast<const unsigned int *>(st);
    unsigned int *dst = reinterpret_cast<unsigned int *>(host);
    for (int i = threadIdx.x; i < (int)(sizeof(DevStatus) / 4); i += blockDim.x) dst[i] = src[i];
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) *reinterpret_cast<volatile unsigned int *>(flag) = seq;
}

__global__ void k_gather_i64(long long *host, const long long *src, const long long *idx, int count) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) host[i] = src[idx[i]];
}

cudaError_t copy_small_to_host(void *host_dst, const void *dev_src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    note_launch(1);
    k_copy_words<<<1, 128, 0, s>>>(static_cast<unsigned int *>(host_dst), static_cast<const unsigned int *>(dev_src),
                                   (long long)(bytes / 4));
    return cudaGetLastError();
}

cudaError_t status_to_host(DevStatus *host_dst, const DevStatus *dev_src, const long long *nnz_src, cudaStream_t s) {
    static_assert(sizeof(DevStatus) % 4 == 0, "status record in words");
    note_launch(1);
    k_status_to_host<<<1, 32, 0, s>>>(host_dst, dev_src, nnz_src);
    return cudaGetLastError();
}

cudaError_t status_to_host_flag(DevStatus *host_dst, const DevStatus *dev_src, unsigned int *host_flag,
                                unsigned int seq, cudaStream_t s) {
    note_launch(1);
    k_status_to_host_flag<<<1, 32, 0, s>>>(host_dst, dev_src, host_flag, seq);
    return cudaGetLastError();
}

bool wait_host_flag(const unsigned int *host_flag, unsigned int seq, double max_us) {
    const volatile unsigned int *f = host_flag;
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned long long it = 0;; ++it) {
        if (*f == seq) {
            std::atomic_thread_fence(std::memory_order_acquire);
            return true;
        }
        if ((it & 1023) == 1023 &&
            std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count() > max_us)
            return false;
    }
}

cudaError_t gather_i64_to_host(long long *host_dst, const long long *src, const long long *idx, int count,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    note_launch(1);
    k_gather_i64<<<1, 128, 0, s>>>(host_dst, src, idx, count);
    return cudaGetLastError();
}

cudaError_t copy_d2d_kernel(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    const long long words = (long long)(bytes / 4);
    if (words == 0) return cudaSuccess;
    long long blocks = (words + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    note_launch(1);
    k_copy_words<<<(unsigned)blocks, 256, 0, s>>>(static_cast<unsigned int *>(dst), static_cast<const unsigned int *>(src),
                                                  words);
    return cudaGetLastError();
}

cudaError_t launch_status_init(DevStatus *st, cudaStream_t s) {
    note_launch(1);
    k_status_init<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_status_reset_counters(DevStatus *st, cudaStream_t s, unsigned long long first_ticket) {
    note_launch(1);
    k_status_reset_counters<<<1, 1, 0, s>>>(st, first_ticket);
    return cudaGetLastError();
}

}  // namespace sph
