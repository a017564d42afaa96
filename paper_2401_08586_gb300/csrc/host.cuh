// host.cuh -- host-side helpers shared by the C-ABI translation units:
// error reporting, stream-ordered device buffers, parameter validation and
// the per-grid constants of the precision tiers (host.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "sph_internal.cuh"

namespace sph {

// Error band of the FP16 "maybe" test and of the FP32 re-decision, in units
// of u^2 (u = h_c / 2).  Derivation (worst case over all pairs with r < kh,
// |x_rel| <= 1): FP16 rounding of x_rel <= 2^-12, of the pre-shifted
// candidate <= 2^-10, of the difference <= 2^-10, so |d - D| <= 2.5 * 2^-10
// per axis; squaring over three axes with |D| <= 2 adds <= 0.0169 and the
// three rounded FMAs of e = d^2 - T add <= 3 * 2^-10: 0.0199 < 0.03.  FP32:
// |d - D| <= 2 * 2^-25 + 2 * 2^-23 per axis -> <= 3.8e-6, plus three FMA
// roundings <= 7.2e-7 and the FP32 rounding of T: 4.7e-6 < 8e-6.
constexpr double TAU16 = 0.03;
constexpr double TAU32 = 8e-6;

// A device buffer that only grows (stream-ordered allocation).
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

template <typename T>
inline T *P(DevBuf &b) {
    return reinterpret_cast<T *>(b.p);
}

// Record a formatted message for sph_last_error (thread-local) and return code.
int fail(int code, const char *fmt, ...);
const char *last_error();

// Grow b to at least `bytes` (contents are not kept); SPH_ERR_NOMEM on failure.
int ensure(DevBuf &b, size_t bytes, cudaStream_t s);
void release(DevBuf &b, cudaStream_t s);

// SPH_OK, or the error of the first status flag set.
int status_to_code(unsigned int flags);

// Checks of one system's parameters and input (n, xyz != NULL when n > 0).
int validate_params(const sph_params *p, int64_t n, const double *xyz);

// The precision-tier thresholds and kernel normalisation of a grid with
// cell size hc (fields kh2 ... w_self64 of GridDev).
void set_constants(GridDev &d, const sph_params &p, double hc);
// The launch-invariant divisors of the grid's cell ids (nk filled first).
void set_divisors(GridDev &d);

// Small device -> host and device -> device copies done by a kernel instead
// of a copy engine.  The control path of a query (status record, nnz, a
// batch's row offsets) and the server's per-request copies then never wait
// in a copy engine's queue behind another stream's large transfer (a client
// copying a 600 MB result back).  host_dst: pinned host memory (mapped into
// the device's address space, as all pinned memory is under unified
// addressing); bytes and both addresses multiples of 4.  The data is visible
// to the host once the stream has been synchronised.
cudaError_t copy_small_to_host(void *host_dst, const void *dev_src, size_t bytes, cudaStream_t s);
// The status record and, if nnz_src != NULL, the value at nnz_src into the
// record's nnz field, in one launch.
cudaError_t status_to_host(DevStatus *host_dst, const DevStatus *dev_src, const long long *nnz_src, cudaStream_t s);
// The same without nnz, then *host_flag = seq once the record is written and
// visible to the host (pinned memory), so that the host can wait for it with
// wait_host_flag instead of synchronising the stream.
cudaError_t status_to_host_flag(DevStatus *host_dst, const DevStatus *dev_src, unsigned int *host_flag,
                                unsigned int seq, cudaStream_t s);
// Spin until *host_flag == seq (then every write the device made before the
// flag is visible), at most max_us microseconds; false if it timed out.
bool wait_host_flag(const unsigned int *host_flag, unsigned int seq, double max_us);
// host_dst[i] = src[idx[i]] for i < count (int64 gathers into pinned memory;
// idx in pinned host memory too).
cudaError_t gather_i64_to_host(long long *host_dst, const long long *src, const long long *idx, int count,
                               cudaStream_t s);
// dst[0, bytes) = src[0, bytes) on the device (4-byte multiples).
cudaError_t copy_d2d_kernel(void *dst, const void *src, size_t bytes, cudaStream_t s);

// Host launchers of the status-record kernels.
cudaError_t launch_status_init(DevStatus *st, cudaStream_t s);
cudaError_t launch_status_reset_counters(DevStatus *st, cudaStream_t s, unsigned long long first_ticket = 0);

}  // namespace sph

#define SPH_CUDA(x)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return ::sph::fail(SPH_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_)); \
        }                                                                                  \
    } while (0)

#define SPH_TRY(x)                   \
    do {                             \
        int r_ = (x);                \
        if (r_ != SPH_OK) return r_; \
    } while (0)
