// sph_internal.cuh -- device-side structures shared by the libsph kernels.
//
// Notation (arXiv 2401.08586): h is the smoothing length, kh the search
// radius, h_c the background cell size, u = h_c / 2 the unit of the
// normalised cell-relative coordinates of Eq. 6 (x_rel = 2 (x - x_cc) / h_c,
// in [-1, 1], x_cc the cell centre).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fastdiv.h"
#include "sph.h"

namespace sph {

// Bits of the per-grid device status word.
enum : unsigned int {
    ST_NONFINITE = 1u << 0,     // a coordinate was NaN or infinite
    ST_OUT_OF_BOX = 1u << 1,    // a particle lies outside the caller's box
    ST_TIMEOUT = 1u << 2,       // a bounded device wait ran out
    ST_CAPACITY = 1u << 3,      // nnz exceeded the col capacity
    ST_DEVICE_CHECK = 1u << 4,  // an internal consistency check fired
};

// Small device-resident record each grid owns: status flags, bounding-box
// reduction slots (doubles mapped to order-preserving unsigned keys) and
// counters of the precision tiers.
struct DevStatus {
    unsigned int flags;
    unsigned int big_cells;          // cells with more than 32 particles (sort fallback list length)
    unsigned long long min_key[3];
    unsigned long long max_key[3];
    unsigned long long fp32_pairs;   // pairs re-decided in FP32
    unsigned long long fp64_pairs;   // pairs decided by the FP64 tier
    long long nnz;
    unsigned long long ticket;       // tile ticket of the single-pass query
};

// Everything a search kernel needs, passed by value.
struct GridDev {
    int dim;
    int n;
    int nk[3];
    long long ncell;
    double lo[3];
    double hc;           // h_c
    double two_over_hc;  // 2 / h_c: FP64 units -> u
    double neg_lo_t[3];  // -lo * 2 / h_c (binning in one FMA, when fma_bin)
    int fma_bin;         // 1: every coordinate is within 2^17 u of the origin
    FastDiv div_nx;      // division by nk[0] (cells per row)
    FastDiv div_nxy;     // division by nk[0] * nk[1] (cells per layer)
    const int *cell_start;
    const uint2 *rel16;   // per sorted particle: half x_rel, y_rel | z_rel, 0
    const float4 *rel32;  // per sorted particle: x_rel, y_rel, z_rel, 0
    const double *x64;    // FP64-CLL mode: cell-ordered coordinates, 4 doubles per particle
    const int *orig_id;   // sorted position -> input index
    const int *scell_x;   // cell x of each sorted particle (row-tile search)
    const double *xyz;    // caller coordinates (input order, n x dim)
    double kh2;           // kh * kh in FP64 (the oracle's threshold)
    float t32_in;         // FP32 tier: r2_u < t32_in  -> neighbour
    float t32_out;        // FP32 tier: r2_u > t32_out -> not a neighbour; between -> FP64 tier
    unsigned int neg_t16; // half2 bits of (-T, -T), T = kh^2 / u^2 rounded to FP16
    unsigned int tau16;   // half2 bits of the FP16 "maybe" bound
    float r_scale;        // u / h: R = sqrt(r2_u) * r_scale
    float w_norm;         // m * alpha_d
    float w_self;         // m * W(0, h)
    double r_scale64;     // FP64-CLL mode: 1 / h
    double w_norm64;      // FP64-CLL mode: m * alpha_d
    double w_self64;
    DevStatus *status;
    int spin_limit;       // polls before a look-back wait gives up (0: LOOKBACK_SPIN_LIMIT)
};

// Cell coordinates of a linear cell id (c = (cz ny + cy) nx + cx).
__device__ __forceinline__ void cell_decompose(const GridDev &g, int c, int &cx, int &cy, int &cz) {
    const int row = (int)fastdiv_div((uint32_t)c, g.div_nx);
    cz = (int)fastdiv_div((uint32_t)c, g.div_nxy);
    cx = c - row * g.nk[0];
    cy = row - cz * g.nk[1];
}

// Order-preserving map from a finite double to an unsigned 64-bit key.
__host__ __device__ inline unsigned long long dkey(double x) {
    unsigned long long b;
    memcpy(&b, &x, 8);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double dkey_inv(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// Cell coordinate along one axis: clamp(floor((x - lo) / h_c), 0, nk - 1),
// evaluated in FP64 exactly as written (IEEE division, no contraction).
__device__ __forceinline__ int cell_coord(double x, double lo, double hc, int nk) {
    double t = floor(__ddiv_rn(__dsub_rn(x, lo), hc));
    t = fmax(t, 0.0);
    t = fmin(t, (double)(nk - 1));
    return (int)t;
}

// Cell index and cell-relative coordinate of one axis, in units of
// u = h_c / 2 (Eq. 6 with the cell centre as reference):
//   s = 2 (x - lo) / h_c,  c = clamp(floor(s / 2), 0, nk - 1),
//   a = s - (2c + 1)  (exact: s and 2c + 1 are within one of each other).
// Five FP64 operations and no division.  s carries a relative error of at
// most 2^-52 (x - lo is exact whenever x and lo are within a factor of two),
// i.e. at most 2^-31 u at the 2^20-cell limit, below the 2^-29 u margin that
// the cell size kh (1 + 2^-30) leaves, so every pair closer than kh sits in
// the same or adjacent cells.
__device__ __forceinline__ int rel_axis_s(double s, int nk, double &a) {
    int c = __double2int_rd(s) >> 1;  // floor(floor(s) / 2) = floor(s / 2); saturating conversion
    c = min(max(c, 0), nk - 1);
    a = __dsub_rn(s, (double)(2 * c + 1));
    return c;
}

__device__ __forceinline__ int rel_axis(double x, double lo, double two_over_hc, int nk, double &a) {
    return rel_axis_s(__dmul_rn(__dsub_rn(x, lo), two_over_hc), nk, a);
}

// The same with s = fma(x, 2 / h_c, -lo 2 / h_c) in one rounding (plus the
// roundings of the two constants): |s - exact| <= 2^-53 (|s| + |x| 2/h_c +
// |lo| 2/h_c), at most 2^-33.4 u when |x| and |lo| are at most 2^17 u, which
// the caller checks for the whole grid before choosing this form.
__device__ __forceinline__ int rel_axis_fma(double x, double neg_lo_t, double two_over_hc, int nk, double &a) {
    return rel_axis_s(__fma_rn(x, two_over_hc, neg_lo_t), nk, a);
}

// RN32(v 2^-sh) for |v| < 2^63 and 32 <= sh <= 62 with 32-bit conversions
// only: v is normalised so that its leading one is bit 63, every bit below
// the top 32 is ORed into the lowest of them (sticky), and the 32-bit value
// is converted; the FP32 rounding looks at no more than the 8 bits below its
// 24, so the sticky bit gives the rounding of the full value.  The power-of-
// two scale is exact (the result stays a normal float).
__device__ __forceinline__ float i64_scaled_to_f32_rn(long long v, int sh) {
    const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = u >> 32 ? __clzll(u) : 32;
    const unsigned long long t = u << lz;  // lz = 32 when u fits 32 bits: exact
    const unsigned int hi = (unsigned int)(t >> 32) | ((unsigned int)t != 0u ? 1u : 0u);
    const float r = __uint2float_rn(hi) * __int_as_float((127 + 32 - lz - sh) << 23);
    return v < 0 ? -r : r;
}

// The same cell and the FP32 relative coordinate RN32(s - (2c + 1)) from the
// bits of s, for 2^-10 <= s < 2^21 (false otherwise: the caller takes the
// FP64 route).  With s = m 2^(e - 52) (m the 53-bit significand), floor(s) =
// m >> (52 - e) and s - (2c + 1) = A 2^(e - 52) exactly, A = m - ((2c + 1) <<
// (52 - e)) with |A| < 2^62, rounded to the nearest FP32 (even on ties) and
// scaled exactly, so the result is bit-identical to rel_axis_s followed by
// the FP32 rounding, without FP64 conversions or subtraction (FP64 issue is
// the slow path on this part).
__device__ __forceinline__ bool rel_axis_bits(double s, int nk, int &c, float &f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const int e = (int)(b >> 52) - 1023;  // the sign bit makes e >= 1025 - 1023 for s < 0
    if (e < -10 || e > 20) return false;
    const unsigned long long m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
    const int sh = 52 - e;  // 32 .. 62
    const long long fl = (long long)(m >> sh);
    c = (int)min(fl >> 1, (long long)(nk - 1));
    const long long A = (long long)m - ((long long)(2 * c + 1) << sh);
    f = i64_scaled_to_f32_rn(A, sh);
    return true;
}

// The stored relative coordinates: FP32 rounded once from the FP64 value,
// FP16 rounded from the FP32 value.  The second rounding adds at most 2^-25
// u to the FP16 coordinate's error (2^-12 u for |x_rel| <= 1), far inside the
// FP16 band's margin.  The FP16 record is x, y, z and the particle's cell x
// modulo 2^16 (an unsigned 16-bit integer): the tile search's candidates lie
// within 3 cells of their group's middle cell, so the 16-bit difference
// gives their cell offset exactly with the coordinates' one load.
__device__ __forceinline__ void round_rel_f(float f0, float f1, float f2, int cx, uint2 &q16, float4 &f32) {
    const __half2 xy = __floats2half2_rn(f0, f1);
    const __half z = __float2half_rn(f2);
    q16.x = *reinterpret_cast<const unsigned int *>(&xy);
    q16.y = (unsigned int)*reinterpret_cast<const unsigned short *>(&z) | ((unsigned int)cx << 16);
    f32 = make_float4(f0, f1, f2, 0.f);
}
__device__ __forceinline__ void round_rel(const double a[3], int cx, uint2 &q16, float4 &f32) {
    round_rel_f(__double2float_rn(a[0]), __double2float_rn(a[1]), __double2float_rn(a[2]), cx, q16, f32);
}
// Cell offset (-3 .. 3) of a candidate's FP16 record from cell x `xm`.
__device__ __forceinline__ int rel_cell_offset(uint2 q16, int xm) {
    return (int)(short)(unsigned short)((q16.y >> 16) - (unsigned int)xm);
}

// Row tiles of the single-pass search: runs of at most TILE_ROWS
// consecutive particles of one row of cells that lie within TILE_SPAN
// consecutive cells, cut greedily from the row's start.  cs: the row's nx + 1
// cell starts; p: the first particle of the tile (p < cs[nx]); c: a cell at
// or before the one holding p (advanced in place).  Returns the end of the
// tile.  A row of len particles has at most len / TILE_ROWS + nx / TILE_SPAN
// + 1 tiles.
constexpr int TILE_ROWS = 32;
constexpr int TILE_SPAN = 4;
__host__ __device__ __forceinline__ int row_tile_end(const int *cs, int nx, int p, int &c) {
    while (cs[c + 1] <= p) ++c;
    const int ce = c + TILE_SPAN < nx ? c + TILE_SPAN : nx;
    const int e = p + TILE_ROWS;
    return e < cs[ce] ? e : cs[ce];
}
__host__ __device__ __forceinline__ long long tiles_max(long long n, long long ncell, long long nrow) {
    return n / TILE_ROWS + ncell / TILE_SPAN + nrow + 1;
}

// What another translation unit of the library may see of a grid
// (filled by grid_view in api.cu).
struct GridView {
    GridDev d;
    const int *scell;  // linear cell id of each sorted particle
    int sm_count;
    int precision;
    int order;
    long long n;
    long long nrow;    // rows of cells along x: nk[1] * nk[2]
    int tile_shape;    // tile-search shape and extra staging the grid's own query would use
    int tile_extra;
};
int grid_view(sph_grid_t grid, GridView *v);
int set_error(int code, const char *msg);
cudaError_t reset_counters_async(DevStatus *st, cudaStream_t s);

// ---- launch helpers (implemented in scan.cu / sort.cu) --------------------

// Exclusive scan of int32 counts into int32 (cell starts) or int64 (row
// pointers) with the grand total written at out[n].  tmp needs
// scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(long long n);
constexpr long long SCAN_SMALL_MAX = 1LL << 14;  // scans this short run in one single-block launch
cudaError_t exclusive_scan_i32(const int *in, int *out, long long n, void *tmp, cudaStream_t s);
cudaError_t exclusive_scan_i64(const int *in, long long *out, long long n, void *tmp,
                               cudaStream_t s);
// The same in one launch (decoupled look-back over tiles of the input):
// state holds scan_lb_state_entries(n) entries, all zero at the launch; a
// bounded wait that runs out sets ST_TIMEOUT in *flags.
long long scan_lb_state_entries(long long n);
cudaError_t exclusive_scan_i32_lb(const int *in, int *out, long long n, unsigned long long *state,
                                  unsigned int *flags, int sm_count, cudaStream_t s);
// A grid's cell counters are followed by the look-back state of their scan,
// so that the one memset that clears the counters clears the state too.
inline long long cnt_words(long long ncell) { return (ncell + 1) & ~1LL; }  // keeps the state 8-byte aligned
inline size_t cnt_bytes(long long ncell) {
    return (size_t)cnt_words(ncell) * sizeof(int) + (size_t)scan_lb_state_entries(ncell) * 8;
}
inline unsigned long long *cnt_scan_state(int *cnt, long long ncell) {
    return reinterpret_cast<unsigned long long *>(cnt + cnt_words(ncell));
}

// Sort every segment [seg_start[c], seg_start[c+1]) of keys ascending, for
// c < nseg.  Segments longer than 128 are listed in big_list (capacity nseg)
// with their count in *big_count (device) and sorted by a second pass.
cudaError_t segmented_sort_i32(int *keys, const int *seg_start, long long nseg, int *big_list,
                               unsigned int *big_count, int sm_count, cudaStream_t s);
// Same for int64-delimited segments (CSR rows).
cudaError_t segmented_sort_rows(int *keys, const long long *row_ptr, long long nrows,
                                int *big_list, unsigned int *big_count, int sm_count, cudaStream_t s);

}  // namespace sph
