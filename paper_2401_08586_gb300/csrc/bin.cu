// bin.cu -- binning of particles into background cells (cell link-list,
// Section "SPH method" / Fig. 3b of arXiv 2401.08586) and conversion to the
// normalised cell-relative coordinates of Eq. 6.
//
// Steps (one pass each over the particles):
//   k_bounds   per-axis min/max of the FP64 coordinates (Eq. 5 uses the
//              domain extent), finiteness check;
//   k_hash     cell index c_k = clamp(floor((x_k - lo_k) / h_c), 0, n_k - 1)
//              and the relative coordinate x_rel = 2 (x - x_cc) / h_c with
//              x_cc the cell centre, as the FP64 value rounded to FP32 and
//              then FP16 (input order); linear id (c_z n_y + c_y) n_x + c_x,
//              warp-aggregated histogram whose returned counter value is the
//              particle's provisional slot;
//   (exclusive scan of the histogram -> cell_start)
//   k_scatter  orig_id[cell_start[cell] + slot] = i;
//   k_sort_convert  per cell: orig_id sorted ascending, so the order inside
//              a cell is the input order and the result does not depend on
//              atomic timing; then for every sorted position its rank, cell
//              id and the relative coordinates gathered into cell order
//              (rel16, rel32), or, for the FP64 cell link-list, the FP64
//              coordinate.
// The FP64 work is one fused multiply-add per axis (s = 2 (x - lo) / h_c);
// the floor, the difference and its FP32 rounding are exact integer work on
// the bits of s, since this part's FP64 rate is a small fraction of its
// FP32 and integer rates.
#include "cellcount.cuh"
#include "launch.cuh"
#include "profile.cuh"
#include "sortnet.cuh"
#include "sph_internal.cuh"

namespace sph {

// Order-preserving integer key of an FP64 value (same map as dkey).
__device__ __forceinline__ unsigned long long key_of(unsigned long long b) {
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ void key_minmax(unsigned long long b, unsigned long long &mn, unsigned long long &mx,
                                           bool &bad) {
    bad |= ((b >> 52) & 0x7ffull) == 0x7ffull;
    const unsigned long long k = key_of(b);
    mn = k < mn ? k : mn;
    mx = k > mx ? k : mx;
}

// Per-axis min/max over the order-preserving integer keys of the FP64
// coordinates (no FP64 arithmetic: this part's FP64 rate is a small fraction
// of its integer rate), and the finiteness check on the exponent bits.
// Each thread step reads six consecutive values as three 16-byte loads
// (six is a multiple of both dimensions, so value j of a step is on axis
// j % dim); a misaligned array or the tail goes value by value.
__global__ void k_bounds(const double *__restrict__ xyz, long long total, int dim, DevStatus *st) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const unsigned long long *bits = reinterpret_cast<const unsigned long long *>(xyz);
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    const bool aligned = (reinterpret_cast<uintptr_t>(xyz) & 15u) == 0;
    const long long nchunk = aligned ? total / 6 : 0;
    const ulonglong2 *v2 = reinterpret_cast<const ulonglong2 *>(xyz);
    // two chunks per iteration: six 16-byte loads in flight per thread
    for (long long c = t; c < nchunk; c += 2 * stride) {
        const long long c2 = c + stride < nchunk ? c + stride : c;  // repeats c at the end (min/max are idempotent)
        const ulonglong2 a = __ldg(v2 + 3 * c), b = __ldg(v2 + 3 * c + 1), d = __ldg(v2 + 3 * c + 2);
        const ulonglong2 a2 = __ldg(v2 + 3 * c2), b2 = __ldg(v2 + 3 * c2 + 1), d2 = __ldg(v2 + 3 * c2 + 2);
        const unsigned long long e[12] = {a.x, a.y, b.x, b.y, d.x, d.y, a2.x, a2.y, b2.x, b2.y, d2.x, d2.y};
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            const int ax = j % 3;
            if (dim == 3) key_minmax(e[j], mn[ax], mx[ax], bad);
            else key_minmax(e[j], mn[j & 1], mx[j & 1], bad);
        }
    }
    for (long long f = nchunk * 6 + t; f < total; f += stride) {
        const int ax = (int)(f % dim);
        key_minmax(__ldg(bits + f), mn[ax], mx[ax], bad);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->flags, ST_NONFINITE);
    __shared__ unsigned long long smin[3][32], smax[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < dim; ++a) {
        unsigned long long vmn = mn[a], vmx = mx[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long pm = __shfl_xor_sync(0xffffffffu, vmn, o);
            const unsigned long long px = __shfl_xor_sync(0xffffffffu, vmx, o);
            vmn = pm < vmn ? pm : vmn;
            vmx = px > vmx ? px : vmx;
        }
        if (lane == 0) {
            smin[a][w] = vmn;
            smax[a][w] = vmx;
        }
    }
    __syncthreads();
    if (threadIdx.x < dim) {
        const int a = threadIdx.x;
        unsigned long long vmn = ~0ull, vmx = 0ull;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            vmn = smin[a][k] < vmn ? smin[a][k] : vmn;
            vmx = smax[a][k] > vmx ? smax[a][k] : vmx;
        }
        if (vmn <= vmx) {
            atomicMin(&st->min_key[a], vmn);
            atomicMax(&st->max_key[a], vmx);
        }
    }
}

template <int PREC, int DIM>
__global__ void k_hash(const double *__restrict__ xyz, int n, GridDev g,
                       int *__restrict__ cnt, int *__restrict__ cid, int *__restrict__ slot,
                       uint2 *__restrict__ rel16u, float4 *__restrict__ rel32u, int check_box) {
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        long long i = base + threadIdx.x;
        bool live = i < n;
        int c = -1;
        if (live) {
            int cc[3] = {0, 0, 0};
            double a[3] = {0.0, 0.0, 0.0};
            float fr[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const double x = xyz[i * DIM + k];
                if (g.fma_bin) {
                    const double sk = __fma_rn(x, g.two_over_hc, g.neg_lo_t[k]);
                    // without a box check the FP64 relative coordinate itself is not needed
                    if (!check_box && rel_axis_bits(sk, g.nk[k], cc[k], fr[k])) continue;
                    cc[k] = rel_axis_s(sk, g.nk[k], a[k]);
                } else {
                    cc[k] = rel_axis(x, g.lo[k], g.two_over_hc, g.nk[k], a[k]);
                }
                fr[k] = __double2float_rn(a[k]);
            }
            if (check_box) {
                bool out = false;
                for (int k = 0; k < DIM; ++k) out |= fabs(a[k]) > 1.0 + 1e-6;
                if (out) atomicOr(&g.status->flags, ST_OUT_OF_BOX);
            }
            c = (cc[2] * g.nk[1] + cc[1]) * g.nk[0] + cc[0];
            if (PREC == SPH_PREC_FP16_RCLL) {
                uint2 q;
                float4 f;
                round_rel_f(fr[0], fr[1], fr[2], cc[0], q, f);
                rel16u[i] = q;
                rel32u[i] = f;
            }
        }
        const int sl = cell_run_slot(c, live, cnt);
        if (live) {
            cid[i] = c;
            slot[i] = sl;
        }
    }
}

__global__ void k_scatter(int n, const int *__restrict__ cell_start, const int *__restrict__ cid,
                          const int *__restrict__ slot, int *__restrict__ orig_id) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        orig_id[cell_start[cid[i]] + slot[i]] = (int)i;
}

// Outputs of sorted position s, holding input particle i of cell c (cell x
// cx): its rank and cell, and (RCLL) the relative coordinates computed by
// k_hash, or (FP64 cell link-list) its FP64 coordinates.
struct ConvertOut {
    int *rank, *scell, *scell_x;
    uint2 *rel16;
    float4 *rel32;
    const uint2 *rel16u;
    const float4 *rel32u;
    const double4_32a *rel64u;
    double4_32a *rel64, *x64;
};

template <int PREC>
__device__ __forceinline__ void convert_pos(const GridDev &g, int dim, const ConvertOut &o, int s, int i, int c,
                                            int cx) {
    o.rank[i] = s;
    o.scell[s] = c;
    if (o.scell_x != nullptr) o.scell_x[s] = cx;
    if (PREC == SPH_PREC_FP64_CLL) {
        double x[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < dim; ++k) x[k] = g.xyz[(long long)i * dim + k];
        o.x64[s] = make_double4_32a(x[0], x[1], x[2], 0.0);
    } else {
        o.rel16[s] = o.rel16u[i];
        o.rel32[s] = o.rel32u[i];
        if (o.rel64 != nullptr) o.rel64[s] = o.rel64u[i];
    }
}

constexpr int SORTCV_NT = 128;
// keys per warp sorted in shared memory: 12 KB per block, so that shared
// memory does not limit the blocks per SM below what the threads and
// registers allow (the grid is sized to one wave of resident blocks)
constexpr int SORTCV_SMEM_KEYS = 768;

// Per cell, one warp: sort the cell's input indices (scattered into
// orig_id in arrival order) ascending -- in registers up to 32, in shared
// memory up to 768, longer cells are listed for k_sort_convert_big -- and
// write every sorted position's outputs.
template <int PREC>
__global__ void __launch_bounds__(SORTCV_NT) k_sort_convert(GridDev g, int dim, ConvertOut o, int *__restrict__ keys,
                                                             const int *__restrict__ cell_start, int *big_list,
                                                             unsigned int *big_count) {
    __shared__ int wbuf[SORTCV_NT / 32][SORTCV_SMEM_KEYS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long nw = ((long long)gridDim.x * SORTCV_NT) >> 5;
    for (long long c = ((long long)blockIdx.x * SORTCV_NT + threadIdx.x) >> 5; c < g.ncell; c += nw) {
        const int a = cell_start[c], len = cell_start[c + 1] - a;
        if (len == 0) continue;
        const int cx = (int)c - (int)fastdiv_div((uint32_t)c, g.div_nx) * g.nk[0];
        if (len <= 32) {
            int v = lane < len ? keys[a + lane] : 0;
            if (len > 1) v = net::warp_sort32(v, lane, len);
            if (lane < len) {
                keys[a + lane] = v;
                convert_pos<PREC>(g, dim, o, a + lane, v, (int)c, cx);
            }
        } else if (len <= SORTCV_SMEM_KEYS) {
            int *buf = wbuf[w];
            for (int k = lane; k < len; k += 32) buf[k] = keys[a + k];
            __syncwarp();
            net::bitonic_all_ascending(buf, len, lane, 32, net::WarpSync());
            for (int k = lane; k < len; k += 32) {
                keys[a + k] = buf[k];
                convert_pos<PREC>(g, dim, o, a + k, buf[k], (int)c, cx);
            }
            __syncwarp();
        } else if (lane == 0) {
            big_list[atomicAdd(big_count, 1u)] = (int)c;
        }
    }
}

// Cells longer than SORTCV_SMEM_KEYS: one block each, sorted in place.
template <int PREC>
__global__ void __launch_bounds__(SORTCV_NT) k_sort_convert_big(GridDev g, int dim, ConvertOut o, int *keys,
                                                                 const int *__restrict__ cell_start,
                                                                 const int *big_list,
                                                                 const unsigned int *big_count) {
    const unsigned int nbig = *big_count;
    for (unsigned int b = blockIdx.x; b < nbig; b += gridDim.x) {
        const int c = big_list[b];
        const int a = cell_start[c], len = cell_start[c + 1] - a;
        net::bitonic_all_ascending(keys + a, len, threadIdx.x, SORTCV_NT, net::BlockSync());
        const int cx = c - (int)fastdiv_div((uint32_t)c, g.div_nx) * g.nk[0];
        for (int k = threadIdx.x; k < len; k += SORTCV_NT) convert_pos<PREC>(g, dim, o, a + k, keys[a + k], c, cx);
        __syncthreads();
    }
}

// ---- host launchers ---------------------------------------------------------

// Resident blocks per SM of k_sort_convert<PREC> (its registers, not its
// shared memory, set the limit), found once per process.
template <int PREC>
static int sortcv_per_sm() {
    static const int per_sm = resident_blocks((const void *)k_sort_convert<PREC>, SORTCV_NT);
    return per_sm;
}

static unsigned grid_for(long long n, int nt, int sm_count, int per_sm) {
    long long b = (n + nt - 1) / nt;
    if (b > (long long)sm_count * per_sm) b = (long long)sm_count * per_sm;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_scatter(int n, const int *cell_start, const int *cid, const int *slot, int *orig_id,
                           int sm_count, cudaStream_t s) {
    ProfScope ps(TAG_SCATTER, s);
    note_launch(1);
    k_scatter<<<grid_for(n, 256, sm_count, 16), 256, 0, s>>>(n, cell_start, cid, slot, orig_id);
    return cudaGetLastError();
}

cudaError_t launch_bounds(const double *xyz, long long n, int dim, DevStatus *st, int sm_count,
                          cudaStream_t s) {
    const int nt = 256;
    ProfScope ps(TAG_BOUNDS, s);
    note_launch(1);
    // few blocks, each thread over several chunks: the block reduction and
    // the per-block atomics on the six bounds stay a small part
    k_bounds<<<grid_for((n * dim + 5) / 6, nt, sm_count, 2), nt, 0, s>>>(xyz, n * dim, dim, st);
    return cudaGetLastError();
}

cudaError_t launch_order_convert(const GridDev &g, int n, int dim, int prec, int *cnt, int *cid, int *slot,
                                 int *cell_start, int *orig_id, int *rank, int *scell, uint2 *rel16, float4 *rel32,
                                 const uint2 *rel16u, const float4 *rel32u, const double4_32a *rel64u, double4_32a *rel64,
                                 double4_32a *x64, int *scell_x, void *scan_tmp, int *big_list, unsigned int *big_count,
                                 int sm_count, cudaStream_t s) {
    const int nt = 256;
    const unsigned blocks = grid_for(n, nt, sm_count, 16);
    // cnt is followed by the zeroed look-back state of its scan
    cudaError_t e =
        exclusive_scan_i32_lb(cnt, cell_start, g.ncell, cnt_scan_state(cnt, g.ncell), &g.status->flags, sm_count, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(TAG_SCATTER, s);
        note_launch(1);
        k_scatter<<<blocks, nt, 0, s>>>(n, cell_start, cid, slot, orig_id);
    }
    // per cell: sort its input indices and write the sorted positions' outputs
    e = cudaMemsetAsync(big_count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    ProfScope ps(TAG_SORT, s);
    note_launch(2);
    const bool r = prec == SPH_PREC_FP16_RCLL;
    const ConvertOut o{rank,  scell, scell_x, r ? rel16 : nullptr, r ? rel32 : nullptr, rel16u, rel32u,
                       rel64u, r ? rel64 : nullptr, r ? nullptr : x64};
    // one wave: the warps loop over the cells, so blocks beyond the resident
    // ones would only start once others finish and run their cells alone
    long long sb = (g.ncell * 32 + SORTCV_NT - 1) / SORTCV_NT;
    const long long wave =
        (long long)sm_count * (r ? sortcv_per_sm<SPH_PREC_FP16_RCLL>() : sortcv_per_sm<SPH_PREC_FP64_CLL>());
    if (sb > wave) sb = wave;
    if (sb < 1) sb = 1;
    if (r) {
        k_sort_convert<SPH_PREC_FP16_RCLL><<<(unsigned)sb, SORTCV_NT, 0, s>>>(g, dim, o, orig_id, cell_start,
                                                                              big_list, big_count);
        k_sort_convert_big<SPH_PREC_FP16_RCLL><<<sm_count, SORTCV_NT, 0, s>>>(g, dim, o, orig_id, cell_start,
                                                                              big_list, big_count);
    } else {
        k_sort_convert<SPH_PREC_FP64_CLL><<<(unsigned)sb, SORTCV_NT, 0, s>>>(g, dim, o, orig_id, cell_start,
                                                                             big_list, big_count);
        k_sort_convert_big<SPH_PREC_FP64_CLL><<<sm_count, SORTCV_NT, 0, s>>>(g, dim, o, orig_id, cell_start,
                                                                             big_list, big_count);
    }
    return cudaGetLastError();
}

cudaError_t launch_hash_scatter_convert(const GridDev &g, const double *xyz, int n, int dim, int prec,
                                        int *cnt, int *cid, int *slot, int *cell_start, int *orig_id,
                                        int *rank, int *scell, uint2 *rel16, float4 *rel32, uint2 *rel16u,
                                        float4 *rel32u, double4_32a *x64, int *scell_x, void *scan_tmp, int *big_list,
                                        unsigned int *big_count, int check_box, int sm_count, cudaStream_t s) {
    const int nt = 256;
    const unsigned blocks = grid_for(n, nt, sm_count, 16);
    cudaError_t e = cudaMemsetAsync(cnt, 0, cnt_bytes(g.ncell), s);  // counters and their scan state
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(TAG_HASH, s);
        note_launch(1);
        const bool r = prec == SPH_PREC_FP16_RCLL;
        auto kern = r ? (dim == 2 ? k_hash<SPH_PREC_FP16_RCLL, 2> : k_hash<SPH_PREC_FP16_RCLL, 3>)
                      : (dim == 2 ? k_hash<SPH_PREC_FP64_CLL, 2> : k_hash<SPH_PREC_FP64_CLL, 3>);
        kern<<<blocks, nt, 0, s>>>(xyz, n, g, cnt, cid, slot, r ? rel16u : nullptr, r ? rel32u : nullptr, check_box);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // a fresh binning leaves the FP64 relative coordinates (kept for time
    // steps) to be derived again on the next step
    return launch_order_convert(g, n, dim, prec, cnt, cid, slot, cell_start, orig_id, rank, scell, rel16, rel32,
                                rel16u, rel32u, nullptr, nullptr, x64, scell_x, scan_tmp, big_list, big_count,
                                sm_count, s);
}

}  // namespace sph
