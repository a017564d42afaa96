// scan_sort.cu -- device-wide exclusive scan and segmented sort used by the
// counting sort of the binning step and by the CSR assembly.
//
// Scan: one launch of one block up to SCAN_SMALL_MAX items, else three
// launches (tile sums, scan of tile sums, tile scan + offset), or, given a
// zeroed state array, one launch with a decoupled look-back over tiles.
// Sort: every segment is sorted ascending with a bitonic network written so
// that all comparators put the minimum at the lower index (the first step of
// each merge compares i with i ^ (k - 1)).  With that form, positions past the
// segment end behave as +infinity and are simply skipped, so no padding is
// stored.  Segments of <= 32 keys are sorted in registers by one warp,
// <= 1024 keys by one warp in shared memory, larger ones by a whole block.
#include "lookback.cuh"
#include "profile.cuh"
#include "sortnet.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

using namespace net;

constexpr int SCAN_NT = 256;
constexpr int SCAN_ITEMS = 4;  // tiles of 1024 items: more blocks in flight for grids of ~10^4-10^5 cells
constexpr int SCAN_TILE = SCAN_NT * SCAN_ITEMS;

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan across a 256-thread block; returns the exclusive prefix of
// v and writes the block total to *total (all threads).
__device__ long long block_excl_scan_256(long long v, long long *total) {
    __shared__ long long wsum[SCAN_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = warp_incl_scan(v, lane);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long s = lane < SCAN_NT / 32 ? wsum[lane] : 0;
        s = warp_incl_scan(s, lane);
        if (lane < SCAN_NT / 32) wsum[lane] = s;
    }
    __syncthreads();
    long long before = w > 0 ? wsum[w - 1] : 0;
    *total = wsum[SCAN_NT / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void __launch_bounds__(SCAN_NT) k_tile_sums(const int *in, long long n, long long *sums) {
    long long base = (long long)blockIdx.x * SCAN_TILE;
    long long s = 0;
#pragma unroll 4
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long idx = base + (long long)k * SCAN_NT + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    long long tot;
    block_excl_scan_256(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: in-place exclusive scan of the tile sums; grand total to sums[ntile].
__global__ void __launch_bounds__(SCAN_NT) k_scan_sums(long long *sums, long long ntile) {
    long long carry = 0;
    for (long long base = 0; base < ntile; base += SCAN_NT) {
        long long idx = base + threadIdx.x;
        long long v = idx < ntile ? sums[idx] : 0;
        long long tot;
        long long ex = block_excl_scan_256(v, &tot);
        if (idx < ntile) sums[idx] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[ntile] = carry;
}

template <typename OutT>
__global__ void __launch_bounds__(SCAN_NT) k_tile_scan(const int *in, OutT *out, long long n,
                                                        const long long *sums, long long ntile) {
    __shared__ long long buf[SCAN_TILE];
    long long base = (long long)blockIdx.x * SCAN_TILE;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long idx = base + (long long)k * SCAN_NT + threadIdx.x;
        buf[k * SCAN_NT + threadIdx.x] = idx < n ? in[idx] : 0;
    }
    __syncthreads();
    long long own[SCAN_ITEMS];
    long long s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        own[k] = buf[threadIdx.x * SCAN_ITEMS + k];
        s += own[k];
    }
    long long tot;
    long long ex = block_excl_scan_256(s, &tot) + sums[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        buf[threadIdx.x * SCAN_ITEMS + k] = ex;
        ex += own[k];
    }
    __syncthreads();
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long idx = base + (long long)k * SCAN_NT + threadIdx.x;
        if (idx < n) out[idx] = (OutT)buf[k * SCAN_NT + threadIdx.x];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (OutT)sums[ntile];
}

constexpr int SMALL_NT = 1024;

// Exclusive scan across a 1024-thread block (as block_excl_scan_256).
__device__ long long block_excl_scan_1024(long long v, long long *total) {
    __shared__ long long wsum[SMALL_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = warp_incl_scan(v, lane);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long t = wsum[lane];
        t = warp_incl_scan(t, lane);
        wsum[lane] = t;
    }
    __syncthreads();
    long long before = w > 0 ? wsum[w - 1] : 0;
    *total = wsum[SMALL_NT / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

// One block, one launch: each thread scans a contiguous run of the input.
template <typename OutT>
__global__ void __launch_bounds__(SMALL_NT) k_scan_small(const int *__restrict__ in, OutT *__restrict__ out,
                                                          long long n) {
    const long long per = (n + SMALL_NT - 1) / SMALL_NT;
    const long long a = (long long)threadIdx.x * per, b = a + per < n ? a + per : n;
    long long sum = 0;
    for (long long i = a; i < b; ++i) sum += in[i];
    long long total;
    long long ex = block_excl_scan_1024(sum, &total);
    for (long long i = a; i < b; ++i) {
        out[i] = (OutT)ex;
        ex += in[i];
    }
    if (threadIdx.x == 0) out[n] = (OutT)total;
}

// Single-launch scan: blocks take tiles of SCAN_TILE items in ticket order
// (state[ntile] is the ticket), scan them in shared memory and add the
// prefix of all earlier tiles found by a decoupled look-back (state[tile]).
template <typename OutT>
__global__ void __launch_bounds__(SCAN_NT) k_scan_lb(const int *__restrict__ in, OutT *__restrict__ out, long long n,
                                                      unsigned long long *__restrict__ state, long long ntile,
                                                      unsigned int *flags) {
    __shared__ long long buf[SCAN_TILE];
    __shared__ long long tile_pre;
    __shared__ unsigned long long tile_id;
    while (true) {
        __syncthreads();  // the previous tile is done with the shared buffers
        if (threadIdx.x == 0) tile_id = atomicAdd(&state[ntile], 1ull);
        __syncthreads();
        const long long t = (long long)tile_id;
        if (t >= ntile) break;
        const long long base = t * SCAN_TILE;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const long long idx = base + (long long)k * SCAN_NT + threadIdx.x;
            buf[k * SCAN_NT + threadIdx.x] = idx < n ? in[idx] : 0;
        }
        __syncthreads();
        long long own[SCAN_ITEMS];
        long long sum = 0;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            own[k] = buf[threadIdx.x * SCAN_ITEMS + k];
            sum += own[k];
        }
        long long tot;
        long long ex = block_excl_scan_256(sum, &tot);
        if (threadIdx.x < 32) {
            lb::look_back_publish(state, t, tot);
            const long long pre = lb::look_back_resolve(state, t, tot, flags);
            if (threadIdx.x == 0) tile_pre = pre;
        }
        __syncthreads();
        ex += tile_pre;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            buf[threadIdx.x * SCAN_ITEMS + k] = ex;
            ex += own[k];
        }
        __syncthreads();
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const long long idx = base + (long long)k * SCAN_NT + threadIdx.x;
            if (idx < n) out[idx] = (OutT)buf[k * SCAN_NT + threadIdx.x];
        }
        if (t == ntile - 1 && threadIdx.x == 0) out[n] = (OutT)(tile_pre + tot);
    }
}

template <typename OutT>
cudaError_t scan_impl(const int *in, OutT *out, long long n, void *tmp, cudaStream_t s) {
    if (n <= SCAN_SMALL_MAX) {
        ProfScope ps(TAG_SCAN, s);
        note_launch(1);
        k_scan_small<OutT><<<1, SMALL_NT, 0, s>>>(in, out, n);
        return cudaGetLastError();
    }
    long long ntile = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntile == 0) ntile = 1;
    long long *sums = (long long *)tmp;
    ProfScope ps(TAG_SCAN, s);
    note_launch(3);
    k_tile_sums<<<(unsigned)ntile, SCAN_NT, 0, s>>>(in, n, sums);
    k_scan_sums<<<1, SCAN_NT, 0, s>>>(sums, ntile);
    k_tile_scan<OutT><<<(unsigned)ntile, SCAN_NT, 0, s>>>(in, out, n, sums, ntile);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sorting

__device__ __forceinline__ int ceil_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

constexpr int SORT_NT = 128;
constexpr int WARP_SMEM_KEYS = 1024;

// Segments of up to 128 keys, one warp each, in registers (1, 2 or 4 keys
// per lane); longer segments are listed in big_list for k_seg_sort_big.  The
// longer paths live in their own kernel so that their registers do not limit
// the residency of this one, which sorts nearly all segments.
template <typename IdxT>
__global__ void __launch_bounds__(SORT_NT) k_seg_sort_small(int *keys, const IdxT *seg, long long nseg,
                                                             int *big_list, unsigned int *big_count) {
    const int lane = threadIdx.x & 31;
    long long gw = ((long long)blockIdx.x * SORT_NT + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * SORT_NT) >> 5;
    for (long long c = gw; c < nseg; c += nw) {
        long long a = seg[c], b = seg[c + 1];
        long long len = b - a;
        if (len <= 1) continue;
        if (len <= 32) {
            int v = lane < len ? keys[a + lane] : 0;
            v = warp_sort32(v, lane, (int)len);
            if (lane < len) keys[a + lane] = v;
        } else if (len <= 64) {
            int v[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) v[t] = t * 32 + lane < len ? keys[a + t * 32 + lane] : 0x7fffffff;
            warp_sort_reg<2>(v, lane);
#pragma unroll
            for (int t = 0; t < 2; ++t)
                if (t * 32 + lane < len) keys[a + t * 32 + lane] = v[t];
        } else if (len <= 128) {
            int v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) v[t] = t * 32 + lane < len ? keys[a + t * 32 + lane] : 0x7fffffff;
            warp_sort_reg<4>(v, lane);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t * 32 + lane < len) keys[a + t * 32 + lane] = v[t];
        } else if (lane == 0) {
            unsigned int slot = atomicAdd(big_count, 1u);
            big_list[slot] = (int)c;
        }
    }
}

// The listed segments (longer than 128 keys), one warp each: up to 256 keys
// in registers (8 per lane), up to WARP_SMEM_KEYS in shared memory, longer
// ones in place in global memory (the same network, the warp's steps ordered
// by __syncwarp).
template <typename IdxT>
__global__ void __launch_bounds__(SORT_NT) k_seg_sort_big(int *keys, const IdxT *seg, const int *big_list,
                                                           const unsigned int *big_count) {
    __shared__ int wbuf[SORT_NT / 32][WARP_SMEM_KEYS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long nbig = *big_count;
    const long long gw = ((long long)blockIdx.x * SORT_NT + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * SORT_NT) >> 5;
    for (long long bi = gw; bi < nbig; bi += nw) {
        const long long c = big_list[bi];
        const long long a = seg[c], len = seg[c + 1] - a;
        if (len <= 256) {
            int v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = t * 32 + lane < len ? keys[a + t * 32 + lane] : 0x7fffffff;
            warp_sort_reg<8>(v, lane);
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t * 32 + lane < len) keys[a + t * 32 + lane] = v[t];
        } else if (len <= WARP_SMEM_KEYS) {
            int *buf = wbuf[w];
            for (long long i = lane; i < len; i += 32) buf[i] = keys[a + i];
            __syncwarp();
            bitonic_all_ascending(buf, len, lane, 32, WarpSync());
            for (long long i = lane; i < len; i += 32) keys[a + i] = buf[i];
            __syncwarp();
        } else {
            bitonic_all_ascending(keys + a, len, lane, 32, WarpSync());
        }
    }
}

template <typename IdxT>
cudaError_t seg_sort_impl(int *keys, const IdxT *seg, long long nseg, int *big_list,
                          unsigned int *big_count, int sm_count, cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    ProfScope ps(TAG_SORT, s);
    note_launch(2);
    const cudaError_t e = cudaMemsetAsync(big_count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    long long blocks = (nseg * 32 + SORT_NT - 1) / SORT_NT;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    k_seg_sort_small<IdxT><<<(unsigned)blocks, SORT_NT, 0, s>>>(keys, seg, nseg, big_list, big_count);
    k_seg_sort_big<IdxT><<<(unsigned)sm_count * 4, SORT_NT, 0, s>>>(keys, seg, big_list, big_count);
    return cudaGetLastError();
}

}  // namespace

size_t scan_tmp_bytes(long long n) {
    long long ntile = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntile == 0) ntile = 1;
    return (size_t)(ntile + 1) * sizeof(long long);
}

long long scan_lb_state_entries(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

cudaError_t exclusive_scan_i32_lb(const int *in, int *out, long long n, unsigned long long *state,
                                  unsigned int *flags, int sm_count, cudaStream_t s) {
    const long long ntile = scan_lb_state_entries(n) - 1;
    if (ntile <= 1) return exclusive_scan_i32(in, out, n, nullptr, s);  // one block: no look-back needed
    long long blocks = ntile < (long long)sm_count * 4 ? ntile : (long long)sm_count * 4;
    ProfScope ps(TAG_SCAN, s);
    note_launch(1);
    k_scan_lb<int><<<(unsigned)blocks, SCAN_NT, 0, s>>>(in, out, n, state, ntile, flags);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_i32(const int *in, int *out, long long n, void *tmp, cudaStream_t s) {
    return scan_impl<int>(in, out, n, tmp, s);
}

cudaError_t exclusive_scan_i64(const int *in, long long *out, long long n, void *tmp,
                               cudaStream_t s) {
    return scan_impl<long long>(in, out, n, tmp, s);
}

cudaError_t segmented_sort_i32(int *keys, const int *seg_start, long long nseg, int *big_list,
                               unsigned int *big_count, int sm_count, cudaStream_t s) {
    return seg_sort_impl<int>(keys, seg_start, nseg, big_list, big_count, sm_count, s);
}

cudaError_t segmented_sort_rows(int *keys, const long long *row_ptr, long long nrows,
                                int *big_list, unsigned int *big_count, int sm_count, cudaStream_t s) {
    return seg_sort_impl<long long>(keys, row_ptr, nrows, big_list, big_count, sm_count, s);
}

}  // namespace sph
