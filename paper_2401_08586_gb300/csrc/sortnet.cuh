// sortnet.cuh -- sorting networks for short segments of int keys: one warp
// in registers (up to 32 keys) and a compare-exchange network over any
// memory run by cooperating threads.  Every comparator puts the minimum at
// the lower index (the first step of each merge compares i with i ^ (k - 1)),
// so positions past the segment end behave as +infinity and are skipped.
#pragma once

namespace sph {
namespace net {

// One warp sorts keys[0, len) (len <= 32) held one per lane.
__device__ __forceinline__ int warp_sort32(int v, int lane, int len) {
    const int INF = 0x7fffffff;
    if (lane >= len) v = INF;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            int partner = (j == (k >> 1)) ? (lane ^ (k - 1)) : (lane ^ j);
            int o = __shfl_sync(0xffffffffu, v, partner);
            bool lower = lane < partner;
            v = lower ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// One warp sorts keys[0, len) (len <= 32 R) held in registers: v[t] is
// position t * 32 + lane.  The same bitonic network as warp_sort32 over 32 R
// positions; a comparator's partner is position p ^ m, i.e. register t ^ (m >>
// 5) of lane lane ^ (m & 31) (a shuffle when m & 31 != 0, else a register of
// the same lane).  Positions past len hold +infinity.
template <int R>
__device__ __forceinline__ void warp_sort_reg(int (&v)[R], int lane) {
    static_assert(R == 2 || R == 4 || R == 8, "32, 64, 128 or 256 keys");
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int m = (j == (k >> 1)) ? (k - 1) : j;
            const int ml = m & 31, mt = m >> 5;
            int o[R];
#pragma unroll
            for (int t = 0; t < R; ++t) o[t] = ml ? __shfl_xor_sync(0xffffffffu, v[t ^ mt], ml) : v[t ^ mt];
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int p = t * 32 + lane, q = p ^ m;
                v[t] = p < q ? min(v[t], o[t]) : max(v[t], o[t]);
            }
        }
    }
}

// Compare-exchange network over keys[0, len) in any memory, executed by
// `nthr` cooperating threads with index `t`; `sync` orders the steps.
template <typename Sync>
__device__ void bitonic_all_ascending(int *keys, long long len, int t, int nthr, Sync sync) {
    long long P = 1;
    while (P < len) P <<= 1;
    for (long long k = 2; k <= P; k <<= 1) {
        for (long long j = k >> 1; j > 0; j >>= 1) {
            for (long long i = t; i < P; i += nthr) {
                long long partner = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
                if (partner > i && partner < len) {
                    int a = keys[i], b = keys[partner];
                    if (a > b) {
                        keys[i] = b;
                        keys[partner] = a;
                    }
                }
            }
            sync();
        }
    }
}

struct WarpSync {
    __device__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

}  // namespace net
}  // namespace sph
