// nnps_tile64.cu -- the FP64 cell link-list search (SPH_PREC_FP64_CLL) on the
// single-pass row-tile structure of the FP16-RCLL search: the same tile list,
// candidate rows of cells, bounding-box cull, look-back CSR offsets and
// output, with the neighbour test and the density in FP64 on the cell-ordered
// caller coordinates (the link-list search of the paper's FP64 runs), so that
// a comparison with the FP16-RCLL search measures precision, not kernel
// design.
//
// Per tile (at most 32 cell-sorted particles of one row of cells within 4
// cells; lane l owns home particle p0 + l, one CSR row):
//   * candidates: the 3^d rows of cells around the tile's row, x-range widened
//     by one cell (same and adjacent cells, Fig. 3b); cull: a candidate whose
//     squared distance to the bounding box of the tile's particles is not
//     below kh^2 (1 + 2^-40) -- the margin covers the FP64 rounding of the box
//     test -- is nobody's neighbour;
//   * windows of kept candidates staged in shared memory (x, y, z, index);
//   * test: r^2 = (dx0 dx0 + dx1 dx1) + dx2 dx2 evaluated exactly as the
//     definition writes it (no contraction); neighbour iff r^2 < kh^2 and
//     j != i: one bit per pair, the decision of the FP64 definition itself;
//   * each lane walks its bits: density W(r / h) of Eq. 3 in FP64, with the
//     kernel written without branches as 6 P(R) = (2 - R)^3 - 4 max(1 - R, 0)^3
//     (the two pieces of Eq. 3 in one expression) and r = r^2 rsqrt(r^2).
// The tile's row counts give its total; the CSR offset comes from the
// decoupled look-back over earlier tiles; each lane writes its row pointer,
// its density and its row from its bits.  A tile whose kept list needs more
// than one pass runs the steps again, emitting in the walk.
#include "launch.cuh"
#include "lookback.cuh"
#include "nnps_common.cuh"
#include "profile.cuh"
#include "tile_rows.cuh"

namespace sph {

using namespace nn;
using namespace lb;

namespace {

constexpr int CMAX64 = 1024;        // kept candidates per pass
constexpr int WIN64 = 128;          // candidates staged per window
constexpr int NW64 = CMAX64 / 32;   // bitmask words per lane and pass
constexpr int WPB64 = 2;            // warps per CTA, each on its own tiles
constexpr int CTA_PER_SM64 = 9;     // 18 resident warps per SM
constexpr double CULL_MARGIN64 = 0x1p-40;

struct Smem64 {
    unsigned int S[32][NW64 + 1];  // odd row stride: a column's words in 32 banks
    int jall[CMAX64];              // kept candidates: sorted index
    int4 rt[9];
    int rcum[10], pad[2];
    double cx[WIN64], cy[WIN64], cz[WIN64];
    int cj[WIN64];
};

__device__ __forceinline__ double warp_min64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The definition's squared distance (no contraction) from a home particle to
// staged candidate c.
template <int DIM>
__device__ __forceinline__ double r2_staged(const Smem64 &S, const double (&xi)[3], int c) {
    const double d0 = __dsub_rn(xi[0], S.cx[c]);
    const double d1 = __dsub_rn(xi[1], S.cy[c]);
    double r2 = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
    if (DIM == 3) {
        const double d2 = __dsub_rn(xi[2], S.cz[c]);
        r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
    }
    return r2;
}

// Cull and compact the tile's candidates from flat index cur (rows in order,
// each row's candidates ascending) until they run out or the kept list is
// full.  Returns the number kept; advances cur.
template <int DIM>
__device__ __forceinline__ int cull64(Smem64 &S, const GridDev &g, const double (&lo)[3], const double (&hi)[3],
                                      double cullT, int &cur) {
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    const int lane = threadIdx.x & 31;
    int rc[NROWS];
#pragma unroll
    for (int r = 0; r < NROWS; ++r) rc[r] = S.rcum[r + 1];
    const int total = rc[NROWS - 1];
    int kept = 0;
    while (cur < total && kept + 32 <= CMAX64) {
        const int k = cur + lane;
        bool keep = false;
        int j = 0;
        if (k < total) {
            j = k + S.rt[tile_row_of<DIM>(k, rc)].x;
            const double *xj = g.x64 + 4ll * j;
            double d2 = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const double x = xj[a];
                const double e = fmax(fmax(__dsub_rn(lo[a], x), __dsub_rn(x, hi[a])), 0.0);
                d2 = __fma_rn(e, e, d2);
            }
            keep = d2 < cullT;
        }
        const unsigned int m = __ballot_sync(0xffffffffu, keep);
        if (keep) S.jall[kept + __popc(m & ((1u << lane) - 1u))] = j;
        kept += __popc(m);
        cur += 32;
    }
    __syncwarp();
    return kept;
}

// Stage kept candidates [w0, w0 + wc) (slots past wc: far away, index -1).
__device__ __forceinline__ void stage64(Smem64 &S, const GridDev &g, int w0, int wc) {
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < WIN64; k += 32) {
        if (k < wc) {
            const int j = S.jall[w0 + k];
            const double *xj = g.x64 + 4ll * j;
            S.cx[k] = xj[0];
            S.cy[k] = xj[1];
            S.cz[k] = xj[2];
            S.cj[k] = j;
        } else {
            S.cx[k] = S.cy[k] = S.cz[k] = 1e300;
            S.cj[k] = -1;
        }
    }
    __syncwarp();
}

// 6 P(R) of Eq. 3 for 0 <= R < 2: (2 - R)^3 - 4 (1 - R)^3 on [0, 1) equals
// 4 - 6 R^2 + 3 R^3 = 6 (2/3 - R^2 + R^3 / 2), and (2 - R)^3 alone on [1, 2).
__device__ __forceinline__ double six_p64(double R) {
    const double t = 2.0 - R, s = fmax(1.0 - R, 0.0);
    return __fma_rn(-4.0 * s, s * s, t * t * t);
}

// r = sqrt(r^2) for the density (the neighbour decision never uses it).
__device__ __forceinline__ double dist64(double r2) { return r2 > 0.0 ? r2 * rsqrt(r2) : 0.0; }

enum { P64_COUNT = 0, P64_EMIT = 1 };

// One pass of kept candidates: windows staged, tested (bits of kept slot k
// into word k / 32 of the lane's row) and walked: PASS count adds the
// neighbours and their density, PASS emit writes them to col[rp + cnt ...]
// in order.
template <int DIM, int PASS>
__device__ __forceinline__ void run_pass64(Smem64 &S, const GridDev &g, const double (&xi)[3], int i, bool mine,
                                           int kept, int &cnt, double &acc, bool dens, int *col, long long rp) {
    const int lane = threadIdx.x & 31;
    const double kh2 = g.kh2;
    for (int w0 = 0; w0 < kept; w0 += WIN64) {
        const int wc = min(WIN64, kept - w0);
        stage64(S, g, w0, wc);
        const int nwin = (wc + 31) >> 5;
        for (int q = 0; q < nwin; ++q) {
            unsigned int word = 0u;
#pragma unroll 4
            for (int b = 0; b < 32; ++b) {
                const int c = q * 32 + b;
                const bool nb = r2_staged<DIM>(S, xi, c) < kh2 && S.cj[c] != i;
                word |= (nb ? 1u : 0u) << b;
            }
            word = mine ? word : 0u;
            S.S[lane][(w0 >> 5) + q] = word;
        }
        // the lane's bits of this window, in candidate order
        for (int q = 0; q < nwin; ++q) {
            unsigned int w = S.S[lane][(w0 >> 5) + q];
            while (__any_sync(0xffffffffu, w != 0u)) {
                if (w != 0u) {
                    const int c = q * 32 + __ffs(w) - 1;
                    w &= w - 1u;
                    if (PASS == P64_EMIT) {
                        col[rp + cnt] = S.cj[c];
                        ++cnt;
                    } else {
                        ++cnt;
                        if (dens) acc += six_p64(dist64(r2_staged<DIM>(S, xi, c)) * g.r_scale64);
                    }
                }
            }
        }
        __syncwarp();
    }
}

template <int DIM>
__global__ void __launch_bounds__(32 * WPB64, CTA_PER_SM64)
    k_nnps_tile64(GridDev g, const int4 *__restrict__ tiles, const long long *__restrict__ ntiles_dev,
                  long long *__restrict__ row_ptr, int *__restrict__ col, long long cap, float *__restrict__ rho,
                  unsigned long long *__restrict__ tstate) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem64 &S = *reinterpret_cast<Smem64 *>(smraw + (threadIdx.x >> 5) * sizeof(Smem64));
    const int lane = threadIdx.x & 31;
    const long long ntiles = *ntiles_dev;
    const double cullT = g.kh2 * (1.0 + CULL_MARGIN64);
    const bool dens = rho != nullptr;
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    while (true) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&g.status->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int4 td = tiles[t];
        const int p0 = td.x, nh = td.y, row = td.z;
        const int cy = row % g.nk[1], cz = row / g.nk[1];
        const bool mine = lane < nh;
        const int i = p0 + lane;
        double xi[3] = {0.0, 0.0, 0.0};
        int cxi = 0;
        if (mine) {
            for (int a = 0; a < DIM; ++a) xi[a] = g.x64[4ll * i + a];
            cxi = g.scell_x[i];
        }
        // the tile's cells (at most TILE_SPAN consecutive ones) and the bounding
        // box of its particles
        const int xa = __shfl_sync(0xffffffffu, cxi, 0);
        const int xb = __shfl_sync(0xffffffffu, cxi, nh - 1);
        double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            lo[a] = warp_min64(mine ? xi[a] : INFINITY);
            hi[a] = warp_max64(mine ? xi[a] : -INFINITY);
        }
        tile_candidate_rows<DIM>(S.rt, S.rcum, g, cy, cz, max(xa - 1, 0), min(xb + 1, g.nk[0] - 1));
        const int total = S.rcum[NROWS];
        // ---- count pass --------------------------------------------------------
        int cnt = 0, cur = 0, passes = 0, kept = 0;
        double acc = 0.0;
        do {
            kept = cull64<DIM>(S, g, lo, hi, cullT, cur);
            run_pass64<DIM, P64_COUNT>(S, g, xi, i, mine, kept, cnt, acc, dens, nullptr, 0);
            ++passes;
        } while (cur < total);
        // ---- CSR offset of the tile --------------------------------------------
        int inc = mine ? cnt : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int agg = __shfl_sync(0xffffffffu, inc, 31);
        const long long rstart = inc - (mine ? cnt : 0);
        look_back_publish(tstate, t, agg);
        const long long pre =
            look_back_resolve(tstate, t, agg, &g.status->flags, g.spin_limit > 0 ? g.spin_limit : LOOKBACK_SPIN_LIMIT);
        const bool wc = col != nullptr && pre + agg <= cap;
        if (col != nullptr && !wc && lane == 0) atomicOr(&g.status->flags, ST_CAPACITY);
        if (mine) {
            row_ptr[i] = pre + rstart;
            if (dens) rho[i] = (float)(g.w_self64 + g.w_norm64 * (acc * (1.0 / 6.0)));
        }
        if (t == ntiles - 1 && lane == 0) row_ptr[g.n] = pre + agg;
        if (!wc) continue;
        if (passes == 1) {
            // every bit of the tile is still in S: the lane's row in order
            long long pos = pre + rstart;
            for (int q = 0; q < (kept + 31) >> 5; ++q) {
                unsigned int w = S.S[lane][q];
                while (w != 0u) {
                    col[pos++] = S.jall[q * 32 + __ffs(w) - 1];
                    w &= w - 1u;
                }
            }
            __syncwarp();
        } else {
            int ecnt = 0;
            double dummy = 0.0;
            cur = 0;
            do {
                kept = cull64<DIM>(S, g, lo, hi, cullT, cur);
                run_pass64<DIM, P64_EMIT>(S, g, xi, i, mine, kept, ecnt, dummy, false, col, pre + rstart);
            } while (cur < total);
        }
    }
}

}  // namespace

cudaError_t launch_nnps_tile64(const GridDev &g, const int4 *tiles, const long long *ntiles_dev,
                               long long ntiles_max, long long *row_ptr, int *col, long long cap, float *rho,
                               unsigned long long *tstate, int sm_count, cudaStream_t s) {
    const size_t sb = sizeof(Smem64) * WPB64;
    auto kern = g.dim == 2 ? k_nnps_tile64<2> : k_nnps_tile64<3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPB64, sb);
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > (ntiles_max + WPB64 - 1) / WPB64) blocks = (ntiles_max + WPB64 - 1) / WPB64;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_FUSED, s);
    note_launch(1);
    kern<<<(unsigned)blocks, 32 * WPB64, sb, s>>>(g, tiles, ntiles_dev, row_ptr, col, cap, rho, tstate);
    return cudaGetLastError();
}

}  // namespace sph
