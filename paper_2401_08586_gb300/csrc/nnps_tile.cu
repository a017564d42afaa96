// nnps_tile.cu -- single-pass FP16-RCLL neighbour search + SPH density with
// one warp per row tile (the production search for cell-order queries).
//
// Tiles: the cell-sorted particles of every x-row of cells (fixed y, z) are
// cut into runs of at most 32; a warp takes tiles in order from an atomic
// ticket and lane l owns home particle p0 + l, i.e. one CSR row.
//
// Per home group (the tile's particles whose cells span at most SPANMAX
// consecutive x-cells; normally the whole tile):
//   candidates = the 3^d x-rows of cells around the group's cells (each a
//   contiguous range of the sorted arrays), cell x-range widened by one.
//   Coordinates are cell-relative (Eq. 6) re-expressed in the frame of the
//   group's middle cell: X = x_rel + 2 (c_x - x_mid), Y = y_rel + 2 dy,
//   Z = z_rel + 2 dz (units of u = h_c / 2), so a pair's difference is the
//   Eq. 7 distance (scale h_c / 2).
//   1. stage a window of candidates in shared memory, two per half2 word;
//   2. FP16 test (all lanes, candidates broadcast): e = ((dx^2 - T) + dy^2)
//      + dz^2 with half2 FMAs; e < tau16 marks a "maybe" pair in the lane's
//      row bitmask (bit order = candidate order = ascending column);
//   3. each lane walks its own maybe bits: FP32 distance from the FP32
//      relative coordinates, decision with the FP32 band (FP64 definition
//      inside it), neighbour count and density sum (Eq. 3) in CSR order;
//      rejected bits are cleared.
// Then the tile's neighbour total is published and the CSR offset of the tile
// found by a decoupled look-back over earlier tiles; each lane writes its row
// pointer and density, emits its row into a shared staging buffer (candidate
// slots), and the warp copies the staged columns out coalesced.
// Tiles with several home groups or more than CMAX candidates run the same
// steps twice (count, then emit straight to their rows after the look-back).
#include "nnps_common.cuh"

namespace sph {

using namespace nn;

namespace {

constexpr int TW = 32;        // rows per tile
constexpr int SPANMAX = 4;    // home cells per group along x (keeps |X| < 8)
constexpr int WIN = 256;      // candidates per staging window
constexpr int CMAX = 1024;    // candidates per super-window (bitmask length)
constexpr int NWORD = CMAX / 32;

constexpr unsigned long long ST_AGG = 1ull << 62;
constexpr unsigned long long ST_INCL = 2ull << 62;
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;
constexpr int LOOKBACK_SPIN_LIMIT = 1 << 20;

struct TileSmem {
    uint4 pw[WIN / 2];          // FP16 pairs: word (g*16 + b) = candidates 32g + b (lo), 32g + 16 + b (hi)
    float4 f32[WIN];            // FP32 frame coordinates, candidate index j in .w
    unsigned int S[TW][NWORD + 1];
    int rstart[9], roff[10], rdy[9], rdz[9], rcb[9][8];
    int C;
    int nbm1;  // internal cell boundaries per candidate row + 1
};

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Publish this tile's total and return the sum over all earlier tiles.
__device__ __forceinline__ long long look_back(unsigned long long *tstate, long long t, long long agg,
                                               unsigned int *flags) {
    const int lane = threadIdx.x & 31;
    if (t == 0) {
        if (lane == 0) atomicExch(&tstate[0], ST_INCL | (unsigned long long)agg);
        return 0;
    }
    if (lane == 0) atomicExch(&tstate[t], ST_AGG | (unsigned long long)agg);
    long long excl = 0, j = t - 1;
    int spins = 0, backoff = 32;
    bool timed_out = false;
    while (true) {
        const long long idx = j - lane;
        const unsigned long long s = idx >= 0 ? ld_volatile(&tstate[idx]) : ST_INCL;
        const unsigned int flag = (unsigned int)(s >> 62);
        const unsigned int m2 = __ballot_sync(0xffffffffu, flag == 2u);
        const unsigned int m0 = __ballot_sync(0xffffffffu, flag == 0u);
        const int stop = m2 ? __ffs(m2) - 1 : 31;
        const unsigned int need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
        if (m0 & need) {
            if (++spins > LOOKBACK_SPIN_LIMIT) {
                timed_out = true;
                break;
            }
            __nanosleep(backoff);
            backoff = min(backoff * 2, 1024);
            continue;
        }
        long long v = lane <= stop ? (long long)(s & ST_VAL) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (m2) break;
        j -= 32;
        backoff = 32;
    }
    if (timed_out && lane == 0) atomicOr(flags, ST_TIMEOUT);
    if (lane == 0) atomicExch(&tstate[t], ST_INCL | (unsigned long long)(excl + agg));
    return excl;
}

__device__ __forceinline__ unsigned int tau16_bits(int mx) {
    // FP16 band in u^2 for frame coordinates |X| <= mx (see sph_precision_bands):
    // |X| < 4 -> 0.03, |X| < 8 -> 0.06.
    const __half t = __float2half_rn(mx < 4 ? 0.03f : 0.06f);
    return h2_bits(__halves2half2(t, t));
}

// Everything one lane needs about its home particle.
struct Home {
    int i;           // sorted index
    int x;           // cell x
    __half2 X, Y, Z; // FP16 frame coordinates, splatted
    float x32, y32, z32;
};

enum { PASS_SINGLE = 0, PASS_COUNT = 1, PASS_EMIT = 2 };

// Candidate row table of a home group (cells [xa, xb] of row (cy, cz)).
template <int DIM>
__device__ __forceinline__ void group_rows(TileSmem &S, const GridDev &g, int cy, int cz, int xa, int xb) {
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    const int lane = threadIdx.x & 31;
    const int nx = g.nk[0], ny = g.nk[1], nz = g.nk[2];
    const int x_lo = max(xa - 1, 0), x_hi = min(xb + 1, nx - 1);
    const int nb = x_hi - x_lo + 2;  // boundaries per row (<= SPANMAX + 3)
    for (int e = lane; e < 9 * 8; e += 32) {
        const int r = e >> 3, k = e & 7;
        int v = 0;
        if (r < NROWS && k < nb) {
            const int dy = DIM == 3 ? (r % 3) - 1 : r - 1;
            const int dz = DIM == 3 ? (r / 3) - 1 : 0;
            const int yy = cy + dy, zz = cz + dz;
            if (yy >= 0 && yy < ny && zz >= 0 && zz < nz)
                v = g.cell_start[((long long)zz * ny + yy) * nx + x_lo + k];
            else
                v = -1;
        }
        S.rcb[r][k] = v;
    }
    __syncwarp();
    int len = 0, start = 0, dy = 0, dz = 0;
    if (lane < 9) {
        const int r = lane;
        if (r < NROWS) {
            dy = DIM == 3 ? (r % 3) - 1 : r - 1;
            dz = DIM == 3 ? (r / 3) - 1 : 0;
            if (S.rcb[r][0] >= 0) {
                start = S.rcb[r][0];
                len = S.rcb[r][nb - 1] - start;
            }
        }
        S.rstart[r] = start;
        S.rdy[r] = dy;
        S.rdz[r] = dz;
    }
    int inc = len;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane < 9) S.roff[lane] = inc - len;
    if (lane == 8) {
        S.roff[9] = inc;
        S.C = inc;
        S.nbm1 = nb - 1;
    }
    __syncwarp();
}

// Stage candidates [w0, w0 + wc) (window-local slots 0..wc-1; the rest of the
// window is padded far away) and their indices into jall[w0 - s0 + .].
__device__ __forceinline__ void stage_window(TileSmem &S, const GridDev &g, int w0, int wc, int s0, int xlo,
                                             int xm) {
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < WIN; k += 32) {
        __half hx, hy, hz;
        float4 f;
        if (k < wc) {
            const int p = w0 + k;
            int r = 0;
#pragma unroll
            for (int q = 1; q < 9; ++q) r = (p >= S.roff[q]) ? q : r;
            const int j = S.rstart[r] + (p - S.roff[r]);
            int cxo = 0;  // cell x offset from x_lo: internal boundaries passed
            const int nbm1 = S.nbm1;
#pragma unroll
            for (int q = 1; q < 7; ++q) cxo += (q < nbm1 && j >= S.rcb[r][q]) ? 1 : 0;
            const float sx = 2.f * (float)(xlo + cxo - xm);
            const float sy = 2.f * (float)S.rdy[r], sz = 2.f * (float)S.rdz[r];
            const uint2 q16 = g.rel16[j];
            const float4 r32 = g.rel32[j];
            const __half2 xy = __hadd2(as_h2(q16.x), __floats2half2_rn(sx, sy));
            hx = __low2half(xy);
            hy = __high2half(xy);
            hz = __hadd(__low2half(as_h2(q16.y)), __float2half_rn(sz));
            f = make_float4(__fadd_rn(r32.x, sx), __fadd_rn(r32.y, sy), __fadd_rn(r32.z, sz), __int_as_float(j));
        } else {
            hx = hy = hz = __float2half_rn(30000.f);
            f = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        }
        S.f32[k] = f;
        const int word = ((k >> 5) << 4) + (k & 15), hi = (k >> 4) & 1;
        __half *pw = reinterpret_cast<__half *>(&S.pw[word]);
        pw[hi] = hx;
        pw[2 + hi] = hy;
        pw[4 + hi] = hz;
    }
    __syncwarp();
}

// FP16 tests of the window against the lane's home particle: one bit per
// candidate, written to S.S[lane][wbase + g] for the WIN/32 words g.
template <int DIM>
__device__ __forceinline__ void test_window(TileSmem &S, const Home &h, bool active, unsigned int negT,
                                            unsigned int tau, int wbase) {
    const int lane = threadIdx.x & 31;
    const __half2 nT = as_h2(negT);
    const __half2 tv = as_h2(tau);
#pragma unroll 1
    for (int gi = 0; gi < WIN / 32; ++gi) {
        unsigned int word = 0;
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const uint4 c = S.pw[gi * 16 + b];
            const __half2 dx = __hsub2(as_h2(c.x), h.X);
            const __half2 dy = __hsub2(as_h2(c.y), h.Y);
            __half2 e = __hfma2(dx, dx, nT);
            e = __hfma2(dy, dy, e);
            if (DIM == 3) {
                const __half2 dz = __hsub2(as_h2(c.z), h.Z);
                e = __hfma2(dz, dz, e);
            }
            word |= __hlt2_mask(e, tv) & ((1u << b) | (1u << (16 + b)));
        }
        S.S[lane][wbase + gi] = active ? word : 0u;
    }
    __syncwarp();
}

// Walk the lane's maybe bits of words [wbase, wbase + nw): FP32 re-decision
// (FP64 inside the band), density; clears rejected bits.  In PASS_EMIT the
// neighbours are written straight to col[rp + cnt].
template <int DIM, int PASS>
__device__ __forceinline__ void walk_window(TileSmem &S, const GridDev &g, const Home &h, int wbase, int nw,
                                            int &cnt, float &acc, bool want_rho, int *col, long long rp,
                                            bool wc, unsigned int &n32, unsigned int &n64) {
    const int lane = threadIdx.x & 31;
    int gi = 0;
    unsigned int w = nw > 0 ? S.S[lane][wbase] : 0u, fin = w;
    while (true) {
        while (w == 0u && gi < nw) {
            S.S[lane][wbase + gi] = fin;
            ++gi;
            if (gi < nw) {
                w = S.S[lane][wbase + gi];
                fin = w;
            }
        }
        if (!__any_sync(0xffffffffu, gi < nw)) break;
        if (gi < nw) {
            const int b = __ffs(w) - 1;
            w &= w - 1u;
            const float4 c = S.f32[gi * 32 + b];
            const int j = __float_as_int(c.w);
            int in = 0;
            float r2 = 0.f;
            if (j != h.i) {
                const float d0 = __fsub_rn(c.x, h.x32);
                const float d1 = __fsub_rn(c.y, h.y32);
                const float d2 = __fsub_rn(c.z, h.z32);
                r2 = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
                if (r2 < g.t32_in) {
                    in = 1;
                } else if (r2 > g.t32_out) {
                    ++n32;
                } else {
                    ++n64;
                    const int oi = g.orig_id[h.i], oj = g.orig_id[j];
                    in = r2_fp64(DIM, g.xyz + (long long)oi * DIM, g.xyz + (long long)oj * DIM) < g.kh2;
                }
            }
            if (in) {
                if (want_rho) acc += g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
                if (PASS == PASS_EMIT && wc) col[rp + cnt] = j;
                ++cnt;
            } else {
                fin &= ~(1u << b);
            }
        }
    }
    __syncwarp();
}

template <int DIM>
__global__ void __launch_bounds__(32) k_nnps_tile(GridDev g, const int4 *__restrict__ tiles,
                                                 const long long *__restrict__ ntiles_dev,
                                                 long long *__restrict__ row_ptr, int *__restrict__ col,
                                                 long long cap, float *__restrict__ rho,
                                                 unsigned long long *__restrict__ tstate) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(smraw);
    const int lane = threadIdx.x;
    const int nx = g.nk[0], ny = g.nk[1];
    const bool want_rho = rho != nullptr;
    const long long ntiles = *ntiles_dev;
    unsigned int n32 = 0, n64 = 0;

    while (true) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&g.status->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int4 td = tiles[t];
        const int p0 = td.x, cnt_home = td.y, row = td.z;
        const int cy = row % ny, cz = row / ny;
        const bool mine = lane < cnt_home;
        Home h;
        h.i = p0 + lane;
        h.x = mine ? g.scell_x[h.i] : 0;

        // home groups: runs of lanes whose cells span <= SPANMAX
        int ngroups = 0;
        {
            int gs = 0;
            while (gs < cnt_home) {
                const int xa = __shfl_sync(0xffffffffu, h.x, gs);
                const unsigned int over = __ballot_sync(0xffffffffu, mine && lane >= gs && h.x > xa + SPANMAX - 1);
                gs = over ? __ffs(over) - 1 : cnt_home;
                ++ngroups;
            }
        }
        int cnt = 0;
        float acc = 0.f;
        const bool simple_try = ngroups == 1;
        bool simple = simple_try;
        // ---- pass 1 (count, or single) ---------------------------------------
        for (int pass = 0; pass < 2; ++pass) {
            const bool emit = pass == 1;
            if (emit && simple) break;
            long long rp = 0;
            if (emit) rp = mine ? row_ptr[h.i] : 0;
            int gs = 0;
            while (gs < cnt_home) {
                const int xa = __shfl_sync(0xffffffffu, h.x, gs);
                const unsigned int over = __ballot_sync(0xffffffffu, mine && lane >= gs && h.x > xa + SPANMAX - 1);
                const int ge = over ? __ffs(over) - 1 : cnt_home;
                const int xb = __shfl_sync(0xffffffffu, h.x, ge - 1);
                const bool act = mine && lane >= gs && lane < ge;
                const int xm = (xa + xb) >> 1;
                const int xlo = max(xa - 1, 0), xhi = min(xb + 1, nx - 1);
                group_rows<DIM>(S, g, cy, cz, xa, xb);
                const int C = S.C;
                if (!emit && C > CMAX) simple = false;
                // home frame coordinates
                {
                    const uint2 q = g.rel16[min(h.i, g.n - 1)];
                    const float4 r = g.rel32[min(h.i, g.n - 1)];
                    const float sx = 2.f * (float)(h.x - xm);
                    const __half X = __hadd(__low2half(as_h2(q.x)), __float2half_rn(sx));
                    h.X = __halves2half2(X, X);
                    h.Y = __high2half2(as_h2(q.x));
                    h.Z = __low2half2(as_h2(q.y));
                    h.x32 = __fadd_rn(r.x, sx);
                    h.y32 = r.y;
                    h.z32 = r.z;
                }
                const int mx = 1 + 2 * max(xm - xlo, xhi - xm);
                const unsigned int tau = tau16_bits(mx);
                for (int s0 = 0; s0 < C; s0 += CMAX) {
                    const int sc = min(CMAX, C - s0);
                    for (int w0 = s0; w0 < s0 + sc; w0 += WIN) {
                        const int wc = min(WIN, s0 + sc - w0);
                        stage_window(S, g, w0, wc, s0, xlo, xm);
                        const int wbase = (w0 - s0) >> 5;
                        test_window<DIM>(S, h, act, g.neg_t16, tau, wbase);
                        const int nw = (wc + 31) >> 5;
                        if (emit)
                            walk_window<DIM, PASS_EMIT>(S, g, h, wbase, act ? nw : 0, cnt, acc, false, col, rp,
                                                        true, n32, n64);
                        else
                            walk_window<DIM, PASS_COUNT>(S, g, h, wbase, act ? nw : 0, cnt, acc, want_rho,
                                                         nullptr, 0, false, n32, n64);
                    }
                }
                gs = ge;
            }
            if (!emit) {
                // ---- offsets across tiles --------------------------------------
                int inc = mine ? cnt : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += v;
                }
                const int agg = __shfl_sync(0xffffffffu, inc, 31);
                const int roff = inc - (mine ? cnt : 0);
                const long long pre = look_back(tstate, t, agg, &g.status->flags);
                const bool wc = col != nullptr && pre + agg <= cap;
                if (col != nullptr && !wc && lane == 0) atomicOr(&g.status->flags, ST_CAPACITY);
                if (mine) {
                    row_ptr[h.i] = pre + roff;
                    if (want_rho) rho[h.i] = g.w_self + acc;
                }
                if (t == ntiles - 1 && lane == 0) row_ptr[g.n] = pre + agg;
                if (simple && wc && col != nullptr) {
                    // emit each row from its kept bits; the column index comes
                    // from the candidate row table (rows are contiguous ranges)
                    const int nw = (S.C + 31) >> 5;
                    long long pos = pre + roff;
                    int gi = 0;
                    unsigned int w = (mine && nw > 0) ? S.S[lane][0] : 0u;
                    while (true) {
                        while (w == 0u && gi < nw) {
                            ++gi;
                            if (gi < nw) w = mine ? S.S[lane][gi] : 0u;
                        }
                        if (!__any_sync(0xffffffffu, gi < nw)) break;
                        if (gi < nw) {
                            const int b = __ffs(w) - 1;
                            w &= w - 1u;
                            const int p = gi * 32 + b;
                            int r = 0;
#pragma unroll
                            for (int q = 1; q < 9; ++q) r = (p >= S.roff[q]) ? q : r;
                            col[pos++] = S.rstart[r] + (p - S.roff[r]);
                        }
                    }
                    __syncwarp();
                }
                if (!simple) {
                    // second pass re-derives the rows and writes them in place
                    cnt = 0;
                    acc = 0.f;
                    if (!wc) break;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n32 += __shfl_xor_sync(0xffffffffu, n32, o);
        n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    }
    if (lane == 0) {
        if (n32) atomicAdd(&g.status->fp32_pairs, (unsigned long long)n32);
        if (n64) atomicAdd(&g.status->fp64_pairs, (unsigned long long)n64);
    }
}

// Tiles per x-row of cells: ceil(particles / 32).
__global__ void k_row_tiles_count(GridDev g, int *__restrict__ tcount) {
    const long long nrow = (long long)g.nk[1] * g.nk[2];
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrow; r += (long long)gridDim.x * blockDim.x) {
        const long long base = r * g.nk[0];
        const int len = g.cell_start[base + g.nk[0]] - g.cell_start[base];
        tcount[r] = (len + TW - 1) / TW;
    }
}

__global__ void k_row_tiles_write(GridDev g, const long long *__restrict__ toff, int4 *__restrict__ tiles) {
    const long long nrow = (long long)g.nk[1] * g.nk[2];
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrow; r += (long long)gridDim.x * blockDim.x) {
        const long long base = r * g.nk[0];
        const int a = g.cell_start[base], b = g.cell_start[base + g.nk[0]];
        long long o = toff[r];
        for (int p = a; p < b; p += TW) tiles[o++] = make_int4(p, min(TW, b - p), (int)r, 0);
    }
}

// Cell x of every sorted particle.
__global__ void k_cell_x(GridDev g, const int *__restrict__ scell, int *__restrict__ sx) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n; s += (long long)gridDim.x * blockDim.x)
        sx[s] = scell[s] % g.nk[0];
}

}  // namespace

size_t tile_smem_bytes() { return sizeof(TileSmem); }

// Build the tile list of a binned grid.  tcount: int[nrow], toff: int64[nrow+1],
// tiles: int4[ntiles_max] with ntiles_max = n / 32 + nrow.
cudaError_t launch_tiles(const GridDev &g, const int *scell, int *scell_x, int *tcount, long long *toff,
                         void *scan_tmp, int4 *tiles, int sm_count, cudaStream_t s) {
    const long long nrow = (long long)g.nk[1] * g.nk[2];
    const int nt = 256;
    long long b = (nrow + nt - 1) / nt;
    if (b > (long long)sm_count * 8) b = (long long)sm_count * 8;
    if (b < 1) b = 1;
    long long bn = (g.n + nt - 1) / nt;
    if (bn > (long long)sm_count * 16) bn = (long long)sm_count * 16;
    if (bn < 1) bn = 1;
    ProfScope ps(TAG_SCAN, s);
    note_launch(3);
    k_cell_x<<<(unsigned)bn, nt, 0, s>>>(g, scell, scell_x);
    k_row_tiles_count<<<(unsigned)b, nt, 0, s>>>(g, tcount);
    cudaError_t e = exclusive_scan_i64(tcount, toff, nrow, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_row_tiles_write<<<(unsigned)b, nt, 0, s>>>(g, toff, tiles);
    return cudaGetLastError();
}

// ntiles_dev: device pointer to the tile count (the last entry of the row
// tile offsets); ntiles_max bounds it (sizes the look-back state).
cudaError_t launch_nnps_tile(const GridDev &g, const int4 *tiles, const long long *ntiles_dev, long long ntiles_max,
                             long long *row_ptr, int *col, long long cap, float *rho, unsigned long long *tstate,
                             int sm_count, cudaStream_t s) {
    const size_t sb = sizeof(TileSmem);
    auto kern = g.dim == 2 ? k_nnps_tile<2> : k_nnps_tile<3>;
    static bool attr_done[2] = {false, false};
    if (!attr_done[g.dim - 2]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
        if (e != cudaSuccess) return e;
        attr_done[g.dim - 2] = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, sb);
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > ntiles_max) blocks = ntiles_max;
    if (blocks < 1) blocks = 1;
    cudaError_t e =
        cudaMemsetAsync(tstate, 0, (size_t)(ntiles_max > 0 ? ntiles_max : 1) * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    ProfScope ps(TAG_FUSED, s);
    note_launch(1);
    kern<<<(unsigned)blocks, 32, sb, s>>>(g, tiles, ntiles_dev, row_ptr, col, cap, rho, tstate);
    return cudaGetLastError();
}

}  // namespace sph
