// nnps_tile.cu -- single-pass FP16-RCLL neighbour search + SPH density with
// one warp per row tile (the production search for cell-order queries).
//
// Tiles: the cell-sorted particles of every x-row of cells (fixed y, z) are
// cut into runs of at most 32; a warp takes tiles in order from an atomic
// ticket and lane l owns home particle p0 + l, i.e. one CSR row.
//
// Per home group (the tile's particles whose cells span at most SPANMAX
// consecutive x-cells; normally the whole tile):
//   * the candidates are the 3^d x-rows of cells around the group's cells
//     (each a contiguous range of the sorted arrays), x-range widened by one
//     cell; coordinates are the cell-relative ones of Eq. 6 re-expressed in
//     the frame of the group's middle cell, X = x_rel + 2 (c_x - x_mid),
//     Y = y_rel + 2 dy, Z = z_rel + 2 dz (units of u = h_c / 2), so a pair's
//     difference is the Eq. 7 distance with the scale h_c / 2; in the dense
//     shape the FP16 x of a group of an even number of cells is shifted by
//     one more (-1: frame centre on the face between the middle two cells,
//     so a two-cell group keeps |X| <= 4 and the narrower FP16 band: fewer
//     pairs to re-decide where many lie near kh); the FP32 coordinates keep
//     the cell-centred frame, so distances and densities do not depend on
//     the shape;
//   * cull: candidates farther than kh (plus a margin) from the bounding box
//     of the group's particles cannot be anybody's neighbour and are dropped;
//     the rest are compacted in candidate order (ascending column);
//   * stage windows of kept candidates in shared memory: FP16 coordinates
//     two per half2 word for the window's test, FP32 coordinates into a
//     ring that holds two windows;
//   * FP16 test (all lanes, candidates broadcast): e = ((dx^2 - T) + dy^2)
//     + dz^2 with half2 FMAs; e < tau16 sets the candidate's bit in the
//     lane's row bitmask;
//   * each lane walks its own bits: FP32 distance from the FP32 relative
//     coordinates, FP32 band decision (FP64 definition inside the band),
//     neighbour count and density sum (Eq. 3) in CSR order; rejected bits are
//     cleared.  Window w is walked once window w + 1 is staged and tested, so
//     a lane that has finished its bits of w goes on with its bits of w + 1
//     while the others finish w (the lanes' bit counts differ per window far
//     more than per tile).
// Then the tile's neighbour total is published and its CSR offset found by a
// decoupled look-back over earlier tiles; each lane writes its row pointer
// and density, and emits its row from the kept bits.  Tiles with several
// home groups or more than CMAX kept candidates run the steps twice (count,
// then emit straight to their rows after the look-back).
#include <stddef.h>

#include <algorithm>

#include <mutex>

#include "launch.cuh"
#include "lookback.cuh"
#include "nnps_common.cuh"
#include "tile_rows.cuh"

namespace sph {

using namespace nn;
using namespace lb;

namespace {

constexpr int TW = TILE_ROWS;     // rows per tile
constexpr int SPANMAX = TILE_SPAN;  // home cells per group along x (keeps |X| < 8)
constexpr float CULL_MARGIN = 0.02f;  // u^2, covers the FP16 rounding of the culling test
constexpr int TILE_MAX_EXTRA_SMEM = 65536;  // largest extra staging a launch may ask for

// Shared-memory shape of the tile search: kept candidates per pass (the
// bitmask length), candidates per staging window, windows whose FP32
// coordinates stay staged together (a ring: the walk of window w may run
// into window w + 1 while the slowest lane finishes w), warps per CTA and the
// resident warps per SM it is built for (the register budget: 96 per thread
// at 20 warps, 128 at 16), the walk's bits in flight per lane (measured: 3 at
// 20 warps, 4 at 16) and spare bytes that only widen the output staging area.
// Each warp works alone on its own tiles in its own shared-memory area; two
// warps per CTA share the SM's per-CTA reservation.  Sparse: 10.8 KB per
// warp, 20 warps per SM; its output area (code, pw, the FP32 ring and the
// spare bytes after the last window) holds 2,640 entries, a tile of 32 rows
// of up to ~80 neighbours.  Dense: 13.7 KB, 16 warps, 832 kept candidates and
// 3,488 output entries for denser particle sets.
template <int CMAX_, int WIN_, int NBUF_, int WPB_, int WSM_, int WB_, int SPARE_, bool FACE_>
struct TileCfg {
    static constexpr int CMAX = CMAX_;
    static constexpr int WIN = WIN_;
    static constexpr int RING = NBUF_ * WIN_;  // FP32 slots of the ring
    static constexpr int RW = RING / 32;        // ring words: kept word q is staged at ring word q % RW
    static constexpr int WPB = WPB_;
    static constexpr int WSM = WSM_;
    static constexpr int WB = WB_;  // bits in flight per lane in the walk (independent loads and arithmetic)
    static constexpr int SPARE = SPARE_;
    // FP16 frame centre of an even number of home cells on the face between
    // the middle two (|X| <= 4 for two-cell groups: the narrower FP16 band)
    static constexpr bool FACE = FACE_;
    static constexpr int NWORD = CMAX_ / 32;
    // Bitmask matrix: NWORD + 1 words per lane.  With an even row stride the
    // words of lanes l and l + 16 in one column share a bank; lanes 16..31
    // then start one word later (in the padding word), which puts the 32
    // lanes' words of a column in 32 different banks.
    static constexpr int SSHIFT = (NWORD + 1) % 2 == 0 ? 1 : 0;
    static_assert(CMAX_ % 32 == 0 && WIN_ % 32 == 0 && WIN_ <= CMAX_, "tile shape");
    static_assert(NBUF_ == 2, "the walk of a window runs into the next one only");
    static_assert(NWORD <= 32, "non-empty word masks are 32 bits");
    static_assert(WSM_ % WPB_ == 0, "warps per CTA");
};
using TileSparse = TileCfg<672, 128, 2, 2, 20, 4, 480, false>;
using TileDense = TileCfg<832, 192, 2, 2, 16, 4, 16, true>;


template <class C>
struct TileSmem {
    unsigned int S[TW][C::NWORD + 1];
    __device__ __forceinline__ unsigned int &bits(int lane, int word) { return S[lane][word + C::SSHIFT * (lane >> 4)]; }
    __device__ __forceinline__ unsigned int bits(int lane, int word) const { return S[lane][word + C::SSHIFT * (lane >> 4)]; }
    int jall[C::CMAX];  // kept candidates: sorted index
    short selfpos[TW];  // kept slot of each lane's own particle (-1: not in this fill)
    // candidate rows r: sorted index minus flat index of the row's candidates,
    // code bits (dy + 1) << 3 | (dz + 1) << 5, frame shifts 2 dy and 2 dz (float bits)
    int4 rt[9];
    int rcum[10], pad[2];  // flat index of row r's first candidate; [nrows] = total
    // code, pw, the ring and spare come last and are contiguous with any
    // extra dynamic shared memory of the launch: after the last window they
    // hold the tile's staged output (16-bit kept-candidate slots), stg_slots
    // of them
    unsigned char code[C::CMAX];  // kept candidates: frame cell offsets (x + 3) | (dy + 1) << 3 | (dz + 1) << 5,
                                  // and 1 << 7 when the FP16 frame centre is on a cell face (x shift 2 x - 1)
    uint4 pw[C::WIN / 2];         // FP16 pairs of the window under test: word (g*16 + b) = its candidates 32g + b (lo), 32g + 16 + b (hi)
    float2 fxy[C::RING + 2];      // FP32 frame coordinates of the staged windows: kept slot 32 q + b at 32 (q % RW) + b,
    float fz[C::RING + 4];        // then a guard slot (read, never used, by the walk's empty bits)
    unsigned char spare[C::SPARE > 0 ? C::SPARE : 16];
    static constexpr size_t staging_bytes() {
        return sizeof(code) + sizeof(pw) + sizeof(fxy) + sizeof(fz) + sizeof(spare);
    }
};


__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 6 P(R) of Eq. 3 (P without alpha_d) for R >= 0, without a branch:
// max(2 - R, 0)^3 - 4 max(1 - R, 0)^3 equals (2 - R)^3 on [1, 2), 4 - 6 R^2 +
// 3 R^3 = 6 (2/3 - R^2 + R^3 / 2) on [0, 1) and 0 from R = 2 on; the second
// clamp is a saturating add.  The factor 1/6 is applied once per row.
__device__ __forceinline__ float w_poly6c(float R) {
    const float t = fmaxf(2.f - R, 0.f), s = __saturatef(1.f - R);
    return __fmaf_rn(-4.f * s, s * s, t * t * t);
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Everything one lane needs about its home particle in the current group.
struct Home {
    int i;            // sorted index
    int x;            // cell x
    __half2 X, Y, Z;  // FP16 frame coordinates, splatted
    float x32, y32, z32;
};

// One home group: its cells, frame and candidate rows.
struct Group {
    int xa, xb, xm, xlo, xhi;      // home cells [xa, xb], middle xm, candidate cells [xlo, xhi]; with
                                   // TileCfg::FACE and an even number of cells the FP16 frame centre is on
                                   // xm's right face
    float lo[3], hi[3];            // bounding box of the group's particles (frame, FP32)
    unsigned int tau;              // FP16 band (half2 bits)
};

// Candidate row table of a group (tile_rows.cuh).
template <int DIM, class C>
__device__ __forceinline__ void group_rows(TileSmem<C> &S, const GridDev &g, int cy, int cz, const Group &G) {
    tile_candidate_rows<DIM>(S.rt, S.rcum, g, cy, cz, G.xlo, G.xhi);
}

constexpr int CULL_CHUNKS = 4;  // chunks of 32 candidates whose loads are in flight together

// Cull and compact candidates of the group, resuming at the flat candidate
// index cur (rows in order, each row's candidates in order: ascending sorted
// index), until the union is exhausted or the kept list cannot take another
// 32.  Returns the number kept; advances the cursor.
template <int DIM, class C>
__device__ __forceinline__ int cull_fill(TileSmem<C> &S, const GridDev &g, const Group &G, float cullT, int &cur,
                                         int p0, int nhome) {
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    constexpr int U = CULL_CHUNKS;
    const int lane = threadIdx.x & 31;
    S.selfpos[lane] = -1;
    __syncwarp();
    int rc[NROWS];
#pragma unroll
    for (int r = 0; r < NROWS; ++r) rc[r] = S.rcum[r + 1];
    const int total = rc[NROWS - 1];
    int kept = 0;
    while (cur < total && kept + 32 <= C::CMAX) {
        const int nu = kept + 32 * U <= C::CMAX ? U : 1;  // warp-uniform
        int jk[U], rr[U];
        bool valid[U];
        uint2 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = cur + 32 * u + lane;
            valid[u] = u < nu && k < total;
            int r = 0;  // row of flat index k: rows before it end at or below k
#pragma unroll
            for (int t = 0; t < NROWS - 1; ++t) r += k >= rc[t] ? 1 : 0;
            rr[u] = r;
            jk[u] = k + S.rt[r].x;
            q[u] = valid[u] ? g.rel16[jk[u]] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u >= nu) break;
            const int4 rt = S.rt[rr[u]];
            const int ox = rel_cell_offset(q[u], G.xm);  // frame cell offset in x, |ox| <= 3
            bool keep = false;
            if (valid[u]) {
                const float2 xy = __half22float2(as_h2(q[u].x));
                const float x = xy.x + 2.f * (float)ox, y = xy.y + __int_as_float(rt.z);
                const float z = __low2float(as_h2(q[u].y)) + __int_as_float(rt.w);
                const float ex = fmaxf(fmaxf(G.lo[0] - x, x - G.hi[0]), 0.f);
                const float ey = fmaxf(fmaxf(G.lo[1] - y, y - G.hi[1]), 0.f);
                const float ez = fmaxf(fmaxf(G.lo[2] - z, z - G.hi[2]), 0.f);
                keep = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < cullT;
            }
            const unsigned int m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = kept + __popc(m & ((1u << lane) - 1u));
                S.jall[pos] = jk[u];
                S.code[pos] = (unsigned char)((ox + 3) | rt.y | (C::FACE ? ((G.xa + G.xb) & 1) << 7 : 0));
                // the tile's own particles are the contiguous range [p0, p0 + nhome)
                if (jk[u] >= p0 && jk[u] < p0 + nhome) S.selfpos[jk[u] - p0] = (short)pos;
            }
            kept += __popc(m);
        }
        cur += 32 * nu;
    }
    __syncwarp();
    return kept;
}

// Stage kept candidates [w0, w0 + wc) (w0 a multiple of 32): FP16 pairs for
// the window's test (slots past wc padded far away) and FP32 coordinates
// into the ring at 32 (w0 / 32 % RW) + k.
template <class C>
__device__ __forceinline__ void stage_window(TileSmem<C> &S, const GridDev &g, int w0, int wc) {
    const int lane = threadIdx.x & 31;
    const int ring0 = ((w0 >> 5) % C::RW) * 32;
#pragma unroll 4
    for (int k = lane; k < C::WIN; k += 32) {
        __half hx, hy, hz;
        if (k < wc) {
            const int j = S.jall[w0 + k];
            const unsigned int c = S.code[w0 + k];
            const float sx = 2.f * (float)((int)(c & 7u) - 3);
            const float sy = 2.f * (float)((int)((c >> 3) & 3u) - 1);
            const float sz = 2.f * (float)((int)((c >> 5) & 3u) - 1);
            const uint2 q16 = g.rel16[j];
            const float4 r32 = g.rel32[j];
            // FP16 x shifted one less when the frame centre is on a cell face
            const __half2 xy = __hadd2(as_h2(q16.x), __floats2half2_rn(C::FACE ? sx - (float)(c >> 7) : sx, sy));
            hx = __low2half(xy);
            hy = __high2half(xy);
            hz = __hadd(__low2half(as_h2(q16.y)), __float2half_rn(sz));
            S.fxy[ring0 + k] = make_float2(__fadd_rn(r32.x, sx), __fadd_rn(r32.y, sy));
            S.fz[ring0 + k] = __fadd_rn(r32.z, sz);
        } else {
            hx = hy = hz = __float2half_rn(30000.f);
        }
        const int word = ((k >> 5) << 4) + (k & 15), hi = (k >> 4) & 1;
        __half *pw = reinterpret_cast<__half *>(&S.pw[word]);
        pw[hi] = hx;
        pw[2 + hi] = hy;
        pw[4 + hi] = hz;
    }
    __syncwarp();
}

// FP16 tests of the window (nwin words of 32) against the lane's home
// particle; bit per kept candidate into S.bits(lane, wbase + gi).  The lane's
// own particle (window slot self_slot, or -1) is left out.
template <int DIM, class C>
__device__ __forceinline__ unsigned int test_window(TileSmem<C> &S, const Home &h, bool active, unsigned int negT,
                                                    unsigned int tau, int wbase, int nwin, int self_slot, int &nbits) {
    const int lane = threadIdx.x & 31;
    const __half2 nT = as_h2(negT);
    const __half2 tv = as_h2(tau);
    unsigned int nem = 0;  // non-empty words, returned for the walk
#pragma unroll 1
    for (int gi = 0; gi < nwin; ++gi) {
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
        if ((self_slot >> 5) == gi) word &= ~(1u << (self_slot & 31));
        word = active ? word : 0u;
        S.bits(lane, wbase + gi) = word;
        nem |= (word != 0u ? 1u : 0u) << gi;
        nbits += __popc(word);
    }
    __syncwarp();
    return nem;
}

enum { PASS_COUNT = 0, PASS_EMIT = 1 };

// The lane's set bits in ascending order, up to WB per call: positions p[k]
// with v[k] marking valid ones (invalid ones still index inside the row's
// ring word or slot word, or one past it).  RING: p is the FP32 ring
// position 32 (q % RW) + b of bit b of kept word q, else the kept slot
// 32 q + b.  State: the current word w (its base rb), the next non-empty word
// wn (base rbn), prefetched once per call, and nem, the lane's non-empty
// words not yet fetched (bit q for word q).  A word that runs out mid-call is
// replaced by a register move; the next word is prefetched before bits k
// with k % RI == 0, so a call may return fewer than WB bits when two words
// run out between prefetches.
struct BitCursor {
    unsigned int w = 0u, wn = 0u, nem = 0u;
    int rb = 0, rbn = 0;
};
template <int WB, class C, bool RING, int RI = WB>
__device__ __forceinline__ void next_bits(const TileSmem<C> &S, int lane, BitCursor &b, int (&p)[WB], bool (&v)[WB]) {
#pragma unroll
    for (int k = 0; k < WB; ++k) {
        if (k % RI == 0 && b.wn == 0u && b.nem != 0u) {
            const int gn = __ffs(b.nem) - 1;
            b.nem &= b.nem - 1u;
            b.wn = S.bits(lane, gn);
            b.rbn = RING ? (gn % C::RW) * 32 : gn * 32;
        }
        if (b.w == 0u) {
            b.w = b.wn;
            b.rb = b.rbn;
            b.wn = 0u;
        }
        v[k] = b.w != 0u;
        p[k] = b.rb + __clz(__brev(b.w));  // lowest set bit; 32 for an empty word
        b.w &= b.w - 1u;
    }
}

// Kept word of ring position p while windows from word q0 on are staged
// (the ring holds the RW consecutive kept words from q0); r0 = q0 % RW, used
// when RW is not a power of two (the dense shape).
template <class C>
__device__ __forceinline__ int ring_word(int p, int q0, int r0) {
    if ((C::RW & (C::RW - 1)) == 0) return q0 + ((p >> 5) - q0 % C::RW + C::RW) % C::RW;
    const int d = (p >> 5) - r0;
    return q0 + (d < 0 ? d + C::RW : d);
}


// The FP64 definition for the rare pairs inside the FP32 band.  Kept out of
// line so that its global loads and FP64 arithmetic are never hoisted into
// the walk loop (FP64 throughput on this part is a small fraction of FP32).
template <int DIM>
__device__ __noinline__ bool fp64_tier(const GridDev &g, int i, int j) {
    const int oi = g.orig_id[i], oj = g.orig_id[j];
    return r2_fp64(DIM, g.xyz + (long long)oi * DIM, g.xyz + (long long)oj * DIM) < g.kh2;
}

// The lane's own particle has been removed from its bits by test_window, so
// every remaining bit is a pair j != i.  The common case (FP32 says
// "neighbour") runs without branches and the density is summed for every
// valid bit (see below); steps in which some lane holds a pair the FP32 tier
// rejects or leaves in its band take a warp-uniform branch to decide those
// (FP64 tier out of line; a rejected bit is cleared).  K bits (ring positions
// p[k], valid v[k]) of the lane's row; q0: first kept word still staged.
template <int DIM, int PASS, class C, int K>
__device__ __forceinline__ void walk_bits(TileSmem<C> &S, const GridDev &g, const Home &h, int q0, int r0,
                                          const int (&p)[K], const bool (&v)[K], int &cnt, float &acc, int *col,
                                          long long rp, unsigned int &n32, unsigned int &n64, bool dens) {
    const int lane = threadIdx.x & 31;
    float r2[K];
    bool in[K];
    bool odd = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float2 cxy = S.fxy[p[k]];  // p[k] <= RING: invalid bits read the guard slot at worst
        const float cz = S.fz[p[k]];
        const float d0 = __fsub_rn(cxy.x, h.x32);
        const float d1 = __fsub_rn(cxy.y, h.y32);
        const float d2 = __fsub_rn(cz, h.z32);
        r2[k] = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
        in[k] = v[k] && r2[k] < g.t32_in;
        odd |= v[k] && !in[k];
    }
    if (PASS != PASS_EMIT && dens) {
        // the weight vanishes from R = 2 on, so pairs the FP32 tier rejects
        // add exactly 0 and band pairs (R within ~1e-6 of 2) less than the
        // sum's last bit: the density needs no decision
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float wk = w_poly6c(sqrt_approx(r2[k]) * g.r_scale);
            acc += v[k] ? wk : 0.f;
        }
    }
    if (__any_sync(0xffffffffu, odd))
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (v[k] && !in[k]) {
            const int q = ring_word<C>(p[k], q0, r0);
            if (r2[k] <= g.t32_out) {
                ++n64;
                in[k] = fp64_tier<DIM>(g, h.i, S.jall[q * 32 + (p[k] & 31)]);
            } else {
                ++n32;
            }
            if (!in[k]) S.bits(lane, q) &= ~(1u << (p[k] & 31));
        }
    }
    if (PASS == PASS_EMIT) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (in[k]) col[rp + cnt++] = S.jall[ring_word<C>(p[k], q0, r0) * 32 + (p[k] & 31)];
    }
}

// Walk the lane's bits in candidate order (the emit pass needs it: columns
// ascending) until every lane has taken `target` bits (all its bits of the
// windows before the current one; `taken` counts them); lanes that are done
// run on into the next staged window.  q0: first kept word still staged.
template <int DIM, int PASS, class C>
__device__ __forceinline__ void walk_until(TileSmem<C> &S, const GridDev &g, const Home &h, BitCursor &cur, int q0,
                                           int target, int &taken, int &cnt, float &acc, int *col, long long rp,
                                           unsigned int &n32, unsigned int &n64, bool dens) {
    const int lane = threadIdx.x & 31;
    const int r0 = (C::RW & (C::RW - 1)) == 0 ? 0 : q0 % C::RW;
    while (__any_sync(0xffffffffu, taken < target)) {
        int p[C::WB];
        bool v[C::WB];
        next_bits<C::WB, C, true>(S, lane, cur, p, v);
#pragma unroll
        for (int k = 0; k < C::WB; ++k) taken += v[k] ? 1 : 0;
        walk_bits<DIM, PASS, C, C::WB>(S, g, h, q0, r0, p, v, cnt, acc, col, rp, n32, n64, dens);
    }
}

// Set up a home group of lanes [gs, ge): frame, bounding box, band, rows.
template <int DIM, class C>
__device__ __forceinline__ void group_setup(TileSmem<C> &S, const GridDev &g, Home &h, bool act, int cy, int cz, int gs,
                                            int ge, Group &G) {
    const int nx = g.nk[0];
    G.xa = __shfl_sync(0xffffffffu, h.x, gs);
    G.xb = __shfl_sync(0xffffffffu, h.x, ge - 1);
    G.xm = (G.xa + G.xb) >> 1;
    G.xlo = max(G.xa - 1, 0);
    G.xhi = min(G.xb + 1, nx - 1);
    const uint2 q = g.rel16[min(h.i, g.n - 1)];
    const float4 r = g.rel32[min(h.i, g.n - 1)];
    const int hf = C::FACE ? (G.xa + G.xb) & 1 : 0;
    const float sx = 2.f * (float)(h.x - G.xm);
    const __half X = __hadd(__low2half(as_h2(q.x)), __float2half_rn(sx - (float)hf));
    h.X = __halves2half2(X, X);
    h.Y = __high2half2(as_h2(q.x));
    h.Z = __low2half2(as_h2(q.y));
    h.x32 = __fadd_rn(r.x, sx);
    h.y32 = r.y;
    h.z32 = r.z;
    G.lo[0] = warp_min(act ? h.x32 : INFINITY);
    G.lo[1] = warp_min(act ? h.y32 : INFINITY);
    G.lo[2] = warp_min(act ? h.z32 : INFINITY);
    G.hi[0] = warp_max(act ? h.x32 : -INFINITY);
    G.hi[1] = warp_max(act ? h.y32 : -INFINITY);
    G.hi[2] = warp_max(act ? h.z32 : -INFINITY);
    // largest FP16 |X| of the group's candidates: 1 + the largest frame shift
    const int mx = C::FACE ? 1 + max(abs(2 * (G.xlo - G.xm) - hf), abs(2 * (G.xhi - G.xm) - hf))
                           : 1 + 2 * max(G.xm - G.xlo, G.xhi - G.xm);
    const __half t = __float2half_rn(mx <= 4 ? 0.03f : 0.06f);  // FP16 band for |X| <= 4 / < 8
    G.tau = h2_bits(__halves2half2(t, t));
    group_rows<DIM, C>(S, g, cy, cz, G);
}

// All candidates of one group against its lanes; returns false when the kept
// list needed more than one pass (the bits in S then cover only the last).
// Per pass: window 0 is staged and tested; then for each window w the next
// one is staged and tested (its FP32 coordinates go to the other half of the
// ring, whose previous window every lane has finished) and the lanes walk
// until all of them are past window w.
template <int DIM, int PASS, class C>
__device__ __forceinline__ bool run_group(TileSmem<C> &S, const GridDev &g, Home &h, bool act, const Group &G,
                                          float cullT, int &cnt, float &acc, int *col, long long rp,
                                          unsigned int &n32, unsigned int &n64, int &kept_out, int p0, int nhome,
                                          bool dens) {
    const int lane = threadIdx.x & 31;
    int cur = 0, passes = 0, kept = 0;
    while (true) {
        kept = cull_fill<DIM, C>(S, g, G, cullT, cur, p0, nhome);
        ++passes;
        const int sp = S.selfpos[lane];
        const int nwords = (kept + 31) >> 5;
        BitCursor bc;
        int tested = 0, taken = 0;  // the lane's bits in the windows tested so far, and taken by the walk
        for (int w0 = 0; w0 < kept + C::WIN; w0 += C::WIN) {
            // stage and test window w0 (if any), then walk window w0 - WIN
            const int before = tested;
            if (w0 < kept) {
                const int wc = min(C::WIN, kept - w0);
                stage_window<C>(S, g, w0, wc);
                const int self_slot = (sp >= w0 && sp < w0 + wc) ? sp - w0 : -1;
                bc.nem |= test_window<DIM, C>(S, h, act, g.neg_t16, G.tau, w0 >> 5, (wc + 31) >> 5, self_slot,
                                              tested)
                          << (w0 >> 5);
            }
            if (w0 > 0) {
                const int q0 = (w0 - C::WIN) >> 5;  // first word still staged
                walk_until<DIM, PASS, C>(S, g, h, bc, q0, w0 < kept ? before : tested, taken, cnt, acc, col, rp,
                                         n32, n64, dens);
            }
        }
        if (PASS == PASS_COUNT) {
            // the neighbours of this pass: its bits that survived the re-decision
            for (int q = 0; q < nwords; ++q) cnt += __popc(S.bits(lane, q));
        }
        __syncwarp();
        constexpr int NROWS = DIM == 3 ? 9 : 3;
        if (cur >= S.rcum[NROWS]) break;
    }
    kept_out = kept;
    return passes == 1;
}

// Emit the lane's kept bits (words [0, nw) of its row) in order: candidate
// slots as 16-bit entries to stg[pos...], or (stg == nullptr) the sorted
// indices jall[slot] to col[pos...].
template <class C>
__device__ __forceinline__ void emit_bits(const TileSmem<C> &S, int lane, int nw, long long pos, unsigned short *stg,
                                          int *col, const int *jall) {
    BitCursor cur;
    for (int q = 0; q < nw; ++q) cur.nem |= (S.bits(lane, q) != 0u ? 1u : 0u) << q;
    constexpr int EB = 8;
    while (true) {
        int p[EB];
        bool v[EB];
        next_bits<EB, C, false, 4>(S, lane, cur, p, v);
        if (!__any_sync(0xffffffffu, v[0])) break;
        // the valid bits of a call need not be a prefix (a word prefetched at
        // k = 4 can follow an empty slot): each goes to the next position
        int o[EB];
#pragma unroll
        for (int k = 0; k < EB; ++k) o[k] = (k == 0 ? 0 : o[k - 1] + (v[k - 1] ? 1 : 0));
        if (stg != nullptr) {
#pragma unroll
            for (int k = 0; k < EB; ++k)
                if (v[k]) stg[pos + o[k]] = (unsigned short)p[k];
        } else {
            int jv[EB];
#pragma unroll
            for (int k = 0; k < EB; ++k) jv[k] = jall[v[k] ? p[k] : 0];
#pragma unroll
            for (int k = 0; k < EB; ++k)
                if (v[k]) col[pos + o[k]] = jv[k];
        }
        pos += o[EB - 1] + (v[EB - 1] ? 1 : 0);
    }
    __syncwarp();
}

// BATCH: tiles of several systems (td.w = system); each tile reads its
// system's GridDev from gsys, g0 carries the shared status record and the
// length of the concatenated sorted arrays.  Otherwise g0 is the grid.
template <int DIM, bool BATCH, class C>
__global__ void __launch_bounds__(32 * C::WPB, C::WSM / C::WPB)
    k_nnps_tile(GridDev g0, const GridDev *__restrict__ gsys, const int4 *__restrict__ tiles,
                const long long *__restrict__ ntiles_dev, long long *__restrict__ row_ptr, int *__restrict__ col,
                long long cap, float *__restrict__ rho, unsigned long long *__restrict__ tstate, int stg_slots,
                int warp_bytes) {
    extern __shared__ __align__(16) unsigned char smraw[];
    // this warp's area: TileSmem, then its share of the extra staging
    TileSmem<C> &S = *reinterpret_cast<TileSmem<C> *>(smraw + (threadIdx.x >> 5) * warp_bytes);
    const int lane = threadIdx.x & 31;
    const bool want_rho = rho != nullptr;
    const long long ntiles = *ntiles_dev;
    unsigned int n32 = 0, n64 = 0;

    while (true) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&g0.status->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int4 td = tiles[t];
        const GridDev &g = BATCH ? gsys[td.w] : g0;
        const int ny = g.nk[1];
        // culling threshold: T plus a margin for the FP16 coordinates it uses
        const float cullT = __half2float(__hneg(__low2half(as_h2(g.neg_t16)))) + CULL_MARGIN;
        const int p0 = td.x, cnt_home = td.y, row = td.z;
        const int cy = row % ny, cz = row / ny;
        const bool mine = lane < cnt_home;
        Home h;
        h.i = p0 + lane;
        h.x = mine ? g.scell_x[h.i] : 0x3fffffff;

        int cnt = 0;
        float acc = 0.f;
        bool simple = true;
        int groups = 0, kept = 0;
        // ---- count pass (emits too when the tile is simple) ------------------
        for (int gs = 0; gs < cnt_home;) {
            const int xa = __shfl_sync(0xffffffffu, h.x, gs);
            const unsigned int over = __ballot_sync(0xffffffffu, lane >= gs && h.x > xa + SPANMAX - 1);
            const int ge = over ? __ffs(over) - 1 : cnt_home;
            const bool act = mine && lane >= gs && lane < ge;
            Group G;
            group_setup<DIM, C>(S, g, h, act, cy, cz, gs, ge, G);
            simple &= run_group<DIM, PASS_COUNT, C>(S, g, h, act, G, cullT, cnt, acc, nullptr, 0, n32, n64, kept, p0,
                                                 cnt_home, want_rho);
            ++groups;
            gs = ge;
        }
        simple &= groups == 1;
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
        // A simple tile whose row segment fits the staging area lays its
        // output out in shared memory before it needs its CSR offset, so the
        // wait on earlier tiles overlaps that work.
        const int *jl = S.jall;
        unsigned short *stg = reinterpret_cast<unsigned short *>(&S.code[0]);
        const bool staged = simple && col != nullptr && agg <= stg_slots;
        if (staged) emit_bits<C>(S, lane, mine ? (kept + 31) >> 5 : 0, rstart, stg, nullptr, nullptr);
        const long long pre =
            look_back_resolve(tstate, t, agg, &g0.status->flags, g0.spin_limit > 0 ? g0.spin_limit : LOOKBACK_SPIN_LIMIT);
        const bool wc = col != nullptr && pre + agg <= cap;
        if (col != nullptr && !wc && lane == 0) atomicOr(&g0.status->flags, ST_CAPACITY);
        if (mine) {
            row_ptr[h.i] = pre + rstart;
            if (want_rho) rho[h.i] = g.w_norm * (2.f / 3.f + acc * (1.f / 6.f));
        }
        if (t == ntiles - 1 && lane == 0) row_ptr[g0.n] = pre + agg;
        if (!wc) continue;
        if (staged) {
            // consecutive lanes on consecutive entries of the tile's segment
#pragma unroll 4
            for (int e = lane; e < agg; e += 32) col[pre + e] = jl[stg[e]];
            __syncwarp();
        } else if (simple) {
            // segment larger than the staging area: rows straight to col
            emit_bits<C>(S, lane, mine ? (kept + 31) >> 5 : 0, pre + rstart, nullptr, col, jl);
        } else {
            // emit pass: same decisions again, written straight to the rows
            int ecnt = 0;
            float dummy = 0.f;
            unsigned int e32 = 0, e64 = 0;
            for (int gs = 0; gs < cnt_home;) {
                const int xa = __shfl_sync(0xffffffffu, h.x, gs);
                const unsigned int over = __ballot_sync(0xffffffffu, lane >= gs && h.x > xa + SPANMAX - 1);
                const int ge = over ? __ffs(over) - 1 : cnt_home;
                const bool act = mine && lane >= gs && lane < ge;
                Group G;
                group_setup<DIM, C>(S, g, h, act, cy, cz, gs, ge, G);
                int kk;
                run_group<DIM, PASS_EMIT, C>(S, g, h, act, G, cullT, ecnt, dummy, col, pre + rstart, e32, e64, kk, p0,
                                          cnt_home, false);
                gs = ge;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n32 += __shfl_xor_sync(0xffffffffu, n32, o);
        n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    }
    if (lane == 0) {
        if (n32) atomicAdd(&g0.status->fp32_pairs, (unsigned long long)n32);
        if (n64) atomicAdd(&g0.status->fp64_pairs, (unsigned long long)n64);
    }
}

// Tiles of one row of cells: span-limited (row_tile_end) or plain runs of
// TW particles (span_limited false: the no-allocation path, whose fixed
// scratch is sized for n / TW + nrow tiles).  cs: the row's nx + 1 starts.
__device__ __forceinline__ int row_tile_count(const int *cs, int nx, bool span_limited) {
    if (!span_limited) return (cs[nx] - cs[0] + TW - 1) / TW;
    int count = 0, c = 0;
    for (int p = cs[0]; p < cs[nx]; ++count) p = row_tile_end(cs, nx, p, c);
    return count;
}

constexpr int ROWTILE_NT = 64;            // threads per block = most rows per chunk
constexpr int ROWTILE_SMEM_INTS = 8192;  // cell starts staged per chunk of rows (32 KB)

// Row tiles, counted (tcount != nullptr) or written (tiles at toff).  Each
// block takes chunks of whole rows whose cell starts fit in shared memory,
// copies them with coalesced loads, and one thread per row walks its row
// there; rows longer than the buffer are walked from global memory.
__global__ void __launch_bounds__(ROWTILE_NT) k_row_tiles(GridDev g, int *__restrict__ tcount,
                                                          const long long *__restrict__ toff,
                                                          int4 *__restrict__ tiles, bool span_limited) {
    __shared__ int cs_s[ROWTILE_SMEM_INTS];
    const long long nrow = (long long)g.nk[1] * g.nk[2];
    const int nx = g.nk[0];
    const bool staged = nx + 1 <= ROWTILE_SMEM_INTS;
    const int rpc = staged ? min(ROWTILE_NT, (ROWTILE_SMEM_INTS - 1) / nx) : ROWTILE_NT;  // rows per chunk
    for (long long r0 = (long long)blockIdx.x * rpc; r0 < nrow; r0 += (long long)gridDim.x * rpc) {
        const int rows = (int)min((long long)rpc, nrow - r0);
        const int *cs = g.cell_start + r0 * nx;
        if (staged) {
            __syncthreads();
            for (int k = threadIdx.x; k <= rows * nx; k += ROWTILE_NT) cs_s[k] = cs[k];
            __syncthreads();
            cs = cs_s;
        }
        if (threadIdx.x < rows) {
            const long long r = r0 + threadIdx.x;
            const int *row = cs + (long long)threadIdx.x * nx;
            if (tcount != nullptr) {
                tcount[r] = row_tile_count(row, nx, span_limited);
            } else {
                long long o = toff[r];
                int c = 0;
                for (int p = row[0]; p < row[nx];) {
                    const int e = span_limited ? row_tile_end(row, nx, p, c) : min(p + TW, row[nx]);
                    tiles[o++] = make_int4(p, e - p, (int)r, 0);
                    p = e;
                }
            }
        }
    }
}

// Row tiles in one launch: each block takes chunks of whole rows in ticket
// order (cstate[nchunks] is the ticket), counts their tiles with the rows'
// cell starts staged in shared memory, finds the chunk's first tile by a
// decoupled look-back over earlier chunks (cstate[chunk]), and writes the
// row offsets toff and the tiles.  cstate[0 .. nchunks] must be zero.
__global__ void __launch_bounds__(ROWTILE_NT) k_row_tiles_lb(GridDev g, long long *__restrict__ toff,
                                                             int4 *__restrict__ tiles, bool span_limited,
                                                             unsigned long long *__restrict__ cstate) {
    __shared__ int cs_s[ROWTILE_SMEM_INTS];
    __shared__ long long wsum[ROWTILE_NT / 32];
    __shared__ long long chunk_pre;
    __shared__ unsigned long long chunk_id;
    static_assert(ROWTILE_NT == 64, "two warps per block");
    const long long nrow = (long long)g.nk[1] * g.nk[2];
    const int nx = g.nk[0];
    const bool staged = nx + 1 <= ROWTILE_SMEM_INTS;
    const int rpc = staged ? min(ROWTILE_NT, (ROWTILE_SMEM_INTS - 1) / nx) : ROWTILE_NT;  // rows per chunk
    const long long nch = (nrow + rpc - 1) / rpc;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    while (true) {
        __syncthreads();  // the previous chunk is done with the shared buffers
        if (threadIdx.x == 0) chunk_id = atomicAdd(&cstate[nch], 1ull);
        __syncthreads();
        const long long ch = (long long)chunk_id;
        if (ch >= nch) break;
        const long long r0 = ch * rpc;
        const int rows = (int)min((long long)rpc, nrow - r0);
        const int *cs = g.cell_start + r0 * nx;
        if (staged) {
            for (int k = threadIdx.x; k <= rows * nx; k += ROWTILE_NT) cs_s[k] = cs[k];
            __syncthreads();
            cs = cs_s;
        }
        const int *row = cs + (long long)threadIdx.x * nx;
        const int cnt = threadIdx.x < rows ? row_tile_count(row, nx, span_limited) : 0;
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int up = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += up;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        const long long total = wsum[0] + wsum[1];
        const long long rex = (w > 0 ? wsum[0] : 0) + inc - cnt;  // the row's first tile within the chunk
        if (w == 0) {
            look_back_publish(cstate, ch, total);
            const long long pre = look_back_resolve(cstate, ch, total, &g.status->flags);
            if (lane == 0) chunk_pre = pre;
        }
        __syncthreads();
        const long long pre = chunk_pre;
        if (threadIdx.x < rows) {
            const long long r = r0 + threadIdx.x;
            long long o = pre + rex;
            toff[r] = o;
            int c = 0;
            for (int p = row[0]; p < row[nx];) {
                const int e = span_limited ? row_tile_end(row, nx, p, c) : min(p + TW, row[nx]);
                tiles[o++] = make_int4(p, e - p, (int)r, 0);
                p = e;
            }
        }
        if (ch == nch - 1 && threadIdx.x == 0) toff[nrow] = pre + total;
    }
}

// The staged output area (code, pw, the ring, spare, then the launch's extra
// dynamic shared memory) must be one contiguous range.
template <class C>
constexpr bool staging_contiguous() {
    using SM = TileSmem<C>;
    return offsetof(SM, pw) == offsetof(SM, code) + sizeof(SM::code) &&
           offsetof(SM, fxy) == offsetof(SM, pw) + sizeof(SM::pw) &&
           offsetof(SM, fz) == offsetof(SM, fxy) + sizeof(SM::fxy) &&
           offsetof(SM, spare) == offsetof(SM, fz) + sizeof(SM::fz) &&
           sizeof(SM) == offsetof(SM, spare) + sizeof(SM::spare) && sizeof(SM) % 16 == 0;
}
static_assert(staging_contiguous<TileSparse>() && staging_contiguous<TileDense>(), "staging layout");
// the largest launch (every warp with the most extra staging) stays within
// the 227 KB a CTA may opt into
template <class C>
constexpr bool fits_cta() { return (sizeof(TileSmem<C>) + TILE_MAX_EXTRA_SMEM) * C::WPB <= 232448; }
static_assert(fits_cta<TileSparse>() && fits_cta<TileDense>(), "shared memory per CTA");

template <class C>
cudaError_t launch_shape(const GridDev &g, const GridDev *gsys, const int4 *tiles, const long long *ntiles_dev,
                         long long ntiles_max, long long *row_ptr, int *col, long long cap, float *rho,
                         unsigned long long *tstate, int extra_smem, bool zeroed, int sm_count, int sm_percent,
                         cudaStream_t s) {
    using SM = TileSmem<C>;
    extra_smem = (extra_smem + 15) & ~15;  // keeps every warp's area 16-byte aligned
    const size_t warp_bytes = sizeof(SM) + (size_t)extra_smem;
    const size_t sb = warp_bytes * C::WPB;
    const bool batch = gsys != nullptr;
    const int ki = (g.dim == 2 ? 0 : 2) + (batch ? 1 : 0);
    auto kern = ki == 0 ? k_nnps_tile<2, false, C> : ki == 1 ? k_nnps_tile<2, true, C>
              : ki == 2 ? k_nnps_tile<3, false, C> : k_nnps_tile<3, true, C>;
    // The shared-memory limit is set once per kernel, to the largest launch
    // any option allows (launches from several threads then never see a
    // limit another thread lowered).
    static std::once_flag once[4];
    static cudaError_t once_err[4];
    std::call_once(once[ki], [&] {
        once_err[ki] = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)((sizeof(SM) + TILE_MAX_EXTRA_SMEM) * C::WPB));
    });
    if (once_err[ki] != cudaSuccess) return once_err[ki];
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * C::WPB, sb);
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)sm_count * per_sm;
    // a share below 100 % leaves resident slots for other streams' kernels
    // (the request server's small requests next to a large one)
    if (sm_percent > 0 && sm_percent < 100) blocks = (blocks * sm_percent + 99) / 100;
    if (blocks > (ntiles_max + C::WPB - 1) / C::WPB) blocks = (ntiles_max + C::WPB - 1) / C::WPB;
    if (blocks < 1) blocks = 1;
    if (!zeroed) {
        const cudaError_t e =
            cudaMemsetAsync(tstate, 0, (size_t)(ntiles_max > 0 ? ntiles_max : 1) * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    const int stg_slots = (int)((SM::staging_bytes() + (size_t)extra_smem) / 2);
    ProfScope ps(TAG_FUSED, s);
    note_launch(1);
    kern<<<(unsigned)blocks, 32 * C::WPB, sb, s>>>(g, gsys, tiles, ntiles_dev, row_ptr, col, cap, rho, tstate,
                                                    stg_slots, (int)warp_bytes);
    return cudaGetLastError();
}

}  // namespace

// Build the tile list of a binned grid.  tcount: int[nrow], toff: int64[nrow+1],
// tiles: int4[ntiles_max].  span_limited: tiles of at most TW particles within
// TILE_SPAN cells (ntiles_max = tiles_max(n, ncell, nrow)), else plain runs of
// TW particles of a row (ntiles_max = n / TW + nrow + 1: the bound the
// no-allocation search sizes its fixed scratch for).  cstate != nullptr: one
// launch with a look-back over chunks of rows (cstate: nrow + 1 zeroed
// entries; tcount and scan_tmp unused), else count, scan and write.
cudaError_t launch_tiles(const GridDev &g, bool span_limited, int *tcount, long long *toff, void *scan_tmp,
                         int4 *tiles, unsigned long long *cstate, int sm_count, cudaStream_t s) {
    const long long nrow = (long long)g.nk[1] * g.nk[2];
    ProfScope ps(TAG_SCAN, s);
    const int nx = g.nk[0];
    const long long rpc = nx + 1 <= ROWTILE_SMEM_INTS ? std::min<long long>(ROWTILE_NT, (ROWTILE_SMEM_INTS - 1) / nx)
                                                      : ROWTILE_NT;
    long long rb = (nrow + rpc - 1) / rpc;
    if (cstate != nullptr) {
        if (rb > (long long)sm_count * 4) rb = (long long)sm_count * 4;
        if (rb < 1) rb = 1;
        note_launch(1);
        k_row_tiles_lb<<<(unsigned)rb, ROWTILE_NT, 0, s>>>(g, toff, tiles, span_limited, cstate);
        return cudaGetLastError();
    }
    if (rb > (long long)sm_count * 16) rb = (long long)sm_count * 16;
    if (rb < 1) rb = 1;
    note_launch(2);
    k_row_tiles<<<(unsigned)rb, ROWTILE_NT, 0, s>>>(g, tcount, nullptr, nullptr, span_limited);
    cudaError_t e = exclusive_scan_i64(tcount, toff, nrow, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_row_tiles<<<(unsigned)rb, ROWTILE_NT, 0, s>>>(g, nullptr, toff, tiles, span_limited);
    return cudaGetLastError();
}

// ntiles_dev: device pointer to the tile count (the last entry of the row
// tile offsets); ntiles_max bounds it (sizes the look-back state, which the
// launch clears unless the caller already has: zeroed).
// gsys != nullptr: batch tiles (td.w = system), g then carries the status
// record and the total particle count.  v: shared-memory shape and extra
// dynamic shared memory (all of it staging area for the tile's output).
cudaError_t launch_nnps_tile(const GridDev &g, const GridDev *gsys, const int4 *tiles, const long long *ntiles_dev,
                             long long ntiles_max, long long *row_ptr, int *col, long long cap, float *rho,
                             unsigned long long *tstate, TileLaunch v, bool zeroed, int sm_count, cudaStream_t s) {
    if (v.extra < 0 || v.extra > TILE_MAX_EXTRA_SMEM || (v.shape != TILE_SPARSE && v.shape != TILE_DENSE))
        return cudaErrorInvalidValue;
    if (v.shape == TILE_DENSE)
        return launch_shape<TileDense>(g, gsys, tiles, ntiles_dev, ntiles_max, row_ptr, col, cap, rho, tstate,
                                       v.extra, zeroed, sm_count, v.sm_percent, s);
    return launch_shape<TileSparse>(g, gsys, tiles, ntiles_dev, ntiles_max, row_ptr, col, cap, rho, tstate, v.extra,
                                    zeroed, sm_count, v.sm_percent, s);
}

// Shape and staging for a grid whose rows hold about `nbr` neighbours on
// average.  The sparse shape (more resident warps) while a tile of 32 such
// rows, with 5% to spare, fits its output area: measured on lattices of 77
// to 89 neighbours per particle, tiles beyond it write their rows directly
// and the dense shape is faster once most do.  Extra staging only when a
// tile of 32 rows (with 15% to spare) needs more than 1.5 times the built-in
// area: measured on 1M and 8M particle sets, the occupancy it costs
// outweighs the coalesced output for the tiles just above the area.
TileLaunch tile_choose_grid(double last_nbr, long long n, long long ncell, int dim, double kh, double hc,
                            int tile_shape, int staging, int sm_percent) {
    // neighbours per particle: the last measured value, else the
    // uniform-density estimate (particles per cell x the search sphere's
    // volume in cells)
    double nbr = last_nbr;
    if (nbr <= 0) {
        const double ppc = (double)n / (double)(ncell > 0 ? ncell : 1), r = kh / hc;
        nbr = dim == 3 ? ppc * 4.18879 * r * r * r : ppc * 3.14159 * r * r;
    }
    TileLaunch tv = tile_choose(nbr, tile_shape);
    if (staging >= 0) tv.extra = staging;
    tv.sm_percent = sm_percent;
    return tv;
}

TileLaunch tile_choose(double nbr, int shape) {
    TileLaunch v;
    const double sparse_slots = (double)TileSmem<TileSparse>::staging_bytes() / 2.0;
    v.shape = shape >= 0 ? shape : (32.0 * nbr * 1.05 <= sparse_slots ? TILE_SPARSE : TILE_DENSE);
    const double have = (double)(v.shape == TILE_DENSE ? TileSmem<TileDense>::staging_bytes()
                                                        : TileSmem<TileSparse>::staging_bytes());
    const double want = 32.0 * nbr * 1.15 * 2.0;  // bytes of 16-bit slots
    v.extra = 0;
    if (want > 1.5 * have) {
        v.extra = (int)((want - have + 2047.0) / 2048.0) * 2048;
        if (v.extra > 16384) v.extra = 16384;
    }
    return v;
}

}  // namespace sph
