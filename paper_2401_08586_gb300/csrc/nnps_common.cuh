// nnps_common.cuh -- pieces shared by the neighbour-search kernels: the
// kernel function of Eq. 3, the FP64 distance of the definition, block
// scans, and the general per-cell search used for cells of any size.
//
// Definition searched for (all-list paragraph, Section "SPH method" of
// arXiv 2401.08586): for each particle i, every j != i with r_ij^2 < kh^2;
// only the 3^d cells around i's cell are scanned (cell link-list, Fig. 3b).
// In FP16-RCLL mode the pair distance comes from cell-relative coordinates
// (Eq. 7, read with the scale h_c/2 that inverts Eq. 6); in units of
// u = h_c/2:  D = (x_rel,j + 2 dc) - x_rel,i,  dc = cell(j) - cell(i).
#pragma once

#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {
namespace nn {

constexpr int CAPC = 1024;        // candidates per window
constexpr int MAXCH = CAPC / 64;  // chunks per window
constexpr int HB = 32;            // home particles per batch
constexpr int PAIRCAP = 2048;     // maybe pairs per classification segment (general path)
constexpr int IN_FLAG = (int)0x80000000;

enum { MODE_COUNT = 0, MODE_FILL = 1 };

template <int PREC>
struct WT {
    using type = float;
};
template <>
struct WT<SPH_PREC_FP64_CLL> {
    using type = double;
};

// Shared memory of the general path.
struct SmemGenBase {
    int row_start[9], row_len[9], row_b0[9], row_b1[9], row_off[10];
    int row_dy[9], row_dz[9];
    int C;
    int hid[HB];
    int rcnt[HB];
    long long rbase[HB];
    long long rend[HB];
    uint2 M[HB * MAXCH];
    int ent_off[HB * MAXCH + 1];
    int wsum[32];
    int pl[PAIRCAP];
    int cand_j[CAPC];
    unsigned char cand_sh[CAPC];
};

template <int PREC>
struct SmemGen;

template <>
struct SmemGen<SPH_PREC_FP16_RCLL> : SmemGenBase {
    unsigned int hx[CAPC / 2], hy[CAPC / 2], hz[CAPC / 2];
    uint4 hq[HB];
    float4 h32[HB];
    float racc[HB];
    float pw[PAIRCAP];
};

template <>
struct SmemGen<SPH_PREC_FP64_CLL> : SmemGenBase {
    double cx[CAPC], cy[CAPC], cz[CAPC];
    double4_32a h64[HB];
    double racc[HB];
    double pw[PAIRCAP];
};

__device__ __forceinline__ __half2 as_h2(unsigned int u) { return *reinterpret_cast<__half2 *>(&u); }

__device__ __forceinline__ unsigned int h2_bits(__half2 h) { return *reinterpret_cast<unsigned int *>(&h); }

// P(R) of Eq. 3 without alpha_d: 2/3 - R^2 + R^3/2 (R < 1), (2 - R)^3 / 6 (R < 2).
__device__ __forceinline__ float w_poly(float R) {
    if (R < 1.f) return fmaf(R * R, fmaf(0.5f, R, -1.f), 2.f / 3.f);
    if (R < 2.f) {
        float t = 2.f - R;
        return t * t * t * (1.f / 6.f);
    }
    return 0.f;
}

__device__ __forceinline__ double w_poly64(double R) {
    if (R < 1.0) return 2.0 / 3.0 - R * R + 0.5 * R * R * R;
    if (R < 2.0) {
        double t = 2.0 - R;
        return t * t * t / 6.0;
    }
    return 0.0;
}

// FP64 squared distance exactly as the definition writes it (no contraction).
__device__ __forceinline__ double r2_fp64(int dim, const double *a, const double *b) {
    double d0 = __dsub_rn(a[0], b[0]);
    double d1 = __dsub_rn(a[1], b[1]);
    double r2 = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
    if (dim == 3) {
        double d2 = __dsub_rn(a[2], b[2]);
        r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
    }
    return r2;
}

// FP16 "maybe" test of two candidates (the halves of X, Y, Z) against one home
// particle q: ballots of e = ((dx^2 - T) + dy^2) + dz^2 < tau for the low and
// high halves.
template <int DIM>
__device__ __forceinline__ void fp16_test_ballot(unsigned int X, unsigned int Y, unsigned int Z, uint4 q,
                                                 unsigned int negT, unsigned int tau, unsigned int &lo,
                                                 unsigned int &hi) {
    const __half2 dx = __hsub2(as_h2(X), as_h2(q.x));
    const __half2 dy = __hsub2(as_h2(Y), as_h2(q.y));
    __half2 e = __hfma2(dx, dx, as_h2(negT));
    e = __hfma2(dy, dy, e);
    if (DIM == 3) {
        const __half2 dz = __hsub2(as_h2(Z), as_h2(q.z));
        e = __hfma2(dz, dz, e);
    }
    const unsigned int eb = h2_bits(e);
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.lt.f16x2 p|q, %2, %3;\n\t"
        "vote.sync.ballot.b32 %0, p, 0xffffffff;\n\t"
        "vote.sync.ballot.b32 %1, q, 0xffffffff;\n\t}"
        : "=r"(lo), "=r"(hi)
        : "r"(eb), "r"(tau));
}

// FP32 re-decision of a kept pair (tier 2) with the FP64 definition inside the
// band (tier 3).  ri, rj: FP32 relative coordinates; s*: 2 dc per axis.
// Returns 1 (neighbour) or 0; *r2o receives the FP32 squared distance in u^2.
template <int DIM>
__device__ __forceinline__ int decide_fp32(const GridDev &g, float4 ri, float4 rj, float sx, float sy, float sz,
                                           int i, int j, float *r2o, unsigned int &n32, unsigned int &n64) {
    const float d0 = __fsub_rn(__fadd_rn(rj.x, sx), ri.x);
    const float d1 = __fsub_rn(__fadd_rn(rj.y, sy), ri.y);
    const float d2 = __fsub_rn(__fadd_rn(rj.z, sz), ri.z);
    const float r2 = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
    *r2o = r2;
    if (r2 < g.t32_in) return 1;
    if (r2 > g.t32_out) {
        ++n32;
        return 0;
    }
    ++n64;
    const int oi = g.orig_id[i], oj = g.orig_id[j];
    return r2_fp64(DIM, g.xyz + (long long)oi * DIM, g.xyz + (long long)oj * DIM) < g.kh2 ? 1 : 0;
}

// Exclusive scan of one int per thread across a block of NT threads.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *total, int *wsum) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        int s = wsum[k];
        before += (k < w) ? s : 0;
        tot += s;
    }
    *total = tot;
    __syncthreads();
    return before + inc - v;
}

// Row table of a home cell: the 3^d neighbour cells as NROWS contiguous
// ranges of the cell-sorted arrays (x-rows of up to 3 cells), ascending.
template <int DIM, typename SM>
__device__ __forceinline__ void build_row_table(SM &S, const GridDev &g, int cx, int cy, int cz) {
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    const int nx = g.nk[0], ny = g.nk[1], nz = g.nk[2];
    const int tid = threadIdx.x;
    if (tid < 9) {
        const int r = tid;
        int dy = 0, dz = 0, start = 0, len = 0, b0 = 0, b1 = 0;
        if (r < NROWS) {
            dy = DIM == 3 ? (r % 3) - 1 : r - 1;
            dz = DIM == 3 ? (r / 3) - 1 : 0;
            const int yy = cy + dy, zz = cz + dz;
            if (yy >= 0 && yy < ny && zz >= 0 && zz < nz) {
                const long long base = ((long long)zz * ny + yy) * nx;
                const int x0 = max(cx - 1, 0), x1 = min(cx + 1, nx - 1);
                start = g.cell_start[base + x0];
                len = g.cell_start[base + x1 + 1] - start;
                b0 = g.cell_start[base + cx];
                b1 = g.cell_start[base + cx + 1];
            }
        }
        S.row_start[r] = start;
        S.row_len[r] = len;
        S.row_b0[r] = b0;
        S.row_b1[r] = b1;
        S.row_dy[r] = dy;
        S.row_dz[r] = dz;
    }
    __syncthreads();
    if (tid == 0) {
        int o = 0;
        for (int r = 0; r < 9; ++r) {
            S.row_off[r] = o;
            o += S.row_len[r];
        }
        S.row_off[9] = o;
        S.C = o;
    }
    __syncthreads();
}

// Stage the FP16 candidates [wb, wb + wc) of a home cell (row table in S):
// candidate index j, shift code (dc + 1 per axis, 2 bits each) and the
// coordinates pre-shifted by 2 dc, packed so that word (c, lane) of hx/hy/hz
// holds candidates 64c + lane (low half) and 64c + 32 + lane (high half).
// Slots up to nch * 64 past wc are padded with a far coordinate.
template <typename SM>
__device__ __forceinline__ void stage_candidates_fp16(SM &S, const GridDev &g, int wb, int wc, int nch, int nthr) {
    for (int p = threadIdx.x; p < nch * 64; p += nthr) {
        const int w = ((p >> 6) << 5) + (p & 31), hi = (p >> 5) & 1;
        __half hx, hy, hz;
        if (p < wc) {
            const int gp = wb + p;
            int r = 0;
#pragma unroll
            for (int k = 1; k < 9; ++k) r = (gp >= S.row_off[k]) ? k : r;
            const int j = S.row_start[r] + (gp - S.row_off[r]);
            const int dxs = j < S.row_b0[r] ? -1 : (j < S.row_b1[r] ? 0 : 1);
            const int dy = S.row_dy[r], dz = S.row_dz[r];
            S.cand_j[p] = j;
            S.cand_sh[p] = (unsigned char)((dxs + 1) | ((dy + 1) << 2) | ((dz + 1) << 4));
            const uint2 q = g.rel16[j];
            const __half2 xy = __hadd2(as_h2(q.x), __floats2half2_rn(2.f * dxs, 2.f * dy));
            hx = __low2half(xy);
            hy = __high2half(xy);
            hz = __hadd(__low2half(as_h2(q.y)), __float2half_rn(2.f * dz));
        } else {
            S.cand_j[p] = -1;
            S.cand_sh[p] = 0;
            hx = hy = hz = __float2half_rn(30000.f);
        }
        reinterpret_cast<__half *>(S.hx)[2 * w + hi] = hx;
        reinterpret_cast<__half *>(S.hy)[2 * w + hi] = hy;
        reinterpret_cast<__half *>(S.hz)[2 * w + hi] = hz;
    }
}

__device__ __forceinline__ void decode_shift(unsigned int sh, float &sx, float &sy, float &sz) {
    sx = 2.f * (float)((int)(sh & 3) - 1);
    sy = 2.f * (float)((int)((sh >> 2) & 3) - 1);
    sz = 2.f * (float)((int)((sh >> 4) & 3) - 1);
}

// General search of one home cell of any size: home particles in batches of
// HB, candidates in windows of CAPC, kept pairs re-decided in segments of
// PAIRCAP.  MODE_COUNT writes the row lengths to cnt_out[i]; MODE_FILL reads
// row_ptr and writes the columns (if write_col) and the density (if rho).
// Rows are walked in candidate order, so columns come out ascending and the
// density is summed in CSR order.  Must be called by all NT threads.
template <int DIM, int PREC, int MODE, int NT>
__device__ void cell_general(SmemGen<PREC> &S, const GridDev &g, long long cell, int *__restrict__ cnt_out,
                             const long long *__restrict__ row_ptr, int *__restrict__ col, bool write_col,
                             float *__restrict__ rho, unsigned int &n32, unsigned int &n64) {
    using W = typename WT<PREC>::type;
    constexpr int NW = NT / 32;
    constexpr int EPT = (HB * MAXCH + NT - 1) / NT;  // entries per thread in the entry scan
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool want_rho = MODE == MODE_FILL && rho != nullptr;
    const int nx = g.nk[0], ny = g.nk[1];
    const int hs = g.cell_start[cell], he = g.cell_start[cell + 1];
    const int nh = he - hs;
    if (nh == 0) return;
    const int cx = (int)(cell % nx);
    const long long t = cell / nx;
    const int cy = (int)(t % ny), cz = (int)(t / ny);

    __syncthreads();  // previous use of shared memory is finished
    build_row_table<DIM>(S, g, cx, cy, cz);
    const int C = S.C;

    for (int hb = 0; hb < nh; hb += HB) {
        const int nb = min(HB, nh - hb);
        __syncthreads();
        if (tid < nb) {
            const int i = hs + hb + tid;
            S.hid[tid] = i;
            S.rcnt[tid] = 0;
            if constexpr (MODE == MODE_FILL) {
                S.rbase[tid] = row_ptr[i];
                S.rend[tid] = row_ptr[i + 1];
            }
            if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                uint2 q = g.rel16[i];
                __half2 xy = as_h2(q.x), z0 = as_h2(q.y);
                S.hq[tid] = make_uint4(h2_bits(__low2half2(xy)), h2_bits(__high2half2(xy)), h2_bits(__low2half2(z0)), 0u);
                S.h32[tid] = g.rel32[i];
                S.racc[tid] = g.w_self;
            } else {
                S.h64[tid] = reinterpret_cast<const double4_32a *>(g.x64)[i];
                S.racc[tid] = g.w_self64;
            }
        }

        for (int wb = 0; wb < C; wb += CAPC) {
            const int wc = min(CAPC, C - wb);
            const int nch = (wc + 63) >> 6;
            __syncthreads();
            // ---- stage candidates [wb, wb + wc) --------------------------------
            for (int p = tid; p < nch * 64; p += NT) {
                if (p < wc) {
                    const int gp = wb + p;
                    int r = 0;
#pragma unroll
                    for (int k = 1; k < 9; ++k) r = (gp >= S.row_off[k]) ? k : r;
                    const int j = S.row_start[r] + (gp - S.row_off[r]);
                    const int dxs = j < S.row_b0[r] ? -1 : (j < S.row_b1[r] ? 0 : 1);
                    const int dy = S.row_dy[r], dz = S.row_dz[r];
                    S.cand_j[p] = j;
                    S.cand_sh[p] = (unsigned char)((dxs + 1) | ((dy + 1) << 2) | ((dz + 1) << 4));
                    if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                        uint2 q = g.rel16[j];
                        __half2 xy = __hadd2(as_h2(q.x), __floats2half2_rn(2.f * dxs, 2.f * dy));
                        __half zz = __hadd(__low2half(as_h2(q.y)), __float2half_rn(2.f * dz));
                        const int w = ((p >> 6) << 5) + (p & 31), hi = (p >> 5) & 1;
                        reinterpret_cast<__half *>(S.hx)[2 * w + hi] = __low2half(xy);
                        reinterpret_cast<__half *>(S.hy)[2 * w + hi] = __high2half(xy);
                        reinterpret_cast<__half *>(S.hz)[2 * w + hi] = zz;
                    } else {
                        double4_32a x = reinterpret_cast<const double4_32a *>(g.x64)[j];
                        S.cx[p] = x.x;
                        S.cy[p] = x.y;
                        S.cz[p] = x.z;
                    }
                } else {
                    S.cand_j[p] = -1;
                    S.cand_sh[p] = 0;
                    if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                        const __half far = __float2half_rn(30000.f);
                        const int w = ((p >> 6) << 5) + (p & 31), hi = (p >> 5) & 1;
                        reinterpret_cast<__half *>(S.hx)[2 * w + hi] = far;
                        reinterpret_cast<__half *>(S.hy)[2 * w + hi] = far;
                        reinterpret_cast<__half *>(S.hz)[2 * w + hi] = far;
                    } else {
                        S.cx[p] = 1e300;
                        S.cy[p] = 1e300;
                        S.cz[p] = 1e300;
                    }
                }
            }
            __syncthreads();

            // ---- candidate tests -------------------------------------------
            for (int c = warp; c < nch; c += NW) {
                if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                    const unsigned int X = S.hx[c * 32 + lane], Y = S.hy[c * 32 + lane], Z = S.hz[c * 32 + lane];
                    for (int k = 0; k < nb; ++k) {
                        unsigned int lo, hi;
                        fp16_test_ballot<DIM>(X, Y, Z, S.hq[k], g.neg_t16, g.tau16, lo, hi);
                        if (lane == 0) S.M[k * MAXCH + c] = make_uint2(lo, hi);
                    }
                } else {
                    const int pa = c * 64 + lane, pb = pa + 32;
                    const double xa[3] = {S.cx[pa], S.cy[pa], S.cz[pa]};
                    const double xb[3] = {S.cx[pb], S.cy[pb], S.cz[pb]};
                    const int ja = S.cand_j[pa], jb = S.cand_j[pb];
                    for (int k = 0; k < nb; ++k) {
                        const double4_32a h = S.h64[k];
                        const double xi[3] = {h.x, h.y, h.z};
                        const int i = S.hid[k];
                        const bool ina = ja != i && r2_fp64(DIM, xi, xa) < g.kh2;
                        const bool inb = jb != i && r2_fp64(DIM, xi, xb) < g.kh2;
                        const unsigned int lo = __ballot_sync(0xffffffffu, ina);
                        const unsigned int hi = __ballot_sync(0xffffffffu, inb);
                        if (lane == 0) S.M[k * MAXCH + c] = make_uint2(lo, hi);
                    }
                }
            }
            __syncthreads();

            // ---- expand, re-decide, kernel values ---------------------------
            const int E = nb * nch;
            {
                int v[EPT], sum = 0;
#pragma unroll
                for (int u = 0; u < EPT; ++u) {
                    const int e = tid * EPT + u;
                    int x = 0;
                    if (e < E) {
                        const uint2 m = S.M[(e / nch) * MAXCH + (e % nch)];
                        x = __popc(m.x) + __popc(m.y);
                    }
                    v[u] = x;
                    sum += x;
                }
                int tot;
                int ex = block_excl_scan<NT>(sum, &tot, S.wsum);
#pragma unroll
                for (int u = 0; u < EPT; ++u) {
                    const int e = tid * EPT + u;
                    if (e < E) S.ent_off[e] = ex;
                    ex += v[u];
                }
                if (tid == 0) S.ent_off[E] = tot;
            }
            __syncthreads();

            int e0 = 0;
            while (e0 < E) {
                const int base = S.ent_off[e0];
                int lo_e = e0 + 1, hi_e = E;
                while (lo_e < hi_e) {
                    const int mid = (lo_e + hi_e + 1) >> 1;
                    if (S.ent_off[mid] - base <= PAIRCAP) lo_e = mid;
                    else hi_e = mid - 1;
                }
                const int e1 = lo_e;
                const int P = S.ent_off[e1] - base;
                for (int e = e0 + tid; e < e1; e += NT) {
                    const int k = e / nch, c = e % nch;
                    const uint2 m = S.M[k * MAXCH + c];
                    unsigned long long bits = ((unsigned long long)m.y << 32) | m.x;
                    int pos = S.ent_off[e] - base;
                    while (bits) {
                        const int b = __ffsll((long long)bits) - 1;
                        bits &= bits - 1;
                        S.pl[pos++] = (c * 64 + b) | (k << 10);
                    }
                }
                __syncthreads();
                for (int q = tid; q < P; q += NT) {
                    const int v = S.pl[q];
                    const int p = v & 1023, k = (v >> 10) & 31;
                    const int j = S.cand_j[p], i = S.hid[k];
                    int in = 0;
                    W w = 0;
                    if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                        if (j != i) {
                            const unsigned int sh = S.cand_sh[p];
                            const float sx = 2.f * (float)((int)(sh & 3) - 1);
                            const float sy = 2.f * (float)((int)((sh >> 2) & 3) - 1);
                            const float sz = 2.f * (float)((int)((sh >> 4) & 3) - 1);
                            float r2;
                            in = decide_fp32<DIM>(g, S.h32[k], g.rel32[j], sx, sy, sz, i, j, &r2, n32, n64);
                            if (in && want_rho) w = g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
                        }
                    } else {
                        in = 1;  // the test was already the exact FP64 one
                        if (want_rho) {
                            const double4_32a h = S.h64[k];
                            const double xi[3] = {h.x, h.y, h.z};
                            const double xj[3] = {S.cx[p], S.cy[p], S.cz[p]};
                            w = g.w_norm64 * w_poly64(sqrt(r2_fp64(DIM, xi, xj)) * g.r_scale64);
                        }
                    }
                    S.pw[q] = w;
                    if (in) S.pl[q] = v | IN_FLAG;
                }
                __syncthreads();
                // rows in order
                if (tid < nb) {
                    const int k = tid;
                    const int ea = max(e0, k * nch), eb = min(e1, (k + 1) * nch);
                    if (ea < eb) {
                        const int qa = S.ent_off[ea] - base, qb = S.ent_off[eb] - base;
                        int cntk = S.rcnt[k];
                        W acc = S.racc[k];
                        const long long rb = MODE == MODE_FILL ? S.rbase[k] : 0;
                        const long long re = MODE == MODE_FILL ? S.rend[k] : 0;
                        for (int q = qa; q < qb; ++q) {
                            const int v = S.pl[q];
                            if (v < 0) {
                                // the count fixed the row length; never write past it
                                if (MODE == MODE_FILL && write_col && rb + cntk < re) col[rb + cntk] = S.cand_j[v & 1023];
                                ++cntk;
                                acc += S.pw[q];
                            }
                        }
                        S.rcnt[k] = cntk;
                        S.racc[k] = acc;
                    }
                }
                __syncthreads();
                e0 = e1;
            }
        }  // windows

        __syncthreads();
        if (tid < nb) {
            const int i = S.hid[tid];
            if constexpr (MODE == MODE_COUNT) {
                cnt_out[i] = S.rcnt[tid];
            } else {
                if (S.rcnt[tid] != (int)(row_ptr[i + 1] - row_ptr[i])) atomicOr(&g.status->flags, ST_DEVICE_CHECK);
                if (want_rho) rho[i] = (float)S.racc[tid];
            }
        }
    }  // home batches
    __syncthreads();
}

}  // namespace nn
}  // namespace sph
