// nnps.cu -- the neighbour search (NNPS) of arXiv 2401.08586 over the
// background-cell grid built by bin.cu, with the SPH density sum fused in.
//
// Definition searched for (all-list paragraph, Section "SPH method"): for each
// particle i, every j != i with r_ij^2 < kh^2.  As in the cell link-list
// (Fig. 3b) only the 3^d cells around i's cell are scanned.  In FP16-RCLL mode
// the pair distance comes from cell-relative coordinates (Eq. 7, read with the
// scale h_c/2 that inverts Eq. 6): in units of u = h_c/2,
//     D = (x_rel,j + 2 dc) - x_rel,i,     dc = cell(j) - cell(i) in {-1,0,1}^d.
//
// Work layout: one CTA (4 warps) per home cell.  The candidates of the cell
// (9 rows of 3 consecutive cells in 3D, 3 rows in 2D; each row is contiguous
// in the cell-sorted arrays) are staged in shared memory, pre-shifted by 2 dc
// and packed two per half2 (candidate p and p + 32 of each 64-wide chunk).
//
// Phase A (FP16 test): each warp owns chunks of 64 candidates held in
//   registers and loops over the home particles; per (home, chunk) it
//   evaluates e = dz^2 + dy^2 + dx^2 - T with three half2 FMAs and keeps the
//   candidates with e < tau16 ("maybe" pairs) as a 64-bit ballot mask.  tau16
//   bounds the FP16 rounding error, so every true neighbour is kept.
// Phase B (re-decision): the maybe pairs are expanded into a list (row-major,
//   candidates ascending) and each is re-decided in FP32 from the FP32
//   relative coordinates:  r2 < t32_in -> neighbour, r2 > t32_out -> not,
//   otherwise the FP64 expression of the definition decides (tier 3).  The
//   FP32 distance also gives the kernel value W (Eq. 3) for the density.
// Phase C (rows): one thread per home particle walks its row in order,
//   counting neighbours, summing the density in CSR order and (fill mode)
//   writing the column indices.
#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int NT = 128;
constexpr int NW = NT / 32;
constexpr int CAPC = 1024;          // candidates per window
constexpr int MAXCH = CAPC / 64;    // chunks per window
constexpr int HB = 32;              // home particles per batch
constexpr int PAIRCAP = 2048;       // maybe pairs per phase-B segment
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

struct SmemBase {
    int row_start[9], row_len[9], row_b0[9], row_b1[9], row_off[10];
    int row_dy[9], row_dz[9];
    int C;
    int hid[HB];
    int rcnt[HB];
    long long rbase[HB];
    long long rend[HB];
    uint2 M[HB * MAXCH];
    int ent_off[HB * MAXCH + 1];
    int wsum[NW];
    int pl[PAIRCAP];
    int cand_j[CAPC];
    unsigned char cand_sh[CAPC];
    unsigned int stat32, stat64;
};

template <int PREC>
struct Smem;

template <>
struct Smem<SPH_PREC_FP16_RCLL> : SmemBase {
    unsigned int hx[CAPC / 2], hy[CAPC / 2], hz[CAPC / 2];
    uint4 hq[HB];
    float4 h32[HB];
    float racc[HB];
    float pw[PAIRCAP];
};

template <>
struct Smem<SPH_PREC_FP64_CLL> : SmemBase {
    double cx[CAPC], cy[CAPC], cz[CAPC];
    double4 h64[HB];
    double racc[HB];
    double pw[PAIRCAP];
};

__device__ __forceinline__ __half2 as_h2(unsigned int u) {
    return *reinterpret_cast<__half2 *>(&u);
}

__device__ __forceinline__ unsigned int h2_bits(__half2 h) {
    return *reinterpret_cast<unsigned int *>(&h);
}

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

// Block-wide exclusive scan of one int per thread (NT threads).
__device__ __forceinline__ int block_excl_scan(int v, int *total, int *wsum) {
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

template <int DIM, int PREC, int MODE>
__global__ void __launch_bounds__(NT) k_nnps(GridDev g, int *__restrict__ cnt_out,
                                            const long long *__restrict__ row_ptr,
                                            int *__restrict__ col, long long col_cap,
                                            float *__restrict__ rho) {
    using W = typename WT<PREC>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<PREC> &S = *reinterpret_cast<Smem<PREC> *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NROWS = DIM == 3 ? 9 : 3;

    bool write_col = false;
    if (MODE == MODE_FILL && col != nullptr) {
        write_col = row_ptr[g.n] <= col_cap;
        if (!write_col && blockIdx.x == 0 && tid == 0) atomicOr(&g.status->flags, ST_CAPACITY);
    }
    const bool want_rho = MODE == MODE_FILL && rho != nullptr;
    if (tid == 0) {
        S.stat32 = 0;
        S.stat64 = 0;
    }

    const int nx = g.nk[0], ny = g.nk[1], nz = g.nk[2];
    for (long long cell = blockIdx.x; cell < g.ncell; cell += gridDim.x) {
        const int hs = g.cell_start[cell], he = g.cell_start[cell + 1];
        const int nh = he - hs;
        if (nh == 0) continue;
        const int cx = (int)(cell % nx);
        const long long t = cell / nx;
        const int cy = (int)(t % ny), cz = (int)(t / ny);

        __syncthreads();  // previous cell's shared-memory use is finished
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
                    auto &SS = S;
                    SS.hq[tid] = make_uint4(h2_bits(__low2half2(xy)), h2_bits(__high2half2(xy)),
                                            h2_bits(__low2half2(z0)), 0u);
                    SS.h32[tid] = g.rel32[i];
                    SS.racc[tid] = g.w_self;
                } else {
                    auto &SS = S;
                    SS.h64[tid] = reinterpret_cast<const double4 *>(g.x64)[i];
                    SS.racc[tid] = g.w_self64;
                }
            }

            for (int wb = 0; wb < C; wb += CAPC) {
                const int wc = min(CAPC, C - wb);
                const int nch = (wc + 63) >> 6;
                __syncthreads();
                // ---- stage candidates [wb, wb + wc) of this cell ----------
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
                            auto &SS = S;
                            uint2 q = g.rel16[j];
                            __half2 xy = __hadd2(as_h2(q.x), __floats2half2_rn(2.f * dxs, 2.f * dy));
                            __half zz = __hadd(__low2half(as_h2(q.y)), __float2half_rn(2.f * dz));
                            const int w = ((p >> 6) << 5) + (p & 31), hi = (p >> 5) & 1;
                            reinterpret_cast<__half *>(SS.hx)[2 * w + hi] = __low2half(xy);
                            reinterpret_cast<__half *>(SS.hy)[2 * w + hi] = __high2half(xy);
                            reinterpret_cast<__half *>(SS.hz)[2 * w + hi] = zz;
                        } else {
                            auto &SS = S;
                            double4 x = reinterpret_cast<const double4 *>(g.x64)[j];
                            SS.cx[p] = x.x;
                            SS.cy[p] = x.y;
                            SS.cz[p] = x.z;
                        }
                    } else {
                        S.cand_j[p] = -1;
                        S.cand_sh[p] = 0;
                        if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                            auto &SS = S;
                            const __half far = __float2half_rn(30000.f);
                            const int w = ((p >> 6) << 5) + (p & 31), hi = (p >> 5) & 1;
                            reinterpret_cast<__half *>(SS.hx)[2 * w + hi] = far;
                            reinterpret_cast<__half *>(SS.hy)[2 * w + hi] = far;
                            reinterpret_cast<__half *>(SS.hz)[2 * w + hi] = far;
                        } else {
                            auto &SS = S;
                            SS.cx[p] = 1e300;
                            SS.cy[p] = 1e300;
                            SS.cz[p] = 1e300;
                        }
                    }
                }
                __syncthreads();

                // ---- phase A: candidate tests --------------------------------
                for (int c = warp; c < nch; c += NW) {
                    if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                        auto &SS = S;
                        const __half2 X = as_h2(SS.hx[c * 32 + lane]);
                        const __half2 Y = as_h2(SS.hy[c * 32 + lane]);
                        const __half2 Z = as_h2(SS.hz[c * 32 + lane]);
                        const __half2 negT = as_h2(g.neg_t16), tau = as_h2(g.tau16);
                        for (int k = 0; k < nb; ++k) {
                            const uint4 q = SS.hq[k];
                            const __half2 dx = __hsub2(X, as_h2(q.x));
                            const __half2 dy = __hsub2(Y, as_h2(q.y));
                            __half2 e = __hfma2(dx, dx, negT);
                            e = __hfma2(dy, dy, e);
                            if (DIM == 3) {
                                const __half2 dz = __hsub2(Z, as_h2(q.z));
                                e = __hfma2(dz, dz, e);
                            }
                            const unsigned int m = __hlt2_mask(e, tau);
                            const unsigned int lo = __ballot_sync(0xffffffffu, (m & 0xffffu) != 0u);
                            const unsigned int hi = __ballot_sync(0xffffffffu, (m >> 16) != 0u);
                            if (lane == 0) S.M[k * MAXCH + c] = make_uint2(lo, hi);
                        }
                    } else {
                        auto &SS = S;
                        const int pa = c * 64 + lane, pb = pa + 32;
                        const double xa[3] = {SS.cx[pa], SS.cy[pa], SS.cz[pa]};
                        const double xb[3] = {SS.cx[pb], SS.cy[pb], SS.cz[pb]};
                        const int ja = S.cand_j[pa], jb = S.cand_j[pb];
                        for (int k = 0; k < nb; ++k) {
                            const double4 h = SS.h64[k];
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

                // ---- phase B: expand, re-decide, kernel values ---------------
                const int E = nb * nch;  // <= HB * MAXCH = NT * 4
                {
                    int v[4], sum = 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = tid * 4 + u;
                        int x = 0;
                        if (e < E) {
                            const uint2 m = S.M[(e / nch) * MAXCH + (e % nch)];
                            x = __popc(m.x) + __popc(m.y);
                        }
                        v[u] = x;
                        sum += x;
                    }
                    int tot;
                    int ex = block_excl_scan(sum, &tot, S.wsum);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = tid * 4 + u;
                        if (e < E) S.ent_off[e] = ex;
                        ex += v[u];
                    }
                    if (tid == 0) S.ent_off[E] = tot;
                }
                __syncthreads();

                int e0 = 0;
                while (e0 < E) {
                    // largest e1 with ent_off[e1] - ent_off[e0] <= PAIRCAP
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
                            // bit b of chunk c: lanes 0..31 hold p = 64c + lane (lo),
                            // 64c + 32 + lane (hi); the 64-bit mask orders them as p.
                            S.pl[pos++] = (c * 64 + b) | (k << 10);
                        }
                    }
                    __syncthreads();
                    for (int q = tid; q < P; q += NT) {
                        const int v = S.pl[q];
                        const int p = v & 1023, k = (v >> 10) & 31;
                        const int j = S.cand_j[p], i = S.hid[k];
                        bool in;
                        W w = 0;
                        if constexpr (PREC == SPH_PREC_FP16_RCLL) {
                            auto &SS = S;
                            in = false;
                            if (j != i) {
                                const unsigned int sh = S.cand_sh[p];
                                const float sx = 2.f * (float)((int)(sh & 3) - 1);
                                const float sy = 2.f * (float)((int)((sh >> 2) & 3) - 1);
                                const float sz = 2.f * (float)((int)((sh >> 4) & 3) - 1);
                                const float4 rj = g.rel32[j];
                                const float4 ri = SS.h32[k];
                                const float d0 = __fsub_rn(__fadd_rn(rj.x, sx), ri.x);
                                const float d1 = __fsub_rn(__fadd_rn(rj.y, sy), ri.y);
                                const float d2 = __fsub_rn(__fadd_rn(rj.z, sz), ri.z);
                                const float r2 =
                                    __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
                                if (r2 < g.t32_in) {
                                    in = true;
                                } else if (r2 > g.t32_out) {
                                    in = false;
                                    atomicAdd(&S.stat32, 1u);
                                } else {
                                    const int oi = g.orig_id[i], oj = g.orig_id[j];
                                    in = r2_fp64(DIM, g.xyz + (long long)oi * DIM,
                                                 g.xyz + (long long)oj * DIM) < g.kh2;
                                    atomicAdd(&S.stat64, 1u);
                                }
                                if (in && want_rho) w = g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
                            }
                        } else {
                            in = true;  // phase A was already the exact test
                            if (want_rho) {
                                auto &SS = S;
                                const double4 h = SS.h64[k];
                                const double xi[3] = {h.x, h.y, h.z};
                                const double xj[3] = {SS.cx[p], SS.cy[p], SS.cz[p]};
                                w = g.w_norm64 * w_poly64(sqrt(r2_fp64(DIM, xi, xj)) * g.r_scale64);
                            }
                        }
                        S.pw[q] = w;
                        if (in) S.pl[q] = v | IN_FLAG;
                    }
                    __syncthreads();
                    // ---- phase C: rows in order ------------------------------
                    if (tid < nb) {
                        const int k = tid;
                        const int ea = max(e0, k * nch), eb = min(e1, (k + 1) * nch);
                        if (ea < eb) {
                            const int qa = S.ent_off[ea] - base, qb = S.ent_off[eb] - base;
                            W *pw = S.pw;
                            W *racc = S.racc;
                            int cntk = S.rcnt[k];
                            W acc = racc[k];
                            const long long rb = MODE == MODE_FILL ? S.rbase[k] : 0;
                            const long long re = MODE == MODE_FILL ? S.rend[k] : 0;
                            for (int q = qa; q < qb; ++q) {
                                const int v = S.pl[q];
                                if (v < 0) {
                                    // the count pass fixed the row length; never write past it
                                    if (MODE == MODE_FILL && write_col && rb + cntk < re)
                                        col[rb + cntk] = S.cand_j[v & 1023];
                                    ++cntk;
                                    acc += pw[q];
                                }
                            }
                            S.rcnt[k] = cntk;
                            racc[k] = acc;
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
                    if (S.rcnt[tid] != (int)(row_ptr[i + 1] - row_ptr[i]))
                        atomicOr(&g.status->flags, ST_DEVICE_CHECK);
                    if (want_rho) {
                        rho[i] = (float)S.racc[tid];
                    }
                }
            }
        }  // home batches
    }      // cells

    __syncthreads();
    if (tid == 0 && MODE == MODE_FILL) {
        if (S.stat32) atomicAdd(&g.status->fp32_pairs, (unsigned long long)S.stat32);
        if (S.stat64) atomicAdd(&g.status->fp64_pairs, (unsigned long long)S.stat64);
    }
}

// Density over an existing CSR (unfused path), thread per row, CSR order.
// order_canonical: rows/cols are input indices (mapped through rank).
template <int DIM, int PREC>
__global__ void k_density(GridDev g, const int *__restrict__ rank, const int *__restrict__ scell,
                          const long long *__restrict__ row_ptr, const int *__restrict__ col,
                          int canonical, float *__restrict__ rho) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.n;
         r += (long long)gridDim.x * blockDim.x) {
        const int si = canonical ? rank[r] : (int)r;
        if constexpr (PREC == SPH_PREC_FP16_RCLL) {
            const float4 ri = g.rel32[si];
            const int ci = scell[si];
            const int cix = ci % g.nk[0], ciy = (ci / g.nk[0]) % g.nk[1], ciz = ci / (g.nk[0] * g.nk[1]);
            float acc = g.w_self;
            for (long long q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
                const int sj = canonical ? rank[col[q]] : col[q];
                const int cj = scell[sj];
                const int cjx = cj % g.nk[0], cjy = (cj / g.nk[0]) % g.nk[1], cjz = cj / (g.nk[0] * g.nk[1]);
                const float4 rj = g.rel32[sj];
                const float d0 = __fsub_rn(__fadd_rn(rj.x, 2.f * (float)(cjx - cix)), ri.x);
                const float d1 = __fsub_rn(__fadd_rn(rj.y, 2.f * (float)(cjy - ciy)), ri.y);
                const float d2 = __fsub_rn(__fadd_rn(rj.z, 2.f * (float)(cjz - ciz)), ri.z);
                const float r2 = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
                acc += g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
            }
            rho[r] = acc;
        } else {
            const double4 h = reinterpret_cast<const double4 *>(g.x64)[si];
            const double xi[3] = {h.x, h.y, h.z};
            double acc = g.w_self64;
            for (long long q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
                const int sj = canonical ? rank[col[q]] : col[q];
                const double4 x = reinterpret_cast<const double4 *>(g.x64)[sj];
                const double xj[3] = {x.x, x.y, x.z};
                acc += g.w_norm64 * w_poly64(sqrt(r2_fp64(DIM, xi, xj)) * g.r_scale64);
            }
            rho[r] = (float)acc;
        }
    }
}

// CELL-order CSR -> row lengths of the CANONICAL rows.
__global__ void k_canon_counts(int n, const int *__restrict__ rank, const long long *__restrict__ rp_cell,
                               int *__restrict__ cnt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = rank[i];
        cnt[i] = (int)(rp_cell[s + 1] - rp_cell[s]);
    }
}

// Copy each row to its canonical place, columns mapped to input indices
// (sorted afterwards), density permuted to input order.
__global__ void k_canon_copy(int n, const int *__restrict__ rank, const int *__restrict__ orig_id,
                             const long long *__restrict__ rp_cell, const int *__restrict__ col_cell,
                             const float *__restrict__ rho_cell, const long long *__restrict__ rp,
                             int *__restrict__ col, float *__restrict__ rho, int write_col) {
    const int lane = threadIdx.x & 31;
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < n; i += nw) {
        const int s = rank[i];
        const long long a = rp_cell[s], len = rp_cell[s + 1] - a, d = rp[i];
        if (write_col)
            for (long long k = lane; k < len; k += 32) col[d + k] = orig_id[col_cell[a + k]];
        if (rho != nullptr && lane == 0) rho[i] = rho_cell[s];
    }
}

}  // namespace

// ---- host-side launchers ---------------------------------------------------

template <int PREC>
static size_t smem_bytes() {
    return sizeof(Smem<PREC>);
}

template <int DIM, int PREC, int MODE>
static cudaError_t launch_nnps_t(const GridDev &g, int *cnt, const long long *row_ptr, int *col,
                                 long long cap, float *rho, int sm_count, cudaStream_t s) {
    auto kern = k_nnps<DIM, PREC, MODE>;
    const size_t sb = smem_bytes<PREC>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sb);
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > g.ncell) blocks = g.ncell;
    if (blocks < 1) blocks = 1;
    ProfScope ps(MODE == MODE_FILL ? TAG_FILL : TAG_COUNT, s);
    note_launch(1);
    kern<<<(unsigned)blocks, NT, sb, s>>>(g, cnt, row_ptr, col, cap, rho);
    return cudaGetLastError();
}

cudaError_t launch_nnps(const GridDev &g, int prec, int mode_fill, int *cnt, const long long *row_ptr,
                        int *col, long long cap, float *rho, int sm_count, cudaStream_t s) {
#define SPH_NNPS_CASE(D, P)                                                                       \
    if (g.dim == D && prec == P)                                                                  \
        return mode_fill ? launch_nnps_t<D, P, MODE_FILL>(g, cnt, row_ptr, col, cap, rho, sm_count, s) \
                         : launch_nnps_t<D, P, MODE_COUNT>(g, cnt, row_ptr, col, cap, rho, sm_count, s);
    SPH_NNPS_CASE(2, SPH_PREC_FP16_RCLL)
    SPH_NNPS_CASE(3, SPH_PREC_FP16_RCLL)
    SPH_NNPS_CASE(2, SPH_PREC_FP64_CLL)
    SPH_NNPS_CASE(3, SPH_PREC_FP64_CLL)
#undef SPH_NNPS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_density(const GridDev &g, int prec, const int *rank, const int *scell,
                           const long long *row_ptr, const int *col, int canonical, float *rho,
                           int sm_count, cudaStream_t s) {
    const int nt = 128;
    long long blocks = (g.n + nt - 1) / nt;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_DENSITY, s);
    note_launch(1);
    if (g.dim == 2 && prec == SPH_PREC_FP16_RCLL)
        k_density<2, SPH_PREC_FP16_RCLL><<<(unsigned)blocks, nt, 0, s>>>(g, rank, scell, row_ptr, col, canonical, rho);
    else if (g.dim == 3 && prec == SPH_PREC_FP16_RCLL)
        k_density<3, SPH_PREC_FP16_RCLL><<<(unsigned)blocks, nt, 0, s>>>(g, rank, scell, row_ptr, col, canonical, rho);
    else if (g.dim == 2)
        k_density<2, SPH_PREC_FP64_CLL><<<(unsigned)blocks, nt, 0, s>>>(g, rank, scell, row_ptr, col, canonical, rho);
    else
        k_density<3, SPH_PREC_FP64_CLL><<<(unsigned)blocks, nt, 0, s>>>(g, rank, scell, row_ptr, col, canonical, rho);
    return cudaGetLastError();
}

cudaError_t launch_canon(int n, const int *rank, const int *orig_id, const long long *rp_cell,
                         const int *col_cell, const float *rho_cell, int *cnt_tmp, void *scan_tmp,
                         long long *rp, int *col, float *rho, int *big_list, unsigned int *big_count,
                         int sm_count, cudaStream_t s) {
    const int nt = 256;
    long long blocks = (n + nt - 1) / nt;
    if (blocks > (long long)sm_count * 8) blocks = (long long)sm_count * 8;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_CANON, s);
    note_launch(col == nullptr && rho == nullptr ? 1 : 2);
    k_canon_counts<<<(unsigned)blocks, nt, 0, s>>>(n, rank, rp_cell, cnt_tmp);
    cudaError_t e = exclusive_scan_i64(cnt_tmp, rp, n, scan_tmp, s);
    if (e != cudaSuccess) return e;
    if (col == nullptr && rho == nullptr) return cudaGetLastError();
    long long wblocks = ((long long)n * 32 + nt - 1) / nt;
    if (wblocks > (long long)sm_count * 16) wblocks = (long long)sm_count * 16;
    if (wblocks < 1) wblocks = 1;
    k_canon_copy<<<(unsigned)wblocks, nt, 0, s>>>(n, rank, orig_id, rp_cell, col_cell, rho_cell, rp, col,
                                                   rho, col != nullptr);
    if (col != nullptr) {
        e = segmented_sort_rows(col, rp, n, big_list, big_count, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace sph
