// nnps_fused.cu -- single-pass FP16-RCLL neighbour search with the density sum
// fused in and the CSR row offsets found by a decoupled look-back across
// cells, so the candidate tests run once (no separate count pass).
//
// One CTA (8 warps) per home cell, cells taken in order from an atomic ticket.
// For a cell with at most 32 particles and 1024 candidates:
//   1. stage the candidates (9 x-rows of 3 cells in 3D, 3 in 2D; FP16,
//      pre-shifted by 2 dc into the home cell's frame) and the home particles;
//   2. FP16 test (Eq. 7 in cell-relative units): warps own 64-candidate chunks
//      and loop over the home particles, keeping "maybe" pairs (e < tau16) as
//      64-bit ballots per (home, chunk);
//   3. expand the kept pairs into a row-major list (8 threads per home row);
//   4. re-decide every kept pair in FP32 (FP64 definition inside the FP32 band)
//      and evaluate W (Eq. 3) from the FP32 distance;
//   5. per row: neighbour count and density (fixed summation order), then
//      compaction of the neighbours into a shared-memory staging buffer;
//   6. publish the cell's neighbour total, look back over earlier cells for its
//      CSR offset, and write row_ptr, rho and the staged columns (coalesced).
// Larger cells fall back to the general path (nnps_common.cuh): a counting
// sweep before the look-back and a writing sweep after it.
#include <mutex>

#include "nnps_common.cuh"

namespace sph {

using namespace nn;

namespace {

constexpr int NTF = 256;
constexpr int NWF = NTF / 32;
constexpr int CAPF = 1024;
constexpr int MAXCHF = CAPF / 64;
constexpr int PAIRF = 4096;
constexpr int PARTS = NTF / HB;  // threads per home row in steps 3 and 5

constexpr unsigned long long ST_AGG = 1ull << 62;
constexpr unsigned long long ST_INCL = 2ull << 62;
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;
constexpr int LOOKBACK_SPIN_LIMIT = 1 << 20;

struct FastSmem {
    int row_start[9], row_len[9], row_b0[9], row_b1[9], row_off[10];
    int row_dy[9], row_dz[9];
    int C;
    unsigned int hx[CAPF / 2], hy[CAPF / 2], hz[CAPF / 2];
    int cand_j[CAPF];
    unsigned char cand_sh[CAPF];
    uint4 hq[HB];
    float4 h32[HB];
    uint2 M[HB * MAXCHF];
    int part_off[NTF + 1];
    int out_off[NTF + 1];
    int pl[PAIRF];
    float pw[PAIRF];  // W of each kept pair; then the column staging
    float rrho[HB];
    int wsum[NWF];
    long long prefix;
    long long tile;
    int agg;
};

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Warp 0: publish this cell's total, find the sum over all earlier cells.
__device__ __forceinline__ long long look_back(unsigned long long *tstate, long long cell, int agg,
                                               unsigned int *flags) {
    const int lane = threadIdx.x & 31;
    long long excl = 0;
    if (cell == 0) {
        if (lane == 0) atomicExch(&tstate[0], ST_INCL | (unsigned long long)agg);
        return 0;
    }
    if (lane == 0) atomicExch(&tstate[cell], ST_AGG | (unsigned long long)agg);
    long long j = cell - 1;
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
    if (lane == 0) atomicExch(&tstate[cell], ST_INCL | (unsigned long long)(excl + agg));
    return excl;
}

template <int DIM>
__global__ void __launch_bounds__(NTF) k_nnps_fused(GridDev g, long long *__restrict__ row_ptr,
                                                   int *__restrict__ col, long long cap, float *__restrict__ rho,
                                                   unsigned long long *__restrict__ tstate, int *__restrict__ rowcnt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FastSmem &S = *reinterpret_cast<FastSmem *>(smraw);
    SmemGen<SPH_PREC_FP16_RCLL> &G = *reinterpret_cast<SmemGen<SPH_PREC_FP16_RCLL> *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = g.nk[0], ny = g.nk[1];
    unsigned int n32 = 0, n64 = 0;
    const bool want_rho = rho != nullptr;

    while (true) {
        __syncthreads();
        if (tid == 0) S.tile = (long long)atomicAdd(&g.status->ticket, 1ull);
        __syncthreads();
        const long long cell = S.tile;
        if (cell >= g.ncell) break;
        const int hs = g.cell_start[cell], he = g.cell_start[cell + 1];
        const int nh = he - hs;
        bool fast = false;
        if (nh > 0) {
            const int cx = (int)(cell % nx);
            const long long t = cell / nx;
            const int cy = (int)(t % ny), cz = (int)(t / ny);
            build_row_table<DIM>(S, g, cx, cy, cz);
            const int C = S.C;
            fast = nh <= HB && C <= CAPF;
            if (fast) {
                const int nch = (C + 63) >> 6;
                stage_candidates_fp16(S, g, 0, C, nch, NTF);
                if (tid < nh) {
                    const int i = hs + tid;
                    const uint2 q = g.rel16[i];
                    const __half2 xy = as_h2(q.x), z0 = as_h2(q.y);
                    S.hq[tid] = make_uint4(h2_bits(__low2half2(xy)), h2_bits(__high2half2(xy)),
                                           h2_bits(__low2half2(z0)), 0u);
                    S.h32[tid] = g.rel32[i];
                }
                __syncthreads();
                // ---- 2. FP16 tests ----------------------------------------
                for (int c = warp; c < nch; c += NWF) {
                    const unsigned int X = S.hx[c * 32 + lane], Y = S.hy[c * 32 + lane], Z = S.hz[c * 32 + lane];
                    for (int k = 0; k < nh; ++k) {
                        unsigned int lo, hi;
                        fp16_test_ballot<DIM>(X, Y, Z, S.hq[k], g.neg_t16, g.tau16, lo, hi);
                        if (lane == 0) S.M[k * MAXCHF + c] = make_uint2(lo, hi);
                    }
                }
                __syncthreads();
                // ---- 3. kept pairs -> row-major list ------------------------
                const int k = tid / PARTS, part = tid % PARTS;
                const int c0 = part * nch / PARTS, c1 = (part + 1) * nch / PARTS;
                int nb = 0;
                if (k < nh)
                    for (int c = c0; c < c1; ++c) {
                        const uint2 m = S.M[k * MAXCHF + c];
                        nb += __popc(m.x) + __popc(m.y);
                    }
                int P;
                const int poff = block_excl_scan<NTF>(nb, &P, S.wsum);
                S.part_off[tid] = poff;
                if (tid == 0) S.part_off[NTF] = P;
                fast = P <= PAIRF;  // block-uniform
                if (fast) {
                    int pos = poff;
                    if (k < nh)
                        for (int c = c0; c < c1; ++c) {
                            const uint2 m = S.M[k * MAXCHF + c];
                            unsigned long long bits = ((unsigned long long)m.y << 32) | m.x;
                            while (bits) {
                                const int b = __ffsll((long long)bits) - 1;
                                bits &= bits - 1;
                                S.pl[pos++] = (c * 64 + b) | (k << 10);
                            }
                        }
                    __syncthreads();
                    // ---- 4. FP32 re-decision + kernel values ----------------
                    for (int q = tid; q < P; q += NTF) {
                        const int v = S.pl[q];
                        const int p = v & 1023, kk = (v >> 10) & 31;
                        const int j = S.cand_j[p], i = hs + kk;
                        float w = 0.f;
                        int in = 0;
                        if (j != i) {
                            float sx, sy, sz, r2;
                            decode_shift(S.cand_sh[p], sx, sy, sz);
                            in = decide_fp32<DIM>(g, S.h32[kk], g.rel32[j], sx, sy, sz, i, j, &r2, n32, n64);
                            if (in && want_rho) w = g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
                        }
                        S.pw[q] = w;
                        if (in) S.pl[q] = v | IN_FLAG;
                    }
                    __syncthreads();
                    // ---- 5. rows: count + density, then compaction ----------
                    int cnt = 0;
                    float acc = 0.f;
                    const int qa = S.part_off[tid], qb = S.part_off[tid + 1];
                    for (int q = qa; q < qb; ++q)
                        if (S.pl[q] < 0) {
                            ++cnt;
                            acc += S.pw[q];
                        }
                    float racc = acc;
#pragma unroll
                    for (int o = 1; o < PARTS; o <<= 1) racc += __shfl_xor_sync(0xffffffffu, racc, o);
                    if (part == 0 && k < nh) S.rrho[k] = g.w_self + racc;
                    int A;
                    const int ooff = block_excl_scan<NTF>(cnt, &A, S.wsum);  // syncs: pw reads are done
                    S.out_off[tid] = ooff;
                    if (tid == 0) {
                        S.out_off[NTF] = A;
                        S.agg = A;
                    }
                    int *stg = reinterpret_cast<int *>(S.pw);
                    int o = ooff;
                    for (int q = qa; q < qb; ++q) {
                        const int v = S.pl[q];
                        if (v < 0) stg[o++] = S.cand_j[v & 1023];
                    }
                }
            }
            if (!fast) {
                __syncthreads();
                cell_general<DIM, SPH_PREC_FP16_RCLL, MODE_COUNT, NTF>(G, g, cell, rowcnt, nullptr, nullptr, false,
                                                                       nullptr, n32, n64);
                int s = 0;
                for (int i = hs + tid; i < he; i += NTF) s += rowcnt[i];
                int A;
                block_excl_scan<NTF>(s, &A, G.wsum);
                if (tid == 0) S.agg = A;
            }
        } else if (tid == 0) {
            S.agg = 0;
        }
        __syncthreads();
        const int agg = S.agg;
        // ---- 6. offsets across cells, write-out ------------------------------
        if (warp == 0) {
            const long long pre = look_back(tstate, cell, agg, &g.status->flags);
            if (lane == 0) S.prefix = pre;
        }
        __syncthreads();
        const long long prefix = S.prefix;
        const bool wc = col != nullptr && prefix + agg <= cap;
        if (col != nullptr && !wc && tid == 0) atomicOr(&g.status->flags, ST_CAPACITY);
        if (nh > 0) {
            if (fast) {
                if (tid < nh) {
                    row_ptr[hs + tid] = prefix + S.out_off[tid * PARTS];
                    if (want_rho) rho[hs + tid] = S.rrho[tid];
                }
                if (wc) {
                    const int *stg = reinterpret_cast<const int *>(S.pw);
                    for (int x = tid; x < agg; x += NTF) col[prefix + x] = stg[x];
                }
            } else {
                // rows of the cell: prefix + running sum of the counts
                long long run = prefix;
                for (int base = hs; base < he; base += NTF) {
                    const int i = base + tid;
                    const int c = i < he ? rowcnt[i] : 0;
                    int tot;
                    const int ex = block_excl_scan<NTF>(c, &tot, G.wsum);
                    if (i < he) row_ptr[i] = run + ex;
                    run += tot;
                }
                if (tid == 0) row_ptr[he] = prefix + agg;  // same value the next cell writes
                __syncthreads();
                cell_general<DIM, SPH_PREC_FP16_RCLL, MODE_FILL, NTF>(G, g, cell, nullptr, row_ptr, col, wc, rho,
                                                                      n32, n64);
            }
        }
        if (cell == g.ncell - 1 && tid == 0) row_ptr[g.n] = prefix + agg;
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

template <int DIM>
cudaError_t launch_fused_t(const GridDev &g, long long *row_ptr, int *col, long long cap, float *rho,
                           unsigned long long *tstate, int *rowcnt, int sm_count, cudaStream_t s) {
    auto kern = k_nnps_fused<DIM>;
    const size_t sb = sizeof(FastSmem) > sizeof(SmemGen<SPH_PREC_FP16_RCLL>) ? sizeof(FastSmem)
                                                                            : sizeof(SmemGen<SPH_PREC_FP16_RCLL>);
    static std::once_flag once;
    static cudaError_t once_err = cudaSuccess;
    std::call_once(once, [&] {
        once_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    });
    if (once_err != cudaSuccess) return once_err;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTF, sb);
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > g.ncell) blocks = g.ncell;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaMemsetAsync(tstate, 0, (size_t)g.ncell * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    ProfScope ps(TAG_FUSED, s);
    note_launch(1);
    kern<<<(unsigned)blocks, NTF, sb, s>>>(g, row_ptr, col, cap, rho, tstate, rowcnt);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_nnps_fused(const GridDev &g, long long *row_ptr, int *col, long long cap, float *rho,
                              unsigned long long *tstate, int *rowcnt, int sm_count, cudaStream_t s) {
    if (g.dim == 2) return launch_fused_t<2>(g, row_ptr, col, cap, rho, tstate, rowcnt, sm_count, s);
    return launch_fused_t<3>(g, row_ptr, col, cap, rho, tstate, rowcnt, sm_count, s);
}

}  // namespace sph
