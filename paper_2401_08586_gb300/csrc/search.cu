// search.cu -- neighbour-search launchers: the general two-pass search
// (count pass, row scan, fill pass), the unfused density over an existing
// CSR, and the canonical-order assembly.  The per-cell search itself is in
// nnps_common.cuh; the single-pass fused search is in nnps_fused.cu.
#include <mutex>

#include "nnps_common.cuh"

namespace sph {

using namespace nn;

namespace {

constexpr int NT = 128;

template <int DIM, int PREC, int MODE>
__global__ void __launch_bounds__(NT) k_nnps(GridDev g, int *__restrict__ cnt_out,
                                            const long long *__restrict__ row_ptr, int *__restrict__ col,
                                            long long col_cap, float *__restrict__ rho) {
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemGen<PREC> &S = *reinterpret_cast<SmemGen<PREC> *>(smraw);
    bool write_col = false;
    if (MODE == MODE_FILL && col != nullptr) {
        write_col = row_ptr[g.n] <= col_cap;
        if (!write_col && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&g.status->flags, ST_CAPACITY);
    }
    unsigned int n32 = 0, n64 = 0;
    for (long long cell = blockIdx.x; cell < g.ncell; cell += gridDim.x)
        cell_general<DIM, PREC, MODE, NT>(S, g, cell, cnt_out, row_ptr, col, write_col, rho, n32, n64);
    if (MODE == MODE_FILL) {
        if (n32) atomicAdd(&g.status->fp32_pairs, (unsigned long long)n32);
        if (n64) atomicAdd(&g.status->fp64_pairs, (unsigned long long)n64);
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
            int cix, ciy, ciz;
            cell_decompose(g, ci, cix, ciy, ciz);
            float acc = g.w_self;
            for (long long q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
                const int sj = canonical ? rank[col[q]] : col[q];
                const int cj = scell[sj];
                int cjx, cjy, cjz;
                cell_decompose(g, cj, cjx, cjy, cjz);
                const float4 rj = g.rel32[sj];
                const float d0 = __fsub_rn(__fadd_rn(rj.x, 2.f * (float)(cjx - cix)), ri.x);
                const float d1 = __fsub_rn(__fadd_rn(rj.y, 2.f * (float)(cjy - ciy)), ri.y);
                const float d2 = __fsub_rn(__fadd_rn(rj.z, 2.f * (float)(cjz - ciz)), ri.z);
                const float r2 = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
                acc += g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
            }
            rho[r] = acc;
        } else {
            const double4_32a h = reinterpret_cast<const double4_32a *>(g.x64)[si];
            const double xi[3] = {h.x, h.y, h.z};
            double acc = g.w_self64;
            for (long long q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
                const int sj = canonical ? rank[col[q]] : col[q];
                const double4_32a x = reinterpret_cast<const double4_32a *>(g.x64)[sj];
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
    return sizeof(SmemGen<PREC>);
}

template <int DIM, int PREC, int MODE>
static cudaError_t launch_nnps_t(const GridDev &g, int *cnt, const long long *row_ptr, int *col,
                                 long long cap, float *rho, int sm_count, cudaStream_t s) {
    auto kern = k_nnps<DIM, PREC, MODE>;
    const size_t sb = smem_bytes<PREC>();
    static std::once_flag once;
    static cudaError_t once_err = cudaSuccess;
    std::call_once(once, [&] {
        once_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    });
    if (once_err != cudaSuccess) return once_err;
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
        e = segmented_sort_rows(col, rp, n, big_list, big_count, sm_count, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace sph
