// Random batch list on the device: cell binning and the core/shell pair kernel.
//
// Sec. 2.3 (Eqs. 13-16) and Algorithm 2 of arXiv 2407.09315.
//  - Cells: the paper uses cubic cells of side r_c (its inner radius) to build a
//    stored neighbour list.  Here cells have side >= r_cut/div (div = 1 or 2),
//    atoms are counting-sorted by cell (stable by atom id, so every evaluation
//    is deterministic) and nothing per pair is stored: the core list and the
//    batch are rebuilt on the fly inside the pair kernel (Algorithm 2 steps 1-2
//    fused), so memory stays O(N) (Sec. 2.3's memory argument taken further).
//  - Membership is integer and exact: d = (int32)(u_j - u_i) per axis (minimum
//    image), D = sum d^2 in uint64; core D < Rc2, shell Rc2 <= D <= Rs2.
//  - Batch: the p shell members with the smallest 64-bit Philox priority keyed
//    by (i, j, step) (ties to the smaller id): a uniform p-subset without
//    replacement that does not depend on the order candidates are visited in.
//  - F_corr (Eq. 16): per-block FP64 sums of the short-range force, reduced in a
//    fixed order.
#include <math.h>

#include "rbmd_internal.cuh"

namespace rbmd {

__device__ __forceinline__ int cell_coord(uint32_t u, int nc)
{
    return (int)(((uint64_t)u * (uint64_t)nc) >> 32);
}

// ---------------------------------------------------------------- binning
__global__ void k_cell_count(const uint4 *__restrict__ u4, int64_t N, int nc,
                             int32_t *__restrict__ count, int32_t *__restrict__ cell_of,
                             int32_t *__restrict__ rank)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 A = u4[i];
    int64_t c = ((int64_t)cell_coord(A.x, nc) * nc + cell_coord(A.y, nc)) * nc + cell_coord(A.z, nc);
    cell_of[i] = (int32_t)c;
    rank[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan of the cell counts in three passes (tile sums, scan of tile sums,
// tile scans).  SCAN_TILE elements per block.
constexpr int SCAN_TILE = 1024;

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ tsum)
{
    __shared__ int32_t s[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int v = 0;
    for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x)
        if (base + k < n) v += in[base + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        tsum[blockIdx.x] = t;
    }
}

__global__ void k_scan_top(int32_t *__restrict__ tsum, int ntiles)
{
    // one block: exclusive scan in chunks of blockDim
    __shared__ int32_t s[1024];
    int carry = 0;
    for (int b = 0; b < ntiles; b += blockDim.x) {
        int k = b + threadIdx.x;
        int v = k < ntiles ? tsum[k] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (k < ntiles) tsum[k] = carry + s[threadIdx.x] - v;
        int tot = s[blockDim.x - 1];
        __syncthreads();
        carry += tot;
    }
}

__global__ void k_scan_final(const int32_t *__restrict__ in, int64_t n,
                             const int32_t *__restrict__ toff, int32_t *__restrict__ out)
{
    // blockDim = 1024, one element per thread
    __shared__ int32_t s[SCAN_TILE];
    int64_t k = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    int v = k < n ? in[k] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_TILE; o <<= 1) {
        int t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (k < n) out[k] = toff[blockIdx.x] + s[threadIdx.x] - v;
    if (k == n - 1) out[n] = toff[blockIdx.x] + s[threadIdx.x];
}

template <typename real>
__global__ void k_cell_scatter(const uint4 *__restrict__ u4, const double *__restrict__ q64,
                               const int32_t *__restrict__ type, int64_t N,
                               const int32_t *__restrict__ cell_of,
                               const int32_t *__restrict__ rank,
                               const int32_t *__restrict__ start, uint4 *__restrict__ spos,
                               real *__restrict__ sq, int32_t *__restrict__ stype)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 A = u4[i];
    int64_t dst = (int64_t)start[cell_of[i]] + rank[i];
    spos[dst] = make_uint4(A.x, A.y, A.z, (uint32_t)i);
    if constexpr (sizeof(real) == 4) sq[dst] = __uint_as_float(A.w);
    else sq[dst] = q64[i];
    stype[dst] = type[i];
}

// Atomic ranks make the order inside a cell arbitrary; restore atom-id order so
// that every later floating-point sum runs in a fixed order.
template <typename real>
__global__ void k_cell_order(const int32_t *__restrict__ start, int64_t ncell,
                             uint4 *__restrict__ spos, real *__restrict__ sq,
                             int32_t *__restrict__ stype)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], e = start[c + 1];
    for (int a = b + 1; a < e; ++a) {
        uint4 P = spos[a];
        real q = sq[a];
        int32_t t = stype[a];
        int k = a - 1;
        while (k >= b && spos[k].w > P.w) {
            spos[k + 1] = spos[k];
            sq[k + 1] = sq[k];
            stype[k + 1] = stype[k];
            --k;
        }
        spos[k + 1] = P;
        sq[k + 1] = q;
        stype[k + 1] = t;
    }
}

rbmd_status cells_build(rbmd_ctx *c)
{
    const int th = 256;
    const unsigned nb = (unsigned)((c->N + th - 1) / th);
    RBMD_CHECK_CUDA(cudaMemsetAsync(c->cell_count, 0, sizeof(int32_t) * c->ncell, c->stream));
    k_cell_count<<<nb, th, 0, c->stream>>>(c->u4, c->N, c->nc, c->cell_count, c->cell_of,
                                           c->cell_rank);
    RBMD_LAUNCH_CHECK();
    const int ntiles = (int)((c->ncell + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_tiles<<<ntiles, 256, 0, c->stream>>>(c->cell_count, c->ncell, c->scan_part);
    RBMD_LAUNCH_CHECK();
    k_scan_top<<<1, 1024, 0, c->stream>>>(c->scan_part, ntiles);
    RBMD_LAUNCH_CHECK();
    k_scan_final<<<ntiles, SCAN_TILE, 0, c->stream>>>(c->cell_count, c->ncell, c->scan_part,
                                                      c->cell_start);
    RBMD_LAUNCH_CHECK();
    const unsigned ncb = (unsigned)((c->ncell + th - 1) / th);
    if (c->fp64) {
        k_cell_scatter<double><<<nb, th, 0, c->stream>>>(c->u4, c->q64, c->type, c->N, c->cell_of,
                                                         c->cell_rank, c->cell_start, c->spos,
                                                         (double *)c->sq, c->stype);
        RBMD_LAUNCH_CHECK();
        k_cell_order<double><<<ncb, th, 0, c->stream>>>(c->cell_start, c->ncell, c->spos,
                                                        (double *)c->sq, c->stype);
    } else {
        k_cell_scatter<float><<<nb, th, 0, c->stream>>>(c->u4, nullptr, c->type, c->N, c->cell_of,
                                                        c->cell_rank, c->cell_start, c->spos,
                                                        (float *)c->sq, c->stype);
        RBMD_LAUNCH_CHECK();
        k_cell_order<float><<<ncb, th, 0, c->stream>>>(c->cell_start, c->ncell, c->spos,
                                                       (float *)c->sq, c->stype);
    }
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// ---------------------------------------------------------------- pair kernel
template <typename real> struct PairArgs {
    const uint4 *spos;
    const real *sq;
    const int32_t *stype;
    const int32_t *cell_start;
    const real *lj;  // [2T]: sqrt(eps_t), sigma_t / 2
    int64_t N;
    int nc, div, T, p, exact;
    uint64_t Rc2, Rs2;
    uint32_t Rlin;
    uint2 key;
    StepRef step;
    uint32_t tag;
    real ck, alpha, sqrt_alpha, c2, lscale;
    real *F;
    int accumulate;
    double *fpart;    // [gridDim][3]
    double *epart;    // [gridDim][2]
    int32_t *imax;    // [0] max N_s
    int32_t *n_core, *n_shell, *batch;
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float erfc_r(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_r(double x) { return erfc(x); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

// Force on i from j (d = r_j - r_i, minimum image) for erfc-Coulomb (Eq. 10) +
// Lennard-Jones (Eq. 2) with Lorentz-Berthelot parameters (Eq. 4); adds w * F_ij
// to f and, with ENERGY, w * u_ij to (ec, el).
template <typename real, bool ENERGY>
__device__ __forceinline__ void pair_eval(const PairArgs<real> &a, real dx, real dy, real dz,
                                          real qq, real eps, real sig, real w, real &fx,
                                          real &fy, real &fz, double &ec, double &el)
{
    const real r2 = dx * dx + dy * dy + dz * dz;
    const real rinv = rsqrt_r(r2);
    const real r = r2 * rinv;
    const real er = erfc_r(a.sqrt_alpha * r);
    const real ex = exp_r(-a.alpha * r2);
    const real gc = qq * (er * rinv + a.c2 * ex);  // r * (-dU_coul/dr)
    const real s2 = sig * sig * rinv * rinv;
    const real s6 = s2 * s2 * s2;
    const real s12 = s6 * s6;
    const real glj = (real)24 * eps * ((real)2 * s12 - s6);  // r * (-dU_lj/dr)
    const real g = w * (gc + glj) * rinv * rinv;
    fx -= g * dx;
    fy -= g * dy;
    fz -= g * dz;
    if constexpr (ENERGY) {
        ec += (double)(w * qq * er * rinv);
        el += (double)(w * (real)4 * eps * (s12 - s6));
    }
}

// Bottom-p selection over (priority, id), kept in registers: the slots are
// addressed with compile-time indices only (predicated), so no local memory.
template <int CAP> struct BottomP {
    uint64_t pri[CAP];
    int32_t k[CAP];
    int n;
    int mpos;  // slot of the current maximum (valid once n == p)

    __device__ __forceinline__ void init() { n = 0; mpos = 0; }

    __device__ __forceinline__ static bool greater(uint64_t pa, int ka, uint64_t pb, int kb,
                                                   const uint4 *spos)
    {
        if (pa != pb) return pa > pb;
        return spos[ka].w > spos[kb].w;  // equal priorities: larger id is "greater"
    }

    __device__ __forceinline__ void find_max(int p, const uint4 *spos)
    {
        uint64_t mp = pri[0];
        int mk = k[0], pos = 0;
#pragma unroll
        for (int e = 1; e < CAP; ++e) {
            if (e < p && greater(pri[e], k[e], mp, mk, spos)) {
                mp = pri[e];
                mk = k[e];
                pos = e;
            }
        }
        mpos = pos;
    }

    __device__ __forceinline__ void insert(uint64_t pr, int kk, int p, const uint4 *spos)
    {
        if (n < p) {
#pragma unroll
            for (int e = 0; e < CAP; ++e)
                if (e == n) { pri[e] = pr; k[e] = kk; }
            ++n;
            if (n == p) find_max(p, spos);
            return;
        }
        uint64_t mp = 0;
        int mk = 0;
#pragma unroll
        for (int e = 0; e < CAP; ++e)
            if (e == mpos) { mp = pri[e]; mk = k[e]; }
        if (!greater(mp, mk, pr, kk, spos)) return;
#pragma unroll
        for (int e = 0; e < CAP; ++e)
            if (e == mpos) { pri[e] = pr; k[e] = kk; }
        find_max(p, spos);
    }
};

template <typename real, int CAP, bool ENERGY, bool LISTS>
__global__ void __launch_bounds__(128) k_rbl_pair(PairArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *s_lj = reinterpret_cast<real *>(smem_raw);
    for (int t = threadIdx.x; t < 2 * a.T; t += blockDim.x) s_lj[t] = a.lj[t];
    __syncthreads();

    const int64_t is = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = is < a.N;
    real fx = 0, fy = 0, fz = 0;
    double ec = 0.0, el = 0.0;
    int ns = 0, ncore = 0;
    uint32_t id_i = 0;
    if (active) {
        const uint4 A = a.spos[is];
        id_i = A.w;
        const real qi = a.sq[is] * a.ck;
        const int ti = a.stype[is];
        const real se_i = s_lj[ti], hs_i = s_lj[a.T + ti];
        const int nc = a.nc, dv = a.div;
        const int cx = cell_coord(A.x, nc), cy = cell_coord(A.y, nc), cz = cell_coord(A.z, nc);
        const bool full = nc >= 2 * dv + 1;  // else every cell along an axis, once
        const int span = full ? 2 * dv + 1 : nc;
        const uint32_t step = (uint32_t)step_of(a.step);
        BottomP<CAP> heap;
        heap.init();
        real bx = 0, by = 0, bz = 0;
        double bec = 0.0, bel = 0.0;

        for (int ox = 0; ox < span; ++ox) {
            int gx = full ? cx - dv + ox : ox;
            gx += (gx < 0) ? nc : 0;
            gx -= (gx >= nc) ? nc : 0;
            for (int oy = 0; oy < span; ++oy) {
                int gy = full ? cy - dv + oy : oy;
                gy += (gy < 0) ? nc : 0;
                gy -= (gy >= nc) ? nc : 0;
                const int64_t row = ((int64_t)gx * nc + gy) * nc;
                // the z cells of this row as at most two contiguous atom ranges
                int r0b, r0e, r1b = 0, r1e = 0;
                if (!full) {
                    r0b = a.cell_start[row];
                    r0e = a.cell_start[row + nc];
                } else {
                    const int zlo = cz - dv, zhi = cz + dv;
                    if (zlo < 0) {
                        r0b = a.cell_start[row + zlo + nc];
                        r0e = a.cell_start[row + nc];
                        r1b = a.cell_start[row];
                        r1e = a.cell_start[row + zhi + 1];
                    } else if (zhi >= nc) {
                        r0b = a.cell_start[row + zlo];
                        r0e = a.cell_start[row + nc];
                        r1b = a.cell_start[row];
                        r1e = a.cell_start[row + zhi - nc + 1];
                    } else {
                        r0b = a.cell_start[row + zlo];
                        r0e = a.cell_start[row + zhi + 1];
                    }
                }
                for (int pass = 0; pass < 2; ++pass) {
                    const int kb = pass ? r1b : r0b, ke = pass ? r1e : r0e;
                    for (int k = kb; k < ke; ++k) {
                        if (k == is) continue;
                        const uint4 B = a.spos[k];
                        const int32_t dx = (int32_t)(B.x - A.x);
                        const int32_t dy = (int32_t)(B.y - A.y);
                        const int32_t dz = (int32_t)(B.z - A.z);
                        // |d| > Rlin on any axis: outside r_cut (unsigned wrap test)
                        if ((uint32_t)dx + a.Rlin > 2u * a.Rlin) continue;
                        if ((uint32_t)dy + a.Rlin > 2u * a.Rlin) continue;
                        if ((uint32_t)dz + a.Rlin > 2u * a.Rlin) continue;
                        const uint64_t D = (uint64_t)((int64_t)dx * dx) +
                                           (uint64_t)((int64_t)dy * dy) +
                                           (uint64_t)((int64_t)dz * dz);
                        if (D > a.Rs2) continue;
                        const bool core = D < a.Rc2;
                        if (core) ++ncore;
                        else ++ns;
                        if (core || a.exact) {
                            const int tj = a.stype[k];
                            pair_eval<real, ENERGY>(a, (real)dx * a.lscale, (real)dy * a.lscale,
                                                    (real)dz * a.lscale, qi * a.sq[k],
                                                    se_i * s_lj[tj], hs_i + s_lj[a.T + tj],
                                                    (real)1, fx, fy, fz, ec, el);
                        } else {
                            const uint4 w = philox10(make_uint4(id_i, B.w, step, a.tag), a.key);
                            heap.insert(((uint64_t)w.x << 32) | w.y, k, a.p, a.spos);
                        }
                    }
                }
            }
        }
        if (!a.exact) {
            const int nb = heap.n;
            const real wgt = ns > a.p ? (real)ns / (real)a.p : (real)1;
#pragma unroll
            for (int e = 0; e < CAP; ++e) {
                if (e < nb) {
                    const int k = heap.k[e];
                    const uint4 B = a.spos[k];
                    const int tj = a.stype[k];
                    pair_eval<real, ENERGY>(a, (real)(int32_t)(B.x - A.x) * a.lscale,
                                            (real)(int32_t)(B.y - A.y) * a.lscale,
                                            (real)(int32_t)(B.z - A.z) * a.lscale, qi * a.sq[k],
                                            se_i * s_lj[tj], hs_i + s_lj[a.T + tj], (real)1, bx,
                                            by, bz, bec, bel);
                }
            }
            fx += wgt * bx;
            fy += wgt * by;
            fz += wgt * bz;
            if constexpr (ENERGY) {
                ec += (double)wgt * bec;
                el += (double)wgt * bel;
            }
            if constexpr (LISTS) {
                int32_t ids[CAP];
#pragma unroll
                for (int e = 0; e < CAP; ++e) ids[e] = e < nb ? (int32_t)a.spos[heap.k[e]].w : INT32_MAX;
                for (int x = 1; x < nb; ++x) {  // insertion sort (verification path only)
                    int32_t v = ids[x];
                    int y = x - 1;
                    while (y >= 0 && ids[y] > v) { ids[y + 1] = ids[y]; --y; }
                    ids[y + 1] = v;
                }
                for (int e = 0; e < a.p; ++e)
                    a.batch[(int64_t)id_i * a.p + e] = (e < nb && e < CAP) ? ids[e] : -1;
            }
        }
        real *f = a.F + 3 * (int64_t)id_i;
        if (a.accumulate) {
            f[0] += fx;
            f[1] += fy;
            f[2] += fz;
        } else {
            f[0] = fx;
            f[1] = fy;
            f[2] = fz;
        }
        if constexpr (LISTS) {
            a.n_core[id_i] = ncore;
            a.n_shell[id_i] = ns;
            if (a.exact)
                for (int e = 0; e < a.p; ++e) a.batch[(int64_t)id_i * a.p + e] = -1;
        }
        if constexpr (ENERGY) atomicMax(a.imax, ns);
    }

    // block partial sums (fixed order) of F_short and of the energies
    double v[5] = {(double)fx, (double)fy, (double)fz, 0.5 * ec, 0.5 * el};
#pragma unroll
    for (int c = 0; c < 5; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    __shared__ double s_acc[5][32];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 5; ++c) s_acc[c][warp] = v[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double t[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w)
            for (int c = 0; c < 5; ++c) t[c] += s_acc[c][w];
        a.fpart[3 * (int64_t)blockIdx.x + 0] = t[0];
        a.fpart[3 * (int64_t)blockIdx.x + 1] = t[1];
        a.fpart[3 * (int64_t)blockIdx.x + 2] = t[2];
        if constexpr (ENERGY) {
            a.epart[2 * (int64_t)blockIdx.x + 0] = t[3];
            a.epart[2 * (int64_t)blockIdx.x + 1] = t[4];
        }
    }
}

template <typename real, int CAP>
static void launch_pair(const PairArgs<real> &a, int blocks, int threads, size_t smem,
                        cudaStream_t st, bool energy, bool lists)
{
    if (lists) {
        if (energy) k_rbl_pair<real, CAP, true, true><<<blocks, threads, smem, st>>>(a);
        else k_rbl_pair<real, CAP, false, true><<<blocks, threads, smem, st>>>(a);
    } else {
        if (energy) k_rbl_pair<real, CAP, true, false><<<blocks, threads, smem, st>>>(a);
        else k_rbl_pair<real, CAP, false, false><<<blocks, threads, smem, st>>>(a);
    }
}

template <typename real>
static rbmd_status rbl_pairs_t(rbmd_ctx *c, StepRef s, void *force, int accumulate, bool energy,
                               int32_t *n_core, int32_t *n_shell, int32_t *batch)
{
    PairArgs<real> a;
    a.spos = c->spos;
    a.sq = (const real *)c->sq;
    a.stype = c->stype;
    a.cell_start = c->cell_start;
    a.lj = c->fp64 ? (const real *)c->lj_d : (const real *)c->lj_f;
    a.N = c->N;
    a.nc = c->nc;
    a.div = c->div;
    a.T = c->T;
    a.p = c->prm.rbl_p;
    a.exact = (c->prm.flags & RBMD_RBL_EXACT) ? 1 : 0;
    a.Rc2 = c->Rc2;
    a.Rs2 = c->Rs2;
    a.Rlin = c->Rlin;
    a.key = make_uint2((uint32_t)(c->prm.seed & 0xFFFFFFFFu), (uint32_t)(c->prm.seed >> 32));
    a.step = s;
    a.tag = RBMD_STREAM_RBL | (c->prm.replica << 8);
    a.ck = (real)c->prm.coulomb_k;
    a.alpha = (real)c->prm.alpha;
    a.sqrt_alpha = (real)sqrt(c->prm.alpha);
    a.c2 = (real)(2.0 * sqrt(c->prm.alpha / kPi));
    a.lscale = (real)c->lscale;
    a.F = (real *)force;
    a.accumulate = accumulate;
    a.fpart = c->fpart;
    a.epart = c->epart;
    a.imax = c->ibuf;
    a.n_core = n_core;
    a.n_shell = n_shell;
    a.batch = batch;
    const bool lists = n_core != nullptr;
    const int threads = c->pair_block;
    const int blocks = c->pair_blocks;
    const size_t smem = sizeof(real) * 2 * c->T;
    const int p = c->prm.rbl_p;
    if (p <= 16) launch_pair<real, 16>(a, blocks, threads, smem, c->stream, energy, lists);
    else if (p <= 32) launch_pair<real, 32>(a, blocks, threads, smem, c->stream, energy, lists);
    else return RBMD_ERR_UNSUPPORTED;
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status rbl_pairs(rbmd_ctx *c, StepRef s, void *force, int accumulate, bool energy,
                      int32_t *n_core, int32_t *n_shell, int32_t *batch)
{
    if (c->fp64) return rbl_pairs_t<double>(c, s, force, accumulate, energy, n_core, n_shell, batch);
    return rbl_pairs_t<float>(c, s, force, accumulate, energy, n_core, n_shell, batch);
}

// ---------------------------------------------------------------- correction
template <typename real>
__global__ void k_add_corr(real *__restrict__ F, int64_t N, const double *__restrict__ fcorr)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    F[3 * i + 0] += (real)fcorr[0];
    F[3 * i + 1] += (real)fcorr[1];
    F[3 * i + 2] += (real)fcorr[2];
}

// F_corr = -(1/N) sum_i (F_core + F_shell*) (Eq. 16, Algorithm 2 step 3) into
// scal[slot..slot+2]; with apply, added to every atom of `force` (Algorithm 2
// step 4).  The integrator keeps its correction in SCAL_FCORR and adds it in the
// kicks instead of in a separate pass.
rbmd_status rbl_correction(rbmd_ctx *c, void *force, bool apply, int slot)
{
    RBMD_CHECK(md_sum(c, c->fpart, c->pair_blocks, 3, c->scal + slot, -1.0 / (double)c->N));
    if (apply) {
        const unsigned nb = (unsigned)((c->N + 255) / 256);
        if (c->fp64) k_add_corr<double><<<nb, 256, 0, c->stream>>>((double *)force, c->N, c->scal + slot);
        else k_add_corr<float><<<nb, 256, 0, c->stream>>>((float *)force, c->N, c->scal + slot);
        RBMD_LAUNCH_CHECK();
    }
    return RBMD_OK;
}

}  // namespace rbmd
