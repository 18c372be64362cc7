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
#include <string.h>

#include <algorithm>

#include "rbmd_internal.cuh"

namespace rbmd {

// ---------------------------------------------------------------- binning
// cond (every kernel of the cell sort): when not NULL the kernel does nothing
// unless *cond is set (the integrator's conditional rebuild inside its graph).
__global__ void k_cell_count(const uint4 *__restrict__ u4, const int2 *__restrict__ map,
                             const Rep *__restrict__ reps, int32_t *__restrict__ count,
                             int32_t *__restrict__ cell_of, int32_t *__restrict__ rank,
                             const int32_t *__restrict__ cond = nullptr)
{
    if (cond && !*cond) return;
    const AtomSlot sl = atom_slot(map, reps);
    if (!sl.ok) return;
    const int64_t i = sl.i;
    const int nc = reps[sl.r].nc;
    const uint4 A = u4[i];
    // each replica owns its own range of cells, so the sorted order keeps the
    // replicas contiguous and in order
    const int64_t c = reps[sl.r].cell0 +
                      ((int64_t)cell_coord(A.x, nc) * nc + cell_coord(A.y, nc)) * nc +
                      cell_coord(A.z, nc);
    cell_of[i] = (int32_t)c;
    rank[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan of the cell counts in three passes (tile sums, scan of tile sums,
// tile scans).  SCAN_TILE elements per block.
constexpr int SCAN_TILE = 1024;

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ tsum,
                             const int32_t *__restrict__ cond = nullptr)
{
    if (cond && !*cond) return;
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

// Inclusive scan of v over the block (blockDim a multiple of 32, at most 1024):
// warp shuffles, then one warp scans the warp totals.  Returns the inclusive
// prefix; *total receives the block sum.
__device__ __forceinline__ int block_scan_incl(int v, int *total)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = (int)(blockDim.x >> 5);
        int y = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        ws[lane] = y;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? ws[w - 1] : 0);
    *total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();  // ws is reused by the next call
    return incl;
}

__global__ void k_scan_top(int32_t *__restrict__ tsum, int ntiles,
                           const int32_t *__restrict__ cond = nullptr)
{
    if (cond && !*cond) return;
    // one block: exclusive scan in chunks of blockDim
    int carry = 0;
    for (int b = 0; b < ntiles; b += blockDim.x) {
        const int k = b + threadIdx.x;
        const int v = k < ntiles ? tsum[k] : 0;
        int tot;
        const int incl = block_scan_incl(v, &tot);
        if (k < ntiles) tsum[k] = carry + incl - v;
        carry += tot;
    }
}

__global__ void k_scan_final(const int32_t *__restrict__ in, int64_t n,
                             const int32_t *__restrict__ toff, int32_t *__restrict__ out,
                             const int32_t *__restrict__ cond = nullptr)
{
    if (cond && !*cond) return;
    // blockDim = SCAN_TILE, one element per thread
    const int64_t k = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    const int v = k < n ? in[k] : 0;
    int tot;
    const int incl = block_scan_incl(v, &tot);
    if (k < n) out[k] = toff[blockIdx.x] + incl - v;
    if (k == n - 1) out[n] = toff[blockIdx.x] + incl;
}

template <typename real>
__global__ void k_cell_scatter(const uint4 *__restrict__ u4, const double *__restrict__ q64,
                               const int32_t *__restrict__ type, int64_t N,
                               const int32_t *__restrict__ cell_of,
                               const int32_t *__restrict__ rank,
                               const int32_t *__restrict__ start, uint4 *__restrict__ spos,
                               real *__restrict__ sq, int32_t *__restrict__ stype,
                               const int32_t *__restrict__ cond = nullptr)
{
    if (cond && !*cond) return;
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
// Then record the sorted index of every atom (sidx[id] = position in spos).
template <typename real>
__global__ void k_cell_order(const int32_t *__restrict__ start, int64_t ncell,
                             uint4 *__restrict__ spos, real *__restrict__ sq,
                             int32_t *__restrict__ stype, int32_t *__restrict__ sidx,
                             const int32_t *__restrict__ cond = nullptr)
{
    if (cond && !*cond) return;
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
    for (int a = b; a < e; ++a) sidx[spos[a].w] = a;
}

// Zeroes n counts when *cond is set (the conditional rebuild's memset).
__global__ void k_vl_zero(int32_t *__restrict__ v, int64_t n, const int32_t *__restrict__ cond)
{
    if (!*cond) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = 0;
}

// Cell counts, cells and ranks of the atoms of the 256-atom blocks [b0, b1) of
// map256 (the counts zeroed beforehand); cells_build(c, true) then completes the sort.
rbmd_status cells_count_blocks(rbmd_ctx *c, int b0, int b1)
{
    if (b1 <= b0) return RBMD_OK;
    k_cell_count<<<(unsigned)(b1 - b0), 256, 0, c->stream>>>(c->u4, c->map256 + b0, c->reps,
                                                             c->cell_count, c->cell_of, c->cell_rank);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// The counting sort of the atoms by cell.  cond == NULL: now (the caller's
// sorted layout replaces the step's candidate lists, which are then rebuilt before
// the next step); else every kernel checks *cond on the device.
static rbmd_status cells_sort(rbmd_ctx *c, bool counted, const int32_t *cond)
{
    c->lists_cached = false;
    const int th = 256;
    const unsigned nb = (unsigned)((c->N + th - 1) / th);
    if (!counted) {
        if (cond) {
            k_vl_zero<<<(unsigned)((c->ncell + 255) / 256), 256, 0, c->stream>>>(c->cell_count,
                                                                                c->ncell, cond);
        } else {
            RBMD_CHECK_CUDA(cudaMemsetAsync(c->cell_count, 0, sizeof(int32_t) * c->ncell, c->stream));
        }
        k_cell_count<<<c->nb256, 256, 0, c->stream>>>(c->u4, c->map256, c->reps, c->cell_count,
                                                       c->cell_of, c->cell_rank, cond);
        RBMD_LAUNCH_CHECK();
    }
    const int ntiles = (int)((c->ncell + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_tiles<<<ntiles, 256, 0, c->stream>>>(c->cell_count, c->ncell, c->scan_part, cond);
    RBMD_LAUNCH_CHECK();
    k_scan_top<<<1, 1024, 0, c->stream>>>(c->scan_part, ntiles, cond);
    RBMD_LAUNCH_CHECK();
    k_scan_final<<<ntiles, SCAN_TILE, 0, c->stream>>>(c->cell_count, c->ncell, c->scan_part,
                                                      c->cell_start, cond);
    RBMD_LAUNCH_CHECK();
    const unsigned ncb = (unsigned)((c->ncell + th - 1) / th);
    if (c->fp64) {
        k_cell_scatter<double><<<nb, th, 0, c->stream>>>(c->u4, c->q64, c->type, c->N, c->cell_of,
                                                         c->cell_rank, c->cell_start, c->spos,
                                                         (double *)c->sq, c->stype, cond);
        RBMD_LAUNCH_CHECK();
        k_cell_order<double><<<ncb, th, 0, c->stream>>>(c->cell_start, c->ncell, c->spos,
                                                        (double *)c->sq, c->stype, c->cell_rank,
                                                        cond);
    } else {
        k_cell_scatter<float><<<nb, th, 0, c->stream>>>(c->u4, nullptr, c->type, c->N, c->cell_of,
                                                        c->cell_rank, c->cell_start, c->spos,
                                                        (float *)c->sq, c->stype, cond);
        RBMD_LAUNCH_CHECK();
        k_cell_order<float><<<ncb, th, 0, c->stream>>>(c->cell_start, c->ncell, c->spos,
                                                       (float *)c->sq, c->stype, c->cell_rank, cond);
    }
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status cells_build(rbmd_ctx *c, bool counted)
{
    c->vl_dirty = true;
    return cells_sort(c, counted, nullptr);
}

// ---------------------------------------------------------------- pair kernels
//
// Algorithm 2 runs as three kernels with one thread per cell-sorted atom, so that
// each stays small and runs at high occupancy (the short-range step is bound by
// memory latency and dependent integer chains, not by arithmetic throughput):
//   k_rbl_scan    step 1: classify every candidate of the neighbour cells and
//                 store the core list (sorted indices) and the shell list (atom
//                 ids), capacity CC and CS per atom; the counts are exact even
//                 when a list is full;
//   k_rbl_select  step 1: Philox priorities of the shell members and the
//                 bottom-p batch (sorted indices);
//   k_rbl_force   step 2: core forces plus the batch forces weighted N_s/p, and
//                 per-warp FP64 partial sums for F_corr (step 3).
// An atom whose lists overflowed is skipped by select and force and handled
// exactly by k_rbl_fused, which recomputes its neighbourhood on its own (it does
// nothing, apart from zeroing its partial sums, when no list overflowed).
template <typename real> struct PairArgs {
    const uint4 *spos;
    const real *sq;
    const int32_t *stype;
    const int32_t *cell_start;
    const real *lj;  // [2T]: sqrt(eps_t), sigma_t / 2
    const Rep *reps;   // per-replica constants (box, cells, radii, Philox key and tag)
    const int2 *map;   // replica-aligned block map of the launch
    int nmap;          // entries of map (blocks of the fallback's grid-stride loop)
    int64_t N;         // all replicas
    int div, T, p, exact;
    StepRef step;
    real ck, alpha, sqrt_alpha, c2;
    const void *tab;   // pair look-up table (pairtab.cu layout, real4 [2 n]) or NULL
    int tab_n, tab_i0;
    real tab_inv_h;
    real *F;
    int accumulate;
    long long *fpart;  // [parts][3]: pair kernel per warp, then the fallback per warp (2^-32)
    double *epart;     // [parts][EPART]
    int64_t fb_part0;  // first partial slot of the fallback kernel
    int32_t *imax;     // [0] max N_s
    int32_t *n_core, *n_shell, *batch;  // verification outputs (caller order) or NULL
    // per-atom lists; entry e of sorted atom i is at lidx(i, e, N, capacity)
    int32_t *lcore;    // [N][CC] sorted indices of the core members
    int32_t *lshell;   // [N][CS] replica-local atom ids of the shell members
    int2 *ncount;      // [N] (|C|, N_s)
    int32_t *bk;       // [N][p] sorted indices of the batch
    const int32_t *sidx;  // [N] sorted index of every atom (by global id)
    int sel_exact;        // every selection by select_exact (RBMD_SELECT_EXACT, tests)
    int sel_key_bits;     // 1..31: priority bits kept in the fast keys (RBMD_SELECT_KEY_BITS, tests)
    int2 *heavy;          // [N] (sorted index, replica) of atoms with N_s > p (p > 10)
    int32_t *heavy_n;     // [1] their count
    int32_t *ovf;      // [0] set when any list overflowed
    int CC, CS;
    int stale;         // the cells are those of the last rebuild of the step's candidate
                       // lists (atoms have moved since): cull at r_cut + skin
    const uint32_t *gid;  // [N] global ids of a slab context's rows (Philox counters and
                          // ties), NULL: the replica-local id
    int *err;             // device error word (bounds-checked builds report through it)
};

// Id of replica-local atom `id` (replica starting at row id0) in the random draws.
template <typename real>
__device__ __forceinline__ uint32_t pid(const PairArgs<real> &a, uint32_t id0, uint32_t id)
{
    return a.gid ? a.gid[id0 + id] : id;
}

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float erfc_r(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_r(double x) { return erfc(x); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

// Energy and virial accumulators of one atom's pairs (ENERGY kernels only): the
// pair energies in FP64, and in the working precision the traces r.(-dU/dr) of
// the erfc-Coulomb and LJ virials and the tensor g d (x) d of both (d = r_j - r_i,
// the pair force on i is -g d, so r_ij (x) F_ij = g d (x) d; xx yy zz xy xz yz).
// The virial is W = -dE/d(strain) of the list energy with its weights held fixed.
// A thread's sums over its pairs (a few tens) in the working precision; the warp
// and global sums of the energies and virials are taken on from there (FP64
// across warps).
template <typename real> struct EAcc {
    real ec, el;
    real wc, wl;
    real w[6];
};

template <typename real>
__device__ __forceinline__ void eacc_zero(EAcc<real> &e)
{
    e.ec = 0;
    e.el = 0;
    e.wc = 0;
    e.wl = 0;
#pragma unroll
    for (int c = 0; c < 6; ++c) e.w[c] = 0;
}

// e += s b (the batch part with its weight N_s/p)
template <typename real>
__device__ __forceinline__ void eacc_add(EAcc<real> &e, const EAcc<real> &b, real s)
{
    e.ec += s * b.ec;
    e.el += s * b.el;
    e.wc += s * b.wc;
    e.wl += s * b.wl;
#pragma unroll
    for (int c = 0; c < 6; ++c) e.w[c] += s * b.w[c];
}

// Force on i from j (d = r_j - r_i, minimum image) for erfc-Coulomb (Eq. 10) +
// Lennard-Jones (Eq. 2) with Lorentz-Berthelot parameters (Eq. 4); adds F_ij to
// f and, with ENERGY, u_ij and the pair virial to e.
template <typename real> struct Real4;
template <> struct Real4<float> { using type = float4; };
template <> struct Real4<double> { using type = double4_32a; };

template <typename real, bool ENERGY, bool TAB>
__device__ __forceinline__ void pair_eval(const PairArgs<real> &a, real dx, real dy, real dz,
                                          real qq, real eps, real sig, real &fx, real &fy,
                                          real &fz, EAcc<real> &e)
{
    const real r2 = dx * dx + dy * dy + dz * dz;
    const real rinv = rsqrt_r(r2);
    const real s2 = sig * sig * rinv * rinv;
    const real s6 = s2 * s2 * s2;
    const real s12 = s6 * s6;
    const real glj = (real)24 * eps * ((real)2 * s12 - s6);  // r * (-dU_lj/dr)
    real g, eu = 0, gcr = 0;  // gcr: r * (-dU_coul/dr)
    if constexpr (TAB) {
        // cubic piece of the tabulated factors at s = r^2; below the knot i0 the
        // pieces hold the remainders and the bare Coulomb terms are added exactly
        const real u = r2 * a.tab_inv_h;
        const int k = min((int)u, a.tab_n - 1);
        const real t = u - (real)k;
        const typename Real4<real>::type *T = static_cast<const typename Real4<real>::type *>(a.tab);
        const typename Real4<real>::type cf = T[2 * k];
        real fc = ((cf.w * t + cf.z) * t + cf.y) * t + cf.x;
        if (k < a.tab_i0) fc += rinv * rinv * rinv;
        g = qq * fc + glj * rinv * rinv;
        if constexpr (ENERGY) {
            const typename Real4<real>::type ce = T[2 * k + 1];
            eu = ((ce.w * t + ce.z) * t + ce.y) * t + ce.x;
            if (k < a.tab_i0) eu += rinv;
            gcr = qq * fc * r2;
        }
    } else {
        const real r = r2 * rinv;
        const real er = erfc_r(a.sqrt_alpha * r);
        const real ex = exp_r(-a.alpha * r2);
        const real gc = qq * (er * rinv + a.c2 * ex);  // r * (-dU_coul/dr)
        g = (gc + glj) * rinv * rinv;
        eu = er * rinv;
        gcr = gc;
    }
    fx -= g * dx;
    fy -= g * dy;
    fz -= g * dz;
    if constexpr (ENERGY) {
        e.ec += qq * eu;
        e.el += (real)4 * eps * (s12 - s6);
        e.wc += gcr;
        e.wl += glj;
        e.w[0] += g * dx * dx;
        e.w[1] += g * dy * dy;
        e.w[2] += g * dz * dz;
        e.w[3] += g * dx * dy;
        e.w[4] += g * dx * dz;
        e.w[5] += g * dy * dz;
    }
}

// Per-atom context for pair evaluations.
template <typename real> struct AtomI {
    uint4 A;
    real qi, se, hs, lscale;
};

template <typename real, bool ENERGY, bool TAB = false>
__device__ __forceinline__ void eval_k(const PairArgs<real> &a, const real *s_lj,
                                       const AtomI<real> &I, int k, real &fx, real &fy, real &fz,
                                       EAcc<real> &e)
{
    k = (int)RBMD_IDX(k, a.N, a.err);
    const uint4 B = a.spos[k];
    const int tj = a.stype[k];
    pair_eval<real, ENERGY, TAB>(a, (real)(int32_t)(B.x - I.A.x) * I.lscale,
                            (real)(int32_t)(B.y - I.A.y) * I.lscale,
                            (real)(int32_t)(B.z - I.A.z) * I.lscale, I.qi * a.sq[k],
                            I.se * s_lj[tj], I.hs + s_lj[a.T + tj], fx, fy, fz, e);
}

// Pair forces of the sorted atoms idx[0..n) in order, the next neighbour's
// position, type and charge loaded before the current pair is evaluated (the
// gathers, not the arithmetic, bound the pair kernel).
template <typename real, bool ENERGY, bool TAB>
__device__ __forceinline__ void eval_list(const PairArgs<real> &a, const real *s_lj,
                                          const AtomI<real> &I, const int32_t *idx, int n,
                                          real &fx, real &fy, real &fz, EAcc<real> &e)
{
    if (n <= 0) return;
    int k = (int)RBMD_IDX(idx[0], a.N, a.err);
    uint4 B = a.spos[k];
    int tj = a.stype[k];
    real qj = a.sq[k];
    for (int t = 0; t < n; ++t) {
        uint4 Bn = B;
        int tn = tj;
        real qn = qj;
        if (t + 1 < n) {
            const int kn = (int)RBMD_IDX(idx[t + 1], a.N, a.err);
            Bn = a.spos[kn];
            tn = a.stype[kn];
            qn = a.sq[kn];
        }
        pair_eval<real, ENERGY, TAB>(a, (real)(int32_t)(B.x - I.A.x) * I.lscale,
                                     (real)(int32_t)(B.y - I.A.y) * I.lscale,
                                     (real)(int32_t)(B.z - I.A.z) * I.lscale, I.qi * qj,
                                     I.se * s_lj[tj], I.hs + s_lj[a.T + tj], fx, fy, fz, e);
        B = Bn;
        tj = tn;
        qj = qn;
    }
}

// eval_list over a 16-byte aligned index row: four indices per load, then the
// four neighbours' gathers issued together (entries past n stay inside the row
// and are not used).  Same pair order as eval_list.
template <typename real, bool ENERGY, bool TAB>
__device__ __forceinline__ void eval_list4(const PairArgs<real> &a, const real *s_lj,
                                           const AtomI<real> &I, const int32_t *idx, int n,
                                           real &fx, real &fy, real &fz, EAcc<real> &e)
{
    for (int e0 = 0; e0 < n; e0 += 4) {
        const int4 kk = reinterpret_cast<const int4 *>(idx)[e0 >> 2];
        const int ks[4] = {kk.x, kk.y, kk.z, kk.w};
        uint4 B[4];
        int tj[4];
        real qj[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = (int)RBMD_IDX(e0 + q < n ? ks[q] : ks[0], a.N, a.err);
            B[q] = a.spos[k];
            tj[q] = a.stype[k];
            qj[q] = a.sq[k];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (e0 + q < n)
                pair_eval<real, ENERGY, TAB>(a, (real)(int32_t)(B[q].x - I.A.x) * I.lscale,
                                             (real)(int32_t)(B[q].y - I.A.y) * I.lscale,
                                             (real)(int32_t)(B[q].z - I.A.z) * I.lscale,
                                             I.qi * qj[q], I.se * s_lj[tj[q]],
                                             I.hs + s_lj[a.T + tj[q]], fx, fy, fz, e);
    }
}

// Table or closed forms chosen at run time (the rarely used fallback kernel).
template <typename real, bool ENERGY>
__device__ __forceinline__ void eval_any(const PairArgs<real> &a, const real *s_lj,
                                         const AtomI<real> &I, int k, real &fx, real &fy, real &fz,
                                         EAcc<real> &e)
{
    if (a.tab) eval_k<real, ENERGY, true>(a, s_lj, I, k, fx, fy, fz, e);
    else eval_k<real, ENERGY, false>(a, s_lj, I, k, fx, fy, fz, e);
}

// Philox4x32-10 of the batch priority for the counter (id_i, id_j, step, tag).
// Round 0 multiplies only the words id_i and step, so its result is the same for
// every j of atom i except for one xor with id_j: it is computed once per atom
// and each candidate runs rounds 1-9 only.
struct Philox0 {
    uint32_t x, y, z, w;  // round-0 output with id_j = 0
};

__device__ __forceinline__ Philox0 philox_round0(uint32_t id_i, uint32_t step, uint32_t tag,
                                                 uint2 key)
{
    uint32_t h0, l0, h1, l1;
    philox_mulhilo(0xD2511F53u, id_i, h0, l0);
    philox_mulhilo(0xCD9E8D57u, step, h1, l1);
    return Philox0{h1 ^ key.x, l1, h0 ^ tag ^ key.y, l0};
}

__device__ __forceinline__ uint2 philox_rest(const Philox0 &r0, uint32_t id_j, uint2 key)
{
    uint4 c = make_uint4(r0.x ^ id_j, r0.y, r0.z, r0.w);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
        uint32_t h0, l0, h1, l1;
        philox_mulhilo(0xD2511F53u, c.x, h0, l0);
        philox_mulhilo(0xCD9E8D57u, c.z, h1, l1);
        c = make_uint4(h1 ^ c.y ^ key.x, l1, h0 ^ c.w ^ key.y, l0);
    }
    return make_uint2(c.x, c.y);  // priority = x << 32 | y
}

// Round keys of rounds 1-9 (the seed plus r Weyl increments), computed once per
// atom for philox_rest4.
struct PhiloxKeys {
    uint2 k[9];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint2 key)
{
    PhiloxKeys K;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
        K.k[r] = key;
    }
    return K;
}

// Four priorities at once (the same rounds as philox_rest, the four chains
// interleaved so that their dependent multiplies overlap): pri[q] = (w0, w1) of
// counter (id_i, id_j[q], step, tag).
__device__ __forceinline__ void philox_rest4(const Philox0 &r0, const uint32_t (&id)[4],
                                             const PhiloxKeys &K, uint2 (&pri)[4])
{
    uint4 c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = make_uint4(r0.x ^ id[q], r0.y, r0.z, r0.w);
#pragma unroll
    for (int r = 0; r < 9; ++r) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t h0, l0, h1, l1;
            philox_mulhilo(0xD2511F53u, c[q].x, h0, l0);
            philox_mulhilo(0xCD9E8D57u, c[q].z, h1, l1);
            c[q] = make_uint4(h1 ^ c[q].y ^ K.k[r].x, l1, h0 ^ c[q].w ^ K.k[r].y, l0);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) pri[q] = make_uint2(c[q].x, c[q].y);
}

// The products of rounds 1 and 2 that do not depend on id_j.  id_j enters round 0's
// output in the x word only (philox_rest), so round 1's second product (of the z
// word) and round 2's first product (of round 1's x word, h1 ^ y ^ key) are the
// same for every j of one atom: precomputed once, they leave 16 of the 18
// multiplies per priority and shorten a single chain by two products.  (Four
// interleaved chains, philox_rest4, measured faster with all 18: there the
// independent products of rounds 1 and 2 hide the multiply latency.)
struct Philox12 {
    uint32_t r0x;   // round-0 x word before id_j is xored in
    uint32_t zk;    // round-0 w word ^ round-1 key y (xored into round 1's z)
    uint32_t y1k;   // round-1 y word ^ round-2 key x
    uint32_t b2hk;  // round-2 high product of the x word ^ round-2 key y
    uint32_t b2l;   // round-2 low product of the x word (round-2 w)
};

// k1, k2: the keys of rounds 1 and 2
__device__ __forceinline__ Philox12 philox_pre12(const Philox0 &r0, uint2 k1, uint2 k2)
{
    uint32_t a1h, a1l, b2h, b2l;
    philox_mulhilo(0xCD9E8D57u, r0.z, a1h, a1l);
    const uint32_t x1 = a1h ^ r0.y ^ k1.x;
    philox_mulhilo(0xD2511F53u, x1, b2h, b2l);
    return Philox12{r0.x, r0.w ^ k1.y, a1l ^ k2.x, b2h ^ k2.y, b2l};
}

// One priority from the precomputed products; k2 the key of round 2 (the later
// round keys are formed on the way, as philox_rest does).  Same output as
// philox_rest.
__device__ __forceinline__ uint2 philox_rest_pre(const Philox12 &P, uint32_t id_j, uint2 k2)
{
    uint32_t h0, l0, h1, l1;
    philox_mulhilo(0xD2511F53u, P.r0x ^ id_j, h0, l0);
    philox_mulhilo(0xCD9E8D57u, h0 ^ P.zk, h1, l1);
    uint4 c = make_uint4(h1 ^ P.y1k, l1, P.b2hk ^ l0, P.b2l);
    uint2 key = k2;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
        philox_mulhilo(0xD2511F53u, c.x, h0, l0);
        philox_mulhilo(0xCD9E8D57u, c.z, h1, l1);
        c = make_uint4(h1 ^ c.y ^ key.x, l1, h0 ^ c.w ^ key.y, l0);
    }
    return make_uint2(c.x, c.y);
}

// Bottom-p selection over (priority, id), in registers, keyed by the high 32
// bits of the priority, as the overflow fallback kernel runs it (select_atom
// uses packed keys and a min/max insertion instead).  The CAP slots hold a
// sorted list, ascending.  For a
// batch size p < CAP the lowest CAP - p slots hold "minus infinity" markers, so
// the largest kept entry is always slot CAP - 1; empty slots hold "plus
// infinity" (key 0xFFFFFFFF).  An insertion is a branch-free shift in which every
// slot is updated independently (no serial compare chain).  If the candidate's
// high word equals a slot's key (probability about 2^-32 per slot) the exact
// path ranks that slot by the full 64-bit priorities and then the atom id.
constexpr int SEL_NEG = -2;  // slot marker: minus infinity
constexpr int SEL_POS = -1;  // slot marker: plus infinity (empty)

struct SelCtx {
    Philox0 r0;
    uint2 key;
    const uint32_t *g;  // global ids of the replica's rows (slab contexts), or NULL
};

// true if slot (replica-local atom id hk) orders before the candidate `id`
// (priorities and ties on the ids of the draws).
__device__ __noinline__ bool sel_slot_before(const SelCtx &s, int hk, uint32_t id)
{
    if (hk == SEL_NEG) return true;
    if (hk == SEL_POS) return false;
    const uint32_t hid = s.g ? s.g[hk] : (uint32_t)hk;
    const uint32_t cid = s.g ? s.g[id] : id;
    const uint2 pa = philox_rest(s.r0, hid, s.key), pb = philox_rest(s.r0, cid, s.key);
    if (pa.x != pb.x) return pa.x < pb.x;
    if (pa.y != pb.y) return pa.y < pb.y;
    return hid < cid;
}

template <int CAP>
__device__ __forceinline__ void sel_init(uint32_t (&hh)[CAP], int (&hk)[CAP], int p)
{
#pragma unroll
    for (int e = 0; e < CAP; ++e) {
        const bool neg = e < CAP - p;
        hh[e] = neg ? 0u : 0xFFFFFFFFu;
        hk[e] = neg ? SEL_NEG : SEL_POS;
    }
}

template <int CAP>
__device__ __forceinline__ void sel_insert(uint32_t (&hh)[CAP], int (&hk)[CAP], uint32_t h, int k,
                                           uint32_t id, const SelCtx &s)
{
    bool below[CAP];  // slot e orders before the candidate (a prefix: the list is sorted)
    bool tie = false;
#pragma unroll
    for (int e = 0; e < CAP; ++e) {
        below[e] = hh[e] < h;
        tie |= hh[e] == h;
    }
    if (tie) {
#pragma unroll
        for (int e = 0; e < CAP; ++e)
            if (hh[e] == h) below[e] = sel_slot_before(s, hk[e], id);
    }
    if (below[CAP - 1]) return;  // not below the largest kept entry
    // drop slot CAP-1 and insert: slots below stay, the first slot not below
    // takes the candidate, the rest take their lower neighbour
#pragma unroll
    for (int e = CAP - 1; e > 0; --e) {
        const bool b = below[e], bp = below[e - 1];
        const uint32_t nh = b ? hh[e] : (bp ? h : hh[e - 1]);
        const int nk = b ? hk[e] : (bp ? k : hk[e - 1]);
        hh[e] = nh;
        hk[e] = nk;
    }
    if (!below[0]) {
        hh[0] = h;
        hk[0] = k;
    }
}

__device__ __forceinline__ float cell_frac(uint32_t u, int nc)
{
    return (float)(uint32_t)((uint64_t)u * (uint64_t)nc) * 2.3283064365386963e-10f;  // 2^-32
}

// Calls f(kb, ke) for the contiguous sorted-atom ranges that cover the neighbour
// cells of position A: the (x, y) rows of the stencil, each as at most two z
// ranges (periodic wrap).  Rows and z cells that cannot hold an atom within r_cut
// are skipped by a conservative float test with a 1e-5 margin: this only saves
// work, membership itself is decided on integers.
template <typename real, class F>
__device__ __forceinline__ void stencil_ranges(const PairArgs<real> &a, const Rep &rp,
                                               const uint4 &A, F &&f)
{
    const int nc = rp.nc, dv = a.div;
    const int32_t *cell_start = a.cell_start + rp.cell0;
    const int cx = cell_coord(A.x, nc), cy = cell_coord(A.y, nc), cz = cell_coord(A.z, nc);
    const bool full = nc >= 2 * dv + 1;  // else every cell along an axis, once
    const int span = full ? 2 * dv + 1 : nc;
    const float fxc = cell_frac(A.x, nc), fyc = cell_frac(A.y, nc), fzc = cell_frac(A.z, nc);
    const float Rw = a.stale ? rp.cull_v : rp.cull_r, Rw2 = Rw * Rw;
    for (int ox = 0; ox < span; ++ox) {
        float wx = 0.f;
        int gx = ox;
        if (full) {
            const int o = ox - dv;
            wx = o > 0 ? (float)o - fxc : (o < 0 ? fxc + (float)(-o - 1) : 0.f);
            if (wx > Rw) continue;
            gx = cx + o;
            gx += (gx < 0) ? nc : 0;
            gx -= (gx >= nc) ? nc : 0;
        }
        for (int oy = 0; oy < span; ++oy) {
            float wy = 0.f;
            int gy = oy;
            if (full) {
                const int o = oy - dv;
                wy = o > 0 ? (float)o - fyc : (o < 0 ? fyc + (float)(-o - 1) : 0.f);
                gy = cy + o;
                gy += (gy < 0) ? nc : 0;
                gy -= (gy >= nc) ? nc : 0;
            }
            const float rem = Rw2 - wx * wx - wy * wy;
            if (full && rem < 0.f) continue;
            const int64_t row = ((int64_t)gx * nc + gy) * nc;
            int rb0, re0, rb1 = 0, re1 = 0;
            if (!full) {
                rb0 = cell_start[row];
                re0 = cell_start[row + nc];
            } else {
                // z cells reachable within the remaining radius, relative to cz
                const float rz = sqrtf(fmaxf(rem, 0.f));
                const int z0 = cz + max(-dv, (int)floorf(fzc - rz));
                const int z1 = cz + min(dv, (int)floorf(fzc + rz));  // inclusive, may wrap
                if (z0 < 0) {
                    rb0 = cell_start[row + z0 + nc];
                    re0 = cell_start[row + nc];
                    rb1 = cell_start[row];
                    re1 = cell_start[row + z1 + 1];
                } else if (z1 >= nc) {
                    rb0 = cell_start[row + z0];
                    re0 = cell_start[row + nc];
                    rb1 = cell_start[row];
                    re1 = cell_start[row + z1 - nc + 1];
                } else {
                    rb0 = cell_start[row + z0];
                    re0 = cell_start[row + z1 + 1];
                }
            }
            f(rb0, re0);
            if (rb1 < re1) f(rb1, re1);
        }
    }
}

// 0: not a neighbour, 1: core (D < Rc2), 2: shell (Rc2 <= D <= Rs2).  Integer
// minimum image d = (int32)(u_j - u_i); D = sum d^2 in uint64 (cannot overflow).
__device__ __forceinline__ int classify(const Rep &a, const uint4 &A, const uint4 &B)
{
    const int32_t dx = (int32_t)(B.x - A.x);
    const int32_t dy = (int32_t)(B.y - A.y);
    const int32_t dz = (int32_t)(B.z - A.z);
    const uint32_t R2x = 2u * a.Rlin;
    // |d| > Rlin on any axis: outside r_cut (unsigned wrap test)
    if (((uint32_t)dx + a.Rlin > R2x) | ((uint32_t)dy + a.Rlin > R2x) |
        ((uint32_t)dz + a.Rlin > R2x))
        return 0;
    const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                       (uint64_t)((int64_t)dz * dz);
    if (D > a.Rs2) return 0;
    return D < a.Rc2 ? 1 : 2;
}

// classify for a pair known to lie within Rv < 2^31 units on every axis (a
// candidate of the step's lists): no per-axis reject, the same result.
__device__ __forceinline__ int classify_near(const Rep &a, const uint4 &A, const uint4 &B)
{
    const int32_t dx = (int32_t)(B.x - A.x);
    const int32_t dy = (int32_t)(B.y - A.y);
    const int32_t dz = (int32_t)(B.z - A.z);
    const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                       (uint64_t)((int64_t)dz * dz);
    if (D > a.Rs2) return 0;
    return D < a.Rc2 ? 1 : 2;
}

template <typename real>
__device__ __forceinline__ bool overflowed(const PairArgs<real> &a, int2 cnt)
{
    return cnt.x > a.CC || cnt.y > a.CS;
}

// Step 1a: lists.
template <typename real, bool ENERGY, bool LISTS>
__global__ void __launch_bounds__(256) k_rbl_scan(PairArgs<real> a)
{
    const AtomSlot sl = atom_slot(a.map, a.reps);  // replica ranges are the same when sorted
    if (!sl.ok) return;
    const int64_t is = sl.i;
    const Rep rp = a.reps[sl.r];  // by value: the fields live in registers
    const uint4 A = a.spos[is];
    const uint32_t id0 = (uint32_t)rp.atom0;
    const int64_t N = a.N;
    int ncore = 0, ns = 0;
    stencil_ranges(a, rp, A, [&](int kb, int ke) {
        for (int k = kb; k < ke; k += 4) {
            uint4 B[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) B[q] = (k + q < ke) ? a.spos[RBMD_IDX(k + q, N, a.err)] : A;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = (k + q < ke && k + q != (int)is) ? classify(rp, A, B[q]) : 0;
                if (c == 1) {
                    if (ncore < a.CC) a.lcore[lidx(is, ncore, N, a.CC)] = k + q;
                    ++ncore;
                } else if (c == 2) {
                    if (ns < a.CS) a.lshell[lidx(is, ns, N, a.CS)] = (int32_t)(B[q].w - id0);
                    ++ns;
                }
            }
        }
    });
    const int2 cnt = make_int2(ncore, ns);
    a.ncount[is] = cnt;
    if (overflowed(a, cnt)) *a.ovf = 1;
    if constexpr (ENERGY) {
        // one atomic per group of converged lanes (all to one address)
        const unsigned m = __activemask();
        const int mx = __reduce_max_sync(m, ns);
        if ((threadIdx.x & 31) == __ffs(m) - 1) atomicMax(a.imax, mx);
    }
    if constexpr (LISTS) {
        a.n_core[A.w] = ncore;
        a.n_shell[A.w] = ns;
        if (a.exact)
            for (int e = 0; e < a.p; ++e) a.batch[(int64_t)A.w * a.p + e] = -1;
    }
}

// Step 1b: the batch B(i), the p shell members with the smallest Philox priority
// (all of them when N_s <= p), as sorted indices in bk[i][0..min(N_s,p)).
// The shell list holds atom ids, so a priority needs one list load and no
// lookup; only the p winners are mapped to sorted indices.

// The exact selection of one atom (full 64-bit priorities, then the id), for the
// rare atoms where the fast selection met equal truncated keys; fills hk with
// CAP - p "minus infinity" markers, then the p smallest ascending (or empty slots).
template <int CAP>
__device__ __noinline__ void select_exact(const Philox0 &r0, uint2 key, const int32_t *ls, int ns,
                                          int p, int (&hk)[CAP], int stride = 1,
                                          const uint32_t *g = nullptr)
{
    uint64_t kk[CAP];
    uint32_t kid[CAP], kloc[CAP];  // ids of the draws (ties), and replica-local ids
    int kept = 0;
    for (int e = 0; e < ns; ++e) {
        const uint32_t loc = (uint32_t)ls[e * stride];
        const uint32_t id = g ? g[loc] : loc;
        const uint2 w = philox_rest(r0, id, key);
        const uint64_t v = ((uint64_t)w.x << 32) | w.y;
        int j;  // the slot the shifting starts from
        if (kept == p) {
            if (!(v < kk[p - 1] || (v == kk[p - 1] && id < kid[p - 1]))) continue;
            j = p - 1;  // the largest kept entry drops out
        } else {
            j = kept;
        }
        while (j > 0 && (v < kk[j - 1] || (v == kk[j - 1] && id < kid[j - 1]))) {
            kk[j] = kk[j - 1];
            kid[j] = kid[j - 1];
            kloc[j] = kloc[j - 1];
            --j;
        }
        kk[j] = v;
        kid[j] = id;
        kloc[j] = loc;
        if (kept < p) ++kept;
    }
    for (int e = 0; e < CAP; ++e) {
        const int j = e - (CAP - p);
        hk[e] = j < 0 ? SEL_NEG : (j < kept ? (int)kloc[j] : SEL_POS);
    }
}

template <typename real, int CAP, bool LISTS>
__device__ __forceinline__ void select_atom(const PairArgs<real> &a, int64_t is, int r)
{
    const Rep rp = a.reps[r];
    const uint32_t id0 = (uint32_t)rp.atom0;
    const int2 cnt = a.ncount[is];
    if (overflowed(a, cnt)) return;
    const int ns = cnt.y;
    const int64_t N = a.N;
    const uint32_t id_i = a.spos[is].w;
    int32_t ids[CAP];
    int nb = 0;
    if (ns <= a.p) {
        for (int e = 0; e < ns; ++e) {
            const int32_t id = a.lshell[lidx(is, e, N, a.CS)];
            if constexpr (LISTS) ids[e < CAP ? e : 0] = id;
            a.bk[lidx(is, e, N, a.p)] = a.sidx[RBMD_IDX(id0 + (uint32_t)id, N, a.err)];
        }
        nb = ns;
    } else {
        const SelCtx sel{philox_round0(pid(a, id0, id_i - id0), (uint32_t)step_of(a.step),
                                       rp.tag_rbl, rp.key),
                         rp.key, a.gid ? a.gid + id0 : nullptr};
        const int32_t *ls = a.lshell + lidx(is, 0, N, a.CS);
        // keys: the priority's high word with its low b bits replaced by the
        // member's list position (2^b > CS, so no key is all ones and no two are
        // equal); the CAP + 1 smallest kept sorted by a min/max insertion
        const int b = 32 - __clz(a.CS);
        const uint32_t lo_mask = (1u << b) - 1u;
        uint32_t keep = ~lo_mask;  // the priority bits a key holds
        if (a.sel_key_bits > 0 && a.sel_key_bits < 32) keep &= ~(0xFFFFFFFFu >> a.sel_key_bits);
        uint32_t sk[CAP + 1];
#pragma unroll
        for (int e = 0; e <= CAP; ++e) sk[e] = 0xFFFFFFFFu;
        const uint2 k1 = make_uint2(rp.key.x + 0x9E3779B9u, rp.key.y + 0xBB67AE85u);
        const uint2 k2 = make_uint2(k1.x + 0x9E3779B9u, k1.y + 0xBB67AE85u);
        const Philox12 P12 = philox_pre12(sel.r0, k1, k2);
        auto insert = [&](uint32_t id, int e) {
            const uint2 w = philox_rest_pre(P12, pid(a, id0, id), k2);
            uint32_t x = (w.x & keep) | (uint32_t)e;
#pragma unroll
            for (int j = 0; j <= CAP; ++j) {
                const uint32_t m = min(sk[j], x);
                x = max(sk[j], x);
                sk[j] = m;
            }
        };
        if ((a.CS & 3) == 0) {
            // 16-byte rows: four list entries per load, the next four loaded
            // before the current ones are ranked (entries past N_s stay inside
            // the row and are skipped)
            const int4 *l4 = reinterpret_cast<const int4 *>(ls);
            int4 cur = l4[0];  // ns > p >= 1
            for (int e0 = 0; e0 < ns; e0 += 4) {
                int4 nxt = cur;
                if (e0 + 4 < ns) nxt = l4[(e0 >> 2) + 1];
                insert((uint32_t)cur.x, e0);
                if (e0 + 1 < ns) insert((uint32_t)cur.y, e0 + 1);
                if (e0 + 2 < ns) insert((uint32_t)cur.z, e0 + 2);
                if (e0 + 3 < ns) insert((uint32_t)cur.w, e0 + 3);
                cur = nxt;
            }
        } else {
            uint32_t idn = (uint32_t)ls[0];  // ns > p >= 1
            for (int e = 0; e < ns; ++e) {
                const uint32_t id = idn;
                if (e + 1 < ns) idn = (uint32_t)ls[e + 1];
                insert(id, e);
            }
        }
        // the key order is the priority order unless two of the p + 1 smallest
        // share their truncated high words (then the exact selection decides)
        bool tie = a.sel_exact != 0;
#pragma unroll
        for (int e = 0; e < CAP; ++e)
            if (e < a.p) tie |= ((sk[e] ^ sk[e + 1]) & keep) == 0u;
        if (!tie) {
#pragma unroll
            for (int e = 0; e < CAP; ++e)
                if (e < a.p) {
                    const int32_t id = ls[sk[e] & lo_mask];
                    if constexpr (LISTS) ids[e] = id;
                    a.bk[lidx(is, e, N, a.p)] = a.sidx[RBMD_IDX(id0 + (uint32_t)id, N, a.err)];
                }
            nb = a.p;
        } else {
            int hk[CAP];
            select_exact<CAP>(sel.r0, rp.key, ls, ns, a.p, hk, 1, sel.g);
            for (int e = 0; e < CAP; ++e)
                if (hk[e] >= 0) {
                    if constexpr (LISTS) ids[nb] = hk[e];
                    a.bk[lidx(is, nb, N, a.p)] = a.sidx[RBMD_IDX(id0 + (uint32_t)hk[e], N, a.err)];
                    ++nb;
                }
        }
    }
    if constexpr (LISTS) {
        // batch ids ascending, -1 padded (verification path only)
        int32_t *out = a.batch + (int64_t)id_i * a.p;
        for (int e = 0; e < a.p; ++e) out[e] = -1;
        for (int e = 0; e < nb; ++e) {
            const int32_t v = (int32_t)(ids[e] + id0);
            int y = e - 1;
            while (y >= 0 && out[y] > v) {
                out[y + 1] = out[y];
                --y;
            }
            out[y + 1] = v;
        }
    }
}

// One thread per cell-sorted atom (p <= 10); four resident blocks per SM (61
// registers, no spills): three measured the same, five (spilling) slower.
template <typename real, int CAP, bool LISTS>
__global__ void __launch_bounds__(256, 4) k_rbl_select(PairArgs<real> a)
{
    const AtomSlot sl = atom_slot(a.map, a.reps);
    if (sl.ok) select_atom<real, CAP, LISTS>(a, sl.i, sl.r);
}

// p > 10: the register heap is large, so the kernel runs a grid-stride loop over
// the compact list of atoms that need a selection (N_s > p), made by
// k_rbl_take_shell; each atom's output depends on that atom only, so the list
// order does not matter.
template <typename real, int CAP, bool LISTS>
__global__ void __launch_bounds__(256) k_rbl_select_list(PairArgs<real> a)
{
    const int32_t n = *a.heavy_n;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int2 h = a.heavy[j];
        select_atom<real, CAP, LISTS>(a, h.x, h.y);
    }
}

// p > 32: one warp per listed atom sorts its whole shell by priority in shared
// memory (bitonic sort of (w0 << 32 | w1, id) pairs, the exact order of the batch
// rule) and keeps the first p.  The priorities are computed by the lanes in
// parallel.  Shared memory: SEL_WARPS warps x n2 entries of 12 bytes, n2 the
// power of two at or above the shell capacity.
constexpr int SEL_WARPS = 4;

template <typename real, bool LISTS>
__global__ void __launch_bounds__(32 * SEL_WARPS) k_rbl_select_warp(PairArgs<real> a, int n2)
{
    extern __shared__ __align__(16) unsigned char smem_sel[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *s_key = reinterpret_cast<uint64_t *>(smem_sel) + (size_t)w * n2;
    uint32_t *s_id = reinterpret_cast<uint32_t *>(reinterpret_cast<uint64_t *>(smem_sel) +
                                                  (size_t)SEL_WARPS * n2) + (size_t)w * n2;
    const int32_t n = *a.heavy_n;
    const int64_t N = a.N;
    for (int64_t j = (int64_t)blockIdx.x * SEL_WARPS + w; j < n;
         j += (int64_t)gridDim.x * SEL_WARPS) {
        const int2 h = a.heavy[j];
        const int64_t is = h.x;
        const Rep rp = a.reps[h.y];
        const uint32_t id0 = (uint32_t)rp.atom0;
        const int ns = a.ncount[is].y;
        const uint32_t id_i = a.spos[is].w;
        const Philox0 r0 =
            philox_round0(pid(a, id0, id_i - id0), (uint32_t)step_of(a.step), rp.tag_rbl, rp.key);
        const int32_t *ls = a.lshell + lidx(is, 0, N, a.CS);
        int m = 1;
        while (m < ns) m <<= 1;  // sort length: power of two, at most n2
        for (int e = lane; e < m; e += 32) {
            if (e < ns) {
                const uint32_t id = (uint32_t)ls[e];
                const uint2 pw = philox_rest(r0, pid(a, id0, id), rp.key);
                s_key[e] = ((uint64_t)pw.x << 32) | pw.y;
                s_id[e] = id;
            } else {
                s_key[e] = ~0ull;  // padding sorts last
                s_id[e] = 0xFFFFFFFFu;
            }
        }
        __syncwarp();
        for (int k = 2; k <= m; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < m; i += 32) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const uint64_t ki = s_key[i], kl = s_key[l];
                        const uint32_t ii = s_id[i], il = s_id[l];
                        const bool gt = ki > kl || (ki == kl && ii > il);
                        if (((i & k) == 0) == gt) {  // ascending where i & k == 0
                            s_key[i] = kl;
                            s_key[l] = ki;
                            s_id[i] = il;
                            s_id[l] = ii;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int e = lane; e < a.p; e += 32)
            a.bk[lidx(is, e, N, a.p)] = a.sidx[id0 + s_id[e]];
        if constexpr (LISTS) {
            // batch ids ascending, -1 padded (verification path only): sort the p kept
            // ids by a second bitonic pass over ids (priorities no longer needed)
            int mp = 1;
            while (mp < a.p) mp <<= 1;
            __syncwarp();
            for (int e = lane; e < mp; e += 32) {
                s_key[e] = e < a.p ? (uint64_t)s_id[e] : ~0ull;
            }
            __syncwarp();
            for (int k = 2; k <= mp; k <<= 1)
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int i = lane; i < mp; i += 32) {
                        const int l = i ^ jj;
                        if (l > i) {
                            const uint64_t ki = s_key[i], kl = s_key[l];
                            if (((i & k) == 0) == (ki > kl)) {
                                s_key[i] = kl;
                                s_key[l] = ki;
                            }
                        }
                    }
                    __syncwarp();
                }
            int32_t *out = a.batch + (int64_t)id_i * a.p;
            for (int e = lane; e < a.p; e += 32) out[e] = (int32_t)(s_key[e] + id0);
        }
        __syncwarp();
    }
}

// Step 1b for atoms with N_s <= p: the batch is the whole shell (weight 1); the
// others go to the list of k_rbl_select_list.
template <typename real, bool LISTS>
__global__ void __launch_bounds__(256) k_rbl_take_shell(PairArgs<real> a)
{
    const AtomSlot sl = atom_slot(a.map, a.reps);
    if (!sl.ok) return;
    const int64_t is = sl.i;
    const int2 cnt = a.ncount[is];
    const bool heavy = !overflowed(a, cnt) && cnt.y > a.p;
    // warp-aggregated append of the atoms that need a selection
    const unsigned m = __ballot_sync(__activemask(), heavy);
    if (heavy) {
        const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(a.heavy_n, __popc(m));
        base = __shfl_sync(m, base, leader);
        a.heavy[base + __popc(m & ((1u << lane) - 1))] = make_int2((int)is, sl.r);
        return;
    }
    if (overflowed(a, cnt)) return;
    const uint32_t id0 = (uint32_t)a.reps[sl.r].atom0;
    const int64_t N = a.N;
    const int32_t *ls = a.lshell + lidx(is, 0, N, a.CS);
    for (int e = 0; e < cnt.y; ++e)
        a.bk[lidx(is, e, N, a.p)] = a.sidx[RBMD_IDX(id0 + (uint32_t)ls[e], N, a.err)];
    if constexpr (LISTS) {
        // batch ids ascending, -1 padded (verification path only)
        int32_t *out = a.batch + (int64_t)a.spos[is].w * a.p;
        for (int e = 0; e < a.p; ++e) out[e] = -1;
        for (int e = 0; e < cnt.y; ++e) {
            const int32_t v = (int32_t)(ls[e] + id0);
            int y = e - 1;
            while (y >= 0 && out[y] > v) {
                out[y + 1] = out[y];
                --y;
            }
            out[y + 1] = v;
        }
    }
}

// Warp sums of the force (and, with ENERGY, of the halved energies and virials)
// into the FP64 partial slot `part` (every lane of the warp calls it).
template <typename real, bool ENERGY>
__device__ __forceinline__ void warp_partials(const PairArgs<real> &a, int64_t part, real fx,
                                              real fy, real fz, const EAcc<real> &e)
{
    // the force sums as exact fixed-point integers (fix32): the momentum correction,
    // and with it the trajectory, does not depend on which atoms share a warp (the
    // sorted order of the last candidate rebuild).  The energies and virials
    // (reported, not integrated) are summed over the warp in the working precision
    // (FP64 operations are scarce on this GPU) and across warps in FP64.
    long long f[3] = {fix32(fx), fix32(fy), fix32(fz)};
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) f[c] += __shfl_down_sync(0xffffffffu, f[c], o);
    real v[EPART] = {e.ec, e.el, e.wc, e.wl};
    if constexpr (ENERGY) {
#pragma unroll
        for (int c = 0; c < 6; ++c) v[4 + c] = e.w[c];
#pragma unroll
        for (int c = 0; c < EPART; ++c)
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    }
    if ((threadIdx.x & 31) == 0) {
        a.fpart[3 * part + 0] = f[0];
        a.fpart[3 * part + 1] = f[1];
        a.fpart[3 * part + 2] = f[2];
        if constexpr (ENERGY) {
#pragma unroll
            for (int c = 0; c < EPART; ++c) a.epart[EPART * part + c] = 0.5 * (double)v[c];
        }
    }
}

// Step 2 (+ the partial sums of step 3).
template <typename real, bool ENERGY, bool TAB>
__global__ void __launch_bounds__(kPairBlock) k_rbl_force(PairArgs<real> a)
{
    __shared__ real s_lj[2 * RBMD_MAX_TYPES];
    for (int t = threadIdx.x; t < 2 * a.T; t += blockDim.x) s_lj[t] = a.lj[t];
    __syncthreads();
    const AtomSlot sl = atom_slot(a.map, a.reps);
    const int64_t is = sl.i;
    real fx = 0, fy = 0, fz = 0;
    EAcc<real> e;
    eacc_zero(e);
    bool own = sl.ok;
    if (own && a.gid) {
        // a slab context's halo rows are neighbours only: zero force, no sums
        const Rep &rq = a.reps[sl.r];
        own = (int64_t)a.spos[is].w - rq.atom0 < rq.n_own;
        if (!own && !a.accumulate) {
            real *f = a.F + 3 * (int64_t)a.spos[is].w;
            f[0] = f[1] = f[2] = (real)0;
        }
    }
    if (own) {
        const int2 cnt = a.ncount[is];
        if (!overflowed(a, cnt)) {
            AtomI<real> I;
            I.A = a.spos[is];
            I.qi = a.sq[is] * a.ck;
            I.lscale = (real)a.reps[sl.r].lscale;
            const int ti = a.stype[is];
            I.se = s_lj[ti];
            I.hs = s_lj[a.T + ti];
            const int64_t N = a.N;
            if ((a.CC & 3) == 0)
                eval_list4<real, ENERGY, TAB>(a, s_lj, I, a.lcore + lidx(is, 0, N, a.CC), cnt.x, fx,
                                              fy, fz, e);
            else
                eval_list<real, ENERGY, TAB>(a, s_lj, I, a.lcore + lidx(is, 0, N, a.CC), cnt.x, fx, fy,
                                             fz, e);
            if (a.exact) {
                const uint32_t id0 = (uint32_t)a.reps[sl.r].atom0;
                for (int k = 0; k < cnt.y; ++k)
                    eval_k<real, ENERGY, TAB>(a, s_lj, I,
                                              a.sidx[id0 + (uint32_t)a.lshell[lidx(is, k, N, a.CS)]],
                                              fx, fy, fz, e);
            } else {
                const int nb = min(cnt.y, a.p);
                const real w = cnt.y > a.p ? (real)cnt.y / (real)a.p : (real)1;
                real bx = 0, by = 0, bz = 0;
                EAcc<real> be;
                eacc_zero(be);
                eval_list<real, ENERGY, TAB>(a, s_lj, I, a.bk + lidx(is, 0, N, a.p), nb, bx, by, bz,
                                             be);
                fx += w * bx;
                fy += w * by;
                fz += w * bz;
                if constexpr (ENERGY) eacc_add(e, be, w);
            }
            real *f = a.F + 3 * (int64_t)I.A.w;
            if (a.accumulate) {
                f[0] += fx;
                f[1] += fy;
                f[2] += fz;
            } else {
                f[0] = fx;
                f[1] = fy;
                f[2] = fz;
            }
        }
    }
    const int64_t part = (int64_t)blockIdx.x * (kPairBlock / 32) + (threadIdx.x >> 5);
    warp_partials<real, ENERGY>(a, part, fx, fy, fz, e);
}

// Exact fallback for atoms whose lists overflowed (Algorithm 2 for one atom,
// fused, with the candidate list in shared memory and flushed when full).  A
// grid-stride loop over the same replica-aligned 128-atom blocks as k_rbl_force,
// so the partial sums stay per replica and deterministic; when no list
// overflowed it only zeroes its partial slots.
constexpr int FB_LIST = 44;

template <typename real, int CAP, bool ENERGY, bool LISTS>
__global__ void __launch_bounds__(kPairBlock) k_rbl_fused(PairArgs<real> a)
{
    __shared__ real s_lj[2 * RBMD_MAX_TYPES];
    __shared__ int32_t s_k[FB_LIST][kPairBlock];
    __shared__ uint32_t s_id[FB_LIST][kPairBlock];
    const int tid = threadIdx.x;
    constexpr int WPB = kPairBlock / 32;  // partial slots (warps) per map block
    // nothing overflowed: the partial sums skip the fallback's slots
    if (*a.ovf == 0) return;
    for (int t = tid; t < 2 * a.T; t += blockDim.x) s_lj[t] = a.lj[t];
    __syncthreads();
    for (int mb = blockIdx.x; mb < a.nmap; mb += gridDim.x) {
        real fx = 0, fy = 0, fz = 0;
        EAcc<real> e;
        eacc_zero(e);
        const AtomSlot sl = atom_slot_at(a.map, a.reps, mb);
        {
            const int64_t is = sl.i;
            bool own = sl.ok;
            if (own && a.gid)
                own = (int64_t)a.spos[is].w - a.reps[sl.r].atom0 < a.reps[sl.r].n_own;
            if (own && overflowed(a, a.ncount[is])) {
                const Rep rp = a.reps[sl.r];
                const uint32_t id0 = (uint32_t)rp.atom0;
                AtomI<real> I;
                I.A = a.spos[is];
                I.qi = a.sq[is] * a.ck;
                I.lscale = (real)rp.lscale;
                const int ti = a.stype[is];
                I.se = s_lj[ti];
                I.hs = s_lj[a.T + ti];
                const uint32_t id_i = I.A.w;
                const SelCtx sel{philox_round0(pid(a, id0, id_i - id0), (uint32_t)step_of(a.step),
                                               rp.tag_rbl, rp.key),
                                 rp.key, a.gid ? a.gid + id0 : nullptr};
                uint32_t hh[CAP];
                int hk[CAP];
                sel_init<CAP>(hh, hk, a.p);
                real ax = 0, ay = 0, az = 0;
                EAcc<real> ae;
                eacc_zero(ae);
                int lc = 0, lsn = 0, ncore = 0, ns = 0;
                auto flush = [&]() {
                    for (int t = 0; t < lsn; ++t) {
                        const int k = s_k[FB_LIST - 1 - t][tid];
                        if (a.exact) {
                            eval_any<real, ENERGY>(a, s_lj, I, k, ax, ay, az, ae);
                        } else {
                            const uint32_t id = s_id[FB_LIST - 1 - t][tid] - id0;
                            const uint2 w = philox_rest(sel.r0, pid(a, id0, id), rp.key);
                            sel_insert<CAP>(hh, hk, w.x, (int)id, id, sel);
                        }
                    }
                    for (int t = 0; t < lc; ++t) eval_any<real, ENERGY>(a, s_lj, I, s_k[t][tid], ax, ay, az, ae);
                    lc = 0;
                    lsn = 0;
                };
                stencil_ranges(a, rp, I.A, [&](int kb, int ke) {
                    for (int k = kb; k < ke; ++k) {
                        if (k == (int)is) continue;
                        const uint4 B = a.spos[RBMD_IDX(k, a.N, a.err)];
                        const int c = classify(rp, I.A, B);
                        if (c == 1) {
                            s_k[lc][tid] = k;
                            ++lc;
                            ++ncore;
                        } else if (c == 2) {
                            s_k[FB_LIST - 1 - lsn][tid] = k;
                            s_id[FB_LIST - 1 - lsn][tid] = B.w;
                            ++lsn;
                            ++ns;
                        }
                        if (lc + lsn == FB_LIST) flush();
                    }
                });
                flush();
                if (!a.exact) {
                    const real w = ns > a.p ? (real)ns / (real)a.p : (real)1;
                    real bx = 0, by = 0, bz = 0;
                    EAcc<real> be;
                    eacc_zero(be);
#pragma unroll
                    for (int t = 0; t < CAP; ++t)
                        if (hk[t] >= 0)
                            eval_any<real, ENERGY>(a, s_lj, I, a.sidx[id0 + (uint32_t)hk[t]], bx, by,
                                                   bz, be);
                    ax += w * bx;
                    ay += w * by;
                    az += w * bz;
                    if constexpr (ENERGY) eacc_add(ae, be, w);
                    if constexpr (LISTS) {
                        int32_t *out = a.batch + (int64_t)id_i * a.p;
                        for (int e = 0; e < a.p; ++e) out[e] = -1;
                        int nb = 0;
#pragma unroll
                        for (int e = 0; e < CAP; ++e) {
                            if (hk[e] < 0) continue;
                            const int32_t v = (int32_t)(id0 + (uint32_t)hk[e]);
                            int y = nb - 1;
                            while (y >= 0 && out[y] > v) {
                                out[y + 1] = out[y];
                                --y;
                            }
                            out[y + 1] = v;
                            ++nb;
                        }
                    }
                }
                real *f = a.F + 3 * (int64_t)id_i;
                if (a.accumulate) {
                    f[0] += ax;
                    f[1] += ay;
                    f[2] += az;
                } else {
                    f[0] = ax;
                    f[1] = ay;
                    f[2] = az;
                }
                fx += ax;
                fy += ay;
                fz += az;
                if constexpr (ENERGY) eacc_add(e, ae, (real)1);
            }
        }
        warp_partials<real, ENERGY>(a, a.fb_part0 + (int64_t)mb * WPB + (tid >> 5), fx, fy, fz, e);
    }
}

// The exact fallback's register heap holds at most 32 entries: with a larger batch
// an atom whose lists overflowed is reported (RBMD_ERR_CELL_OVERFLOW), not
// computed; the fallback's partial sums are zero.
template <bool ENERGY>
__global__ void k_rbl_no_fallback(const int32_t *__restrict__ ovf, int *__restrict__ err,
                                  long long *__restrict__ fpart, double *__restrict__ epart,
                                  int64_t part0, int64_t nparts)
{
    if (*ovf == 0) return;  // the partial sums skip the fallback's slots
    const int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j0 == 0) latch_error(err, RBMD_ERR_CELL_OVERFLOW);
    for (int64_t j = j0; j < nparts; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t part = part0 + j;
        fpart[3 * part + 0] = 0;
        fpart[3 * part + 1] = 0;
        fpart[3 * part + 2] = 0;
        if constexpr (ENERGY) {
            for (int c = 0; c < EPART; ++c) epart[EPART * part + c] = 0.0;
        }
    }
}

// Largest shell capacity the large-batch selection sorts in shared memory.
constexpr int SEL_WARP_MAX_CS = 4096;

rbmd_status rbl_configure(rbmd_ctx *c)
{
    if (c->prm.rbl_p <= 32) return RBMD_OK;
    if (c->list_cs > SEL_WARP_MAX_CS) return RBMD_ERR_UNSUPPORTED;
    const size_t smem = (size_t)SEL_WARPS * SEL_WARP_MAX_CS * (sizeof(uint64_t) + sizeof(uint32_t));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_select_warp<float, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_select_warp<float, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_select_warp<double, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_select_warp<double, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return RBMD_OK;
}

// Batch selection over the 256-atom block map: one kernel for p <= 10; above, the
// light kernel takes whole shells and lists the rest for the heap kernel.
template <typename real, int CAP, bool LISTS>
static void launch_select(const PairArgs<real> &a256, unsigned nb256, cudaStream_t st)
{
    if constexpr (CAP <= 10) {
        k_rbl_select<real, CAP, LISTS><<<nb256, 256, 0, st>>>(a256);
    } else if constexpr (CAP > 32) {
        cudaMemsetAsync(a256.heavy_n, 0, sizeof(int32_t), st);
        k_rbl_take_shell<real, LISTS><<<nb256, 256, 0, st>>>(a256);
        int n2 = 1;
        while (n2 < a256.CS) n2 <<= 1;
        const size_t smem = (size_t)SEL_WARPS * n2 * (sizeof(uint64_t) + sizeof(uint32_t));
        k_rbl_select_warp<real, LISTS><<<4u * 148u, 32 * SEL_WARPS, smem, st>>>(a256, n2);
    } else {
        cudaMemsetAsync(a256.heavy_n, 0, sizeof(int32_t), st);
        k_rbl_take_shell<real, LISTS><<<nb256, 256, 0, st>>>(a256);
        // one resident block per SM at this register count, a few waves of work
        k_rbl_select_list<real, CAP, LISTS><<<min(nb256, 2u * 148u), 256, 0, st>>>(a256);
    }
}

template <typename real, int CAP>
static void launch_rbl(rbmd_ctx *c, const PairArgs<real> &a, cudaStream_t st, bool energy,
                       bool lists, bool marks)
{
    PairArgs<real> a256 = a, a128 = a;
    a256.map = c->map256;
    a256.nmap = c->nb256;
    a128.map = c->map128;
    a128.nmap = c->nb128;
    const unsigned nb256 = (unsigned)c->nb256, nbp = (unsigned)c->nb128;
    const unsigned nfb = (unsigned)min(c->nb128, 4 * 148);  // fallback: a few waves at most
    if (lists) {
        if (energy) k_rbl_scan<real, true, true><<<nb256, 256, 0, st>>>(a256);
        else k_rbl_scan<real, false, true><<<nb256, 256, 0, st>>>(a256);
        if (marks) prof_mark(c, 3);
        if (!a.exact) launch_select<real, CAP, true>(a256, nb256, st);
    } else {
        if (energy) k_rbl_scan<real, true, false><<<nb256, 256, 0, st>>>(a256);
        else k_rbl_scan<real, false, false><<<nb256, 256, 0, st>>>(a256);
        if (marks) prof_mark(c, 3);
        if (!a.exact) launch_select<real, CAP, false>(a256, nb256, st);
    }
    if (marks) prof_mark(c, 4);
    if (a.tab) {
        if (energy) k_rbl_force<real, true, true><<<nbp, kPairBlock, 0, st>>>(a128);
        else k_rbl_force<real, false, true><<<nbp, kPairBlock, 0, st>>>(a128);
    } else {
        if (energy) k_rbl_force<real, true, false><<<nbp, kPairBlock, 0, st>>>(a128);
        else k_rbl_force<real, false, false><<<nbp, kPairBlock, 0, st>>>(a128);
    }
    if constexpr (CAP > 32) {
        const int64_t nparts = (int64_t)c->nb128 * (kPairBlock / 32);
        if (energy)
            k_rbl_no_fallback<true><<<nfb, kPairBlock, 0, st>>>(a.ovf, c->err, a.fpart, a.epart,
                                                                a.fb_part0, nparts);
        else
            k_rbl_no_fallback<false><<<nfb, kPairBlock, 0, st>>>(a.ovf, c->err, a.fpart, a.epart,
                                                                 a.fb_part0, nparts);
    } else if (lists) {
        if (energy) k_rbl_fused<real, CAP, true, true><<<nfb, kPairBlock, 0, st>>>(a128);
        else k_rbl_fused<real, CAP, false, true><<<nfb, kPairBlock, 0, st>>>(a128);
    } else {
        if (energy) k_rbl_fused<real, CAP, true, false><<<nfb, kPairBlock, 0, st>>>(a128);
        else k_rbl_fused<real, CAP, false, false><<<nfb, kPairBlock, 0, st>>>(a128);
    }
}

// Launch arguments of the RBL kernels from the context (force output, flags and
// verification outputs left for the caller).
template <typename real>
static PairArgs<real> pair_args(rbmd_ctx *c, StepRef s)
{
    PairArgs<real> a;
    memset(&a, 0, sizeof(a));
    a.spos = c->spos;
    a.sq = (const real *)c->sq;
    a.stype = c->stype;
    a.cell_start = c->cell_start;
    a.lj = c->fp64 ? (const real *)c->lj_d : (const real *)c->lj_f;
    a.N = c->N;
    a.reps = c->reps;
    a.map = c->map256;
    a.div = c->div;
    a.T = c->T;
    a.p = c->prm.rbl_p;
    a.exact = (c->prm.flags & RBMD_RBL_EXACT) ? 1 : 0;
    a.step = s;
    a.ck = (real)c->prm.coulomb_k;
    a.alpha = (real)c->prm.alpha;
    a.sqrt_alpha = (real)sqrt(c->prm.alpha);
    a.c2 = (real)(2.0 * sqrt(c->prm.alpha / kPi));
    a.tab = c->use_table ? c->ptab : nullptr;
    a.tab_n = c->ptab_n;
    a.tab_i0 = c->ptab_i0;
    a.tab_inv_h = (real)c->ptab_inv_h;
    a.fpart = c->fpart;
    a.epart = c->epart;
    a.fb_part0 = 4 * (int64_t)c->nb128;
    a.imax = c->ibuf;
    a.lcore = c->lcore;
    a.lshell = c->lshell;
    a.sidx = c->cell_rank;
    a.heavy = c->heavy;
    a.heavy_n = c->ibuf + 3;
    a.sel_exact = c->sel_exact;
    a.sel_key_bits = c->sel_key_bits;
    a.ncount = c->ncount;
    a.bk = c->bk;
    a.ovf = c->ibuf + 2;
    a.CC = c->list_cc;
    a.CS = c->list_cs;
    a.gid = c->gid;
    a.err = c->err;
    return a;
}

template <typename real>
static rbmd_status rbl_pairs_t(rbmd_ctx *c, StepRef s, void *force, int accumulate, bool energy,
                               int32_t *n_core, int32_t *n_shell, int32_t *batch, bool marks)
{
    PairArgs<real> a = pair_args<real>(c, s);
    a.F = (real *)force;
    a.accumulate = accumulate;
    a.n_core = n_core;
    a.n_shell = n_shell;
    a.batch = batch;
    RBMD_CHECK_CUDA(cudaMemsetAsync(c->ibuf + 2, 0, sizeof(int32_t), c->stream));
    const bool lists = n_core != nullptr;
    const int p = c->prm.rbl_p;
    if (p > 32 && c->list_cs > SEL_WARP_MAX_CS) return RBMD_ERR_UNSUPPORTED;
    if (p <= 10) launch_rbl<real, 10>(c, a, c->stream, energy, lists, marks);
    else if (p <= 16) launch_rbl<real, 16>(c, a, c->stream, energy, lists, marks);
    else if (p <= 32) launch_rbl<real, 32>(c, a, c->stream, energy, lists, marks);
    else launch_rbl<real, 1024>(c, a, c->stream, energy, lists, marks);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Lists and batches of step s only (Algorithm 2 step 1), for the adjoint.
template <typename real>
static rbmd_status rbl_lists_t(rbmd_ctx *c, StepRef s)
{
    PairArgs<real> a = pair_args<real>(c, s);
    RBMD_CHECK_CUDA(cudaMemsetAsync(c->ibuf, 0, 3 * sizeof(int32_t), c->stream));
    const unsigned nb256 = (unsigned)c->nb256;
    k_rbl_scan<real, true, false><<<nb256, 256, 0, c->stream>>>(a);
    if (!a.exact) {
        const int p = c->prm.rbl_p;
        if (p > 32 && c->list_cs > SEL_WARP_MAX_CS) return RBMD_ERR_UNSUPPORTED;
        if (p <= 10) launch_select<real, 10, false>(a, nb256, c->stream);
        else if (p <= 16) launch_select<real, 16, false>(a, nb256, c->stream);
        else if (p <= 32) launch_select<real, 32, false>(a, nb256, c->stream);
        else launch_select<real, 1024, false>(a, nb256, c->stream);
    }
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

__global__ void k_max_counts(const int2 *__restrict__ cnt, int64_t N, int32_t *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int2 c = i < N ? cnt[i] : make_int2(0, 0);
    const int mx = __reduce_max_sync(0xffffffffu, c.x), my = __reduce_max_sync(0xffffffffu, c.y);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, mx);
        atomicMax(out + 1, my);
    }
}

rbmd_status rbl_lists(rbmd_ctx *c, StepRef s)
{
    c->lists_cached = false;
    if (c->fp64) return rbl_lists_t<double>(c, s);
    return rbl_lists_t<float>(c, s);
}

rbmd_status rbl_max_counts(rbmd_ctx *c, int32_t *out_dev)
{
    RBMD_CHECK_CUDA(cudaMemsetAsync(out_dev, 0, 2 * sizeof(int32_t), c->stream));
    k_max_counts<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->ncount, c->N, out_dev);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status rbl_pairs(rbmd_ctx *c, StepRef s, void *force, int accumulate, bool energy,
                      int32_t *n_core, int32_t *n_shell, int32_t *batch, bool marks)
{
    c->lists_cached = false;
    if (c->fp64)
        return rbl_pairs_t<double>(c, s, force, accumulate, energy, n_core, n_shell, batch, marks);
    return rbl_pairs_t<float>(c, s, force, accumulate, energy, n_core, n_shell, batch, marks);
}

// ---------------------------------------------------------------- the step's candidate lists
//
// The integrator's short-range part keeps, per cell-sorted atom, the list of its
// candidates: every atom within Rv of it at the last rebuild (Rv = Rlin + 1 + 2h
// fixed-point units, h = floor(skin/2 in units)), and keeps the sorted order of
// that rebuild between rebuilds (positions gathered into it every step).  A
// rebuild happens when some atom's displacement d since the rebuild has
// |d|^2 > h^2 (exact integers).  Until then every pair with D <= Rs2 is on the
// candidate list: with |d_i|, |d_j| <= h, the rebuild's separation satisfies
// |r_ref| <= |r_now| + 2h < Rlin + 1 + 2h = Rv.  Every step classifies the
// candidates exactly (core D < Rc2, shell Rc2 <= D <= Rs2, as classify), so the
// core list, N_s and the batch are the sets the cell walk gives; the core list
// and a whole-shell batch are put in atom-id order and a drawn batch is in
// priority order, so the pair sums do not depend on when the lists were built.
struct VlArgs {
    const int32_t *cand;  // [ceil(N/32)][cv][32]
    int32_t *cand_w;      // the same array, written by the rebuild
    int32_t *ncand;
    uint4 *sref;
    int32_t *flag;        // rebuild pending
    int32_t *nrebuild;
    int cv, ccs;
    int core_rows;        // max(ccs, p): rows of k_rbl_vsel's core-id array
    int32_t *imax;        // when set: the largest N_s (atomicMax, one per warp)
};



__device__ __forceinline__ int64_t vl_slot(int64_t is, int t, int cv)
{
    return (is >> 5) * (int64_t)cv * 32 + (int64_t)t * 32 + (is & 31);
}


// Positions of the current state in the sorted order of the last rebuild, and
// the displacement test that asks for a rebuild.  Nothing to do when a rebuild is
// already pending (it sorts the state afresh).
__global__ void k_vl_gather(const Rep *__restrict__ reps, const int2 *__restrict__ map,
                            uint4 *__restrict__ spos, const uint4 *__restrict__ u4,
                            const uint4 *__restrict__ sref, int32_t *__restrict__ flag,
                            int64_t N, int *__restrict__ err)
{
    if (*flag) return;
    const AtomSlot sl = atom_slot(map, reps);
    if (!sl.ok) return;
    const uint32_t id = spos[sl.i].w;
    const uint4 U = u4[RBMD_IDX(id, N, err)];
    spos[sl.i] = make_uint4(U.x, U.y, U.z, id);
    const uint4 R = sref[sl.i];
    const int32_t dx = (int32_t)(U.x - R.x), dy = (int32_t)(U.y - R.y), dz = (int32_t)(U.z - R.z);
    const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                       (uint64_t)((int64_t)dz * dz);
    if (D > reps[sl.r].H2) *flag = 1;
}

// Rebuild (only when *flag): every atom within Rv of each sorted atom, from the
// freshly sorted cells (stencil culled at r_cut + skin), and the reference
// positions.
template <typename real>
__global__ void __launch_bounds__(256) k_vl_build(PairArgs<real> a, VlArgs v)
{
    if (!*v.flag) return;
    const AtomSlot sl = atom_slot(a.map, a.reps);
    if (!sl.ok) return;
    const int64_t is = sl.i;
    const Rep rp = a.reps[sl.r];
    const uint4 A = a.spos[is];
    v.sref[is] = A;
    const uint32_t R2x = 2u * rp.Rv;
    int n = 0;
    stencil_ranges(a, rp, A, [&](int kb, int ke) {
        for (int k = kb; k < ke; ++k) {
            const uint4 B = a.spos[RBMD_IDX(k, a.N, a.err)];
            const int32_t dx = (int32_t)(B.x - A.x), dy = (int32_t)(B.y - A.y),
                          dz = (int32_t)(B.z - A.z);
            if (((uint32_t)dx + rp.Rv > R2x) | ((uint32_t)dy + rp.Rv > R2x) |
                ((uint32_t)dz + rp.Rv > R2x) | (k == (int)is))
                continue;
            const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                               (uint64_t)((int64_t)dz * dz);
            if (D > rp.Rv2) continue;
            if (n < v.cv) v.cand_w[vl_slot(is, n, v.cv)] = k;
            ++n;
        }
    });
    v.ncand[is] = n;
}

__global__ void k_vl_done(int32_t *__restrict__ flag, int32_t *__restrict__ nrebuild)
{
    if (*flag) {
        *flag = 0;
        ++*nrebuild;
    }
}

// Ascending insertion sort of n values at v[0], v[s], v[2s], ...
__device__ __forceinline__ void sort_strided(int32_t *v, int n, int s)
{
    for (int e = 1; e < n; ++e) {
        const int32_t x = v[e * s];
        int y = e - 1;
        while (y >= 0 && v[y * s] > x) {
            v[(y + 1) * s] = v[y * s];
            --y;
        }
        v[(y + 1) * s] = x;
    }
}

// The exact batch of one atom from its candidates (full 64-bit priorities, ties
// to the smaller id), for the rare atoms whose truncated keys tie: fills hk as
// select_exact does (replica-local ids).
template <int CAP>
__device__ __noinline__ void vl_select_exact(const Philox0 &r0, uint2 key, const Rep &rp,
                                             const uint4 A, const uint4 *spos, const int32_t *cl,
                                             int n, uint32_t id0, int p, int (&hk)[CAP])
{
    uint64_t kk[CAP];
    uint32_t kid[CAP];
    int kept = 0;
    for (int t = 0; t < n; ++t) {
        const uint4 B = spos[cl[t * 32]];
        if (classify_near(rp, A, B) != 2) continue;
        const uint32_t id = B.w - id0;
        const uint2 w = philox_rest(r0, id, key);
        const uint64_t v = ((uint64_t)w.x << 32) | w.y;
        int j;
        if (kept == p) {
            if (!(v < kk[p - 1] || (v == kk[p - 1] && id < kid[p - 1]))) continue;
            j = p - 1;
        } else {
            j = kept;
        }
        while (j > 0 && (v < kk[j - 1] || (v == kk[j - 1] && id < kid[j - 1]))) {
            kk[j] = kk[j - 1];
            kid[j] = kid[j - 1];
            --j;
        }
        kk[j] = v;
        kid[j] = id;
        if (kept < p) ++kept;
    }
    for (int e = 0; e < CAP; ++e) {
        const int j = e - (CAP - p);
        hk[e] = j < 0 ? SEL_NEG : (j < kept ? (int)kid[j] : SEL_POS);
    }
}

// The CAP + 1 smallest of the kept keys sk (ascending) and four new keys x, into
// sk.  For CAP + 5 <= 32 a bitonic merge: x sorted descending after sk and
// all-ones padding makes one bitonic sequence, which log2 of its length
// compare-exchange stages sort (a dependency chain of 5 or so instead of the
// 4 (CAP + 1) of inserting the keys one by one); larger CAP insert one by one.
// The kept set is the same either way.
template <int CAP>
__device__ __forceinline__ void merge4(uint32_t (&sk)[CAP + 1], uint32_t (&x)[4])
{
    constexpr int M = CAP + 1;
    if constexpr (M + 4 <= 32) {
        constexpr int NP = M + 4 <= 16 ? 16 : 32;
        auto ce = [](uint32_t &lo, uint32_t &hi) {  // lo <- min, hi <- max
            const uint32_t a = min(lo, hi), b = max(lo, hi);
            lo = a;
            hi = b;
        };
        ce(x[1], x[0]);  // descending
        ce(x[3], x[2]);
        ce(x[2], x[0]);
        ce(x[3], x[1]);
        ce(x[2], x[1]);
        uint32_t v[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) v[i] = 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < M; ++i) v[i] = sk[i];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[NP - 4 + q] = x[q];
#pragma unroll
        for (int j = NP >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < NP; ++i)
                if ((i & j) == 0) ce(v[i], v[i + j]);
#pragma unroll
        for (int i = 0; i < M; ++i) sk[i] = v[i];
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t y = x[q];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const uint32_t m = min(sk[j], y);
                y = max(sk[j], y);
                sk[j] = m;
            }
        }
    }
}

// Algorithm 2 step 1 for the step: classification of the candidates, N_s, the
// batch and the core list, one thread per sorted atom (128 per block).  The shell
// is never stored.  A lane classifies four candidates per round and queues its
// shell members (replica-local id, candidate position) in a 16-entry ring in
// shared memory; the warp computes Philox priorities four per lane at once (four
// interleaved chains) when every lane has four queued or has finished its list,
// or when some lane's ring is three-quarters full, so that the priorities are
// computed for shell members only and mostly with all lanes busy.  The bottom-p
// keys of select_atom are kept in registers, keyed by the candidate's position
// in the list, so a winner's sorted index is its candidate entry; the kept set
// does not depend on the order the keys arrive in.  Shared memory: the core
// members' replica-local ids, [max(ccs, p)][128] int32, put in id order, then the
// rings, [16][128] uint2.  Outputs: lcore and bk rows (sorted indices) and
// ncount, read by k_rbl_force.  An atom beyond a capacity is marked overflowed
// for the exact fallback.
template <typename real, int CAP>
__global__ void __launch_bounds__(128) k_rbl_vsel(PairArgs<real> a, VlArgs v)
{
    extern __shared__ int32_t s_vl[];
    constexpr unsigned FULL = 0xFFFFFFFFu;
    // every lane runs to the end: the warp votes on when to compute priorities
    const AtomSlot sl = atom_slot(a.map, a.reps);
    const int64_t is = sl.i;
    const Rep rp = a.reps[sl.r];
    const uint4 A = sl.ok ? a.spos[is] : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t id0 = (uint32_t)rp.atom0;
    int32_t *s_core = s_vl + threadIdx.x;
    uint2 *s_ring = reinterpret_cast<uint2 *>(s_vl + v.core_rows * 128) + threadIdx.x;
    const int n_all = sl.ok ? v.ncand[is] : 0;
    const int n = n_all <= v.cv ? n_all : 0;  // beyond the capacity: the fallback
    const int32_t *cl = v.cand + vl_slot(is, 0, v.cv);
    const Philox0 r0 = philox_round0(A.w - id0, (uint32_t)step_of(a.step), rp.tag_rbl, rp.key);
    const PhiloxKeys K = philox_keys(rp.key);
    const int b = 32 - __clz(v.cv);  // 2^b > cv > every candidate position
    const uint32_t lo_mask = (1u << b) - 1u;
    uint32_t keep = ~lo_mask;
    if (a.sel_key_bits > 0 && a.sel_key_bits < 32) keep &= ~(0xFFFFFFFFu >> a.sel_key_bits);
    uint32_t sk[CAP + 1];
#pragma unroll
    for (int e = 0; e <= CAP; ++e) sk[e] = 0xFFFFFFFFu;
    int nc = 0, ns = 0;
    int head = 0, cnt = 0;  // the ring holds entries head .. head + cnt - 1 (mod 16)
    // up to four queued members: their priorities, their keys into the kept set
    auto drain4 = [&]() {
        uint32_t id4[4], t4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint2 e = q < cnt ? s_ring[((head + q) & 15) * 128] : make_uint2(0u, FULL);
            id4[q] = e.x;
            t4[q] = e.y;
        }
        const int took = min(cnt, 4);
        head += took;
        cnt -= took;
        uint2 w[4];
        philox_rest4(r0, id4, K, w);
        uint32_t x4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x4[q] = t4[q] != FULL ? (w[q].x & keep) | t4[q] : FULL;
        merge4<CAP>(sk, x4);
    };
    {
        // four candidates per round: their positions are gathered one round
        // ahead and their indices (one coalesced row of the warp each) two rounds
        // ahead, so the gathers overlap the previous round's work
        constexpr int VB = 4;
        int kk[VB];
        uint4 Bn[VB];
#pragma unroll
        for (int q = 0; q < VB; ++q) {
            const int k0 = q < n ? cl[q * 32] : -1;
            Bn[q] = k0 >= 0 ? a.spos[RBMD_IDX(k0, a.N, a.err)] : A;
            kk[q] = VB + q < n ? cl[(VB + q) * 32] : -1;
        }
        for (int t0 = 0; __any_sync(FULL, t0 < n); t0 += VB) {
            uint4 B[VB];
#pragma unroll
            for (int q = 0; q < VB; ++q) {
                B[q] = Bn[q];
                Bn[q] = kk[q] >= 0 ? a.spos[RBMD_IDX(kk[q], a.N, a.err)] : A;
                kk[q] = t0 + 2 * VB + q < n ? cl[(t0 + 2 * VB + q) * 32] : -1;
            }
#pragma unroll
            for (int q = 0; q < VB; ++q) {
                const int cls = t0 + q < n ? classify_near(rp, A, B[q]) : 0;
                const uint32_t id = B[q].w - id0;
                if (cls == 1) {
                    if (nc < v.ccs) s_core[nc * 128] = (int32_t)id;
                    ++nc;
                } else if (cls == 2) {
                    s_ring[((head + cnt) & 15) * 128] = make_uint2(id, (uint32_t)(t0 + q));
                    ++cnt;
                    ++ns;
                }
            }
            // before the pushes every ring holds at most 11 (else the warp drained
            // four from each), so it never exceeds 15
            const bool go = __all_sync(FULL, cnt >= 4 || t0 + VB >= n) | __any_sync(FULL, cnt >= 12);
            if (go) drain4();
        }
        while (__any_sync(FULL, cnt > 0)) drain4();
    }
    if (v.imax) {
        const int m = __reduce_max_sync(FULL, sl.ok ? ns : 0);
        if ((threadIdx.x & 31) == 0) atomicMax(v.imax, m);
    }
    if (!sl.ok) return;
    if (n_all > v.cv || nc > v.ccs || nc > a.CC) {
        a.ncount[is] = make_int2(a.CC + 1, 0);
        *a.ovf = 1;
        return;
    }
    const int32_t *sidx = a.sidx + id0;
    int32_t *lc = a.lcore + is * a.CC;
    if (nc <= 16) {
        int32_t r[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) r[e] = e < nc ? s_core[e * 128] : 0x7FFFFFFF;
        sort16(r);
#pragma unroll
        for (int e = 0; e < 16; ++e)
            if (e < nc) lc[e] = sidx[r[e]];
    } else {
        sort_strided(s_core, nc, 128);
        for (int e = 0; e < nc; ++e) lc[e] = sidx[s_core[e * 128]];
    }
    int32_t *bk = a.bk + is * a.p;
    if (ns <= a.p && ns <= 16) {
        // the whole shell (its keys are all kept), in atom-id order
        int32_t r[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
            r[e] = e < ns && e <= CAP
                       ? (int32_t)(a.spos[RBMD_IDX(cl[(sk[e < CAP ? e : CAP] & lo_mask) * 32], a.N,
                                                   a.err)].w - id0)
                       : 0x7FFFFFFF;
        sort16(r);
#pragma unroll
        for (int e = 0; e < 16; ++e)
            if (e < ns) bk[e] = sidx[r[e]];
    } else if (ns <= a.p) {
#pragma unroll
        for (int e = 0; e < CAP; ++e)
            if (e < ns)
                s_core[e * 128] =
                    (int32_t)(a.spos[RBMD_IDX(cl[(sk[e] & lo_mask) * 32], a.N, a.err)].w - id0);
        sort_strided(s_core, ns, 128);
        for (int e = 0; e < ns; ++e) bk[e] = sidx[s_core[e * 128]];
    } else {
        bool tie = a.sel_exact != 0;
#pragma unroll
        for (int e = 0; e < CAP; ++e)
            if (e < a.p) tie |= ((sk[e] ^ sk[e + 1]) & keep) == 0u;
        if (!tie) {
#pragma unroll
            for (int e = 0; e < CAP; ++e)
                if (e < a.p) bk[e] = cl[(sk[e] & lo_mask) * 32];
        } else {
            int hk[CAP];
            vl_select_exact<CAP>(r0, rp.key, rp, A, a.spos, cl, n, id0, a.p, hk);
            int nb = 0;
            for (int e = 0; e < CAP; ++e)
                if (hk[e] >= 0) bk[nb++] = sidx[hk[e]];
        }
    }
    a.ncount[is] = make_int2(nc, ns);
}

template <typename real>
static VlArgs vl_args(rbmd_ctx *c)
{
    VlArgs v;
    v.cand = c->vl_cand;
    v.cand_w = c->vl_cand;
    v.ncand = c->vl_ncand;
    v.sref = c->vl_sref;
    v.flag = c->ibuf + 4;
    v.nrebuild = c->ibuf + 5;
    v.cv = c->vl_cv;
    v.ccs = c->vl_ccs;
    v.core_rows = std::max(c->vl_ccs, c->prm.rbl_p);
    v.imax = nullptr;
    return v;
}

// The rebuild of the candidate lists when *flag is set (every kernel checks it).
template <typename real>
static rbmd_status vl_rebuild(rbmd_ctx *c, int32_t *flag)
{
    RBMD_CHECK(cells_sort(c, false, flag));
    PairArgs<real> a = pair_args<real>(c, StepRef{nullptr, 0});
    a.stale = 1;  // cull at r_cut + skin: the candidates reach Rv
    k_vl_build<real><<<c->nb256, 256, 0, c->stream>>>(a, vl_args<real>(c));
    RBMD_LAUNCH_CHECK();
    k_vl_done<<<1, 1, 0, c->stream>>>(flag, c->ibuf + 5);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Opens the conditional node of the step graph when the displacement test found a
// rebuild due.
__global__ void k_vl_cond(const int32_t *__restrict__ flag, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, *flag != 0 ? 1u : 0u);
}

// Inside the capture of the step graph: the rebuild kernels become the body of a
// conditional (if) node that k_vl_cond opens on the steps whose displacement test
// asks for a rebuild, so the other steps launch none of them.  Returns false,
// with nothing captured, when the node cannot be made (the caller then captures
// the device-conditional kernels themselves).
template <typename real>
static bool vl_rebuild_node(rbmd_ctx *c, int32_t *flag, rbmd_status *st)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle h;
    if (!c->cond_stream &&
        cudaStreamCreateWithFlags(&c->cond_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->cond_stream = nullptr;
        cudaGetLastError();
        return false;
    }
    if (cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive ||
        cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    *st = RBMD_OK;
    k_vl_cond<<<1, 1, 0, c->stream>>>(flag, h);
    if (cudaGetLastError() != cudaSuccess ||
        cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess) {
        *st = RBMD_ERR_CUDA;
        return true;
    }
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};  // the rest zero
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, ed, nd, &np) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess ||
        cudaStreamBeginCaptureToGraph(c->cond_stream, np.conditional.phGraph_out[0], nullptr,
                                      nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        *st = RBMD_ERR_CUDA;
        return true;
    }
    const cudaStream_t main = c->stream;
    c->stream = c->cond_stream;
    *st = vl_rebuild<real>(c, flag);
    c->stream = main;
    cudaGraph_t body;
    if (cudaStreamEndCapture(c->cond_stream, &body) != cudaSuccess && *st == RBMD_OK)
        *st = RBMD_ERR_CUDA;
    size_t nn = 0;
    if (*st == RBMD_OK) cudaGraphGetNodes(np.conditional.phGraph_out[0], nullptr, &nn);
    c->graph_cond_kernels = (int32_t)nn;  // kernel nodes only: the body holds nothing else
    return true;
}

template <typename real>
static rbmd_status verlet_prepare_t(rbmd_ctx *c)
{
    int32_t *flag = c->ibuf + 4;
    k_vl_gather<<<c->nb256, 256, 0, c->stream>>>(c->reps, c->map256, c->spos, c->u4, c->vl_sref,
                                                  flag, c->N, c->err);
    RBMD_LAUNCH_CHECK();
    rbmd_status st = RBMD_OK;
    if (c->capturing && c->cond_nodes && vl_rebuild_node<real>(c, flag, &st)) {
        // a failed node fails this capture; the next one uses plain graph nodes
        if (st != RBMD_OK) c->cond_nodes = false;
        return st;
    }
    return vl_rebuild<real>(c, flag);
}

rbmd_status verlet_prepare(rbmd_ctx *c)
{
    if (c->fp64) return verlet_prepare_t<double>(c);
    return verlet_prepare_t<float>(c);
}

static size_t vl_smem(const rbmd_ctx *c)
{
    return (size_t)std::max(c->vl_ccs, c->prm.rbl_p) * 128 * sizeof(int32_t) +
           (size_t)16 * 128 * sizeof(uint2);
}

// energy: the pair kernels also sum the energies and virials, and the selection
// records the largest N_s; pairs = false: the lists only (for the adjoint)
template <typename real, int CAP>
static void launch_vl(rbmd_ctx *c, const PairArgs<real> &a, bool marks, bool energy, bool pairs)
{
    PairArgs<real> a128 = a;
    a128.map = c->map128;
    a128.nmap = c->nb128;
    const unsigned nbp = (unsigned)c->nb128;
    const unsigned nfb = (unsigned)min(c->nb128, 4 * 148);
    VlArgs v = vl_args<real>(c);
    if (energy) v.imax = c->ibuf;
    k_rbl_vsel<real, CAP><<<nbp, 128, vl_smem(c), c->stream>>>(a128, v);
    if (marks) {
        prof_mark(c, 3);
        prof_mark(c, 4);
    }
    if (!pairs) return;
    if (energy) {
        if (a.tab) k_rbl_force<real, true, true><<<nbp, kPairBlock, 0, c->stream>>>(a128);
        else k_rbl_force<real, true, false><<<nbp, kPairBlock, 0, c->stream>>>(a128);
        k_rbl_fused<real, CAP, true, false><<<nfb, kPairBlock, 0, c->stream>>>(a128);
    } else {
        if (a.tab) k_rbl_force<real, false, true><<<nbp, kPairBlock, 0, c->stream>>>(a128);
        else k_rbl_force<real, false, false><<<nbp, kPairBlock, 0, c->stream>>>(a128);
        k_rbl_fused<real, CAP, false, false><<<nfb, kPairBlock, 0, c->stream>>>(a128);
    }
}

template <typename real>
static rbmd_status rbl_pairs_verlet_t(rbmd_ctx *c, StepRef s, void *force, bool marks, bool energy,
                                      bool pairs)
{
    PairArgs<real> a = pair_args<real>(c, s);
    a.F = (real *)force;
    a.accumulate = 0;
    a.stale = 1;  // the fallback walks the cells of the last rebuild
    RBMD_CHECK_CUDA(cudaMemsetAsync(c->ibuf + 2, 0, sizeof(int32_t), c->stream));
    if (c->prm.rbl_p <= 10) launch_vl<real, 10>(c, a, marks, energy, pairs);
    else if (c->prm.rbl_p <= 16) launch_vl<real, 16>(c, a, marks, energy, pairs);
    else launch_vl<real, 32>(c, a, marks, energy, pairs);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status rbl_pairs_verlet(rbmd_ctx *c, StepRef s, void *force, bool marks, bool energy)
{
    c->lists_cached = false;
    if (c->fp64) return rbl_pairs_verlet_t<double>(c, s, force, marks, energy, true);
    return rbl_pairs_verlet_t<float>(c, s, force, marks, energy, true);
}

// The core lists, batches and counts of step s from the candidates (after
// verlet_prepare), without the pair forces; an atom beyond a capacity sets the
// overflow word (ibuf[2]) as in the cell walk.
rbmd_status rbl_lists_verlet(rbmd_ctx *c, StepRef s)
{
    c->lists_cached = false;
    if (c->fp64) return rbl_pairs_verlet_t<double>(c, s, nullptr, false, false, false);
    return rbl_pairs_verlet_t<float>(c, s, nullptr, false, false, false);
}

rbmd_status verlet_configure(rbmd_ctx *c)
{
    if (!c->verlet) return RBMD_OK;
    const int bytes = (int)vl_smem(c);
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_vsel<float, 10>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_vsel<float, 16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_vsel<double, 10>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_vsel<double, 16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_vsel<float, 32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rbl_vsel<double, 32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return RBMD_OK;
}

// ---------------------------------------------------------------- correction
template <typename real>
__global__ void k_add_corr(real *__restrict__ F, const int2 *__restrict__ map,
                           const Rep *__restrict__ reps, const double *__restrict__ scal, int slot)
{
    const AtomSlot sl = atom_slot(map, reps);
    if (!sl.ok) return;
    const double *fc = scal + (int64_t)sl.r * SCAL_COUNT + slot;
    F[3 * sl.i + 0] += (real)fc[0];
    F[3 * sl.i + 1] += (real)fc[1];
    F[3 * sl.i + 2] += (real)fc[2];
}

// F_corr = -(1/N_r) sum_{i in r} (F_core + F_shell*) per replica (Eq. 16,
// Algorithm 2 step 3) into its scalars [slot, slot + 3); with apply, added to
// every atom of `force` (Algorithm 2 step 4).  The integrator keeps its
// correction in SCAL_FCORR and adds it in the kicks instead of in a separate pass.
rbmd_status rbl_correction(rbmd_ctx *c, void *force, bool apply, int slot)
{
    RBMD_CHECK(md_sum_replicas_fix(c, c->fpart, slot, -1.0, true, true));
    if (apply) {
        if (c->fp64)
            k_add_corr<double><<<c->nb256, 256, 0, c->stream>>>((double *)force, c->map256, c->reps,
                                                                c->scal, slot);
        else
            k_add_corr<float><<<c->nb256, 256, 0, c->stream>>>((float *)force, c->map256, c->reps,
                                                               c->scal, slot);
        RBMD_LAUNCH_CHECK();
    }
    return RBMD_OK;
}

}  // namespace rbmd
