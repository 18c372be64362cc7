// Adjoint of the total potential (rbmd_energy_backward): gradients of
//   E = E_coul_real + E_lj + E_rbe + E_self
// with respect to positions, charges and the per-type LJ parameters, with the
// random draws of the step held fixed.  The paper gives forces only; this is
// the gradient of its energy expressions (Eqs. 2, 4, 8, 10 with the random-batch
// estimators of Eqs. 12 and 15):
//   E_RBL = 1/2 sum_i sum_j W_ij u_ij,  W_ij = 1 (j in C(i)), N_s(i)/p (j in B(i));
// since the lists are one-sided, dE/dr_k = sum_j 1/2 (W_kj + W_jk) u'(r_kj) r_hat.
// W_jk is nonzero for a shell neighbour j of k only when k is in j's batch, so the
// kernel walks three lists per atom: its core (weight 1 both ways), its batch
// (1/2 W_kj) and its reverse batch, the atoms whose batch holds k (1/2 W_jk),
// built by scattering every batch entry before the kernel runs.
#include <math.h>

#include "rbmd_internal.cuh"

namespace rbmd {

// d_pos = 0, d_q = g * dE_self/dq = -2 g coulomb_k sqrt(alpha/pi) q
template <typename real>
__global__ void k_adj_init(real *__restrict__ dpos, real *__restrict__ dq,
                           const uint4 *__restrict__ u4, const double *__restrict__ q64,
                           int64_t N, double gself)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (dpos) {
        dpos[3 * i] = 0;
        dpos[3 * i + 1] = 0;
        dpos[3 * i + 2] = 0;
    }
    if (dq) {
        double q;
        if constexpr (sizeof(real) == 4) q = (double)__uint_as_float(u4[i].w);
        else q = q64[i];
        dq[i] = (real)(gself * q);
    }
}

template <typename real> struct AdjArgs {
    const Rep *reps;
    const int2 *map;        // replica-aligned 128-atom blocks
    const uint4 *spos;
    const real *sq;
    const int32_t *stype;
    const int32_t *lcore, *lshell, *bk;  // per-atom lists, entry e of atom i at lidx(i, e, N, cap)
    int32_t *rb;                         // reverse batches, [N][RC] sorted indices (each row
                                         // sorted in place by its own atom's thread)
    int RC;                              // their capacity (>= CS: never exceeded)
    const int32_t *rbn;                  // reverse-batch counts
    const int32_t *sidx;                 // sorted index of every atom (by global id)
    const int2 *ncount;
    int64_t N;
    int CC, CS, p, T, exact;
    real ck, alpha, sqrt_alpha, c2;
    const real *eps, *sig;  // per type (host values copied in)
    const real *pairtab;    // [4][T][T]: 1/2 sqrt(eps_t2/eps_t1), 1/sigma_t1t2, eps_t1t2, sigma_t1t2
    double g;               // grad_out
    real *dpos, *dq;
    double *tpart;          // [blocks][2T] per-block (d eps, d sigma) partial sums
};

__device__ __forceinline__ float erfc_a(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_a(double x) { return erfc(x); }
__device__ __forceinline__ float exp_a(float x) { return expf(x); }
__device__ __forceinline__ double exp_a(double x) { return exp(x); }
__device__ __forceinline__ float sqrt_a(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_a(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrt_a(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_a(double x) { return 1.0 / sqrt(x); }

constexpr int ADJ_BLOCK = 128;

// acc[t] += v for a run-time type t < TT: TT <= 8 keeps the accumulators in
// registers (an unrolled select), larger TT index an array.
template <typename real, int TT>
__device__ __forceinline__ void acc_add(real (&acc)[2 * TT], int t, real v)
{
    if constexpr (TT <= 8) {
#pragma unroll
        for (int u = 0; u < 2 * TT; ++u)
            if (u == t) acc[u] += v;
    } else {
        acc[t] += v;
    }
}

// One thread per cell-sorted atom k, over its core (weight W = 1), its batch
// (W = w_k / 2) and its reverse batch (the atoms j whose batch holds k, W = w_j / 2):
// the symmetric weights of dE/dr and dE/dq.  The eps and sigma sums follow the same
// visits.  An ordered pair (k, j) of one-sided weight W_kj adds 1/2 W_kj du/d eps_kj
// times d eps_kj/d eps_t = [t = t_k] a_kj + [t = t_j] a_jk (a_kj = 1/2 sqrt(eps_j /
// eps_k), Eq. 4); the [t = t_j] part of (k, j) is the [t = t_k] part of the reversed
// pair seen from k, so each visit adds W du/d eps_kj a_kj (and W du/d sigma_kj / 2)
// to k's own type only.  TT >= the number of LJ types.
template <typename real, int TT>
__global__ void __launch_bounds__(ADJ_BLOCK) k_rbl_adjoint(AdjArgs<real> a)
{
    __shared__ double s_t[2 * TT][ADJ_BLOCK / 32];
    // type-pair factors of the eps and sigma derivatives (Eq. 4), TT <= 16:
    // [tk TT + tj] = 1/2 sqrt(eps_j / eps_k) and 1 / sigma_kj
    constexpr int TP = TT <= 16 ? TT * TT : 1;
    __shared__ real s_er[TP], s_is[TP], s_e[TP], s_s[TP];  // + eps_kj and sigma_kj (Eq. 4)
    if constexpr (TT <= 16) {
        // from the table the host computed once per set of parameters
        const int T2 = a.T * a.T;
        for (int u = threadIdx.x; u < T2; u += blockDim.x) {
            const int t1 = u / a.T, t2 = u % a.T;
            s_er[t1 * TT + t2] = a.pairtab[u];
            s_is[t1 * TT + t2] = a.pairtab[T2 + u];
            s_e[t1 * TT + t2] = a.pairtab[2 * T2 + u];
            s_s[t1 * TT + t2] = a.pairtab[3 * T2 + u];
        }
        __syncthreads();
    }
    // per-thread type sums in the working precision (a few tens of pairs), warp sums
    // too; the block and type sums are FP64
    real acc[2 * TT];
#pragma unroll
    for (int t = 0; t < 2 * TT; ++t) acc[t] = 0;
    const AtomSlot sl = atom_slot(a.map, a.reps);
    const int64_t ks = sl.i;
    if (sl.ok) {
        const real lscale = (real)a.reps[sl.r].lscale;
        const uint4 A = a.spos[ks];
        const real qk = a.sq[ks];
        const int tk = a.stype[ks];
        const int2 cnt = a.ncount[ks];
        const int nbk = min(cnt.y, a.p);
        const real wk = cnt.y > a.p ? (real)cnt.y / (real)a.p : (real)1;
        const int64_t N = a.N;
        const uint32_t id0 = (uint32_t)a.reps[sl.r].atom0;
        real gx = 0, gy = 0, gz = 0, gq = 0;
        real ak_e = 0, ak_s = 0;  // the type sums of k's own type, added to acc at the end
        // one pair (k, js) of symmetric weight W
        struct Nb {  // a neighbour's record; its counts only on the reverse batch
            uint4 B;
            int tj;
            real qj;
            int2 cj;
        };
        auto load = [&](int32_t js, bool counts) {
            Nb n;
            n.B = a.spos[js];
            n.tj = a.stype[js];
            n.qj = a.sq[js];
            n.cj = counts ? a.ncount[js] : make_int2(0, 0);
            return n;
        };
        auto pair = [&](const Nb &nb, real W) {
            const uint4 B = nb.B;
            const real dx = (real)(int32_t)(B.x - A.x) * lscale;  // r_j - r_k
            const real dy = (real)(int32_t)(B.y - A.y) * lscale;
            const real dz = (real)(int32_t)(B.z - A.z) * lscale;
            const real r2 = dx * dx + dy * dy + dz * dz;
            const real rinv = rsqrt_a(r2);
            const real r = r2 * rinv;
            const int tj = nb.tj;
            const real qj = nb.qj;
            real eij, sij;
            if constexpr (TT <= 16) {
                eij = s_e[tk * TT + tj];
                sij = s_s[tk * TT + tj];
            } else {
                eij = sqrt_a(a.eps[tk] * a.eps[tj]);
                sij = (real)0.5 * (a.sig[tk] + a.sig[tj]);
            }
            const real s2 = sij * sij * rinv * rinv;
            const real s6 = s2 * s2 * s2, s12 = s6 * s6;
            const real er = erfc_a(a.sqrt_alpha * r);
            // u'(r) of erfc-Coulomb and LJ
            const real du = -a.ck * qk * qj * (er * rinv * rinv + a.c2 * exp_a(-a.alpha * r2) * rinv) -
                            (real)24 * eij * ((real)2 * s12 - s6) * rinv;
            // dE/dr_k: u'(r) (r_k - r_j)/r = -u'(r) d / r
            const real f = W * du * rinv;
            gx -= f * dx;
            gy -= f * dy;
            gz -= f * dz;
            gq += W * a.ck * qj * er * rinv;
            // k's own type: W du/d eps_kj a_kj and W du/d sigma_kj / 2 (Eq. 4)
            const real due = (real)4 * (s12 - s6);
            real dus = (real)4 * eij * ((real)12 * s12 - (real)6 * s6);
            real rkj;
            if constexpr (TT <= 16) {
                dus *= s_is[tk * TT + tj];
                rkj = s_er[tk * TT + tj];
            } else {
                dus /= sij;
                rkj = (real)0.5 * sqrt_a(a.eps[tj] / a.eps[tk]);
            }
            ak_e += W * due * rkj;
            ak_s += W * dus * (real)0.5;
        };
        // a list of n neighbours, each one's loads issued before the previous pair is
        // computed; weight(nb) gives the pair's weight
        auto walk = [&](auto index, int n, bool counts, auto weight) {
            if (n <= 0) return;
            int32_t js = index(0);
            Nb cur = load(js, counts);
            for (int e = 0; e < n; ++e) {
                const int32_t jn = e + 1 < n ? index(e + 1) : js;
                const Nb nxt = load(jn, counts);
                pair(cur, weight(cur));
                cur = nxt;
                js = jn;
            }
        };
        auto ones = [](const Nb &) { return (real)1; };
        walk([&](int e) { return a.lcore[lidx(ks, e, N, a.CC)]; }, cnt.x, false, ones);
        if (a.exact) {
            walk([&](int e) { return a.sidx[id0 + (uint32_t)a.lshell[lidx(ks, e, N, a.CS)]]; },
                 cnt.y, false, ones);
        } else {
            walk([&](int e) { return a.bk[lidx(ks, e, N, a.p)]; }, nbk, false,
                 [&](const Nb &) { return (real)0.5 * wk; });
            // the reverse batch in ascending sorted index (the scatter's order is not
            // fixed): sorted in place, one row per thread
            int32_t *rrow = a.rb + lidx(ks, 0, N, a.RC);
            const int nrb = min(a.rbn[ks], a.RC);
            if (nrb <= 16) {
                // up to 16 entries (most rows: about p on average) in registers; the
                // loads and stores are independent
                int32_t r[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) r[i] = i < nrb ? rrow[i] : 0x7FFFFFFF;
                sort16(r);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < nrb) rrow[i] = r[i];
            } else {
                for (int e = 1; e < nrb; ++e) {
                    const int32_t x = rrow[e];
                    int y = e - 1;
                    while (y >= 0 && rrow[y] > x) {
                        rrow[y + 1] = rrow[y];
                        --y;
                    }
                    rrow[y + 1] = x;
                }
            }
            walk([&](int e) { return rrow[e]; }, nrb, true, [&](const Nb &nb) {
                const real wj = nb.cj.y > a.p ? (real)nb.cj.y / (real)a.p : (real)1;
                return (real)0.5 * wj;
            });
        }
        acc_add<real, TT>(acc, tk, ak_e);
        acc_add<real, TT>(acc, TT + tk, ak_s);
        const int64_t id = A.w;
        if (a.dpos) {
            a.dpos[3 * id] += (real)a.g * gx;
            a.dpos[3 * id + 1] += (real)a.g * gy;
            a.dpos[3 * id + 2] += (real)a.g * gz;
        }
        if (a.dq) a.dq[id] += (real)a.g * gq;
    }
    // per-type block partials, fixed order (eps of type t at acc[t], sigma at acc[TT + t]):
    // warp sums in the working precision, then FP64
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 2 * TT; ++t) {
        if ((t % TT) >= a.T) continue;
        real v = acc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_t[t][warp] = (double)v * a.g;
    }
    __syncthreads();
    if (threadIdx.x < 2 * a.T) {
        const int t = threadIdx.x < a.T ? threadIdx.x : TT + threadIdx.x - a.T;
        double v = 0.0;
        for (int w = 0; w < ADJ_BLOCK / 32; ++w) v += s_t[t][w];
        a.tpart[(int64_t)blockIdx.x * 2 * a.T + threadIdx.x] = v;
    }
}

// Reverse batches: for every batch entry j of atom k (sorted indices), k is
// appended to j's row.  A batch member is a shell member and the shell relation is
// symmetric, so a row never holds more than N_s(j) entries, at most the shell
// capacity on complete lists; a count beyond the row capacity latches an error
// instead of writing.
template <typename real>
__global__ void k_adj_reverse_batches(AdjArgs<real> a, int32_t *__restrict__ rb,
                                      int32_t *__restrict__ rbn, int *__restrict__ err)
{
    const AtomSlot sl = atom_slot(a.map, a.reps);
    if (!sl.ok) return;
    const int64_t ks = sl.i;
    const int nb = min(a.ncount[ks].y, a.p);
    for (int e = 0; e < nb; ++e) {
        const int32_t j = a.bk[lidx(ks, e, a.N, a.p)];
        const int pos = atomicAdd(rbn + j, 1);
        if (pos < a.RC) rb[lidx(j, pos, a.N, a.RC)] = (int32_t)ks;
        else latch_error(err, RBMD_ERR_CELL_OVERFLOW);
    }
}

// RBE part: dE/dr_i = -F_i (Eq. 12) and dE/dq_i = -sum_l (B_l cos th + A_l sin th),
// with the coefficients of the forward pass (A = c Im rho, B = c Re rho).
template <typename real, int CHUNK>
__global__ void k_rbe_adjoint(const uint4 *__restrict__ u4, const double *__restrict__ q64,
                              const int2 *__restrict__ map, const Rep *__restrict__ reps,
                              const ModeCoef<real> *__restrict__ coef_all, int64_t Pm, double g,
                              const double2 *__restrict__ ptab, real *__restrict__ dpos,
                              real *__restrict__ dq)
{
    __shared__ ModeCoef<real> s_c[CHUNK];
    const AtomSlot sl = atom_slot(map, reps);
    const int64_t i = sl.i;
    const bool active = sl.ok;
    const ModeCoef<real> *coef = coef_all + (int64_t)sl.r * Pm;
    const real tk = (real)(2.0 * kPi / reps[sl.r].L);
    const uint4 A = active ? u4[i] : make_uint4(0, 0, 0, 0);
    real fx = 0, fy = 0, fz = 0, phi = 0;
    for (int64_t c0 = 0; c0 < Pm; c0 += CHUNK) {
        const int nc = (int)min((int64_t)CHUNK, Pm - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < nc; k += blockDim.x) s_c[k] = coef[c0 + k];
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < nc; ++k) {
            const ModeCoef<real> mc = s_c[k];
            const uint32_t ph = (uint32_t)mc.mx * A.x + (uint32_t)mc.my * A.y + (uint32_t)mc.mz * A.z;
            real sn, cs;
            if constexpr (sizeof(real) == 4) phase_sincos(ph, sn, cs);  // as the force pass
            else phase_sincos_tab(ptab, ph, sn, cs);
            const real gg = mc.A * cs - mc.B * sn;
            fx += gg * mc.kx;
            fy += gg * mc.ky;
            fz += gg * mc.kz;
            phi -= mc.B * cs + mc.A * sn;
        }
    }
    if (!active) return;
    real q;
    if constexpr (sizeof(real) == 4) q = __uint_as_float(A.w);
    else q = q64[i];
    const real s = (real)g * q * tk;
    if (dpos) {
        dpos[3 * i] -= s * fx;
        dpos[3 * i + 1] -= s * fy;
        dpos[3 * i + 2] -= s * fz;
    }
    if (dq) dq[i] += (real)g * phi;
}

template <typename real>
static rbmd_status adjoint_t(rbmd_ctx *c, double g, void *dpos, void *dq, double *tsum_dev,
                             const double *eps_h, const double *sig_h)
{
    const unsigned nb = (unsigned)((c->N + 255) / 256);
    const double gself = -2.0 * g * c->prm.coulomb_k * sqrt(c->prm.alpha / kPi);
    gprof_mark(c, 2);
    k_adj_init<real><<<nb, 256, 0, c->stream>>>((real *)dpos, (real *)dq, c->u4, c->q64, c->N, gself);
    RBMD_LAUNCH_CHECK();
    gprof_mark(c, 3);
    if (!(c->prm.flags & RBMD_NO_RBL)) {
        AdjArgs<real> a;
        a.reps = c->reps;
        a.map = c->map128;
        a.spos = c->spos;
        a.sq = (const real *)c->sq;
        a.stype = c->stype;
        a.lcore = c->lcore;
        a.lshell = c->lshell;
        a.sidx = c->cell_rank;
        a.bk = c->bk;
        a.ncount = c->ncount;
        a.N = c->N;
        a.CC = c->list_cc;
        a.CS = c->list_cs;
        a.p = c->prm.rbl_p;
        a.T = c->T;
        a.exact = (c->prm.flags & RBMD_RBL_EXACT) ? 1 : 0;
        a.ck = (real)c->prm.coulomb_k;
        a.alpha = (real)c->prm.alpha;
        a.sqrt_alpha = (real)sqrt(c->prm.alpha);
        a.c2 = (real)(2.0 * sqrt(c->prm.alpha / kPi));
        a.eps = (const real *)c->adj_lj;
        a.sig = (const real *)c->adj_lj + c->T;
        a.pairtab = (const real *)c->adj_lj + 2 * c->T;
        a.g = g;
        a.dpos = (real *)dpos;
        a.dq = (real *)dq;
        a.tpart = c->adj_tpart;
        const unsigned nba = (unsigned)c->nb128;
        // reverse batches in their own array (allocated on the first use, for the
        // shell capacity: the lists the step keeps are left as they are) and their
        // counts in the scratch array
        if (!a.exact && c->adj_rb_cap < c->list_cs) {
            if (c->adj_rb) cudaFree(c->adj_rb);
            c->adj_rb = nullptr;
            c->adj_rb_cap = 0;
            RBMD_CHECK(dev_alloc(reinterpret_cast<void **>(&c->adj_rb),
                                 sizeof(int32_t) * (size_t)c->N * c->list_cs));
            c->adj_rb_cap = c->list_cs;
        }
        int32_t *rb = c->adj_rb, *rbn = (int32_t *)c->scratch_force;
        a.rb = rb;
        a.RC = c->adj_rb_cap;
        a.rbn = rbn;
        if (!a.exact) {
            RBMD_CHECK_CUDA(cudaMemsetAsync(rbn, 0, sizeof(int32_t) * (size_t)c->N, c->stream));
            k_adj_reverse_batches<real><<<nba, ADJ_BLOCK, 0, c->stream>>>(a, rb, rbn, c->err);
            RBMD_LAUNCH_CHECK();
        }
        if (c->T <= 4) k_rbl_adjoint<real, 4><<<nba, ADJ_BLOCK, 0, c->stream>>>(a);
        else if (c->T <= 16) k_rbl_adjoint<real, 16><<<nba, ADJ_BLOCK, 0, c->stream>>>(a);
        else k_rbl_adjoint<real, RBMD_MAX_TYPES><<<nba, ADJ_BLOCK, 0, c->stream>>>(a);
        RBMD_LAUNCH_CHECK();
        RBMD_CHECK(md_sum(c, c->adj_tpart, (int)nba, 2 * c->T, tsum_dev, 1.0));
    } else {
        RBMD_CHECK_CUDA(cudaMemsetAsync(tsum_dev, 0, sizeof(double) * 2 * c->T, c->stream));
    }
    gprof_mark(c, 4);
    if (!(c->prm.flags & RBMD_NO_RBE)) {
        if constexpr (sizeof(real) == 4)
            k_rbe_adjoint<float, 256><<<c->nb256, 256, 0, c->stream>>>(
                c->u4, nullptr, c->map256, c->reps, (const ModeCoef<float> *)c->coef, c->Pm, g,
                nullptr, (float *)dpos, (float *)dq);
        else
            k_rbe_adjoint<double, 128><<<c->nb256, 256, 0, c->stream>>>(
                c->u4, c->q64, c->map256, c->reps, (const ModeCoef<double> *)c->coef, c->Pm, g,
                c->phtab, (double *)dpos, (double *)dq);
        RBMD_LAUNCH_CHECK();
    }
    (void)eps_h;
    (void)sig_h;
    return RBMD_OK;
}

rbmd_status adjoint_run(rbmd_ctx *c, double g, void *dpos, void *dq, double *tsum_dev)
{
    if (c->fp64) return adjoint_t<double>(c, g, dpos, dq, tsum_dev, nullptr, nullptr);
    return adjoint_t<float>(c, g, dpos, dq, tsum_dev, nullptr, nullptr);
}

}  // namespace rbmd
