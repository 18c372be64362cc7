// C ABI of the library (declared in include/rbmd.h): context set-up, the force,
// step and energy entry points, checkpoints and verification hooks.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rbmd_internal.cuh"

using namespace rbmd;

namespace {

// Host-side fault injection for the failure-path tests: RBMD_FAIL_ALLOC_AFTER=k
// makes the k-th device allocation of the next rbmd_init report failure.
int g_alloc_countdown = -1;

}  // namespace

rbmd_status rbmd::dev_alloc(void **p, size_t bytes)
{
    if (g_alloc_countdown == 0) {
        *p = nullptr;
        return RBMD_ERR_OOM;
    }
    if (g_alloc_countdown > 0) --g_alloc_countdown;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return RBMD_ERR_OOM;
    }
    return RBMD_OK;
}

namespace {

// Entries of the step's candidate lists ([ceil(N/32)][cv][32] int32), 0 without them.
static size_t cand_entries(const rbmd_ctx *c)
{
    return c->verlet ? (size_t)((c->N + 31) / 32) * 32 * c->vl_cv : 0;
}

template <typename T> rbmd_status alloc_n(T **p, size_t n)
{
    return dev_alloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

uint32_t isqrt64(uint64_t x)
{
    uint64_t r = (uint64_t)sqrt((double)x);
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return (uint32_t)r;
}

uint64_t radius2_units(double r, double L)
{
    const double s = r * (kTwo32 / L);
    return (uint64_t)floor(s * s);
}

// Ordering with the caller's work when it passed the legacy default stream.
void enter(rbmd_ctx *c)
{
    if (c->own_stream) {
        cudaEventRecord(c->ev_in, 0);
        cudaStreamWaitEvent(c->stream, c->ev_in, 0);
    }
}
rbmd_status leave(rbmd_ctx *c, rbmd_status s)
{
    if (c->own_stream) {
        cudaEventRecord(c->ev_out, c->stream);
        cudaStreamWaitEvent(0, c->ev_out, 0);
    }
    if (s == RBMD_OK && cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return RBMD_ERR_CUDA;
    }
    return s;
}

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

// Sorted slots hold valid atom ids from the start (every later sort rewrites them).
__global__ void k_iota_spos(uint4 *spos, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) spos[i] = make_uint4(0u, 0u, 0u, (uint32_t)i);
}
__global__ void k_init_scal(double *scal, int R)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < R * SCAL_COUNT)
        scal[t] = (t % SCAL_COUNT == SCAL_LAMBDA || t % SCAL_COUNT == SCAL_LAMBDA_KICK) ? 1.0 : 0.0;
}
__global__ void k_set_lambda(double *scal, int R, double v)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) {
        scal[(int64_t)r * SCAL_COUNT + SCAL_LAMBDA] = v;
        scal[(int64_t)r * SCAL_COUNT + SCAL_LAMBDA_KICK] = v;
    }
}

template <typename real>
__global__ void k_pack(const real *__restrict__ q, const int32_t *__restrict__ type, int64_t N,
                       uint4 *__restrict__ u4, double *__restrict__ q64,
                       int32_t *__restrict__ tout, int n_types, int *__restrict__ err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double qi = (double)q[i];
    u4[i].w = __float_as_uint((float)qi);
    if (q64) q64[i] = qi;
    int t = type ? type[i] : 0;
    if (t < 0 || t >= n_types) {
        latch_error(err, RBMD_ERR_INVALID);
        t = 0;
    }
    tout[i] = t;
}

// Charge sums for the neutrality check and the self energy: [sum q, sum |q|, sum q^2]
// per replica-aligned 256-atom block.
__global__ void k_charge_parts(const double *__restrict__ q64, const uint4 *__restrict__ u4,
                               const int2 *__restrict__ map, const Rep *__restrict__ reps,
                               double *__restrict__ parts)
{
    const AtomSlot sl = atom_slot(map, reps);
    const int64_t i = sl.i;
    double q = 0.0;
    if (sl.ok) q = q64 ? q64[i] : (double)__uint_as_float(u4[i].w);
    double v[3] = {q, fabs(q), q * q};
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    __shared__ double s[3][8];
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) s[c][threadIdx.x >> 5] = v[c];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[c][w];
            parts[3 * (int64_t)blockIdx.x + c] = t;
        }
}

__global__ void k_modes_to_m3(const int4 *__restrict__ modes, int64_t P, int32_t *__restrict__ m3)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    int4 m = modes[l];
    m3[3 * l] = m.x;
    m3[3 * l + 1] = m.y;
    m3[3 * l + 2] = m.z;
}

__global__ void k_u4_to_u3(const uint4 *__restrict__ u4, int64_t N, uint32_t *__restrict__ u3)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 A = u4[i];
    u3[3 * i] = A.x;
    u3[3 * i + 1] = A.y;
    u3[3 * i + 2] = A.z;
}

__global__ void k_u3_to_u4(const uint32_t *__restrict__ u3, int64_t N, uint4 *__restrict__ u4)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 A = u4[i];
    A.x = u3[3 * i];
    A.y = u3[3 * i + 1];
    A.z = u3[3 * i + 2];
    u4[i] = A;
}

// F += fc on the owned rows of every replica (the momentum correction of a slab
// context, Eq. 16, with a correction summed over all ranks).
template <typename real>
__global__ void k_add_owned(real *__restrict__ F, const int2 *__restrict__ map,
                            const Rep *__restrict__ reps, double fx, double fy, double fz)
{
    const AtomSlot sl = atom_slot(map, reps);
    if (!sl.ok || sl.i - reps[sl.r].atom0 >= reps[sl.r].n_own) return;
    F[3 * sl.i + 0] += (real)fx;
    F[3 * sl.i + 1] += (real)fy;
    F[3 * sl.i + 2] += (real)fz;
}

__global__ void k_zero_slots(double *scal, int R, int slot0, int count)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < R * count) scal[(int64_t)(t / count) * SCAL_COUNT + slot0 + t % count] = 0.0;
}

// One block (256 threads) per replica: the sum of its P mode energies e_l into
// scal[SCAL_ERBE] and the RBE virial estimate into scal[SCAL_VRBE + 0..5]:
//   W_ab = sum_l e_l [delta_ab - 2 k_a k_b (1/k^2 + 1/(4 alpha))],
// the strain derivative of the Fourier energy of Eq. 8 (V -> V (1 + tr e),
// k -> (1 - e^T) k, rho unchanged) applied to the sampled modes with weight S/P:
// an unbiased estimate of the Ewald virial.  FP64, fixed order.
__global__ void k_sum_modes(const double *__restrict__ emode, const int4 *__restrict__ modes,
                            const Rep *__restrict__ reps, int64_t P, double alpha,
                            double *__restrict__ scal)
{
    __shared__ double s[7][256];
    const double tk = 2.0 * kPi / reps[blockIdx.x].L;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t l = threadIdx.x; l < P; l += blockDim.x) {
        const int64_t g = (int64_t)blockIdx.x * P + l;
        const double e = emode[g];
        const int4 m = modes[g];
        const double kx = tk * m.x, ky = tk * m.y, kz = tk * m.z;
        const double k2 = kx * kx + ky * ky + kz * kz;
        v[0] += e;
        if (k2 > 0.0) {
            const double b = 2.0 * (1.0 / k2 + 1.0 / (4.0 * alpha));
            v[1] += e * (1.0 - b * kx * kx);
            v[2] += e * (1.0 - b * ky * ky);
            v[3] += e * (1.0 - b * kz * kz);
            v[4] -= e * b * kx * ky;
            v[5] -= e * b * kx * kz;
            v[6] -= e * b * ky * kz;
        }
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) s[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) {
#pragma unroll
            for (int c = 0; c < 7; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) {
        double *sc = scal + (int64_t)blockIdx.x * SCAL_COUNT;
        if (threadIdx.x == 0) sc[SCAL_ERBE] = s[0][0];
        else sc[SCAL_VRBE + threadIdx.x - 1] = s[threadIdx.x][0];
    }
}

rbmd_status sum_modes(rbmd_ctx *c)
{
    k_sum_modes<<<c->R, 256, 0, c->stream>>>(c->emode, c->modes, c->reps, c->Pm, c->prm.alpha, c->scal);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Largest of n counts into *out: a grid-stride loop, a block maximum and one
// atomic per block (every block's atomics go to one address).
__global__ void k_max_count(const int32_t *__restrict__ count, int64_t n, int32_t *__restrict__ out)
{
    int v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v = max(v, count[i]);
    v = __reduce_max_sync(0xffffffffu, v);
    __shared__ int s_m[32];
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? s_m[threadIdx.x] : 0;
        v = __reduce_max_sync(0xffffffffu, v);
        if (threadIdx.x == 0) atomicMax(out, v);
    }
}

void free_ctx(rbmd_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph_ready) cudaGraphExecDestroy(c->graph);
    void *ptrs[] = {c->u4,        c->q64,       c->type,     c->vel,        c->force,
                    c->scratch_force, c->scal,  c->err,      c->d_step,     c->cdf,
                    c->modes,     c->W,         c->rho_part, c->rho,        c->emode,
                    c->coef,      c->cell_count, c->cell_start, c->cell_of, c->cell_rank,
                    c->scan_part, c->spos,      c->sq,       c->stype,      c->fpart,
                    c->epart,     c->kepart,    c->ibuf,     c->lj_f,       c->lj_d,
                    c->lcore,     c->lshell,    c->ncount,   c->bk,         c->red_tmp,
                    c->adj_lj,    c->adj_tpart, c->adj_tsum, c->reps,       c->map256,
                    c->map128,    c->tiles,     c->red_rep,   c->ptab,       c->heavy,
                    c->modes0,    c->acc,       c->chain_step, c->phtab,
                    c->vl_cand != c->lshell ? c->vl_cand : nullptr,
                    c->vl_ncand,  c->vl_sref,   c->rho_acc,   c->gid,      c->adj_rb};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int k = 0; k <= RBMD_PROFILE_STAGES; ++k)
        if (c->prof_ev[k]) cudaEventDestroy(c->prof_ev[k]);
    for (int k = 0; k <= RBMD_PROFILE_GRAD_STAGES; ++k)
        if (c->gprof_ev[k]) cudaEventDestroy(c->gprof_ev[k]);
    delete[] c->reps_h;
    if (c->side) cudaStreamDestroy(c->side);
    if (c->cond_stream) cudaStreamDestroy(c->cond_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->copy) cudaStreamDestroy(c->copy);
    for (int k = 0; k < 8; ++k) {
        if (c->ev_h2d[k]) cudaEventDestroy(c->ev_h2d[k]);
        if (c->ev_enc[k]) cudaEventDestroy(c->ev_enc[k]);
        if (c->ev_fin[k]) cudaEventDestroy(c->ev_fin[k]);
    }
    if (c->own_stream) {
        cudaStreamDestroy(c->stream);
        cudaEventDestroy(c->ev_in);
        cudaEventDestroy(c->ev_out);
    }
    delete c;
}

size_t real_size(const rbmd_ctx *c) { return c->fp64 ? sizeof(double) : sizeof(float); }

// Per-type LJ tables for the pair kernels (sqrt(eps), sigma/2) and the adjoint
// (eps, sigma), from host arrays.
rbmd_status upload_lj(rbmd_ctx *c, const double *eps, const double *sig)
{
    const int T = c->T, T2 = T * T;
    std::vector<double> ljd(2 * T), raw(2 * T + 4 * T2);
    std::vector<float> ljf(2 * T), rawf(2 * T + 4 * T2);
    for (int t = 0; t < T; ++t) {
        if (!(eps[t] >= 0.0) || !(sig[t] >= 0.0)) return RBMD_ERR_INVALID;
        ljd[t] = sqrt(eps[t]);
        ljd[T + t] = 0.5 * sig[t];
        raw[t] = eps[t];
        raw[T + t] = sig[t];
    }
    for (int t = 0; t < 2 * T; ++t) {
        ljf[t] = (float)ljd[t];
        rawf[t] = (float)raw[t];
    }
    // the adjoint's type-pair factors (Eq. 4), from the eps and sigma it holds in
    // its working precision: [t1 T + t2] = 1/2 sqrt(eps_t2 / eps_t1), 1 / sigma_t1t2,
    // eps_t1t2, sigma_t1t2 (IEEE operations, the same bits as on the device)
    for (int t1 = 0; t1 < T; ++t1)
        for (int t2 = 0; t2 < T; ++t2) {
            const int u = t1 * T + t2;
            const double e1 = raw[t1], e2 = raw[t2], s1 = raw[T + t1], s2 = raw[T + t2];
            raw[2 * T + u] = 0.5 * sqrt(e2 / e1);
            raw[2 * T + T2 + u] = 1.0 / (0.5 * (s1 + s2));
            raw[2 * T + 2 * T2 + u] = sqrt(e1 * e2);
            raw[2 * T + 3 * T2 + u] = 0.5 * (s1 + s2);
            const float f1 = rawf[t1], f2 = rawf[t2], g1 = rawf[T + t1], g2 = rawf[T + t2];
            rawf[2 * T + u] = (float)(0.5 * sqrt((double)f2 / (double)f1));
            rawf[2 * T + T2 + u] = (float)(1.0 / (0.5 * ((double)g1 + (double)g2)));
            rawf[2 * T + 2 * T2 + u] = sqrtf(f1 * f2);
            rawf[2 * T + 3 * T2 + u] = 0.5f * (g1 + g2);
        }
    RBMD_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    if (c->fp64) {
        RBMD_CHECK_CUDA(cudaMemcpy(c->lj_d, ljd.data(), sizeof(double) * 2 * T, cudaMemcpyHostToDevice));
        RBMD_CHECK_CUDA(cudaMemcpy(c->adj_lj, raw.data(), sizeof(double) * raw.size(), cudaMemcpyHostToDevice));
    } else {
        RBMD_CHECK_CUDA(cudaMemcpy(c->lj_f, ljf.data(), sizeof(float) * 2 * T, cudaMemcpyHostToDevice));
        RBMD_CHECK_CUDA(cudaMemcpy(c->adj_lj, rawf.data(), sizeof(float) * rawf.size(), cudaMemcpyHostToDevice));
    }
    return RBMD_OK;
}

// Forces of the current configuration, keyed by `s`, into `force` (RBE + RBL);
// F_corr is written to scal (and added to `force` when apply_corr).
rbmd_status check_latched(rbmd_ctx *c);

// One block per replica: the 3 charge sums of its 256-atom blocks.
__global__ void k_sum_charges(const double *__restrict__ parts, const Rep *__restrict__ reps,
                              double *__restrict__ out)
{
    __shared__ double s[3][256];
    const Rep rp = reps[blockIdx.x];
    double v[3] = {0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < rp.nb256; j += blockDim.x)
        for (int k = 0; k < 3; ++k) v[k] += parts[3 * (int64_t)(rp.b256_0 + j) + k];
    for (int k = 0; k < 3; ++k) s[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[3 * (int64_t)blockIdx.x + k] = s[k][0];
}

// Cells of every replica for `div` cells per r_list = r_cut (+ skin when the step
// keeps candidate lists) (Sec. 2.3 binning): the side is at least r_list / div,
// and the count is capped so that sparse boxes do not get more cells than atoms
// (bigger cells stay correct: the stencil still covers r_list).  Returns the
// total; with apply, stores nc, the culling radii and the cell ranges in the host
// replica table.
int64_t cell_layout(rbmd_ctx *c, int div, bool apply)
{
    const double r_cut = c->prm.r_cut;
    const double r_list = r_cut + (c->verlet ? c->skin : 0.0);
    int64_t cell0 = 0;
    for (int r = 0; r < c->R; ++r) {
        Rep &rp = c->reps_h[r];
        int nc = (int)floor(rp.L * div / r_list);
        if (nc < 1) nc = 1;
        while (nc > 1 && (double)rp.Rv * (double)nc > (double)div * kTwo32) --nc;
        const double max_cells = fmax(8.0 * (double)rp.N, 1048576.0);
        while (nc > 1 && (double)nc * nc * nc > max_cells) --nc;
        if (apply) {
            rp.nc = nc;
            rp.cull_r = (float)(r_cut * nc / rp.L * (1.0 + 1e-5) + 1e-6);
            rp.cull_v = (float)(r_list * nc / rp.L * (1.0 + 1e-5) + 1e-6);
            rp.cell0 = cell0;
            rp.ncell = (int64_t)nc * nc * nc;
        }
        cell0 += (int64_t)nc * nc * nc;
    }
    return cell0;
}

// Structure-factor tiles of `tile` atoms that never straddle replicas; returns
// their count and, with apply, fills the map and the replicas' tile ranges.
int tile_layout(rbmd_ctx *c, int tile, bool apply, std::vector<int2> &tl)
{
    tl.clear();
    for (int r = 0; r < c->R; ++r) {
        Rep &rp = c->reps_h[r];
        const int t0 = (int)tl.size();
        for (int64_t a = 0; a < rp.n_own; a += tile) tl.push_back(make_int2(r, (int)(rp.atom0 + a)));
        if (apply) {
            rp.tile0 = t0;
            rp.ntiles = (int32_t)tl.size() - t0;
        }
    }
    return (int)tl.size();
}

// Neutrality of every replica (Sec. 2.2, when check_neutral) and its self energy
// -coulomb_k sqrt(alpha/pi) sum q^2 (third term of Eq. 8).  Synchronises.
rbmd_status charge_sums(rbmd_ctx *c, bool check_neutral = true)
{
    double *parts = (double *)c->scratch_force;  // 3 nb256 doubles fit in 3N doubles + 64 B
    double *sums = c->kepart;                     // 3 R doubles fit in 3 nb256
    k_charge_parts<<<c->nb256, 256, 0, c->stream>>>(c->q64, c->u4, c->map256, c->reps, parts);
    k_sum_charges<<<c->R, 256, 0, c->stream>>>(parts, c->reps, sums);
    RBMD_LAUNCH_CHECK();
    std::vector<double> h(3 * (size_t)c->R);
    RBMD_CHECK_CUDA(cudaMemcpyAsync(h.data(), sums, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                                    c->stream));
    RBMD_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    RBMD_CHECK(check_latched(c));
    for (int r = 0; r < c->R && check_neutral; ++r)
        if (fabs(h[3 * r]) > 1e-6 * (h[3 * r + 1] > 0 ? h[3 * r + 1] : 1.0)) return RBMD_ERR_NOT_NEUTRAL;
    for (int r = 0; r < c->R; ++r)
        c->reps_h[r].e_self = -c->prm.coulomb_k * sqrt(c->prm.alpha / kPi) * h[3 * r + 2];
    RBMD_CHECK_CUDA(cudaMemcpy(c->reps, c->reps_h, sizeof(Rep) * c->R, cudaMemcpyHostToDevice));
    return RBMD_OK;
}

// kick != NULL (the integrator's step): the RBE force kernel also does the second
// half kick; *kicked tells whether it ran.
// verlet: the short-range part of the integrator's step on its candidate lists
// (rbl_pairs_verlet); the same lists, batches and forces as the cell walk.
// A force evaluation outside the step graph uses the candidate lists when the
// context keeps them; after a cell walk or a new layout they are rebuilt first (on
// the device, as in rbmd_step).  Returns whether to use them.
static bool candidates_for_call(rbmd_ctx *c, int accumulate)
{
    if (!c->verlet || accumulate) return false;
    if (c->vl_dirty) {
        if (cudaMemsetAsync(c->ibuf + 4, 1, sizeof(int32_t), c->stream) != cudaSuccess) return false;
        c->vl_dirty = false;
        c->vl_current = false;  // the rebuild has to run
    }
    return true;
}

// verlet_prepare outside the step graph, skipped when the sorted positions and the
// candidate lists are already those of the current state: the last one ran on
// these positions (they move only in the step's drift, which clears the mark, and
// in the calls that set a new state, which make the layout dirty) and nothing
// re-sorted the atoms since.
static rbmd_status verlet_prepare_call(rbmd_ctx *c)
{
    if (!c->capturing && c->vl_current) return RBMD_OK;
    const rbmd_status s = verlet_prepare(c);
    c->vl_current = s == RBMD_OK && !c->capturing;
    return s;
}

// energy: also the potential's terms into scal (SCAL_EPAIR, SCAL_ERBE; the energy bath)
rbmd_status forces_into(rbmd_ctx *c, StepRef s, void *force, int accumulate, bool apply_corr,
                        bool marks = false, const StepRef *kick = nullptr, bool *kicked = nullptr,
                        bool counted = false, bool verlet = false, bool energy = false)
{
    if (kicked) *kicked = false;
    const bool do_rbe = !(c->prm.flags & RBMD_NO_RBE);
    const bool do_rbl = !(c->prm.flags & RBMD_NO_RBL);
    int acc = accumulate;
    // the RBE sampling and structure factors depend on the positions only: on the
    // side stream they overlap the cell sort and the RBL kernels (not while the
    // stages are timed one by one)
    const bool fork = do_rbe && do_rbl && c->side && !c->profiling;
    if (fork) {
        RBMD_CHECK_CUDA(cudaEventRecord(c->ev_fork, c->stream));
        RBMD_CHECK_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        const cudaStream_t main = c->stream;
        c->stream = c->side;
        rbmd_status st = rbe_sample(c, s);
        if (st == RBMD_OK) st = rbe_structure_factors(c, -1);
        if (st == RBMD_OK && energy) st = sum_modes(c);
        c->stream = main;
        RBMD_CHECK_CUDA(cudaEventRecord(c->ev_join, c->side));
        if (st != RBMD_OK) {
            cudaStreamWaitEvent(c->stream, c->ev_join, 0);
            return st;
        }
    }
    if (marks) prof_mark(c, 1);
    if (do_rbl) {
        NvtxRange nvtx_range("rbl");
        rbmd_status st = RBMD_OK;
        if (verlet && !accumulate) {
            st = verlet_prepare_call(c);
            if (marks) prof_mark(c, 2);  // stages 3 and 4 are marked inside
            if (st == RBMD_OK) st = rbl_pairs_verlet(c, s, force, marks, energy);
        } else {
            st = cells_build(c, counted);
            if (marks) prof_mark(c, 2);  // stages 3 and 4 are marked inside
            if (st == RBMD_OK) st = rbl_pairs(c, s, force, acc, energy, nullptr, nullptr, nullptr, marks);
        }
        if (st == RBMD_OK && energy) st = md_sum_replicas(c, c->epart, EPART, SCAL_EPAIR, 1.0, false, true);
        if (marks) prof_mark(c, 5);
        if (st == RBMD_OK)
            st = rbl_correction(c, force, apply_corr, apply_corr ? SCAL_FCORR_AUX : SCAL_FCORR);
        if (st != RBMD_OK) {
            if (fork) cudaStreamWaitEvent(c->stream, c->ev_join, 0);  // no side work left unjoined
            return st;
        }
        acc = 1;
    } else {
        for (int k = 2; k <= 5 && marks; ++k) prof_mark(c, k);
        if (energy) {
            k_zero_slots<<<(c->R * EPART + 255) / 256, 256, 0, c->stream>>>(c->scal, c->R, SCAL_EPAIR, EPART);
            RBMD_LAUNCH_CHECK();
        }
        if (!apply_corr) {
            k_zero_slots<<<(c->R * 3 + 255) / 256, 256, 0, c->stream>>>(c->scal, c->R, SCAL_FCORR, 3);
            RBMD_LAUNCH_CHECK();
        }
    }
    if (marks) prof_mark(c, 6);
    if (fork) {
        RBMD_CHECK_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    } else if (do_rbe) {
        RBMD_CHECK(rbe_sample(c, s));
        if (marks) prof_mark(c, 7);
        RBMD_CHECK(rbe_structure_factors(c, marks ? 8 : -1));
        if (energy) RBMD_CHECK(sum_modes(c));
        if (marks) prof_mark(c, 9);
    } else if (energy) {
        k_zero_slots<<<(c->R + 255) / 256, 256, 0, c->stream>>>(c->scal, c->R, SCAL_ERBE, 1);
        RBMD_LAUNCH_CHECK();
    }
    if (do_rbe) {
        RBMD_CHECK(rbe_apply_forces(c, force, acc, kick));
        if (kicked && kick) *kicked = true;
        acc = 1;
    } else if (marks) {
        for (int k = 7; k <= 9; ++k) prof_mark(c, k);
    }
    if (!acc)
        RBMD_CHECK_CUDA(cudaMemsetAsync(force, 0, 3 * c->N * real_size(c), c->stream));
    return RBMD_OK;
}

rbmd_status record_step(rbmd_ctx *c)
{
    StepRef next{c->d_step, 1};
    prof_mark(c, 0);
    // the drift kernel also bins the atoms (not when the candidate lists are used:
    // they re-sort only at a rebuild)
    const bool bin = !(c->prm.flags & RBMD_NO_RBL) && !c->verlet;
    RBMD_CHECK(md_kick_drift(c, bin));
    c->vl_current = false;  // the drift moved the atoms
    bool kicked = false;
    RBMD_CHECK(forces_into(c, next, c->force, 0, false, true, &next, &kicked, bin, c->verlet,
                           c->prm.thermostat == 4));
    prof_mark(c, 10);
    RBMD_CHECK(md_kick_thermo(c, true, next, kicked));
    prof_mark(c, 11);
    return RBMD_OK;
}

rbmd_status check_latched(rbmd_ctx *c)
{
    int e = 0;
    RBMD_CHECK_CUDA(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        int z = 0;
        cudaMemcpy(c->err, &z, sizeof(int), cudaMemcpyHostToDevice);
        return (rbmd_status)e;
    }
    return RBMD_OK;
}

}  // namespace

extern "C" {

const char *rbmd_status_string(rbmd_status s)
{
    switch (s) {
    case RBMD_OK: return "ok";
    case RBMD_ERR_INVALID: return "invalid argument";
    case RBMD_ERR_NOT_NEUTRAL: return "system is not charge neutral";
    case RBMD_ERR_BOX_TOO_SMALL: return "r_cut must be below L/2";
    case RBMD_ERR_OOM: return "device allocation failed";
    case RBMD_ERR_CUDA: return "CUDA runtime error";
    case RBMD_ERR_CELL_OVERFLOW: return "cell or list capacity exceeded";
    case RBMD_ERR_NONFINITE: return "non-finite force or velocity";
    case RBMD_ERR_TIMEOUT: return "bounded device wait timed out";
    case RBMD_ERR_UNSUPPORTED: return "unsupported option";
    case RBMD_ERR_BOUNDS: return "index out of range (bounds-checked build)";
    }
    return "unknown status";
}

const char *rbmd_version(void) { return "rbmd-b300 0.1 (sm_103a)"; }

rbmd_status rbmd_sampler_table(double box_length, double alpha, int32_t *M, uint64_t *T, double *H)
{
    return sampler_table_host(box_length, alpha, M, T, H);
}

rbmd_status rbmd_metropolis_table(double box_length, double alpha, uint64_t *A)
{
    int32_t M = 0;
    RBMD_CHECK(sampler_table_host(box_length, alpha, &M, nullptr, nullptr));
    if (!A) return RBMD_ERR_INVALID;
    return metropolis_table_host(box_length, alpha, M, A);
}

}  // extern "C"

namespace {

// A slab context of a spatial decomposition (rbmd_init_slab).
struct SlabInit {
    int64_t n_owned, n_global;
    const uint32_t *gid;  // device [N]
};

rbmd_status init_ctx(const rbmd_params *prms, int32_t R, const void *pos, const void *vel,
                     const void *charge, const int32_t *type, const double *lj_eps,
                     const double *lj_sigma, void *stream, const SlabInit *slab, rbmd_ctx **out)
{
    if (!out) return RBMD_ERR_INVALID;
    *out = nullptr;
    if (!prms || R < 1 || R > 65536 || !pos || !charge || !lj_eps || !lj_sigma) return RBMD_ERR_INVALID;
    const rbmd_params p = prms[0];
    int64_t Ntot = 0;
    for (int r = 0; r < R; ++r) {
        const rbmd_params &q = prms[r];
        if (q.n_atoms < 1 || q.n_atoms > (int64_t)2000000000) return RBMD_ERR_INVALID;
        if (!(q.box_length > 0.0)) return RBMD_ERR_INVALID;
        // everything but the size, box, seed, replica tag and T0 is shared
        if (q.n_types != p.n_types || q.rbe_P != p.rbe_P || q.alpha != p.alpha ||
            q.r_core != p.r_core || q.r_cut != p.r_cut || q.rbl_p != p.rbl_p ||
            q.thermostat != p.thermostat || q.coulomb_k != p.coulomb_k || q.dt != p.dt ||
            q.tau_T != p.tau_T || q.precision != p.precision || q.flags != p.flags ||
            q.cell_div != p.cell_div || q.mh_moves != p.mh_moves || q.skin != p.skin)
            return RBMD_ERR_INVALID;
        if (!(q.r_cut < 0.5 * q.box_length)) return RBMD_ERR_BOX_TOO_SMALL;
        Ntot += q.n_atoms;
    }
    if (Ntot > (int64_t)2000000000) return RBMD_ERR_INVALID;
    if (p.n_types < 1 || p.n_types > RBMD_MAX_TYPES) return RBMD_ERR_INVALID;
    if (!(p.alpha > 0.0) || !(p.r_cut > 0.0)) return RBMD_ERR_INVALID;
    if (!(p.r_core >= 0.0) || p.r_core > p.r_cut) return RBMD_ERR_INVALID;
    if (p.rbe_P < 1 || p.rbl_p < 1 || p.rbl_p > 1024) return RBMD_ERR_INVALID;
    if (p.precision != RBMD_FP32 && p.precision != RBMD_FP64) return RBMD_ERR_INVALID;
    if (p.thermostat < 0 || p.thermostat > 4) return RBMD_ERR_INVALID;
    if (p.cell_div < 0 || p.cell_div > 2) return RBMD_ERR_INVALID;
    if ((p.flags & RBMD_FULL_EWALD_MODES) && R != 1) return RBMD_ERR_UNSUPPORTED;
    if ((p.flags & RBMD_FULL_EWALD_MODES) && (p.flags & RBMD_METROPOLIS_MODES))
        return RBMD_ERR_INVALID;
    if (p.mh_moves < 0) return RBMD_ERR_INVALID;
    for (int t = 0; t < p.n_types; ++t)
        if (!(lj_eps[t] >= 0.0) || !(lj_sigma[t] >= 0.0)) return RBMD_ERR_INVALID;

    {
        const char *env = getenv("RBMD_FAIL_ALLOC_AFTER");
        g_alloc_countdown = env ? atoi(env) : -1;
    }

    rbmd_ctx *c = new rbmd_ctx;
    memset(c, 0, sizeof(*c));
    c->prm = p;
    c->R = R;
    c->N = Ntot;
    c->T = p.n_types;
    c->fp64 = p.precision == RBMD_FP64;
    c->tau = p.tau_T > 0.0 ? p.tau_T : 0.1;
    c->sqrt_alpha = sqrt(p.alpha);
    c->full_modes = (p.flags & RBMD_FULL_EWALD_MODES) != 0;
    c->div = p.cell_div == 0 ? 2 : p.cell_div;
    c->rho_tile = 1024;
    c->rho_mode_tile = 256;
    c->reps_h = new Rep[R];
    memset(c->reps_h, 0, sizeof(Rep) * R);

    rbmd_status st = RBMD_OK;
#define TRY(x)                     \
    do {                           \
        st = (x);                  \
        if (st != RBMD_OK) {       \
            g_alloc_countdown = -1; \
            free_ctx(c);           \
            return st;             \
        }                          \
    } while (0)

    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        c->own_stream = true;
        TRY(cuda_status(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)));
        TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)));
        TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)));
    }
    c->cond_nodes = !(getenv("RBMD_GRAPH_COND") && atoi(getenv("RBMD_GRAPH_COND")) == 0);
    // RBMD_ONE_STREAM=1 keeps every force evaluation on the context's stream
    // (the two-stream and one-stream evaluations compute the same bits)
    if (!(getenv("RBMD_ONE_STREAM") && atoi(getenv("RBMD_ONE_STREAM")) != 0)) {
        TRY(cuda_status(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)));
        TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)));
        TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)));
        TRY(cuda_status(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking)));
        for (int k = 0; k < 8; ++k) {
            TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_h2d[k], cudaEventDisableTiming)));
            TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_enc[k], cudaEventDisableTiming)));
            TRY(cuda_status(cudaEventCreateWithFlags(&c->ev_fin[k], cudaEventDisableTiming)));
        }
    }
    enter(c);

    // per-replica constants: sampler (Eq. 12), RBL radii and cells (Sec. 2.3)
    std::vector<uint64_t> T;
    std::vector<int2> m256, m128, tl;
    double max_mc = 0.0, max_ms = 0.0;
    int64_t atom0 = 0;
    for (int r = 0; r < R; ++r) {
        const rbmd_params &q = prms[r];
        Rep &rp = c->reps_h[r];
        rp.L = q.box_length;
        rp.lscale = rp.L / kTwo32;
        rp.dtc = q.dt * (kTwo32 / rp.L);
        rp.dtc_hi = (float)rp.dtc;
        rp.dtc_lo = (float)(rp.dtc - (double)rp.dtc_hi);
        rp.T0 = q.temperature;
        rp.key = make_uint2((uint32_t)(q.seed & 0xFFFFFFFFu), (uint32_t)(q.seed >> 32));
        rp.tag_rbe = RBMD_STREAM_RBE | (q.replica << 8);
        rp.tag_rbl = RBMD_STREAM_RBL | (q.replica << 8);
        int32_t M = 0;
        double H = 0.0;
        TRY(sampler_table_host(rp.L, p.alpha, &M, nullptr, nullptr));
        rp.M = M;
        rp.cdf0 = (int64_t)T.size();
        T.resize(T.size() + 2 * (size_t)M + 1);
        TRY(sampler_table_host(rp.L, p.alpha, &M, T.data() + rp.cdf0, &H));
        rp.S = H * H * H - 1.0;
        rp.Wrbe = rp.S / (double)p.rbe_P;
        rp.Rc2 = radius2_units(p.r_core, rp.L);
        rp.Rs2 = radius2_units(p.r_cut, rp.L);
        rp.Rlin = isqrt64(rp.Rs2);
        rp.Rv = rp.Rlin;
        rp.atom0 = atom0;
        rp.N = q.n_atoms;
        rp.n_own = slab ? slab->n_owned : q.n_atoms;
        rp.b256_0 = (int32_t)m256.size();
        for (int64_t a = 0; a < rp.N; a += 256) m256.push_back(make_int2(r, (int)(atom0 + a)));
        rp.nb256 = (int32_t)m256.size() - rp.b256_0;
        rp.b128_0 = (int32_t)m128.size();
        for (int64_t a = 0; a < rp.N; a += 128) m128.push_back(make_int2(r, (int)(atom0 + a)));
        rp.nb128 = (int32_t)m128.size() - rp.b128_0;
        atom0 += rp.N;
        const double n = (double)rp.N / (rp.L * rp.L * rp.L);
        const double mc = n * 4.0 / 3.0 * kPi * p.r_core * p.r_core * p.r_core;
        max_mc = fmax(max_mc, mc);
        max_ms = fmax(max_ms, n * 4.0 / 3.0 * kPi * (p.r_cut * p.r_cut * p.r_cut) - mc);
    }
    // candidate lists of the integrator's step (the lists, batches and forces are
    // the same without them; they only save the per-step cell walk): a skin of
    // p.skin (0: 0.4 sigma), off for exact lists, large batches, RBL off, or a box
    // where r_cut + skin reaches half the box
    c->skin = p.skin == 0.0 ? 0.4 : p.skin;
    c->verlet = c->skin > 0.0 && !(p.flags & (RBMD_RBL_EXACT | RBMD_NO_RBL)) && p.rbl_p <= 32 &&
                !slab;
    if (const char *env = getenv("RBMD_NO_CANDIDATES")) c->verlet = c->verlet && atoi(env) == 0;
    double max_mv = 0.0;
    for (int r = 0; r < R && c->verlet; ++r) {
        Rep &rp = c->reps_h[r];
        const double h = floor(0.5 * c->skin * (kTwo32 / rp.L));
        const double Rv = (double)rp.Rlin + 1.0 + 2.0 * h;
        if (!(p.r_cut + c->skin < 0.5 * rp.L) || Rv >= 2147483000.0) {
            c->verlet = false;
            break;
        }
        rp.H2 = (uint64_t)h * (uint64_t)h;
        rp.Rv = (uint32_t)Rv;
        rp.Rv2 = (uint64_t)rp.Rv * (uint64_t)rp.Rv;
        const double n = (double)rp.N / (rp.L * rp.L * rp.L);
        const double rl = p.r_cut + c->skin;
        max_mv = fmax(max_mv, n * 4.0 / 3.0 * kPi * rl * rl * rl);
    }
    if (!c->verlet)
        for (int r = 0; r < R; ++r) c->reps_h[r].Rv = c->reps_h[r].Rlin;
    // capacities: candidates mean + 4 sd + 8 (a liquid's counts vary less than
    // Poisson's); the core members a thread keeps in shared memory mean + 5 sd + 4
    // (beyond them: the exact fallback)
    c->vl_cv = ((int)ceil(max_mv + 4.0 * sqrt(max_mv) + 8.0) + 3) / 4 * 4;
    c->vl_ccs = (int)ceil(max_mc + 5.0 * sqrt(max_mc) + 4.0);
    if (std::max(c->vl_ccs, p.rbl_p) * 128 * 4 > 160 * 1024) c->verlet = false;
    c->vl_dirty = true;

    // cell arrays and tile partials sized for every layout rbmd_set_tiles allows
    c->ncell_max = std::max(cell_layout(c, 1, false), cell_layout(c, 2, false));
    c->ntiles_max = tile_layout(c, 512, false, tl);
    c->ncell = cell_layout(c, c->div, true);
    c->ntiles = tile_layout(c, c->rho_tile, true, tl);
    c->cdf_total = (int64_t)T.size();
    c->nb256 = (int)m256.size();
    c->nb128 = (int)m128.size();
    c->pair_parts = 2 * 4 * c->nb128;  // per warp: pair kernel, then the fallback
    // list capacities: mean + 5 sd + 8 (core) and mean + 8 sd + 8 (shell) of a
    // uniform fluid at the densest replica's density, rounded up to a multiple of
    // 4; atoms beyond them take the exact fallback
    c->list_cc = ((int)ceil(max_mc + 5.0 * sqrt(max_mc) + 8.0) + 3) / 4 * 4;
    c->list_cs = ((int)ceil(max_ms + 8.0 * sqrt(max_ms) + 8.0) + 3) / 4 * 4;
    // RBMD_SELECT_EXACT=1 sends every batch selection through the exact path that
    // otherwise only atoms with equal priority words take, so that tests reach it
    if (const char *env = getenv("RBMD_SELECT_EXACT")) c->sel_exact = atoi(env) != 0;
    // RBMD_SELECT_KEY_BITS=k keeps only the k high bits of the priority word in the
    // fast selection's keys, so that equal truncated keys (and with them the
    // exact path) become common; the batches must not change
    if (const char *env = getenv("RBMD_SELECT_KEY_BITS")) c->sel_key_bits = atoi(env);
    // RBMD_LIST_CAPS="cc,cs" shrinks the capacities so that tests can drive
    // atoms through the overflow path
    if (const char *env = getenv("RBMD_LIST_CAPS")) {
        int cc = 0, cs = 0;
        if (sscanf(env, "%d,%d", &cc, &cs) == 2 && cc >= 1 && cs >= 1) {
            c->list_cc = cc;
            c->list_cs = cs;
            c->vl_ccs = std::min(c->vl_ccs, cc);
        }
    }

    // mode list (the full Ewald series of one replica, Eq. 11)
    std::vector<int4> full;
    std::vector<double> fullW;
    if (c->full_modes) {
        const double a = kPi * kPi / (p.alpha * c->reps_h[0].L * c->reps_h[0].L);
        const int M = c->reps_h[0].M;
        for (int mx = -M; mx <= M; ++mx)
            for (int my = -M; my <= M; ++my)
                for (int mz = -M; mz <= M; ++mz) {
                    if (!mx && !my && !mz) continue;
                    full.push_back(make_int4(mx, my, mz, 0));
                    fullW.push_back(exp(-a * (double)(mx * mx + my * my + mz * mz)));
                }
        c->Pm = (int64_t)full.size();
    } else {
        c->Pm = p.rbe_P;
    }

    const size_t rs = real_size(c);
    const int64_t N = c->N;
    TRY(alloc_n(&c->reps, (size_t)R));
    TRY(alloc_n(&c->map256, (size_t)c->nb256));
    TRY(alloc_n(&c->map128, (size_t)c->nb128));
    TRY(alloc_n(&c->tiles, (size_t)c->ntiles_max));
    TRY(alloc_n(&c->u4, N));
    if (c->fp64) TRY(alloc_n(&c->q64, N));
    TRY(alloc_n(&c->type, N));
    TRY(dev_alloc(&c->vel, 3 * N * rs));
    TRY(dev_alloc(&c->force, 3 * N * rs));
    TRY(dev_alloc(&c->scratch_force, 3 * N * (rs > 4 ? rs : 8) + 64));
    TRY(alloc_n(&c->scal, (size_t)R * SCAL_COUNT));
    TRY(alloc_n(&c->red_tmp, (size_t)RED_BLOCKS * 8));
    TRY(alloc_n(&c->red_rep, (size_t)R * RED_SPLIT * RED_STRIDE));
    TRY(alloc_n(&c->err, 1));
    TRY(alloc_n(&c->d_step, 1));
    TRY(alloc_n(&c->cdf, T.size()));
    TRY(alloc_n(&c->modes, (size_t)R * c->Pm));
    if (p.flags & RBMD_METROPOLIS_MODES) {
        TRY(alloc_n(&c->modes0, (size_t)R * c->Pm));
        TRY(alloc_n(&c->acc, T.size()));
        TRY(alloc_n(&c->chain_step, 1));
        c->mh_moves = p.mh_moves > 0 ? p.mh_moves : 8;
    }
    if (c->full_modes) TRY(alloc_n(&c->W, c->Pm));
    TRY(alloc_n(&c->rho_part, (size_t)c->ntiles_max * c->Pm));
    TRY(alloc_n(&c->rho, (size_t)R * c->Pm));
    TRY(alloc_n(&c->rho_acc, (size_t)R * c->Pm * 2));
    TRY(alloc_n(&c->emode, (size_t)R * c->Pm));
    TRY(dev_alloc(&c->coef, (size_t)R * c->Pm * (c->fp64 ? sizeof(ModeCoef<double>) : sizeof(ModeCoef<float>))));
    TRY(alloc_n(&c->cell_count, c->ncell_max));
    TRY(alloc_n(&c->cell_start, c->ncell_max + 1));
    TRY(alloc_n(&c->cell_of, N));
    TRY(alloc_n(&c->cell_rank, N));
    TRY(alloc_n(&c->scan_part, (c->ncell_max + 1023) / 1024 + 1));
    TRY(alloc_n(&c->spos, N));
    TRY(dev_alloc(&c->sq, N * rs));
    TRY(alloc_n(&c->stype, N));
    TRY(alloc_n(&c->fpart, 3 * (size_t)c->pair_parts));
    TRY(alloc_n(&c->lcore, (size_t)N * c->list_cc));
    // the cell walk's shell lists and the step's candidate lists share one array: a
    // cell walk re-sorts the atoms, which makes the candidates stale anyway (every
    // cell walk marks them for a rebuild before the next step)
    TRY(alloc_n(&c->lshell, std::max((size_t)N * c->list_cs, cand_entries(c))));
    TRY(alloc_n(&c->ncount, (size_t)N));
    TRY(alloc_n(&c->bk, (size_t)N * p.rbl_p));
    if (p.rbl_p > 10) TRY(alloc_n(&c->heavy, (size_t)N));
    TRY(dev_alloc(&c->adj_lj, (2 * (size_t)c->T + 4 * (size_t)c->T * c->T) * rs));
    TRY(alloc_n(&c->adj_tpart, (size_t)c->nb128 * 2 * c->T));
    TRY(alloc_n(&c->adj_tsum, 2 * (size_t)c->T));
    TRY(alloc_n(&c->epart, EPART * (size_t)c->pair_parts));
    TRY(alloc_n(&c->kepart, (size_t)c->nb256 * 3));
    TRY(alloc_n(&c->ibuf, 8));
    c->n_glob = slab ? slab->n_global : Ntot;
    if (slab) {
        TRY(alloc_n(&c->gid, (size_t)N));
        TRY(cuda_status(cudaMemcpyAsync(c->gid, slab->gid, sizeof(uint32_t) * N, cudaMemcpyDefault,
                                        c->stream)));
    }
    if (c->verlet) {
        c->vl_cand = c->lshell;
        TRY(alloc_n(&c->vl_ncand, (size_t)N));
        TRY(alloc_n(&c->vl_sref, (size_t)N));
    }
    g_alloc_countdown = -1;

    // LJ tables: sqrt(eps_t), sigma_t/2 (Lorentz-Berthelot, Eq. 4)
    if (c->fp64) TRY(alloc_n(&c->lj_d, 2 * c->T));
    else TRY(alloc_n(&c->lj_f, 2 * c->T));
    {
        // pair look-up table (Sec. 3.3), used when RBMD_PAIR_TABLE is set or the
        // autotuner picks it
        std::vector<double> coef;
        c->ptab_n = c->fp64 ? 8192 : 1024;
        double inv_h = 0.0;
        TRY(pair_table_host(p.alpha, p.r_cut, c->ptab_n, coef, &c->ptab_i0, &inv_h));
        c->ptab_inv_h = inv_h;
        if (c->fp64) {
            TRY(dev_alloc(&c->ptab, sizeof(double) * coef.size()));
            TRY(cuda_status(cudaMemcpy(c->ptab, coef.data(), sizeof(double) * coef.size(),
                                       cudaMemcpyHostToDevice)));
        } else {
            std::vector<float> cf(coef.begin(), coef.end());
            TRY(dev_alloc(&c->ptab, sizeof(float) * cf.size()));
            TRY(cuda_status(cudaMemcpy(c->ptab, cf.data(), sizeof(float) * cf.size(),
                                       cudaMemcpyHostToDevice)));
        }
        c->use_table = (p.flags & RBMD_PAIR_TABLE) != 0;
    }
    TRY(upload_lj(c, lj_eps, lj_sigma));
    TRY(rbe_configure(c));
    TRY(rbl_configure(c));
    TRY(verlet_configure(c));
    TRY(cuda_status(cudaMemcpy(c->reps, c->reps_h, sizeof(Rep) * R, cudaMemcpyHostToDevice)));
    TRY(cuda_status(cudaMemcpy(c->map256, m256.data(), sizeof(int2) * m256.size(), cudaMemcpyHostToDevice)));
    TRY(cuda_status(cudaMemcpy(c->map128, m128.data(), sizeof(int2) * m128.size(), cudaMemcpyHostToDevice)));
    TRY(cuda_status(cudaMemcpy(c->tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice)));
    TRY(cuda_status(cudaMemcpy(c->cdf, T.data(), sizeof(uint64_t) * T.size(), cudaMemcpyHostToDevice)));
    if (c->modes0) {
        std::vector<uint64_t> A(T.size());
        for (int r = 0; r < R; ++r)
            TRY(metropolis_table_host(c->reps_h[r].L, p.alpha, c->reps_h[r].M, A.data() + c->reps_h[r].cdf0));
        TRY(cuda_status(cudaMemcpy(c->acc, A.data(), sizeof(uint64_t) * A.size(), cudaMemcpyHostToDevice)));
        TRY(rbe_metropolis_init(c));
    }
    if (c->full_modes) {
        TRY(cuda_status(cudaMemcpy(c->modes, full.data(), sizeof(int4) * full.size(), cudaMemcpyHostToDevice)));
        TRY(cuda_status(cudaMemcpy(c->W, fullW.data(), sizeof(double) * fullW.size(), cudaMemcpyHostToDevice)));
    }
    TRY(cuda_status(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream)));
    TRY(cuda_status(cudaMemsetAsync(c->u4, 0, sizeof(uint4) * N, c->stream)));
    TRY(cuda_status(cudaMemsetAsync(c->ibuf, 0, 8 * sizeof(int32_t), c->stream)));
    k_iota_spos<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->spos, N);
    k_init_scal<<<(R * SCAL_COUNT + 255) / 256, 256, 0, c->stream>>>(c->scal, R);
    k_set_i64<<<1, 1, 0, c->stream>>>(c->d_step, 0);

    // particle data (Sec. 2.1: map the arrays to the device)
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (c->fp64)
        k_pack<double><<<nb, 256, 0, c->stream>>>((const double *)charge, type, N, c->u4, c->q64,
                                                  c->type, c->T, c->err);
    else
        k_pack<float><<<nb, 256, 0, c->stream>>>((const float *)charge, type, N, c->u4, nullptr,
                                                 c->type, c->T, c->err);
    TRY(md_encode_positions(c, pos));
    if (vel) TRY(cuda_status(cudaMemcpyAsync(c->vel, vel, 3 * N * rs, cudaMemcpyDefault, c->stream)));
    else TRY(cuda_status(cudaMemsetAsync(c->vel, 0, 3 * N * rs, c->stream)));

    // neutrality of every replica (Sec. 2.2) and the self energies (third term of Eq. 8)
    TRY(charge_sums(c, !slab));  // a slab need not be neutral (the whole system is)
#undef TRY
    c->step = 0;
    c->have_force = false;
    c->vl_dirty = true;
    leave(c, RBMD_OK);
    *out = c;
    return RBMD_OK;
}

}  // namespace

extern "C" {

rbmd_status rbmd_init_batch(const rbmd_params *prms, int32_t R, const void *pos, const void *vel,
                            const void *charge, const int32_t *type, const double *lj_eps,
                            const double *lj_sigma, void *stream, rbmd_ctx **out)
{
    return init_ctx(prms, R, pos, vel, charge, type, lj_eps, lj_sigma, stream, nullptr, out);
}

rbmd_status rbmd_init_slab(const rbmd_params *params, int64_t n_owned, int64_t n_global,
                           const uint32_t *gid, const void *pos, const void *vel,
                           const void *charge, const int32_t *type, const double *lj_eps,
                           const double *lj_sigma, void *stream, rbmd_ctx **out)
{
    if (!out) return RBMD_ERR_INVALID;
    *out = nullptr;
    if (!params || !gid || n_owned < 1 || n_owned > params->n_atoms || n_global < n_owned ||
        n_global > (int64_t)UINT32_MAX || params->rbl_p > 32 ||
        (params->flags & RBMD_FULL_EWALD_MODES))
        return RBMD_ERR_INVALID;
    const SlabInit sl{n_owned, n_global, gid};
    return init_ctx(params, 1, pos, vel, charge, type, lj_eps, lj_sigma, stream, &sl, out);
}

rbmd_status rbmd_init(const rbmd_params *prm, const void *pos, const void *vel, const void *charge,
                      const int32_t *type, const double *lj_eps, const double *lj_sigma,
                      void *stream, rbmd_ctx **out)
{
    return rbmd_init_batch(prm, 1, pos, vel, charge, type, lj_eps, lj_sigma, stream, out);
}

void rbmd_destroy(rbmd_ctx *c) { free_ctx(c); }

rbmd_status rbmd_rbe_forces(rbmd_ctx *c, int64_t step, void *force, int accumulate)
{
    NvtxRange nvtx_range("rbmd_rbe_forces");
    if (!c || !force) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    enter(c);
    rbmd_status s = RBMD_OK;
    if (c->prm.flags & RBMD_NO_RBE) {
        if (!accumulate) s = cuda_status(cudaMemsetAsync(force, 0, 3 * c->N * real_size(c), c->stream));
        return leave(c, s);
    }
    StepRef r{nullptr, step};
    s = rbe_sample(c, r);
    if (s == RBMD_OK) s = rbe_structure_factors(c);
    if (s == RBMD_OK) s = rbe_apply_forces(c, force, accumulate);
    return leave(c, s);
}

rbmd_status rbmd_rbl_forces(rbmd_ctx *c, int64_t step, void *force, int accumulate)
{
    NvtxRange nvtx_range("rbmd_rbl_forces");
    if (!c || !force) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    enter(c);
    rbmd_status s = RBMD_OK;
    if (c->prm.flags & RBMD_NO_RBL) {
        if (!accumulate) s = cuda_status(cudaMemsetAsync(force, 0, 3 * c->N * real_size(c), c->stream));
        return leave(c, s);
    }
    StepRef r{nullptr, step};
    s = cells_build(c);
    if (s == RBMD_OK) s = rbl_pairs(c, r, force, accumulate, false, nullptr, nullptr, nullptr);
    if (s == RBMD_OK) s = rbl_correction(c, force, true, SCAL_FCORR_AUX);
    return leave(c, s);
}

rbmd_status rbmd_forces(rbmd_ctx *c, int64_t step, void *force, int accumulate)
{
    NvtxRange nvtx_range("rbmd_forces");
    if (!c || !force) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    enter(c);
    const bool vl = candidates_for_call(c, accumulate);
    return leave(c, forces_into(c, StepRef{nullptr, step}, force, accumulate, true, false, nullptr,
                                nullptr, false, vl));
}

rbmd_status rbmd_forces_host(rbmd_ctx *c, const void *pos, void *force, int64_t step)
{
    NvtxRange nvtx_range("rbmd_forces_host");
    if (!c || !pos || !force) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    const size_t row = 3 * real_size(c);
    void *dev = c->scratch_force;  // staged positions, then the forces
    const bool do_rbe = !(c->prm.flags & RBMD_NO_RBE);
    const bool do_rbl = !(c->prm.flags & RBMD_NO_RBL);
    if (!c->copy || !do_rbe || !do_rbl || c->profiling) {
        // nothing to overlap (or stages being timed): the same work in sequence
        rbmd_status s = rbmd_set_state(c, pos, nullptr, step);
        if (s == RBMD_OK) s = rbmd_forces(c, step, dev, 0);
        if (s != RBMD_OK) return s;
        enter(c);
        s = cuda_status(cudaMemcpyAsync(force, dev, c->N * row, cudaMemcpyDefault, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
        return leave(c, s);
    }
    enter(c);
    // chunks: ranges of structure-factor tiles; a tile starts on a 256-atom block
    // boundary of its replica, so each chunk is also a range of map256 blocks and
    // of atoms
    std::vector<int64_t> ta;
    for (int r = 0; r < c->R; ++r)
        for (int64_t a = 0; a < c->reps_h[r].N; a += c->rho_tile) ta.push_back(c->reps_h[r].atom0 + a);
    const int ntl = (int)ta.size();
    int nch = std::min(4, ntl);
    if (const char *e = getenv("RBMD_HOST_CHUNKS")) nch = std::max(1, std::min(std::min(8, atoi(e)), ntl));
    int T[9], B[9];
    int64_t A[9];
    for (int k = 0; k <= nch; ++k) {
        T[k] = (int)((int64_t)k * ntl / nch);
        A[k] = T[k] < ntl ? ta[T[k]] : c->N;
        B[k] = c->nb256;
        for (int r = 0; r < c->R && T[k] < ntl; ++r) {
            const Rep &rp = c->reps_h[r];
            if (A[k] >= rp.atom0 && A[k] < rp.atom0 + rp.N) B[k] = rp.b256_0 + (int)((A[k] - rp.atom0) / 256);
        }
    }
    const StepRef s{nullptr, step};
    const cudaStream_t main = c->stream;
    rbmd_status st = RBMD_OK;
    auto on = [&](cudaStream_t q, auto &&f) {  // host helpers launch on c->stream
        c->stream = q;
        if (st == RBMD_OK) st = f();
        c->stream = main;
    };
    // the copies reuse the staging buffer only after the caller's earlier work
    cudaEventRecord(c->ev_fork, main);
    cudaStreamWaitEvent(c->copy, c->ev_fork, 0);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    // the candidate lists (rebuilt on the device when an atom moved too far), else
    // the cell walk with the atoms binned chunk by chunk as they arrive
    const bool vl = candidates_for_call(c, 0);
    if (!vl) st = cuda_status(cudaMemsetAsync(c->cell_count, 0, sizeof(int32_t) * c->ncell, main));
    on(c->side, [&] { return rbe_sample(c, s); });
    for (int k = 0; k < nch; ++k) {
        // positions of chunk k: copied in, encoded and binned, then its tiles' partial
        // structure factors on the side stream while the next chunk is copied
        const size_t off = (size_t)A[k] * row, bytes = (size_t)(A[k + 1] - A[k]) * row;
        if (st == RBMD_OK)
            st = cuda_status(cudaMemcpyAsync((char *)dev + off, (const char *)pos + off, bytes,
                                             cudaMemcpyDefault, c->copy));
        cudaEventRecord(c->ev_h2d[k], c->copy);
        cudaStreamWaitEvent(main, c->ev_h2d[k], 0);
        if (st == RBMD_OK) st = md_encode_blocks(c, dev, B[k], B[k + 1]);
        if (st == RBMD_OK && !vl) st = cells_count_blocks(c, B[k], B[k + 1]);
        cudaEventRecord(c->ev_enc[k], main);
        cudaStreamWaitEvent(c->side, c->ev_enc[k], 0);
        on(c->side, [&] { return rbe_rho_partial(c, T[k], T[k + 1]); });
    }
    on(c->side, [&] { return rbe_rho_final(c); });
    cudaEventRecord(c->ev_join, c->side);
    // the short-range part (same kernels as rbmd_forces), then the RBE force pass
    // chunk by chunk, each chunk's forces copied out while the next is computed
    c->vl_current = false;  // new positions
    if (vl) {
        if (st == RBMD_OK) st = verlet_prepare_call(c);
        if (st == RBMD_OK) st = rbl_pairs_verlet(c, s, dev, false);
    } else {
        if (st == RBMD_OK) st = cells_build(c, true);
        if (st == RBMD_OK) st = rbl_pairs(c, s, dev, 0, false, nullptr, nullptr, nullptr);
    }
    if (st == RBMD_OK) st = rbl_correction(c, dev, true, SCAL_FCORR_AUX);
    cudaStreamWaitEvent(main, c->ev_join, 0);
    for (int k = 0; k < nch; ++k) {
        const size_t off = (size_t)A[k] * row, bytes = (size_t)(A[k + 1] - A[k]) * row;
        if (st == RBMD_OK) st = rbe_apply_forces(c, dev, 1, nullptr, B[k], B[k + 1]);
        cudaEventRecord(c->ev_fin[k], main);
        cudaStreamWaitEvent(c->copy, c->ev_fin[k], 0);
        if (st == RBMD_OK)
            st = cuda_status(cudaMemcpyAsync((char *)force + off, (const char *)dev + off, bytes,
                                             cudaMemcpyDefault, c->copy));
    }
    const rbmd_status sync = cuda_status(cudaStreamSynchronize(c->copy));
    if (st == RBMD_OK) st = sync;
    cudaStreamSynchronize(c->side);
    c->step = step;
    c->have_force = false;
    c->bath_set = false;  // a new state or potential: a new bath energy
    if (!vl) c->vl_dirty = true;  // the cell walk re-sorted the atoms
    return leave(c, st);
}

rbmd_status rbmd_step(rbmd_ctx *c, int64_t n_steps)
{
    NvtxRange nvtx_range("rbmd_step");
    if (!c || n_steps < 0) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    if (n_steps == 0) return RBMD_OK;
    enter(c);
    c->lists_cached = c->rho_cached = false;
    rbmd_status s = RBMD_OK;
    if (c->verlet && c->vl_dirty) {
        // the sorted layout was changed outside the step: rebuild the candidates
        if (cudaMemsetAsync(c->ibuf + 4, 1, sizeof(int32_t), c->stream) != cudaSuccess)
            return leave(c, RBMD_ERR_CUDA);
        c->vl_dirty = false;
        c->vl_current = false;  // the rebuild has to run
    }
    if (!c->have_force) {
        k_set_i64<<<1, 1, 0, c->stream>>>(c->d_step, c->step);
        s = forces_into(c, StepRef{nullptr, c->step}, c->force, 0, false, false, nullptr, nullptr,
                        false, c->verlet, c->prm.thermostat == 4);  // the step's kernels
        if (s == RBMD_OK) s = md_thermo_prepare(c);
        if (s != RBMD_OK) return leave(c, s);
        c->have_force = true;
    }
    if (c->profiling && c->prof_eager) {
        // profiled steps launched one kernel at a time, events between stages
        for (int64_t k = 0; k < n_steps; ++k) {
            s = record_step(c);
            if (s != RBMD_OK) return leave(c, s);
            if (cudaEventSynchronize(c->prof_ev[RBMD_PROFILE_STAGES]) != cudaSuccess)
                return leave(c, RBMD_ERR_CUDA);
            for (int st = 0; st < RBMD_PROFILE_STAGES; ++st) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, c->prof_ev[st], c->prof_ev[st + 1]) == cudaSuccess)
                    c->prof_ms[st] += ms;
                else
                    cudaGetLastError();
            }
            ++c->prof_steps;
        }
        c->step += n_steps;
        return leave(c, RBMD_OK);
    }
    if (!c->graph_ready) {
        cudaGraph_t g;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return leave(c, RBMD_ERR_CUDA);
        c->capturing = true;
        c->graph_cond_kernels = 0;
        rbmd_status rs = record_step(c);
        c->capturing = false;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rs != RBMD_OK || e != cudaSuccess) {
            cudaGetLastError();
            return leave(c, rs != RBMD_OK ? rs : RBMD_ERR_CUDA);
        }
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        int nk = 0;
        for (size_t k = 0; k < nn; ++k) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
        }
        c->graph_kernels = nk;
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return leave(c, RBMD_ERR_CUDA);
        c->graph_ready = true;
    }
    for (int64_t k = 0; k < n_steps; ++k) {
        if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) return leave(c, RBMD_ERR_CUDA);
        if (c->profiling) {
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return leave(c, RBMD_ERR_CUDA);
            float ms[RBMD_PROFILE_STAGES];
            bool ok = true;
            for (int st = 0; st < RBMD_PROFILE_STAGES && ok; ++st)
                ok = cudaEventElapsedTime(&ms[st], c->prof_ev[st], c->prof_ev[st + 1]) == cudaSuccess;
            if (!ok) {
                // event nodes of this graph cannot be timed: drop the graph and
                // profile the following steps with eager launches
                cudaGetLastError();
                cudaGraphExecDestroy(c->graph);
                c->graph_ready = false;
                c->prof_eager = true;
                c->step += k + 1;
                return leave(c, rbmd_step(c, n_steps - k - 1));
            }
            for (int st = 0; st < RBMD_PROFILE_STAGES; ++st) c->prof_ms[st] += ms[st];
            ++c->prof_steps;
        }
    }
    c->step += n_steps;
    // the step's candidate-list check ran after its drift: the lists are current
    c->vl_current = c->verlet && !(c->prm.flags & RBMD_NO_RBL);
    return leave(c, RBMD_OK);
}

// Adds the stage times of the last profiled forward (which = 0, nst stages) or
// backward (which = 1) call, once its work has finished.
static void gprof_collect(rbmd_ctx *c, int which, int nst)
{
    if (!c->profiling || !c->gprof_ev[0]) return;
    if (cudaEventSynchronize(c->gprof_ev[nst]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    double *acc = which == 0 ? c->gprof_fwd : c->gprof_bwd;
    for (int k = 0; k < nst; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->gprof_ev[k], c->gprof_ev[k + 1]) == cudaSuccess)
            acc[k] += ms;
        else
            cudaGetLastError();
    }
    ++c->gprof_calls[which];
}

rbmd_status rbmd_energy_batch(rbmd_ctx *c, int64_t step, rbmd_energy_terms *out)
{
    NvtxRange nvtx_range("rbmd_energy");
    if (!c || !out) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    enter(c);
    const int R = c->R;
    memset(out, 0, sizeof(*out) * (size_t)R);
    StepRef r{nullptr, step};
    rbmd_status s = RBMD_OK;
    cudaMemsetAsync(c->ibuf, 0, 4 * sizeof(int32_t), c->stream);
    k_zero_slots<<<(R * 6 + 255) / 256, 256, 0, c->stream>>>(c->scal, R, SCAL_FSUM, 6);
    k_zero_slots<<<(R * (SCAL_COUNT - SCAL_EPAIR) + 255) / 256, 256, 0, c->stream>>>(
        c->scal, R, SCAL_EPAIR, SCAL_COUNT - SCAL_EPAIR);
    gprof_mark(c, 0);
    // as in a force evaluation, the RBE part (which writes only its own scal slots)
    // runs on the side stream beside the RBL part, when the stages are not timed
    const bool fork = !(c->prm.flags & RBMD_NO_RBE) && !(c->prm.flags & RBMD_NO_RBL) && c->side &&
                      !c->profiling;
    if (!(c->prm.flags & RBMD_NO_RBE)) {
        const cudaStream_t main = c->stream;
        if (fork) {
            s = cuda_status(cudaEventRecord(c->ev_fork, main));
            if (s == RBMD_OK) s = cuda_status(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            c->stream = c->side;
        }
        if (s == RBMD_OK) s = rbe_sample(c, r);
        if (s == RBMD_OK) s = rbe_structure_factors(c);
        if (s == RBMD_OK) s = sum_modes(c);
        // the kinetic energy (velocities only, its own scal slot) there too
        if (s == RBMD_OK && fork) s = md_kinetic(c, SCAL_KE_TRUE);
        if (fork) {
            c->stream = main;
            const rbmd_status sj = cuda_status(cudaEventRecord(c->ev_join, c->side));
            if (s == RBMD_OK) s = sj;
        }
    }
    gprof_mark(c, 1);
    if (s == RBMD_OK && !(c->prm.flags & RBMD_NO_RBL)) {
        // through the candidate lists when the context keeps them, else the cell walk
        const bool vl = candidates_for_call(c, 0);
        s = vl ? verlet_prepare_call(c) : cells_build(c);
        gprof_mark(c, 2);
        if (s == RBMD_OK)
            s = vl ? rbl_pairs_verlet(c, r, c->scratch_force, false, true)
                   : rbl_pairs(c, r, c->scratch_force, 0, true, nullptr, nullptr, nullptr);
        gprof_mark(c, 3);
        if (s == RBMD_OK) s = md_sum_replicas_fix(c, c->fpart, SCAL_FSUM, 1.0, false, true);
        if (s == RBMD_OK) s = md_sum_replicas(c, c->epart, EPART, SCAL_EPAIR, 1.0, false, true);
        if (s == RBMD_OK) {
            k_max_count<<<(unsigned)std::min<int64_t>((c->ncell + 255) / 256, 1024), 256, 0,
                          c->stream>>>(c->cell_count, c->ncell, c->ibuf + 1);
        }
    }
    else {
        gprof_mark(c, 2);
        gprof_mark(c, 3);
    }
    if (s == RBMD_OK && !fork) s = md_kinetic(c, SCAL_KE_TRUE);
    if (fork) {
        const rbmd_status sj = cuda_status(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        if (s == RBMD_OK) s = sj;
    }
    gprof_mark(c, 4);
    std::vector<double> h((size_t)R * SCAL_COUNT);
    int32_t hi[4];
    int herr = 0;  // the latched error word, read back with the results
    if (s == RBMD_OK)
        s = cuda_status(cudaMemcpyAsync(h.data(), c->scal, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(hi, c->ibuf, sizeof(hi), cudaMemcpyDeviceToHost, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    s = leave(c, s);
    if (s != RBMD_OK) return s;
    gprof_collect(c, 0, RBMD_PROFILE_FWD_STAGES);
    if (herr != 0) {
        const int z = 0;
        cudaMemcpy(c->err, &z, sizeof(int), cudaMemcpyHostToDevice);
        return (rbmd_status)herr;
    }
    // the lists (complete when no atom overflowed: hi[2]) and the modes and
    // structure factors of this state and step stay for rbmd_energy_backward
    if (!(c->prm.flags & RBMD_NO_RBL) && hi[2] == 0) {
        c->lists_cached = true;
        c->lists_step = step;
    }
    if (!(c->prm.flags & RBMD_NO_RBE)) {
        c->rho_cached = true;
        c->rho_step = step;
    }
    for (int q = 0; q < R; ++q) {
        const double *hr = h.data() + (size_t)q * SCAL_COUNT;
        const Rep &rp = c->reps_h[q];
        rbmd_energy_terms &o = out[q];
        o.e_coul_real = hr[SCAL_EPAIR + 0];
        o.e_lj = hr[SCAL_EPAIR + 1];
        o.e_rbe = hr[SCAL_ERBE];
        o.e_self = rp.e_self;
        o.e_potential = o.e_coul_real + o.e_lj + o.e_rbe + o.e_self;
        o.e_kinetic = hr[SCAL_KE_TRUE];
        o.temperature = rp.N > 1 ? 2.0 * o.e_kinetic / (3.0 * (double)rp.N - 3.0) : 0.0;
        o.S = rp.S;
        for (int d = 0; d < 3; ++d) o.fsum_short[d] = hr[SCAL_FSUM + d];
        o.step = step;
        o.max_shell = hi[0];
        o.max_cell = hi[1];
        o.virial_coul_real = hr[SCAL_EPAIR + 2];
        o.virial_lj = hr[SCAL_EPAIR + 3];
        o.virial_rbe = hr[SCAL_VRBE + 0] + hr[SCAL_VRBE + 1] + hr[SCAL_VRBE + 2];
        for (int k = 0; k < 6; ++k) o.virial[k] = hr[SCAL_EPAIR + 4 + k] + hr[SCAL_VRBE + k];
        const double V = rp.L * rp.L * rp.L;
        o.pressure = (2.0 * o.e_kinetic + o.virial[0] + o.virial[1] + o.virial[2]) / (3.0 * V);
    }
    return RBMD_OK;
}

rbmd_status rbmd_energy(rbmd_ctx *c, int64_t step, rbmd_energy_terms *out)
{
    if (!c || !out || c->R != 1) return RBMD_ERR_INVALID;
    return rbmd_energy_batch(c, step, out);
}

int32_t rbmd_replica_count(rbmd_ctx *c) { return c ? c->R : 0; }

int64_t rbmd_candidate_rebuilds(rbmd_ctx *c)
{
    if (!c) return -1;
    if (!c->verlet) return 0;
    int32_t n = 0;
    if (cudaMemcpyAsync(&n, c->ibuf + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return -1;
    return n;
}

rbmd_status rbmd_set_tiles(rbmd_ctx *c, int32_t cell_div, int32_t rho_tile, int32_t rho_mode_tile)
{
    if (!c) return RBMD_ERR_INVALID;
    if (cell_div != 1 && cell_div != 2) return RBMD_ERR_INVALID;
    if (rho_tile != 512 && rho_tile != 1024 && rho_tile != 2048) return RBMD_ERR_INVALID;
    if (rho_mode_tile != 64 && rho_mode_tile != 128 && rho_mode_tile != 256) return RBMD_ERR_INVALID;
    RBMD_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int2> tl;
    c->ncell = cell_layout(c, cell_div, true);
    c->vl_dirty = true;
    c->ntiles = tile_layout(c, rho_tile, true, tl);
    c->div = cell_div;
    c->rho_tile = rho_tile;
    c->rho_mode_tile = rho_mode_tile;
    RBMD_CHECK_CUDA(cudaMemcpy(c->tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice));
    RBMD_CHECK_CUDA(cudaMemcpy(c->reps, c->reps_h, sizeof(Rep) * c->R, cudaMemcpyHostToDevice));
    if (c->graph_ready) {  // the step graph holds the old grids
        cudaGraphExecDestroy(c->graph);
        c->graph_ready = false;
    }
    return RBMD_OK;
}

rbmd_status rbmd_get_tiles(rbmd_ctx *c, int32_t *out)
{
    if (!c || !out) return RBMD_ERR_INVALID;
    out[0] = c->div;
    out[1] = c->rho_tile;
    out[2] = c->rho_mode_tile;
    out[3] = c->use_table ? 1 : 0;
    return RBMD_OK;
}

rbmd_status rbmd_set_pair_table(rbmd_ctx *c, int32_t on)
{
    if (!c) return RBMD_ERR_INVALID;
    RBMD_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    c->use_table = on != 0;
    if (c->graph_ready) {  // the step graph holds the old kernel arguments
        cudaGraphExecDestroy(c->graph);
        c->graph_ready = false;
    }
    return RBMD_OK;
}

// Times `reps` runs of the RBL part (div only changes the cells) or the
// structure factors (the tile shape only changes those), after one untimed run.
static rbmd_status tune_time(rbmd_ctx *c, bool rbl, StepRef s, int reps, float *ms)
{
    cudaEvent_t e0, e1;
    RBMD_CHECK_CUDA(cudaEventCreate(&e0));
    RBMD_CHECK_CUDA(cudaEventCreate(&e1));
    rbmd_status st = RBMD_OK;
    for (int k = 0; k <= reps && st == RBMD_OK; ++k) {
        if (k == 1) cudaEventRecord(e0, c->stream);
        if (rbl) {
            st = cells_build(c);
            if (st == RBMD_OK) st = rbl_pairs(c, s, c->scratch_force, 0, false, nullptr, nullptr, nullptr);
        } else {
            st = rbe_sample(c, s);
            if (st == RBMD_OK) st = rbe_structure_factors(c);
        }
    }
    cudaEventRecord(e1, c->stream);
    if (st == RBMD_OK) st = cuda_status(cudaEventSynchronize(e1));
    if (st == RBMD_OK) st = cuda_status(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

rbmd_status rbmd_autotune(rbmd_ctx *c, int64_t step, int32_t *chosen)
{
    NvtxRange nvtx_range("rbmd_autotune");
    if (!c) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    enter(c);
    const StepRef s{nullptr, step};
    const int reps = 3;
    int best_div = c->div, best_tile = c->rho_tile, best_mt = c->rho_mode_tile;
    rbmd_status st = RBMD_OK;
    if (!(c->prm.flags & RBMD_NO_RBL)) {
        float best = 1e30f;
        for (int div = 1; div <= 2 && st == RBMD_OK; ++div) {
            float ms = 0.f;
            st = rbmd_set_tiles(c, div, best_tile, best_mt);
            if (st == RBMD_OK) st = tune_time(c, true, s, reps, &ms);
            if (st == RBMD_OK && ms < best) {
                best = ms;
                best_div = div;
            }
        }
    }
    if (!(c->prm.flags & RBMD_NO_RBE)) {
        float best = 1e30f;
        const int tiles[3] = {512, 1024, 2048}, mts[3] = {64, 128, 256};
        for (int a = 0; a < 3 && st == RBMD_OK; ++a)
            for (int b = 0; b < 3 && st == RBMD_OK; ++b) {
                float ms = 0.f;
                st = rbmd_set_tiles(c, best_div, tiles[a], mts[b]);
                if (st == RBMD_OK) st = tune_time(c, false, s, reps, &ms);
                if (st == RBMD_OK && ms < best) {
                    best = ms;
                    best_tile = tiles[a];
                    best_mt = mts[b];
                }
            }
    }
    if (st == RBMD_OK) st = rbmd_set_tiles(c, best_div, best_tile, best_mt);
    if (st == RBMD_OK && !(c->prm.flags & RBMD_NO_RBL)) {
        float ms[2] = {0.f, 0.f};
        for (int on = 0; on < 2 && st == RBMD_OK; ++on) {
            st = rbmd_set_pair_table(c, on);
            if (st == RBMD_OK) st = tune_time(c, true, s, reps, &ms[on]);
        }
        if (st == RBMD_OK) st = rbmd_set_pair_table(c, ms[1] < ms[0]);
    }
    if (st == RBMD_OK && chosen) st = rbmd_get_tiles(c, chosen);
    st = leave(c, st);
    if (st != RBMD_OK) return st;
    return check_latched(c);
}

rbmd_status rbmd_energy_backward(rbmd_ctx *c, int64_t step, double grad_out, void *d_pos, void *d_q,
                                 double *d_eps, double *d_sigma)
{
    NvtxRange nvtx_range("rbmd_energy_backward");
    if (!c) return RBMD_ERR_INVALID;
    if (c->gid) return RBMD_ERR_UNSUPPORTED;  // slab contexts: the calls of rbmd_init_slab
    enter(c);
    StepRef r{nullptr, step};
    rbmd_status s = RBMD_OK;
    gprof_mark(c, 0);
    bool have_lists = !(c->prm.flags & RBMD_NO_RBL) && c->lists_cached && c->lists_step == step;
    if (!(c->prm.flags & RBMD_NO_RBL) && !have_lists && candidates_for_call(c, 0)) {
        // the lists from the candidates, when no atom overflows a capacity
        int32_t ovf = 1;
        s = verlet_prepare_call(c);
        if (s == RBMD_OK) s = rbl_lists_verlet(c, r);
        if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(&ovf, c->ibuf + 2, sizeof(ovf), cudaMemcpyDeviceToHost, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
        if (s != RBMD_OK) return leave(c, s);
        have_lists = ovf == 0;
    }
    if (!(c->prm.flags & RBMD_NO_RBL) && !have_lists) {
        // complete lists of the step: grow the capacities until nothing overflows
        for (int attempt = 0; attempt < 8; ++attempt) {
            s = cells_build(c);
            if (s == RBMD_OK) s = rbl_lists(c, r);
            int32_t h[3] = {0, 0, 0};
            if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(h, c->ibuf, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
            if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
            if (s != RBMD_OK) return leave(c, s);
            if (h[2] == 0) break;
            s = rbl_max_counts(c, c->ibuf);
            if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(h, c->ibuf, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
            if (s != RBMD_OK) return leave(c, s);
            const int cc = (max(h[0], c->list_cc) + 8 + 3) / 4 * 4, cs = (max(h[1], c->list_cs) + 8 + 3) / 4 * 4;
            uint32_t *lc = nullptr, *ls = nullptr;
            if (dev_alloc((void **)&lc, sizeof(int32_t) * (size_t)c->N * cc) != RBMD_OK ||
                dev_alloc((void **)&ls, sizeof(int32_t) * std::max((size_t)c->N * cs, cand_entries(c))) != RBMD_OK) {
                if (lc) cudaFree(lc);
                return leave(c, RBMD_ERR_OOM);
            }
            cudaFree(c->lcore);
            cudaFree(c->lshell);
            c->lcore = (int32_t *)lc;
            c->lshell = (int32_t *)ls;
            if (c->verlet) c->vl_cand = c->lshell;  // shared (the lists were rebuilt anyway)
            c->vl_dirty = true;
            c->list_cc = cc;
            c->list_cs = cs;
            if (c->graph_ready) {  // the step graph holds the old list pointers
                cudaGraphExecDestroy(c->graph);
                c->graph_ready = false;
            }
        }
    }
    gprof_mark(c, 1);
    if (!(c->prm.flags & RBMD_NO_RBE) && !(c->rho_cached && c->rho_step == step)) {
        s = rbe_sample(c, r);
        if (s == RBMD_OK) s = rbe_structure_factors(c);
        if (s != RBMD_OK) return leave(c, s);
    }
    s = adjoint_run(c, grad_out, d_pos, d_q, c->adj_tsum);  // marks stages 2-4
    gprof_mark(c, 5);
    if (s == RBMD_OK && (d_eps || d_sigma)) {
        std::vector<double> h(2 * c->T);
        s = cuda_status(cudaMemcpyAsync(h.data(), c->adj_tsum, sizeof(double) * 2 * c->T,
                                        cudaMemcpyDeviceToHost, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
        if (s == RBMD_OK)
            for (int t = 0; t < c->T; ++t) {
                if (d_eps) d_eps[t] = h[t];
                if (d_sigma) d_sigma[t] = h[c->T + t];
            }
    }
    s = leave(c, s);
    if (s == RBMD_OK) gprof_collect(c, 1, RBMD_PROFILE_GRAD_STAGES);
    return s;
}

rbmd_status rbmd_set_charges(rbmd_ctx *c, const void *charge)
{
    if (!c || !charge) return RBMD_ERR_INVALID;
    enter(c);
    const unsigned nb = (unsigned)((c->N + 255) / 256);
    if (c->fp64)
        k_pack<double><<<nb, 256, 0, c->stream>>>((const double *)charge, c->type, c->N, c->u4, c->q64,
                                                  c->type, c->T, c->err);
    else
        k_pack<float><<<nb, 256, 0, c->stream>>>((const float *)charge, c->type, c->N, c->u4, nullptr,
                                                 c->type, c->T, c->err);
    rbmd_status s = charge_sums(c, false);
    c->have_force = false;
    c->bath_set = false;  // a new state or potential: a new bath energy
    c->vl_dirty = true;
    c->lists_cached = c->rho_cached = false;
    return leave(c, s);
}

rbmd_status rbmd_set_lj(rbmd_ctx *c, const double *lj_eps, const double *lj_sigma)
{
    if (!c || !lj_eps || !lj_sigma) return RBMD_ERR_INVALID;
    enter(c);
    rbmd_status s = upload_lj(c, lj_eps, lj_sigma);
    c->have_force = false;
    c->bath_set = false;  // a new state or potential: a new bath energy
    c->vl_dirty = true;
    return leave(c, s);
}

rbmd_status rbmd_get_state(rbmd_ctx *c, void *pos, void *vel, int64_t *step)
{
    if (!c) return RBMD_ERR_INVALID;
    enter(c);
    const size_t bytes = 3 * c->N * real_size(c);
    void *stage = c->scratch_force;
    rbmd_status s = RBMD_OK;
    if (pos) {
        s = md_decode_state(c, stage, nullptr);
        if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(pos, stage, bytes, cudaMemcpyDefault, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    }
    if (s == RBMD_OK && vel) {
        s = md_decode_state(c, nullptr, stage);
        if (s == RBMD_OK) s = cuda_status(cudaMemcpyAsync(vel, stage, bytes, cudaMemcpyDefault, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    }
    if (step) *step = c->step;
    s = leave(c, s);
    if (s != RBMD_OK) return s;
    return check_latched(c);
}

rbmd_status rbmd_set_state(rbmd_ctx *c, const void *pos, const void *vel, int64_t step)
{
    if (!c) return RBMD_ERR_INVALID;
    enter(c);
    const size_t bytes = 3 * c->N * real_size(c);
    rbmd_status s = RBMD_OK;
    if (pos) {
        s = cuda_status(cudaMemcpyAsync(c->scratch_force, pos, bytes, cudaMemcpyDefault, c->stream));
        if (s == RBMD_OK) s = md_encode_positions(c, c->scratch_force);
    }
    if (s == RBMD_OK && vel) {
        s = cuda_status(cudaMemcpyAsync(c->vel, vel, bytes, cudaMemcpyDefault, c->stream));
        k_set_lambda<<<(c->R + 255) / 256, 256, 0, c->stream>>>(c->scal, c->R, 1.0);
    }
    c->step = step;
    c->have_force = false;
    c->bath_set = false;  // a new state or potential: a new bath energy
    c->vl_dirty = true;
    return leave(c, s);
}

rbmd_status rbmd_get_state_u(rbmd_ctx *c, uint32_t *u, void *vel, int64_t *step)
{
    if (!c) return RBMD_ERR_INVALID;
    enter(c);
    rbmd_status s = RBMD_OK;
    void *stage = c->scratch_force;
    if (u) {
        k_u4_to_u3<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->u4, c->N, (uint32_t *)stage);
        s = cuda_status(cudaMemcpyAsync(u, stage, 3 * c->N * sizeof(uint32_t), cudaMemcpyDefault, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    }
    if (s == RBMD_OK && vel) {
        s = md_decode_state(c, nullptr, stage);
        if (s == RBMD_OK)
            s = cuda_status(cudaMemcpyAsync(vel, stage, 3 * c->N * real_size(c), cudaMemcpyDefault, c->stream));
        if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    }
    if (step) *step = c->step;
    s = leave(c, s);
    if (s != RBMD_OK) return s;
    return check_latched(c);
}

rbmd_status rbmd_set_state_u(rbmd_ctx *c, const uint32_t *u, const void *vel, int64_t step)
{
    if (!c) return RBMD_ERR_INVALID;
    enter(c);
    rbmd_status s = RBMD_OK;
    if (u) {
        s = cuda_status(cudaMemcpyAsync(c->scratch_force, u, 3 * c->N * sizeof(uint32_t), cudaMemcpyDefault, c->stream));
        k_u3_to_u4<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>((const uint32_t *)c->scratch_force, c->N, c->u4);
    }
    if (s == RBMD_OK && vel) {
        s = cuda_status(cudaMemcpyAsync(c->vel, vel, 3 * c->N * real_size(c), cudaMemcpyDefault, c->stream));
        k_set_lambda<<<(c->R + 255) / 256, 256, 0, c->stream>>>(c->scal, c->R, 1.0);
    }
    c->step = step;
    c->have_force = false;
    c->bath_set = false;  // a new state or potential: a new bath energy
    c->vl_dirty = true;
    c->lists_cached = c->rho_cached = false;
    return leave(c, s);
}

rbmd_status rbmd_get_thermostat(rbmd_ctx *c, double *xi)
{
    if (!c || !xi) return RBMD_ERR_INVALID;
    enter(c);
    std::vector<double> h((size_t)c->R * SCAL_COUNT);
    rbmd_status s = cuda_status(cudaMemcpyAsync(h.data(), c->scal, sizeof(double) * h.size(),
                                                cudaMemcpyDeviceToHost, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    if (s == RBMD_OK)
        for (int r = 0; r < c->R; ++r) xi[r] = h[(size_t)r * SCAL_COUNT + SCAL_XI];
    if (s == RBMD_OK && c->prm.thermostat == 4 && !c->bath_set)
        for (int r = 0; r < c->R; ++r) xi[r] = NAN;  // taken by the next rbmd_step
    return leave(c, s);
}

rbmd_status rbmd_set_thermostat(rbmd_ctx *c, const double *xi)
{
    if (!c || !xi) return RBMD_ERR_INVALID;
    enter(c);
    rbmd_status s = RBMD_OK;
    for (int r = 0; r < c->R && s == RBMD_OK; ++r)
        s = cuda_status(cudaMemcpyAsync(c->scal + (size_t)r * SCAL_COUNT + SCAL_XI, xi + r,
                                        sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    c->have_force = false;
    c->bath_set = s == RBMD_OK;
    c->vl_dirty = true;  // the next rbmd_step redoes the first half update
    return leave(c, s);
}

rbmd_status rbmd_sync(rbmd_ctx *c)
{
    if (!c) return RBMD_ERR_INVALID;
    RBMD_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    return check_latched(c);
}

int64_t rbmd_rbe_mode_count(rbmd_ctx *c) { return c ? c->Pm : 0; }

rbmd_status rbmd_rbe_modes(rbmd_ctx *c, int64_t step, int32_t *m, double *rho)
{
    if (!c) return RBMD_ERR_INVALID;
    enter(c);
    StepRef r{nullptr, step};
    rbmd_status s = rbe_sample(c, r);
    if (s == RBMD_OK) s = rbe_structure_factors(c);
    if (s == RBMD_OK && m) {
        const int64_t nm = (int64_t)c->R * c->Pm;
        k_modes_to_m3<<<(unsigned)((nm + 255) / 256), 256, 0, c->stream>>>(c->modes, nm, (int32_t *)c->rho_part);
        s = cuda_status(cudaMemcpyAsync(m, c->rho_part, 3 * nm * sizeof(int32_t), cudaMemcpyDefault, c->stream));
    }
    if (s == RBMD_OK && rho)
        s = cuda_status(cudaMemcpyAsync(rho, c->rho, 2 * (int64_t)c->R * c->Pm * sizeof(double), cudaMemcpyDefault, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    return leave(c, s);
}

rbmd_status rbmd_rbl_lists(rbmd_ctx *c, int64_t step, int32_t *n_core, int32_t *n_shell, int32_t *batch)
{
    if (!c || !n_core || !n_shell || !batch) return RBMD_ERR_INVALID;
    enter(c);
    rbmd_status s = cells_build(c);
    if (s == RBMD_OK)
        s = rbl_pairs(c, StepRef{nullptr, step}, c->scratch_force, 0, false, n_core, n_shell, batch);
    return leave(c, s);
}

rbmd_status rbmd_profile(rbmd_ctx *c, int enable)
{
    if (!c) return RBMD_ERR_INVALID;
    const bool on = enable != 0;
    if (on && !c->prof_ev[0])
        for (int k = 0; k <= RBMD_PROFILE_STAGES; ++k)
            RBMD_CHECK_CUDA(cudaEventCreate(&c->prof_ev[k]));
    if (on && !c->gprof_ev[0])
        for (int k = 0; k <= RBMD_PROFILE_GRAD_STAGES; ++k)
            RBMD_CHECK_CUDA(cudaEventCreate(&c->gprof_ev[k]));
    if (on != c->profiling) {
        RBMD_CHECK_CUDA(cudaStreamSynchronize(c->stream));
        if (c->graph_ready) cudaGraphExecDestroy(c->graph);
        c->graph_ready = false;  // re-captured with (or without) the stage events
        c->profiling = on;
    }
    return RBMD_OK;
}

rbmd_status rbmd_profile_read_grad(rbmd_ctx *c, double *fwd_ms, double *bwd_ms, int64_t *calls,
                                   int reset)
{
    if (!c) return RBMD_ERR_INVALID;
    for (int k = 0; k < RBMD_PROFILE_FWD_STAGES && fwd_ms; ++k) fwd_ms[k] = c->gprof_fwd[k];
    for (int k = 0; k < RBMD_PROFILE_GRAD_STAGES && bwd_ms; ++k) bwd_ms[k] = c->gprof_bwd[k];
    if (calls) {
        calls[0] = c->gprof_calls[0];
        calls[1] = c->gprof_calls[1];
    }
    if (reset) {
        for (int k = 0; k < RBMD_PROFILE_FWD_STAGES; ++k) c->gprof_fwd[k] = 0.0;
        for (int k = 0; k < RBMD_PROFILE_GRAD_STAGES; ++k) c->gprof_bwd[k] = 0.0;
        c->gprof_calls[0] = c->gprof_calls[1] = 0;
    }
    return RBMD_OK;
}

rbmd_status rbmd_profile_read(rbmd_ctx *c, double *ms, int64_t *steps, int reset)
{
    if (!c) return RBMD_ERR_INVALID;
    if (ms)
        for (int k = 0; k < RBMD_PROFILE_STAGES; ++k) ms[k] = c->prof_ms[k];
    if (steps) *steps = c->prof_steps;
    if (reset) {
        for (int k = 0; k < RBMD_PROFILE_STAGES; ++k) c->prof_ms[k] = 0.0;
        c->prof_steps = 0;
    }
    return RBMD_OK;
}

int32_t rbmd_step_kernel_count(rbmd_ctx *c) { return c ? c->graph_kernels : 0; }
int32_t rbmd_rebuild_kernel_count(rbmd_ctx *c) { return c ? c->graph_cond_kernels : 0; }

rbmd_status rbmd_rbe_rho_partial(rbmd_ctx *c, int64_t step, int64_t *acc)
{
    NvtxRange nvtx_range("rbmd_rbe_rho_partial");
    if (!c || !acc) return RBMD_ERR_INVALID;
    if (c->prm.flags & RBMD_NO_RBE) return RBMD_ERR_UNSUPPORTED;
    enter(c);
    rbmd_status s = rbe_sample(c, StepRef{nullptr, step});
    if (s == RBMD_OK) s = rbe_structure_factors(c);
    if (s == RBMD_OK)
        s = cuda_status(cudaMemcpyAsync(acc, c->rho_acc, sizeof(__int128) * 2 * c->R * c->Pm,
                                        cudaMemcpyDeviceToHost, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    s = leave(c, s);
    if (s != RBMD_OK) return s;
    return check_latched(c);
}

void rbmd_rho_acc_add(int64_t *sum, const int64_t *part, int64_t n_modes)
{
    if (!sum || !part) return;
    for (int64_t k = 0; k < 2 * n_modes; ++k) {
        // words (low as unsigned, high as signed) of 128-bit two's-complement integers
        const unsigned __int128 a = ((unsigned __int128)(uint64_t)sum[2 * k + 1] << 64) |
                                    (uint64_t)sum[2 * k];
        const unsigned __int128 b = ((unsigned __int128)(uint64_t)part[2 * k + 1] << 64) |
                                    (uint64_t)part[2 * k];
        const unsigned __int128 t = a + b;
        sum[2 * k] = (int64_t)(uint64_t)t;
        sum[2 * k + 1] = (int64_t)(uint64_t)(t >> 64);
    }
}

rbmd_status rbmd_rbe_forces_rho(rbmd_ctx *c, int64_t step, const int64_t *acc, void *force,
                                int accumulate)
{
    NvtxRange nvtx_range("rbmd_rbe_forces_rho");
    if (!c || !acc || !force) return RBMD_ERR_INVALID;
    if (c->prm.flags & RBMD_NO_RBE) return RBMD_ERR_UNSUPPORTED;
    enter(c);
    rbmd_status s = rbe_sample(c, StepRef{nullptr, step});
    if (s == RBMD_OK)
        s = cuda_status(cudaMemcpyAsync(c->rho_acc, acc, sizeof(__int128) * 2 * c->R * c->Pm,
                                        cudaMemcpyHostToDevice, c->stream));
    if (s == RBMD_OK) s = rbe_rho_from_acc(c, c->rho_acc);
    if (s == RBMD_OK) s = rbe_apply_forces(c, force, accumulate);
    return leave(c, s);
}

rbmd_status rbmd_rbl_forces_slab(rbmd_ctx *c, int64_t step, void *force, int accumulate,
                                 double *fsum)
{
    NvtxRange nvtx_range("rbmd_rbl_forces_slab");
    if (!c || !force || !fsum) return RBMD_ERR_INVALID;
    if (c->prm.flags & RBMD_NO_RBL) return RBMD_ERR_UNSUPPORTED;
    enter(c);
    const StepRef r{nullptr, step};
    rbmd_status s = cells_build(c);
    if (s == RBMD_OK) s = rbl_pairs(c, r, force, accumulate, false, nullptr, nullptr, nullptr);
    if (s == RBMD_OK) s = md_sum_replicas_fix(c, c->fpart, SCAL_FSUM, 1.0, false, true);
    if (s == RBMD_OK)
        s = cuda_status(cudaMemcpyAsync(fsum, c->scal + SCAL_FSUM, 3 * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream));
    if (s == RBMD_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    c->have_force = false;
    c->vl_dirty = true;
    s = leave(c, s);
    if (s != RBMD_OK) return s;
    return check_latched(c);
}

rbmd_status rbmd_add_correction(rbmd_ctx *c, void *force, const double *fsum_total)
{
    if (!c || !force || !fsum_total) return RBMD_ERR_INVALID;
    enter(c);
    const double sc = -1.0 / (double)c->n_glob;
    if (c->fp64)
        k_add_owned<double><<<c->nb256, 256, 0, c->stream>>>((double *)force, c->map256, c->reps,
                                                             sc * fsum_total[0], sc * fsum_total[1],
                                                             sc * fsum_total[2]);
    else
        k_add_owned<float><<<c->nb256, 256, 0, c->stream>>>((float *)force, c->map256, c->reps,
                                                            sc * fsum_total[0], sc * fsum_total[1],
                                                            sc * fsum_total[2]);
    return leave(c, cuda_status(cudaPeekAtLastError()));
}

rbmd_status rbmd_debug_latch_error(rbmd_ctx *c, int32_t code)
{
    if (!c) return RBMD_ERR_INVALID;
    RBMD_CHECK_CUDA(cudaMemcpy(c->err, &code, sizeof(int32_t), cudaMemcpyHostToDevice));
    return RBMD_OK;
}

}  // extern "C"
