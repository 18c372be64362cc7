// Velocity-Verlet with the Berendsen thermostat, fixed-point state conversion and
// deterministic FP64 reductions.
//
// Sec. 2.1 of arXiv 2407.09315 (velocity-Verlet, Berendsen/NVT).  Positions are
// 32-bit fixed-point fractions of the box: the drift adds rint(v dt 2^32 / L)
// (computed in FP64) and wraps modulo 2^32, which is the periodic wrap.  The
// Berendsen factor lambda = sqrt(1 + (dt/tau)(T0/T - 1)), clamped to [0.8, 1.25]
// with T = 2 KE / (3N - 3), is computed per replica after the second half kick
// and applied lazily: the stored velocities are multiplied by it in the next
// kick (and in every read-out), which saves a separate rescaling pass.
#include <math.h>

#include "rbmd_internal.cuh"

namespace rbmd {

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Deterministic FP64 sum of nparts partial vectors of ncomp components
// (parts[j * ncomp + c]), one block, fixed order: out[c] = scale * sum_j.
__global__ void k_sum_parts(const double *__restrict__ parts, int nparts, int ncomp,
                            double *__restrict__ out, double scale)
{
    __shared__ double s[256];
    for (int c = 0; c < ncomp; ++c) {
        double v = 0.0;
        for (int j = threadIdx.x; j < nparts; j += blockDim.x) v += parts[(int64_t)j * ncomp + c];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
            if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = scale * s[0];
        __syncthreads();
    }
}

// First stage for long inputs: block b sums the contiguous chunk b of the
// partials (fixed order inside the block), one vector per block.
__global__ void k_sum_chunks(const double *__restrict__ parts, int nparts, int ncomp, int chunk,
                             double *__restrict__ out)
{
    __shared__ double s[256];
    const int j0 = blockIdx.x * chunk, j1 = min(nparts, j0 + chunk);
    for (int c = 0; c < ncomp; ++c) {
        double v = 0.0;
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) v += parts[(int64_t)j * ncomp + c];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
            if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[(int64_t)blockIdx.x * ncomp + c] = s[0];
        __syncthreads();
    }
}

rbmd_status md_sum(rbmd_ctx *c, const double *parts, int nparts, int ncomp, double *out,
                   double scale)
{
    if (nparts > 4096 && ncomp <= 8) {
        // two fixed-order stages: RED_BLOCKS chunk sums, then one block
        const int chunk = (nparts + RED_BLOCKS - 1) / RED_BLOCKS;
        const int nb = (nparts + chunk - 1) / chunk;
        k_sum_chunks<<<nb, 256, 0, c->stream>>>(parts, nparts, ncomp, chunk, c->red_tmp);
        RBMD_LAUNCH_CHECK();
        k_sum_parts<<<1, 256, 0, c->stream>>>(c->red_tmp, nb, ncomp, out, scale);
    } else {
        k_sum_parts<<<1, 256, 0, c->stream>>>(parts, nparts, ncomp, out, scale);
    }
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Per-replica sums of the 4 nb128 per-warp partials of its 128-atom blocks (and
// the same range of the second segment, the overflow fallback's, when *use2 is
// set: a pass without overflowed atoms leaves that segment unwritten, and adding
// its zeros would change no bit) in two fixed-order stages: block
// (k, r) sums chunk k of RED_SPLIT equal chunks of replica r's range, then one
// block per replica adds its RED_SPLIT chunk sums.  The chunking depends only on
// the replica's own size, so a replica sums identically alone or in a batch.
// T: double, or long long for fixed-point partials (exact sums).
template <int NC, typename T>
__global__ void k_sum_replicas1(const T *__restrict__ parts, int64_t seg2,
                                const int32_t *__restrict__ use2, const Rep *__restrict__ reps,
                                T *__restrict__ tmp)
{
    __shared__ T s[NC][256];
    if (seg2 >= 0 && *use2 == 0) seg2 = -1;
    const Rep rp = reps[blockIdx.y];
    const int64_t j0 = 4 * (int64_t)rp.b128_0, nj = 4 * (int64_t)rp.nb128;
    const int64_t chunk = (nj + RED_SPLIT - 1) / RED_SPLIT;
    const int64_t b = blockIdx.x * chunk, e = min(nj, b + chunk);
    T v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = 0;
    for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            v[c] += parts[(j0 + j) * NC + c];
            if (seg2 >= 0) v[c] += parts[(seg2 + j0 + j) * NC + c];
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) {
#pragma unroll
            for (int c = 0; c < NC; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < NC)
        tmp[((int64_t)blockIdx.y * RED_SPLIT + blockIdx.x) * RED_STRIDE + threadIdx.x] = s[threadIdx.x][0];
}

// unit: the value of one unit of T (2^-32 for the fixed-point force sums)
template <typename T>
__global__ void k_sum_replicas2(const T *__restrict__ tmp, int ncomp,
                                const Rep *__restrict__ reps, double *__restrict__ scal, int slot,
                                double scale, int per_atom, double unit)
{
    const int c = threadIdx.x;
    if (c >= ncomp) return;
    const double sc = per_atom ? scale / (double)reps[blockIdx.x].N : scale;
    T v = 0;
    for (int k = 0; k < RED_SPLIT; ++k) v += tmp[((int64_t)blockIdx.x * RED_SPLIT + k) * RED_STRIDE + c];
    scal[(int64_t)blockIdx.x * SCAL_COUNT + slot + c] = sc * ((double)v * unit);
}

rbmd_status md_sum_replicas(rbmd_ctx *c, const double *parts, int ncomp, int slot, double scale,
                            bool per_atom, bool two_segments)
{
    const int64_t seg2 = two_segments ? 4 * (int64_t)c->nb128 : -1;
    const dim3 grid(RED_SPLIT, c->R);
    if (ncomp == 3)
        k_sum_replicas1<3, double><<<grid, 256, 0, c->stream>>>(parts, seg2, c->ibuf + 2, c->reps,
                                                                c->red_rep);
    else if (ncomp == 2)
        k_sum_replicas1<2, double><<<grid, 256, 0, c->stream>>>(parts, seg2, c->ibuf + 2, c->reps,
                                                                c->red_rep);
    else if (ncomp == EPART)
        k_sum_replicas1<EPART, double><<<grid, 256, 0, c->stream>>>(parts, seg2, c->ibuf + 2,
                                                                    c->reps, c->red_rep);
    else return RBMD_ERR_INVALID;
    RBMD_LAUNCH_CHECK();
    k_sum_replicas2<double><<<c->R, 32, 0, c->stream>>>(c->red_rep, ncomp, c->reps, c->scal, slot,
                                                        scale, per_atom ? 1 : 0, 1.0);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status md_sum_replicas_fix(rbmd_ctx *c, const long long *parts, int slot, double scale,
                                bool per_atom, bool two_segments)
{
    const int64_t seg2 = two_segments ? 4 * (int64_t)c->nb128 : -1;
    const dim3 grid(RED_SPLIT, c->R);
    long long *tmp = reinterpret_cast<long long *>(c->red_rep);  // same 8-byte slots
    k_sum_replicas1<3, long long><<<grid, 256, 0, c->stream>>>(parts, seg2, c->ibuf + 2, c->reps,
                                                               tmp);
    RBMD_LAUNCH_CHECK();
    k_sum_replicas2<long long><<<c->R, 32, 0, c->stream>>>(tmp, 3, c->reps, c->scal, slot, scale,
                                                           per_atom ? 1 : 0, 0x1p-32);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// The first half kick and drift of one atom (the state update of the integrator's
// step): v = lambda v + hdt (F + F_corr), u += rint(v dt 2^32 / L) mod 2^32.
template <typename real>
__device__ __forceinline__ void kick_drift_atom(uint4 &A, real (&v)[3], const real (&f)[3],
                                                real lam, const real (&fc)[3], real hdt,
                                                const Rep &rp)
{
    uint32_t *pu = &A.x;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // lambda * v rounds on its own (no contraction), exactly as a checkpoint
        // read-out does, so a resumed run is bit-identical to an unbroken one
        real vd = mul_rn(lam, v[d]) + hdt * (f[d] + fc[d]);
        v[d] = vd;
        long long du;
        if constexpr (sizeof(real) == 4) {
            // vd * dtc with dtc = dhi + dlo (two floats): p1 + e1 = vd dhi exactly,
            // t = vd dlo + e1; the rounding of p1 + t to an integer, in FP32 (FP64
            // operations are scarce on this GPU).  The product is good to about
            // 1e-10 units, so the integer is that of the FP64 product except within
            // that distance of a half-integer.
            const float dhi = rp.dtc_hi, dlo = rp.dtc_lo;
            const float p1 = __fmul_rn(vd, dhi);
            const float e1 = __fmaf_rn(vd, dhi, -p1);
            const float t = __fmaf_rn(vd, dlo, e1);
            const float r = rintf(p1);
            du = (long long)r + (long long)rintf(__fadd_rn(__fsub_rn(p1, r), t));
        } else {
            du = llrint((double)vd * rp.dtc);
        }
        pu[d] = pu[d] + (uint32_t)du;
    }
}

// First half kick (with the pending thermostat factor) and drift: AT atoms per
// thread (atoms j, j + 256/AT, ... of the 256-atom block), their loads issued
// together.
template <typename real, int AT>
__global__ void __launch_bounds__(256 / AT) k_kick_drift(uint4 *__restrict__ u4, real *__restrict__ v,
                             const real *__restrict__ F, const int2 *__restrict__ map,
                             const Rep *__restrict__ reps, const double *__restrict__ scal,
                             real hdt, int32_t *__restrict__ count, int32_t *__restrict__ cell_of,
                             int32_t *__restrict__ rank)
{
    constexpr int TB = 256 / AT;
    const int2 mb = map[blockIdx.x];
    const int r = mb.x;
    const Rep &rp = reps[r];
    const int64_t end = rp.atom0 + rp.N;
    const double *sc = scal + (int64_t)r * SCAL_COUNT;
    const real lam = (real)sc[SCAL_LAMBDA_KICK];
    const real fc[3] = {(real)sc[SCAL_FCORR], (real)sc[SCAL_FCORR + 1], (real)sc[SCAL_FCORR + 2]};
    uint4 A[AT];
    real vv[AT][3], ff[AT][3];
#pragma unroll
    for (int h = 0; h < AT; ++h) {
        const int64_t i = (int64_t)mb.y + threadIdx.x + h * TB;
        if (i < end) {
            A[h] = u4[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                vv[h][d] = v[3 * i + d];
                ff[h][d] = F[3 * i + d];
            }
        }
    }
#pragma unroll
    for (int h = 0; h < AT; ++h) {
        const int64_t i = (int64_t)mb.y + threadIdx.x + h * TB;
        if (i >= end) continue;
        kick_drift_atom(A[h], vv[h], ff[h], lam, fc, hdt, rp);
#pragma unroll
        for (int d = 0; d < 3; ++d) v[3 * i + d] = vv[h][d];
        u4[i] = A[h];
        if (count) {
            const int nc = rp.nc;
            const int64_t c = rp.cell0 +
                              ((int64_t)cell_coord(A[h].x, nc) * nc + cell_coord(A[h].y, nc)) * nc +
                              cell_coord(A[h].z, nc);
            cell_of[i] = (int32_t)c;
            rank[i] = atomicAdd(&count[c], 1);
        }
    }
}

// Second half kick and FP64 kinetic-energy block partials (second_kick); used when
// the step has no RBE force kernel to carry the kick in its epilogue.
template <typename real>
__global__ void k_kick_ke(real *__restrict__ v, real *__restrict__ F,
                          const int2 *__restrict__ map, const Rep *__restrict__ reps,
                          KickArgs<real> k)
{
    const AtomSlot a = atom_slot(map, reps);
    double ke = 0.0;
    if (a.ok) {
        real f[3] = {F[3 * a.i], F[3 * a.i + 1], F[3 * a.i + 2]};
        real fc[3];
        kick_fcorr(k, a.r, fc);
        ke = second_kick(k, reps[a.r], a.r, a.i, v, F, f, fc);
    }
    block_ke_partial(ke, k.kepart);
}

// One block per replica: KE, temperature and the thermostat factors; block 0
// optionally advances the device step counter.
//   Berendsen:   lambda = sqrt(1 + (dt/tau)(T0/T - 1)) in [0.8, 1.25], applied on
//                read-out and by the next kick;
//   Langevin:    no rescale;
//   Nose-Hoover: lambda1 = e^{-xi dt/2} (second half of the step), the end-of-
//                step update xi += dt/2 (2K' - g T0)/Q with K' = lambda1^2 K, then
//                the next step's first update (same K') and lambda2 = e^{-xi dt/2};
//                read-out uses lambda1, the next kick lambda1 lambda2;
//   energy bath: lambda^2 = a = 1 + (dt/tau)((E0 - U)/K - 1), a clamped to
//                [0.64, 1.5625], no rescale at K = 0; U the potential of the step's
//                force evaluation (its energy sums in scal), E0 in SCAL_XI; applied
//                like the Berendsen factor.
__global__ void k_thermo(const double *__restrict__ kepart, const Rep *__restrict__ reps,
                         double *__restrict__ scal, int thermostat, double dt, double tau,
                         int64_t *__restrict__ d_step, int advance)
{
    __shared__ double s[1024];
    const Rep rp = reps[blockIdx.x];
    double v = 0.0;
    for (int j = threadIdx.x; j < rp.nb256; j += blockDim.x) v += kepart[rp.b256_0 + j];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double ke = 0.5 * s[0];
    double *sc = scal + (int64_t)blockIdx.x * SCAL_COUNT;
    double lam = 1.0, lam_kick = 1.0;
    const double g = 3.0 * (double)rp.N - 3.0;
    if (thermostat == 1 && rp.N > 1) {
        const double T = 2.0 * ke / g;
        lam = sqrt(1.0 + (dt / tau) * (rp.T0 / T - 1.0));
        lam = fmin(fmax(lam, 0.8), 1.25);
        lam_kick = lam;
    } else if (thermostat == 3 && rp.N > 1) {
        const double Q = g * rp.T0 * tau * tau;
        const double lam1 = exp(-0.5 * dt * sc[SCAL_XI_RUN]);
        const double k1 = lam1 * lam1 * ke;
        const double xi_b = sc[SCAL_XI_RUN] + 0.5 * dt * (2.0 * k1 - g * rp.T0) / Q;
        const double xi_r = xi_b + 0.5 * dt * (2.0 * k1 - g * rp.T0) / Q;
        sc[SCAL_XI] = xi_b;
        sc[SCAL_XI_RUN] = xi_r;
        lam = lam1;
        lam_kick = lam1 * exp(-0.5 * dt * xi_r);
    } else if (thermostat == 4 && ke > 0.0) {
        const double U = sc[SCAL_EPAIR] + sc[SCAL_EPAIR + 1] + sc[SCAL_ERBE] + rp.e_self;
        const double a = 1.0 + (dt / tau) * ((sc[SCAL_XI] - U) / ke - 1.0);
        lam = a <= 0.64 ? 0.8 : (a >= 1.5625 ? 1.25 : sqrt(a));
        lam_kick = lam;
    }
    sc[SCAL_KE] = ke;
    sc[SCAL_LAMBDA] = lam;
    sc[SCAL_LAMBDA_KICK] = lam_kick;
    if (advance && blockIdx.x == 0) *d_step += 1;
}

// Before the first step of a run (Nose-Hoover only): the first half update of the
// step, xi_run = xi + dt/2 (2K - g T0)/Q with K the kinetic energy of the read-out
// velocities (SCAL_KE_TRUE), and the kick factor lambda e^{-xi_run dt/2}.
__global__ void k_nh_prepare(const Rep *__restrict__ reps, int R, double *__restrict__ scal,
                             double dt, double tau)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const Rep rp = reps[r];
    double *sc = scal + (int64_t)r * SCAL_COUNT;
    if (rp.N < 2) {
        sc[SCAL_LAMBDA_KICK] = sc[SCAL_LAMBDA];
        return;
    }
    const double g = 3.0 * (double)rp.N - 3.0, Q = g * rp.T0 * tau * tau;
    const double xi_r = sc[SCAL_XI] + 0.5 * dt * (2.0 * sc[SCAL_KE_TRUE] - g * rp.T0) / Q;
    sc[SCAL_XI_RUN] = xi_r;
    sc[SCAL_LAMBDA_KICK] = sc[SCAL_LAMBDA] * exp(-0.5 * dt * xi_r);
}

rbmd_status md_kick_drift(rbmd_ctx *c, bool bin)
{
    const double hdt = 0.5 * c->prm.dt;
    int32_t *count = bin ? c->cell_count : nullptr;
    if (bin)
        RBMD_CHECK_CUDA(cudaMemsetAsync(c->cell_count, 0, sizeof(int32_t) * c->ncell, c->stream));
    if (c->fp64)
        k_kick_drift<double, 1><<<c->nb256, 256, 0, c->stream>>>(
            c->u4, (double *)c->vel, (const double *)c->force, c->map256, c->reps, c->scal, hdt,
            count, c->cell_of, c->cell_rank);
    else
        k_kick_drift<float, 2><<<c->nb256, 128, 0, c->stream>>>(
            c->u4, (float *)c->vel, (const float *)c->force, c->map256, c->reps, c->scal,
            (float)hdt, count, c->cell_of, c->cell_rank);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

template <typename real>
KickArgs<real> kick_args(rbmd_ctx *c, StepRef sref)
{
    KickArgs<real> k;
    k.v = (real *)c->vel;
    k.scal = c->scal;
    k.hdt = (real)(0.5 * c->prm.dt);
    k.kepart = c->kepart;
    k.err = c->err;
    k.langevin = c->prm.thermostat == 2 ? 1 : 0;
    k.gamma = 1.0 / c->tau;
    k.dt = c->prm.dt;
    k.sref = sref;
    return k;
}
template KickArgs<float> kick_args<float>(rbmd_ctx *, StepRef);
template KickArgs<double> kick_args<double>(rbmd_ctx *, StepRef);

rbmd_status md_kick_thermo(rbmd_ctx *c, bool advance_step, StepRef sref, bool kicked)
{
    if (!kicked) {
        if (c->fp64)
            k_kick_ke<double><<<c->nb256, 256, 0, c->stream>>>(
                (double *)c->vel, (double *)c->force, c->map256, c->reps, kick_args<double>(c, sref));
        else
            k_kick_ke<float><<<c->nb256, 256, 0, c->stream>>>(
                (float *)c->vel, (float *)c->force, c->map256, c->reps, kick_args<float>(c, sref));
        RBMD_LAUNCH_CHECK();
    }
    k_thermo<<<c->R, 1024, 0, c->stream>>>(c->kepart, c->reps, c->scal, c->prm.thermostat,
                                          c->prm.dt, c->tau, c->d_step, advance_step ? 1 : 0);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Kinetic energy of the true velocities (lambda * stored), per 256-atom block.
template <typename real>
__global__ void k_ke_true(const real *__restrict__ v, const int2 *__restrict__ map,
                          const Rep *__restrict__ reps, const double *__restrict__ scal,
                          double *__restrict__ kepart)
{
    const AtomSlot a = atom_slot(map, reps);
    double ke = 0.0;
    if (a.ok) {
        const double lam = scal[(int64_t)a.r * SCAL_COUNT + SCAL_LAMBDA];
        for (int d = 0; d < 3; ++d) {
            const double x = lam * (double)v[3 * a.i + d];
            ke += x * x;
        }
    }
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        kepart[blockIdx.x] = t;
    }
}

// One block per replica: 1/2 * sum of its 256-atom block partials into slot.
__global__ void k_sum_ke(const double *__restrict__ kepart, const Rep *__restrict__ reps,
                         double *__restrict__ scal, int slot)
{
    __shared__ double s[1024];
    const Rep rp = reps[blockIdx.x];
    double v = 0.0;
    for (int j = threadIdx.x; j < rp.nb256; j += blockDim.x) v += kepart[rp.b256_0 + j];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[(int64_t)blockIdx.x * SCAL_COUNT + slot] = 0.5 * s[0];
}

rbmd_status md_kinetic(rbmd_ctx *c, int slot)
{
    if (c->fp64)
        k_ke_true<double><<<c->nb256, 256, 0, c->stream>>>((const double *)c->vel, c->map256,
                                                           c->reps, c->scal, c->kepart);
    else
        k_ke_true<float><<<c->nb256, 256, 0, c->stream>>>((const float *)c->vel, c->map256,
                                                          c->reps, c->scal, c->kepart);
    RBMD_LAUNCH_CHECK();
    k_sum_ke<<<c->R, 1024, 0, c->stream>>>(c->kepart, c->reps, c->scal, slot);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Energy bath at the start of a run without a set E0: E0 = K + U of the state the
// run starts from (K of the read-out velocities, U from the energy sums of the
// force evaluation of that state).
__global__ void k_bath_prepare(const Rep *__restrict__ reps, int R, double *__restrict__ scal)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double *sc = scal + (int64_t)r * SCAL_COUNT;
    const double U = sc[SCAL_EPAIR] + sc[SCAL_EPAIR + 1] + sc[SCAL_ERBE] + reps[r].e_self;
    sc[SCAL_XI] = sc[SCAL_KE_TRUE] + U;
}

rbmd_status md_thermo_prepare(rbmd_ctx *c)
{
    if (c->prm.thermostat == 4 && !c->bath_set) {
        RBMD_CHECK(md_kinetic(c, SCAL_KE_TRUE));
        k_bath_prepare<<<(c->R + 127) / 128, 128, 0, c->stream>>>(c->reps, c->R, c->scal);
        RBMD_LAUNCH_CHECK();
        c->bath_set = true;
        return RBMD_OK;
    }
    if (c->prm.thermostat != 3) return RBMD_OK;
    RBMD_CHECK(md_kinetic(c, SCAL_KE_TRUE));
    k_nh_prepare<<<(c->R + 127) / 128, 128, 0, c->stream>>>(c->reps, c->R, c->scal, c->prm.dt,
                                                            c->tau);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// ---------------------------------------------------------------- state I/O
// Positions -> fixed point: u = floor(frac(x / L) 2^32), computed in FP64.
template <typename real>
__global__ void k_encode(const real *__restrict__ pos, const int2 *__restrict__ map,
                         const Rep *__restrict__ reps, uint4 *__restrict__ u4)
{
    const AtomSlot a = atom_slot(map, reps);
    if (!a.ok) return;
    const double L = reps[a.r].L;
    uint4 A = u4[a.i];
    uint32_t *pu = &A.x;
    for (int d = 0; d < 3; ++d) {
        double f = (double)pos[3 * a.i + d] / L;
        f -= floor(f);
        double s = floor(f * kTwo32);
        if (s >= kTwo32) s = kTwo32 - 1.0;
        if (!(s >= 0.0)) s = 0.0;
        pu[d] = (uint32_t)s;
    }
    u4[a.i] = A;
}

template <typename real>
__global__ void k_decode(const uint4 *__restrict__ u4, const real *__restrict__ v,
                         const int2 *__restrict__ map, const Rep *__restrict__ reps,
                         const double *__restrict__ scal, real *__restrict__ pos,
                         real *__restrict__ vel)
{
    const AtomSlot a = atom_slot(map, reps);
    if (!a.ok) return;
    const int64_t i = a.i;
    const uint4 A = u4[i];
    if (pos) {
        const double ls = reps[a.r].lscale;
        pos[3 * i + 0] = (real)((double)A.x * ls);
        pos[3 * i + 1] = (real)((double)A.y * ls);
        pos[3 * i + 2] = (real)((double)A.z * ls);
    }
    if (vel) {
        const real lam = (real)scal[(int64_t)a.r * SCAL_COUNT + SCAL_LAMBDA];
        for (int d = 0; d < 3; ++d) vel[3 * i + d] = mul_rn(lam, v[3 * i + d]);
    }
}

rbmd_status md_encode_positions(rbmd_ctx *c, const void *pos)
{
    c->lists_cached = c->rho_cached = false;
    if (c->fp64) k_encode<double><<<c->nb256, 256, 0, c->stream>>>((const double *)pos, c->map256, c->reps, c->u4);
    else k_encode<float><<<c->nb256, 256, 0, c->stream>>>((const float *)pos, c->map256, c->reps, c->u4);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// The same for the atoms of the 256-atom blocks [b0, b1) of map256.
rbmd_status md_encode_blocks(rbmd_ctx *c, const void *pos, int b0, int b1)
{
    c->lists_cached = c->rho_cached = false;
    if (b1 <= b0) return RBMD_OK;
    const unsigned nb = (unsigned)(b1 - b0);
    if (c->fp64) k_encode<double><<<nb, 256, 0, c->stream>>>((const double *)pos, c->map256 + b0, c->reps, c->u4);
    else k_encode<float><<<nb, 256, 0, c->stream>>>((const float *)pos, c->map256 + b0, c->reps, c->u4);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status md_decode_state(rbmd_ctx *c, void *pos, void *vel)
{
    if (c->fp64)
        k_decode<double><<<c->nb256, 256, 0, c->stream>>>(c->u4, (const double *)c->vel, c->map256,
                                                          c->reps, c->scal, (double *)pos,
                                                          (double *)vel);
    else
        k_decode<float><<<c->nb256, 256, 0, c->stream>>>(c->u4, (const float *)c->vel, c->map256,
                                                         c->reps, c->scal, (float *)pos,
                                                         (float *)vel);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

}  // namespace rbmd
