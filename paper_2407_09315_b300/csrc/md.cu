// Velocity-Verlet with the Berendsen thermostat, fixed-point state conversion and
// deterministic FP64 reductions.
//
// Sec. 2.1 of arXiv 2407.09315 (velocity-Verlet, Berendsen/NVT).  Positions are
// 32-bit fixed-point fractions of the box: the drift adds rint(v dt 2^32 / L)
// (computed in FP64) and wraps modulo 2^32, which is the periodic wrap.  The
// Berendsen factor lambda = sqrt(1 + (dt/tau)(T0/T - 1)), clamped to [0.8, 1.25]
// with T = 2 KE / (3N - 3), is computed after the second half kick and applied
// lazily: the stored velocities are multiplied by it in the next kick (and in
// every read-out), which saves a separate rescaling pass over the velocities.
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

// First half kick (with the pending Berendsen factor) and drift.
template <typename real>
__global__ void k_kick_drift(uint4 *__restrict__ u4, real *__restrict__ v,
                             const real *__restrict__ F, int64_t N,
                             const double *__restrict__ scal, real hdt, double dtc)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const real lam = (real)scal[SCAL_LAMBDA];
    uint4 A = u4[i];
    uint32_t *pu = &A.x;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // lambda * v rounds on its own (no contraction), exactly as a checkpoint
        // read-out does, so a resumed run is bit-identical to an unbroken one
        real vd = mul_rn(lam, v[3 * i + d]) + hdt * (F[3 * i + d] + (real)scal[SCAL_FCORR + d]);
        v[3 * i + d] = vd;
        const long long du = llrint((double)vd * dtc);
        pu[d] = pu[d] + (uint32_t)du;
    }
    u4[i] = A;
}

// Second half kick and FP64 kinetic-energy block partials; non-finite
// velocities latch RBMD_ERR_NONFINITE.
template <typename real>
__global__ void k_kick_ke(real *__restrict__ v, const real *__restrict__ F, int64_t N,
                          const double *__restrict__ scal, real hdt,
                          double *__restrict__ kepart, int *__restrict__ err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < N) {
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            real vd = v[3 * i + d] + hdt * (F[3 * i + d] + (real)scal[SCAL_FCORR + d]);
            v[3 * i + d] = vd;
            bad |= !isfinite(vd);
            ke += (double)vd * (double)vd;
        }
        if (bad) latch_error(err, RBMD_ERR_NONFINITE);
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

// KE, temperature and the Berendsen factor; optionally advances the device step.
__global__ void k_thermo(const double *__restrict__ kepart, int nparts, int64_t N,
                         double *__restrict__ scal, int thermostat, double dt, double tau,
                         double T0, int64_t *__restrict__ d_step, int advance)
{
    __shared__ double s[256];
    double v = 0.0;
    for (int j = threadIdx.x; j < nparts; j += blockDim.x) v += kepart[j];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double ke = 0.5 * s[0];
    double lam = 1.0;
    if (thermostat == 1 && N > 1) {
        const double T = 2.0 * ke / (3.0 * (double)N - 3.0);
        lam = sqrt(1.0 + (dt / tau) * (T0 / T - 1.0));
        lam = fmin(fmax(lam, 0.8), 1.25);
    }
    scal[SCAL_KE] = ke;
    scal[SCAL_LAMBDA] = lam;
    if (advance) *d_step += 1;
}

rbmd_status md_kick_drift(rbmd_ctx *c)
{
    const int th = 256;
    const unsigned nb = (unsigned)((c->N + th - 1) / th);
    const double hdt = 0.5 * c->prm.dt;
    if (c->fp64)
        k_kick_drift<double><<<nb, th, 0, c->stream>>>(c->u4, (double *)c->vel,
                                                       (const double *)c->force, c->N, c->scal,
                                                       hdt, c->dtc);
    else
        k_kick_drift<float><<<nb, th, 0, c->stream>>>(c->u4, (float *)c->vel,
                                                      (const float *)c->force, c->N, c->scal,
                                                      (float)hdt, c->dtc);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status md_kick_thermo(rbmd_ctx *c, bool advance_step)
{
    const int th = 256;
    const unsigned nb = (unsigned)((c->N + th - 1) / th);
    const double hdt = 0.5 * c->prm.dt;
    if (c->fp64)
        k_kick_ke<double><<<nb, th, 0, c->stream>>>((double *)c->vel, (const double *)c->force,
                                                    c->N, c->scal, hdt, c->kepart, c->err);
    else
        k_kick_ke<float><<<nb, th, 0, c->stream>>>((float *)c->vel, (const float *)c->force, c->N,
                                                   c->scal, (float)hdt, c->kepart, c->err);
    RBMD_LAUNCH_CHECK();
    k_thermo<<<1, 256, 0, c->stream>>>(c->kepart, (int)nb, c->N, c->scal, c->prm.thermostat,
                                       c->prm.dt, c->tau, c->prm.temperature, c->d_step,
                                       advance_step ? 1 : 0);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// Kinetic energy of the true velocities (lambda * stored) into out_dev[0].
template <typename real>
__global__ void k_ke_true(const real *__restrict__ v, int64_t N, const double *__restrict__ scal,
                          double *__restrict__ kepart)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    const double lam = scal[SCAL_LAMBDA];
    if (i < N)
        for (int d = 0; d < 3; ++d) {
            double x = lam * (double)v[3 * i + d];
            ke += x * x;
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

rbmd_status md_kinetic(rbmd_ctx *c, double *out_dev)
{
    const int th = 256;
    const unsigned nb = (unsigned)((c->N + th - 1) / th);
    if (c->fp64) k_ke_true<double><<<nb, th, 0, c->stream>>>((const double *)c->vel, c->N, c->scal, c->kepart);
    else k_ke_true<float><<<nb, th, 0, c->stream>>>((const float *)c->vel, c->N, c->scal, c->kepart);
    RBMD_LAUNCH_CHECK();
    return md_sum(c, c->kepart, (int)nb, 1, out_dev, 0.5);
}

// ---------------------------------------------------------------- state I/O
// Positions -> fixed point: u = floor(frac(x / L) 2^32), computed in FP64.
template <typename real>
__global__ void k_encode(const real *__restrict__ pos, int64_t N, double L, uint4 *__restrict__ u4)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 A = u4[i];
    uint32_t *pu = &A.x;
    for (int d = 0; d < 3; ++d) {
        double f = (double)pos[3 * i + d] / L;
        f -= floor(f);
        double s = floor(f * kTwo32);
        if (s >= kTwo32) s = kTwo32 - 1.0;
        if (!(s >= 0.0)) s = 0.0;
        pu[d] = (uint32_t)s;
    }
    u4[i] = A;
}

template <typename real>
__global__ void k_decode(const uint4 *__restrict__ u4, const real *__restrict__ v, int64_t N,
                         double lscale, const double *__restrict__ scal, real *__restrict__ pos,
                         real *__restrict__ vel)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint4 A = u4[i];
    if (pos) {
        pos[3 * i + 0] = (real)((double)A.x * lscale);
        pos[3 * i + 1] = (real)((double)A.y * lscale);
        pos[3 * i + 2] = (real)((double)A.z * lscale);
    }
    if (vel) {
        const real lam = (real)scal[SCAL_LAMBDA];
        for (int d = 0; d < 3; ++d) vel[3 * i + d] = mul_rn(lam, v[3 * i + d]);
    }
}

rbmd_status md_encode_positions(rbmd_ctx *c, const void *pos)
{
    const unsigned nb = (unsigned)((c->N + 255) / 256);
    if (c->fp64) k_encode<double><<<nb, 256, 0, c->stream>>>((const double *)pos, c->N, c->L, c->u4);
    else k_encode<float><<<nb, 256, 0, c->stream>>>((const float *)pos, c->N, c->L, c->u4);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status md_decode_state(rbmd_ctx *c, void *pos, void *vel)
{
    const unsigned nb = (unsigned)((c->N + 255) / 256);
    if (c->fp64)
        k_decode<double><<<nb, 256, 0, c->stream>>>(c->u4, (const double *)c->vel, c->N, c->lscale,
                                                    c->scal, (double *)pos, (double *)vel);
    else
        k_decode<float><<<nb, 256, 0, c->stream>>>(c->u4, (const float *)c->vel, c->N, c->lscale,
                                                   c->scal, (float *)pos, (float *)vel);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

}  // namespace rbmd
