// Random batch Ewald on the device: mode sampling, structure factors and forces.
//
// Sec. 2.2 (Eqs. 9, 11, 12) and Algorithm 1 of arXiv 2407.09315.  The paper
// samples the P modes with a Metropolis chain on the CPU and copies them to the
// GPU every step; here they are drawn i.i.d. on the device (exact inverse CDF per
// dimension, Philox4x32-10 keyed by seed, step and mode index), which keeps the
// step free of host round trips and lets it be captured in a CUDA graph.
//
// Phases are computed exactly in integer arithmetic: with fixed-point positions
// u (units of L/2^32), k.r = 2 pi (m . u mod 2^32) / 2^32, so the wrapped phase
// is known to 2^-32 of a turn whatever the box size; only the final conversion
// to a fraction of a turn rounds.
#include <math.h>

#include <algorithm>

#include "rbmd_internal.cuh"

namespace rbmd {

// --------------------------------------------------------------------------
// Sampler thresholds (host).  The density of Eq. 12 factorises over the three
// axes, exp(-k^2/4alpha) = prod_d exp(-a m_d^2) with a = pi^2/(alpha L^2).
// M is the smallest half-width with a M^2 >= ln(1e16); T[j] = min(2^64 - 1,
// floor(CDF_j 2^64)) for j = 0..2M, CDF_j the cumulative weight of m = -M..j-M.
// --------------------------------------------------------------------------
rbmd_status sampler_table_host(double L, double alpha, int32_t *Mout, uint64_t *T, double *Hout)
{
    if (!(L > 0.0) || !(alpha > 0.0)) return RBMD_ERR_INVALID;
    const double a = kPi * kPi / (alpha * L * L);
    const double half_width = ceil(sqrt(16.0 * log(10.0) / a));
    if (half_width > 1.0e7) return RBMD_ERR_INVALID;
    const int M = (int)half_width;
    if (Mout) *Mout = M;
    if (!T && !Hout) return RBMD_OK;
    const int n = 2 * M + 1;
    double *cum = new double[n];
    double total = 0.0;
    for (int j = 0; j < n; ++j) {
        double m = (double)(j - M);
        total += exp(-a * m * m);
        cum[j] = total;
    }
    if (T) {
        for (int j = 0; j < n; ++j) {
            double x = (cum[j] / total) * kTwo64;
            T[j] = (x >= kTwo64) ? UINT64_MAX : (uint64_t)x;
        }
    }
    if (Hout) *Hout = total;
    delete[] cum;
    return RBMD_OK;
}

// Number of thresholds T[0..2M-1] not above U, minus M: the inverse CDF.
__device__ __forceinline__ int draw_axis(uint64_t U, const uint64_t *__restrict__ T, int M)
{
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (T[mid] <= U) lo = mid + 1;
        else hi = mid;
    }
    return lo - M;
}

// One thread per mode l: attempt t draws U_x, U_y from Philox(l, t, step, stream)
// and U_z from Philox(l, t | 2^31, step, stream); m = 0 is redrawn (k != 0 in
// Eq. 12).  After RBMD_MAX_ATTEMPTS zero draws the mode stays 0 (zero weight).
// Grid (mode blocks, replicas): each block stages its replica's threshold table in
// shared memory when it fits (SAMPLE_SMEM_MAX entries) and searches it there.
constexpr int SAMPLE_SMEM_MAX = 6144;  // 48 KB of thresholds

__global__ void k_rbe_sample(const uint64_t *__restrict__ Tall, const Rep *__restrict__ reps,
                             int64_t P, StepRef sref, int4 *__restrict__ modes)
{
    extern __shared__ uint64_t s_T[];
    const int r = blockIdx.y;
    const Rep rp = reps[r];
    const int M = rp.M, nT = 2 * M + 1;
    const uint64_t *T = Tall + rp.cdf0;
    if (nT <= SAMPLE_SMEM_MAX) {
        for (int j = threadIdx.x; j < nT; j += blockDim.x) s_T[j] = T[j];
        __syncthreads();
        T = s_T;
    }
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    const uint2 key = rp.key;
    const uint32_t step = (uint32_t)step_of(sref);
    const uint32_t tag = rp.tag_rbe;
    int mx = 0, my = 0, mz = 0;
    for (uint32_t t = 0; t < RBMD_MAX_ATTEMPTS; ++t) {
        uint4 w = philox10(make_uint4((uint32_t)l, t, step, tag), key);
        uint4 w2 = philox10(make_uint4((uint32_t)l, t | 0x80000000u, step, tag), key);
        mx = draw_axis(((uint64_t)w.x << 32) | w.y, T, M);
        my = draw_axis(((uint64_t)w.z << 32) | w.w, T, M);
        mz = draw_axis(((uint64_t)w2.x << 32) | w2.y, T, M);
        if (mx != 0 || my != 0 || mz != 0) break;
    }
    modes[(int64_t)r * P + l] = make_int4(mx, my, mz, 0);
}

// --------------------------------------------------------------------------
// Metropolis mode chains (Algorithm 1 step 1), one thread per (replica, chain).
// Acceptance thresholds A_k = min(2^64 - 1, floor(exp(-a (2k + 1)) 2^64)) on the
// host; the chains advance from the step they hold to the requested one (or are
// replayed from step 0 when it lies before), `moves` moves per step.
// --------------------------------------------------------------------------
rbmd_status metropolis_table_host(double L, double alpha, int M, uint64_t *A)
{
    if (!(L > 0.0) || !(alpha > 0.0) || M < 1) return RBMD_ERR_INVALID;
    const double a = kPi * kPi / (alpha * L * L);
    for (int k = 0; k <= 2 * M; ++k) {
        const double x = exp(-a * (2.0 * k + 1.0)) * kTwo64;
        A[k] = (x >= kTwo64) ? UINT64_MAX : (uint64_t)x;
    }
    return RBMD_OK;
}

__global__ void k_rbe_metropolis(const uint64_t *__restrict__ Aall, const Rep *__restrict__ reps,
                                 int64_t P, StepRef sref, const int64_t *__restrict__ chain_step,
                                 const int4 *__restrict__ modes0, int4 *__restrict__ modes,
                                 int moves)
{
    const int r = blockIdx.y;
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    const Rep rp = reps[r];
    const uint64_t *A = Aall + rp.cdf0;
    const int kmax = 2 * rp.M;
    const int64_t target = step_of(sref);
    int64_t s0 = *chain_step;
    const int64_t t = (int64_t)r * P + l;
    int4 m = modes[t];
    if (target < s0) {  // replay from step 0
        m = modes0[t];
        s0 = 0;
    }
    const uint32_t tag = (rp.tag_rbe & ~0xFFu) | RBMD_STREAM_METROPOLIS;
    for (int64_t st = s0 + 1; st <= target; ++st) {
        for (int mv = 0; mv < moves; ++mv) {
            const uint4 w = philox10(make_uint4((uint32_t)l, (uint32_t)mv, (uint32_t)st, tag), rp.key);
            const int d = (int)(w.x % 3u);
            const int delta = (w.y & 1u) ? 1 : -1;
            const uint64_t U = ((uint64_t)w.z << 32) | w.w;
            const int md = d == 0 ? m.x : (d == 1 ? m.y : m.z);
            const int mn = md + delta;
            // m' = 0 is rejected
            const bool zero = mn == 0 && (d == 0 ? (m.y == 0 && m.z == 0)
                                                 : d == 1 ? (m.x == 0 && m.z == 0)
                                                          : (m.x == 0 && m.y == 0));
            bool accept;
            if (delta * md < 0) {
                accept = true;
            } else {
                const int k = md < 0 ? -md : md;
                accept = k <= kmax && U < A[k];
            }
            if (accept && !zero) {
                if (d == 0) m.x = mn;
                else if (d == 1) m.y = mn;
                else m.z = mn;
            }
        }
    }
    modes[t] = m;
}

__global__ void k_set_chain_step(int64_t *chain_step, StepRef sref) { *chain_step = step_of(sref); }

rbmd_status rbe_metropolis_init(rbmd_ctx *c)
{
    const int threads = 128;
    const dim3 grid((unsigned)((c->Pm + threads - 1) / threads), (unsigned)c->R);
    int nmax = 0;
    for (int r = 0; r < c->R; ++r) nmax = std::max(nmax, 2 * c->reps_h[r].M + 1);
    const size_t smem = sizeof(uint64_t) * (size_t)std::min(nmax, SAMPLE_SMEM_MAX);
    k_rbe_sample<<<grid, threads, smem, c->stream>>>(c->cdf, c->reps, c->Pm, StepRef{nullptr, 0},
                                                      c->modes0);
    RBMD_LAUNCH_CHECK();
    RBMD_CHECK_CUDA(cudaMemcpyAsync(c->modes, c->modes0, sizeof(int4) * (size_t)c->R * c->Pm,
                                    cudaMemcpyDeviceToDevice, c->stream));
    RBMD_CHECK_CUDA(cudaMemsetAsync(c->chain_step, 0, sizeof(int64_t), c->stream));
    return RBMD_OK;
}

rbmd_status rbe_sample(rbmd_ctx *c, StepRef s)
{
    c->rho_cached = false;
    if (c->full_modes) return RBMD_OK;  // fixed list built at init
    const int threads = 128;
    if (c->modes0) {
        const dim3 g((unsigned)((c->Pm + threads - 1) / threads), (unsigned)c->R);
        k_rbe_metropolis<<<g, threads, 0, c->stream>>>(c->acc, c->reps, c->Pm, s, c->chain_step,
                                                       c->modes0, c->modes, c->mh_moves);
        RBMD_LAUNCH_CHECK();
        k_set_chain_step<<<1, 1, 0, c->stream>>>(c->chain_step, s);
        RBMD_LAUNCH_CHECK();
        return RBMD_OK;
    }
    const dim3 grid((unsigned)((c->Pm + threads - 1) / threads), (unsigned)c->R);
    int nmax = 0;
    for (int r = 0; r < c->R; ++r) nmax = std::max(nmax, 2 * c->reps_h[r].M + 1);
    const size_t smem = sizeof(uint64_t) * (size_t)std::min(nmax, SAMPLE_SMEM_MAX);
    k_rbe_sample<<<grid, threads, smem, c->stream>>>(c->cdf, c->reps, c->Pm, s, c->modes);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// --------------------------------------------------------------------------
// Structure factors, Eq. 9 (Algorithm 1 steps 2-3, the paper's Reduce-by-Key).
// Block (x = atom tile, y = mode tile): the atom tile and the modes are staged
// in shared memory; work item (mode l, sub-tile s) sums q_j e^{i theta_jl} over
// its atoms with the thread's own compensated (Kahan) FP32 accumulators, one
// compensated addition per four atoms (plain FP64 in FP64 contexts).  Items of
// one warp share s, so every lane reads the same atom: a shared-memory broadcast.  The sub-tile sums are combined in FP64
// in a fixed order and one partial per (atom tile, mode) goes to HBM.
// --------------------------------------------------------------------------
// FP64 phase factors by angle addition.  The phase is an exact 32-bit fraction of
// a turn, so with ph = h 2^16 + l, e^{i theta} = T[h] T'[l] where
// T[h] = e^{2 pi i h/2^16} and T'[l] = e^{2 pi i l/2^32}: two reads of a 2 MB
// table (L2-resident) and one complex product replace a sincospi, whose cost
// bounds the FP64 kernels (B300 runs few FP64 operations per clock).  The entries
// are sincospi of exact arguments; the product adds a few units in the last
// place.  Layout: {cos, sin}, T at [0, 65536), T' at [65536, 131072).  (A
// 10 + 11 + 11-bit split with an 80 KB table and two products measured slower:
// the FP64 operations, not the table reads, bound these kernels.)
// (phase_sincos_tab in rbmd_internal.cuh reads it.)
constexpr int PHASE_TAB = 131072;

__global__ void k_phase_table(double2 *__restrict__ tab)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= PHASE_TAB) return;
    const double x = j < 65536 ? (double)j * 0x1p-15 : (double)(j - 65536) * 0x1p-31;  // angle / pi
    double s, c;
    sincospi(x, &s, &c);
    tab[j] = make_double2(c, s);
}

// Explicitly rounded operations for the force passes: the same force must come out
// of the kernel variants with and without the integrator's kick (a resumed run
// computes its first force without it), so no contraction is left to the compiler.
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_r(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_r(double a, double b) { return __dadd_rn(a, b); }

__device__ __forceinline__ void kahan_add(float &s, float &comp, float x)
{
    float y = x - comp;
    float t = s + y;
    comp = (t - s) - y;
    s = t;
}

template <typename real>
__global__ void __launch_bounds__(1024, sizeof(real) == 4 ? 2 : 1) k_rho_partial(const uint4 *__restrict__ u4, const double *__restrict__ q64,
                              const int2 *__restrict__ tiles, const Rep *__restrict__ reps,
                              const int4 *__restrict__ modes_all, int64_t Pm, int tile_atoms,
                              int mode_tile, int sub, double2 *__restrict__ part, int tile0,
                              int ntiles_all, const double2 *__restrict__ ptab)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint4 *s_at = reinterpret_cast<uint4 *>(smem);
    double *s_q = reinterpret_cast<double *>(s_at + tile_atoms);  // FP64 contexts only
    int4 *s_m = reinterpret_cast<int4 *>(s_q + (sizeof(real) == 8 ? tile_atoms : 0));
    double2 *s_acc = reinterpret_cast<double2 *>(s_m + mode_tile);

    const int tix = tile0 + (int)blockIdx.x;  // launches may cover a range of the tiles
    const int2 tl = tiles[tix];  // (replica, first atom); tiles never straddle replicas
    const int64_t a0 = tl.y;
    const int na = (int)min((int64_t)tile_atoms, reps[tl.x].atom0 + reps[tl.x].n_own - a0);
    const int4 *modes = modes_all + (int64_t)tl.x * Pm;
    const int64_t l0 = (int64_t)blockIdx.y * mode_tile;
    const int nl = (int)min((int64_t)mode_tile, Pm - l0);

    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        s_at[k] = u4[a0 + k];
        if constexpr (sizeof(real) == 8) s_q[k] = q64[a0 + k];
    }
    for (int k = threadIdx.x; k < nl; k += blockDim.x) s_m[k] = modes[l0 + k];
    __syncthreads();

    const int per = (na + sub - 1) / sub;
    for (int it = threadIdx.x; it < nl * sub; it += blockDim.x) {
        const int l = it % nl;
        const int s = it / nl;
        const int b = s * per;
        const int e = min(na, b + per);
        const int4 m = s_m[l];
        const uint32_t mx = (uint32_t)m.x, my = (uint32_t)m.y, mz = (uint32_t)m.z;
        double2 out;
        if constexpr (sizeof(real) == 4) {
            float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
            int a = b;
            // four atoms per compensated addition: their plain FP32 sum, then Kahan
            for (; a + 3 < e; a += 4) {
                float pc, ps;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 A0 = s_at[a + 2 * h], A1 = s_at[a + 2 * h + 1];
                    float s0, c0, s1, c1;
                    phase_sincos(mx * A0.x + my * A0.y + mz * A0.z, s0, c0);
                    phase_sincos(mx * A1.x + my * A1.y + mz * A1.z, s1, c1);
                    const float q0 = __uint_as_float(A0.w), q1 = __uint_as_float(A1.w);
                    const float tc = q0 * c0 + q1 * c1, ts = q0 * s0 + q1 * s1;
                    pc = h ? pc + tc : tc;
                    ps = h ? ps + ts : ts;
                }
                kahan_add(sr, cr, pc);
                kahan_add(si, ci, ps);
            }
            for (; a + 1 < e; a += 2) {
                const uint4 A0 = s_at[a], A1 = s_at[a + 1];
                float s0, c0, s1, c1;
                phase_sincos(mx * A0.x + my * A0.y + mz * A0.z, s0, c0);
                phase_sincos(mx * A1.x + my * A1.y + mz * A1.z, s1, c1);
                const float q0 = __uint_as_float(A0.w), q1 = __uint_as_float(A1.w);
                kahan_add(sr, cr, q0 * c0 + q1 * c1);
                kahan_add(si, ci, q0 * s0 + q1 * s1);
            }
            for (; a < e; ++a) {
                const uint4 A = s_at[a];
                const uint32_t ph = mx * A.x + my * A.y + mz * A.z;
                float sn, cs;
                phase_sincos(ph, sn, cs);
                const float q = __uint_as_float(A.w);
                kahan_add(sr, cr, q * cs);
                kahan_add(si, ci, q * sn);
            }
            out = make_double2((double)sr - (double)cr, (double)si - (double)ci);
        } else {
            double sr = 0.0, si = 0.0;
            for (int a = b; a < e; ++a) {
                const uint4 A = s_at[a];
                const uint32_t ph = mx * A.x + my * A.y + mz * A.z;
                double sn, cs;
                phase_sincos_tab(ptab, ph, sn, cs);
                sr += s_q[a] * cs;
                si += s_q[a] * sn;
            }
            out = make_double2(sr, si);
        }
        s_acc[s * mode_tile + l] = out;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int s = 0; s < sub; ++s) {
            re += s_acc[s * mode_tile + l].x;
            im += s_acc[s * mode_tile + l].y;
        }
        part[(l0 + l) * (int64_t)ntiles_all + tix] = make_double2(re, im);
    }
}

// Exact, order-independent sums of the tile partials: every FP64 partial is
// turned into a 128-bit fixed-point integer in units of 2^-64 (bits below are
// dropped, deterministically), and integers add associatively, so a mode's sum
// is the same for any grouping of its tiles: one context summing all of them, or
// the slab contexts of a spatial decomposition adding their partial sums.
__device__ __forceinline__ __int128 fx_from_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) return 0;  // zero (or below 2^-1022)
    const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int sh = ex - 1075 + 64;  // |x| 2^64 = mant 2^sh (|x| < 2^62 keeps it below 2^127)
    if (sh <= -53) return 0;
    __int128 v = (__int128)mant;
    v = sh >= 0 ? (v << sh) : (v >> (-sh));
    return (b >> 63) ? -v : v;
}

__device__ __forceinline__ double fx_to_double(__int128 v)
{
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return (double)hi + (double)lo * 5.421010862427522170e-20;  // 2^-64
}

__device__ __forceinline__ __int128 shfl_xor_128(__int128 v, int o)
{
    const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(v >> 64), o);
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    return ((__int128)hi << 64) | (__int128)lo;
}

// Force and energy coefficients of mode l (replica rp, local index lm) from its
// structure factor:
//   c_l = -(4 pi coulomb_k / V) W_l / k_l^2,  A_l = c_l Im rho_l,  B_l = c_l Re rho_l,
//   e_l = coulomb_k (2 pi / V) W_l |rho_l|^2 / k_l^2   (energy estimate term).
template <typename real>
__device__ __forceinline__ void mode_coef(const Rep &rp, int64_t l, int64_t lm, int4 m,
                                          const double *__restrict__ W, double ck, double re,
                                          double im, double2 *__restrict__ rho,
                                          double *__restrict__ emode, ModeCoef<real> *__restrict__ coef)
{
    const double L = rp.L;
    const double V = L * L * L;
    const double tk = 2.0 * kPi / L;
    const double kx = tk * m.x, ky = tk * m.y, kz = tk * m.z;
    const double k2 = kx * kx + ky * ky + kz * kz;
    const double w = W ? W[lm] : rp.Wrbe;
    double cl = 0.0, e = 0.0;
    if (k2 > 0.0) {
        cl = -(4.0 * kPi * ck / V) * w / k2;
        e = ck * (2.0 * kPi / V) * w * (re * re + im * im) / k2;
    }
    rho[l] = make_double2(re, im);
    emode[l] = e;
    ModeCoef<real> mc;
    mc.mx = m.x;
    mc.my = m.y;
    mc.mz = m.z;
    if constexpr (sizeof(real) == 8) mc.pad = 0;
    mc.A = (real)(cl * im);
    mc.B = (real)(cl * re);
    mc.kx = (real)m.x;
    mc.ky = (real)m.y;
    mc.kz = (real)m.z;
    if constexpr (sizeof(real) == 8) mc.pad2 = mc.pad3 = mc.pad4 = (real)0;
    coef[l] = mc;
}

// Second stage: one block of 128 threads (32 when every replica has at most 128
// tiles) per (replica, mode) sums the atom-tile partials exactly (fixed point,
// above), stores the sums (acc, [R][Pm][2] re, im) and derives rho and the
// coefficients (mode_coef).
template <typename real>
__global__ void k_rho_final(const double2 *__restrict__ part, int ntiles, const Rep *__restrict__ reps, int R,
                            int64_t Pm, const int4 *__restrict__ modes,
                            const double *__restrict__ W, double ck, double2 *__restrict__ rho,
                            double *__restrict__ emode, ModeCoef<real> *__restrict__ coef,
                            __int128 *__restrict__ acc)
{
    __shared__ __int128 s_p[4][2];
    const int64_t t = blockIdx.x;  // r Pm + l
    const int lane = threadIdx.x & 31;
    const int r = (int)(t / Pm);
    const int64_t lm = t - (int64_t)r * Pm;
    const Rep rp = reps[r];
    __int128 re = 0, im = 0;
    for (int k = threadIdx.x; k < rp.ntiles; k += blockDim.x) {
        const double2 p = part[lm * (int64_t)ntiles + rp.tile0 + k];
        re += fx_from_double(p.x);
        im += fx_from_double(p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += shfl_xor_128(re, o);
        im += shfl_xor_128(im, o);
    }
    if (blockDim.x > 32) {
        if (lane == 0) {
            s_p[threadIdx.x >> 5][0] = re;
            s_p[threadIdx.x >> 5][1] = im;
        }
        __syncthreads();
        if (threadIdx.x != 0) return;
        re = s_p[0][0] + s_p[1][0] + s_p[2][0] + s_p[3][0];
        im = s_p[0][1] + s_p[1][1] + s_p[2][1] + s_p[3][1];
    } else if (lane != 0) {
        return;
    }
    acc[2 * t] = re;
    acc[2 * t + 1] = im;
    mode_coef<real>(rp, t, lm, modes[t], W, ck, fx_to_double(re), fx_to_double(im), rho, emode, coef);
}

// rho and the coefficients of every mode from given exact sums (acc, [R][Pm][2]),
// for a structure factor summed over several contexts.
template <typename real>
__global__ void k_rho_from_acc(const __int128 *__restrict__ acc, const Rep *__restrict__ reps,
                               int64_t RPm, int64_t Pm, const int4 *__restrict__ modes,
                               const double *__restrict__ W, double ck, double2 *__restrict__ rho,
                               double *__restrict__ emode, ModeCoef<real> *__restrict__ coef)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= RPm) return;
    const int r = (int)(t / Pm);
    mode_coef<real>(reps[r], t, t - (int64_t)r * Pm, modes[t], W, ck, fx_to_double(acc[2 * t]),
                    fx_to_double(acc[2 * t + 1]), rho, emode, coef);
}

// Dynamic shared memory of k_rho_partial for a tile shape.
static size_t rho_smem(bool fp64, int tile, int mode_tile, int sub)
{
    return (size_t)tile * sizeof(uint4) + (fp64 ? (size_t)tile * sizeof(double) : 0) +
           (size_t)mode_tile * sizeof(int4) + (size_t)mode_tile * sub * sizeof(double2);
}

rbmd_status rbe_configure(rbmd_ctx *c)
{
    if (c->fp64 && !c->phtab) {
        RBMD_CHECK_CUDA(cudaMalloc(&c->phtab, sizeof(double2) * PHASE_TAB));
        k_phase_table<<<(PHASE_TAB + 255) / 256, 256, 0, c->stream>>>(c->phtab);
        RBMD_LAUNCH_CHECK();
    }
    // the largest tile shape (2048 atoms, 256 modes x 4 sub-tiles) needs 68 KB in FP64
    const int bytes = (int)rho_smem(true, 2048, 256, 4);
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rho_partial<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    RBMD_CHECK_CUDA(cudaFuncSetAttribute(k_rho_partial<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return RBMD_OK;
}

// Partial sums of the tiles [t0, t1) (Eq. 9 per tile and mode).
rbmd_status rbe_rho_partial(rbmd_ctx *c, int t0, int t1)
{
    c->rho_cached = false;
    if (t1 <= t0) return RBMD_OK;
    const int tile = c->rho_tile;
    const int mode_tile = (int)(c->Pm < c->rho_mode_tile ? c->Pm : c->rho_mode_tile);
    int sub = max(1, 1024 / mode_tile);
    sub = min(sub, tile);
    int threads = ((mode_tile * sub + 31) / 32) * 32;
    threads = min(threads, 1024);
    dim3 grid((unsigned)(t1 - t0), (unsigned)((c->Pm + mode_tile - 1) / mode_tile));
    const size_t smem = rho_smem(c->fp64, tile, mode_tile, sub);
    if (c->fp64)
        k_rho_partial<double><<<grid, threads, smem, c->stream>>>(
            c->u4, c->q64, c->tiles, c->reps, c->modes, c->Pm, tile, mode_tile, sub, c->rho_part, t0,
            c->ntiles, c->phtab);
    else
        k_rho_partial<float><<<grid, threads, smem, c->stream>>>(
            c->u4, nullptr, c->tiles, c->reps, c->modes, c->Pm, tile, mode_tile, sub, c->rho_part, t0,
            c->ntiles, nullptr);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// rho of every mode from the tile partials, then the force-pass coefficients.
rbmd_status rbe_rho_final(rbmd_ctx *c)
{
    c->rho_cached = false;
    const unsigned fin_blocks = (unsigned)(c->R * c->Pm);
    int max_tiles = 0;
    for (int r = 0; r < c->R; ++r) max_tiles = std::max(max_tiles, (int)c->reps_h[r].ntiles);
    const int fin_threads = max_tiles > 128 ? 128 : 32;
    if (c->fp64)
        k_rho_final<double><<<fin_blocks, fin_threads, 0, c->stream>>>(
            c->rho_part, c->ntiles, c->reps, c->R, c->Pm, c->modes, c->W, c->prm.coulomb_k, c->rho, c->emode,
            (ModeCoef<double> *)c->coef, c->rho_acc);
    else
        k_rho_final<float><<<fin_blocks, fin_threads, 0, c->stream>>>(
            c->rho_part, c->ntiles, c->reps, c->R, c->Pm, c->modes, c->W, c->prm.coulomb_k, c->rho, c->emode,
            (ModeCoef<float> *)c->coef, c->rho_acc);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

// rho and the coefficients from given exact sums (device [R][Pm][2] __int128).
rbmd_status rbe_rho_from_acc(rbmd_ctx *c, const void *acc)
{
    c->rho_cached = false;
    const int64_t RPm = (int64_t)c->R * c->Pm;
    const unsigned nb = (unsigned)((RPm + 127) / 128);
    if (c->fp64)
        k_rho_from_acc<double><<<nb, 128, 0, c->stream>>>(
            (const __int128 *)acc, c->reps, RPm, c->Pm, c->modes, c->W, c->prm.coulomb_k, c->rho,
            c->emode, (ModeCoef<double> *)c->coef);
    else
        k_rho_from_acc<float><<<nb, 128, 0, c->stream>>>(
            (const __int128 *)acc, c->reps, RPm, c->Pm, c->modes, c->W, c->prm.coulomb_k, c->rho,
            c->emode, (ModeCoef<float> *)c->coef);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

rbmd_status rbe_structure_factors(rbmd_ctx *c, int mark_between)
{
    RBMD_CHECK(rbe_rho_partial(c, 0, c->ntiles));
    if (mark_between >= 0) prof_mark(c, mark_between);
    return rbe_rho_final(c);
}

// --------------------------------------------------------------------------
// Force pass, Eq. 12 (Algorithm 1 step 4).  One thread per atom; the mode
// coefficients stream through shared memory in chunks (every lane reads the same
// mode: a broadcast).  The phase is recomputed exactly from the integers rather
// than stored per atom-mode (N P complex numbers would cost more HBM traffic
// than the recomputation).
// --------------------------------------------------------------------------
// With KICK (the integrator's step) the epilogue also performs the second half
// kick of the atom with its final force and writes the block's kinetic-energy
// partial, saving a pass over the forces and velocities.
template <typename real, int CHUNK, bool KICK>
__global__ void k_rbe_force(const uint4 *__restrict__ u4, const double *__restrict__ q64,
                            const int2 *__restrict__ map, const Rep *__restrict__ reps,
                            const ModeCoef<real> *__restrict__ coef_all, int64_t Pm,
                            real *__restrict__ F, int accumulate, KickArgs<real> kick,
                            const double2 *__restrict__ ptab)
{
    __shared__ ModeCoef<real> s_c[CHUNK];
    const AtomSlot sl = atom_slot(map, reps);  // the whole block belongs to replica sl.r
    const int64_t i = sl.i;
    const bool active = sl.ok;
    const ModeCoef<real> *coef = coef_all + (int64_t)sl.r * Pm;
    const real tk = (real)(2.0 * kPi / reps[sl.r].L);
    uint4 A = active ? u4[i] : make_uint4(0, 0, 0, 0);
    real fx = 0, fy = 0, fz = 0;
    for (int64_t c0 = 0; c0 < Pm; c0 += CHUNK) {
        const int nc = (int)min((int64_t)CHUNK, Pm - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < nc; k += blockDim.x) s_c[k] = coef[c0 + k];
        __syncthreads();
        if (active) {
            for (int k = 0; k < nc; ++k) {
                const ModeCoef<real> mc = s_c[k];
                const uint32_t ph = (uint32_t)mc.mx * A.x + (uint32_t)mc.my * A.y +
                                    (uint32_t)mc.mz * A.z;
                real sn, cs;
                if constexpr (sizeof(real) == 8) phase_sincos_tab(ptab, ph, sn, cs);
                else phase_sincos(ph, sn, cs);  // (the FP32 path runs k_rbe_force_at)
                const real g = fma_r(mc.A, cs, -mul_r(mc.B, sn));
                fx = fma_r(g, mc.kx, fx);
                fy = fma_r(g, mc.ky, fy);
                fz = fma_r(g, mc.kz, fz);
            }
        }
    }
    double ke = 0.0;
    if (active) {
        real q;
        if constexpr (sizeof(real) == 4) q = __uint_as_float(A.w);
        else q = q64[i];
        const real s = mul_r(q, tk);
        real *f = F + 3 * i;
        real fo[3] = {mul_r(s, fx), mul_r(s, fy), mul_r(s, fz)};
        if (accumulate) {
            fo[0] = add_r(fo[0], f[0]);
            fo[1] = add_r(fo[1], f[1]);
            fo[2] = add_r(fo[2], f[2]);
        }
        f[0] = fo[0];
        f[1] = fo[1];
        f[2] = fo[2];
        if constexpr (KICK) {
            real fc[3];
            kick_fcorr(kick, sl.r, fc);
            ke = second_kick(kick, reps[sl.r], sl.r, i, kick.v, F, fo, fc);
        }
    }
    if constexpr (KICK) block_ke_partial(ke, kick.kepart);
}

// FP32 force pass with AT atoms per thread (atoms j, j + 256/AT, ... of the
// 256-atom block): each staged mode coefficient is read once for all of them,
// dividing the shared-memory traffic per atom-mode by AT; otherwise as k_rbe_force.
constexpr int FORCE_AT = 2;  // measured: 2 beats 1 (mode-table reads) and 4 (registers)

template <int CHUNK, bool KICK, int AT>
__global__ void __launch_bounds__(256 / AT) k_rbe_force_at(const uint4 *__restrict__ u4,
                                                           const int2 *__restrict__ map,
                                                           const Rep *__restrict__ reps,
                                                           const ModeCoef<float> *__restrict__ coef_all,
                                                           int64_t Pm, float *__restrict__ F,
                                                           int accumulate, KickArgs<float> kick)
{
    constexpr int TB = 256 / AT;  // threads per block
    __shared__ ModeCoef<float> s_c[CHUNK];
    const int2 mb = map[blockIdx.x];
    const int r = mb.x;
    const Rep rp = reps[r];
    const int64_t end = rp.atom0 + rp.N;
    const ModeCoef<float> *coef = coef_all + (int64_t)r * Pm;
    const float tk = (float)(2.0 * kPi / rp.L);
    uint4 A[AT];
    float f3[AT][3];
#pragma unroll
    for (int h = 0; h < AT; ++h) {
        const int64_t i = (int64_t)mb.y + threadIdx.x + h * TB;
        A[h] = i < end ? u4[i] : make_uint4(0, 0, 0, 0);
        f3[h][0] = f3[h][1] = f3[h][2] = 0.f;
    }
    const bool any = (int64_t)mb.y + threadIdx.x < end;
    for (int64_t c0 = 0; c0 < Pm; c0 += CHUNK) {
        const int nc = (int)min((int64_t)CHUNK, Pm - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < nc; k += blockDim.x) s_c[k] = coef[c0 + k];
        __syncthreads();
        if (any) {
            for (int k = 0; k < nc; ++k) {
                const ModeCoef<float> mc = s_c[k];
#pragma unroll
                for (int h = 0; h < AT; ++h) {
                    float sn, cs;
                    phase_sincos((uint32_t)mc.mx * A[h].x + (uint32_t)mc.my * A[h].y +
                                     (uint32_t)mc.mz * A[h].z,
                                 sn, cs);
                    const float g = fma_r(mc.A, cs, -mul_r(mc.B, sn));
                    f3[h][0] = fma_r(g, mc.kx, f3[h][0]);
                    f3[h][1] = fma_r(g, mc.ky, f3[h][1]);
                    f3[h][2] = fma_r(g, mc.kz, f3[h][2]);
                }
            }
        }
    }
    double ke = 0.0;
    float fc[3] = {0.f, 0.f, 0.f};
    if constexpr (KICK) kick_fcorr(kick, r, fc);  // once for the thread's atoms
#pragma unroll
    for (int h = 0; h < AT; ++h) {
        const int64_t i = (int64_t)mb.y + threadIdx.x + h * TB;
        if (i >= end) continue;
        const float sc = mul_r(__uint_as_float(A[h].w), tk);
        float *f = F + 3 * i;
        float fo[3] = {mul_r(sc, f3[h][0]), mul_r(sc, f3[h][1]), mul_r(sc, f3[h][2])};
        if (accumulate) {
            fo[0] = add_r(fo[0], f[0]);
            fo[1] = add_r(fo[1], f[1]);
            fo[2] = add_r(fo[2], f[2]);
        }
        f[0] = fo[0];
        f[1] = fo[1];
        f[2] = fo[2];
        if constexpr (KICK) ke += second_kick(kick, rp, r, i, kick.v, F, fo, fc);
    }
    if constexpr (KICK) block_ke_partial(ke, kick.kepart);
}

rbmd_status rbe_apply_forces(rbmd_ctx *c, void *force, int accumulate, const StepRef *kick,
                             int b0, int b1)
{
    // the atoms of the 256-atom blocks [b0, b1) of map256 (all of them when b1 < 0);
    // the integrator's kick (kinetic-energy partials per block) covers all blocks
    if (b1 < 0) b1 = c->nb256;
    if (kick && (b0 != 0 || b1 != c->nb256)) return RBMD_ERR_INVALID;
    if (b1 <= b0) return RBMD_OK;
    const unsigned nb = (unsigned)(b1 - b0);
    const int2 *map = c->map256 + b0;
    if (c->fp64) {
        KickArgs<double> k{};
        if (kick) k = kick_args<double>(c, *kick);
        if (kick)
            k_rbe_force<double, 128, true><<<nb, 256, 0, c->stream>>>(
                c->u4, c->q64, map, c->reps, (const ModeCoef<double> *)c->coef, c->Pm,
                (double *)force, accumulate, k, c->phtab);
        else
            k_rbe_force<double, 128, false><<<nb, 256, 0, c->stream>>>(
                c->u4, c->q64, map, c->reps, (const ModeCoef<double> *)c->coef, c->Pm,
                (double *)force, accumulate, k, c->phtab);
    } else {
        KickArgs<float> k{};
        if (kick) k = kick_args<float>(c, *kick);
        if (kick)
            k_rbe_force_at<256, true, FORCE_AT><<<nb, 256 / FORCE_AT, 0, c->stream>>>(
                c->u4, map, c->reps, (const ModeCoef<float> *)c->coef, c->Pm,
                (float *)force, accumulate, k);
        else
            k_rbe_force_at<256, false, FORCE_AT><<<nb, 256 / FORCE_AT, 0, c->stream>>>(
                c->u4, map, c->reps, (const ModeCoef<float> *)c->coef, c->Pm,
                (float *)force, accumulate, k);
    }
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}

}  // namespace rbmd
