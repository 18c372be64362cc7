// Allocation-free RBE force entry point (rbmd_rbe_forces_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while another framework
// owns the whole device memory through its own pool, or code on a latency-
// critical path where an allocation would synchronise the device.  For them this
// file computes the random batch Ewald force (the same method as
// rbmd_rbe_forces: device mode sampling, structure factors, force pass) with no
// context and no allocation.  Every intermediate lives in one file-scope device
// array of fixed size, so each GPU that loads the library holds these
// RBMD_NOALLOC_SCRATCH_BYTES until the process exits.
//
// Host code must not hand the array's name to a kernel: on the host it is only a
// stand-in for the symbol.  The device address is looked up once per device with
// cudaGetSymbolAddress (first call on that device, with the device current).
#include <math.h>
#include <string.h>

#include "rbmd_internal.cuh"

namespace {

using namespace rbmd;

constexpr int NA_MAX_P = RBMD_NOALLOC_MAX_P;
constexpr int NA_MAX_TABLE = RBMD_NOALLOC_MAX_TABLE;
constexpr int NA_BLOCKS = 256;  // structure-factor blocks: partial sums per mode
constexpr int NA_TILE = 512;    // atoms staged per structure-factor tile
constexpr int NA_MAX_DEVICES = 64;

// scratch layout (bytes)
constexpr size_t NA_OFF_CDF = 0;
constexpr size_t NA_OFF_MODES = NA_OFF_CDF + sizeof(uint64_t) * NA_MAX_TABLE;
constexpr size_t NA_OFF_COEF = NA_OFF_MODES + sizeof(int4) * NA_MAX_P;
constexpr size_t NA_OFF_PART = NA_OFF_COEF + sizeof(float4) * 2 * NA_MAX_P;
constexpr size_t NA_END = NA_OFF_PART + sizeof(double2) * (size_t)NA_BLOCKS * NA_MAX_P;
static_assert(NA_END <= RBMD_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the static array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[RBMD_NOALLOC_SCRATCH_BYTES];

void *g_scratch_dev[NA_MAX_DEVICES];  // device address of the array, per device

__device__ __forceinline__ int na_draw(uint64_t U, const uint64_t *__restrict__ T, int M)
{
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T[mid] <= U) lo = mid + 1;
        else hi = mid;
    }
    return lo - M;
}

// Mode l of `step`: the same inverse-CDF draw as the context path (Philox words
// (l, t, step, tag) -> m_x, m_y; (l, t | 2^31, step, tag) -> m_z; m = 0 redrawn).
__global__ void na_sample(unsigned char *scr, int M, int P, uint2 key, uint32_t step, uint32_t tag)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    const uint64_t *T = reinterpret_cast<const uint64_t *>(scr + NA_OFF_CDF);
    int mx = 0, my = 0, mz = 0;
    for (uint32_t t = 0; t < RBMD_MAX_ATTEMPTS; ++t) {
        const uint4 w = philox10(make_uint4((uint32_t)l, t, step, tag), key);
        const uint4 w2 = philox10(make_uint4((uint32_t)l, t | 0x80000000u, step, tag), key);
        mx = na_draw(((uint64_t)w.x << 32) | w.y, T, M);
        my = na_draw(((uint64_t)w.z << 32) | w.w, T, M);
        mz = na_draw(((uint64_t)w2.x << 32) | w2.y, T, M);
        if (mx != 0 || my != 0 || mz != 0) break;
    }
    reinterpret_cast<int4 *>(scr + NA_OFF_MODES)[l] = make_int4(mx, my, mz, 0);
}

__device__ __forceinline__ void na_kahan(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Structure factors (Eq. 9): a fixed grid of NA_BLOCKS blocks walks the atom
// tiles; thread t owns modes t and t + 256 and keeps compensated FP32 sums across
// all tiles of its block, then writes one FP64 partial per (block, mode).  Every
// slot of the partial array that is read later is written here, so nothing has
// to be cleared between calls.
__global__ void __launch_bounds__(256) na_rho(unsigned char *scr, const uint32_t *__restrict__ u,
                                              const float *__restrict__ q, int64_t N, int P)
{
    __shared__ uint4 s_at[NA_TILE];
    const int4 *modes = reinterpret_cast<const int4 *>(scr + NA_OFF_MODES);
    int4 m0 = make_int4(0, 0, 0, 0), m1 = make_int4(0, 0, 0, 0);
    const int l0 = threadIdx.x, l1 = threadIdx.x + 256;
    if (l0 < P) m0 = modes[l0];
    if (l1 < P) m1 = modes[l1];
    float r0 = 0.f, c0 = 0.f, i0 = 0.f, d0 = 0.f, r1 = 0.f, c1 = 0.f, i1 = 0.f, d1 = 0.f;
    for (int64_t base = (int64_t)blockIdx.x * NA_TILE; base < N; base += (int64_t)gridDim.x * NA_TILE) {
        const int na = (int)min((int64_t)NA_TILE, N - base);
        __syncthreads();
        for (int k = threadIdx.x; k < na; k += blockDim.x) {
            const int64_t j = base + k;
            s_at[k] = make_uint4(u[3 * j], u[3 * j + 1], u[3 * j + 2], __float_as_uint(q[j]));
        }
        __syncthreads();
        for (int a = 0; a < na; ++a) {
            const uint4 A = s_at[a];
            const float qa = __uint_as_float(A.w);
            if (l0 < P) {
                const uint32_t ph = (uint32_t)m0.x * A.x + (uint32_t)m0.y * A.y + (uint32_t)m0.z * A.z;
                float sn, cs;
                sincospif((float)(int32_t)ph * 4.656612873077392578125e-10f, &sn, &cs);
                na_kahan(r0, c0, qa * cs);
                na_kahan(i0, d0, qa * sn);
            }
            if (l1 < P) {
                const uint32_t ph = (uint32_t)m1.x * A.x + (uint32_t)m1.y * A.y + (uint32_t)m1.z * A.z;
                float sn, cs;
                sincospif((float)(int32_t)ph * 4.656612873077392578125e-10f, &sn, &cs);
                na_kahan(r1, c1, qa * cs);
                na_kahan(i1, d1, qa * sn);
            }
        }
    }
    double2 *part = reinterpret_cast<double2 *>(scr + NA_OFF_PART) + (int64_t)blockIdx.x * NA_MAX_P;
    if (l0 < P) part[l0] = make_double2((double)r0 - (double)c0, (double)i0 - (double)d0);
    if (l1 < P) part[l1] = make_double2((double)r1 - (double)c1, (double)i1 - (double)d1);
}

// One warp per mode: fixed-order FP64 sum of the block partials and the force
// coefficients c_l = -(4 pi coulomb_k / V)(S/P)/k^2, A = c Im rho, B = c Re rho.
__global__ void na_final(unsigned char *scr, int P, double Wl, double L, double ck)
{
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= P) return;
    const double2 *part = reinterpret_cast<const double2 *>(scr + NA_OFF_PART);
    double re = 0.0, im = 0.0;
    for (int b = lane; b < NA_BLOCKS; b += 32) {
        const double2 v = part[(int64_t)b * NA_MAX_P + l];
        re += v.x;
        im += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane != 0) return;
    const int4 m = reinterpret_cast<const int4 *>(scr + NA_OFF_MODES)[l];
    const double tk = 2.0 * kPi / L;
    const double kx = tk * m.x, ky = tk * m.y, kz = tk * m.z;
    const double k2 = kx * kx + ky * ky + kz * kz;
    const double cl = k2 > 0.0 ? -(4.0 * kPi * ck / (L * L * L)) * Wl / k2 : 0.0;
    float4 *coef = reinterpret_cast<float4 *>(scr + NA_OFF_COEF);
    coef[2 * l] = make_float4((float)(cl * im), (float)(cl * re), (float)m.x, (float)m.y);
    coef[2 * l + 1] = make_float4((float)m.z, __int_as_float(m.x), __int_as_float(m.y),
                                  __int_as_float(m.z));
}

// Force pass (Eq. 12): thread per atom, coefficients staged in shared memory.
__global__ void __launch_bounds__(256) na_force(const unsigned char *scr, const uint32_t *__restrict__ u,
                                                const float *__restrict__ q, int64_t N, int P,
                                                float tk, float *__restrict__ F)
{
    __shared__ float4 s_c[2 * NA_MAX_P];
    const float4 *coef = reinterpret_cast<const float4 *>(scr + NA_OFF_COEF);
    for (int k = threadIdx.x; k < 2 * P; k += blockDim.x) s_c[k] = coef[k];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t ux = u[3 * i], uy = u[3 * i + 1], uz = u[3 * i + 2];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int l = 0; l < P; ++l) {
        const float4 c0 = s_c[2 * l], c1 = s_c[2 * l + 1];
        const uint32_t ph = (uint32_t)__float_as_int(c1.y) * ux +
                            (uint32_t)__float_as_int(c1.z) * uy +
                            (uint32_t)__float_as_int(c1.w) * uz;
        float sn, cs;
        sincospif((float)(int32_t)ph * 4.656612873077392578125e-10f, &sn, &cs);
        const float g = c0.x * cs - c0.y * sn;
        fx += g * c0.z;
        fy += g * c0.w;
        fz += g * c1.x;
    }
    const float s = q[i] * tk;
    F[3 * i] = s * fx;
    F[3 * i + 1] = s * fy;
    F[3 * i + 2] = s * fz;
}

// Inverse-CDF thresholds (same definition as rbmd_sampler_table), computed into
// caller-provided fixed storage: no heap allocation.
bool na_table(double L, double alpha, int *Mout, uint64_t *T, double *H)
{
    const double a = kPi * kPi / (alpha * L * L);
    const double hw = ceil(sqrt(16.0 * log(10.0) / a));
    if (!(hw >= 0.0) || 2.0 * hw + 1.0 > (double)NA_MAX_TABLE) return false;
    const int M = (int)hw;
    double cum[NA_MAX_TABLE];
    double total = 0.0;
    for (int j = 0; j < 2 * M + 1; ++j) {
        const double m = (double)(j - M);
        total += exp(-a * m * m);
        cum[j] = total;
    }
    for (int j = 0; j < 2 * M + 1; ++j) {
        const double x = (cum[j] / total) * kTwo64;
        T[j] = (x >= kTwo64) ? UINT64_MAX : (uint64_t)x;
    }
    *Mout = M;
    *H = total;
    return true;
}

}  // namespace

extern "C" rbmd_status rbmd_rbe_forces_noalloc(const uint32_t *u, const float *charge,
                                               int64_t n_atoms, double box_length, double alpha,
                                               double coulomb_k, int32_t P, uint64_t seed,
                                               int64_t step, uint32_t replica, float *force,
                                               void *stream)
{
    if (!u || !charge || !force || n_atoms < 1 || n_atoms > (int64_t)INT32_MAX) return RBMD_ERR_INVALID;
    if (!(box_length > 0.0) || !(alpha > 0.0)) return RBMD_ERR_INVALID;
    if (P < 1 || P > NA_MAX_P) return RBMD_ERR_INVALID;
    static uint64_t T[NA_MAX_TABLE];  // host staging of the thresholds (not thread-safe)
    int M = 0;
    double H = 0.0;
    if (!na_table(box_length, alpha, &M, T, &H)) return RBMD_ERR_INVALID;

    int dev = 0;
    RBMD_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return RBMD_ERR_UNSUPPORTED;
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return RBMD_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    unsigned char *scr = static_cast<unsigned char *>(g_scratch_dev[dev]);
    cudaStream_t st = (cudaStream_t)stream;

    RBMD_CHECK_CUDA(cudaMemcpyAsync(scr + NA_OFF_CDF, T, sizeof(uint64_t) * (2 * M + 1),
                                    cudaMemcpyHostToDevice, st));
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    na_sample<<<(P + 127) / 128, 128, 0, st>>>(scr, M, P, key, (uint32_t)step,
                                                RBMD_STREAM_RBE | (replica << 8));
    na_rho<<<NA_BLOCKS, 256, 0, st>>>(scr, u, charge, n_atoms, P);
    const double S = H * H * H - 1.0;
    na_final<<<(P * 32 + 255) / 256, 256, 0, st>>>(scr, P, S / (double)P, box_length, coulomb_k);
    na_force<<<(unsigned)((n_atoms + 255) / 256), 256, 0, st>>>(
        scr, u, charge, n_atoms, P, (float)(2.0 * kPi / box_length), force);
    RBMD_LAUNCH_CHECK();
    return RBMD_OK;
}
