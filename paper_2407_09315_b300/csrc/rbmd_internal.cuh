// Internal declarations of the B300 random-batch MD library.
//
// Data layout in HBM (atom id = the caller's row index):
//   u4     uint4[N]   fixed-point fractional coordinates (x, y, z) in units of
//                     L/2^32, and the FP32 charge bits in .w (id order, master)
//   q64    double[N]  charges (FP64 contexts)
//   type   int32[N]   LJ type
//   vel    real[N][3] velocities (stored before the pending Berendsen factor)
//   force  real[N][3] forces of the current configuration (without F_corr)
//   spos   uint4[N]   cell-sorted copy {ux, uy, uz, id}, rebuilt every evaluation
//   sq     real[N]    cell-sorted charges;  stype int32[N] cell-sorted types
//   cell_start int32[ncell+1]  CSR offsets of the cells (x-major, z fastest)
//
// All floating-point reductions whose results leave a kernel run in FP64 and in a
// fixed order, so two runs of the same state are bit-identical.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "../../include/rbmd.h"

#define RBMD_STREAM_RBE 1u
#define RBMD_STREAM_RBL 2u
#define RBMD_STREAM_LANGEVIN 3u
#define RBMD_STREAM_METROPOLIS 4u
#define RBMD_MAX_ATTEMPTS 256
#define RBMD_MAX_TYPES 64
#define RBMD_MAX_P 128

namespace rbmd {

constexpr double kTwo32 = 4294967296.0;
constexpr double kTwo64 = 18446744073709551616.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kPairBlock = 128;  // threads per block of the RBL pair kernel
constexpr int RED_BLOCKS = 256;  // first-stage blocks of the long FP64 reductions
constexpr int RED_SPLIT = 32;    // first-stage chunks per replica of the per-replica sums
constexpr int RED_STRIDE = 16;   // components per first-stage chunk slot (at most 16)

// Step number used by a kernel: (*ptr) + add when ptr is set (graph replays read
// the device counter), else add.
struct StepRef {
    const int64_t *ptr;
    int64_t add;
};

__device__ __forceinline__ int64_t step_of(StepRef s) { return (s.ptr ? *s.ptr : 0) + s.add; }

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// 10 rounds of two 32x32->64 multiplies with Weyl-sequence key increments.
__host__ __device__ __forceinline__ void philox_mulhilo(uint32_t a, uint32_t b, uint32_t &hi,
                                                        uint32_t &lo)
{
#ifdef __CUDA_ARCH__
    hi = __umulhi(a, b);
    lo = a * b;
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        uint32_t h0, l0, h1, l1;
        philox_mulhilo(0xD2511F53u, c.x, h0, l0);
        philox_mulhilo(0xCD9E8D57u, c.z, h1, l1);
        c = make_uint4(h1 ^ c.y ^ k.x, l1, h0 ^ c.w ^ k.y, l0);
    }
    return c;
}

// Device error word: first error wins.
__device__ __forceinline__ void latch_error(int *err, int code) { atomicCAS(err, 0, code); }

// Index i of an array of n elements.  Built with -DRBMD_CHECKED, an index outside
// [0, n) latches RBMD_ERR_BOUNDS and reads element 0 instead (a debugging build in
// place of a memory checker: nothing faults, the error is reported by the next
// synchronising call); otherwise the index itself.
__device__ __forceinline__ int64_t checked_index(int64_t i, int64_t n, int *err)
{
    if (i < 0 || i >= n) {
        if (err) latch_error(err, RBMD_ERR_BOUNDS);
        return 0;
    }
    return i;
}
#ifdef RBMD_CHECKED
#define RBMD_IDX(i, n, err) rbmd::checked_index((int64_t)(i), (int64_t)(n), (err))
#else
#define RBMD_IDX(i, n, err) (i)
#endif

// sin and cos of the wrapped phase 2 pi ph / 2^32.  ph is read as a signed
// fraction of a turn, so the angle lies in [-pi, pi): there the hardware SFU
// sin/cos (__sincosf) needs no range reduction and its documented absolute error
// is at most 2^-21.41.  The FP64 kernels use phase_sincos_tab below.
__device__ __forceinline__ void phase_sincos(uint32_t ph, float &s, float &c)
{
    __sincosf((float)(int32_t)ph * 1.4629180792671596e-09f, &s, &c);  // 2 pi / 2^32
}

// FP64 phase factors by angle addition from the table of k_phase_table (rbe.cu):
// with ph = h 2^16 + l, e^{i theta} = T[h] T'[l], T at [0, 65536), T' at
// [65536, 131072), entries {cos, sin}.
__device__ __forceinline__ void phase_sincos_tab(const double2 *__restrict__ tab, uint32_t ph,
                                                 double &s, double &c)
{
    const double2 a = __ldg(tab + (ph >> 16));
    const double2 d = __ldg(tab + 65536 + (ph & 65535u));
    c = __fma_rn(a.x, d.x, -__dmul_rn(a.y, d.y));
    s = __fma_rn(a.x, d.y, __dmul_rn(a.y, d.x));
}

// x 2^32 truncated toward zero, from the bits of x (|x| < 2^31): the force sums of
// the momentum correction are added as these integers, exactly, so they do not
// depend on how the atoms are grouped (warps, blocks, the sorted order of a
// candidate rebuild).
__device__ __forceinline__ long long fix32(float x)
{
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 0xFFu);
    if (ex == 0) return 0;
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = min(ex - 118, 39);  // x = m 2^(ex - 150)
    const long long v = sh >= 0 ? (m << sh) : (sh > -24 ? (m >> -sh) : 0);
    return (b >> 31) ? -v : v;
}

__device__ __forceinline__ long long fix32(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FFu);
    if (ex == 0) return 0;
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int sh = min(ex - 1043, 10);  // x = m 2^(ex - 1075)
    const long long v = sh >= 0 ? (m << sh) : (sh > -53 ? (m >> -sh) : 0);
    return (b >> 63) ? -v : v;
}

// Ascending sort of n <= 16 values (the rest of r padded with INT_MAX) by a
// bitonic network in registers: no dependent memory accesses.
__device__ __forceinline__ void sort16(int32_t (&r)[16])
{
#pragma unroll
    for (int k = 2; k <= 16; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t lo = min(r[i], r[l]), hi = max(r[i], r[l]);
                    const bool up = (i & k) == 0;
                    r[i] = up ? lo : hi;
                    r[l] = up ? hi : lo;
                }
            }
}

// A named host range for profilers (nothing happens without one attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Per-replica constants, on the device (array of R) and on the host.  A context
// holds R >= 1 independent replicas concatenated: atoms [atom0, atom0 + N),
// cells [cell0, cell0 + ncell), modes [r P, (r + 1) P), FP64 scalars
// [r SCAL_COUNT, (r + 1) SCAL_COUNT).
struct Rep {
    double L, lscale, dtc, Wrbe, S, T0, e_self;
    uint64_t Rc2, Rs2;
    uint2 key;              // Philox key (seed)
    uint32_t Rlin;          // floor(sqrt(Rs2)): per-axis early reject
    uint32_t Rv;            // candidate radius of the step's lists: Rlin + 1 + 2 h (= Rlin without them)
    uint64_t Rv2, H2;       // Rv^2; h^2 with h = floor(skin/2 in fixed-point units)
    uint32_t tag_rbe, tag_rbl;
    int32_t nc, M;          // cells per axis, sampler half-width
    float cull_r;           // r_cut in cell widths (+ margin): cells sorted for these positions
    float cull_v;           // r_cut + skin in cell widths (+ margin): cells of the last rebuild
    float dtc_hi, dtc_lo;   // dtc as a sum of two floats (FP32 drift)
    int64_t atom0, N;
    int64_t n_own;          // atoms [atom0, atom0 + n_own) own forces and structure-factor
                            // terms; the rest (a slab context's halo) are neighbours only
    int64_t cell0, ncell;
    int64_t cdf0;           // offset of the replica's sampler thresholds
    int32_t b256_0, nb256;  // blocks of the 256-thread atom kernels
    int32_t b128_0, nb128;  // blocks of the 128-thread atom kernels
    int32_t tile0, ntiles;  // structure-factor atom tiles
};

// Atom handled by this thread in a replica-aligned launch: map[blockIdx.x] =
// (replica, first atom of the block); blocks never straddle two replicas.
struct AtomSlot {
    int r;
    int64_t i;
    bool ok;
};

// Position of entry e of sorted atom i in a per-atom list of capacity cap.  Row
// major: a thread's appends stay in its own row, which measured faster than the
// column-major layout (coalesced reads, but scattered partial-line writes).
__device__ __forceinline__ int64_t lidx(int64_t i, int e, int64_t /*N*/, int cap)
{
    return i * cap + e;
}

// Cell index along one axis of a fixed-point coordinate for nc cells per axis.
__device__ __forceinline__ int cell_coord(uint32_t u, int nc)
{
    return (int)(((uint64_t)u * (uint64_t)nc) >> 32);
}

__device__ __forceinline__ AtomSlot atom_slot_at(const int2 *__restrict__ map,
                                                 const Rep *__restrict__ reps, int b)
{
    const int2 m = map[b];
    AtomSlot s;
    s.r = m.x;
    s.i = (int64_t)m.y + threadIdx.x;
    s.ok = s.i < reps[m.x].atom0 + reps[m.x].N;
    return s;
}

__device__ __forceinline__ AtomSlot atom_slot(const int2 *__restrict__ map,
                                              const Rep *__restrict__ reps)
{
    return atom_slot_at(map, reps, blockIdx.x);
}

// Per-mode coefficients for the force pass (Eq. 12 expanded):
//   F_i = q_i sum_l (A_l cos th - B_l sin th) k_l,  A = c rho_im, B = c rho_re,
//   c_l = -(4 pi coulomb_k / V) W_l / k_l^2.
template <typename real> struct ModeCoef {
    int32_t mx, my, mz, pad;
    real A, B, kx, ky, kz, pad2, pad3, pad4;
};
// FP32: 32 bytes, two 16-byte shared-memory loads per mode.
template <> struct __align__(16) ModeCoef<float> {
    int32_t mx, my, mz;
    float A, B, kx, ky, kz;
};

}  // namespace rbmd

struct rbmd_ctx {
    rbmd_params prm;
    int64_t N;
    int32_t T;
    bool fp64;
    cudaStream_t stream;
    bool own_stream;      // created here because the caller passed the legacy stream
    cudaEvent_t ev_in, ev_out;
    // second stream of a force evaluation: the RBE sampling and structure factors
    // run on it beside the RBL kernels (they share no buffer), joined before the
    // RBE force pass; null when the evaluation stays on one stream
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    // rbmd_forces_host: a copy stream and per-chunk events (positions copied in,
    // positions encoded, forces final), 8 chunks at most
    cudaStream_t copy;
    cudaEvent_t ev_h2d[8], ev_enc[8], ev_fin[8];
    // the step graph: the candidate-list rebuild kernels form the body of a
    // conditional node (captured on cond_stream); off with RBMD_GRAPH_COND=0
    cudaStream_t cond_stream = nullptr;
    bool cond_nodes = false;
    int32_t graph_cond_kernels = 0;  // kernels in that body (launched on rebuild steps only)

    // spatial decomposition (rbmd_init_slab): global atom ids of the rows (every
    // random draw is keyed by them) and the global atom count; NULL / N otherwise
    uint32_t *gid;
    int64_t n_glob;

    // replicas
    int32_t R;
    rbmd::Rep *reps_h;    // [R] host copy
    rbmd::Rep *reps;      // [R] device
    int2 *map256;         // [nb256] replica-aligned blocks of 256 atoms
    int2 *map128;         // [nb128] replica-aligned blocks of 128 atoms
    int2 *tiles;          // [ntiles] structure-factor tiles (replica, first atom)
    int nb256, nb128, ntiles;

    // shared constants
    double sqrt_alpha, tau;
    int32_t div;          // cells per r_cut
    int64_t ncell;        // all replicas
    int64_t Pm;           // modes per replica per evaluation (P or the full count)
    int64_t cdf_total;
    bool full_modes;

    // master state
    uint4 *u4;
    double *q64;
    int32_t *type;
    void *vel;
    void *force;          // internal force buffer for the integrator
    void *scratch_force;  // force buffer for energy evaluations
    double *scal;         // [R][SCAL_COUNT] FP64 scalars, see SCAL_* below
    double *red_tmp;      // [RED_BLOCKS][8] first stage of long reductions
    double *red_rep;      // [R][RED_SPLIT][RED_STRIDE] first stage of the per-replica sums
    int *err;
    int64_t *d_step;

    // RBE
    uint64_t *cdf;        // sampler thresholds of every replica (2M_r + 1 each)
    int4 *modes;          // [R][Pm]
    int4 *modes0;         // [R][Pm] Metropolis chains at step 0 (RBMD_METROPOLIS_MODES)
    uint64_t *acc;        // Metropolis acceptance thresholds, same offsets as cdf
    int64_t *chain_step;  // [1] step the chains in `modes` belong to
    int mh_moves;
    double *W;            // [Pm] weights (full-mode list, one replica), else NULL
    double2 *rho_part;    // [Pm][ntiles] mode-major, so a warp sums one mode over consecutive tiles
    double2 *rho;         // [R][Pm]
    __int128 *rho_acc;    // [R][Pm][2] exact sums of the tile partials (units of 2^-64)
    double *emode;        // [R][Pm]
    void *coef;           // ModeCoef<real>[R][Pm]
    void *ptab;           // pair look-up table, real4 [2 ptab_n] (pairtab.cu)
    double2 *phtab;       // FP64 contexts: phase factors {cos, sin} for the RBE kernels (rbe.cu)
    int ptab_n, ptab_i0;
    double ptab_inv_h;
    bool use_table;       // pair kernels read the table instead of erfc/exp
    int rho_tile;         // atoms per structure-factor tile (512, 1024 or 2048)
    int rho_mode_tile;    // modes per structure-factor block (64, 128 or 256)
    int ntiles_max;       // tiles at the smallest tile size (rho_part capacity)
    int64_t ncell_max;    // cells at the finest cell division (cell array capacity)

    // RBL
    int32_t *cell_count;  // [ncell]
    int32_t *cell_start;  // [ncell+1]
    int32_t *cell_of;     // [N]
    int32_t *cell_rank;   // [N] rank inside the cell while binning, then the sorted index
    int32_t *scan_part;   // scan block sums
    uint4 *spos;          // [N]
    void *sq;             // real [N]
    int32_t *stype;       // [N]
    long long *fpart;     // [pair_parts][3] force partial sums (per warp), fixed point 2^-32
    double *epart;        // [pair_parts][EPART] energy and virial partial sums
    double *kepart;       // [nb256]
    int32_t *ibuf;        // [8] integer diagnostics and flags: 0 max N_s, 1 max cell,
                          // 2 list overflow, 3 heavy atoms, 4 rebuild the step's candidates,
                          // 5 rebuilds so far
    float *lj_f;          // [2*T] sqrt(eps), sigma/2 (FP32 path)
    double *lj_d;         // [2*T] (FP64 path)
    int pair_parts;       // per-warp partial sums: pair kernel (4 nb128), then the fallback (4 nb128)
    int32_t *lcore;       // [N][list_cc] core lists (sorted indices)
    int32_t *lshell;      // [N][list_cs] shell lists (replica-local atom ids)
    int2 *ncount;         // [N] (|C|, N_s)
    int32_t *bk;          // [N][p] batch (sorted indices)
    int2 *heavy;          // [N] atoms that need a batch selection (p > 10 only)
    int sel_exact;        // RBMD_SELECT_EXACT: every batch by the exact slow path (tests)
    int sel_key_bits;     // RBMD_SELECT_KEY_BITS: fewer priority bits in the fast keys (tests)
    int list_cc, list_cs; // list capacities per atom
    void *adj_lj;         // real [2T + 4T^2]: eps_t, sigma_t, then the adjoint's type-pair factors
    double *adj_tpart;    // [adjoint blocks][2T]
    double *adj_tsum;     // [2T]

    // neighbour candidates of the integrator's step (Verlet lists with a skin):
    // built from the cells at a rebuild, classified exactly every step
    bool verlet;          // the step uses them (skin > 0, p <= 32, batches not exact)
    // what the list and mode arrays hold, so that rbmd_energy_backward right after
    // rbmd_energy of the same state and step reuses them: set by rbmd_energy,
    // cleared by every call that writes the lists, the modes or structure factors,
    // the positions or the charges
    bool lists_cached = false, rho_cached = false;
    int32_t *adj_rb = nullptr;  // reverse batches of the adjoint, [N][adj_rb_cap] (on first use)
    int adj_rb_cap = 0;
    int64_t lists_step = 0, rho_step = 0;
    bool vl_current = false;  // the sorted positions and candidate lists are those of the state
    bool vl_dirty;        // the sorted layout changed outside the step: rebuild before the next
    double skin;
    int vl_cv;            // candidate capacity per atom
    int vl_ccs;           // core members per thread kept in shared memory
    int32_t *vl_cand;     // [ceil(N/32)][vl_cv][32] sorted indices (entry t of atom i at
                          //  (i/32) cv 32 + 32 t + i%32: a warp's loads of entry t coalesce)
    int32_t *vl_ncand;    // [N] candidate count (> vl_cv: the atom takes the exact fallback)
    uint4 *vl_sref;       // [N] sorted positions at the last rebuild

    // integrator state
    int64_t step;
    bool have_force;
    bool bath_set = false;  // energy bath: SCAL_XI holds E0 (set, or taken at a run's start)
    cudaGraphExec_t graph;
    bool graph_ready;
    int32_t graph_kernels;

    // per-stage timing (rbmd_profile)
    bool profiling;
    bool capturing;       // inside the stream capture of the step graph
    bool prof_eager;      // graph event nodes not timeable: profile without the graph
    cudaEvent_t prof_ev[RBMD_PROFILE_STAGES + 1];
    double prof_ms[RBMD_PROFILE_STAGES];
    int64_t prof_steps;
    // stages of rbmd_energy (forward) and rbmd_energy_backward while profiling
    cudaEvent_t gprof_ev[RBMD_PROFILE_GRAD_STAGES + 1];
    double gprof_fwd[RBMD_PROFILE_FWD_STAGES];
    double gprof_bwd[RBMD_PROFILE_GRAD_STAGES];
    int64_t gprof_calls[2];
};

// FP64 scalar slots in ctx->scal
enum {
    SCAL_FCORR = 0,   // [3] momentum correction F_corr
    SCAL_LAMBDA = 3,  // pending Berendsen factor of the stored velocities
    SCAL_KE = 4,      // kinetic energy after the last kick (before lambda)
    SCAL_FSUM = 5,    // [3] sum of short-range forces before the correction
    SCAL_ERBE = 8,    // RBE energy estimate
    SCAL_KE_TRUE = 11,
    SCAL_FCORR_AUX = 12,  // [3] correction of stand-alone force calls
    SCAL_ESELF = 15,      // self energy (kept on the device for batched read-out)
    SCAL_LAMBDA_KICK = 16,  // factor applied to the stored velocities by the next kick
    SCAL_XI = 17,         // Nose-Hoover variable at the step boundary; the energy bath's E0
    SCAL_XI_RUN = 18,     // Nose-Hoover variable during the step (after its first half update)
    SCAL_EPAIR = 20,      // [EPART] pair-list sums: E_coul, E_lj, tr W_coul, tr W_lj, W[6]
    SCAL_VRBE = 30,       // [6] RBE virial estimate xx yy zz xy xz yz
    SCAL_COUNT = 36
};

// Components of the pair kernels' energy partial sums (per warp, FP64): the
// erfc-Coulomb and LJ energies of the lists, the traces of their virials and the
// virial tensor of both (xx yy zz xy xz yz), each already halved (every ordered
// pair of the lists is visited once from each side).
constexpr int EPART = 10;

namespace rbmd {

// Records the event that opens stage `k` of rbmd_energy or rbmd_energy_backward
// (profiling only; eager launches).
inline void gprof_mark(rbmd_ctx *c, int k)
{
    if (c->profiling && c->gprof_ev[0]) cudaEventRecord(c->gprof_ev[k], c->stream);
}

// Records the event that opens stage `k` of the step (profiling only).
inline void prof_mark(rbmd_ctx *c, int k)
{
    if (!c->profiling) return;
    if (c->capturing) cudaEventRecordWithFlags(c->prof_ev[k], c->stream, cudaEventRecordExternal);
    else cudaEventRecord(c->prof_ev[k], c->stream);
}

// ---- host-side helpers implemented in the .cu files ----
rbmd_status sampler_table_host(double L, double alpha, int32_t *M, uint64_t *T, double *H);

// RBE (rbe.cu)
// Standard normal deviates of the Langevin force (thermostat 2) of replica-local
// atom `id` at force evaluation `step`: Philox4x32-10, key = seed, counter
// (id, step, 0, 3 | replica << 8), uniforms (w + 1/2) 2^-32, Box-Muller.
__device__ __forceinline__ void langevin_normals(uint32_t id, uint32_t step, const Rep &rp,
                                                 double g[3])
{
    const uint4 w = philox10(make_uint4(id, step, 0u, (rp.tag_rbe & ~0xFFu) | RBMD_STREAM_LANGEVIN),
                             rp.key);
    const double u0 = ((double)w.x + 0.5) * 2.3283064365386963e-10;
    const double u1 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)w.z + 0.5) * 2.3283064365386963e-10;
    const double u3 = ((double)w.w + 0.5) * 2.3283064365386963e-10;
    const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s3, &c3);
    g[0] = r0 * c1;
    g[1] = r0 * s1;
    g[2] = r1 * c3;
}
__device__ __forceinline__ void langevin_normals(uint32_t id, uint32_t step, const Rep &rp,
                                                 float g[3])
{
    const uint4 w = philox10(make_uint4(id, step, 0u, (rp.tag_rbe & ~0xFFu) | RBMD_STREAM_LANGEVIN),
                             rp.key);
    const float u0 = ((float)(w.x >> 8) + 0.5f) * 5.9604644775390625e-8f;  // 2^-24
    const float u1 = ((float)(w.y >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float u2 = ((float)(w.z >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float u3 = ((float)(w.w >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    g[0] = r0 * c1;
    g[1] = r0 * s1;
    g[2] = r1 * c3;
}

// Arguments of the second half kick.
template <typename real> struct KickArgs {
    real *v;
    const double *scal;
    real hdt;
    double *kepart;  // [nb256] kinetic-energy partial of each 256-atom block
    int *err;
    int langevin;    // thermostat 2: add the friction and random force first
    double gamma, dt;
    StepRef sref;    // step of the force evaluation (Langevin counter)
};

__device__ __forceinline__ float kick_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double kick_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// F_corr of replica r in the working precision (the kick's constant force term).
template <typename real>
__device__ __forceinline__ void kick_fcorr(const KickArgs<real> &k, int r, real fc[3])
{
    const double *sc = k.scal + (int64_t)r * SCAL_COUNT;
#pragma unroll
    for (int d = 0; d < 3; ++d) fc[d] = (real)sc[SCAL_FCORR + d];
}

// Second half kick of atom i of replica r with force f (the atom's final force
// of the step, stored to F when the Langevin force is added to it) and F_corr fc
// (kick_fcorr); returns |v|^2, summed in the working precision (the block and
// replica sums are FP64).  Non-finite velocities latch RBMD_ERR_NONFINITE.
template <typename real>
__device__ __forceinline__ double second_kick(const KickArgs<real> &k, const Rep &rp, int r,
                                              int64_t i, real *__restrict__ v, real *__restrict__ F,
                                              real f[3], const real fc[3])
{
    (void)r;
    if (k.langevin) {
        real gn[3];
        langevin_normals((uint32_t)(i - rp.atom0), (uint32_t)step_of(k.sref), rp, gn);
        const real gm = (real)k.gamma, sd = (real)sqrt(2.0 * k.gamma * rp.T0 / k.dt);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            f[d] += -gm * v[3 * i + d] + sd * gn[d];
            F[3 * i + d] = f[d];
        }
    }
    real ke = 0;
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const real vd = v[3 * i + d] + k.hdt * (f[d] + fc[d]);
        v[3 * i + d] = vd;
        bad |= !isfinite(vd);
        ke = kick_fma(vd, vd, ke);
    }
    if (bad) latch_error(k.err, RBMD_ERR_NONFINITE);
    return (double)ke;
}

// Block sum of ke (every thread of the 256-thread block calls it) to kepart[block].
__device__ __forceinline__ void block_ke_partial(double ke, double *__restrict__ kepart)
{
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    __shared__ double s_ke[32];
    if ((threadIdx.x & 31) == 0) s_ke[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_ke[w];
        kepart[blockIdx.x] = t;
    }
}

template <typename real> KickArgs<real> kick_args(rbmd_ctx *c, StepRef sref);

rbmd_status rbe_sample(rbmd_ctx *c, StepRef s);
rbmd_status rbe_metropolis_init(rbmd_ctx *c);  // chains at step 0 (exact draw)
rbmd_status metropolis_table_host(double L, double alpha, int M, uint64_t *A);
rbmd_status rbe_structure_factors(rbmd_ctx *c, int mark_between = -1);
rbmd_status rbe_rho_partial(rbmd_ctx *c, int t0, int t1);  // tile partials of tiles [t0, t1)
rbmd_status rbe_rho_final(rbmd_ctx *c);                    // rho and coefficients from them
rbmd_status rbe_rho_from_acc(rbmd_ctx *c, const void *acc);  // the same from given exact sums
rbmd_status rbe_configure(rbmd_ctx *c);  // kernel attributes (dynamic shared memory)
rbmd_status rbl_configure(rbmd_ctx *c);  // the same for the large-batch selection
rbmd_status pair_table_host(double alpha, double r_cut, int n, std::vector<double> &coef,
                            int32_t *i0, double *inv_h);
// kick != NULL: the integrator's step; the kernel also does the second half kick
// (KickArgs of that step) and the kinetic-energy partials.  [b0, b1): the 256-atom
// blocks of map256 to cover (b1 < 0: all; a kick needs all).
rbmd_status rbe_apply_forces(rbmd_ctx *c, void *force, int accumulate,
                             const StepRef *kick = nullptr, int b0 = 0, int b1 = -1);

// RBL (rbl.cu)
// counted: the cell counts, cells and ranks are already there (the integrator's
// drift kernel bins the atoms it moves).
rbmd_status cells_build(rbmd_ctx *c, bool counted = false);
// cudaMalloc with the test hook of RBMD_FAIL_ALLOC_AFTER (api.cu)
rbmd_status dev_alloc(void **p, size_t bytes);
rbmd_status cells_count_blocks(rbmd_ctx *c, int b0, int b1);
rbmd_status rbl_pairs(rbmd_ctx *c, StepRef s, void *force, int accumulate, bool energy,
                      int32_t *n_core, int32_t *n_shell, int32_t *batch, bool marks = false);
rbmd_status rbl_correction(rbmd_ctx *c, void *force, bool apply, int slot);

rbmd_status rbl_lists(rbmd_ctx *c, StepRef s);
// The integrator's short-range part on the candidate lists: the sorted positions
// gathered from the current state, the cell sort and the candidate lists rebuilt
// on the device when an atom has moved more than half the skin since the last
// rebuild (or the layout was changed outside the step), then the exact
// classification, batch selection and pair forces (same sets as rbl_pairs).
rbmd_status verlet_prepare(rbmd_ctx *c);
rbmd_status rbl_pairs_verlet(rbmd_ctx *c, StepRef s, void *force, bool marks, bool energy = false);
rbmd_status rbl_lists_verlet(rbmd_ctx *c, StepRef s);
rbmd_status verlet_configure(rbmd_ctx *c);
rbmd_status rbl_max_counts(rbmd_ctx *c, int32_t *out_dev);

// adjoint (adjoint.cu)
rbmd_status adjoint_run(rbmd_ctx *c, double g, void *dpos, void *dq, double *tsum_dev);

// MD (md.cu)
// First half kick and drift; with bin, the moved atoms are also binned into the
// (zeroed) cell counts, as k_cell_count does, for cells_build(c, true).
rbmd_status md_kick_drift(rbmd_ctx *c, bool bin = false);
// Second half kick (unless `kicked`: the RBE force kernel already did it) and the
// thermostat; advance_step increments the device step counter.
rbmd_status md_kick_thermo(rbmd_ctx *c, bool advance_step, StepRef s, bool kicked);
rbmd_status md_thermo_prepare(rbmd_ctx *c);  // Nose-Hoover first half update before a run
rbmd_status md_sum(rbmd_ctx *c, const double *parts, int nparts, int ncomp, double *out,
                   double scale);
// Per replica r: out[r * SCAL_COUNT + slot + comp] = scale_r * (sum of the parts of
// its 128-atom blocks, 4 per block, in pass 0 and, with two_segments, pass 1 at
// offset 4 nb128).  scale_r = scale, or scale / N_r when per_atom.
// The same for the fixed-point (2^-32) force partials: exact integer sums, scaled
// to FP64 at the end.
rbmd_status md_sum_replicas_fix(rbmd_ctx *c, const long long *parts, int slot, double scale,
                                bool per_atom, bool two_segments);
rbmd_status md_sum_replicas(rbmd_ctx *c, const double *parts, int ncomp, int slot, double scale,
                            bool per_atom, bool two_segments);
rbmd_status md_decode_state(rbmd_ctx *c, void *pos, void *vel);
rbmd_status md_encode_positions(rbmd_ctx *c, const void *pos);
rbmd_status md_encode_blocks(rbmd_ctx *c, const void *pos, int b0, int b1);
rbmd_status md_kinetic(rbmd_ctx *c, int slot);

inline rbmd_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RBMD_OK : RBMD_ERR_CUDA; }

}  // namespace rbmd

#define RBMD_CHECK_CUDA(call)                                          \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return RBMD_ERR_CUDA;                  \
    } while (0)

#define RBMD_CHECK(call)                                               \
    do {                                                               \
        rbmd_status s__ = (call);                                      \
        if (s__ != RBMD_OK) return s__;                                \
    } while (0)

#define RBMD_LAUNCH_CHECK() RBMD_CHECK_CUDA(cudaGetLastError())
