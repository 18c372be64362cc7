/*
 * rbmd.h -- C ABI of the B300 random-batch nonbonded step (arXiv 2407.09315).
 *
 * The library computes, for N point charges with Lennard-Jones types in a cubic
 * periodic box of side L (Sec. 2.2: neutral system, V = L^3):
 *   - the random batch Ewald (RBE) long-range force (Sec. 2.2, Eq. 12,
 *     Algorithm 1): P Fourier modes k = 2 pi m / L, m != 0, drawn i.i.d. with
 *     probability exp(-k^2/4 alpha)/S, the structure factors
 *     rho(k) = sum_j q_j exp(i k.r_j) (Eq. 9), and
 *     F_i = -sum_l (S/P) 4 pi coulomb_k q_i k_l / (V k_l^2) Im(e^{-i k_l.r_i} rho_l);
 *   - the random batch list (RBL) short-range force (Sec. 2.3, Eqs. 13-16,
 *     Algorithm 2): an exact core list (r < r_core), a reweighted random batch of
 *     p shell neighbours (r_core <= r <= r_cut, weight N_s/p), erfc-Coulomb
 *     (Eq. 10) plus Lennard-Jones (Eq. 2, Lorentz-Berthelot mixing Eq. 4), and
 *     the momentum correction F_corr = -(1/N) sum_i (F_core + F_shell*) (Eq. 16);
 *   - velocity-Verlet with an optional Berendsen, Langevin or Nose-Hoover
 *     thermostat (Sec. 2.1).
 *
 * Naming: r_core is the paper's inner radius r_c and r_cut its outer radius r_s.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" must be device memory of the context's GPU
 *     (for example torch CUDA tensors); "host" marks host memory; "host or
 *     device" accepts either (copied with cudaMemcpyDefault under unified
 *     addressing; pinned host memory keeps the copy asynchronous).
 *   - Real-valued arrays are float for RBMD_FP32 contexts and double for
 *     RBMD_FP64 contexts ("real" below).  Vectors are [N][3], row-major,
 *     in the caller's atom order (atom id = row index).
 *   - The caller owns every buffer it passes; rbmd_init copies the inputs into
 *     the context's own layout and the context owns all its device state.
 *   - Work is queued on the stream given to rbmd_init.  Calls that return host
 *     values (rbmd_energy, rbmd_get_state, rbmd_sync, rbmd_rbe_modes) wait for
 *     the stream; the others return as soon as the work is queued.  A force
 *     evaluation (every step, rbmd_forces) forks the RBE sampling and structure
 *     factors onto a second stream owned by the context and joins it back before
 *     the RBE force pass, so work queued on the caller's stream after the call
 *     sees the whole evaluation.  The environment variable RBMD_ONE_STREAM=1 at
 *     rbmd_init keeps everything on the caller's stream (same results, bit for
 *     bit).
 *   - Test hooks, read by rbmd_init unless noted (none changes a result):
 *     RBMD_LIST_CAPS="cc,cs" shrinks the core and shell list capacities so that
 *     atoms take the exact overflow path; RBMD_SELECT_EXACT=1 sends every batch selection
 *     through the exact 64-bit path; RBMD_SELECT_KEY_BITS=k keeps only k
 *     priority bits in the fast selection's keys (equal keys then send atoms
 *     to the exact path); RBMD_HOST_CHUNKS=k (1..8, read per call) sets the
 *     chunk count of rbmd_forces_host (default 4).
 *   - Errors are returned, never raised or aborted on.  Device-side faults
 *     (non-finite forces, timeouts) are latched in a device error word and
 *     returned by the next call that synchronises.
 *   - `step` keys every random draw (RBE modes and RBL batches): the same state
 *     and step give bit-identical results.
 *   - A context is not thread-safe; use one context per stream.
 */
#ifndef RBMD_H
#define RBMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbmd_ctx rbmd_ctx;

typedef enum {
    RBMD_OK = 0,
    RBMD_ERR_INVALID = 1,        /* bad argument or parameter */
    RBMD_ERR_NOT_NEUTRAL = 2,    /* |sum q| > 1e-6 * sum |q| (Sec. 2.2 needs neutrality) */
    RBMD_ERR_BOX_TOO_SMALL = 3,  /* r_cut >= L/2: minimum image not unique */
    RBMD_ERR_OOM = 4,            /* a device allocation failed */
    RBMD_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    RBMD_ERR_CELL_OVERFLOW = 6,  /* a cell or list exceeded its capacity */
    RBMD_ERR_NONFINITE = 7,      /* a force or velocity became NaN/Inf */
    RBMD_ERR_TIMEOUT = 8,        /* a bounded device wait gave up (reserved: no kernel of
                                    this library waits on another, so no call returns it;
                                    rbmd_debug_latch_error can latch it for tests) */
    RBMD_ERR_UNSUPPORTED = 9,    /* combination of options not built */
    RBMD_ERR_BOUNDS = 10         /* an index out of range (bounds-checked builds only:
                                    compiled with -DRBMD_CHECKED, the access is skipped) */
} rbmd_status;

typedef enum { RBMD_FP32 = 0, RBMD_FP64 = 1 } rbmd_precision;

/* rbmd_params.flags */
#define RBMD_FULL_EWALD_MODES 1u /* RBE uses every m != 0 with |m_d| <= M and weights
                                    exp(-k^2/4 alpha): the Ewald series of Eq. 11 */
#define RBMD_RBL_EXACT 2u        /* RBL keeps every shell neighbour with weight 1 */
#define RBMD_NO_RBE 4u           /* skip the long-range part (LJ-fluid runs) */
#define RBMD_NO_RBL 8u           /* skip the short-range part */
#define RBMD_PAIR_TABLE 16u      /* erfc-Coulomb pair terms from a cubic look-up table
                                    (Sec. 3.3; rbmd_pair_table) instead of erfc/exp */
#define RBMD_METROPOLIS_MODES 32u /* RBE modes from Metropolis chains (Algorithm 1 step 1)
                                     instead of exact i.i.d. draws; see rbmd_metropolis_table */

typedef struct {
    int64_t n_atoms;     /* N >= 1 */
    int32_t n_types;     /* LJ types, 1..64 */
    int32_t rbe_P;       /* RBE batch size P >= 1 (Eq. 12) */
    double box_length;   /* L > 0 */
    double alpha;        /* splitting parameter of Eq. 6 (erfc(sqrt(alpha) r)) */
    double r_core;       /* inner radius (paper r_c), 0 <= r_core <= r_cut */
    double r_cut;        /* outer radius (paper r_s), r_cut < L/2 */
    int32_t rbl_p;       /* RBL shell batch size p, 1..1024 (Eq. 15); above 32 an atom
                            whose lists overflow latches RBMD_ERR_CELL_OVERFLOW */
    int32_t thermostat;  /* 0 none (NVE), 1 Berendsen, 2 Langevin, 3 Nose-Hoover, 4 energy
                            bath (NVE held at the bath energy E0, Sec. 2.1; rbmd_step) */
    double coulomb_k;    /* Coulomb prefactor (1/(4 pi eps0) of Eq. 3; Bjerrum length in reduced units) */
    double dt;           /* time step */
    double temperature;  /* thermostat target T0 (k_B = 1) */
    double tau_T;        /* thermostat time: Berendsen and energy-bath coupling time,
                            Langevin 1/gamma, Nose-Hoover period scale (Q = g T0 tau^2);
                            <= 0 selects 0.1 */
    uint64_t seed;       /* Philox key of every random draw */
    uint32_t replica;    /* replica index mixed into the random streams */
    int32_t precision;   /* rbmd_precision */
    uint32_t flags;      /* RBMD_* flags above */
    int32_t cell_div;    /* cells per r_cut along each axis: 1 or 2; 0 = 2 (rbmd_set_tiles
                            and rbmd_autotune change it later) */
    int32_t mh_moves;    /* RBMD_METROPOLIS_MODES: moves per chain per step (0 = 8) */
    double skin;         /* rbmd_step's neighbour candidates: every atom within r_cut + skin
                            at the last rebuild (sigma units); 0 selects 0.4, < 0 turns the
                            candidate lists off (every step walks the cells).  The lists,
                            batches and forces do not depend on it (see rbmd_step). */
} rbmd_params;

/* Energies and diagnostics (host, FP64).  Potential terms follow Eq. 8 with the
 * random-batch estimators: e_rbe = coulomb_k (2 pi S/(V P)) sum_l |rho_l|^2/k_l^2
 * (unbiased for Eq. 8's long-range term), e_coul_real and e_lj use the RBL list
 * with 1/2 sum_i [sum_{C(i)} u_ij + (N_s/p) sum_{B(i)} u_ij]. */
typedef struct {
    double e_coul_real;   /* erfc-Coulomb over the RBL lists */
    double e_lj;          /* Lennard-Jones over the RBL lists */
    double e_rbe;         /* RBE estimate of the Fourier-space energy */
    double e_self;        /* -coulomb_k sqrt(alpha/pi) sum q^2 */
    double e_potential;   /* sum of the four terms above */
    double e_kinetic;     /* 1/2 sum v^2 (unit masses) */
    double temperature;   /* 2 KE / (3N - 3) */
    double S;             /* normaliser sum_{m != 0} exp(-k^2/4 alpha) */
    double fsum_short[3]; /* sum_i (F_core + F_shell*) before the correction */
    int64_t step;         /* step the energies were evaluated at */
    int32_t max_shell;    /* largest N_s over atoms */
    int32_t max_cell;     /* largest cell occupancy */
    /* Virial W_ab = -dE/d(strain_ab) at fixed fractional coordinates (the box and
     * every position deformed together).  Pair part (list weights held fixed):
     * 1/2 sum_i [sum_{C(i)} r_ij (x) F_ij + (N_s/p) sum_{B(i)} r_ij (x) F_ij],
     * r_ij = r_i - r_j (minimum image), F_ij the erfc-Coulomb + LJ pair force on i
     * (Eqs. 2, 10, 15).  Fourier part: sum_l e_l [delta_ab - 2 k_a k_b (1/k_l^2 +
     * 1/(4 alpha))] over the drawn modes with e_l the terms of e_rbe, an unbiased
     * estimate of the virial of Eq. 8's Fourier term (the strain derivative of
     * its Gaussian weights and 1/V).  The self term and the momentum correction
     * (Eq. 16) add nothing.  FP64 reductions. */
    double virial[6];        /* xx, yy, zz, xy, xz, yz of the total */
    double virial_coul_real; /* trace of the erfc-Coulomb pair part */
    double virial_lj;        /* trace of the LJ pair part */
    double virial_rbe;       /* trace of the Fourier (RBE) part */
    double pressure;         /* (2 e_kinetic + trace of virial) / (3 V) */
} rbmd_energy_terms;

/* Name of a status code (static string). */
const char *rbmd_status_string(rbmd_status s);

/* Library version string (static). */
const char *rbmd_version(void);

/*
 * rbmd_init -- create a context (Sec. 2.1 workflow: read the configuration,
 * map the particle arrays to the device).
 *   params   host, read once.
 *   pos      device, real [N][3]; wrapped into [0, L) and stored as 32-bit
 *            fixed-point fractions u = floor(x * 2^32 / L).
 *   vel      device, real [N][3], or NULL for zero velocities.
 *   charge   device, real [N]; must be neutral (RBMD_ERR_NOT_NEUTRAL).
 *   type     device, int32 [N] in [0, n_types), or NULL for all type 0.
 *   lj_eps, lj_sigma  host, double [n_types]; mixed by Lorentz-Berthelot (Eq. 4).
 *   stream   cudaStream_t to queue all work on (NULL = legacy default stream).
 *   out      receives the context; NULL on error.
 * Errors: INVALID (bad sizes, r_core > r_cut, p or P out of range, bad type),
 * BOX_TOO_SMALL (r_cut >= L/2), NOT_NEUTRAL, OOM, CUDA.
 */
rbmd_status rbmd_init(const rbmd_params *params, const void *pos, const void *vel,
                      const void *charge, const int32_t *type, const double *lj_eps,
                      const double *lj_sigma, void *stream, rbmd_ctx **out);

/*
 * rbmd_init_batch -- one context over R independent systems (replicas) that are
 * stepped together: every kernel of a step covers all of them in one launch, so
 * small systems fill the GPU.  Replicas never interact; each has its own box,
 * cells, modes, momentum correction, thermostat and energies.  The paper runs
 * one system per job; batching is this library's addition (the per-system
 * arithmetic is unchanged, so replica r of a batch gives the same lists, modes
 * and draws as a stand-alone context with the same parameters).
 *   params   host, rbmd_params [R].  Per replica: n_atoms, box_length, seed,
 *            replica, temperature.  Every other field must equal params[0]'s
 *            (INVALID otherwise).  RBMD_FULL_EWALD_MODES needs R == 1
 *            (UNSUPPORTED otherwise).
 *   pos, vel, charge, type  as in rbmd_init, concatenated in replica order
 *            (replica r's atoms start at n_atoms[0] + ... + n_atoms[r-1]);
 *            each replica must be neutral on its own.
 *   lj_eps, lj_sigma  host, double [n_types], shared by all replicas.
 * Every per-atom buffer of the other entry points (forces, state, gradients,
 * lists) is the concatenated [N_total] array; atom ids in rbmd_rbl_lists are
 * indices into it.  rbmd_rbe_modes returns R blocks of P modes.  The gradients of
 * rbmd_energy_backward are those of the sum of the replicas' potentials (so
 * d_pos and d_q are per replica, d_eps and d_sigma summed over replicas).
 * Errors: as rbmd_init, plus INVALID for R < 1 or mismatched shared fields.
 */
rbmd_status rbmd_init_batch(const rbmd_params *params, int32_t R, const void *pos,
                            const void *vel, const void *charge, const int32_t *type,
                            const double *lj_eps, const double *lj_sigma, void *stream,
                            rbmd_ctx **out);

/* Number of replicas of the context (1 for rbmd_init), 0 for NULL. */
int32_t rbmd_replica_count(rbmd_ctx *ctx);

/*
 * Tile shapes of the hot kernels (the paper has no counterpart: these are
 * implementation choices of this library, with no effect on the integer work).
 *   cell_div       cells per r_cut along each axis, 1 or 2 (binning and the
 *                  neighbour stencil, Sec. 2.3).  Lists and batches are the same
 *                  sets for both; only the order in which pairs are summed changes.
 *   rho_tile       atoms per structure-factor block, 512, 1024 or 2048.
 *   rho_mode_tile  modes per structure-factor block, 64, 128 or 256.
 * The tile shape only changes the FP rounding order of rho(k) (results stay
 * within the precision's tolerance).  Defaults: cell_div from the parameters (2
 * when 0), 1024, 256.
 * rbmd_set_tiles  sets them (INVALID for other values).  Synchronises.
 * rbmd_get_tiles  out: host int32 [4] = cell_div, rho_tile, rho_mode_tile, and 1
 *                 when the pair look-up table is in use (rbmd_set_pair_table).
 * rbmd_autotune   times the RBL part for each cell_div and the structure factors
 *                 for each (rho_tile, rho_mode_tile) on the current state with the
 *                 draws of `step`, after one untimed run, 3 timed runs each, and
 *                 keeps the fastest, then times the pair kernels with and without
 *                 the look-up table; chosen (host int32 [4], or NULL) receives
 *                 them as rbmd_get_tiles does.  Synchronises.  A batch context
 *                 tunes once for all replicas.  Scratch force buffers are
 *                 overwritten; the state
 *                 (positions, velocities, step counter) is not changed.
 */
rbmd_status rbmd_set_tiles(rbmd_ctx *ctx, int32_t cell_div, int32_t rho_tile,
                           int32_t rho_mode_tile);
rbmd_status rbmd_get_tiles(rbmd_ctx *ctx, int32_t *out);
rbmd_status rbmd_autotune(rbmd_ctx *ctx, int64_t step, int32_t *chosen);

/*
 * rbmd_set_pair_table -- pair kernels evaluate the erfc-Coulomb force and energy
 * from the look-up table (on != 0) or from erfc/exp (0); the initial choice is
 * the RBMD_PAIR_TABLE flag.  rbmd_autotune also times both and keeps the faster
 * (chosen[3], rbmd_get_tiles out[3]: 1 = table).  Synchronises.
 *
 * rbmd_pair_table -- the table itself (host), Sec. 3.3's look-up method: n cubic
 * pieces over s = r^2 in [0, r_cut^2 (1 + 1e-6)], h = that / n; piece k, local
 * t = s/h - k in [0, 1]: coef[8k..8k+3] = c0..c3 of the force factor
 *   f(s) = [erfc(sqrt(alpha s))/sqrt(s) + 2 sqrt(alpha/pi) e^{-alpha s}] / s,
 * coef[8k+4..8k+7] of the energy factor e(s) = erfc(sqrt(alpha s))/sqrt(s); for
 * k < *i0 the pieces hold f - s^{-3/2} and e - s^{-1/2} (the bare terms are added
 * exactly).  Cubics through the exact values at t = 0, 1/3, 2/3, 1.  coef (may be
 * NULL) must hold 8 n doubles; *inv_h = 1/h.  Contexts use n = 1024 (FP32) and
 * 8192 (FP64).  INVALID for alpha <= 0, r_cut <= 0 or n < 16.
 */
rbmd_status rbmd_set_pair_table(rbmd_ctx *ctx, int32_t on);
rbmd_status rbmd_pair_table(double alpha, double r_cut, int32_t n, int32_t *i0, double *inv_h,
                            double *coef);

/* Free every device buffer of the context (waits for its stream). NULL is a no-op. */
void rbmd_destroy(rbmd_ctx *ctx);

/*
 * rbmd_rbe_forces -- RBE long-range force of the current positions, Eq. 12 and
 * Algorithm 1: draw the P modes of `step` on the device, reduce rho(k_l) over all
 * N charges, then F_i for every atom.
 *   force      device, real [N][3]; overwritten, or added to when accumulate != 0.
 * With RBMD_FULL_EWALD_MODES the full Ewald Fourier force of Eq. 11 is computed.
 */
rbmd_status rbmd_rbe_forces(rbmd_ctx *ctx, int64_t step, void *force, int accumulate);

/*
 * rbmd_rbl_forces -- RBL short-range force, Eqs. 13-16 and Algorithm 2: cell
 * binning, exact core list, a random batch of p shell neighbours of `step`
 * weighted N_s/p, erfc-Coulomb + LJ pair forces and the momentum correction of
 * Eq. 16 added to every atom.
 *   force      device, real [N][3]; overwritten, or added to when accumulate != 0.
 */
rbmd_status rbmd_rbl_forces(rbmd_ctx *ctx, int64_t step, void *force, int accumulate);

/*
 * rbmd_forces -- RBE + RBL (with correction) in one call; same arguments.  Without
 * accumulate, a context that keeps the step's candidate lists (see rbmd_step)
 * evaluates the short-range part through them at the current positions,
 * rebuilding them on the device when an atom has moved more than skin/2 (the same
 * sets as the cell walk of rbmd_rbl_forces, summed in the step's order: equal to
 * it up to the last bits).  rbmd_energy and rbmd_energy_backward do the same.
 */
rbmd_status rbmd_forces(rbmd_ctx *ctx, int64_t step, void *force, int accumulate);

/*
 * rbmd_forces_host -- host buffers in and out: the positions become the state
 * (as rbmd_set_state(ctx, pos, NULL, step)) and the forces of rbmd_forces(step)
 * are written to the host array, bit for bit the same as that sequence followed
 * by a copy.  The positions are copied in chunks on a copy stream; each chunk is
 * encoded and binned, and its structure-factor tiles summed, while the next one
 * is copied, the short-range part goes through the candidate lists as in
 * rbmd_forces, and the RBE force pass runs in chunks whose forces are copied out
 * while the next chunk is computed.  Returns when the forces are on the host.
 *   pos        host (pinned for overlap), real [N][3], caller's atom order.
 *   force      host, real [N][3]; overwritten.
 * With RBMD_NO_RBE or RBMD_NO_RBL, or while stages are timed (rbmd_profile), the
 * same work runs in sequence on the context's stream.  Device-side faults are
 * latched as for rbmd_forces.
 */
rbmd_status rbmd_forces_host(rbmd_ctx *ctx, const void *pos, void *force, int64_t step);

/*
 * rbmd_step -- advance n_steps velocity-Verlet steps (Sec. 2.1): half kick,
 * drift of the fixed-point positions (wrapping is modular), forces of the new
 * configuration keyed by the new step number, half kick, thermostat.  Unit
 * masses, k_B = 1, g = 3N - 3 degrees of freedom per system, T = 2 KE / g.
 *   1 Berendsen: v *= lambda = sqrt(1 + (dt/tau)(T0/T - 1)), clamped to [0.8, 1.25].
 *   2 Langevin (Schneider-Stoll): after the forces of the new configuration every
 *     atom gets F_L = -gamma v + sqrt(2 gamma T0 / dt) G, gamma = 1/tau, v the
 *     half-step velocity, G standard normal (Philox4x32-10, key = seed, counter
 *     (replica-local atom id, step of that force evaluation, 0, 3 | replica << 8),
 *     uniforms (w + 1/2) 2^-32 (FP32 contexts: ((w >> 8) + 1/2) 2^-24), Box-Muller:
 *     (G_x, G_y) = sqrt(-2 ln u0)(cos, sin)(2 pi u1), G_z = sqrt(-2 ln u2) cos(2 pi u3));
 *     F + F_L drives the second half-kick and the next first half-kick.
 *   3 Nose-Hoover, one variable xi, Q = g T0 tau^2: xi += dt/2 (2 KE - g T0)/Q,
 *     v *= e^{-xi dt/2}, kick-drift-force-kick, v *= e^{-xi dt/2},
 *     xi += dt/2 (2 KE - g T0)/Q.
 * The context's step counter advances by n_steps.  Queued as one CUDA graph per
 * step after the first call.
 * Short-range lists of the step (Algorithm 2 step 1): unless params.skin < 0 (or
 * with RBMD_RBL_EXACT, p > 32 or r_cut + skin >= L/2), the step keeps for every
 * atom its candidates, the atoms within r_cut + skin at the last rebuild, and
 * classifies them exactly each step on the integer positions.  A rebuild (cell
 * sort and candidates) runs inside the step, on the device, when some atom has
 * moved more than skin/2 since the last one (an exact integer test) or when
 * another call changed the sorted layout.  The core list, N_s and the batch are
 * the sets of the cell walk that rbmd_rbl_forces does; the core list and a whole
 * shell are summed in atom-id order and a drawn batch in priority order, so the
 * forces do not depend on when rebuilds happen (a resumed run stays
 * bit-identical), but they may differ from rbmd_rbl_forces in the last bits.  An
 * atom beyond the lists' capacities (a density fluctuation of over 5 standard
 * deviations) is computed by the exact cell walk instead.
 */
rbmd_status rbmd_step(rbmd_ctx *ctx, int64_t n_steps);

/* Rebuilds of the step's candidate lists so far (0 when they are off, see
 * rbmd_step); -1 for NULL.  Synchronises. */
int64_t rbmd_candidate_rebuilds(rbmd_ctx *ctx);

/*
 * Nose-Hoover variable xi of every replica at the step boundary (host double [R]),
 * for checkpoints; rbmd_set_thermostat also makes the next rbmd_step recompute the
 * forces.  Energy bath (thermostat 4): the bath energy E0 of every replica.  The
 * bath relaxes the total energy H = K + U toward E0 after every second half kick,
 * lambda^2 = 1 + (dt/tau_T)((E0 - U)/K - 1) clamped to [0.64, 1.5625], U the
 * potential of the step's force evaluation (its random batches) -- a reading of
 * the energy-stable scheme that Sec. 2.1 names without its steps.  Unless set,
 * the first rbmd_step of a run takes E0 = K + U of the state it starts from (NaN
 * is returned until then); rbmd_set_state, rbmd_set_state_u, rbmd_set_charges,
 * rbmd_set_lj and rbmd_forces_host clear it, so set it after them.  Each step of
 * this thermostat also evaluates the potential (the energy sums of the pair
 * kernels and of the modes).  A Berendsen factor is folded into the velocities that rbmd_get_state
 * returns; the Langevin random force of the last step is not part of the state
 * (a resumed Langevin run draws the same later noise but restarts its first
 * half-kick from the conservative force).
 */
rbmd_status rbmd_get_thermostat(rbmd_ctx *ctx, double *xi);
rbmd_status rbmd_set_thermostat(rbmd_ctx *ctx, const double *xi);

/*
 * rbmd_energy -- energies and diagnostics of the current state, with the random
 * draws of `step` (out: host).  Synchronises; returns a latched device error.
 */
rbmd_status rbmd_energy(rbmd_ctx *ctx, int64_t step, rbmd_energy_terms *out);

/*
 * rbmd_energy_batch -- rbmd_energy for every replica: out is host
 * rbmd_energy_terms [R] (replica order).  rbmd_energy is INVALID on a context
 * with R > 1.  max_shell and max_cell are taken over the whole batch.
 */
rbmd_status rbmd_energy_batch(rbmd_ctx *ctx, int64_t step, rbmd_energy_terms *out);

/*
 * rbmd_energy_backward -- gradients of E = e_coul_real + e_lj + e_rbe + e_self
 * (rbmd_energy's potential, draws of `step`) times grad_out.
 *   d_pos    device, real [N][3], dE/dr (or NULL)
 *   d_q      device, real [N], dE/dq (or NULL)
 *   d_eps    host, double [n_types], dE/d eps_t (or NULL)
 *   d_sigma  host, double [n_types], dE/d sigma_t (or NULL)
 * The RBL energy weights a pair by its list weight, so dE/dr is the
 * symmetrised force -(1/2) sum_j (W_ij + W_ji) u'(r_ij) r_hat (the paper's
 * one-sided RBL force is not a gradient); with RBMD_RBL_EXACT it equals -F
 * without the momentum correction.  The list weights are those of `step` and
 * are held fixed (E jumps where a membership changes).  Always synchronises
 * (the lists of the step must be complete: list capacities grow if needed).
 * dE/d eps_t needs eps_t > 0.  Right after rbmd_energy of the same state and
 * step (no call in between that writes the lists, modes, positions or charges)
 * its lists, modes and structure factors are reused: the same bits as computing
 * them again.  The first call allocates the reverse-batch array ([N] x the
 * shell capacity, int32) that the gradient pass keeps.
 */
rbmd_status rbmd_energy_backward(rbmd_ctx *ctx, int64_t step, double grad_out, void *d_pos,
                                 void *d_q, double *d_eps, double *d_sigma);

/*
 * rbmd_set_charges -- replace the per-atom charges (device, real [N], caller
 * order).  Neutrality is not re-checked, so that charge derivatives can be taken
 * by perturbation; the Fourier sum omits k = 0 either way (Sec. 2.2).
 * Synchronises.  The next rbmd_step recomputes the forces.
 * rbmd_set_lj -- replace the per-type LJ parameters (host, double [n_types];
 * Lorentz-Berthelot mixing, Eq. 4).  Synchronises.
 */
rbmd_status rbmd_set_charges(rbmd_ctx *ctx, const void *charge);
rbmd_status rbmd_set_lj(rbmd_ctx *ctx, const double *lj_eps, const double *lj_sigma);

/* Checkpoint: positions (real [N][3], decoded x = u L / 2^32), velocities
 * (real [N][3]) and the step counter.  Buffers host or device. get_state
 * synchronises. */
rbmd_status rbmd_get_state(rbmd_ctx *ctx, void *pos, void *vel, int64_t *step);
rbmd_status rbmd_set_state(rbmd_ctx *ctx, const void *pos, const void *vel, int64_t step);

/* Exact checkpoint: fixed-point positions u (uint32 [N][3]), velocities
 * (real [N][3], or NULL to keep them) and the step counter.  Host or device
 * buffers.  A save + load round trip is bit-identical. */
rbmd_status rbmd_get_state_u(rbmd_ctx *ctx, uint32_t *u, void *vel, int64_t *step);
rbmd_status rbmd_set_state_u(rbmd_ctx *ctx, const uint32_t *u, const void *vel, int64_t step);

/* Wait for the stream and return (then clear) the latched device error. */
rbmd_status rbmd_sync(rbmd_ctx *ctx);

/*
 * Inspection of the random draws, for verification.
 * rbmd_rbe_modes: the P modes m_l of `step` (host int32 [P][3], or NULL) and the
 *   structure factors rho_l (host double [P][2] = re, im, or NULL), reduced on the
 *   device in the context's precision.  In full-Ewald mode P is the full mode count
 *   (rbmd_rbe_mode_count).  A batch context returns R consecutive blocks of P
 *   ([R][P][3] and [R][P][2]).  Synchronises.
 * rbmd_rbl_lists: per atom (caller order) the core count |C(i)|, shell count N_s,
 *   and the batch B(i) as atom ids ascending, -1 padded (device int32 [N], [N],
 *   [N][p]; all three required).
 */
int64_t rbmd_rbe_mode_count(rbmd_ctx *ctx);
rbmd_status rbmd_rbe_modes(rbmd_ctx *ctx, int64_t step, int32_t *m, double *rho);
rbmd_status rbmd_rbl_lists(rbmd_ctx *ctx, int64_t step, int32_t *n_core, int32_t *n_shell,
                           int32_t *batch);

/*
 * rbmd_metropolis_table -- acceptance thresholds of the Metropolis mode chains
 * (RBMD_METROPOLIS_MODES; the paper draws the modes by the Metropolis procedure,
 * Algorithm 1 step 1).  Chain l of a context is one mode slot: a random walk on
 * Z^3 \ {0} with the symmetric proposal m' = m + delta e_d, accepted with
 * min(1, exp(-a (|m'|^2 - |m|^2))), a = pi^2/(alpha L^2), m' = 0 rejected.  A move
 * that raises |m| (delta m_d >= 0, k = |m_d|) is accepted when the 64-bit uniform
 * U < A[k] = min(2^64 - 1, floor(exp(-a (2k + 1)) 2^64)), k = 0..2M (rejected for
 * k > 2M).  The chains start at step 0 from the exact draw of step 0 (stationary);
 * each later step s makes mh_moves moves, move t from Philox4x32-10 (key = seed,
 * counter (l, t, s, 4 | replica << 8)): d = w0 mod 3, delta = +1 if w1 is odd
 * else -1, U = w2 << 32 | w3.  The modes of a step are a function of (seed,
 * replica, step): a call for an earlier step replays the chains from step 0.
 * A must hold 2M + 1 entries (M from rbmd_sampler_table).
 */
rbmd_status rbmd_metropolis_table(double box_length, double alpha, uint64_t *A);

/*
 * rbmd_sampler_table -- host-side inverse-CDF thresholds of the per-dimension
 * sampler (Eq. 12 density factorises as prod_d exp(-a m_d^2), a = pi^2/(alpha L^2)):
 * M = ceil(sqrt(ln(1e16)/a)); T[j] = min(2^64-1, floor(CDF_j 2^64)), j = 0..2M.
 * Call with T == NULL to get M; T must hold 2M+1 entries.  H (may be NULL)
 * receives sum_{|m|<=M} exp(-a m^2), so S = H^3 - 1.
 */
rbmd_status rbmd_sampler_table(double box_length, double alpha, int32_t *M, uint64_t *T,
                               double *H);

/*
 * Measurement hooks.
 * rbmd_profile: enable (1) or disable (0) per-stage timing of rbmd_step; CUDA
 *   events are recorded between the stages inside the step graph and read after
 *   each step (profiling makes rbmd_step wait for every step).  Stages:
 *   0 kick+drift, 1 cell sort, 2 RBL list scan, 3 RBL batch selection,
 *   4 RBL pair forces (+ overflow fallback), 5 F_corr reduction,
 *   6 RBE mode sampling, 7 structure-factor partials, 8 structure-factor
 *   final reduction, 9 RBE force kernel (which also does the second half kick),
 *   10 thermostat (and the second half kick when RBE is off).
 * rbmd_profile_read: accumulated milliseconds per stage (host double
 *   [RBMD_PROFILE_STAGES]) and the number of profiled steps; reset != 0 zeroes them.
 * rbmd_step_kernel_count: kernel launches in one step graph (captured on the
 *   first rbmd_step; 0 before that) on a step without a candidate-list rebuild.
 * rbmd_rebuild_kernel_count: the kernels a step adds when it rebuilds the
 *   candidate lists (the body of the graph's conditional node; 0 when the rebuild
 *   kernels are ordinary graph nodes that return at once on other steps, which
 *   rbmd_step_kernel_count then includes, as with RBMD_GRAPH_COND=0 in the
 *   environment, or when the step has no candidate lists).
 */
#define RBMD_PROFILE_STAGES 11
rbmd_status rbmd_profile(rbmd_ctx *ctx, int enable);
rbmd_status rbmd_profile_read(rbmd_ctx *ctx, double *ms, int64_t *steps, int reset);
int32_t rbmd_step_kernel_count(rbmd_ctx *ctx);
int32_t rbmd_rebuild_kernel_count(rbmd_ctx *ctx);

/*
 * rbmd_profile_read_grad: while profiling is enabled, rbmd_energy and
 * rbmd_energy_backward also record events between their stages; accumulated
 * milliseconds (host double) and call counts (host int64 [2]: forward,
 * backward; any pointer may be NULL); reset != 0 zeroes them.
 *   forward [RBMD_PROFILE_FWD_STAGES]: 0 RBE sampling, structure factors and mode
 *     energy/virial sums, 1 cell sort, 2 RBL lists, batches and pair
 *     energies/virials, 3 FP64 sums and kinetic energy;
 *   backward [RBMD_PROFILE_GRAD_STAGES]: 0 cell sort and complete lists, 1 RBE
 *     sampling and structure factors, 2 output initialisation and the self
 *     term, 3 RBL adjoint (pair gradients and per-type sums), 4 RBE adjoint.
 */
#define RBMD_PROFILE_FWD_STAGES 4
#define RBMD_PROFILE_GRAD_STAGES 5
rbmd_status rbmd_profile_read_grad(rbmd_ctx *ctx, double *fwd_ms, double *bwd_ms, int64_t *calls,
                                   int reset);

/*
 * rbmd_rbe_forces_noalloc -- the RBE force of rbmd_rbe_forces (same mode draws,
 * same structure factors and force pass, FP32 arithmetic) for callers that
 * cannot allocate device memory: code that runs while another framework owns
 * all device memory through its own pool, or a latency-critical path where a
 * cudaMalloc would synchronise the device.  It needs no context and allocates
 * nothing (no cudaMalloc, cudaFree or allocating library call); the paper has
 * no counterpart of this call.
 *   u          device, uint32 [N][3]: fixed-point fractional positions,
 *              x = u L / 2^32 (as rbmd_get_state_u returns them).
 *   charge     device, float [N].
 *   force      device, float [N][3], overwritten.
 *   alpha, coulomb_k, P, seed, step, replica: as in rbmd_params / rbmd_rbe_forces.
 *   stream     cudaStream_t to queue on (NULL = legacy default stream).
 * Scratch: one static device array of RBMD_NOALLOC_SCRATCH_BYTES, held by every
 * GPU that loads the library until the process exits and shared by all calls.
 * Each call writes every scratch value it reads, so nothing carries over from
 * the previous call, but calls that overlap on the GPU (two streams of the
 * same device) race on it; calls are also not thread-safe on the host.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The address is kept for the life of the process, so a
 * device reset (cudaDeviceReset) between calls is not supported.
 * Errors: RBMD_ERR_INVALID for null pointers, N < 1 or N > 2^31 - 1,
 * P > RBMD_NOALLOC_MAX_P, or a sampler table longer than RBMD_NOALLOC_MAX_TABLE
 * entries (box too large for alpha); RBMD_ERR_CUDA if a launch fails.
 */
#define RBMD_NOALLOC_MAX_P 512
#define RBMD_NOALLOC_MAX_TABLE 4096
#define RBMD_NOALLOC_SCRATCH_BYTES 2359296u /* 2.25 MiB */
rbmd_status rbmd_rbe_forces_noalloc(const uint32_t *u, const float *charge, int64_t n_atoms,
                                    double box_length, double alpha, double coulomb_k,
                                    int32_t P, uint64_t seed, int64_t step, uint32_t replica,
                                    float *force, void *stream);

/*
 * Spatial decomposition of one system over several contexts (one per GPU): the
 * paper names running on several GPUs as future work (Sec. 5); the split follows
 * the RBE's structure (Sec. 2.2 below Eq. 12: the structure factors are sums over
 * atoms, so each rank sums its own atoms and the ranks exchange 2P numbers) and
 * the short range of the RBL (Sec. 2.3: an atom needs the atoms within r_cut).
 *
 * rbmd_init_slab -- a context over the atoms one rank owns, rows 0 .. n_owned-1,
 *   followed by its halo, rows n_owned .. N-1: atoms of other ranks within r_cut
 *   (with a margin) of the owned ones, all in the global box.  params->n_atoms =
 *   N (owned + halo); gid (device, uint32 [N]) the global ids of the rows: every
 *   random draw (RBE modes, RBL batch priorities and their ties) is keyed by the
 *   global ids, so the modes, |C(i)|, N_s and B(i) of an owned atom are those of
 *   one context holding all n_global atoms.  The slab need not be neutral.
 *   Supported calls on a slab context: rbmd_rbe_rho_partial, rbmd_rbe_forces_rho,
 *   rbmd_rbl_forces_slab, rbmd_add_correction, rbmd_rbl_lists, rbmd_set_state(_u),
 *   rbmd_get_state(_u), rbmd_sync, rbmd_destroy (others: RBMD_ERR_UNSUPPORTED).
 *   Errors: as rbmd_init; INVALID for n_owned outside [1, N], n_global < n_owned,
 *   p > 32 or RBMD_FULL_EWALD_MODES.
 *
 * rbmd_rbe_rho_partial -- the structure factors of the owned atoms for the modes
 *   of `step` as exact sums (Eq. 9): acc (host, int64 [P][4]) holds, per mode,
 *   Re and Im as 128-bit fixed-point integers in units of 2^-64, each two int64
 *   words (low word first, as unsigned, then the signed high word).  The atoms'
 *   tile partials are added as integers, so the sum over ranks (rbmd_rho_acc_add,
 *   in any order) equals bit for bit the sums of one context whose atom tiles hold
 *   the same atoms (an ordinary context returns its full sums here too).
 *   Synchronises.
 * rbmd_rho_acc_add -- sum[k] += part[k] for n_modes modes of acc words (host
 *   arithmetic on 128-bit integers, wrapping like the device sums).
 * rbmd_rbe_forces_rho -- the RBE force (Eq. 12) of the owned atoms of `step` from
 *   given summed structure factors acc (host, int64 [P][4]): every rank passing the
 *   same sums computes the same rho and coefficients.  force (device, real [N][3]):
 *   owned rows overwritten (or added to when accumulate != 0); halo rows are
 *   unspecified.
 * rbmd_rbl_forces_slab -- the RBL force of the owned atoms without the momentum
 *   correction (Eqs. 13-15; halo rows set to zero unless accumulate), and in
 *   fsum (host double [3]) the sum of those forces over the owned atoms.
 *   Synchronises.
 * rbmd_add_correction -- adds -fsum_total / n_global (Eq. 16: fsum_total the sum
 *   of every rank's fsum) to the owned rows of force (device, real [N][3]).
 */
rbmd_status rbmd_init_slab(const rbmd_params *params, int64_t n_owned, int64_t n_global,
                           const uint32_t *gid, const void *pos, const void *vel,
                           const void *charge, const int32_t *type, const double *lj_eps,
                           const double *lj_sigma, void *stream, rbmd_ctx **out);
rbmd_status rbmd_rbe_rho_partial(rbmd_ctx *ctx, int64_t step, int64_t *acc);
void rbmd_rho_acc_add(int64_t *sum, const int64_t *part, int64_t n_modes);
rbmd_status rbmd_rbe_forces_rho(rbmd_ctx *ctx, int64_t step, const int64_t *acc, void *force,
                                int accumulate);
rbmd_status rbmd_rbl_forces_slab(rbmd_ctx *ctx, int64_t step, void *force, int accumulate,
                                 double *fsum);
rbmd_status rbmd_add_correction(rbmd_ctx *ctx, void *force, const double *fsum_total);

/* Device error word injection for failure-path tests: sets the latched error to
 * `code` exactly as a kernel would. */
rbmd_status rbmd_debug_latch_error(rbmd_ctx *ctx, int32_t code);

#ifdef __cplusplus
}
#endif

#endif /* RBMD_H */
