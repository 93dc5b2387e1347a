/*
 * rbsog.h -- C ABI of the GB300 (sm_103a) RBSOG + RBL force evaluation and MD
 * step for Born-Mayer-Huggins (BMH) ionic systems.
 *
 * Method: arXiv 2512.24970, Sec. 2 ("Method").  The Coulomb kernel is split by
 * the sum-of-Gaussians u-series (Sec. 2.1, Eqs. (1r), (far), (short), C^1 cutoff
 * at r_c = r_shell); the short-range residual plus the BMH repulsion and
 * dispersion (Eq. (BMH), Eq. (Fshort)) are summed over the random batch list
 * (Sec. 2.2: exact core r < r_core, P_R sampled shell neighbours weighted
 * N_shell/P_R, momentum correction F^corr); the long-range part is the RBSOG
 * estimator (Eq. (long-rangeforce)) over P_F k-vectors drawn from
 * P(k) = k^2 Fhat(k)/S (Eq. (Pk)) with structure factors rho(k) (Sec. 2.1).
 * The step integrates the underdamped Langevin equation of Sec. 2.3 (BAOAB)
 * or NVE velocity Verlet.
 *
 * Units: metal -- Angstrom, eV, ps, amu, elementary charge.  Coulomb terms
 * carry k_e = 14.3996454784 eV*Angstrom.
 *
 * Conventions for every entry point:
 *   - Return 0 on success or a negative RBSOG_E_* code; rbsog_last_error()
 *     gives a one-line message.  No call traps or aborts.
 *   - Pointer arguments are host or device memory as ptr_kind says
 *     (RBSOG_PTR_HOST / RBSOG_PTR_DEVICE, device = the context's device).
 *   - The caller owns every buffer it passes; the library copies inputs and
 *     keeps no caller pointer after a call returns.
 *   - Atom order at the ABI is the caller's order.  Per-atom arrays are AoS
 *     [n][3] FP64 unless stated.
 *   - Work runs on a library stream ordered after, and before, the stream
 *     given to rbsog_create (events both ways); host-pointer outputs are
 *     complete when the call returns, device-pointer outputs are ordered on
 *     the caller's stream.
 *   - Errors raised inside kernels (capacity overflow) are latched in a device
 *     error word and reported by rbsog_sync() or the next synchronising call.
 *   - Only the device given to rbsog_create is used; there is no CPU path.
 */
#ifndef RBSOG_H
#define RBSOG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define RBSOG_OK 0
#define RBSOG_E_INVAL (-1)          /* bad argument or state */
#define RBSOG_E_NONNEUTRAL (-2)     /* |sum of charges| > 1e-10 (Sec. 2.1 assumes neutrality) */
#define RBSOG_E_BOX_TOO_SMALL (-3)  /* min L_d < 2 r_shell (minimum image) */
#define RBSOG_E_CAP_OVERFLOW (-4)   /* a fixed capacity (core list, per-cell shell count) overflowed */
#define RBSOG_E_CUDA (-5)           /* CUDA runtime error */
#define RBSOG_E_TIMEOUT (-6)        /* bounded device wait expired */
#define RBSOG_E_NO_SOG_ROOT (-7)    /* no s with N'(r_c) = 0 in [r_c/6, r_c/2] */
#define RBSOG_E_NO_SYSTEM (-8)      /* call needs rbsog_set_system first */
#define RBSOG_E_SKIN (-9)           /* kept lists: an atom moved by more than skin/2 since the
                                       lists were built (that step and later ones are invalid) */

/* ---- enums ---------------------------------------------------------------- */
#define RBSOG_FP64 0   /* analytic FP64 pair terms (M+1 Gaussians), FP64 sincospi and sums */
#define RBSOG_MIXED 1  /* FP32 pair math (tabulated SOG residual), exact integer phases,
                          FP32 minimax sin/cos polynomials after an exact half-turn
                          reduction, FP64 structure-factor / energy / position sums */

#define RBSOG_NVE_VV 0          /* velocity Verlet */
#define RBSOG_LANGEVIN_BAOAB 1  /* BAOAB splitting of the Langevin SDE of Sec. 2.3 */
#define RBSOG_NOSE_HOOVER 2     /* Nose-Hoover chain NVT, the thermostat of the runs of Sec. 3:
                                   a half step of the chain (Martyna-Tuckerman-Klein splitting,
                                   masses Q_0 = (3N-3) kT tdamp^2, Q_j = kT tdamp^2) before the
                                   first and after the second half kick of velocity Verlet */

#define RBSOG_LISTS_AUTO (-1)  /* list_every: rebuild kept lists when an atom moved by skin/2 */

#define RBSOG_PTR_HOST 0
#define RBSOG_PTR_DEVICE 1

/* Capacities of the device path (exceeding one sets RBSOG_E_CAP_OVERFLOW). */
#define RBSOG_MAX_SPECIES 8
#define RBSOG_MAX_PR 64        /* shell batch size P_R */
#define RBSOG_MAX_CORE 64      /* core neighbours per atom */
#define RBSOG_MAX_ROW_SLOTS 128 /* candidate slots of one stencil row: the x-cells a run of
                                   8 sorted atoms needs, each cell padded to a multiple of 4
                                   (also: a run of 8 atoms spans at most 4 cells along x) */
#define RBSOG_MAX_SHELL 1024   /* shell neighbours of one atom when the batch is sampled */
#define RBSOG_MAX_KEPT 512     /* kept lists: members of B (r_core <= r < r_shell + skin) per atom */
#define RBSOG_MAX_M 128        /* Gaussians m = 0..M */
#define RBSOG_MAX_NH_CHAIN 8   /* Nose-Hoover chain length */

typedef struct rbsog_ctx rbsog_ctx; /* opaque, library-owned */

/* Method parameters (Sec. 2.1-2.3).  r_shell is both the RBL shell radius and
 * the SOG cutoff r_c; BMH terms are truncated (unshifted) at r_shell. */
typedef struct {
  double b;        /* SOG base b > 1 (Eq. (1-r)) */
  int32_t M;       /* Gaussians m = 0..M of Eq. (far) */
  double s;        /* SOG bandwidth; s <= 0 or w0 <= 0: solve (s, w0) for C^1 at r_shell */
  double w0;       /* modified narrowest weight (value continuity at r_c) */
  double r_core;   /* RBL core radius (Sec. 2.2) */
  double r_shell;  /* RBL shell radius = SOG cutoff */
  int32_t P_R;     /* shell batch size, 1..RBSOG_MAX_PR */
  int32_t P_F;     /* Fourier batch size >= 1 */
  uint64_t seed;   /* key of every Philox4x32-10 draw */
  int32_t precision;   /* RBSOG_FP64 | RBSOG_MIXED */
  int32_t integrator;  /* RBSOG_NVE_VV | RBSOG_LANGEVIN_BAOAB */
  double dt;       /* time step [ps] */
  double T;        /* Langevin temperature [K] */
  double gamma;    /* Langevin collision rate gamma/m [1/ps], same for all species */
  /* Random batch lists (Sec. 2.2).  list_every = 0: core and shell are found
   * from the current positions at every evaluation.  list_every = n >= 1:
   * kept lists, as with the paper's skin neighbour lists (Sec. 3): built from
   * the positions of the first evaluation after set_system / set_state and of
   * every step that is a multiple of n (RBSOG_LISTS_AUTO: of every step where
   * some atom has moved by more than skin/2 since the last build, checked on
   * the device every step), with the outer radius
   * r_list = r_shell + skin; A = {r < r_core}, B = {r_core <= r < r_list} at
   * those positions.  Each evaluation sums A exactly and a Floyd batch of P_R
   * of B with weight |B| / P_R; every term carries the indicator
   * r < r_shell at the current positions, so the estimator stays unbiased for
   * the r_shell-cutoff force while no atom moves by skin/2 between builds
   * (checked every step: RBSOG_E_SKIN with a fixed n).  Needs every box
   * length >= 2 r_list. */
  int32_t list_every;
  double skin;     /* [A], >= 0; used when list_every != 0 */
  double tdamp;    /* Nose-Hoover time constant [ps] > 0 (RBSOG_NOSE_HOOVER) */
  int32_t nh_chain;  /* Nose-Hoover chain length, 1..RBSOG_MAX_NH_CHAIN (RBSOG_NOSE_HOOVER) */
} rbsog_params;

/* Create a context on CUDA device `cuda_device`.  `cuda_stream` is the
 * caller's cudaStream_t: if non-NULL the library's kernels and its captured
 * step graph run on it directly; if NULL the library creates its own
 * non-blocking stream and orders it after, and before, the legacy default
 * stream with events.  Errors: RBSOG_E_INVAL, RBSOG_E_CUDA. */
int rbsog_create(rbsog_ctx **out, int cuda_device, void *cuda_stream);

/* Destroy a context and free its device memory (NULL is ignored). */
void rbsog_destroy(rbsog_ctx *ctx);

/* Define the system (Sec. 2.1: N charges in a cuboid periodic box, neutral).
 *   n        atoms, >= 2
 *   pos      [n][3] FP64 positions (any image; wrapped internally)
 *   species  [n] int32 in [0, n_species)
 *   charge   [n_species] FP64 charges [e]; sum over atoms must vanish
 *   mass     [n_species] FP64 masses [amu]
 *   bmh      [n_species][n_species][5] FP64 = (A [eV], sigma [A], rho [A],
 *            C [eV A^6], D [eV A^8]) of Eq. (BMH); must be symmetric
 *   box      [3] FP64 box lengths, each >= 2 r_shell
 *   params   method parameters (host pointer always)
 * Resets velocities to zero and the step counter to 0; forces are evaluated
 * on the first compute/step.  All arrays are copied.
 * Errors: RBSOG_E_INVAL, RBSOG_E_NONNEUTRAL, RBSOG_E_BOX_TOO_SMALL,
 * RBSOG_E_NO_SOG_ROOT, RBSOG_E_CUDA. */
int rbsog_set_system(rbsog_ctx *ctx, int64_t n, const double *pos, const int32_t *species,
                     int32_t n_species, const double *charge, const double *mass,
                     const double *bmh, const double box[3], const rbsog_params *params,
                     int ptr_kind);

/* Species-dependent core radii (the adaptive, species-dependent cutoff of
 * Sec. 1, whose rule the paper does not print): r_core_pair [n_species]
 * [n_species] FP64 [A], symmetric, each in (0, r_core]; the pair (i, j) is in
 * the exact core iff r_ij < r_core_pair[s_i][s_j] (FP32 predicate), else in
 * the shell up to r_shell.  Any split leaves the estimator unbiased; only its
 * variance and cost change.  NULL restores the single r_core.  Host pointer;
 * lists are rebuilt at the next evaluation.  Errors: RBSOG_E_INVAL. */
int rbsog_set_core_radii(rbsog_ctx *ctx, const double *r_core_pair);

/* Set velocities [n][3] FP64 [A/ps]. */
int rbsog_set_velocities(rbsog_ctx *ctx, const double *vel, int ptr_kind);

/* One IRBSOG force evaluation at the current state and step counter s
 * (Sec. 2.2: F* = F_core + F*_shell - F^corr + F*_F; shell batch and k-batch
 * drawn with RNG step index s).  Outputs (each may be NULL):
 *   forces [n][3] FP64 [eV/A]
 *   energy [4] FP64 [eV] = (U_N, U_F*, U_F^self, U_N + U_F* - U_F^self), the
 *          sampled estimators of Eqs. (short2), (UF): U_N = 1/2 sum_i
 *          (sum_core e_ij + N_shell/P_R sum_B e_ij), U_F* = k_e S/(2 V P_F)
 *          sum_p |rho_p|^2/|k_p|^2, U_self = k_e/2 sum_i q_i^2 sum_m w_m
 *   virial [6] FP64 [eV] = (W_xx, W_yy, W_zz, W_xy, W_xz, W_yz), minus the
 *          derivative of U_N + U_F* under a homogeneous strain of positions
 *          and box, with the same samples: W_N = 1/2 sum_i (sum_core
 *          r_ij (x) f_ij + N_shell/P_R sum_B r_ij (x) f_ij) and W_F* =
 *          delta U_F* + (k_e/V) sum_p c_p (Fhat'/Fhat)(|k_p|^2) k_p (x) k_p
 *          |rho_p|^2; F^corr, not a pair force, has none.  The pressure is
 *          (2 E_kin + tr W) / (3V).
 * Synchronous for host outputs.  Errors: RBSOG_E_NO_SYSTEM, RBSOG_E_INVAL,
 * RBSOG_E_CAP_OVERFLOW, RBSOG_E_CUDA. */
int rbsog_compute_forces(rbsog_ctx *ctx, double *forces, double *energy, double *virial,
                         int ptr_kind);

/* Advance nsteps MD steps (asynchronous on the caller's stream).  Step
 * s -> s+1: half kick, drift (BAOAB: half drift, Ornstein-Uhlenbeck with
 * Philox noise of step index s+1, half drift), force evaluation with RNG step
 * index s+1, half kick.  One step is captured once as a CUDA graph and
 * replayed.  Errors: RBSOG_E_NO_SYSTEM, RBSOG_E_CUDA. */
int rbsog_step(rbsog_ctx *ctx, int64_t nsteps);

/* Kinetic tensor of the current velocities, K [6] FP64 [eV] = (K_xx, K_yy,
 * K_zz, K_xy, K_xz, K_yz), K_ab = sum_i m_i v_ia v_ib (the order of the
 * virial), summed on the device in a fixed order (block sums, then the blocks
 * in order).  With the virial W of rbsog_compute_forces it gives the stress
 * tensor S = K + W; S_xy is the shear stress of the Green-Kubo viscosity of
 * Sec. 3 (sum_i m_i v_xi v_yi plus the pair term 1/2 sum_{j != i} x_ij f_y,
 * here with the far field's strain derivative as well), and tr K = 2 E_kin.
 * ptr_kind: host (synchronous) or device (asynchronous on the caller's
 * stream).  Errors: RBSOG_E_NO_SYSTEM, RBSOG_E_INVAL, RBSOG_E_CUDA. */
int rbsog_get_kinetic_tensor(rbsog_ctx *ctx, double *K, int ptr_kind);

/* Read the state: pos/vel [n][3] FP64 (each may be NULL), step counter. */
int rbsog_get_state(rbsog_ctx *ctx, double *pos, double *vel, int64_t *step, int ptr_kind);

/* Overwrite the state (pos/vel may be NULL to keep them); forces are
 * re-evaluated at the new state before the next step.  Because every draw
 * depends only on (seed, step, index), save + restore + run(n) reproduces
 * run(2n) bit for bit; with kept lists the lists depend on the positions of
 * their last build too, so a restore passes those on as well
 * (rbsog_get_list_origin / rbsog_set_list_origin), else the restored run
 * builds its lists at the restored positions (an equally valid sample path,
 * not the same one). */
int rbsog_set_state(rbsog_ctx *ctx, const double *pos, const double *vel, int64_t step,
                    int ptr_kind);

/* Move the atoms to pos [n][3] FP64 [A] and set the step counter, keeping
 * velocities and the kept lists: for a caller that integrates on its side
 * and evaluates forces here every step.  As between two steps, the next
 * evaluation reuses the lists of the last build unless some atom is more than
 * skin/2 from its build position (automatic mode: rebuilt on the device;
 * fixed schedule: RBSOG_E_SKIN, as the lists are rebuilt only by steps at
 * multiples of list_every).  With per-step lists the same as rbsog_set_state
 * with vel = NULL.  ptr_kind: host (synchronous) or device.  Errors:
 * RBSOG_E_NO_SYSTEM, RBSOG_E_INVAL, RBSOG_E_CUDA. */
int rbsog_move_atoms(rbsog_ctx *ctx, const double *pos, int64_t step, int ptr_kind);

/* Forces at given positions in one call: rbsog_move_atoms(pos, step) followed
 * by the force-only rbsog_compute_forces(forces), with the same results bit
 * for bit (Eqs. (Fshort), (long-rangeforce) and F^corr of Sec. 2.2, drawn
 * with RNG step index step).  For a caller that integrates on its side (an
 * external MD engine) and hands over positions and reads forces every step:
 * the positions' copy, the layout conversions, the evaluation graph and the
 * forces' copy are enqueued together and the host waits once.
 *   pos    [n][3] FP64 [A], caller order (read)
 *   forces [n][3] FP64 [eV/A] (written)
 * ptr_kind: host (both pointers host memory; synchronous: both buffers may be
 * reused on return) or device (both device memory of the context's device;
 * asynchronous on the caller's stream, pos read and forces written in stream
 * order).  Errors: RBSOG_E_NO_SYSTEM, RBSOG_E_INVAL (null pointer, step < 0,
 * unknown ptr_kind), RBSOG_E_SKIN and RBSOG_E_CAP_OVERFLOW (host pointers; with
 * device pointers they are reported by the next synchronizing call, e.g.
 * rbsog_sync), RBSOG_E_CUDA. */
int rbsog_forces_at(rbsog_ctx *ctx, const double *pos, int64_t step, double *forces, int ptr_kind);

/* Kept lists (list_every != 0): the positions [n][3] FP64 [A] of the last
 * build of the lists the next evaluation uses, caller order.  Errors:
 * RBSOG_E_INVAL without kept lists or before the first evaluation. */
int rbsog_get_list_origin(rbsog_ctx *ctx, double *pos_b, int ptr_kind);

/* Kept lists: the next evaluation builds its lists from the positions pos_b
 * (binned, listed and recorded as the build positions exactly as a build at
 * pos_b would be) and evaluates at the current positions.  Call after
 * rbsog_set_state (which lets lists be rebuilt at the restored positions);
 * with the saved state it resumes a run bit for bit.  The caller keeps the
 * build within skin/2 of the current positions, as a run does (a fixed
 * schedule reports RBSOG_E_SKIN otherwise, the automatic one rebuilds).
 * Errors: RBSOG_E_INVAL without kept lists, RBSOG_E_CUDA. */
int rbsog_set_list_origin(rbsog_ctx *ctx, const double *pos_b, int ptr_kind);

/* Builds of the kept random batch lists since rbsog_set_system (waits for the
 * context's work).  Host pointer. */
int rbsog_get_list_builds(rbsog_ctx *ctx, int64_t *builds);

/* Nose-Hoover chain state between steps (RBSOG_NOSE_HOOVER): eta[nh_chain]
 * and its velocities v_eta[nh_chain] [1/ps].  Host pointers; get waits for
 * the context's work.  set_system starts the chain at rest; together with
 * rbsog_get_state / rbsog_set_state these make a run resumable bit for bit.
 * Errors: RBSOG_E_INVAL (another integrator), RBSOG_E_CUDA. */
int rbsog_get_thermostat(rbsog_ctx *ctx, double *eta, double *v_eta);
int rbsog_set_thermostat(rbsog_ctx *ctx, const double *eta, const double *v_eta);

/* Wait for the context's work; return the latched device error, if any. */
int rbsog_sync(rbsog_ctx *ctx);

/* SOG parameters in use: s, w[0..M] (w[0] modified), S = sum_{k!=0} k^2 Fhat(k). */
int rbsog_get_sog(rbsog_ctx *ctx, double *s, double *w, double *S);

/* ---- kernel schedule -------------------------------------------------------- */

/* Launch shapes of the mixed-precision far field (Sec. 2.2: the structure
 * factors rho(k_p) over all atoms and the force of Eq. (long-rangeforce),
 * O(N P_F) work each, Sec. 2.4) and of the near field beside it.  They split that work over the GPU and
 * change nothing but the order in which FP32 and FP64 partial sums are added;
 * paper_2512_24970_gb300/autotune.py picks them by timing.  Defaults (0, 2, 2, 4, 1, 0, 0, 0, 0). */
typedef struct {
  int32_t rho_variant;           /* structure factor block shape: 0 = two groups of 256 threads,
                                    one pair of modes per thread; 1 = one group of 256; 2 = two
                                    groups of 128 threads, two pairs each; 3 = four such groups;
                                    4..7 = 0..3 in scalar FP32 instead of packed FP32x2; 8, 9 =
                                    0, 1 with the cosine packed too */
  int32_t rho_blocks_per_sm;     /* structure factor: tiles of atoms per SM the tiling aims at, 1..8 */
  int32_t far_atoms_per_thread;  /* far force: atoms per thread, 1, 2 or 4 */
  int32_t far_segments;          /* far force: k segments per block of 8 warps, 1, 2, 4 or 8 */
  int32_t far_packed;            /* far force: 1 = two modes per packed FP32x2 instruction, 0 = scalar,
                                    2 = packed and the sums kept in packed lanes too */
  int32_t near_blocks_per_sm;    /* near field with kept lists: 0 = one block per 32 slots; k = 1..16:
                                    k blocks per SM loop over the slots, so that the far field's
                                    kernels, which run beside it, always find free SM slots */
  int32_t rho_tile_atoms;        /* structure factor: 0 = tiles from rho_blocks_per_sm; 32..65536 =
                                    that many atoms per tile (tiles in proportion to N, e.g. for the
                                    replicas of a packed ensemble) */
  int32_t near_wide;             /* near field with kept lists: 1 = a thread gathers its first 8 members
                                    of A and its first batch members at once (more loads in flight, more
                                    registers); 0 = in rounds of 4 and 5 (same sums bit for bit) */
  int32_t rho_reduce;            /* sum of the structure factor's tile partials: 0 = a warp per mode up
                                    to 160 tiles, else a block per mode; 1 = always a block per mode;
                                    2 = always a warp per mode (8 modes per block: fewer blocks to
                                    schedule beside the near field) */
} rbsog_schedule;

/* Set the schedule (host pointer).  Takes effect at the next evaluation (the
 * step graph is captured again).  Errors: RBSOG_E_INVAL (a value out of
 * range), RBSOG_E_CUDA. */
int rbsog_set_schedule(rbsog_ctx *ctx, const rbsog_schedule *sched);

/* The schedule in use (host pointer). */
int rbsog_get_schedule(rbsog_ctx *ctx, rbsog_schedule *sched);

/* ---- allocation-free entry point -------------------------------------------- */

#define RBSOG_SF_STATIC_PMAX 1024  /* largest P of rbsog_structure_factor_static */

/* Structure factors rho(k_p) = sum_j q_j exp(i k_p . r_j), k_p = 2 pi m_p / L,
 * of the context's current positions for P caller modes, with the same exact integer phase m.u mod 2^32 and FP64
 * sincos as the FP64 force path.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory, e.g. an
 * analysis hook that samples S(k) = |rho(k)|^2 / N between MD steps while
 * other work is in flight (cudaFree synchronises the whole device, and a
 * caching allocator may already hold all free memory).  It allocates
 * nothing: its scratch is a static 2 MiB device array of RBSOG_SF_STATIC_PMAX x
 * 128 tile partials, whose device address is looked up once per device, on that
 * device's first call (make that first call outside stream capture).  Like
 * every context, the cached address does not survive a cudaDeviceReset of the
 * device: do not use the library across one.  Nothing in the scratch
 * has to start at zero (every partial read is written in the same call).
 *   m   [P][3] int32, DEVICE pointer (mode indices m_x, m_y, m_z)
 *   rho [P][2] FP64, DEVICE pointer (Re, Im), written
 * Asynchronous on the context's stream.  The scratch is shared by every
 * context of a device, so two calls that overlap in time (two contexts or
 * streams of one device, or host threads) race on it: serialise them.
 * Errors: RBSOG_E_INVAL (P < 0, P > RBSOG_SF_STATIC_PMAX, null pointer, or a
 * pointer that is not memory of the context's device), RBSOG_E_NO_SYSTEM,
 * RBSOG_E_CUDA.  P = 0 does nothing. */
int rbsog_structure_factor_static(rbsog_ctx *ctx, int32_t P, const int32_t *m, double *rho);

/* ---- parity hooks (test use) ---------------------------------------------- */

/* Lists and shell batch of atoms sel[0..nsel) at the current state and step
 * counter, computed by the device list kernel that shares the hot path's
 * predicate and canonical order: core/shell rows of width cap_core/cap_shell
 * hold caller atom indices in canonical order (ascending (cell index of j,
 * fixed-point x coordinate u_x of j, j)), batch rows of width P_R the sampled shell neighbours in the same order,
 * weight = N_shell/P_R (1 if the whole shell is taken).  Host pointers. */
int rbsog_debug_get_lists(rbsog_ctx *ctx, const int64_t *sel, int64_t nsel, int32_t cap_core,
                          int32_t cap_shell, int32_t *core, int32_t *ncore, int32_t *shell,
                          int32_t *nshell, int32_t *batch, int32_t *nbatch, double *weight);

/* Kept lists (list_every >= 1) of atoms sel[0..nsel) as last built, and the
 * shell batch the current step counter draws from them: A rows (width
 * cap_a) and B rows (width cap_b) hold caller atom indices in the canonical
 * order of the build positions (ascending (cell index of j on the r_list/2
 * grid, u_x of j, j)); batch rows of width P_R hold the sampled members of B
 * (all of B, weight 1, if |B| <= P_R), weight = |B| / P_R.  Needs a force
 * evaluation since the lists were last invalidated.  Host pointers.
 * Errors: RBSOG_E_INVAL (per-step lists in use, bad arguments). */
int rbsog_debug_get_kept_lists(rbsog_ctx *ctx, const int64_t *sel, int64_t nsel, int32_t cap_a,
                               int32_t cap_b, int32_t *A, int32_t *nA, int32_t *B, int32_t *nB,
                               int32_t *batch, int32_t *nbatch, double *weight);

/* Kept lists: the shell batch the last force evaluation's pair sums read
 * (drawn by the batch kernel from B, Sec. 2.2 F*_shell), batch [nsel][P_R]
 * caller ids in draw order; rows of atoms that took all of B stay -1.
 * Compare with rbsog_debug_get_kept_lists at the same step.  Host pointers. */
int rbsog_debug_get_kept_batch_used(rbsog_ctx *ctx, const int64_t *sel, int64_t nsel, int32_t *batch);

/* Kept lists store B also as 16-bit slot offsets (modulo the slot count),
 * which the batch kernel reads when every offset of the last build fits.
 * force_wide != 0 makes it read the 32-bit rows always (same batch);
 * *fits (may be NULL) = 1 when the last build's offsets all fit 16 bits. */
int rbsog_debug_kept_b16(rbsog_ctx *ctx, int force_wide, int32_t *fits);

/* k-batch of the last force evaluation: m [P][3] int32, c [P] FP64 with
 * c_p = S/(P_F |k_p|^2) (or the weights set below).  Host pointers. */
int rbsog_debug_get_kbatch(rbsog_ctx *ctx, int32_t *m, double *c);

/* Replace the sampled k-batch by a fixed list of P modes m [P][3] with
 * weights c [P] (c_p = Fhat(k_p) over all k gives Eq. (Long)); P = 0 restores
 * sampling.  Host pointers. */
int rbsog_debug_set_kbatch(rbsog_ctx *ctx, int32_t P, const int32_t *m, const double *c);

/* Parts of the last force evaluation: uncorrected near field F_core +
 * F*_shell [n][3], far field F*_F [n][3], F^corr [3], structure factors
 * rho [P][2].  Host pointers, each may be NULL. */
int rbsog_debug_get_parts(rbsog_ctx *ctx, double *near, double *far, double *fcorr,
                          double *rho);

/* FP32 phase factors of the mixed-precision far field: s[i], c[i] = sin, cos
 * of 2 pi th[i] / 2^32 evaluated by the device routine the structure-factor
 * and far-force kernels use.  Host pointers; needs a context for its device. */
int rbsog_debug_sincos(rbsog_ctx *ctx, int64_t n, const uint32_t *th, float *s, float *c);

/* Take the whole shell with weight 1 for every atom (flag != 0), i.e. the
 * deterministic r_shell-cutoff near field; 0 restores the P_R batch. */
int rbsog_debug_set_whole_shell(rbsog_ctx *ctx, int flag);

/* ---- measurement ----------------------------------------------------------- */

/* Stages timed by the profiling events.  The structure factor runs on a side
 * stream concurrently with binning and the near field, so stage times do not
 * add up to the total, which is reported last. */
#define RBSOG_NSTAGE 9  /* integrator + fixed point + histograms; bin (row scan, cell
                           prefix, scatter, rank); near field; far-field branch on the
                           side stream (k-batch, structure factor, its reduction, far
                           force); F^corr; total force + closing kick; total; inside the
                           far-field branch: the structure-factor kernel alone, the
                           far-force kernel alone */

/* Record a CUDA event between consecutive stages of every force evaluation
 * (also inside the captured step graph, as event nodes) when on != 0. */
int rbsog_set_profiling(rbsog_ctx *ctx, int on);

/* Durations [ms] of the RBSOG_NSTAGE stages of the most recent force
 * evaluation (waits for it).  Requires profiling on.  Host pointer. */
int rbsog_get_stage_times(rbsog_ctx *ctx, float *ms, int32_t nstage);

#define RBSOG_NMARK 12  /* main stream: start, after the integrator, after binning, after the
                           near field, after F^corr, after the join of the branches, end;
                           side stream: branch start, structure factor start (after the
                           k-batch and the integrator), structure factor end, its
                           reduction end, far-field force end */

/* Times [ms] of the RBSOG_NMARK stage marks of the most recent force
 * evaluation, from its start (waits for it): the timeline behind the stage
 * durations, both branches on one clock.  Requires profiling on.  Host
 * pointer; the first min(nmark, RBSOG_NMARK) entries are written. */
int rbsog_get_stage_marks(rbsog_ctx *ctx, float *ms, int32_t nmark);

/* Throughput of one arithmetic pipe of `cuda_device`, measured: every thread
 * of 4 blocks of 512 per SM runs 8 independent multiply-add chains (FP32 fma,
 * packed FP32x2 fma, FP64 fma or 32-bit integer multiply-add, as `kind`
 * says); one warm-up launch, then one launch timed with CUDA events.
 * *ops_per_s = lane multiply-adds per second (an FP32x2 instruction counts
 * two).  These are the denominators of the rooflines the benchmark reports
 * (Sec. 2.4 gives the method's cost as operation counts).  Host pointer;
 * allocates and frees a small buffer.  Errors: RBSOG_E_INVAL, RBSOG_E_CUDA. */
#define RBSOG_PROBE_FP32 0
#define RBSOG_PROBE_FP32X2 1
#define RBSOG_PROBE_FP64 2
#define RBSOG_PROBE_IMAD 3
int rbsog_probe_peak(int cuda_device, int kind, double *ops_per_s);

/* Message of the last error of this context (never NULL). */
const char *rbsog_last_error(const rbsog_ctx *ctx);

/* ---- ensemble of independent replicas ---------------------------------------- */

/* Many independent systems of uneven size on one GPU (e.g. a screen over
 * compositions and temperatures).  Each replica is a full context (its own
 * system, parameters, RNG key, step counter and step graph) running on its own
 * non-blocking stream pair, so the replicas' steps overlap on the device; the
 * calls below order that work after, and before, the ensemble's stream with
 * events.  Results per replica are bit-identical to stepping it alone. */
typedef struct rbsog_ensemble rbsog_ensemble; /* opaque, library-owned */

/* Create an empty ensemble on CUDA device `cuda_device` for at most
 * max_replicas replicas.  `cuda_stream` as in rbsog_create (NULL: the legacy
 * stream).  Errors: RBSOG_E_INVAL, RBSOG_E_CUDA. */
int rbsog_ensemble_create(rbsog_ensemble **out, int cuda_device, void *cuda_stream,
                          int32_t max_replicas);

/* Destroy the ensemble and all its replicas (waits for their work). */
void rbsog_ensemble_destroy(rbsog_ensemble *ens);

/* Add a replica: arguments exactly as rbsog_set_system.  *replica receives its
 * index (0, 1, ...).  Errors: those of rbsog_set_system, RBSOG_E_INVAL when
 * the ensemble is full. */
int rbsog_ensemble_add(rbsog_ensemble *ens, int64_t n, const double *pos, const int32_t *species,
                       int32_t n_species, const double *charge, const double *mass,
                       const double *bmh, const double box[3], const rbsog_params *params,
                       int ptr_kind, int32_t *replica);

/* The context of replica r (owned by the ensemble): every rbsog_* call on a
 * context applies to it (velocities, state, forces, parity hooks).  NULL for
 * a bad index. */
rbsog_ctx *rbsog_ensemble_replica(rbsog_ensemble *ens, int32_t r);

/* Advance every replica nsteps MD steps (rbsog_step of each replica, all on
 * their own streams, joined into the ensemble's stream; asynchronous).
 * Errors: RBSOG_E_INVAL, the first failing replica's code. */
int rbsog_ensemble_step(rbsog_ensemble *ens, int64_t nsteps);

/* Wait for all replicas; return the first latched device error, if any. */
int rbsog_ensemble_sync(rbsog_ensemble *ens);

/* How rbsog_ensemble_step runs the replicas (each replica's estimator needs
 * only its own state, Sec. 2.2, so they are independent problems):
 *   RBSOG_ENSEMBLE_PACKED (default): every stage of the step is one kernel
 *     launch over the blocks of all replicas, in one CUDA graph per ensemble
 *     step, when the replicas are all mixed precision, share the integrator
 *     (velocity Verlet or BAOAB), the list mode (per-step lists or kept lists
 *     rebuilt when needed) and the far-field schedule, and none is profiling;
 *     otherwise the step falls back to
 *   RBSOG_ENSEMBLE_GRAPHS: one CUDA graph whose child nodes are the replicas'
 *     own step graphs (replicas on a fixed list schedule: each launches its
 *     own graphs).
 * Results per replica are bit-identical either way.  Errors: RBSOG_E_INVAL. */
#define RBSOG_ENSEMBLE_PACKED 0
#define RBSOG_ENSEMBLE_GRAPHS 1
int rbsog_ensemble_set_mode(rbsog_ensemble *ens, int32_t mode);

/* Packed mode: deal the replicas into `groups` groups of about equal atoms;
 * each group's stages are packed launches, and the groups run as parallel
 * branches of the step graph, so that one group's reductions overlap another's
 * arithmetic (1 = every replica in one group, the default; more than the
 * number of replicas = one replica per group).  The tuner of
 * paper_2512_24970_gb300/autotune.py picks it by timing.  Errors: RBSOG_E_INVAL. */
int rbsog_ensemble_set_groups(rbsog_ensemble *ens, int32_t groups);

/* The way the last rbsog_ensemble_step ran (RBSOG_ENSEMBLE_PACKED or
 * RBSOG_ENSEMBLE_GRAPHS; -1 before the first step).  Host pointer. */
int rbsog_ensemble_get_mode(rbsog_ensemble *ens, int32_t *used);

/* Message of the last error of the ensemble (never NULL). */
const char *rbsog_ensemble_last_error(const rbsog_ensemble *ens);

#ifdef __cplusplus
}
#endif
#endif /* RBSOG_H */
