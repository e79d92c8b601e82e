/*
 * nb.h — C ABI of the B300 hybrid symplectic N-body library (libnb.so).
 *
 * The library integrates a planetary system with the hybrid symplectic
 * method of Grimm & Stadel ("Terrestrial planet formation in the era of GPU
 * computing", section "The hybrid symplectic integrator"):
 *   H = H_A + H_B + H_C                                            (Eq. H)
 *   H_A  Kepler motion about the star + the (1 - K) close part     (Eq. Ha)
 *   H_B  mutual interaction weighted by the changeover K(r_ij)     (Eq. Hb)
 *   H_C  |sum p|^2 / (2 m0), the momentum term of mixed variables  (Eq. Hc)
 *   r_crit,i = max(3 R_Hill,i, 0.4 dt v_i)                         (Eq. rcrit)
 * One step is B(h/2) C(h/2) A(h) C(h/2) B(h/2); A is the Kepler drift of
 * every body, replaced by a Bulirsch-Stoer integration of H_A for bodies in
 * a close-encounter group (the "direct solver" of the same section), with
 * perfect merging on contact (section "Detailing the outcomes of collisions").
 *
 * Conventions
 *  - Units: AU, day, solar mass. The star is implicit (mass m0). Bodies carry
 *    heliocentric positions x and barycentric velocities v (democratic
 *    heliocentric coordinates), interleaved [n][3] in every argument.
 *  - All device memory is provided by the caller: the library never calls
 *    cudaMalloc or cudaFree. nb_workspace_bytes() sizes the workspace.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy stream.
 *  - Functions return NB_OK (0) or a negative NB_E_* code; they never throw.
 *    nb_last_error() gives a message for the last failure on a handle.
 *  - Body order is the caller's order; ids must be strictly increasing, so
 *    index order and id order agree. A merger keeps the lower id.
 *  - nb_step() is atomic: on any error the state is restored to what it was
 *    when the call started.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_OK 0
#define NB_E_INVALID (-1)   /* bad argument, NaN/Inf input, n < 1, ids not increasing */
#define NB_E_CUDA (-2)      /* a CUDA runtime call failed */
#define NB_E_OVERFLOW (-3)  /* flagged-pair or group buffer full; grow pair_capacity */
#define NB_E_NOCONV (-4)    /* Kepler or Bulirsch-Stoer iteration cap reached */
#define NB_E_TIMEOUT (-5)   /* a bounded device loop gave up */
#define NB_E_WORKSPACE (-6) /* workspace too small or not 256-byte aligned */

#define NB_PREC_FP64 0  /* kick pair terms in FP64 */
#define NB_PREC_MIXED 1 /* FP32 r^-3 seed, one FP64 Newton step, compensated sums */
#define NB_PREC_DS 2    /* FP64 relative coordinates; r^2, r^-3, products and sums in   \
                           double-single (float pairs) on the FP32 pipe; tile sums in FP64 */

typedef struct {
  double G;            /* gravitational constant; default k^2 = 2.959122082855911e-4 */
  double m0;           /* central mass; default 1 */
  double dt_rcrit;     /* time step in the velocity term of Eq. rcrit; default 6 days */
  double hill_factor;  /* Eq. rcrit, default 3 */
  double vel_factor;   /* Eq. rcrit, default 0.4 */
  int vel_mode;        /* 0: |v - v_circ(x)| (default); 1: |v| */
  int merge;           /* 1: perfect merging on contact (default) */
  int precision;       /* NB_PREC_FP64 (default), NB_PREC_MIXED or NB_PREC_DS */
  int kepler_max_iter; /* Kepler iteration cap, default 30 */
  double bs_tol;       /* Bulirsch-Stoer relative tolerance, default 1e-14 */
  int bs_kmax;         /* extrapolation columns (substeps 2k), default 8, at most 12 */
  int bs_max_halvings; /* default 20 */
  int pair_capacity;   /* flagged-pair buffer, pairs; 0 = max(4096, 4n) */
  int log_capacity;    /* encounter-log entries per nb_step call; 0 = 1<<20 */
  int kick_split;      /* j-chunks per i-tile in the kick; 0 = automatic */
  int rcrit_refresh;   /* cadence of Eq. rcrit. 0 (default): rc from the initial state, recomputed
                          only for a merged survivor, so one force evaluation per step serves the
                          step's end and the next step's start. 1: rc recomputed for every body
                          from its state at the start of every step, and the force and flags
                          re-evaluated with the new radii (two evaluations per step). Only
                          nb_init_system / nb_step take 1; the batch and adjoint entry points
                          reject it (NB_E_INVALID). */
  /* Gas drag (section "Modelling additional dynamical effects"), applied as
   * G(h/2) B(h/2) C(h/2) A(h) C(h/2) B(h/2) G(h/2), each G(tau) the implicit
   * midpoint update of Eq. implicit, v' = v + tau a_f(x, (v + v') / 2),
   * solved by fixed-point iteration to 1e-15 relative (NB_E_NOCONV after
   * gas_iter). Drag law (a reading; the paper names none): the quadratic law
   * a_f = -(C_D pi R^2 rho / (2 m)) |u| u, u the velocity relative to gas that
   * circles the star at (1 - eta) times the circular speed sqrt(G m0 / s) of
   * the cylindrical radius s, midplane density rho = rho0 (s / 1 AU)^-p.
   * Bodies with R = 0 feel no drag. Single-system path only (the batch and
   * adjoint entry points reject gas != 0). */
  int gas;             /* 1: gas drag on; default 0 */
  double gas_rho0;     /* Msun / AU^3; default 2.36e-3 (1.4e-9 g cm^-3) */
  double gas_p;        /* default 2.75 */
  double gas_eta;      /* default 2e-3 */
  double gas_cd;       /* default 1 */
  int gas_iter;        /* default 30 */
  /* Ejection: at the start of every step, bodies farther than eject_r (AU)
   * from the star are removed (their mass and the energy they carry away,
   * mutual and Eq. Hc terms included, are booked; the cached force is then
   * re-evaluated). 0 (default) = never. Single-system path only. */
  double eject_r;
  /* Groups of at least bs_cluster_min bodies are integrated by a cluster of
   * 8 CTAs (one thread per extrapolation column and member, the cluster's
   * hardware barrier between phases) instead of one CTA; same results bit
   * for bit. Default 64; 0 = one CTA for every group. */
  int bs_cluster_min;
  /* Multi-level changeover (section "Increasing N": the step is reduced level
   * by level for the bodies of a close encounter, each level with its own
   * changeover, the direct solver only at the last level). Level l has
   * critical radii r_crit ml_factor^-l and substeps tau / ml_factor; a group
   * of level l is integrated by ml_factor substeps of a kick with weight
   * w_(l+1) - w_l, the Kepler drift of its bodies and, for the pairs within
   * the level-(l+1) radii, groups of level l + 1; at l = ml_levels by the
   * direct solver with the radii of that level. 0 (default) = the direct
   * solver for every group; at most 3. With levels on, every group runs on
   * one CTA (bs_cluster_min does not apply). Single-system path only. */
  int ml_levels;
  int ml_factor;       /* default 3; 2..64 */
  /* Speculative half-size attempts in the direct solver: 1 (default) = a group
   * of up to 4 bodies run by one warp also integrates, in its spare lanes,
   * the half-size attempt that a failure of the current attempt would lead
   * to, and takes it on a failure; 0 = attempts one after the other. The
   * results, counters and adjoint records are the same bit for bit. */
  int bs_speculate;
  /* Unordered-pair kick (FP64 and double-single precision, unsharded
   * systems): each pair {i, j} is evaluated once and its term applied to both
   * bodies (Newton's third law); in FP64, 4.5 FP64 instructions per ordered
   * pair against 7 in the row kick.
   * 0 (default) = automatic: on for 4096 <= n <= 262144; 1 = on for any
   * n <= 262144 (nb_init_system returns NB_E_INVALID above); -1 = off (the
   * row kick). The mixed precision always runs the row kick. Results agree
   * with the row kick to rounding (the products and the order of the sums
   * differ), deterministic for a given n. A sharded system (nb_set_shard,
   * world > 1) runs the row kick whatever the setting; the shards equal the
   * one-GPU step with -1 bit for bit. Batches (nb_batch_*): 0 or 1 (default)
   * = the unordered-pair kick on 32-body block pairs of each system, -1 = the
   * row kick in tiles of the schedule's tile rows. */
  int kick_symmetric;
} nb_params;

typedef struct {
  long long steps;           /* integrator steps completed */
  long long force_evals;     /* full O(N^2) kick evaluations */
  long long encounter_pairs; /* sum over steps of |E| */
  long long groups;          /* close-encounter groups integrated */
  long long bs_substeps;     /* accepted BS substeps */
  long long bs_halvings;     /* BS substep halvings */
  long long bs_derivs;       /* BS right-hand-side evaluations */
  long long merges;          /* perfect mergers */
  long long kepler_iters;    /* Kepler iterations summed over bodies and steps */
  long long moved_bodies;    /* bodies re-integrated by BS (incremental force update) */
  long long log_dropped;     /* encounter-log entries that did not fit */
  int n_active;              /* bodies not absorbed by a merger or ejected */
  int last_pairs;            /* |F| of the last force evaluation */
  long long ejections;       /* bodies removed beyond eject_r */
  double m_ejected;          /* their mass */
  long long ml_substeps;     /* substeps on the intermediate changeover levels */
  long long ml_groups;       /* groups formed on the intermediate levels */
  int kick_symmetric;        /* 1 when the step's kicks evaluate each pair once (the
                                unordered-pair kick), 0 for the row kick */
} nb_stats_t;

typedef struct nb_system nb_system; /* opaque host handle (small, malloc'd by the library) */

/* Fill p with the defaults listed above. */
void nb_default_params(nb_params* p);

/* Bytes of device workspace that nb_init_system() needs for n bodies. */
size_t nb_workspace_bytes(const nb_params* p, int n);

/* Create a system in the caller's device workspace (>= nb_workspace_bytes,
 * 256-byte aligned) and evaluate the first kick and flags (the cached
 * "first same as last" force). x, v: [n][3]; m, R: [n]; rc_override: [n] or
 * NULL (then r_crit follows Eq. rcrit); ids: [n] strictly increasing or NULL
 * (then 0..n-1). The inputs are host pointers when inputs_on_device == 0,
 * device pointers otherwise; they are copied in and not retained. The
 * workspace must stay allocated until nb_destroy(). Returns NB_E_INVALID for
 * NaN/Inf, m <= 0, R < 0, rc <= 0 or ids not increasing. */
int nb_init_system(nb_system** out, const nb_params* p, int n, const double* x, const double* v,
                   const double* m, const double* R, const double* rc_override, const int* ids,
                   void* workspace, size_t ws_bytes, void* stream, int inputs_on_device);

/* Replace the cached force and flag set (resume a run bit-exactly): a is
 * [n][3] over all n slots, pairs_ij holds npairs (i, j) index pairs, i < j. */
int nb_set_fsal(nb_system* s, const double* a, const int* pairs_ij, int npairs, int on_device);

/* Load a complete state into an existing system of the same n (checkpoint
 * restore, or feeding a new batch into a resident workspace): x, v [n][3],
 * m, R, rc [n] (rc required), ids [n] or NULL, the cached force a [n][3] and
 * npairs flagged index pairs. No force is evaluated. Host pointers when
 * on_device == 0. Validation as in nb_init_system (NB_E_INVALID; the previous
 * state is then undefined and must be reloaded). */
int nb_set_state(nb_system* s, const double* x, const double* v, const double* m,
                 const double* R, const double* rc, const int* ids, const double* a,
                 const int* pairs_ij, int npairs, int on_device);

/* Event timing of the kick launches inside nb_step (off by default).
 * nb_timing() returns the summed kick time in ms and the number of timed kick
 * launches since timing was enabled, and the total number of kernels the
 * handle has launched. */
int nb_set_timing(nb_system* s, int enable);
int nb_timing(nb_system* s, double* kick_ms, long long* kick_launches, long long* launches);

/* Advance nsteps steps of size dt (dt may be negative). Synchronises the
 * stream before returning. The encounter log is cleared at entry. Without
 * split phases (rcrit_refresh, gas, ejection), row sharding or timing, the
 * steps replay two CUDA graphs captured at the first call with this dt (the
 * same kernels; results are identical to direct launches, which are used when
 * capture is unavailable). */
int nb_step(nb_system* s, int nsteps, double dt);

/* Total energy E = H_A + H_B + H_C (K cancels, Eqs. Ha-Hc), angular
 * momentum L = sum m x cross v, P = sum m v and the energy removed by
 * mergers. Host outputs; any pointer may be NULL. */
int nb_energy_momentum(nb_system* s, double* E, double L[3], double P[3], double* E_lost);

/* Active bodies in ascending id: x, v [k][3], m, R, rc [k], ids [k]. Any
 * pointer may be NULL. Outputs are device pointers when out_on_device != 0.
 * *n_active (host) receives k. */
int nb_get_state(nb_system* s, double* x, double* v, double* m, double* R, double* rc, int* ids,
                 int* n_active, int out_on_device);

/* Cached force of all n slots [n][3] and the cached flag set (index pairs).
 * *npairs (host) receives the pair count; at most cap pairs are written. */
int nb_get_fsal(nb_system* s, double* a, int* pairs_ij, int cap, int* npairs, int out_on_device);

/* Encounter pairs of the last nb_step() call as (step, id_i, id_j) triples,
 * id_i < id_j, sorted by step then ids (host output). *count receives the
 * total; if it exceeds cap, cap triples are written and NB_E_OVERFLOW is
 * returned. */
int nb_encounter_list(nb_system* s, int* step_ij, int cap, int* count);

int nb_stats(nb_system* s, nb_stats_t* out);
void nb_destroy(nb_system* s);
const char* nb_last_error(const nb_system* s);
const char* nb_status_string(int status);

/* ---------------------------------------------------------------------
 * Row sharding across ranks (section "Increasing N": large N is the point of
 * the GPU method, and the O(N^2) kick is split by target rows). Every rank
 * holds the whole system (the same inputs, so the same state bit for bit)
 * and calls nb_step with the same arguments. Each rank evaluates the kick,
 * and the row-wise part of the force update after the direct solver, for
 * its own block of target rows only; everything else (the O(N) drifts, the
 * encounter set, the groups, the direct solver, the members' rows) runs on
 * every rank on identical data. Two exchanges per step join the blocks:
 *   1. after the trial kick, every rank's flagged pairs (a header of 4 ints,
 *      count, status, unclipped count, 0, then pair_capacity (i, j) int
 *      pairs, count of them valid), so that every rank forms the same
 *      encounter set; a rank's kick error (overflow, a bad coordinate)
 *      reaches every rank through the status and the step rolls back on all;
 *   2. after the force update, every rank's rows of the acceleration (three
 *      blocks of `chunk` doubles, ax, ay, az, zero beyond its last row), so
 *      that every rank closes the step with the whole force.
 * The blocks are contiguous: rank r owns rows [r c, min(n, (r + 1) c)),
 * c = ceil(n / world) (nb_shard_rows). With the same n and kick split the
 * rows are bit-identical to those of the unsharded kick, so a sharded run
 * equals nb_step bit for bit for any world size.
 * --------------------------------------------------------------------- */

/* The exchange: gather `bytes` bytes from every rank's send buffer into recv
 * (world x bytes, rank r's block at offset r x bytes), both device memory of
 * this rank, ordered after the work already enqueued on `stream` and before
 * the work enqueued on it afterwards (an NCCL all-gather on that stream, for
 * example). Returns 0 on success; anything else fails the step. */
typedef int (*nb_allgather_fn)(void* user, const void* send, void* recv, size_t bytes,
                               void* stream);

/* Rows [row0, row1) of rank `rank` out of `world` for n bodies (host
 * function; an empty block when n < world). NB_E_INVALID for bad arguments. */
int nb_shard_rows(int n, int rank, int world, int* row0, int* row1);

/* Bytes of exchange buffer (device memory, 256-byte aligned) that
 * nb_set_shard needs for this system and world size; 0 if invalid. */
size_t nb_shard_buffer_bytes(const nb_system* s, int world);

/* Shard the system's kick across `world` ranks as rank `rank`, with the
 * caller's all-gather `fn` (called from inside nb_step with `user`) and an
 * exchange buffer of nb_shard_buffer_bytes() bytes that stays allocated while
 * the system is sharded. world = 1 (fn and buf may be NULL) returns to the
 * unsharded step. Not combinable with rcrit_refresh, gas drag or ejection
 * (their extra force evaluations are not sharded): NB_E_INVALID. */
int nb_set_shard(nb_system* s, int rank, int world, nb_allgather_fn fn, void* user, void* buf,
                 size_t buf_bytes);

/* ---------------------------------------------------------------------
 * Batched ensembles: many independent systems (each its own star and
 * bodies, the same method and parameters) integrated together. Each step of
 * every system is three launches: the O(N) opening phase (a CTA takes whole
 * systems, largest first), the O(N^2) kick over tiles of 128 target rows of
 * one system, and the closing phase (encounters, groups, Bulirsch-Stoer,
 * the incremental force update, closing kicks) with a system in shared
 * memory. Chunks of steps are replayed from a captured CUDA graph. System s
 * owns body slots offsets[s] .. offsets[s+1]-1 of the concatenated arrays;
 * 1 <= N_s <= NB_BATCH_MAX_N.
 * --------------------------------------------------------------------- */
#define NB_BATCH_MAX_N 512
typedef struct nb_batch nb_batch;

/* Workspace bytes for nsys systems with the given offsets (host, nsys + 1). */
size_t nb_batch_workspace_bytes(const nb_params* p, int nsys, const int* offsets);

/* x, v [total][3], m, R [total], rc_override [total] or NULL; host pointers
 * unless inputs_on_device. offsets are host. Evaluates the first force and
 * flags of every system. Errors as nb_init_system. */
int nb_batch_init(nb_batch** out, const nb_params* p, int nsys, const int* offsets,
                  const double* x, const double* v, const double* m, const double* R,
                  const double* rc_override, void* workspace, size_t ws_bytes, void* stream,
                  int inputs_on_device);

/* Advance every system by nsteps steps of dt: full chunks replay a captured
 * graph, the remainder is launched directly. Synchronises; atomic like
 * nb_step (any error restores the state at entry). */
int nb_batch_step(nb_batch* b, int nsteps, double dt);

/* Launch shape: threads per CTA of the per-system launches (64, 128 or 256)
 * and steps per captured graph (1..1000). Schedule: target rows per kick
 * tile (32, 64 or 128) and the number of buckets (1..16), independent chains
 * of launches on their own streams, each holding every k-th system of the
 * largest-first order (one bucket's latency-bound direct solver then overlaps
 * the others' kicks). nb_batch_autotune() times threads {64, 128, 256} x
 * buckets {4, 8, 16} at 32-row tiles and 25-step graphs, then tile rows 64
 * and 128 (the row kick only: the unordered-pair kick's tiles are 32-body
 * block pairs), then chunks of 10, 25 and 50 steps (each timed afresh over
 * the same 50 steps, best of three interleaved rounds), on graph replays of a copy of the state (restored
 * afterwards), and keeps the fastest; *ms_per_step is the chosen chunk's time;
 * nb_batch_get_shape() reports what is in use. None of these changes a
 * result: every system's arithmetic is the same in any shape. */
int nb_batch_set_shape(nb_batch* b, int threads, int chunk);
int nb_batch_set_schedule(nb_batch* b, int tile_rows, int buckets);
int nb_batch_autotune(nb_batch* b, double dt, int* threads, double* ms_per_step);
int nb_batch_get_shape(nb_batch* b, int* threads, int* chunk, int* tile_rows, int* buckets);

/* All slots (offsets layout): x, v [total][3], m, R [total], alive [total]
 * (0 for bodies absorbed by mergers). Any pointer may be NULL. */
int nb_batch_get_state(nb_batch* b, double* x, double* v, double* m, double* R, int* alive,
                       int out_on_device);

/* Encounter pairs of system `sys` during the last nb_batch_step() call as
 * (step, i, j) triples, i < j the body's index within the system, sorted by
 * step then indices (the same list nb_encounter_list gives for that system on
 * its own). *count receives the total; the library keeps the first 256 per
 * system and call. NB_E_OVERFLOW when the total exceeds 256 or cap. */
int nb_batch_encounter_list(nb_batch* b, int sys, int* step_ij, int cap, int* count);

/* Per-system energy (Eqs. Ha + Hb + Hc) and energy removed by mergers, host
 * arrays of nsys. */
int nb_batch_energy(nb_batch* b, double* E, double* E_lost);
int nb_batch_stats(nb_batch* b, nb_stats_t* out);

/* Time budget of one persistent launch: a CTA takes no further system once it
 * has run longer than max_ms_per_launch, and the call then returns
 * NB_E_TIMEOUT with the state rolled back to the call's start (0 = no budget,
 * the default). Keeps any launch bounded on a shared GPU. */
int nb_batch_set_budget(nb_batch* b, double max_ms_per_launch);

/* Load balance of the last launch: efficiency = sum over CTAs of their busy
 * time / (CTAs x the longest), the longest CTA time in ms, and the CTA count. */
int nb_batch_balance(nb_batch* b, double* efficiency, double* max_cta_ms, int* ctas);
void nb_batch_destroy(nb_batch* b);

/* ---------------------------------------------------------------------
 * Single-kernel entry points (one launch each, on caller device buffers).
 * --------------------------------------------------------------------- */

/* Kick accelerations (gradient of Eq. Hb) and close-pair flags of n bodies.
 * x [n][3], m [n], rc [n] device inputs; a [n][3] device output; pairs_ij
 * device output of up to cap (i, j) pairs, i < j, unordered; *npairs (host)
 * receives the total count. scratch: device buffer of
 * nb_kick_scratch_bytes(n, split) bytes. precision: NB_PREC_*. Returns
 * NB_E_OVERFLOW when more than cap pairs were found (all others written) and
 * NB_E_INVALID when a coordinate is not finite or |x| >= 2^37 AU (the FP64
 * kick forms its differences from 128-bit fixed-point positions, exact below
 * 2^38 AU; nb_init_system and nb_set_state apply the same bound). */
size_t nb_kick_scratch_bytes(int n, int split);
int nb_kick(int n, const double* x, const double* m, const double* rc, double G, int precision,
            int split, double* a, int* pairs_ij, int cap, int* npairs, void* scratch,
            size_t scratch_bytes, void* stream);

/* The kick of nb_kick() for the target rows row0 <= i < row1 only, every one
 * of the n bodies acting on them: the unit of a row-sharded kick (each
 * device owning a block of rows after gathering all positions). a receives
 * (row1 - row0) x 3 doubles, row i at a[3 (i - row0)]; pairs_ij the flagged
 * pairs (i, j), i < j, with i in the block. With the same n and split the
 * rows are bit-identical to those of nb_kick(), so blocks that partition
 * 0..n-1 reproduce the full kick and its pair set. NB_E_INVALID unless
 * 0 <= row0 < row1 <= n; scratch and errors as nb_kick(). */
int nb_kick_rows(int n, int row0, int row1, const double* x, const double* m, const double* rc,
                 double G, int precision, int split, double* a, int* pairs_ij, int cap,
                 int* npairs, void* scratch, size_t scratch_bytes, void* stream);

/* The kick of nb_kick() for callers that cannot allocate device memory (a
 * framework allocator owns the device, allocation is forbidden after
 * start-up, or the caller must never touch the CUDA allocator). The paper
 * has no counterpart; this is a deployment convenience. Arguments as in
 * nb_kick() minus the scratch: the library keeps a static device array of
 * about 8.4 MB on every GPU that loads it, so n must not exceed
 * NB_NOALLOC_MAX_N (NB_E_INVALID otherwise). The first call in each CUDA
 * context (a device's primary context, again after cudaDeviceReset, or a
 * caller's own driver-API context) looks up that array's device address:
 * make it before any stream capture. Calls share the array: calls that
 * overlap on the GPU race, so serialise them. The pair set equals nb_kick()'s;
 * the accelerations agree with it to rounding (at most 4 source chunks here,
 * so the partial sums are added in another order), not bit for bit.
 * Allocates nothing; synchronises the stream before returning. */
#define NB_NOALLOC_MAX_N 65600
int nb_kick_noalloc(int n, const double* x, const double* m, const double* rc, double G,
                    int precision, double* a, int* pairs_ij, int cap, int* npairs, void* stream);

/* Gradient of the total energy E = H_A + H_B + H_C (Eqs. Ha-Hc; the
 * changeover K cancels, leaving the Newtonian pair sum) with respect to the
 * state of the live bodies, for losses that contain the energy (the adjoint's
 * cotangent of a final-energy term):
 *   dE/dx_i = G m_i (m0 x_i / |x_i|^3 + sum_j m_j (x_i - x_j) / r_ij^3)
 *   dE/dv_i = m_i (v_i + P / m0),  P = sum_j m_j v_j
 *   dE/dm_i = |v_i|^2 / 2 - G m0 / |x_i| - G sum_j m_j / r_ij + P . v_i / m0
 * Device arrays: x, v [n][3], m [n], alive [n] int32 (0 = absorbed; NULL =
 * every body live); outputs gx, gv [n][3], gm [n] (zero for absorbed
 * bodies). scratch: nb_energy_grad_scratch_bytes(n) bytes of device memory,
 * 8-byte aligned (the pair sums' per-chunk partials, at most 256 n doubles,
 * and the momentum's per-block sums). Asynchronous on the stream. NB_E_INVALID for n < 1, null
 * arrays or m0 <= 0; NB_E_WORKSPACE for a short or misaligned scratch. */
size_t nb_energy_grad_scratch_bytes(int n);
int nb_energy_grad(int n, const double* x, const double* v, const double* m, const int* alive,
                   double G, double m0, double* gx, double* gv, double* gm, void* scratch,
                   size_t scratch_bytes, void* stream);

/* Universal-variable Kepler drift (first sum of Eq. Ha) of n bodies about
 * mu = G m0 by dt, in place on device x, v [n][3]. Returns NB_E_NOCONV if a
 * body hit max_iter. scratch: 16 bytes of device memory. */
int nb_kepler_drift(int n, double mu, double* x, double* v, double dt, int max_iter,
                    void* scratch, void* stream);

/* Measured throughput of the chip's FP64 (DFMA) and FP32 (FFMA) pipes in
 * FLOP/s, from the library's own dependent-free FMA loops. scratch: at least
 * nb_peak_scratch_bytes() of device memory. */
size_t nb_peak_scratch_bytes(void);
int nb_measure_peaks(double* fp64_flops, double* fp32_flops, void* scratch, void* stream);

/* Element-wise evaluation, on device arrays in[n] -> out[n], of the device
 * arithmetic helpers the kernels are built from, for checking them one by one
 * (the integrator never calls this):
 *   NB_MATH_EXP            exp(x), table-driven (|x| <= 700)
 *   NB_MATH_RCP            1/x (x positive normal, 2^-126 <= x < 2^128)
 *   NB_MATH_RSQRT          1/sqrt(x) (same range)
 *   NB_MATH_RPOW32         x^(-3/2) as the FP64 kick forms m r^-3 from x = r^2
 *   NB_MATH_RPOW32_MIXED   the same with the mixed kick's single Newton step
 *   NB_MATH_RPOW32_M       the same as NB_MATH_RPOW32 from the mass alone (the
 *                          form used by the finishing and batched kernels)
 *   NB_MATH_CLOSE_WEIGHT   1 - w(r) of the changeover (w = K - r dK/dr, the
 *                          paragraph after Eq. Hc) for rc = 1, x = r
 *   NB_MATH_MASS15         1.5 m as the kernels build it from a mass x
 *   NB_MATH_MASS1875       1.875 m likewise (x = 0 or 2^-126 <= x <= 2^127)
 *   NB_MATH_NEVILLE        the direct solver's Neville weight (j - q)^2 /
 *                          (q (2j - q)) for x = 16 j + q, 1 <= q < j <= 12
 *                          (0 otherwise), as the solver reads it
 *   NB_MATH_RATIO_LE       the solver's acceptance test fl(a / b) <= tol as
 *                          1 or 0, reading in[3i .. 3i+2] = (a, b, tol), b > 0,
 *                          tol >= 0 (in then holds 3n doubles)
 *   NB_MATH_RINV3          x^(-3/2) as the unordered-pair kick forms r^-3 from
 *                          x = r^2 (residual and series on the integer pipe,
 *                          one FP64 product; 2^-126 <= x < 2^128)
 * NB_E_INVALID for an unknown fn, n < 0 or null arrays (n > 0); asynchronous
 * on the stream. */
enum {
  NB_MATH_EXP = 0,
  NB_MATH_RCP = 1,
  NB_MATH_RSQRT = 2,
  NB_MATH_RPOW32 = 3,
  NB_MATH_RPOW32_MIXED = 4,
  NB_MATH_RPOW32_M = 5,
  NB_MATH_CLOSE_WEIGHT = 6,
  NB_MATH_MASS15 = 7,
  NB_MATH_MASS1875 = 8,
  NB_MATH_NEVILLE = 9,
  NB_MATH_RATIO_LE = 10,
  NB_MATH_RINV3 = 11
};
int nb_math_eval(int fn, int n, const double* in, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Discrete adjoint of nb_step: the gradient of a scalar loss L(x_T, v_T, m_T)
 * of the state after nsteps steps with respect to the initial x_0, v_0, m_0.
 * The paper integrates forward only (Eqs. H, Ha-Hc); this is the transposed
 * linearisation of exactly the forward algorithm: the kick of Eq. Hb, the
 * drift of Eq. Hc, the Kepler drift of Eq. Ha (6x6 Jacobian of the f/g map
 * with the implicit derivative of the universal anomaly) and, for bodies in
 * close-encounter groups, the recorded Bulirsch-Stoer substeps (modified
 * midpoint and Neville extrapolation) and perfect mergers. Encounter flags,
 * groups, BS substep sizes and columns, mergers and the critical radii rc are
 * held at their forward values (rc gets no gradient). FP64 only.
 *
 * Memory: the caller provides nb_adjoint_workspace_bytes() of device memory,
 * 256-byte aligned; it holds an nb_system for the forward state, a
 * checkpoint of the full state every checkpoint_every steps, per-step
 * records of one segment and the BS replay scratch. The backward pass
 * replays each segment from its checkpoint (the forward is deterministic,
 * so the replay takes every decision of the forward again).
 * Layout of host/device arrays as nb_init_system: x, v [n][3], m, R, rc [n].
 * ------------------------------------------------------------------------ */
typedef struct nb_adjoint nb_adjoint;

/* Bytes of workspace for n bodies and up to nsteps steps; 0 if invalid. */
size_t nb_adjoint_workspace_bytes(const nb_params* p, int n, int nsteps, int checkpoint_every);

/* Create the handle and load the initial state (as nb_init_system; rc must
 * be given so that the forward and its finite-difference checks keep it).
 * p->precision must be NB_PREC_FP64. NB_E_WORKSPACE if ws is too small or
 * misaligned; NB_E_INVALID for bad inputs. */
int nb_adjoint_init(nb_adjoint** out, const nb_params* p, int n, const double* x,
                    const double* v, const double* m, const double* R, const double* rc,
                    int nsteps, int checkpoint_every, void* workspace, size_t ws_bytes,
                    void* stream, int inputs_on_device);

/* Run nsteps steps of size dt from the initial state, keeping checkpoints.
 * May be called again; each call restarts from the initial state. Returns
 * NB_E_OVERFLOW if nsteps exceeds the count the workspace was sized for, or
 * the forward's status. */
int nb_adjoint_forward(nb_adjoint* a, int nsteps, double dt);

/* Final state of the forward (all n slots; absorbed bodies have m = 0,
 * alive = 0). Any pointer may be NULL. Synchronises the stream. */
int nb_adjoint_state(nb_adjoint* a, double* x, double* v, double* m, int* alive,
                     int out_on_device);

/* Pull back dL/dx_T, dL/dv_T [n][3] and dL/dm_T [n] to dL/dx_0, dL/dv_0
 * [n][3] and dL/dm_0 [n]. Entries of bodies absorbed by the end are ignored
 * (their final state is a constant). Output pointers may be NULL. Leaves the
 * handle at the forward's final state, so backward can be called again with
 * other cotangents. NB_E_OVERFLOW if a group needed more than 256 BS
 * substeps or 16 mergers in one step (the records' capacity). */
int nb_adjoint_backward(nb_adjoint* a, const double* gx, const double* gv, const double* gm,
                        double* dx0, double* dv0, double* dm0, int on_device);

const char* nb_adjoint_last_error(const nb_adjoint* a);
void nb_adjoint_destroy(nb_adjoint* a);

#ifdef __cplusplus
}
#endif
#endif
