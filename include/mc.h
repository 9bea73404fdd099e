/*
 * mc.h -- C ABI of libmcgb: GB300 (sm_103a) multigroup, time-dependent Monte Carlo random walk.
 *
 * The library implements the transport method whose problem class the MC/DC paper states in
 * its Section 3: fixed-source multigroup transport on quadric-surface constructive solid geometry
 * (planes, cylinders, spheres, general quadrics and a pin lattice with optional axial layers), a
 * time-dependent source, a time
 * census and time-dependent mesh tallies scored with the track-length estimator (Section 3.1) or
 * the time-crossing estimator, with analog collisions or implicit capture (Section 3's runs).
 * Per particle the walk samples the distance to collision, compares it with the distance to the
 * next surface and to the census, moves the particle and scores its track length into an
 * (x, y, z, group, time) mesh, then samples the collision: scatter to a new group, secondary
 * production into a particle bank, or capture.
 *
 * Conventions for every entry point:
 *   - Return value: MC_OK (0) or a negative mc_status.  Nothing aborts, traps or asserts; the
 *     message of the last failure on the calling thread is returned by mc_last_error().
 *   - Ownership: every array in a descriptor is copied by mc_problem_create; the caller keeps
 *     ownership of its memory.  Output buffers are caller-allocated host memory unless an
 *     argument says "device".
 *   - Streams: `stream` is a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) or NULL
 *     for the legacy default stream.  mc_run is asynchronous on that stream; device-side errors
 *     (bank overflow, watchdog) are reported by mc_wait / mc_tally_get, which synchronise.
 *   - Units: cm, s, 1/cm, cm/s.  Tally values are per source particle.
 */
#ifndef MCGB_MC_H
#define MCGB_MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------- status codes */
typedef enum {
  MC_OK = 0,
  MC_ERR_INVALID = -1,   /* a descriptor or argument failed validation */
  MC_ERR_CUDA = -2,      /* a CUDA runtime call failed (message in mc_last_error) */
  MC_ERR_OOM = -3,       /* device allocation failed */
  MC_ERR_BANK_FULL = -4, /* the secondary/birth bank overflowed during the run */
  MC_ERR_TIMEOUT = -5,   /* the device watchdog (iteration or barrier-wait budget) expired */
  MC_ERR_STATE = -6,     /* call out of order (e.g. tally read before any run) */
  MC_ERR_LOST = -7,      /* particles left the geometry (no cell contains them) */
  MC_ERR_BOUNDS = -8     /* bounds-checked build only: an index into a table, a tally or the
                            lattice was out of range (the access was skipped) */
} mc_status;

/* ------------------------------------------------------------------------- limits */
#define MC_MAX_GROUPS 32
#define MC_MAX_MATERIALS 255
#define MC_MAX_SURFACES 255
#define MC_MAX_CELLS 255
#define MC_MAX_HALFSPACES 16
#define MC_MAX_LATTICE 255 /* per axis */
#define MC_MAX_LATTICE_ELEMENTS 65536 /* nx x ny x max(nz, 1) */
#define MC_MAX_TALLIES 4

/* ------------------------------------------------------------------------- geometry */
typedef enum {
  MC_SURF_PX = 0, MC_SURF_PY = 1, MC_SURF_PZ = 2, /* planes x, y, z = coef[0] */
  MC_SURF_CZ = 3, /* cylinder parallel to z: (x - coef[0])^2 + (y - coef[1])^2 - coef[2]^2 */
  MC_SURF_CX = 4, /* cylinder parallel to x: (y - coef[0])^2 + (z - coef[1])^2 - coef[2]^2 */
  MC_SURF_CY = 5, /* cylinder parallel to y: (x - coef[0])^2 + (z - coef[1])^2 - coef[2]^2 */
  MC_SURF_SQ = 6, /* sphere: (x - coef[0])^2 + (y - coef[1])^2 + (z - coef[2])^2 - coef[3]^2 */
  MC_SURF_GQ = 7  /* general quadric A x^2 + B y^2 + C z^2 + D xy + E yz + F zx + G x + H y + I z + J,
                     coef = A..J */
} mc_surface_kind;
typedef enum { MC_BC_INTERIOR = 0, MC_BC_VACUUM = 1, MC_BC_REFLECT = 2 } mc_boundary;

/* Surface f(x,y,z) = 0 of the kind's form (mc_surface_kind), the paper's quadric-surface CSG.  A
 * particle leaves the half-space it is in at the first point ahead where f changes sign in that
 * direction; a grazing entry into a sphere, cylinder or convex quadric whose chord is shorter than
 * 2e-5 cm (FP32 tracking) or 1e-12 cm (FP64) is no crossing.  Reflection is supported on planes only. */
typedef struct {
  int kind;        /* mc_surface_kind */
  double coef[10]; /* as the kind says; unused entries ignored */
  int bc;          /* mc_boundary */
} mc_surface;

/* A cell is the intersection of half-spaces; sense +1 means f >= 0, -1 means f < 0.
 * material >= 0 fills the cell; material == -1 fills it with the lattice, which must cover the
 * cell's extent exactly (the lattice's outer walls are the cell's own surfaces). */
typedef struct {
  int n_halfspaces;
  int surface[MC_MAX_HALFSPACES];
  int sense[MC_MAX_HALFSPACES];
  int material;
} mc_cell;

/* Square pin lattice (the paper's lattice geometry, Section 3): nx x ny elements of side `pitch`,
 * lower-left corner (x0, y0).  With nz >= 2 it has nz axial layers of height pitch_z stacked from
 * z0 (a 3D lattice: axially zoned assemblies, partially inserted rods); with nz = 0 or 1 it is one
 * layer, unbounded in z.  Element (i, j, k) holds a z-cylinder of `radius` centred in it, filled with
 * pin_material[(k*ny + j)*nx + i] (no pin if that entry is -1), inside matrix_material.  The lattice
 * fills the cells whose material is -1 and must cover their extent exactly (its outer walls are
 * the cells' own surfaces).  nx, ny, nz <= MC_MAX_LATTICE and nx*ny*max(nz,1) <= 65536; invalid
 * sizes, pitches or materials make mc_problem_create return MC_ERR_INVALID. */
typedef struct {
  int nx, ny;
  double x0, y0, pitch, radius;
  const int* pin_material; /* [max(nz,1)][ny][nx] */
  int matrix_material;
  int nz;                  /* axial layers (0 or 1: one layer, unbounded in z) */
  double z0, pitch_z;      /* bottom of layer 0 and the layer height (used when nz >= 2) */
} mc_lattice;

/* ------------------------------------------------------------------------- source */
typedef enum { MC_SRC_BOX = 0, MC_SRC_SURFACE_X0 = 1 } mc_source_pos;
typedef enum { MC_DIR_ISO = 0, MC_DIR_BEAM_X = 1, MC_DIR_COS_X = 2 } mc_source_dir;

/* Position uniform in the box [lo, hi] (or on the plane x = lo[0] with y, z uniform in
 * [lo, hi]); direction isotropic, the +x beam, or cosine-distributed into +x (the entering
 * current of an isotropic angular flux); group from group_pdf; time uniform in [t0, t1]. */
typedef struct {
  int pos;  /* mc_source_pos */
  double lo[3], hi[3];
  int dir;  /* mc_source_dir */
  const double* group_pdf; /* [n_groups], non-negative, not necessarily normalised */
  double t0, t1;
} mc_source;

/* ------------------------------------------------------------------------- tallies */
/* Estimators of a mesh tally (both appear in the paper's Section 3 runs).
 *   MC_EST_TRACK_LENGTH: the track-length estimator of the flux integrated over each of the nt time
 *     bins between the nt+1 time edges t (and over each mesh cell): a flight scores w x (its
 *     length inside the cell and time bin).  Per source particle, units cm (flux x volume x time).
 *   MC_EST_TIME_CROSSING: the time-crossing estimator of the flux at each of the nt+1 time points t
 *     themselves (the paper's multigroup pulse and C5G7 transients): a particle alive at t_j scores
 *     w v_g into the mesh cell it occupies at t_j, i.e. a flight over [t_a, t_b) scores every
 *     t_j with t_a <= t_j < t_b.  Per source particle, units cm^3/s (flux x volume).  The
 *     device accumulates the weight w (int64 fixed point stays in range for fast groups); the
 *     readback multiplies by v_g.  A point at or after the census time gets no score: the census
 *     ends every particle there. */
typedef enum { MC_EST_TRACK_LENGTH = 0, MC_EST_TIME_CROSSING = 1 } mc_estimator;

/* Mesh tally over strictly increasing edges (the outermost spatial edges may be +-inf; the time
 * points of a time-crossing tally must be finite).  Values are laid out [z][y][x][group][t]: nt
 * time bins (track length) or nt+1 time points (time crossing). */
typedef struct {
  int nx, ny, nz, nt;
  const double *x, *y, *z, *t; /* nx+1, ny+1, nz+1, nt+1 edges */
  int estimator;               /* mc_estimator (0 = track length) */
} mc_mesh_tally;

/* ------------------------------------------------------------------------- problem */
typedef struct {
  int n_groups;     /* G */
  int n_materials;  /* M */
  const double* sigma_t; /* [M][G] total cross section */
  const double* sigma_s; /* [M][G][G] scattering, row = from-group, column = to-group */
  const double* sigma_f; /* [M][G] production cross section */
  const double* nu;      /* [M][G] mean secondaries per production event (<= 64) */
  const double* chi;     /* [M][G] secondary group spectrum */
  const double* speed;   /* [G] group speeds */
  int n_surfaces;
  const mc_surface* surfaces;
  int n_cells;
  const mc_cell* cells;
  const mc_lattice* lattice; /* NULL if no cell uses a lattice */
  mc_source source;
  int n_tallies;
  const mc_mesh_tally* tallies;
  double t_census;           /* final census time; +inf for steady state */
} mc_problem_desc;

typedef struct mc_problem mc_problem; /* opaque, library-owned */

/* ------------------------------------------------------------------------- run options */
typedef enum { MC_FP32 = 0, MC_FP64 = 1 } mc_precision;
typedef enum { MC_TALLY_FIXED64 = 0, MC_TALLY_FP64 = 1 } mc_tally_mode;
/* Event-based: every iteration advances each live particle by one event and one flight and
 * writes it back to the bank partitioned by its next event (collisions, surfaces).
 * History-based: each thread carries its particle from source to death without write-back.
 * Both draw the same random numbers per particle and give identical fixed-point tallies.
 * Auto: the algorithm mc_run_tune found faster for the problem (event-based until it has run;
 * mc_run_tune called with MC_ALG_AUTO times both). */
typedef enum { MC_ALG_EVENT = 0, MC_ALG_HISTORY = 1, MC_ALG_AUTO = 2 } mc_algorithm;

typedef struct {
  int precision;          /* mc_precision: arithmetic of positions/directions/distances */
  int tally_mode;         /* mc_tally_mode: int64 fixed point (deterministic) or FP64 atomics */
  int fixed_bits;         /* fixed-point scale 2^fixed_bits (default 32) */
  int n_batches;          /* statistical batches, >= 2 (default 32) */
  uint64_t bank_capacity; /* particles in flight (0 = library default: the power of two >= 2 x the
                             histories, at most 2^22, or 2^28 with census_times); FP32 mc_run runs
                             without census_times or weight windows also keep, for the
                             history-style tail, a stack of min(256, bank_capacity / warps)
                             secondaries per warp (none below 32: the run is then one launch) */
  int block_size;         /* threads per CTA (0 = mc_run_tune's choice if it ran, else 128 for
                             the 96-register build above and 256 otherwise) */
  int blocks_per_sm;      /* CTAs per SM, counted in 256-thread CTAs (the cap is blocks_per_sm x
                             256 / block_size CTAs): 2 selects the 128-register build of the kernel
                             (2 x 256 threads per SM), another value the 80-register build (3 x 256
                             fit; FP32 runs whose tallies all take the plain track-length walk use
                             a 96-register build at 128 threads per CTA, 5 CTAs per SM); 0 =
                             mc_run_tune's choice if it ran, else the 128-register build when a
                             tally deals its time pieces out over the warp and the 80- or
                             96-register build otherwise, as many CTAs as fit */
  uint64_t max_iterations;/* watchdog: event iterations before MC_ERR_TIMEOUT (0 = 2^20) */
  int aggregate_atomics;  /* 1 = warp-aggregated tally atomics (staged per warp, same-bin scores
                             summed before one atomic), 0 = one atomic per score at once,
                             -1 = default (currently 0: faster on every measured workload) */
  int ww_enable;          /* 1 = apply the weight-window table set by mc_ww_set_table */
  uint64_t log_first, log_count; /* log every event of histories [log_first, +log_count) */
  uint64_t log_capacity;  /* event records kept (0 = 64 per logged history) */
  uint64_t first_history; /* history indices run are [first_history, first_history + n) */
  int algorithm;          /* mc_algorithm (default MC_ALG_EVENT) */
  uint64_t drain_threshold; /* event mode: once every history is sourced and at most this many
                               particles remain, finish them history-style (0 = 2 per thread; in
                               mc_run_eigen 32 per thread; mc_run_tune may pick another).  FP32
                               mc_run runs without census_times or weight windows do this in a
                               second launch, in which each warp flies its secondaries from its
                               own stack; the results equal those of one launch */
  int tally_stripes;      /* copies of the batch tallies that CTAs score into round-robin, summed
                             by the statistics (0 = up to 16 within a 64 MB budget) */
  int batch_unit;         /* mc_run_batch: histories per work unit a warp claims (0 = tuned or 128) */
  /* Implicit capture (survival biasing; the paper's Kobayashi transient runs with it): a collision
   * never captures.  Its channel is drawn among scatter and production with probabilities
   * Sigma_s / (Sigma_s + Sigma_f) and Sigma_f / (Sigma_s + Sigma_f), and the weight (of the scattered
   * particle or of each of the floor(nu + xi) secondaries) is multiplied by the non-capture
   * probability (Sigma_s + Sigma_f) / Sigma_t; where that is 0 the collision captures as in the
   * analog walk.  After a scatter, a weight below wr_cutoff survives a roulette with probability
   * w / wr_survival at weight wr_survival (the u_spare draw of the collision), which ends histories
   * without bias; roulette kills count as MC_C_WW_KILL.  Needs 0 <= wr_cutoff < wr_survival.  Every
   * tally stays unbiased; FP64 or fixed-point tallies both work (weights stay near 1). */
  int implicit_capture;   /* 0 = analog (default), 1 = implicit capture */
  double wr_cutoff;       /* weight cutoff (default 0.25) */
  double wr_survival;     /* survival weight of the roulette (default 0.5) */
  /* Population control at interior census times (the paper's time census with population control,
   * Section 3), by splitting-roulette within each statistical batch, which makes every batch an
   * independent simulation of its N_b histories.  The run is split into intervals ending at
   * census_times[0..n_census-1] and then at the problem's t_census.  A particle reaching an interior
   * census is banked; then per batch W_b = the sum of llrint(w 2^40) of its banked particles (exact),
   * w_t = W_b 2^-40 / N_b, and a banked particle of weight w becomes floor(w / w_t + xi) copies of
   * weight w_t at the census time (xi = the first FP64 uniform of block 1 of its census flight; copy
   * j tagged as a child with mark 0x40000000 | j), which start the next interval.  The tallies'
   * errors come from the batches.  The array is copied during the call; times must increase and lie
   * below t_census.  mc_run synchronises once per interval.  Not for mc_run_batch / mc_run_eigen /
   * mc_run_static. */
  int n_census;
  const double* census_times;
  /* Population-control method (mc_pc_method).  MC_PC_COMB combs instead of splitting-roulette
   * (systematic sampling of the census bank, one of the population-control techniques the paper
   * cites): per batch the banked particles are ordered by their 64-bit tag, C_j = the running sum of
   * llrint(w 2^40) up to and including particle j, W_b = C_M, and particle j becomes F(C_j) - F(C_{j-1})
   * copies with F(C) = min(N_b, max(0, ceil(C N_b / W_b - xi_b))) evaluated in FP64 in that order
   * (xi_b = the first FP64 uniform of block 5 of event i of tag 0xFFFFFFFE + 2^32 b, i the census
   * index): the N_b teeth (k + xi_b) W_b / N_b that fall in its weight interval.  Every census then
   * restores exactly N_b particles per batch.  Copies as for splitting-roulette. */
  int pc_method;
} mc_run_opts;

typedef enum { MC_PC_SPLIT_ROULETTE = 0, MC_PC_COMB = 1 } mc_pc_method;

/* Fills the defaults listed above. */
void mc_run_opts_default(mc_run_opts* o);

/* Event record of the debug log (one per flight of a logged history).  kind: 0 collision,
 * 1 surface, 2 census, 3 lost.  outcome: collision 0 scatter / 1 production / 2 capture;
 * surface 0 transmit / 1 reflect / 2 leak / 3 lattice wall / 4 pin.  Position, direction, group,
 * time and weight are the values at the end of the flight, before the event is handled. */
typedef struct {
  uint64_t tag, root;
  uint32_t k;
  int32_t kind, outcome, n_child, cell, elem, in_pin, g;
  double x, y, z, ux, uy, uz, t, w;
} mc_event;

/* Counters summed over a run, in this order.  MC_C_SCORES counts tally updates (track length: one
 * per mesh cell and time bin a flight crosses; time crossing: one per time point a flight spans).
 * MC_C_WW_KILL counts particles removed by a roulette (weight windows or the implicit-capture
 * weight cutoff).  MC_C_WW_HELD counts weight-window splits
 * not made because the particle store was more than half full: a split is optional (the particle
 * keeps its weight, which is unbiased), so bad windows slow a run down instead of overflowing
 * it; a run with held splits is no longer independent of the GPU's schedule.  MC_C_PC_BANKED counts
 * particles stopped at an interior census of population control, MC_C_PC_COPIES the particles that
 * splitting-roulette started from them. */
typedef enum {
  MC_C_SOURCE = 0, MC_C_SECONDARY, MC_C_CAPTURE, MC_C_PRODUCTION, MC_C_LEAK, MC_C_CENSUS,
  MC_C_LOST, MC_C_FLIGHT, MC_C_COLLISION, MC_C_SCATTER, MC_C_SURFACE, MC_C_REFLECT,
  MC_C_WW_SPLIT, MC_C_WW_KILL, MC_C_ITERATIONS, MC_C_SCORES, MC_C_WW_HELD, MC_C_PC_BANKED, MC_C_PC_COPIES,
  MC_NCOUNTERS
} mc_counter;

/* ------------------------------------------------------------------------- entry points */

/* Validates `d` on the host (returns MC_ERR_INVALID before touching the GPU), builds the
 * per-material sampling tables (scatter-group CDFs, channel thresholds, chi CDFs) and the
 * geometry/tally tables, and uploads them to the current device.  *out receives a handle owned
 * by the library; release it with mc_problem_destroy. */
int mc_problem_create(const mc_problem_desc* d, mc_problem** out);

/* Runs n_histories source particles (history indices first_history + 0..n-1, each with its whole lineage of
 * secondaries) with the given 64-bit seed, asynchronously on `stream`.  Tallies and counters of
 * the previous run are replaced.  Histories are split into opts->n_batches contiguous batches
 * whose tallies give the statistical error.  The paper's time census, track-length estimator and
 * secondary production are Section 3 features; the random walk itself is the textbook analog one.
 * Returns MC_ERR_INVALID for bad options, or when the problem's tables (per material and group
 * cross sections and scatter CDFs, surfaces, cells, the lattice's one-byte-per-element pin map, tally
 * edges) and the per-warp queues do not fit in one CTA's shared memory, where the kernels keep
 * them (about 180 KB of tables at 256 threads per CTA); MC_ERR_OOM / MC_ERR_CUDA for launch failures. */
int mc_run(mc_problem* p, uint64_t n_histories, uint64_t seed, const mc_run_opts* opts,
           void* stream);

/* k-eigenvalue power iteration (the paper's C5G7 runs, Section 3: k-eigenvalue, inactive and active
 * cycles), analog transport of n_inactive + n_active cycles of n_per_cycle histories each on a
 * steady-state problem (t_census = inf) with production cross sections.
 *   Cycle 0 starts from the problem's source.  A production event does not transport secondaries:
 *   it banks floor(nu / k + xi) fission sites (position, group drawn from chi) for the next cycle,
 *   k being the previous cycle's estimate (1 before cycle 0), in slots of the producing history, so
 *   that the sites are ordered by producing history and production order whatever the schedule.
 *   Cycle c >= 1 starts history h (particle tag h + 2^32 c) at site floor((h + u0) M / N) of the M
 *   sites of cycle c - 1 (systematic sampling; u0 = the first uniform of Philox(seed, counter
 *   (2^32 - 1, c, 2^32 - 1, 4))), isotropic, in the site's group, at t = 0 with weight 1.
 *   k of a cycle is the track-length estimate: the sum over its flights of w l nu Sigma_f (summed
 *   exactly in int64 fixed point at 2^-32), divided by N.  Tallies are scored in the active cycles
 *   only, each active cycle being one statistical batch (mc_tally_get then gives the mean over the
 *   active cycles per source particle and its standard error).
 *   opts: precision, tally mode, kernel configuration, algorithm and event logging as for mc_run
 *   (a log covers histories [log_first, +log_count) of every cycle); n_batches is replaced by
 *   n_active; weight windows, implicit capture and first_history are rejected.
 *   Outputs (host, nullable): k_cycle[n_inactive + n_active], sites_cycle[same], *k_mean and
 *   *k_std_err over the active cycles.  Synchronises once per cycle (to read k).  MC_ERR_STATE if a
 *   cycle banks no site; device errors as for mc_wait. */
int mc_run_eigen(mc_problem* p, uint64_t n_per_cycle, int n_inactive, int n_active, uint64_t seed,
                 const mc_run_opts* opts, void* stream, double* k_cycle, uint64_t* sites_cycle, double* k_mean,
                 double* k_std_err);

/* Autotuner of mc_run for one problem: runs n_histories with each candidate configuration (256 or
 * 128 threads per CTA; the 80-register build at 3 CTAs of 256 per SM, or the 128-register build at
 * 2; with opts->algorithm == MC_ALG_AUTO each under both algorithms), times each run with CUDA
 * events (best of two after a warm-up) and stores the fastest in the problem.  When
 * opts->drain_threshold is 0, drain thresholds of 16 and 64 times the default (twice the resident
 * threads) are timed as well, at the fastest event-based configuration.  Later mc_run calls on the
 * problem whose block_size and blocks_per_sm are both 0 use the stored configuration (and its drain
 * threshold when theirs is 0), those with MC_ALG_AUTO its algorithm.  tuned (nullable) receives a
 * copy of opts with those fields set (drain_threshold 0 = the default), best_ms (nullable) its time.
 * Synchronises; the tallies left behind are those of the last candidate. */
int mc_run_tune(mc_problem* p, uint64_t n_histories, uint64_t seed, const mc_run_opts* opts, void* stream,
                mc_run_opts* tuned, double* best_ms);

/* Waits for the runs issued so far and returns the first device error any of them raised since
 * the previous mc_wait (MC_OK, MC_ERR_BANK_FULL, MC_ERR_TIMEOUT, MC_ERR_LOST), so that back-to-back
 * runs cannot hide a failed one. */
int mc_wait(mc_problem* p);

/* Shape of a tally: {nz, ny, nx, G, nt} (track length) or {nz, ny, nx, G, nt + 1} (time
 * crossing).  tally_id == n_tallies addresses the leakage tally, shape {1, 1, n_surfaces, 1, 1}:
 * weight leaving through each vacuum surface. */
int mc_tally_shape(const mc_problem* p, int tally_id, int64_t shape[5]);

/* Copies the per-source-particle mean and its standard error (from the spread of the batch
 * means) of every bin of a tally into host arrays of n >= bins elements (time-crossing bins
 * already multiplied by their group speed).  Synchronises. */
int mc_tally_get(mc_problem* p, int tally_id, double* mean, double* std_err, size_t n);

/* Copies the per-batch means per source particle, out[n_batches][bins] (n >= n_batches * bins),
 * of a tally, so that the error of any function of several bins (e.g. a total) can be formed
 * from the spread of the batch values.  Synchronises. */
int mc_tally_batches(mc_problem* p, int tally_id, double* out, size_t n, int* n_batches);

/* Exact int64 fixed-point sums (units of 2^-fixed_bits) over all histories of the last run, one
 * per bin of a tally (the track-length scores of Section 3 summed over batches and stripes, before
 * any floating-point division), into sums[n >= bins]; *fixed_bits (may be NULL) receives the scale.
 * Integer sums do not depend on the order of their terms: runs over disjoint history ranges
 * (mc_run_opts::first_history) add up to the run over their union bit for bit, which is how
 * histories shard across processes or GPUs and how a run cut short resumes.  MC_ERR_STATE after a
 * run with FP64 tallies.  Synchronises. */
int mc_tally_sums(mc_problem* p, int tally_id, int64_t* sums, size_t n, int* fixed_bits);

/* Copies the MC_NCOUNTERS run counters into counters[n]. Synchronises. */
int mc_counters_get(mc_problem* p, int64_t* counters, size_t n);

/* Copies up to `cap` event records of the last run's logged histories; *n_out receives the
 * number copied.  Records are in device completion order (sort by (tag, k) to compare). */
int mc_event_log(mc_problem* p, mc_event* out, size_t cap, size_t* n_out);

/* Per-iteration trace of the last run's persistent kernel: t_ns[i] (%globaltimer, ns, relative
 * to kernel start), items[i] (particles handled in iteration i), sources[i] (new histories
 * among them; bit 63 set when the iteration ran history-style).  *n_out = iterations recorded
 * (at most cap and at most 65536).  Synchronises. */
int mc_trace_get(mc_problem* p, uint64_t* t_ns, uint64_t* items, uint64_t* sources, size_t cap,
                 size_t* n_out);

/* Device time of the last run's phases, from CUDA events recorded on the run's stream around
 * the transport kernel and around the batch-statistics kernel (milliseconds).  Synchronises. */
int mc_run_timing(mc_problem* p, double* transport_ms, double* stats_ms);

/* Kernels the last mc_run of p launched on its stream: the transport (one launch, or two for a
 * split run: FP32 tracking without census times or weight windows runs its event-based iterations
 * and its history-style tail as two launches), the range-walk reconstruction when a tally is
 * scored by the range walk, and the batch statistics.  *n receives the count.  MC_ERR_STATE when
 * p has not run, or when its last run was not a plain mc_run (census times, mc_run_batch,
 * mc_run_eigen), whose launches are not counted; mc_run_static leaves the count of p's last
 * run as it was.  Does not synchronise. */
int mc_run_launches(const mc_problem* p, int* n);

/* Device layout of the last run's batch tallies (the track-length tally scoring of Section 3 writes
 * into it): *stripes copies of *n_batches rows of *row int64 (or double) elements each, so the
 * scoring atomics of a run spread over stripes x n_batches x row elements.  Any pointer may be
 * NULL.  MC_ERR_STATE before the first run. */
int mc_tally_layout(const mc_problem* p, int* stripes, int* n_batches, uint64_t* row);

/* Weight windows (variance reduction for deep penetration; the paper's runs are analog or use
 * implicit capture, §3).  Sets the window-centre table w_c over an (x, y, z) mesh and all groups:
 * edges = x[nx+1], y[ny+1], z[nz+1] (increasing), centre[nz][ny][nx][G] (host arrays, copied;
 * 0 disables windows in a cell).  With opts->ww_enable, after every collision or surface event a
 * particle of weight w in a cell with centre w_c is split into k = min(ceil(w / w_c), 10) copies
 * of weight w / k if w > 2 w_c, or rouletted (kept with probability w / w_c at weight w_c, using
 * the event's u_ww draw) if w < w_c / 2.  Both keep every tally unbiased.  Weighted runs should
 * use FP64 tallies (weights can span many decades). */
int mc_ww_set_table(mc_problem* p, int nx, int ny, int nz, const double* edges, const double* centre);

/* The same with time bins (the time-dependent problems of Section 3: a pulse source and a time
 * census, where the importance of a particle depends on when it is somewhere): edges = x[nx+1],
 * y[ny+1], z[nz+1], t[nt+1] (increasing), centre[nt][nz][ny][nx][G].  A particle takes the window of
 * the time bin t[i] <= t < t[i+1] holding its time (outside every bin: no window).
 * mc_ww_set_table is this call with one time bin [0, +inf). */
int mc_ww_set_table_t(mc_problem* p, int nx, int ny, int nz, int nt, const double* edges, const double* centre);

/* ------------------------------------------------------------------------- importance network */
/* A 5 -> 64 -> 64 -> 64 -> 1 perceptron (tanh hidden units, linear output) mapping a phase-space
 * point (x, y, z, group, t, each scaled to [-1, 1]) to the log of a weight-window centre.  FP32
 * master parameters with Adam state; the forward and backward passes run on the tensor cores in
 * BF16 with FP32 accumulation.  Parameter order: W1[64][5], b1[64], W2[64][64], b2[64],
 * W3[64][64], b3[64], W4[64], b4 (mc_mlp_param_count() values).  The paper has no such network:
 * it is this library's learned variance reduction for deep-penetration problems. */
typedef struct mc_mlp mc_mlp;
int mc_mlp_param_count(void);
/* Creates a network on the current device with all parameters 0. */
int mc_mlp_create(mc_mlp** out);
void mc_mlp_destroy(mc_mlp* m);
/* Copies n == mc_mlp_param_count() parameters from / to host memory (set resets the Adam state). */
int mc_mlp_set_params(mc_mlp* m, const double* params, size_t n);
int mc_mlp_get_params(mc_mlp* m, double* params, size_t n);
/* y[i] = net(x[i]) for n points; x DEVICE [n][5] float, y DEVICE [n] float. */
int mc_mlp_forward(mc_mlp* m, const float* x, float* y, int n, void* stream);
/* loss = (1/n) sum_i wt[i] (net(x[i]) - target[i])^2 and grad = d loss / d params (DEVICE arrays;
 * wt may be NULL for unit weights; grad has mc_mlp_param_count() floats; both are overwritten). */
int mc_mlp_loss_grad(mc_mlp* m, const float* x, const float* target, const float* wt, int n, float* grad,
                     float* loss, void* stream);
/* `epochs` full-batch Adam steps (beta 0.9 / 0.999) at learning rate lr on the DEVICE arrays,
 * continuing the network's Adam state; *last_loss (DEVICE, may be NULL) gets the last epoch's loss.
 * One CTA runs all epochs; the set is limited to 2^20 points. */
int mc_mlp_train(mc_mlp* m, const float* x, const float* target, const float* wt, int n, int epochs, float lr,
                 float* last_loss, void* stream);
/* One learning round of the weight windows from the problem's last run (synchronous):
 *   1. from mesh tally `tally_id` take the flux phi of every (cell, group, time bin) resolved to a
 *      relative error below 0.5 (with one time bin, or none resolved in time: the flux summed over
 *      time); target = log(phi / phi_ref), phi_ref = that of the source point's cell in the source's
 *      main group (and the time bin of the source's start time), weight = 1 / relative variance
 *      (capped); the network input is (x, y, z, group, time bin index), each scaled to [-1, 1];
 *   2. if extrap_slope > 0, continue the windows past the resolved region along x: for every x line
 *      of the mesh (fixed y, z cell and time bin) and each group with r >= 3 resolved cells, fit a
 *      least-squares line to the targets of its outermost max(3, r/4) resolved cells; take the
 *      flattest of these slopes that fall away from the resolved region as the line's common
 *      slope (deep in a medium all groups decay at the common asymptotic rate); from each group's
 *      outermost resolved cell, lower the target at extrap_slope (in (0, 1]) times that slope until
 *      it has fallen by extrap_efolds, then hold it to the end of the line.  These extra targets
 *      have weight 4 (a 50% relative error) and are clamped at -700.  The windows then reach past
 *      the depth the last run resolved, so that each round resolves deeper, and extrap_efolds
 *      bounds how far a wrong slope can take them from the flux.  (A table whose splitting
 *      overflows the bank shows as MC_ERR_BANK_FULL on the next run: learn again with less.)
 *   3. train the network on these targets on the GPU (`epochs` Adam steps at `lr`);
 *   4. evaluate it on every (cell, group, time bin) of that tally's mesh and set the window centres
 *      w_c = phi_ref-normalised exp(net) as the problem's weight-window table, with the tally's
 *      time bins when step 1 resolved them in time (the forward-flux weight windows of the MAGIC
 *      method, learned instead of tabulated).
 * info (host, may be NULL) receives {resolved training points, final loss, target scale, phi_ref,
 * extrapolated training points}. */
int mc_ww_learn(mc_problem* p, mc_mlp* m, int tally_id, int epochs, float lr, double extrap_slope,
                double extrap_efolds, double info[5]);

/* The same with a network the problem owns (created by the first mc_ww_set_mlp, released with the
 * problem), for callers that do not manage an mc_mlp.  mc_ww_set_mlp loads n == mc_mlp_param_count()
 * parameters given as BF16 bit patterns (host array; the order of mc_mlp_set_params; non-finite
 * values are MC_ERR_INVALID).  mc_ww_train runs one learning round on mesh tally tally_id of the
 * problem's last run (mc_ww_learn steps 1, 3 and 4: no extrapolation past the resolved region), or
 * returns MC_ERR_STATE when no weights were loaded. */
int mc_ww_set_mlp(mc_problem* p, const uint16_t* bf16_weights, size_t n);
int mc_ww_train(mc_problem* p, int tally_id, int epochs, float lr);

/* Bytes of sampling, geometry and tally tables that mc_problem_create copied to the device
 * (both tracking precisions); 0 for NULL. */
size_t mc_problem_table_bytes(const mc_problem* p);

/* Releases the problem and its device memory.  NULL is ignored. */
void mc_problem_destroy(mc_problem* p);

/* Thread-local message describing the last failure ("" if none). */
const char* mc_last_error(void);

/* ------------------------------------------------------------------------- allocation-free run */
/* Bytes of the library's static device scratch used by mc_run_static. */
#define MC_STATIC_SCRATCH_BYTES (32u << 20)

/* mc_run for callers that cannot allocate device memory: applications that hand all device memory
 * to their own pool or allocator up front (a further cudaMalloc fails or steals from the pool),
 * allocator or memory-pressure callbacks that must not re-enter the allocator, and hosts that fix
 * their device-memory budget at start-up.  This call takes no memory from cudaMalloc, cudaFree or any allocating
 * library: its control block, particle banks (32768 particles each), batch tallies and statistics
 * live in one MC_STATIC_SCRATCH_BYTES array that the library declares at file scope, reserved on
 * every GPU that loads the library until the process exits.  The paper has no counterpart; it is
 * an interface for such callers only.
 *   p            problem from mc_problem_create (created beforehand, outside the restricted code)
 *   n_histories, seed, opts   as for mc_run; opts may not ask for an event log, more than 32768
 *                particles in flight, fewer than 1024 (a non-zero bank_capacity below 1024), or
 *                tally_stripes > 1 (MC_ERR_INVALID)
 *   mean, std_err  DEVICE arrays of the problem's device (8-byte aligned; host, misaligned or
 *                other-device pointers are MC_ERR_INVALID before any launch) of at least the
 *                problem's total bin count (every mesh tally's
 *                bins in tally order, then the leakage bins), caller-allocated; they receive the
 *                per-source-particle mean and standard error, or NaN in every entry if the run
 *                failed on the device (bank overflow, watchdog, lost particle)
 * The tallies must fit the scratch: (n_batches + 3) x bins x 8 bytes plus the banks; larger
 * problems are rejected with MC_ERR_INVALID and a message giving the bytes needed.  Asynchronous on
 * `stream`.  The first call on a device looks up the array's device address (a runtime query, no
 * allocation) with that device current; make that first call before any stream capture.  Every
 * call shares the one array, which keeps the last call's contents (the call clears what must start
 * at zero): calls that overlap on the GPU, e.g. on two streams, race and corrupt each other. */
int mc_run_static(const mc_problem* p, uint64_t n_histories, uint64_t seed, const mc_run_opts* opts,
                  double* mean, double* std_err, void* stream);

/* ------------------------------------------------------------------------- batched launch */
/* Runs n independent problems (n <= 65536) in one persistent launch, replayed from a CUDA graph
 * that the library captures once per launch shape.  Problem i runs histories [0, n_hist[i]) with
 * the seed `seed + i`: exactly the particles that mc_run(ps[i], n_hist[i], seed + i, o) transports,
 * so fixed-point tallies and event counters equal those of n separate runs bit for bit.
 *   Scheduling: the histories of every problem are cut into work units of o->batch_unit
 *   consecutive histories; problems are ordered by geometry kind (plain cells, then lattices, so
 *   that concurrent warps mostly run the same code) and by ascending n_hist within a kind (short
 *   problems finish first).
 *   Every warp of the grid claims units one at a time, stages the unit's problem tables in its own
 *   slice of shared memory (only when the problem changes), and carries the unit's particles and
 *   all their secondaries to completion; a warp claims the next unit of the same problem before its
 *   lanes run dry.  Secondaries and weight-window copies wait in a warp-private stack of
 *   o->bank_capacity particles (0 = 2048) in device memory; no CTA waits for another, so the
 *   launch has no grid barrier.
 *   Options apply to every problem (precision, tally_mode, fixed_bits, n_batches, ww_enable,
 *   aggregate_atomics, max_iterations as the per-particle event budget); algorithm, event logging,
 *   first_history, tally_stripes and drain_threshold do not apply.  block_size, blocks_per_sm and
 *   batch_unit left at 0 take the configuration mc_batch_tune stored for a batch of the same
 *   shape, else 256 threads, as many CTAs per SM as fit, 128 histories.
 *   Results are read per problem with mc_tally_get, mc_tally_batches, mc_counters_get; mc_wait on
 *   a problem returns that problem's device error (bank overflow, watchdog, lost particle), which
 *   stops its remaining units but not the other problems'.  mc_run_timing on a problem gives the
 *   span from its first claimed unit to its last finished particle (device clock) as transport
 *   time.
 *   Asynchronous on `stream`, unless per_problem_wall_s is non-NULL: then the call synchronises and
 *   writes, for each problem, the seconds from the start of the launch until its last particle
 *   finished.  The problems must live on the current device and be distinct. */
int mc_run_batch(mc_problem* const* ps, int n, const uint64_t* n_hist, uint64_t seed,
                 const mc_run_opts* o, void* stream, double* per_problem_wall_s);

/* Autotuner of mc_run_batch: runs the batch (seed, o) under each candidate configuration (block
 * size 128 or 256; the 80- or 128-register build of the kernel; units of 32 to 512 histories),
 * times each launch with CUDA events (best of two after a warm-up), and stores the fastest for
 * every later batch of the same shape (problem count, precision, tally mode, batches, and per
 * problem its group count, geometry kind, bin count and history count rounded to a power of 2).
 * tuned (nullable) receives a copy of o with block_size, blocks_per_sm and batch_unit set;
 * best_ms (nullable) the launch time of that configuration, in ms.  Synchronises.  The tallies
 * left behind are those of the last candidate run. */
int mc_batch_tune(mc_problem* const* ps, int n, const uint64_t* n_hist, uint64_t seed,
                  const mc_run_opts* o, void* stream, mc_run_opts* tuned, double* best_ms);

/* Measures the device's L2 atomic throughput for the scoring access pattern: 64-bit atomic adds
 * to pseudo-random slots of a zeroed array of `span` elements (1 .. 2^27), issued by 8 CTAs of
 * 256 threads per SM; *atomics_per_s receives adds per second.  Allocates and frees its array.
 * Used as the atomic roofline of track-length scoring. */
int mc_atomic_peak(uint64_t span, double* atomics_per_s);

/* Instruction throughput on the current GPU, in operations per SM clock per SM (a measurement tool
 * like mc_atomic_peak; it explains why the FP32 walk keeps FP64 work off its path): out[0] FP32 FMA,
 * [1] FP64 add, [2] 32-bit umulhi (with an add), [3] int -> float conversion, [4] float -> int64
 * conversion, [5] __logf (with an add); four independent chains per thread, 8 CTAs of 256 threads
 * per SM.  n >= 6.  Synchronous. */
int mc_op_rates(double* ops_per_clk_per_sm, int n);

/* Philox4x32-10 (Salmon et al., SC'11) on the device: out[i] = Philox(key = seed, ctr = ctr[i])
 * for n counters; ctr and out are DEVICE arrays of 4*n uint32 (counter words c0..c3).  This is
 * the generator every random draw of the walk uses, exposed for verification. */
int mc_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, uint64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MCGB_MC_H */
