/*
 * CPU oracle for the multigroup, time-dependent Monte Carlo random walk.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library.  It shares no code, header, table or constant generator
 * with the CUDA path; the two meet only in the seeded problem dicts.
 *
 * What it computes: the analog history-based random walk of the paper's Section 3 problem class
 * (fixed source, multigroup, quadric CSG -- planes, cylinders, spheres, general quadrics -- plus
 * a square pin lattice with optional axial layers,
 * time-dependent source, time census, track-length mesh tallies, secondary production), in FP64,
 * one history at a time, with the per-history variance of every tally bin.  Two variants the
 * paper's Section 3 runs use: the time-crossing estimator of the flux at time points (the
 * multigroup pulse and C5G7 transients) and implicit capture (the Kobayashi transient).  The
 * paper prints no transport equations; the steps follow textbook multigroup Monte Carlo in order
 *   distance to collision -> distance to surface -> distance to census -> move + score ->
 *   collision (scatter / production / capture) or surface (leak / reflect / transmit).
 */
#ifndef MC_ORACLE_H
#define MC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_HS 16

/* surfaces: planes x/y/z = c; cylinders parallel to z, x, y; spheres; general quadrics
 * A x^2 + B y^2 + C z^2 + D xy + E yz + F zx + G x + H y + I z + J = 0 */
enum { OR_PX = 0, OR_PY = 1, OR_PZ = 2, OR_CZ = 3, OR_CX = 4, OR_CY = 5, OR_SQ = 6, OR_GQ = 7 };
enum { OR_INTERIOR = 0, OR_VACUUM = 1, OR_REFLECT = 2 };
enum { OR_SRC_BOX = 0, OR_SRC_SURFACE_X0 = 1 };
enum { OR_DIR_ISO = 0, OR_DIR_BEAM_X = 1, OR_DIR_COS_X = 2 };
enum { OR_EV_COLLISION = 0, OR_EV_SURFACE = 1, OR_EV_CENSUS = 2, OR_EV_LOST = 3 };
/* tally estimators: track length over time bins, or the time-crossing estimator at time points */
enum { OR_EST_TRACK = 0, OR_EST_CROSSING = 1 };

/* counters, summed over all histories */
enum {
  OR_C_SOURCE = 0,      /* primaries started */
  OR_C_SECONDARY,       /* children produced by the production channel */
  OR_C_CAPTURE,         /* removed by capture */
  OR_C_PRODUCTION,      /* removed by the production channel (parent absorbed) */
  OR_C_LEAK,            /* removed through a vacuum surface */
  OR_C_CENSUS,          /* removed at the census time */
  OR_C_LOST,            /* removed because no cell contained the particle */
  OR_C_FLIGHT,          /* flights */
  OR_C_COLLISION,       /* collisions */
  OR_C_SCATTER,         /* scatters */
  OR_C_SURFACE,         /* surface events (including lattice walls and pins) */
  OR_C_REFLECT,         /* reflections */
  OR_C_WW_SPLIT,        /* extra particles created by weight-window splitting */
  OR_C_WW_KILL,         /* particles removed by roulette (weight windows or weight cutoff) */
  OR_C_PC_BANKED,       /* particles stopped at an interior census (population control) */
  OR_C_PC_COPIES,       /* particles started after an interior census by splitting-roulette */
  OR_NCOUNT
};

typedef struct {
  int G, M;
  const double* sigma_t;   /* [M][G] */
  const double* sigma_s;   /* [M][G][G], from -> to */
  const double* sigma_f;   /* [M][G] */
  const double* nu;        /* [M][G] */
  const double* chi;       /* [M][G] */
  const double* speed;     /* [G] */
  int n_surf;
  const int* surf_kind;    /* [n_surf] OR_PX.. */
  const double* surf_coef; /* [n_surf][10]: plane c; z-cylinder x0, y0, r; x-cylinder y0, z0, r;
                              y-cylinder x0, z0, r; sphere x0, y0, z0, r; quadric A..J */
  const int* surf_bc;      /* [n_surf] */
  int n_cell;
  const int* cell_nhs;     /* [n_cell] */
  const int* cell_hs_surf; /* [n_cell][OR_MAX_HS] */
  const int* cell_hs_sense;/* [n_cell][OR_MAX_HS] +1 / -1 */
  const int* cell_mat;     /* [n_cell], -1 = filled by the lattice */
  int has_lattice, lat_nx, lat_ny;
  double lat_x0, lat_y0, lat_pitch, lat_r;
  const int* lat_pin_mat;  /* [nz][ny][nx] (nz = 1 when lat_nz <= 1), -1 = no pin */
  int lat_matrix;
  int lat_nz;              /* axial layers; <= 1: one layer, unbounded in z */
  double lat_z0, lat_pitch_z;
  int src_pos, src_dir;
  double src_lo[3], src_hi[3];
  const double* src_group_pdf; /* [G] */
  double src_t0, src_t1;
  int n_tally;
  const int* tally_dims;   /* [n_tally][4]: nx, ny, nz, nt */
  const double* tally_edges; /* per tally: x[nx+1], y[ny+1], z[nz+1], t[nt+1] */
  double t_census;
  /* weight windows: centre w_c per (cell of the ww mesh, group); 0 disables */
  int ww_on;
  int ww_nx, ww_ny, ww_nz;
  const double* ww_edges;  /* x[ww_nx+1], y[ww_ny+1], z[ww_nz+1] */
  const double* ww_center; /* [ww_nz][ww_ny][ww_nx][G] */
  double ww_upper, ww_lower; /* split above upper*w_c, roulette below lower*w_c */
  int ww_split_max;
  /* per tally: OR_EST_TRACK (nt time bins between the nt+1 edges) or OR_EST_CROSSING (values at
   * the nt+1 time points themselves); NULL means every tally is a track-length tally */
  const int* tally_est;
  /* time bins of the weight windows: ww_center is [ww_nt][ww_nz][ww_ny][ww_nx][G] and a particle
   * takes the window of the time bin t[i] <= t < t[i+1] holding its time; ww_nt <= 1 or NULL edges:
   * one bin holding every time */
  int ww_nt;
  const double* ww_tedges; /* t[ww_nt+1] */
} or_problem;

typedef struct {
  uint64_t tag, root;
  uint32_t k;
  int32_t kind, outcome, n_child, cell, elem, in_pin, g;
  double x, y, z, ux, uy, uz, t, w;
} or_event;

/* outcome codes: collision 0 scatter, 1 production, 2 capture;
 * surface 0 transmit, 1 reflect, 2 leak, 3 lattice wall, 4 pin */

typedef struct {
  uint64_t first_history, n_histories, seed;
  int threads;
  uint64_t log_first, log_count; /* histories [log_first, +log_count) are logged */
  or_event* log;                 /* caller buffer, may be NULL */
  uint64_t log_cap;
  uint64_t* log_n;               /* events written (clipped to log_cap) */
  int fixed_bits;                /* fixed-point scale 2^fixed_bits for the int64 sums */
  /* implicit capture: collisions never capture; the weight is multiplied by the non-capture
   * probability (Sigma_s + Sigma_f) / Sigma_t and the channel is drawn among scatter and
   * production; a particle whose weight falls below wr_cutoff after a scatter survives a
   * roulette with probability w / wr_survival at weight wr_survival */
  int implicit_capture;
  double wr_cutoff, wr_survival;
} or_opts;

/* Outputs are laid out over all tallies' bins concatenated (tally 0 first, bins in
 * [z][y][x][g][t] order; a time-crossing tally has nt+1 time values), followed by n_surf leakage
 * bins.  s1 = sum over histories of the history's score, s2 = sum of its square; fixed = sum of
 * llrint(score_piece * 2^fixed_bits), where a time-crossing score piece counts its weight w
 * (its flux score is w v). */
typedef struct {
  double* s1;
  double* s2;
  int64_t* fixed;
  int64_t counters[OR_NCOUNT];
} or_result;

int or_total_bins(const or_problem* p);
int or_run(const or_problem* p, const or_opts* o, or_result* r);

/* Time-dependent run with population control at interior census times (the paper's Section 3
 * feature list: time census with population control).  The histories are split into n_batches
 * contiguous batches (history h in batch floor(h nb / N)), and each batch is an independent
 * simulation of its N_b histories.  Interval i runs from the previous census (or the source) to
 * census_times[i] (the problem's t_census after the last one): every particle and its secondaries
 * are transported; one reaching an interior census is banked.  Then, per batch, splitting-roulette:
 * W_b = sum of llrint(w 2^40) over the batch's banked particles (exact), w_t = W_b 2^-40 / N_b, and a
 * banked particle of weight w (tag T, census flight k) becomes floor(w / w_t + xi) copies, xi = the
 * first FP64 uniform of block 1 of event k, copy j with tag child_tag(T, k, 0x40000000 | j), weight
 * w_t, time = the census time exactly, event index 0, the same position, direction and group.  The
 * copies start the next interval.  Tallies are returned per batch (tally_batch[b][bin], per source
 * particle of the batch).
 * method 1 combs instead (systematic sampling of the census bank): the batch's banked particles are
 * ordered by tag, C_j = the running sum of llrint(w 2^40) up to and including particle j, W_b = C_M,
 * and with F(C) = min(N_b, max(0, ceil(C N_b / W_b - xi_b))) (FP64, each operation rounded in this
 * order; xi_b = the first FP64 uniform of block 5 of event i of tag 0xFFFFFFFE + 2^32 b, i the
 * census index) particle j becomes F(C_j) - F(C_{j-1}) copies (the N_b teeth (k + xi_b) W_b / N_b
 * that fall in its weight interval), each as above. */
typedef struct {
  uint64_t n_histories, seed;
  int n_batches, threads;
  int n_census;
  const double* census_times;    /* [n_census], increasing, below the problem's t_census */
  uint64_t log_first, log_count;
  or_event* log;
  uint64_t log_cap;
  uint64_t* log_n;
  int method;                    /* 0 splitting-roulette, 1 combing */
} or_pc_opts;

typedef struct {
  double* tally_batch;           /* [n_batches][total bins] */
  uint64_t* banked;              /* [n_census] particles banked at each interior census (all batches) */
  int64_t counters[OR_NCOUNT];
} or_pc_result;

int or_run_pc(const or_problem* p, const or_pc_opts* o, or_pc_result* r);

/* The comb of method 1 applied to n weights in the given order: out[j] = copies of weight j
 * (exposed for the pins). */
void or_comb_counts(const double* w, int64_t n, uint64_t Nb, double xi, int64_t* out);

/* k-eigenvalue power iteration (the paper's C5G7 runs, Section 3), analog: n_inactive + n_active
 * cycles of n_per_cycle histories.  Cycle 0 starts at the problem's source; cycle c >= 1 starts
 * history h (tag h + 2^32 c) at site floor((h + u0) M / N) of the previous cycle's M fission sites
 * (systematic sampling; u0 = first uniform of Philox(seed, (2^32 - 1, c, 2^32 - 1, 4))), with an
 * isotropic direction from its source draws (blocks 1, 2), the site's group, t = 0, w = 1.  A
 * production event banks floor(nu / k + xi) sites (k = the previous cycle's estimate, 1 before
 * cycle 0; groups from chi by each child tag's source draw) instead of transporting secondaries.
 * Sites are ordered by producing history, then production order.  k of a cycle is the
 * track-length estimate: sum over flights of w l nu Sigma_f, divided by N, summed in int64 fixed
 * point at 2^-32 (llrint per flight) so that it does not depend on the thread count.  Tallies are
 * scored in active cycles only. */
typedef struct {
  uint64_t n_per_cycle, seed;
  int n_inactive, n_active, threads, fixed_bits;
  uint64_t log_first, log_count; /* histories [log_first, +log_count) of every cycle are logged */
  or_event* log;
  uint64_t log_cap;
  uint64_t* log_n;
} or_eigen_opts;

typedef struct {
  double* k_cycle;       /* [n_inactive + n_active] */
  uint64_t* sites_cycle; /* [n_inactive + n_active] fission sites banked in each cycle */
  double* tally_cycle;   /* [n_active][total bins]: each active cycle's tallies per source particle */
  int64_t counters[OR_NCOUNT]; /* summed over all cycles; OR_C_SECONDARY counts banked sites */
} or_eigen_result;

/* 0 on success; -1 for bad options; -2 if a cycle banked no fission site. */
int or_run_eigen(const or_problem* p, const or_eigen_opts* o, or_eigen_result* r);

/* unit-level entry points used by the tests */
void or_philox(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4]);
double or_u01(uint32_t a, uint32_t b);
double or_dist_cylinder(double x, double y, double ux, double uy, double x0, double y0, double r,
                        int inside);
double or_dist_plane(double pos, double u, double c, int sense);
/* distance to surface s of the problem from (x,y,z) along (ux,uy,uz) for a particle in its
 * half-space `sense` (the distance at which it leaves that half-space; inf if never) */
double or_dist_surface(const or_problem* p, int s, double x, double y, double z, double ux, double uy, double uz,
                       int sense);
/* source sample of history h: writes x,y,z,ux,uy,uz,t and group; returns cell or -1 */
int or_source_sample(const or_problem* p, uint64_t seed, uint64_t h, double out[7], int* g);
/* cell of the point (x, y, z); skip >= 0: the point was reached by crossing surface `skip`,
 * flying along (ux, uy, uz), and lies on it with sense skip_sense afterwards; -1 if no cell
 * holds it */
int or_find_cell(const or_problem* p, double x, double y, double z, int skip, int skip_sense, double ux,
                 double uy, double uz);
/* sample a scatter group for material m, group g at uniform u */
int or_sample_scatter_group(const or_problem* p, int m, int g, double u);
/* derive the tag of child j produced at event k by a parent */
uint64_t or_child_tag(uint64_t seed, uint64_t parent, uint32_t k, uint32_t j, uint32_t marker);

/* Reference MLP for the weight-window map: 5 -> H -> H -> H -> 1, tanh hidden units, FP64.
 * params = [W1 (H x 5), b1 (H), W2 (H x H), b2, W3 (H x H), b3, W4 (1 x H), b4].
 * Forward over n inputs x[n][5] -> y[n]; loss = mean over n of wt[i] (y - target)^2;
 * grad receives d loss / d params. */
int or_mlp_param_count(int H);
double or_mlp_loss_grad(int H, const double* params, int n, const double* x, const double* target,
                        const double* wt, double* y, double* grad);

#ifdef __cplusplus
}
#endif
#endif
