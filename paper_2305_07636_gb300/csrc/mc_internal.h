// Internal layout shared by the host half (mc_api.cu) and the device half (mc_transport.cu) of
// libmcgb.  Not part of the public ABI.
#pragma once
#include <stdint.h>

#include "../../include/mc.h"

namespace mcgb {

constexpr int kMaxTallies = MC_MAX_TALLIES;
constexpr int kSurfStride = 16;   // table values per surface (plane / cylinder, quadric, centre)
constexpr int kMaxLanes = 6;      // 16-byte state lanes per particle (FP64 layout)
constexpr int kLanesFP32 = 4;     // 64 B per particle
constexpr int kLanesFP64 = 6;     // 96 B per particle
// per-warp shared memory of the transport kernels: flight queue slots and tally staging entries
// (8-byte value + 4-byte slot each)
constexpr unsigned kWarpQ = 64;
constexpr unsigned kStage = 128;
// segments waiting to be scored: records per warp (31 waiting + 32 new from one flight round; a
// scoring pass puts back at most as many as it took) of kSegLanes 16-byte lanes, in a per-warp
// region of shared memory (the persistent kernel) or device memory (the batched kernel)
constexpr unsigned kSegCap = 64;
constexpr int kSegLanes = 4;
constexpr uint32_t kSourceEvent = 0xFFFFFFFFu;
constexpr uint32_t kChildMark = 0x80000000u;
constexpr uint32_t kSplitMark = 0xC0000000u;
constexpr uint32_t kChildKeyXor = 0xA5A5A5A5u;

// ---- `elem` word: bits 0-15 lattice element (iz ny + iy) nx + ix, 16-31 statistical batch
// ---- packed per-particle word (lane 3 .w in FP32, lane 4 .w in FP64)
//   bits 0-4   group (G <= 32)
//   bits 5-12  cell index
//   bit  13    inside the pin of the current lattice element
//   bits 14-15 pending event: 0 none (needs a flight), 1 collision, 2 surface
//   bits 16-17 surface hit type: 0 cell surface, 1 lattice wall, 3 pin
//   bit  18    lattice wall direction (1 = +1, 0 = -1)
//   bits 19-26 index of the crossed cell surface, or the axis of the crossed lattice wall (0 x, 1 y, 2 z)
//   bits 27-28 channel of a pending collision (drawn with the flight): 0 scatter, 1 production
enum : uint32_t { PEND_NONE = 0, PEND_COLL = 1, PEND_SURF = 2 };
enum : uint32_t { CHAN_SCATTER = 0, CHAN_PRODUCTION = 1, CHAN_CAPTURE = 2 };
enum : uint32_t { HIT_CELL = 0, HIT_LAT = 1, HIT_PIN = 3 };
constexpr uint8_t kNoPin = 0xFF;

// Bounds-checked build (libmcgb_checked.so, compiled with -DMCGB_CHECKED): the walk checks every
// index it computes into the tables, the tallies and the lattice's element map before use; a bad
// one records MC_ERR_BOUNDS in the run's status, the access is skipped and the particle ends.  It
// stands in for a memory checker.  In the normal build the checks are constant-true.
#ifdef MCGB_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif  // pin map entry of an element without a pin (materials are < 255)

__host__ __device__ inline uint32_t pk_g(uint32_t w) { return w & 0x1Fu; }
__host__ __device__ inline uint32_t pk_cell(uint32_t w) { return (w >> 5) & 0xFFu; }
__host__ __device__ inline uint32_t pk_pin(uint32_t w) { return (w >> 13) & 1u; }
__host__ __device__ inline uint32_t pk_pend(uint32_t w) { return (w >> 14) & 3u; }
__host__ __device__ inline uint32_t pk_hit(uint32_t w) { return (w >> 16) & 3u; }
__host__ __device__ inline int pk_dir(uint32_t w) { return ((w >> 18) & 1u) ? 1 : -1; }
__host__ __device__ inline uint32_t pk_surf(uint32_t w) { return (w >> 19) & 0xFFu; }
__host__ __device__ inline uint32_t pk_chan(uint32_t w) { return (w >> 27) & 3u; }
__host__ __device__ inline uint32_t pk_set_chan(uint32_t w, uint32_t c) { return (w & ~(3u << 27)) | ((c & 3u) << 27); }
__host__ __device__ inline uint32_t pk_make(uint32_t g, uint32_t cell, uint32_t pin) {
  return (g & 0x1Fu) | ((cell & 0xFFu) << 5) | ((pin & 1u) << 13);
}
__host__ __device__ inline uint32_t pk_set_pending(uint32_t w, uint32_t pend, uint32_t hit,
                                                   int dir, uint32_t surf) {
  w &= 0x3FFFu;
  return w | (pend << 14) | (hit << 16) | ((dir > 0 ? 1u : 0u) << 18) | ((surf & 0xFFu) << 19);
}

// ---- per-problem table blob: header followed by typed arrays, all 16-byte aligned.  `Real`
// arrays are float in FP32 mode and double in FP64 mode; time edges are always double.
struct TallyDesc {
  int nx, ny, nz, nt;
  int o_ex, o_ey, o_ez, o_et;  // byte offsets of the edge arrays
  int bin_offset;              // first bin of this tally in the concatenated bin space
  int n_bins;
  int o_etf;                   // time edges rounded to float (FP32 tracking)
  int range;                   // 1: scored by the range walk (full time bins as difference marks)
  int est;                     // MC_EST_TRACK_LENGTH or MC_EST_TIME_CROSSING
  int nval;                    // values per (cell, group) along time: nt bins or nt + 1 points
  int diff_offset;             // range walk: first difference slot after the batch row's bins
  int ndiff;                   // range walk: difference slots per (cell, group): nt + 1 (track
                               // length) or nt + 2 (time crossing)
  // First guess of a segment's starting bin along x, y, z, t from the float edges (FP32 walk):
  // kind 0 none (bisection); 1 equal spacing, bin floor((u - a) b); 2 geometric from edge 1 on,
  // bin 1 + floor(log2(u a) b) (bin 0 below edge 1).  The guess is corrected against the edges,
  // so the bin found is the one bisection finds whatever the spacing.
  int gkind[4];
  float ga[4], gb[4];
};

// A tally is scored by the range walk when its time axis is much finer than its spatial mesh
// (flights then cross many more time edges or points than mesh planes).
inline bool ranges_time_bins(int nx, int ny, int nz, int nt) { return nt >= 3 && nt >= 4 * (nx + ny + nz); }

struct TableHeader {
  int G, M, n_surf, n_cell;
  int has_lat, lat_nx, lat_ny, lat_matrix;
  int n_tally, total_bins, leak_offset, real_bytes;
  int src_pos, src_dir, total_diff, pad1;  // total_diff: difference slots after the bins of a row
  double t_census;
  double src_lo[3], src_hi[3], src_t0, src_t1;
  double lat_x0, lat_y0, lat_pitch, lat_r;
  double lat_z0, lat_pz;                  // axial layers (lat_nz >= 2): bottom and height
  unsigned long long lat_mx, lat_my;      // ceil(2^32 / nx), ceil(2^32 / ny): element index division
  // float copies for FP32 tracking (no double->float conversion on the device)
  float src_lo_f[4], src_hi_f[4];
  float src_t0_f, src_t1_f, tc_hi, tc_lo;  // census time as the float pair hi + lo
  int has_census, lat_nz, pad6, pad7;  // lat_nz: axial layers (1: one layer, unbounded in z)
  // byte offsets
  int o_st, o_ss, o_ssf, o_nu;        // [M][G] Real: sigma_t, scatter threshold, scatter+production threshold, nu
  int o_v, o_inv_v, o_scdf, o_chi;    // [G] Real speed, 1/speed; [M][G][G] scatter CDF; [M][G] chi CDF
  int o_src_cdf, o_skind, o_sbc, o_scoef;  // [G] Real; [n_surf] int; [n_surf] int; [n_surf][16] Real
  int o_nhs, o_hs, o_cmat, o_lpin;    // [n_cell] int; [n_cell][16] int (surf | sense<<16); [n_cell] int;
                                      // [nz][ny][nx] uint8 pin material (kNoPin = no pin)
  TallyDesc tally[kMaxTallies];
  int blob_bytes, o_nusf, o_cbox, pad4;  // o_nusf: [M][G] Real nu Sigma_f (k-eigenvalue estimator)
  // o_cbox: [n_cell][7] int: 1 for a cell bounded by axis-aligned planes only, at most one lower
  // and one upper plane per axis; then per axis its lower and upper plane as surface | (position
  // in the cell's halfspace list << 16), or -1
};

// Factor that turns a bin's accumulated score into the tally value: v_g for a time-crossing bin
// (the device accumulates the weight w of a particle at a time point; its flux score is w v_g),
// 1 otherwise.  `blob` is the FP64 table blob (speeds stored as double).
__host__ __device__ inline double bin_value_factor(const char* blob, uint64_t bin) {
  const TableHeader* H = reinterpret_cast<const TableHeader*>(blob);
  for (int t = 0; t < H->n_tally; ++t) {
    const TallyDesc& D = H->tally[t];
    if (bin >= (uint64_t)D.bin_offset && bin < (uint64_t)D.bin_offset + (uint64_t)D.n_bins) {
      if (D.est != MC_EST_TIME_CROSSING) return 1.0;
      const int g = (int)(((bin - (uint64_t)D.bin_offset) / (uint64_t)D.nval) % (uint64_t)H->G);
      return reinterpret_cast<const double*>(blob + H->o_v)[g];
    }
  }
  return 1.0;
}

// ---- device control block, one per problem
struct Ctl {
  // rotated per iteration (mod 3): the next transport bank's fill (collision-pending particles from
  // the front in the low 32 bits, surface-pending ones from the back in the high 32 bits; cap_s <
  // 2^32), the birth bank's fill and the first history not yet started
  unsigned long long fb[3], birth[3], hstart[3];
  unsigned long long splits[3];  // weight-window split copies counted in the iteration (rotated too)
  unsigned long long next[3];                                 // dynamic item claim counters
  unsigned int bar_count, bar_gen;
  int status, pad;
  unsigned long long counters[MC_NCOUNTERS + 1];
  unsigned long long log_n;
  unsigned long long iterations;
  unsigned long long t_start, t_end;  // %globaltimer at kernel start / end (ns)
  unsigned long long k_acc;           // k-eigenvalue cycle: sum of fixed(w l nu Sigma_f 2^32)
  unsigned long long pc_n;            // particles banked at this launch's interior census
  unsigned long long tail_it;         // split run: the iteration the history-style tail launch starts at
};

struct RunParams {
  uint4* S[2][kMaxLanes];  // ping-pong transport banks (front: pending collision, back: surface)
  uint4* B[2][kMaxLanes];  // ping-pong birth banks (sources' children, split copies)
  uint64_t cap_s, cap_b;
  Ctl* ctl;
  int* sticky;             // first error of any run since the host last read it
  uint32_t tally_stripes;  // copies of the batch tallies; CTA b scores into copy b % stripes
  uint32_t pad_ts;
  uint64_t stripe_stride;  // elements per copy (n_batches * row)
  uint64_t row;            // elements per batch row: total_bins, then total_diff difference slots
  void* tally;             // [stripes][n_batches][row] int64 (fixed point) or double
  int tally_fp64, aggregate;
  double fixed_scale;      // 2^fixed_bits
  float fixed_scale_f;
  int history_mode;        // 1: every iteration runs its particles to completion (no write-back)
  uint64_t drain_threshold;// event mode: finish the run history-style once all histories are
                           // sourced and at most this many particles remain
  unsigned long long* trace;  // per iteration: globaltimer, items, sources|drain<<63
  uint64_t trace_cap;
  uint64_t n_hist, hist_per_batch, h_first;
  uint32_t batch_magic, pad_bm;  // floor(2^32 nb / N) (clamped), for the batch index
  int n_batches, blob_bytes;
  uint64_t seed;
  const uint4* blob;
  uint64_t max_iter;
  unsigned long long spin_limit;  // barrier wait budget (polls)
  mc_event* log;
  uint64_t log_cap, log_first, log_count;
  // weight windows (optional)
  int ww_on, ww_nx, ww_ny, ww_nz;
  int ww_nt, pad_ww;
  const double* ww_edges;  // x[nx+1], y[ny+1], z[nz+1], t[nt+1]
  const double* ww_center; // [nt][nz][ny][nx][G]
  double ww_upper, ww_lower;
  int ww_split_max;
  int implicit;            // implicit capture with a weight-cutoff roulette
  double wr_cutoff, wr_survival;
  // histories this launch starts (n_hist, or 0 for a population-control interval after the first)
  uint64_t n_sources;
  // census of this launch: time (double and float pair), and whether it is an interior census of
  // population control (reached particles go to the census bank C instead of ending)
  int has_census, pc_interior;
  float tc_hi, tc_lo;
  double tc;
  uint4* C[kMaxLanes];
  uint64_t cap_c;
  // k-eigenvalue cycle (eigen = 1): sources come from src_site[h] (cycle >= 1), production banks
  // floor(nu inv_k + xi) fission sites at site_next[h * nmax + j] with count_next[h], every flight
  // adds fixed(w l nu Sigma_f) to Ctl::k_acc, tallies are scored only when eigen_score, into batch
  // row batch_fixed; particle tags are (h, cycle)
  int eigen, eigen_score;
  uint32_t cycle, batch_fixed;
  uint32_t nmax, pad_e;
  double inv_k;
  const uint4* src_site;   // [N] sites of this cycle's sources (cycle >= 1)
  uint4* site_next;        // [N * nmax] sites banked this cycle
  uint32_t* count_next;    // [N] sites banked by each history (zeroed before the cycle)
  // FP32 tracking, plain-walk tallies only: 1 = flown segments wait in a per-warp region of shared
  // memory and are scored 32 at a time; 0: every flight is scored at once
  int seg, pad_seg;
  // split run (event-based launch, then a history-style tail launch): per-warp stacks of the tail's
  // secondaries, lane l of warp w's slot j at WS[l][w * ws_cap + j]; nullptr: one launch
  uint4* WS[kMaxLanes];
  unsigned long long ws_cap;
};

// fission sites: FP32 tracking 1 x 16 B (x, y, z, g), FP64 2 x 16 B ((x, y), (z, g))
constexpr int kSiteLanesFP32 = 1, kSiteLanesFP64 = 2;

}  // namespace mcgb
