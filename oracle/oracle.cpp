// CPU oracle for the multigroup, time-dependent Monte Carlo random walk.
//
// TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU-baseline leg of the
// benchmark, never by the product path.  Plain FP64, one history at a time, no blocking or
// reordering beyond what the method states.  Shares nothing with the CUDA path.
//
// The paper (MC/DC, Section 3) names the problem class -- fixed-source multigroup transport on
// quadric-surface CSG, time-dependent source, time census, time-dependent mesh tallies with the
// track-length estimator (Section 3.1), secondary production (the supercritical AZURV1 case of
// Section 3) -- but prints no transport equations.  The steps here are textbook analog multigroup
// Monte Carlo, in this order per flight:
//   1. distance to collision  d_c = -ln(xi) / Sigma_t[m][g]
//   2. distance to the nearest bounding surface d_s (planes, quadrics, lattice walls and pins)
//   3. distance to census     d_t = v[g] (t_census - t)
//   4. l = min(...), move, score w * l into the (x, y, z, g, t) mesh (track-length estimator)
//   5. collision: scatter (g' by CDF of the Sigma_s row, isotropic), production
//      (floor(nu + xi) children, g' ~ chi, isotropic; parent absorbed) or capture;
//      surface: leak (vacuum), reflect (flip the normal component) or move to the next cell.
// Variants used by the paper's Section 3 runs: the time-crossing estimator (the flux at time
// points t_j: every particle alive at t_j scores w v into the mesh cell it occupies then) and
// implicit capture (no capture channel; the weight carries the survival probability, and a
// weight-cutoff roulette ends histories).
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11) keyed by the seed, with the counter (tag, event index, block).
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double INF = std::numeric_limits<double>::infinity();
const double TWO_PI = 6.283185307179586476925286766559;
const uint32_t SOURCE_EVENT = 0xFFFFFFFFu;
const uint32_t CHILD_MARK = 0x80000000u;
const uint32_t SPLIT_MARK = 0xC0000000u;

// ---------------------------------------------------------------- Philox4x32-10 (SC'11 paper)
void philox(uint32_t k0, uint32_t k1, uint32_t c[4]) {
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// uniform on the open interval (0,1) from 52 random bits: ((a >> 6) 2^26 + (b >> 6) + 1/2) 2^-52.
// With 52 bits the half-offset stays exact, so the largest value is 1 - 2^-53 < 1.
double u01(uint32_t a, uint32_t b) {
  return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 4503599627370496.0);
}

struct Pair {
  double a, b;
};

// two uniforms of block `block` of event `k` of the particle with tag `tag`
Pair draw(uint64_t seed, uint64_t tag, uint32_t k, uint32_t block) {
  uint32_t c[4] = {(uint32_t)tag, (uint32_t)(tag >> 32), k, block};
  philox((uint32_t)seed, (uint32_t)(seed >> 32), c);
  return {u01(c[0], c[1]), u01(c[2], c[3])};
}

uint64_t child_tag(uint64_t seed, uint64_t parent, uint32_t k, uint32_t j, uint32_t marker) {
  uint32_t c[4] = {(uint32_t)parent, (uint32_t)(parent >> 32), k, marker | j};
  philox((uint32_t)seed ^ 0xA5A5A5A5u, (uint32_t)(seed >> 32), c);
  return (uint64_t)c[0] | ((uint64_t)c[1] << 32);
}

// ---------------------------------------------------------------- problem copy
struct Tally {
  std::vector<double> e[4];  // x, y, z, t edges (time points for a time-crossing tally)
  int n[4];
  int est;     // OR_EST_TRACK or OR_EST_CROSSING
  int nval;    // values per (cell, group) along time: n[3] bins, or n[3] + 1 points
  int offset;  // first bin in the concatenated output
};

// how one history is transported: analog, or with implicit capture and a weight cutoff
struct Physics {
  bool implicit;
  double cutoff, survival;
};

// k-eigenvalue cycle state of one history: production banks fission sites for the next cycle
// (floor(nu / k + xi) of them, k the previous cycle's estimate) instead of transporting
// secondaries; every flight adds w l nu Sigma_f to the track-length estimate of k
struct Site {
  double x, y, z;
  int g;
};
struct Eig {
  double inv_k;             // 1 / k of the previous cycle
  bool score;               // tallies are scored (active cycles)
  std::vector<Site>* sites; // this history's sites, in the order they are produced
  int64_t ktl;              // sum of llrint(w l nu Sigma_f 2^32) over this thread's flights: an
                            // exact integer sum, so k does not depend on the thread count
};

// A quadric surface written about a centre point c: with (X, Y, Z) = p - c,
// f = A X^2 + B Y^2 + C Z^2 + D XY + E YZ + F ZX + G X + H Y + I Z + J.  Cylinders and spheres are
// centred on their axis or centre (g = 0, J = -r^2), which keeps f well conditioned far from the
// origin; a general quadric is taken as given, about the origin.
struct Quad {
  double q[10];
  double c[3];
};

Quad quad_of(int kind, const double* k) {
  Quad Q{};
  switch (kind) {
    case OR_CX: Q.q[1] = Q.q[2] = 1.0; Q.q[9] = -k[2] * k[2]; Q.c[1] = k[0]; Q.c[2] = k[1]; break;
    case OR_CY: Q.q[0] = Q.q[2] = 1.0; Q.q[9] = -k[2] * k[2]; Q.c[0] = k[0]; Q.c[2] = k[1]; break;
    case OR_SQ: Q.q[0] = Q.q[1] = Q.q[2] = 1.0; Q.q[9] = -k[3] * k[3]; Q.c[0] = k[0]; Q.c[1] = k[1]; Q.c[2] = k[2]; break;
    case OR_GQ: for (int i = 0; i < 10; ++i) Q.q[i] = k[i]; break;
    default: break;
  }
  return Q;
}

// the quadric along the ray p + t u: f(t) = a t^2 + b t + c
void quad_ray(const Quad& Q, double x, double y, double z, double ux, double uy, double uz, double& a, double& b,
              double& c) {
  const double* q = Q.q;
  const double X = x - Q.c[0], Y = y - Q.c[1], Z = z - Q.c[2];
  a = q[0] * ux * ux + q[1] * uy * uy + q[2] * uz * uz + q[3] * ux * uy + q[4] * uy * uz + q[5] * uz * ux;
  b = 2.0 * (q[0] * X * ux + q[1] * Y * uy + q[2] * Z * uz) + q[3] * (X * uy + Y * ux) + q[4] * (Y * uz + Z * uy) +
      q[5] * (Z * ux + X * uz) + q[6] * ux + q[7] * uy + q[8] * uz;
  c = q[0] * X * X + q[1] * Y * Y + q[2] * Z * Z + q[3] * X * Y + q[4] * Y * Z + q[5] * Z * X + q[6] * X + q[7] * Y +
      q[8] * Z + q[9];
}

// Distance along the ray at which the particle leaves its half-space of a quadric (sense +1: f >= 0,
// -1: f < 0): the root of f(t) where f falls (sense +1) or rises (sense -1).  A root just behind
// counts as 0 where the particle is on the surface heading out of a convex section; a grazing
// entry into a convex section whose chord is shorter than 1e-12 cm is no crossing.
double dist_quadric(double a, double b, double c, int sense) {
  const double INFD = std::numeric_limits<double>::infinity();
  if (a == 0.0) {
    if (b == 0.0 || (sense > 0) == (b > 0.0)) return INFD;  // f linear along the ray, not leaving
    double t = -c / b;
    return t > 0.0 ? t : 0.0;
  }
  double disc = b * b - 4.0 * a * c;
  if (sense < 0) {  // the root where f rises: (-b + sqrt(disc)) / 2a
    if (disc < 0.0) {
      if (a > 0.0) disc = 0.0;  // inside a convex section: rounding
      else return INFD;
    }
    double sq = std::sqrt(disc);
    double t = b <= 0.0 ? (-b + sq) / (2.0 * a) : (-2.0 * c) / (b + sq);
    if (!(t > 0.0)) return a > 0.0 ? 0.0 : INFD;
    return t;
  }
  if (disc <= 0.0) return INFD;  // the root where f falls: (-b - sqrt(disc)) / 2a
  double sq = std::sqrt(disc);
  if (a > 0.0 && sq < 1e-12 * a) return INFD;
  double t = b >= 0.0 ? (-b - sq) / (2.0 * a) : (-2.0 * c) / (b - sq);
  if (!(t > 0.0)) return (a > 0.0 && b < 0.0) ? 0.0 : INFD;
  return t;
}

struct Prob {
  int G, M;
  std::vector<double> st, ss, sf, nu, chi, v;
  std::vector<double> ss_tot;    // [M][G]
  std::vector<double> scat_cdf;  // [M][G][G]
  std::vector<double> chi_cdf;   // [M][G]
  std::vector<double> src_cdf;   // [G]
  int n_surf;
  std::vector<int> skind, sbc;
  std::vector<double> scoef;   // [n_surf][10] as given
  std::vector<Quad> quad;       // surfaces other than planes and z-cylinders, as quadrics
  int n_cell;
  std::vector<int> nhs, hs_surf, hs_sense, cmat;
  bool lat;
  int lnx, lny, lnz, lmatrix;  // lnz = 1: one layer, unbounded in z (no z walls)
  double lx0, ly0, lz0, lp, lpz, lr;
  std::vector<int> lpin;       // [lnz][lny][lnx]
  int src_pos, src_dir;
  double src_lo[3], src_hi[3], t0, t1;
  std::vector<Tally> tallies;
  int total_bins;  // mesh bins; leakage bins follow
  double t_census;
  bool ww;
  std::vector<double> ww_e[4];  // x, y, z and time edges
  int ww_n[4];
  std::vector<double> ww_c;
  double ww_up, ww_lo;
  int ww_max;
};

// cumulative distribution of a non-negative row, normalised; last entry forced to exactly 1
void make_cdf(const double* row, int n, double* cdf) {
  double total = 0.0;
  for (int i = 0; i < n; ++i) total += row[i];
  double run = 0.0;
  for (int i = 0; i < n; ++i) {
    run += row[i];
    cdf[i] = total > 0.0 ? run / total : (i == n - 1 ? 1.0 : 0.0);
  }
  // index of the last positive entry gets 1 so that u < 1 always finds a bin
  int last = n - 1;
  while (last > 0 && row[last] <= 0.0) --last;
  for (int i = last; i < n; ++i) cdf[i] = 1.0;
}

int sample_cdf(const double* cdf, int n, double u) {
  for (int i = 0; i < n; ++i)
    if (u < cdf[i]) return i;
  return n - 1;
}

Prob copy_problem(const or_problem* p) {
  Prob P;
  P.G = p->G;
  P.M = p->M;
  int G = P.G, M = P.M;
  P.st.assign(p->sigma_t, p->sigma_t + M * G);
  P.ss.assign(p->sigma_s, p->sigma_s + M * G * G);
  P.sf.assign(p->sigma_f, p->sigma_f + M * G);
  P.nu.assign(p->nu, p->nu + M * G);
  P.chi.assign(p->chi, p->chi + M * G);
  P.v.assign(p->speed, p->speed + G);
  P.ss_tot.assign(M * G, 0.0);
  P.scat_cdf.assign(M * G * G, 0.0);
  P.chi_cdf.assign(M * G, 0.0);
  for (int m = 0; m < M; ++m) {
    for (int g = 0; g < G; ++g) {
      const double* row = &P.ss[(m * G + g) * G];
      double s = 0.0;
      for (int h = 0; h < G; ++h) s += row[h];
      P.ss_tot[m * G + g] = s;
      make_cdf(row, G, &P.scat_cdf[(m * G + g) * G]);
    }
    make_cdf(&P.chi[m * G], G, &P.chi_cdf[m * G]);
  }
  P.src_cdf.assign(G, 0.0);
  make_cdf(p->src_group_pdf, G, P.src_cdf.data());
  P.n_surf = p->n_surf;
  P.skind.assign(p->surf_kind, p->surf_kind + P.n_surf);
  P.sbc.assign(p->surf_bc, p->surf_bc + P.n_surf);
  P.scoef.assign(p->surf_coef, p->surf_coef + 10 * P.n_surf);
  P.quad.resize(P.n_surf);
  for (int s = 0; s < P.n_surf; ++s) P.quad[s] = quad_of(P.skind[s], &P.scoef[10 * s]);
  P.n_cell = p->n_cell;
  P.nhs.assign(p->cell_nhs, p->cell_nhs + P.n_cell);
  P.hs_surf.assign(p->cell_hs_surf, p->cell_hs_surf + OR_MAX_HS * P.n_cell);
  P.hs_sense.assign(p->cell_hs_sense, p->cell_hs_sense + OR_MAX_HS * P.n_cell);
  P.cmat.assign(p->cell_mat, p->cell_mat + P.n_cell);
  P.lat = p->has_lattice != 0;
  P.lnx = p->lat_nx;
  P.lny = p->lat_ny;
  P.lx0 = p->lat_x0;
  P.ly0 = p->lat_y0;
  P.lp = p->lat_pitch;
  P.lr = p->lat_r;
  P.lmatrix = p->lat_matrix;
  P.lnz = p->lat_nz > 1 ? p->lat_nz : 1;
  P.lz0 = p->lat_z0;
  P.lpz = p->lat_pitch_z;
  if (P.lat) P.lpin.assign(p->lat_pin_mat, p->lat_pin_mat + P.lnx * P.lny * P.lnz);
  P.src_pos = p->src_pos;
  P.src_dir = p->src_dir;
  for (int i = 0; i < 3; ++i) {
    P.src_lo[i] = p->src_lo[i];
    P.src_hi[i] = p->src_hi[i];
  }
  P.t0 = p->src_t0;
  P.t1 = p->src_t1;
  const double* e = p->tally_edges;
  int off = 0;
  for (int t = 0; t < p->n_tally; ++t) {
    Tally T;
    for (int d = 0; d < 4; ++d) {
      T.n[d] = p->tally_dims[4 * t + d];
      T.e[d].assign(e, e + T.n[d] + 1);
      e += T.n[d] + 1;
    }
    T.est = p->tally_est ? p->tally_est[t] : OR_EST_TRACK;
    T.nval = T.est == OR_EST_CROSSING ? T.n[3] + 1 : T.n[3];
    T.offset = off;
    off += T.n[0] * T.n[1] * T.n[2] * G * T.nval;
    P.tallies.push_back(T);
  }
  P.total_bins = off;
  P.t_census = p->t_census;
  P.ww = p->ww_on != 0;
  if (P.ww) {
    P.ww_n[0] = p->ww_nx;
    P.ww_n[1] = p->ww_ny;
    P.ww_n[2] = p->ww_nz;
    const double* we = p->ww_edges;
    for (int d = 0; d < 3; ++d) {
      P.ww_e[d].assign(we, we + P.ww_n[d] + 1);
      we += P.ww_n[d] + 1;
    }
    if (p->ww_nt > 1 && p->ww_tedges) {
      P.ww_n[3] = p->ww_nt;
      P.ww_e[3].assign(p->ww_tedges, p->ww_tedges + p->ww_nt + 1);
    } else {
      P.ww_n[3] = 1;
      P.ww_e[3] = {0.0, std::numeric_limits<double>::infinity()};
    }
    P.ww_c.assign(p->ww_center, p->ww_center + (size_t)P.ww_n[0] * P.ww_n[1] * P.ww_n[2] * P.ww_n[3] * G);
    P.ww_up = p->ww_upper;
    P.ww_lo = p->ww_lower;
    P.ww_max = p->ww_split_max;
  }
  return P;
}

// ---------------------------------------------------------------- geometry
struct Particle {
  double x, y, z, ux, uy, uz, t, w;
  uint64_t tag, root;
  uint32_t k;
  int g, cell, ix, iy, iz, in_pin;
};

// surface function f(p): plane x - c (or y, z); cylinder (x-x0)^2 + (y-y0)^2 - r^2
double surf_f(const Prob& P, int s, double x, double y, double z) {
  const double* c = &P.scoef[10 * s];
  switch (P.skind[s]) {
    case OR_PX: return x - c[0];
    case OR_PY: return y - c[0];
    case OR_PZ: return z - c[0];
    case OR_CZ: {
      double dx = x - c[0], dy = y - c[1];
      return dx * dx + dy * dy - c[2] * c[2];
    }
    default: {
      double a, b, f;
      quad_ray(P.quad[s], x, y, z, 0.0, 0.0, 0.0, a, b, f);
      return f;
    }
  }
}

// sense +1 <=> f >= 0, sense -1 <=> f < 0
bool sense_ok(double f, int sense) { return sense > 0 ? f >= 0.0 : f < 0.0; }

// size of the terms surf_f subtracts: what its rounding error is relative to
double surf_terms(const Prob& P, int s, double x, double y, double z) {
  const double* c = &P.scoef[10 * s];
  switch (P.skind[s]) {
    case OR_PX: return 1.0 + std::fabs(x) + std::fabs(c[0]);
    case OR_PY: return 1.0 + std::fabs(y) + std::fabs(c[0]);
    case OR_PZ: return 1.0 + std::fabs(z) + std::fabs(c[0]);
    case OR_CZ: {
      double dx = x - c[0], dy = y - c[1];
      return 1.0 + dx * dx + dy * dy + c[2] * c[2];
    }
    default: {
      const Quad& Q = P.quad[s];
      const double* q = Q.q;
      const double X = x - Q.c[0], Y = y - Q.c[1], Z = z - Q.c[2];
      return 1.0 + std::fabs(q[0] * X * X) + std::fabs(q[1] * Y * Y) + std::fabs(q[2] * Z * Z) +
             std::fabs(q[3] * X * Y) + std::fabs(q[4] * Y * Z) + std::fabs(q[5] * Z * X) + std::fabs(q[6] * X) +
             std::fabs(q[7] * Y) + std::fabs(q[8] * Z) + std::fabs(q[9]);
    }
  }
}

// normal component of the direction on surface s: which side a point on s is heading into
double surf_dir(const Prob& P, int s, double x, double y, double z, double ux, double uy, double uz) {
  const double* c = &P.scoef[10 * s];
  switch (P.skind[s]) {
    case OR_PX: return ux;
    case OR_PY: return uy;
    case OR_PZ: return uz;
    case OR_CZ: return (x - c[0]) * ux + (y - c[1]) * uy;
    default: {
      double a, b, f;
      quad_ray(P.quad[s], x, y, z, ux, uy, uz, a, b, f);
      return b;  // the rate at which f changes along the direction
    }
  }
}

// The cell a point is in.  When the point was reached by crossing skip_surf, that surface's sense
// is given (skip_sense) rather than evaluated, only cells bounded by it qualify, and the
// direction of flight settles the other surfaces:
//   - a point lying exactly on another surface belongs to the side the particle is moving into
//     (the + side if it moves along the surface);
//   - if no cell holds the point -- a crossing next to where two surfaces meet can land a rounding
//     error outside the neighbouring surface -- a cell that holds it to within 1e-12 of the size
//     of each surface function's terms is accepted, the first in cell order.
// Without a crossing, a point on a surface is on its + side.
int find_cell(const Prob& P, double x, double y, double z, int skip_surf, int skip_sense, double ux,
              double uy, double uz) {
  const int passes = skip_surf < 0 ? 1 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    for (int c = 0; c < P.n_cell; ++c) {
      bool ok = true;
      bool has_skip = skip_surf < 0;
      for (int i = 0; i < P.nhs[c] && ok; ++i) {
        int s = P.hs_surf[c * OR_MAX_HS + i], sn = P.hs_sense[c * OR_MAX_HS + i];
        if (s == skip_surf) {
          has_skip = true;
          ok = (sn == skip_sense);
        } else if (pass == 0) {
          double f = surf_f(P, s, x, y, z);
          if (f == 0.0) f = surf_dir(P, s, x, y, z, ux, uy, uz);
          ok = sense_ok(f, sn);
        } else {
          double f = surf_f(P, s, x, y, z), tol = 1e-12 * surf_terms(P, s, x, y, z);
          ok = sn > 0 ? f >= -tol : f < tol;
        }
      }
      if (ok && has_skip) return c;
    }
  }
  return -1;
}

// element (ix, iy, iz) of the lattice, z layer iz outermost
int elem_index(const Prob& P, int ix, int iy, int iz) { return (iz * P.lny + iy) * P.lnx + ix; }

bool has_pin(const Prob& P, const Particle& q) { return P.lpin[elem_index(P, q.ix, q.iy, q.iz)] >= 0; }

int pin_sense_inside(const Prob& P, const Particle& q) {
  if (!has_pin(P, q)) return 0;
  double xc = P.lx0 + (q.ix + 0.5) * P.lp, yc = P.ly0 + (q.iy + 0.5) * P.lp;
  double dx = q.x - xc, dy = q.y - yc;
  return (dx * dx + dy * dy - P.lr * P.lr) < 0.0 ? 1 : 0;
}

void lattice_locate(const Prob& P, Particle& q) {
  int ix = (int)std::floor((q.x - P.lx0) / P.lp);
  int iy = (int)std::floor((q.y - P.ly0) / P.lp);
  q.ix = std::min(std::max(ix, 0), P.lnx - 1);
  q.iy = std::min(std::max(iy, 0), P.lny - 1);
  q.iz = 0;
  if (P.lnz > 1) {
    int iz = (int)std::floor((q.z - P.lz0) / P.lpz);
    q.iz = std::min(std::max(iz, 0), P.lnz - 1);
  }
  q.in_pin = pin_sense_inside(P, q);
}

int material(const Prob& P, const Particle& q) {
  int m = P.cmat[q.cell];
  if (m >= 0) return m;
  if (q.in_pin) return P.lpin[elem_index(P, q.ix, q.iy, q.iz)];
  return P.lmatrix;
}

// distance along u to a plane at c, counted only when the motion leaves the half-space
double dist_plane(double pos, double u, double c, int sense) {
  bool leaving = sense > 0 ? (u < 0.0) : (u > 0.0);
  if (!leaving) return INF;
  double d = (c - pos) / u;
  return d > 0.0 ? d : 0.0;
}

// distance to the z-cylinder (x0, y0, r); inside: far root, outside: near root if approaching
double dist_cyl(double x, double y, double ux, double uy, double x0, double y0, double r,
                bool inside) {
  double a = ux * ux + uy * uy;
  if (a == 0.0) return INF;
  double dx = x - x0, dy = y - y0;
  double b = dx * ux + dy * uy;
  double c = dx * dx + dy * dy - r * r;
  double disc = b * b - a * c;
  if (inside) {
    if (disc < 0.0) disc = 0.0;
    double sq = std::sqrt(disc);
    double d = (b <= 0.0) ? (-b + sq) / a : -c / (b + sq);
    return d > 0.0 ? d : 0.0;
  }
  if (b >= 0.0 || disc <= 0.0) return INF;
  // a grazing line whose chord inside the cylinder, 2 sqrt(disc) / a, is shorter than 1e-12 cm
  // does not enter it (otherwise rounding can bounce a particle in and out on the spot)
  double sq = std::sqrt(disc);
  if (2.0 * sq < 1e-12 * a) return INF;
  double d = c / (-b + sq);
  return d > 0.0 ? d : 0.0;
}

enum { HIT_CELL = 0, HIT_LAT_X = 1, HIT_LAT_Y = 2, HIT_PIN = 3, HIT_LAT_Z = 4 };
struct Hit {
  double d;
  int type, idx;
};

Hit distance_to_boundary(const Prob& P, const Particle& q) {
  Hit h{INF, -1, -1};
  int c = q.cell;
  for (int i = 0; i < P.nhs[c]; ++i) {
    int s = P.hs_surf[c * OR_MAX_HS + i], sn = P.hs_sense[c * OR_MAX_HS + i];
    const double* cf = &P.scoef[10 * s];
    double d;
    switch (P.skind[s]) {
      case OR_PX: d = dist_plane(q.x, q.ux, cf[0], sn); break;
      case OR_PY: d = dist_plane(q.y, q.uy, cf[0], sn); break;
      case OR_PZ: d = dist_plane(q.z, q.uz, cf[0], sn); break;
      case OR_CZ: d = dist_cyl(q.x, q.y, q.ux, q.uy, cf[0], cf[1], cf[2], sn < 0); break;
      default: {
        double a, b, f;
        quad_ray(P.quad[s], q.x, q.y, q.z, q.ux, q.uy, q.uz, a, b, f);
        d = dist_quadric(a, b, f, sn);
        break;
      }
    }
    if (d < h.d) h = {d, HIT_CELL, s};
  }
  if (P.cmat[c] < 0) {
    // inside the lattice: element walls (outer walls belong to the cell), then the pin
    Hit l{INF, -1, 0};
    double xlo = P.lx0 + q.ix * P.lp, ylo = P.ly0 + q.iy * P.lp;
    if (q.ux > 0.0 && q.ix + 1 < P.lnx) {
      double d = (xlo + P.lp - q.x) / q.ux;
      d = d > 0.0 ? d : 0.0;
      if (d < l.d) l = {d, HIT_LAT_X, +1};
    } else if (q.ux < 0.0 && q.ix > 0) {
      double d = (xlo - q.x) / q.ux;
      d = d > 0.0 ? d : 0.0;
      if (d < l.d) l = {d, HIT_LAT_X, -1};
    }
    if (q.uy > 0.0 && q.iy + 1 < P.lny) {
      double d = (ylo + P.lp - q.y) / q.uy;
      d = d > 0.0 ? d : 0.0;
      if (d < l.d) l = {d, HIT_LAT_Y, +1};
    } else if (q.uy < 0.0 && q.iy > 0) {
      double d = (ylo - q.y) / q.uy;
      d = d > 0.0 ? d : 0.0;
      if (d < l.d) l = {d, HIT_LAT_Y, -1};
    }
    if (P.lnz > 1) {
      // axial layers: the z walls between them
      double zlo = P.lz0 + q.iz * P.lpz;
      if (q.uz > 0.0 && q.iz + 1 < P.lnz) {
        double d = (zlo + P.lpz - q.z) / q.uz;
        d = d > 0.0 ? d : 0.0;
        if (d < l.d) l = {d, HIT_LAT_Z, +1};
      } else if (q.uz < 0.0 && q.iz > 0) {
        double d = (zlo - q.z) / q.uz;
        d = d > 0.0 ? d : 0.0;
        if (d < l.d) l = {d, HIT_LAT_Z, -1};
      }
    }
    if (has_pin(P, q)) {
      double d = dist_cyl(q.x, q.y, q.ux, q.uy, xlo + 0.5 * P.lp, ylo + 0.5 * P.lp, P.lr,
                          q.in_pin != 0);
      if (d < l.d) l = {d, HIT_PIN, 0};
    }
    if (l.d < h.d) h = l;
  }
  return h;
}

int bin_of(const std::vector<double>& e, double v) {
  // edges[i] <= v < edges[i+1]
  if (!(v >= e.front()) || !(v < e.back())) return -1;
  auto it = std::upper_bound(e.begin(), e.end(), v);
  return (int)(it - e.begin()) - 1;
}

// ---------------------------------------------------------------- accumulation
struct Acc {
  std::vector<double> s1, s2, hist;
  std::vector<int64_t> fixed;
  std::vector<int> touched;
  std::vector<char> mark;
  int64_t cnt[OR_NCOUNT];
  double fscale;
  std::vector<or_event> log;

  void init(int n, int fixed_bits) {
    s1.assign(n, 0.0);
    s2.assign(n, 0.0);
    hist.assign(n, 0.0);
    fixed.assign(n, 0);
    mark.assign(n, 0);
    std::memset(cnt, 0, sizeof(cnt));
    fscale = std::ldexp(1.0, fixed_bits);
  }
  // adds score v to the history's bin; the fixed-point sum counts fx (the score itself, or the
  // weight of a time-crossing score, whose flux w v can exceed the fixed-point range)
  void add(int bin, double v, double fx) {
    if (!mark[bin]) {
      mark[bin] = 1;
      touched.push_back(bin);
    }
    hist[bin] += v;
    fixed[bin] += (int64_t)std::llrint(fx * fscale);
  }
  void add(int bin, double v) { add(bin, v, v); }
  void end_history() {
    for (int b : touched) {
      s1[b] += hist[b];
      s2[b] += hist[b] * hist[b];
      hist[b] = 0.0;
      mark[b] = 0;
    }
    touched.clear();
  }
};

// track-length scoring of the segment from q over length l: cut the segment at every mesh plane
// and time edge it crosses, score each piece into the bin that contains its midpoint
void score_segment(const Prob& P, const Particle& q, double l, Acc& acc) {
  double v = P.v[q.g];
  double p0[3] = {q.x, q.y, q.z}, u[3] = {q.ux, q.uy, q.uz};
  for (const Tally& T : P.tallies) {
    if (T.est == OR_EST_CROSSING) {
      // time-crossing estimator: the flight spans the times [t, t + l / v); at every time point
      // t_j inside that span the particle contributes w v to the flux of the cell it is in
      double t_end = q.t + l / v;
      for (int j = 0; j <= T.n[3]; ++j) {
        double tj = T.e[3][j];
        if (!(tj >= q.t && tj < t_end)) continue;
        double s = (tj - q.t) * v;
        int ix = bin_of(T.e[0], p0[0] + s * u[0]);
        int iy = bin_of(T.e[1], p0[1] + s * u[1]);
        int iz = bin_of(T.e[2], p0[2] + s * u[2]);
        if (ix < 0 || iy < 0 || iz < 0) continue;
        int bin = (((iz * T.n[1] + iy) * T.n[0] + ix) * P.G + q.g) * T.nval + j;
        acc.add(T.offset + bin, q.w * v, q.w);
      }
      continue;
    }
    std::vector<double> cuts;
    cuts.push_back(0.0);
    cuts.push_back(l);
    for (int d = 0; d < 3; ++d) {
      if (u[d] == 0.0) continue;
      for (double e : T.e[d]) {
        double s = (e - p0[d]) / u[d];
        if (s > 0.0 && s < l) cuts.push_back(s);
      }
    }
    for (double e : T.e[3]) {
      double s = (e - q.t) * v;
      if (s > 0.0 && s < l) cuts.push_back(s);
    }
    std::sort(cuts.begin(), cuts.end());
    for (size_t i = 0; i + 1 < cuts.size(); ++i) {
      double a = cuts[i], b = cuts[i + 1];
      if (!(b > a)) continue;
      double m = 0.5 * (a + b);
      int ix = bin_of(T.e[0], p0[0] + m * u[0]);
      int iy = bin_of(T.e[1], p0[1] + m * u[1]);
      int iz = bin_of(T.e[2], p0[2] + m * u[2]);
      int it = bin_of(T.e[3], q.t + m / v);
      if (ix < 0 || iy < 0 || iz < 0 || it < 0) continue;
      int bin = (((iz * T.n[1] + iy) * T.n[0] + ix) * P.G + q.g) * T.nval + it;
      acc.add(T.offset + bin, q.w * (b - a));
    }
  }
}

void isotropic(double mu, double u_phi, double& ux, double& uy, double& uz) {
  double s = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  double phi = TWO_PI * u_phi;
  ux = mu;
  uy = s * std::cos(phi);
  uz = s * std::sin(phi);
}

// source particle of history h: event index SOURCE_EVENT, blocks 0..3 give
// (u_x, u_y), (u_z, u_mu), (u_phi, u_g), (u_t, -)
Particle source_particle(const Prob& P, uint64_t seed, uint64_t h) {
  Particle q{};
  q.tag = h;
  q.root = h;
  Pair b0 = draw(seed, h, SOURCE_EVENT, 0), b1 = draw(seed, h, SOURCE_EVENT, 1);
  Pair b2 = draw(seed, h, SOURCE_EVENT, 2), b3 = draw(seed, h, SOURCE_EVENT, 3);
  if (P.src_pos == OR_SRC_BOX) {
    q.x = P.src_lo[0] + (P.src_hi[0] - P.src_lo[0]) * b0.a;
    q.y = P.src_lo[1] + (P.src_hi[1] - P.src_lo[1]) * b0.b;
    q.z = P.src_lo[2] + (P.src_hi[2] - P.src_lo[2]) * b1.a;
  } else {
    q.x = P.src_lo[0];
    q.y = P.src_lo[1] + (P.src_hi[1] - P.src_lo[1]) * b0.b;
    q.z = P.src_lo[2] + (P.src_hi[2] - P.src_lo[2]) * b1.a;
  }
  if (P.src_dir == OR_DIR_BEAM_X) {
    q.ux = 1.0;
    q.uy = 0.0;
    q.uz = 0.0;
  } else {
    double mu = P.src_dir == OR_DIR_COS_X ? std::sqrt(b1.b) : 2.0 * b1.b - 1.0;
    isotropic(mu, b2.a, q.ux, q.uy, q.uz);
  }
  q.g = sample_cdf(P.src_cdf.data(), P.G, b2.b);
  q.t = P.t0 + (P.t1 - P.t0) * b3.a;
  q.w = 1.0;
  q.k = 0;
  q.cell = find_cell(P, q.x, q.y, q.z, -1, 0, 0.0, 0.0, 0.0);
  q.ix = q.iy = q.iz = q.in_pin = 0;
  if (q.cell >= 0 && P.cmat[q.cell] < 0) lattice_locate(P, q);
  return q;
}

// weight-window check at the particle's current state; returns false if roulette killed it
bool weight_window(const Prob& P, uint64_t seed, Particle& q, uint32_t k_used,
                   std::vector<Particle>& stack, Acc& acc) {
  if (!P.ww) return true;
  // the window of the cell the particle moves into: a particle on a window-mesh edge (e.g. just
  // after crossing a layer plane that is also a mesh plane) is looked up 1e-9 cm ahead
  const double ah = 1e-9;
  int ix = bin_of(P.ww_e[0], q.x + ah * q.ux), iy = bin_of(P.ww_e[1], q.y + ah * q.uy),
      iz = bin_of(P.ww_e[2], q.z + ah * q.uz);
  // and of the time bin holding the particle's time
  int it = bin_of(P.ww_e[3], q.t);
  if (ix < 0 || iy < 0 || iz < 0 || it < 0) return true;
  double wc = P.ww_c[(((it * P.ww_n[2] + iz) * P.ww_n[1] + iy) * P.ww_n[0] + ix) * P.G + q.g];
  if (!(wc > 0.0)) return true;
  if (q.w > P.ww_up * wc) {
    int n = (int)std::ceil(q.w / wc);
    if (n > P.ww_max) n = P.ww_max;
    double w = q.w / n;
    q.w = w;
    for (int j = 1; j < n; ++j) {
      Particle c = q;
      c.tag = child_tag(seed, q.tag, k_used, (uint32_t)j, SPLIT_MARK);
      c.k = 0;
      stack.push_back(c);
      acc.cnt[OR_C_WW_SPLIT]++;
    }
  } else if (q.w < P.ww_lo * wc) {
    double u = draw(seed, q.tag, k_used, 2).b;
    if (u < q.w / wc) {
      q.w = wc;
    } else {
      acc.cnt[OR_C_WW_KILL]++;
      return false;
    }
  }
  return true;
}

// population control interval of one batch: the census time of the interval, and where particles
// that reach an interior census are banked
struct PcBanked {
  Particle q;
  uint32_t kc;  // event index of the flight that reached the census
};
struct Pc {
  double t_census;
  bool interior;
  std::vector<PcBanked>* bank;
};

struct Logger {
  bool on;
  uint64_t first, count;
};

void transport(const Prob& P, const Physics& ph, uint64_t seed, Particle q, std::vector<Particle>& stack,
               Acc& acc, const Logger& lg, Eig* eig = nullptr, Pc* pc = nullptr) {
  const double t_census = pc ? pc->t_census : P.t_census;
  const int G = P.G;
  while (true) {
    int m = material(P, q);
    double St = P.st[m * G + q.g];
    Pair b0 = draw(seed, q.tag, q.k, 0);
    double dc = St > 0.0 ? -std::log(b0.a) / St : INF;
    Hit hit = distance_to_boundary(P, q);
    double dt = INF;
    if (t_census < INF) {
      dt = P.v[q.g] * (t_census - q.t);
      if (dt < 0.0) dt = 0.0;
    }
    int ev;
    double l;
    if (dc < hit.d && dc < dt) {
      ev = OR_EV_COLLISION;
      l = dc;
    } else if (hit.d <= dt) {
      ev = OR_EV_SURFACE;
      l = hit.d;
    } else {
      ev = OR_EV_CENSUS;
      l = dt;
    }
    acc.cnt[OR_C_FLIGHT]++;
    if (!(l < INF)) ev = OR_EV_LOST;
    if (ev != OR_EV_LOST) {
      if (!eig || eig->score) score_segment(P, q, l, acc);
      if (eig) eig->ktl += (int64_t)std::llrint(q.w * l * (P.nu[m * G + q.g] * P.sf[m * G + q.g]) * 4294967296.0);
      q.x += l * q.ux;
      q.y += l * q.uy;
      q.z += l * q.uz;
      q.t += l / P.v[q.g];
    }
    uint32_t k = q.k;
    q.k = k + 1;
    or_event rec{};
    bool logit = lg.on && q.root >= lg.first && q.root < lg.first + lg.count;
    if (logit) {
      rec.tag = q.tag;
      rec.root = q.root;
      rec.k = k;
      rec.kind = ev;
      rec.cell = q.cell;
      rec.elem = P.lat ? elem_index(P, q.ix, q.iy, q.iz) : q.ix;
      rec.in_pin = q.in_pin;
      rec.g = q.g;
      rec.x = q.x;
      rec.y = q.y;
      rec.z = q.z;
      rec.ux = q.ux;
      rec.uy = q.uy;
      rec.uz = q.uz;
      rec.t = q.t;
      rec.w = q.w;
    }
    bool alive = true;
    if (ev == OR_EV_LOST) {
      acc.cnt[OR_C_LOST]++;
      alive = false;
    } else if (ev == OR_EV_CENSUS) {
      if (pc && pc->interior) {
        pc->bank->push_back({q, k});
        acc.cnt[OR_C_PC_BANKED]++;
      } else {
        acc.cnt[OR_C_CENSUS]++;
      }
      alive = false;
    } else if (ev == OR_EV_SURFACE) {
      acc.cnt[OR_C_SURFACE]++;
      if (hit.type == HIT_CELL) {
        int s = hit.idx;
        if (P.sbc[s] == OR_VACUUM) {
          if (!eig || eig->score) acc.add(P.total_bins + s, q.w);
          acc.cnt[OR_C_LEAK]++;
          rec.outcome = 2;
          alive = false;
        } else if (P.sbc[s] == OR_REFLECT) {
          acc.cnt[OR_C_REFLECT]++;
          rec.outcome = 1;
          if (P.skind[s] == OR_PX) q.ux = -q.ux;
          else if (P.skind[s] == OR_PY) q.uy = -q.uy;
          else q.uz = -q.uz;
        } else {
          int old_sense = 0;
          for (int i = 0; i < P.nhs[q.cell]; ++i)
            if (P.hs_surf[q.cell * OR_MAX_HS + i] == s) old_sense = P.hs_sense[q.cell * OR_MAX_HS + i];
          int nc = find_cell(P, q.x, q.y, q.z, s, -old_sense, q.ux, q.uy, q.uz);
          rec.outcome = 0;
          if (nc < 0) {
            acc.cnt[OR_C_LOST]++;
            alive = false;
          } else {
            q.cell = nc;
            if (P.cmat[nc] < 0) lattice_locate(P, q);
          }
        }
      } else if (hit.type == HIT_LAT_X || hit.type == HIT_LAT_Y || hit.type == HIT_LAT_Z) {
        rec.outcome = 3;
        if (hit.type == HIT_LAT_X) q.ix += hit.idx;
        else if (hit.type == HIT_LAT_Y) q.iy += hit.idx;
        else q.iz += hit.idx;
        q.in_pin = pin_sense_inside(P, q);
      } else {
        rec.outcome = 4;
        q.in_pin = !q.in_pin;
      }
      if (alive) alive = weight_window(P, seed, q, k, stack, acc);
    } else {
      acc.cnt[OR_C_COLLISION]++;
      double Ss = P.ss_tot[m * G + q.g], Sf = P.sf[m * G + q.g];
      // analog: the channel is drawn over Sigma_t (scatter, production, capture).  Implicit
      // capture: it is drawn over Sigma_s + Sigma_f only, and the weight takes the factor
      // (Sigma_s + Sigma_f) / Sigma_t, the probability that the collision is not a capture
      double xi = b0.b * St;
      if (ph.implicit) {
        double keep = Ss + Sf;
        xi = b0.b * keep;
        if (keep > 0.0) q.w *= keep / St;
        else xi = INF;  // a pure absorber: the weight would be zero, the particle is captured
      }
      if (xi < Ss) {
        acc.cnt[OR_C_SCATTER]++;
        Pair b1 = draw(seed, q.tag, k, 1), b2 = draw(seed, q.tag, k, 2);
        q.g = sample_cdf(&P.scat_cdf[(m * G + q.g) * G], G, b1.a);
        isotropic(2.0 * b1.b - 1.0, b2.a, q.ux, q.uy, q.uz);
        rec.outcome = 0;
        if (ph.implicit && q.w < ph.cutoff) {
          // weight cutoff: survive with probability w / w_s at weight w_s (unbiased)
          double u = draw(seed, q.tag, k, 3).b;
          if (u < q.w / ph.survival) {
            q.w = ph.survival;
          } else {
            acc.cnt[OR_C_WW_KILL]++;
            alive = false;
          }
        }
        if (alive) alive = weight_window(P, seed, q, k, stack, acc);
      } else if (xi < Ss + Sf) {
        acc.cnt[OR_C_PRODUCTION]++;
        Pair b3 = draw(seed, q.tag, k, 3);
        if (eig) {
          // fission sites for the next cycle: floor(nu / k + xi), group from chi, at this point
          int n = (int)std::floor(P.nu[m * G + q.g] * eig->inv_k + b3.a);
          for (int j = 0; j < n; ++j) {
            uint64_t ct = child_tag(seed, q.tag, k, (uint32_t)j, CHILD_MARK);
            Pair c2 = draw(seed, ct, SOURCE_EVENT, 2);
            eig->sites->push_back({q.x, q.y, q.z, sample_cdf(&P.chi_cdf[m * G], G, c2.b)});
            acc.cnt[OR_C_SECONDARY]++;
          }
          rec.outcome = 1;
          rec.n_child = n;
          alive = false;
          if (logit) acc.log.push_back(rec);
          return;
        }
        int n = (int)std::floor(P.nu[m * G + q.g] + b3.a);
        for (int j = 0; j < n; ++j) {
          Particle c = q;
          c.tag = child_tag(seed, q.tag, k, (uint32_t)j, CHILD_MARK);
          c.k = 0;
          Pair c1 = draw(seed, c.tag, SOURCE_EVENT, 1), c2 = draw(seed, c.tag, SOURCE_EVENT, 2);
          isotropic(2.0 * c1.b - 1.0, c2.a, c.ux, c.uy, c.uz);
          c.g = sample_cdf(&P.chi_cdf[m * G], G, c2.b);
          stack.push_back(c);
          acc.cnt[OR_C_SECONDARY]++;
        }
        rec.outcome = 1;
        rec.n_child = n;
        alive = false;
      } else {
        acc.cnt[OR_C_CAPTURE]++;
        rec.outcome = 2;
        alive = false;
      }
    }
    if (logit) acc.log.push_back(rec);
    if (!alive) return;
  }
}

void run_range(const Prob& P, const Physics& ph, uint64_t seed, uint64_t h0, uint64_t h1, Acc& acc,
               const Logger& lg) {
  std::vector<Particle> stack;
  for (uint64_t h = h0; h < h1; ++h) {
    Particle q = source_particle(P, seed, h);
    acc.cnt[OR_C_SOURCE]++;
    if (q.cell < 0) {
      acc.cnt[OR_C_LOST]++;
    } else {
      stack.push_back(q);
      while (!stack.empty()) {
        Particle c = stack.back();
        stack.pop_back();
        transport(P, ph, seed, c, stack, acc, lg);
      }
    }
    acc.end_history();
  }
}

// one batch of a population-controlled run (see or_run_pc): its histories [h0, h1), interval by
// interval, with splitting-roulette of the banked particles at every interior census
// copies of banked particle j by the comb: teeth at (k + xi) W / N_b, k = 0 .. N_b - 1, counted in
// its cumulative-weight interval [C_{j-1}, C_j) through F(C) = #{k : tooth k < C}
int64_t comb_teeth_below(int64_t C, int64_t W, uint64_t Nb, double xi) {
  const double x = (double)C * (double)Nb / (double)W - xi;
  const double f = std::ceil(x);
  if (!(f > 0.0)) return 0;
  return f >= (double)Nb ? (int64_t)Nb : (int64_t)f;
}

void run_pc_batch(const Prob& P, const or_pc_opts* o, uint64_t b, uint64_t h0, uint64_t h1, Acc& acc,
                  const Logger& lg, std::vector<uint64_t>& banked) {
  const Physics ph{false, 0.0, 0.0};
  const uint64_t Nb = h1 - h0;
  std::vector<Particle> cur, stack;
  for (uint64_t h = h0; h < h1; ++h) {
    Particle q = source_particle(P, o->seed, h);
    acc.cnt[OR_C_SOURCE]++;
    if (q.cell < 0) acc.cnt[OR_C_LOST]++;
    else cur.push_back(q);
  }
  for (int i = 0; i <= o->n_census; ++i) {
    std::vector<PcBanked> bank;
    Pc pc{i < o->n_census ? o->census_times[i] : P.t_census, i < o->n_census, &bank};
    for (const Particle& q : cur) {
      stack.push_back(q);
      while (!stack.empty()) {
        Particle c = stack.back();
        stack.pop_back();
        transport(P, ph, o->seed, c, stack, acc, lg, nullptr, &pc);
      }
    }
    cur.clear();
    if (!pc.interior) break;
    banked[i] += bank.size();
    // splitting-roulette to the batch's N_b histories: exact fixed-point total weight
    int64_t Wq = 0;
    for (const PcBanked& b : bank) Wq += (int64_t)std::llrint(b.q.w * 1099511627776.0);
    if (Wq <= 0) break;
    const double wt = (double)Wq / 1099511627776.0 / (double)Nb;
    std::vector<int> ncopy(bank.size());
    if (o->method == 1) {
      // combing: the bank in tag order, one offset per batch and census
      std::sort(bank.begin(), bank.end(), [](const PcBanked& x, const PcBanked& y) { return x.q.tag < y.q.tag; });
      const double xi = draw(o->seed, 0xFFFFFFFEull | (b << 32), (uint32_t)i, 5).a;
      int64_t C = 0;
      for (size_t j = 0; j < bank.size(); ++j) {
        const int64_t Cp = C;
        C += (int64_t)std::llrint(bank[j].q.w * 1099511627776.0);
        ncopy[j] = (int)(comb_teeth_below(C, Wq, Nb, xi) - comb_teeth_below(Cp, Wq, Nb, xi));
      }
    } else {
      for (size_t j = 0; j < bank.size(); ++j)
        ncopy[j] = (int)std::floor(bank[j].q.w / wt + draw(o->seed, bank[j].q.tag, bank[j].kc, 1).a);
    }
    for (size_t jb = 0; jb < bank.size(); ++jb) {
      const PcBanked& bk = bank[jb];
      for (int j = 0; j < ncopy[jb]; ++j) {
        Particle c = bk.q;
        c.tag = child_tag(o->seed, bk.q.tag, bk.kc, (uint32_t)j, 0x40000000u);
        c.k = 0;
        c.t = pc.t_census;
        c.w = wt;
        cur.push_back(c);
        acc.cnt[OR_C_PC_COPIES]++;
      }
    }
  }
}

// k-eigenvalue power iteration (the paper's C5G7 runs, Section 3): cycle 0 starts N histories
// from the problem's source; every later cycle starts N histories at the previous cycle's fission
// sites, picked by systematic sampling (combing) with one random offset per cycle, so the
// population stays N.  Sites are ordered by the source history that produced them, then in
// production order, which fixes the order whatever the thread count.
struct EigRun {
  const Prob& P;
  const Physics& ph;
  uint64_t seed, N;
  int threads;
};

// source particle h of cycle c >= 1 at site i of the previous cycle's bank
Particle site_source(const Prob& P, uint64_t seed, uint64_t h, uint32_t cycle, const Site& s) {
  Particle q{};
  q.tag = h | ((uint64_t)cycle << 32);
  q.root = h;
  Pair b1 = draw(seed, q.tag, SOURCE_EVENT, 1), b2 = draw(seed, q.tag, SOURCE_EVENT, 2);
  q.x = s.x;
  q.y = s.y;
  q.z = s.z;
  isotropic(2.0 * b1.b - 1.0, b2.a, q.ux, q.uy, q.uz);
  q.g = s.g;
  q.t = 0.0;
  q.w = 1.0;
  q.k = 0;
  q.cell = find_cell(P, q.x, q.y, q.z, -1, 0, 0.0, 0.0, 0.0);
  q.ix = q.iy = q.iz = q.in_pin = 0;
  if (q.cell >= 0 && P.cmat[q.cell] < 0) lattice_locate(P, q);
  return q;
}

// the combing offset of cycle c: first uniform of the counter (2^32 - 1, c, 2^32 - 1, 4)
double comb_offset(uint64_t seed, uint32_t cycle) {
  return draw(seed, 0xFFFFFFFFull | ((uint64_t)cycle << 32), SOURCE_EVENT, 4).a;
}

}  // namespace

extern "C" {

void or_comb_counts(const double* w, int64_t n, uint64_t Nb, double xi, int64_t* out) {
  int64_t W = 0;
  for (int64_t j = 0; j < n; ++j) W += (int64_t)std::llrint(w[j] * 1099511627776.0);
  int64_t C = 0;
  for (int64_t j = 0; j < n; ++j) {
    const int64_t Cp = C;
    C += (int64_t)std::llrint(w[j] * 1099511627776.0);
    out[j] = comb_teeth_below(C, W, Nb, xi) - comb_teeth_below(Cp, W, Nb, xi);
  }
}

int or_run_pc(const or_problem* p, const or_pc_opts* o, or_pc_result* r) {
  Prob P = copy_problem(p);
  const uint64_t N = o->n_histories;
  const int nb = o->n_batches;
  if (N == 0 || nb < 1 || (uint64_t)nb > N || o->n_census < 0) return -1;
  for (int i = 0; i < o->n_census; ++i)
    if (!(o->census_times[i] > (i ? o->census_times[i - 1] : 0.0)) || !(o->census_times[i] < P.t_census)) return -1;
  const int bins = P.total_bins + P.n_surf;
  std::vector<Acc> accs(nb);
  std::vector<std::vector<uint64_t>> banked(nb, std::vector<uint64_t>(o->n_census > 0 ? o->n_census : 1, 0));
  Logger lg{o->log != nullptr, o->log_first, o->log_count};
  int nt = o->threads > 0 ? o->threads : 1;
  if (nt > nb) nt = nb;
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    th.emplace_back([&, t] {
      for (int b = t; b < nb; b += nt) {
        accs[b].init(bins, 32);
        // histories of batch b: floor(h nb / N) == b
        const uint64_t h0 = ((uint64_t)b * N + nb - 1) / nb, h1 = ((uint64_t)(b + 1) * N + nb - 1) / nb;
        run_pc_batch(P, o, (uint64_t)b, h0, h1, accs[b], lg, banked[b]);
        accs[b].end_history();
      }
    });
  }
  for (auto& x : th) x.join();
  for (int k = 0; k < OR_NCOUNT; ++k) {
    r->counters[k] = 0;
    for (int b = 0; b < nb; ++b) r->counters[k] += accs[b].cnt[k];
  }
  for (int b = 0; b < nb; ++b) {
    const uint64_t h0 = ((uint64_t)b * N + nb - 1) / nb, h1 = ((uint64_t)(b + 1) * N + nb - 1) / nb;
    if (r->tally_batch)
      for (int i = 0; i < bins; ++i) r->tally_batch[(size_t)b * bins + i] = accs[b].s1[i] / (double)(h1 - h0);
  }
  if (r->banked)
    for (int i = 0; i < o->n_census; ++i) {
      r->banked[i] = 0;
      for (int b = 0; b < nb; ++b) r->banked[i] += banked[b][i];
    }
  if (o->log) {
    uint64_t w = 0;
    for (int b = 0; b < nb; ++b)
      for (const or_event& e : accs[b].log)
        if (w < o->log_cap) o->log[w++] = e;
    if (o->log_n) *o->log_n = w;
  }
  return 0;
}

int or_run_eigen(const or_problem* p, const or_eigen_opts* o, or_eigen_result* r) {
  Prob P = copy_problem(p);
  Physics ph{false, 0.0, 0.0};
  const uint64_t N = o->n_per_cycle;
  const int n_cycles = o->n_inactive + o->n_active;
  if (N == 0 || n_cycles <= 0 || o->n_active < 0) return -1;
  int nt = o->threads > 0 ? o->threads : 1;
  if ((uint64_t)nt > N) nt = (int)N;
  const int nb = P.total_bins + P.n_surf;
  std::vector<Site> prev, next;
  double k_prev = 1.0;
  for (int k = 0; k < OR_NCOUNT; ++k) r->counters[k] = 0;
  Logger lg{o->log != nullptr, o->log_first, o->log_count};
  std::vector<or_event> log;
  for (int cyc = 0; cyc < n_cycles; ++cyc) {
    const bool active = cyc >= o->n_inactive;
    const double u0 = comb_offset(o->seed, (uint32_t)cyc);
    std::vector<Acc> accs(nt);
    std::vector<std::vector<Site>> sites(nt);
    std::vector<int64_t> ktl(nt, 0);
    std::vector<std::thread> th;
    for (int i = 0; i < nt; ++i) {
      accs[i].init(nb, o->fixed_bits);
      uint64_t h0 = N * (uint64_t)i / (uint64_t)nt, h1 = N * (uint64_t)(i + 1) / (uint64_t)nt;
      th.emplace_back([&, i, h0, h1] {
        Eig eig{1.0 / k_prev, active, &sites[i], 0};
        std::vector<Particle> stack;
        for (uint64_t h = h0; h < h1; ++h) {
          Particle q;
          if (cyc == 0) {
            q = source_particle(P, o->seed, h);
          } else {
            const uint64_t M = prev.size();
            uint64_t idx = (uint64_t)std::floor(((double)h + u0) * (double)M / (double)N);
            if (idx >= M) idx = M - 1;
            q = site_source(P, o->seed, h, (uint32_t)cyc, prev[idx]);
          }
          accs[i].cnt[OR_C_SOURCE]++;
          if (q.cell < 0) {
            accs[i].cnt[OR_C_LOST]++;
          } else {
            transport(P, ph, o->seed, q, stack, accs[i], lg, &eig);
          }
          accs[i].end_history();
        }
        ktl[i] = eig.ktl;
      });
    }
    for (auto& t : th) t.join();
    next.clear();
    int64_t ksum = 0;
    for (int i = 0; i < nt; ++i) {
      next.insert(next.end(), sites[i].begin(), sites[i].end());
      ksum += ktl[i];
      for (int k = 0; k < OR_NCOUNT; ++k) r->counters[k] += accs[i].cnt[k];
      for (const or_event& e : accs[i].log) log.push_back(e);
    }
    const double k_cyc = (double)ksum / 4294967296.0 / (double)N;
    if (r->k_cycle) r->k_cycle[cyc] = k_cyc;
    if (r->sites_cycle) r->sites_cycle[cyc] = next.size();
    if (active && r->tally_cycle) {
      double* out = r->tally_cycle + (size_t)(cyc - o->n_inactive) * nb;
      for (int b = 0; b < nb; ++b) {
        double a = 0.0;
        for (int i = 0; i < nt; ++i) a += accs[i].s1[b];
        out[b] = a / (double)N;
      }
    }
    if (next.empty()) return -2;  // no fission site: the chain died out
    prev.swap(next);
    k_prev = k_cyc;
  }
  if (o->log) {
    uint64_t w = 0;
    for (const or_event& e : log)
      if (w < o->log_cap) o->log[w++] = e;
    if (o->log_n) *o->log_n = w;
  }
  return 0;
}

int or_total_bins(const or_problem* p) {
  int off = 0;
  for (int t = 0; t < p->n_tally; ++t) {
    const int* d = &p->tally_dims[4 * t];
    const int nval = (p->tally_est && p->tally_est[t] == OR_EST_CROSSING) ? d[3] + 1 : d[3];
    off += d[0] * d[1] * d[2] * p->G * nval;
  }
  return off + p->n_surf;
}

int or_run(const or_problem* p, const or_opts* o, or_result* r) {
  Prob P = copy_problem(p);
  int nb = P.total_bins + P.n_surf;
  int nt = o->threads > 0 ? o->threads : 1;
  uint64_t n = o->n_histories;
  if ((uint64_t)nt > n && n > 0) nt = (int)n;
  if (nt < 1) nt = 1;
  std::vector<Acc> accs(nt);
  Logger lg{o->log != nullptr, o->log_first, o->log_count};
  Physics ph{o->implicit_capture != 0, o->wr_cutoff, o->wr_survival};
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) {
    accs[i].init(nb, o->fixed_bits);
    uint64_t h0 = o->first_history + n * (uint64_t)i / (uint64_t)nt;
    uint64_t h1 = o->first_history + n * (uint64_t)(i + 1) / (uint64_t)nt;
    th.emplace_back([&, i, h0, h1] { run_range(P, ph, o->seed, h0, h1, accs[i], lg); });
  }
  for (auto& t : th) t.join();
  for (int b = 0; b < nb; ++b) {
    double a = 0.0, c = 0.0;
    int64_t f = 0;
    for (int i = 0; i < nt; ++i) {
      a += accs[i].s1[b];
      c += accs[i].s2[b];
      f += accs[i].fixed[b];
    }
    if (r->s1) r->s1[b] = a;
    if (r->s2) r->s2[b] = c;
    if (r->fixed) r->fixed[b] = f;
  }
  for (int k = 0; k < OR_NCOUNT; ++k) {
    r->counters[k] = 0;
    for (int i = 0; i < nt; ++i) r->counters[k] += accs[i].cnt[k];
  }
  if (o->log) {
    uint64_t w = 0;
    for (int i = 0; i < nt; ++i)
      for (const or_event& e : accs[i].log)
        if (w < o->log_cap) o->log[w++] = e;
    if (o->log_n) *o->log_n = w;
  }
  return 0;
}

void or_philox(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  philox(k0, k1, c);
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

double or_u01(uint32_t a, uint32_t b) { return u01(a, b); }

double or_dist_cylinder(double x, double y, double ux, double uy, double x0, double y0, double r,
                        int inside) {
  return dist_cyl(x, y, ux, uy, x0, y0, r, inside != 0);
}

double or_dist_surface(const or_problem* p, int s, double x, double y, double z, double ux, double uy, double uz,
                       int sense) {
  Prob P = copy_problem(p);
  const double* cf = &P.scoef[10 * s];
  switch (P.skind[s]) {
    case OR_PX: return dist_plane(x, ux, cf[0], sense);
    case OR_PY: return dist_plane(y, uy, cf[0], sense);
    case OR_PZ: return dist_plane(z, uz, cf[0], sense);
    case OR_CZ: return dist_cyl(x, y, ux, uy, cf[0], cf[1], cf[2], sense < 0);
    default: {
      double a, b, f;
      quad_ray(P.quad[s], x, y, z, ux, uy, uz, a, b, f);
      return dist_quadric(a, b, f, sense);
    }
  }
}

double or_dist_plane(double pos, double u, double c, int sense) {
  return dist_plane(pos, u, c, sense);
}

int or_find_cell(const or_problem* p, double x, double y, double z, int skip, int skip_sense, double ux,
                 double uy, double uz) {
  Prob P = copy_problem(p);
  return find_cell(P, x, y, z, skip, skip_sense, ux, uy, uz);
}

int or_source_sample(const or_problem* p, uint64_t seed, uint64_t h, double out[7], int* g) {
  Prob P = copy_problem(p);
  Particle q = source_particle(P, seed, h);
  out[0] = q.x;
  out[1] = q.y;
  out[2] = q.z;
  out[3] = q.ux;
  out[4] = q.uy;
  out[5] = q.uz;
  out[6] = q.t;
  *g = q.g;
  return q.cell;
}

int or_sample_scatter_group(const or_problem* p, int m, int g, double u) {
  Prob P = copy_problem(p);
  return sample_cdf(&P.scat_cdf[(m * P.G + g) * P.G], P.G, u);
}

uint64_t or_child_tag(uint64_t seed, uint64_t parent, uint32_t k, uint32_t j, uint32_t marker) {
  return child_tag(seed, parent, k, j, marker);
}

// ---------------------------------------------------------------- reference MLP (FP64)
int or_mlp_param_count(int H) { return H * 5 + H + 2 * (H * H + H) + H + 1; }

double or_mlp_loss_grad(int H, const double* prm, int n, const double* x, const double* target,
                        const double* wt, double* y, double* grad) {
  const double* W1 = prm;
  const double* b1 = W1 + H * 5;
  const double* W2 = b1 + H;
  const double* b2 = W2 + H * H;
  const double* W3 = b2 + H;
  const double* b3 = W3 + H * H;
  const double* W4 = b3 + H;
  const double* b4 = W4 + H;
  int np = or_mlp_param_count(H);
  if (grad)
    for (int i = 0; i < np; ++i) grad[i] = 0.0;
  double* gW1 = grad;
  double* gb1 = grad ? gW1 + H * 5 : nullptr;
  double* gW2 = grad ? gb1 + H : nullptr;
  double* gb2 = grad ? gW2 + H * H : nullptr;
  double* gW3 = grad ? gb2 + H : nullptr;
  double* gb3 = grad ? gW3 + H * H : nullptr;
  double* gW4 = grad ? gb3 + H : nullptr;
  double* gb4 = grad ? gW4 + H : nullptr;
  std::vector<double> h1(H), h2(H), h3(H), d1(H), d2(H), d3(H);
  double loss = 0.0;
  for (int i = 0; i < n; ++i) {
    const double* xi = &x[5 * i];
    // forward: h_l = tanh(W_l h_{l-1} + b_l), output linear
    for (int j = 0; j < H; ++j) {
      double s = b1[j];
      for (int k = 0; k < 5; ++k) s += W1[j * 5 + k] * xi[k];
      h1[j] = std::tanh(s);
    }
    for (int j = 0; j < H; ++j) {
      double s = b2[j];
      for (int k = 0; k < H; ++k) s += W2[j * H + k] * h1[k];
      h2[j] = std::tanh(s);
    }
    for (int j = 0; j < H; ++j) {
      double s = b3[j];
      for (int k = 0; k < H; ++k) s += W3[j * H + k] * h2[k];
      h3[j] = std::tanh(s);
    }
    double out = b4[0];
    for (int k = 0; k < H; ++k) out += W4[k] * h3[k];
    if (y) y[i] = out;
    double wi = wt ? wt[i] : 1.0;
    double r = target ? out - target[i] : 0.0;
    loss += wi * r * r / n;
    if (!grad) continue;
    // backward, chain rule layer by layer
    double dout = 2.0 * wi * r / n;
    gb4[0] += dout;
    for (int k = 0; k < H; ++k) {
      gW4[k] += dout * h3[k];
      d3[k] = dout * W4[k] * (1.0 - h3[k] * h3[k]);
    }
    for (int j = 0; j < H; ++j) {
      gb3[j] += d3[j];
      for (int k = 0; k < H; ++k) gW3[j * H + k] += d3[j] * h2[k];
    }
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int j = 0; j < H; ++j) s += W3[j * H + k] * d3[j];
      d2[k] = s * (1.0 - h2[k] * h2[k]);
    }
    for (int j = 0; j < H; ++j) {
      gb2[j] += d2[j];
      for (int k = 0; k < H; ++k) gW2[j * H + k] += d2[j] * h1[k];
    }
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int j = 0; j < H; ++j) s += W2[j * H + k] * d2[j];
      d1[k] = s * (1.0 - h1[k] * h1[k]);
    }
    for (int j = 0; j < H; ++j) {
      gb1[j] += d1[j];
      for (int k = 0; k < 5; ++k) gW1[j * 5 + k] += d1[j] * xi[k];
    }
  }
  return loss;
}

}  // extern "C"
