// Host half of libmcgb: the C ABI declared in include/mc.h.
//
// mc_problem_create validates a problem description, builds the sampling tables (channel
// thresholds, scatter-group and secondary-spectrum CDFs, geometry and tally tables) once in FP64
// and packs them into two blobs (FP32 and FP64 tracking) that every CTA stages into shared memory.
// mc_run zeroes the per-batch tallies, launches the persistent transport kernel cooperatively and
// the batch-statistics kernel on the caller's stream.  Readback calls synchronise and turn batch
// sums into per-source-particle means and standard errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mc_host.h"
#include "mc_tables.h"

namespace mcgb {
template <typename R>
cudaError_t launch_transport(const RunParams& P, int grid, int block, size_t smem, cudaStream_t s, bool wide,
                             bool range);
template <typename R>
cudaError_t transport_occupancy(int block, size_t smem, int* per_sm, bool wide, bool range, bool seg);
cudaError_t launch_scan_sites(const uint32_t* counts, unsigned long long* scan, unsigned long long* block_sums, uint64_t n,
                              cudaStream_t s);
cudaError_t launch_comb(const uint32_t* counts, const unsigned long long* scan, const uint4* sites, uint32_t nmax,
                        uint64_t n, uint64_t seed, uint32_t next_cycle, uint4* src, int lanes, cudaStream_t s);
template <typename R>
cudaError_t launch_pc(const RunParams& P, const RunParams& Q, const unsigned long long* pc_n, long long* wq,
                      unsigned long long* out_n, unsigned long long* copies, int* status, bool split, cudaStream_t s);
size_t comb_scratch_bytes(uint64_t n, int nb);
template <typename R>
cudaError_t launch_comb_pc(const RunParams& P, const RunParams& Q, uint64_t n, const long long* wb, uint32_t census,
                           void* scratch, size_t scratch_bytes, unsigned long long* out_n, unsigned long long* copies,
                           int* status, cudaStream_t s);
cudaError_t launch_reconstruct(void* tally, const char* blob64, uint64_t rows, uint64_t row, int nb, int stripes,
                               int fp64, cudaStream_t s);
cudaError_t launch_batch_stats(const void* tally, int fp64, uint64_t bins, uint64_t row, int nb, int stripes,
                               uint64_t n_hist, void* out, cudaStream_t s);
cudaError_t launch_op_probe(int op, int grid, int iters, unsigned long long* sink, unsigned long long* clk,
                            cudaStream_t s);
cudaError_t launch_philox(uint64_t seed, const uint4* ctr, uint4* out, uint64_t n, cudaStream_t s);
cudaError_t launch_atomic_probe(unsigned long long* a, unsigned long long span, int grid, int iters, unsigned salt,
                                cudaStream_t s);
}  // namespace mcgb

using namespace mcgb;

static const uint64_t kTraceCap = 65536;

// ------------------------------------------------------------------------------------------ errors
static thread_local std::string g_err;

namespace mcgb {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  // reset the runtime's last-error state, so that a failed call (an attribute, an allocation) is not
  // reported again by the next library call that checks cudaGetLastError after a launch
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

int check_shared_memory(int dev, size_t bytes, const char* what) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (bytes > (size_t)optin)
    return fail(MC_ERR_INVALID,
                "%s needs %zu B of shared memory per CTA (the problem's tables and the per-warp queues); "
                "the device allows %d B: fewer materials x groups, surfaces, cells or lattice elements",
                what, bytes, optin);
  return MC_OK;
}

int current_device(int* dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  return MC_OK;
}

// ------------------------------------------------------------------------------------------ memory pool
// Device blocks are recycled across problems instead of returned to the driver, so creating and
// destroying problems in a loop does not pay cudaMalloc/cudaFree each time.
struct PoolBlock {
  int dev;
  void* ptr;
};
static std::mutex g_pool_mu;
static std::multimap<size_t, PoolBlock> g_pool;

int check_implicit_opts(const mc_run_opts& o) {
  if (o.implicit_capture != 0 && o.implicit_capture != 1) return fail(MC_ERR_INVALID, "implicit_capture must be 0 or 1");
  if (o.implicit_capture &&
      !(std::isfinite(o.wr_cutoff) && std::isfinite(o.wr_survival) && o.wr_cutoff >= 0.0 && o.wr_survival > o.wr_cutoff))
    return fail(MC_ERR_INVALID, "implicit capture needs 0 <= wr_cutoff < wr_survival (finite)");
  return MC_OK;
}

int pool_alloc(void** out, size_t bytes, int dev) {
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto it = g_pool.lower_bound(bytes); it != g_pool.end() && it->first <= 2 * bytes + (1 << 20); ++it) {
      if (it->second.dev == dev) {
        *out = it->second.ptr;
        g_pool.erase(it);
        return MC_OK;
      }
    }
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    // release cached blocks of this device and retry once
    std::vector<void*> drop;
    {
      std::lock_guard<std::mutex> lk(g_pool_mu);
      for (auto it = g_pool.begin(); it != g_pool.end();) {
        if (it->second.dev == dev) {
          drop.push_back(it->second.ptr);
          it = g_pool.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (void* d : drop) cudaFree(d);
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  }
  *out = p;
  return MC_OK;
}

// a block must be returned with the size it was requested with
void pool_free(void* p, size_t bytes, int dev) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  g_pool.insert({bytes, PoolBlock{dev, p}});
}

}  // namespace mcgb

namespace {

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

int validate(const mc_problem_desc* d) {
  if (!d) return fail(MC_ERR_INVALID, "descriptor is NULL");
  const int G = d->n_groups, M = d->n_materials;
  if (G < 1 || G > MC_MAX_GROUPS) return fail(MC_ERR_INVALID, "n_groups=%d outside [1,%d]", G, MC_MAX_GROUPS);
  if (M < 1 || M > MC_MAX_MATERIALS) return fail(MC_ERR_INVALID, "n_materials=%d outside [1,%d]", M, MC_MAX_MATERIALS);
  if (!d->sigma_t || !d->sigma_s || !d->sigma_f || !d->nu || !d->chi || !d->speed)
    return fail(MC_ERR_INVALID, "cross-section array is NULL");
  for (int g = 0; g < G; ++g)
    if (!(std::isfinite(d->speed[g]) && d->speed[g] > 0.0)) return fail(MC_ERR_INVALID, "speed[%d] must be > 0", g);
  for (int m = 0; m < M; ++m) {
    double chi_sum = 0.0;
    bool any_f = false;
    for (int g = 0; g < G; ++g) {
      const double st = d->sigma_t[m * G + g], sf = d->sigma_f[m * G + g], nu = d->nu[m * G + g];
      const double ch = d->chi[m * G + g];
      if (!finite_nonneg(st) || !finite_nonneg(sf) || !finite_nonneg(nu) || !finite_nonneg(ch))
        return fail(MC_ERR_INVALID, "material %d group %d: negative or non-finite data", m, g);
      if (nu > 64.0) return fail(MC_ERR_INVALID, "material %d group %d: nu above 64", m, g);
      double ss = 0.0;
      for (int h = 0; h < G; ++h) {
        const double v = d->sigma_s[(m * G + g) * G + h];
        if (!finite_nonneg(v)) return fail(MC_ERR_INVALID, "material %d sigma_s[%d][%d] invalid", m, g, h);
        ss += v;
      }
      if (ss + sf > st * (1.0 + 1e-12))
        return fail(MC_ERR_INVALID, "material %d group %d: sigma_s + sigma_f exceeds sigma_t", m, g);
      chi_sum += ch;
      any_f = any_f || (sf > 0.0 && nu > 0.0);
    }
    if (any_f && !(chi_sum > 0.0)) return fail(MC_ERR_INVALID, "material %d produces secondaries but chi sums to 0", m);
  }
  if (d->n_surfaces < 1 || d->n_surfaces > MC_MAX_SURFACES || !d->surfaces)
    return fail(MC_ERR_INVALID, "n_surfaces=%d outside [1,%d]", d->n_surfaces, MC_MAX_SURFACES);
  for (int s = 0; s < d->n_surfaces; ++s) {
    const mc_surface& S = d->surfaces[s];
    if (S.kind < MC_SURF_PX || S.kind > MC_SURF_GQ) return fail(MC_ERR_INVALID, "surface %d: bad kind", s);
    if (S.bc < MC_BC_INTERIOR || S.bc > MC_BC_REFLECT) return fail(MC_ERR_INVALID, "surface %d: bad bc", s);
    if (S.kind > MC_SURF_PZ && S.bc == MC_BC_REFLECT)
      return fail(MC_ERR_INVALID, "surface %d: reflection is supported on planes only", s);
    for (int i = 0; i < 10; ++i)
      if (!std::isfinite(S.coef[i])) return fail(MC_ERR_INVALID, "surface %d: non-finite coefficient", s);
    const double radius = S.kind == MC_SURF_SQ ? S.coef[3] : S.coef[2];
    if ((S.kind == MC_SURF_CZ || S.kind == MC_SURF_CX || S.kind == MC_SURF_CY || S.kind == MC_SURF_SQ) &&
        !(radius > 0.0))
      return fail(MC_ERR_INVALID, "surface %d: radius must be > 0", s);
  }
  if (d->n_cells < 1 || d->n_cells > MC_MAX_CELLS || !d->cells)
    return fail(MC_ERR_INVALID, "n_cells=%d outside [1,%d]", d->n_cells, MC_MAX_CELLS);
  bool uses_lattice = false;
  for (int c = 0; c < d->n_cells; ++c) {
    const mc_cell& C = d->cells[c];
    if (C.n_halfspaces < 1 || C.n_halfspaces > MC_MAX_HALFSPACES)
      return fail(MC_ERR_INVALID, "cell %d: n_halfspaces=%d outside [1,%d]", c, C.n_halfspaces, MC_MAX_HALFSPACES);
    for (int i = 0; i < C.n_halfspaces; ++i) {
      if (C.surface[i] < 0 || C.surface[i] >= d->n_surfaces) return fail(MC_ERR_INVALID, "cell %d: bad surface", c);
      if (C.sense[i] != 1 && C.sense[i] != -1) return fail(MC_ERR_INVALID, "cell %d: sense must be +-1", c);
    }
    if (C.material == -1) uses_lattice = true;
    else if (C.material < 0 || C.material >= M) return fail(MC_ERR_INVALID, "cell %d: bad material", c);
  }
  if (uses_lattice || d->lattice) {
    const mc_lattice* L = d->lattice;
    if (!L) return fail(MC_ERR_INVALID, "a cell uses the lattice but no lattice is given");
    if (L->nx < 1 || L->ny < 1 || L->nx > MC_MAX_LATTICE || L->ny > MC_MAX_LATTICE || L->nz < 0 ||
        L->nz > MC_MAX_LATTICE)
      return fail(MC_ERR_INVALID, "lattice size outside [1,%d] (nz in [0,%d])", MC_MAX_LATTICE, MC_MAX_LATTICE);
    const int nz = L->nz > 1 ? L->nz : 1;
    if (L->nx * L->ny * nz > MC_MAX_LATTICE_ELEMENTS)
      return fail(MC_ERR_INVALID, "lattice has more than %d elements", MC_MAX_LATTICE_ELEMENTS);
    if (!(L->pitch > 0.0) || !(L->radius > 0.0) || !(2.0 * L->radius < L->pitch) || !std::isfinite(L->x0) ||
        !std::isfinite(L->y0))
      return fail(MC_ERR_INVALID, "lattice needs pitch > 2 radius > 0");
    if (nz > 1 && (!(L->pitch_z > 0.0) || !std::isfinite(L->pitch_z) || !std::isfinite(L->z0)))
      return fail(MC_ERR_INVALID, "an axially layered lattice needs a finite z0 and pitch_z > 0");
    if (!L->pin_material) return fail(MC_ERR_INVALID, "lattice pin_material is NULL");
    for (int i = 0; i < L->nx * L->ny * nz; ++i)
      if (L->pin_material[i] < -1 || L->pin_material[i] >= M) return fail(MC_ERR_INVALID, "lattice pin %d: bad material", i);
    if (L->matrix_material < 0 || L->matrix_material >= M) return fail(MC_ERR_INVALID, "lattice matrix material");
  }
  const mc_source& S = d->source;
  if (S.pos < MC_SRC_BOX || S.pos > MC_SRC_SURFACE_X0 || S.dir < MC_DIR_ISO || S.dir > MC_DIR_COS_X)
    return fail(MC_ERR_INVALID, "source kind");
  if (!S.group_pdf) return fail(MC_ERR_INVALID, "source group_pdf is NULL");
  double gs = 0.0;
  for (int g = 0; g < G; ++g) {
    if (!finite_nonneg(S.group_pdf[g])) return fail(MC_ERR_INVALID, "source group_pdf[%d] invalid", g);
    gs += S.group_pdf[g];
  }
  if (!(gs > 0.0)) return fail(MC_ERR_INVALID, "source group_pdf sums to 0");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(S.lo[i]) || !std::isfinite(S.hi[i]) || S.hi[i] < S.lo[i])
      return fail(MC_ERR_INVALID, "source box must be finite with hi >= lo");
  if (!std::isfinite(S.t0) || !std::isfinite(S.t1) || S.t1 < S.t0 || S.t0 < 0.0)
    return fail(MC_ERR_INVALID, "source times need 0 <= t0 <= t1");
  if (d->n_tallies < 0 || d->n_tallies > MC_MAX_TALLIES || (d->n_tallies > 0 && !d->tallies))
    return fail(MC_ERR_INVALID, "n_tallies=%d outside [0,%d]", d->n_tallies, MC_MAX_TALLIES);
  uint64_t bins = 0;
  for (int t = 0; t < d->n_tallies; ++t) {
    const mc_mesh_tally& T = d->tallies[t];
    const int n[4] = {T.nx, T.ny, T.nz, T.nt};
    const double* e[4] = {T.x, T.y, T.z, T.t};
    if (T.estimator != MC_EST_TRACK_LENGTH && T.estimator != MC_EST_TIME_CROSSING)
      return fail(MC_ERR_INVALID, "tally %d: unknown estimator %d", t, T.estimator);
    const bool crossing = T.estimator == MC_EST_TIME_CROSSING;
    for (int k = 0; k < 4; ++k) {
      if (n[k] < 1 || n[k] > (1 << 16) || !e[k]) return fail(MC_ERR_INVALID, "tally %d axis %d: bad size", t, k);
      for (int i = 0; i <= n[k]; ++i) {
        if (std::isnan(e[k][i])) return fail(MC_ERR_INVALID, "tally %d: NaN edge", t);
        if ((i > 0 && i < n[k] && !std::isfinite(e[k][i])) || (i > 0 && !(e[k][i] > e[k][i - 1])))
          return fail(MC_ERR_INVALID, "tally %d axis %d: edges must increase (infinite only at the ends)", t, k);
        if (k == 3 && crossing && !std::isfinite(e[k][i]))
          return fail(MC_ERR_INVALID, "tally %d: time-crossing points must be finite", t);
      }
    }
    bins += (uint64_t)T.nx * T.ny * T.nz * (T.nt + (crossing ? 1 : 0)) * G;
    if (ranges_time_bins(T.nx, T.ny, T.nz, T.nt)) bins += (uint64_t)T.nx * T.ny * T.nz * (T.nt + 2) * G;
  }
  if (bins + d->n_surfaces > (1ull << 30)) return fail(MC_ERR_INVALID, "tallies too large");
  if (!(d->t_census > 0.0)) return fail(MC_ERR_INVALID, "t_census must be > 0 (inf for steady state)");
  return MC_OK;
}

// cumulative distribution of a non-negative row (summed in index order), normalised; entries from
// the last positive one on are exactly 1 so that any u < 1 selects a bin with positive weight
void cdf_row(const double* row, int n, double* out) {
  double total = 0.0;
  for (int i = 0; i < n; ++i) total += row[i];
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    acc += row[i];
    out[i] = total > 0.0 ? acc / total : (i == n - 1 ? 1.0 : 0.0);
  }
  int last = n - 1;
  while (last > 0 && !(row[last] > 0.0)) --last;
  for (int i = last; i < n; ++i) out[i] = 1.0;
}

struct Blob {
  std::vector<uint8_t> b;
  Blob() : b(sizeof(TableHeader), 0) {}
  int put(const void* src, size_t bytes) {
    size_t off = (b.size() + 15) & ~size_t(15);
    b.resize(off + ((bytes + 15) & ~size_t(15)), 0);
    if (bytes) std::memcpy(b.data() + off, src, bytes);
    return (int)off;
  }
  template <typename T>
  int put(const std::vector<T>& v) {
    return put(v.data(), v.size() * sizeof(T));
  }
  TableHeader* hdr() { return reinterpret_cast<TableHeader*>(b.data()); }
};

template <typename R>
std::vector<uint8_t> build_blob(const mc_problem_desc* d) {
  const int G = d->n_groups, M = d->n_materials;
  Blob B;
  TableHeader H;
  std::memset(&H, 0, sizeof(H));
  H.G = G;
  H.M = M;
  H.n_surf = d->n_surfaces;
  H.n_cell = d->n_cells;
  H.real_bytes = (int)sizeof(R);
  H.t_census = d->t_census;
  for (int i = 0; i < 3; ++i) {
    H.src_lo[i] = d->source.lo[i];
    H.src_hi[i] = d->source.hi[i];
  }
  H.src_t0 = d->source.t0;
  H.src_t1 = d->source.t1;
  H.src_pos = d->source.pos;
  H.src_dir = d->source.dir;
  for (int i = 0; i < 3; ++i) {
    H.src_lo_f[i] = (float)d->source.lo[i];
    H.src_hi_f[i] = (float)d->source.hi[i];
  }
  H.src_t0_f = (float)d->source.t0;
  H.src_t1_f = (float)d->source.t1;
  H.has_census = std::isfinite(d->t_census) ? 1 : 0;
  if (H.has_census) {
    H.tc_hi = (float)d->t_census;
    H.tc_lo = (float)(d->t_census - (double)H.tc_hi);
  }
  std::vector<R> st(M * G), ss(M * G), ssf(M * G), nu(M * G), nusf(M * G), scdf(M * G * G), chi(M * G);
  std::vector<double> tmp(G);
  for (int m = 0; m < M; ++m) {
    for (int g = 0; g < G; ++g) {
      const double* row = d->sigma_s + (m * G + g) * G;
      double s = 0.0;
      for (int h = 0; h < G; ++h) s += row[h];
      st[m * G + g] = (R)d->sigma_t[m * G + g];
      ss[m * G + g] = (R)s;
      ssf[m * G + g] = (R)(s + d->sigma_f[m * G + g]);
      nu[m * G + g] = (R)d->nu[m * G + g];
      nusf[m * G + g] = (R)(d->nu[m * G + g] * d->sigma_f[m * G + g]);
      cdf_row(row, G, tmp.data());
      for (int h = 0; h < G; ++h) scdf[(m * G + g) * G + h] = (R)tmp[h];
    }
    cdf_row(d->chi + m * G, G, tmp.data());
    for (int h = 0; h < G; ++h) chi[m * G + h] = (R)tmp[h];
  }
  std::vector<R> v(G), inv_v(G), src(G);
  for (int g = 0; g < G; ++g) {
    v[g] = (R)d->speed[g];
    inv_v[g] = (R)(1.0 / d->speed[g]);
  }
  cdf_row(d->source.group_pdf, G, tmp.data());
  for (int g = 0; g < G; ++g) src[g] = (R)tmp[g];
  H.o_st = B.put(st);
  H.o_ss = B.put(ss);
  H.o_ssf = B.put(ssf);
  H.o_nu = B.put(nu);
  H.o_nusf = B.put(nusf);
  H.o_v = B.put(v);
  H.o_inv_v = B.put(inv_v);
  H.o_scdf = B.put(scdf);
  H.o_chi = B.put(chi);
  H.o_src_cdf = B.put(src);
  std::vector<int> skind(H.n_surf), sbc(H.n_surf);
  // per surface kSurfStride values: [0..2] the plane / z-cylinder coefficients, [3..12] the quadric
  // A..J about the centre [13..15] for the other kinds (cylinders and spheres centred on their axis
  // or centre, so that their f stays well conditioned far from the origin)
  std::vector<R> scoef(kSurfStride * H.n_surf, R(0));
  for (int s = 0; s < H.n_surf; ++s) {
    const mc_surface& S = d->surfaces[s];
    skind[s] = S.kind;
    sbc[s] = S.bc;
    R* c = &scoef[kSurfStride * s];
    for (int i = 0; i < 3; ++i) c[i] = (R)S.coef[i];
    double q[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, ctr[3] = {0, 0, 0};
    switch (S.kind) {
      case MC_SURF_CX: q[1] = q[2] = 1.0; q[9] = -S.coef[2] * S.coef[2]; ctr[1] = S.coef[0]; ctr[2] = S.coef[1]; break;
      case MC_SURF_CY: q[0] = q[2] = 1.0; q[9] = -S.coef[2] * S.coef[2]; ctr[0] = S.coef[0]; ctr[2] = S.coef[1]; break;
      case MC_SURF_SQ:
        q[0] = q[1] = q[2] = 1.0;
        q[9] = -S.coef[3] * S.coef[3];
        for (int i = 0; i < 3; ++i) ctr[i] = S.coef[i];
        break;
      case MC_SURF_GQ: for (int i = 0; i < 10; ++i) q[i] = S.coef[i]; break;
      default: break;
    }
    for (int i = 0; i < 10; ++i) c[3 + i] = (R)q[i];
    for (int i = 0; i < 3; ++i) c[13 + i] = (R)ctr[i];
  }
  H.o_skind = B.put(skind);
  H.o_sbc = B.put(sbc);
  H.o_scoef = B.put(scoef);
  std::vector<int> nhs(H.n_cell), hs(H.n_cell * MC_MAX_HALFSPACES, 0), cmat(H.n_cell);
  for (int c = 0; c < H.n_cell; ++c) {
    const mc_cell& C = d->cells[c];
    nhs[c] = C.n_halfspaces;
    for (int i = 0; i < C.n_halfspaces; ++i)
      hs[c * MC_MAX_HALFSPACES + i] = C.surface[i] | (C.sense[i] < 0 ? (1 << 16) : 0);
    cmat[c] = C.material;
    if (C.material < 0) H.has_lat = 1;
  }
  H.o_nhs = B.put(nhs);
  H.o_hs = B.put(hs);
  H.o_cmat = B.put(cmat);
  // box cells: the walk takes the one plane per axis that the direction of motion can leave by
  std::vector<int> cbox((size_t)H.n_cell * 7, -1);
  for (int c = 0; c < H.n_cell; ++c) box_cell_entry(d->cells[c], d->surfaces, &cbox[(size_t)c * 7]);
  H.o_cbox = B.put(cbox);
  if (d->lattice) {
    const mc_lattice* L = d->lattice;
    H.has_lat = 1;
    H.lat_nx = L->nx;
    H.lat_ny = L->ny;
    H.lat_matrix = L->matrix_material;
    H.lat_x0 = L->x0;
    H.lat_y0 = L->y0;
    H.lat_pitch = L->pitch;
    H.lat_r = L->radius;
    H.lat_nz = L->nz > 1 ? L->nz : 1;
    H.lat_z0 = H.lat_nz > 1 ? L->z0 : 0.0;
    H.lat_pz = H.lat_nz > 1 ? L->pitch_z : 1.0;
    H.lat_mx = ((1ull << 32) + (unsigned long long)L->nx - 1) / (unsigned long long)L->nx;
    H.lat_my = ((1ull << 32) + (unsigned long long)L->ny - 1) / (unsigned long long)L->ny;
    // one byte per element (the tables live in shared memory): material, or kNoPin
    std::vector<uint8_t> pins((size_t)L->nx * L->ny * H.lat_nz);
    for (size_t i = 0; i < pins.size(); ++i) pins[i] = L->pin_material[i] < 0 ? kNoPin : (uint8_t)L->pin_material[i];
    H.o_lpin = B.put(pins);
  } else {
    H.has_lat = 0;
    H.lat_nz = 1;
    H.lat_mx = H.lat_my = 1ull << 32;
    std::vector<uint8_t> none(1, kNoPin);
    H.o_lpin = B.put(none);
  }
  H.n_tally = d->n_tallies;
  int off = 0, doff = 0;
  for (int t = 0; t < d->n_tallies; ++t) {
    const mc_mesh_tally& T = d->tallies[t];
    TallyDesc& D = H.tally[t];
    D.nx = T.nx;
    D.ny = T.ny;
    D.nz = T.nz;
    D.nt = T.nt;
    std::vector<R> ex(T.x, T.x + T.nx + 1), ey(T.y, T.y + T.ny + 1), ez(T.z, T.z + T.nz + 1);
    std::vector<double> et(T.t, T.t + T.nt + 1);
    std::vector<float> etf(T.t, T.t + T.nt + 1);
    D.o_ex = B.put(ex);
    D.o_ey = B.put(ey);
    D.o_ez = B.put(ez);
    D.o_et = B.put(et);
    D.o_etf = B.put(etf);
    {
      const std::vector<float> exf(T.x, T.x + T.nx + 1), eyf(T.y, T.y + T.ny + 1), ezf(T.z, T.z + T.nz + 1);
      const std::vector<float>* axes[4] = {&exf, &eyf, &ezf, &etf};
      for (int a = 0; a < 4; ++a) bin_guess_params(*axes[a], D.gkind[a], D.ga[a], D.gb[a]);
    }
    D.bin_offset = off;
    D.est = T.estimator;
    D.nval = T.nt + (T.estimator == MC_EST_TIME_CROSSING ? 1 : 0);
    D.n_bins = T.nx * T.ny * T.nz * G * D.nval;
    D.range = ranges_time_bins(T.nx, T.ny, T.nz, T.nt) ? 1 : 0;
    D.diff_offset = doff;
    D.ndiff = T.nt + (T.estimator == MC_EST_TIME_CROSSING ? 2 : 1);
    if (D.range) doff += T.nx * T.ny * T.nz * G * D.ndiff;
    off += D.n_bins;
  }
  H.leak_offset = off;
  H.total_bins = off + H.n_surf;
  H.total_diff = doff;
  B.b.resize((B.b.size() + 15) & ~size_t(15), 0);
  H.blob_bytes = (int)B.b.size();
  *B.hdr() = H;
  return B.b;
}

}  // namespace

// ------------------------------------------------------------------------------------------ ABI
namespace mcgb {

// Shared memory of one warp of the transport kernel besides the tables: its flight queue (64
// particles) and, where the tally adds are warp-aggregated, its tally staging buffer (128 x 12 B).
size_t transport_warp_smem(int fp64, bool aggregate) {
  return (size_t)kWarpQ * 16 * (fp64 ? kLanesFP64 : kLanesFP32) + (aggregate ? (size_t)kStage * 12 : 0);
}

// NVTX range over a library call or a phase of it (visible to nsys / ncu when a tool is attached;
// header-only, no cost otherwise)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// the launch's census: the problem's t_census unless population control sets an interior one
void set_census(RunParams& P, double t, bool interior) {
  P.has_census = std::isfinite(t) ? 1 : 0;
  P.tc = t;
  P.tc_hi = P.has_census ? (float)t : 0.0f;
  P.tc_lo = P.has_census ? (float)(t - (double)P.tc_hi) : 0.0f;
  P.pc_interior = interior ? 1 : 0;
}

void fill_run_params(const mc_problem* p, const mc_run_opts& o, uint64_t n_histories, uint64_t seed,
                     uint32_t stripes, RunParams& P) {
  const int fp64 = o.precision == MC_FP64;
  const int nb = o.n_batches;
  const uint64_t bins = (uint64_t)p->total_bins;
  P.n_sources = n_histories;
  set_census(P, reinterpret_cast<const TableHeader*>(p->blob[1].data())->t_census, false);
  P.ctl = (Ctl*)p->d_ctl.ptr;
  P.sticky = (int*)p->d_sticky.ptr;
  P.tally = p->d_tally.ptr;
  P.tally_stripes = stripes;
  P.row = p->row;
  P.stripe_stride = (uint64_t)nb * p->row;
  P.tally_fp64 = o.tally_mode == MC_TALLY_FP64;
  // auto: one fire-and-forget atomic per score.  Warp aggregation (match + shuffle tree through a
  // shared-memory stage) was the default for small unstriped tallies, i.e. the batched launch; there
  // it measured slower (the 256-problem workload: 85 ms per launch aggregated, 69 ms direct), so it
  // is kept only as an option for tallies with a few very hot bins.
  (void)bins;
  P.aggregate = o.aggregate_atomics >= 0 ? o.aggregate_atomics : 0;
  P.fixed_scale = std::ldexp(1.0, o.fixed_bits);
  P.fixed_scale_f = (float)P.fixed_scale;
  P.n_hist = n_histories;
  P.hist_per_batch = (n_histories + nb - 1) / nb;
  {
    const double mg = std::floor(4294967296.0 * (double)nb / (double)n_histories);
    P.batch_magic = mg >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)mg;
  }
  P.n_batches = nb;
  P.blob_bytes = (int)p->blob[fp64].size();
  P.blob = (const uint4*)p->d_blob[fp64].ptr;
  P.seed = seed;
  P.max_iter = o.max_iterations ? o.max_iterations : (1ull << 20);
  P.implicit = o.implicit_capture;
  P.wr_cutoff = o.wr_cutoff;
  P.wr_survival = o.wr_survival;
  if (o.ww_enable) {
    const double* base = (const double*)p->d_ww.ptr;
    P.ww_on = 1;
    P.ww_nx = p->ww_n[0];
    P.ww_ny = p->ww_n[1];
    P.ww_nz = p->ww_n[2];
    P.ww_nt = p->ww_n[3];
    P.ww_edges = base;
    P.ww_center = base + (p->ww_n[0] + 1) + (p->ww_n[1] + 1) + (p->ww_n[2] + 1) + (p->ww_n[3] + 1);
    P.ww_upper = 2.0;
    P.ww_lower = 0.5;
    P.ww_split_max = 10;
  }
}

}  // namespace mcgb

extern "C" {

const char* mc_last_error(void) { return g_err.c_str(); }

void mc_run_opts_default(mc_run_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MC_FP32;
  o->tally_mode = MC_TALLY_FIXED64;
  o->fixed_bits = 32;
  o->n_batches = 32;
  o->aggregate_atomics = -1;
  o->wr_cutoff = 0.25;
  o->wr_survival = 0.5;
}

int mc_problem_create(const mc_problem_desc* d, mc_problem** out) {
  g_err.clear();
  if (!out) return fail(MC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = validate(d);
  if (rc != MC_OK) return rc;
  mc_problem* p = new mc_problem();
  p->G = d->n_groups;
  p->M = d->n_materials;
  p->n_surf = d->n_surfaces;
  p->n_cell = d->n_cells;
  p->n_tally = d->n_tallies;
  for (int t = 0; t < d->n_tallies; ++t) {
    const mc_mesh_tally& T = d->tallies[t];
    HostTally h;
    h.n[0] = T.nx;
    h.n[1] = T.ny;
    h.n[2] = T.nz;
    h.n[3] = T.nt;
    h.est = T.estimator;
    h.nval = T.nt + (T.estimator == MC_EST_TIME_CROSSING ? 1 : 0);
    const double* e[4] = {T.x, T.y, T.z, T.t};
    for (int k = 0; k < 4; ++k) h.e[k].assign(e[k], e[k] + h.n[k] + 1);
    p->range = p->range || ranges_time_bins(T.nx, T.ny, T.nz, T.nt);
    p->tallies.push_back(h);
  }
  for (int i = 0; i < 3; ++i) p->src_center[i] = 0.5 * (d->source.lo[i] + d->source.hi[i]);
  if (d->source.pos == MC_SRC_SURFACE_X0) p->src_center[0] = d->source.lo[0];
  for (int g = 1; g < p->G; ++g)
    if (d->source.group_pdf[g] > d->source.group_pdf[p->src_group]) p->src_group = g;
  p->blob[0] = build_blob<float>(d);
  p->blob[1] = build_blob<double>(d);
  const TableHeader* H = reinterpret_cast<const TableHeader*>(p->blob[0].data());
  p->total_bins = H->total_bins;
  p->leak_offset = H->leak_offset;
  p->row = (uint64_t)H->total_bins + (uint64_t)H->total_diff;
  for (int i = 0; i < p->M * p->G; ++i) p->nu_max = std::max(p->nu_max, d->sigma_f[i] > 0.0 ? d->nu[i] : 0.0);
  for (int t = 0; t < H->n_tally; ++t)
    if (H->tally[t].range) p->range_rows += (uint64_t)H->tally[t].nx * H->tally[t].ny * H->tally[t].nz * H->G;
  rc = current_device(&p->dev);
  for (int i = 0; i < 2 && rc == MC_OK; ++i) {
    rc = p->d_blob[i].ensure(p->blob[i].size(), p->dev);
    if (rc == MC_OK) {
      cudaError_t e = cudaMemcpy(p->d_blob[i].ptr, p->blob[i].data(), p->blob[i].size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) rc = cuda_fail(e, "upload tables");
    }
  }
  if (rc == MC_OK) rc = p->d_ctl.ensure(sizeof(Ctl), p->dev);
  if (rc == MC_OK) rc = p->d_sticky.ensure(16, p->dev);
  if (rc == MC_OK) {
    cudaError_t e = cudaMemset(p->d_sticky.ptr, 0, 16);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset");
  }
  for (int i = 0; i < 3 && rc == MC_OK; ++i) {
    cudaError_t e = cudaEventCreate(&p->ev[i]);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventCreate");
  }
  if (rc != MC_OK) {
    mc_problem_destroy(p);
    return rc;
  }
  *out = p;
  return MC_OK;
}

void mc_problem_destroy(mc_problem* p) {
  if (!p) return;
  if (p->has_run && p->stream) cudaStreamSynchronize(p->stream);
  p->d_blob[0].release();
  p->d_blob[1].release();
  p->d_ctl.release();
  p->d_tally.release();
  p->d_stats.release();
  p->d_log.release();
  p->d_banks.release();
  p->d_trace.release();
  p->d_sticky.release();
  p->d_ww.release();
  p->d_wstack.release();
  // k-eigenvalue and population-control buffers
  p->d_sites.release();
  p->d_counts.release();
  p->d_scan.release();
  p->d_blocksums.release();
  p->d_src.release();
  p->d_cbank.release();
  p->d_pc.release();
  p->d_comb.release();
  if (p->own_mlp) mc_mlp_destroy(p->own_mlp);
  for (int i = 0; i < 3; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  delete p;
}

// Population control: one transport launch per interval between census times.  After an interior
// census the banked particles' batch weights are summed exactly, splitting-roulette or the comb
// writes the copies into the next launch's birth bank, and the next launch starts from them alone.  The run's
// counters (and the event log count) are summed over the intervals on the host and written back
// into the control block at the end.
int run_population_controlled(mc_problem* p, const RunParams& P0, const std::vector<double>& census, double t_final,
                              int grid, int block, size_t smem, bool wide, bool range, int fp64, int lanes,
                              uint64_t cap, bool comb, cudaStream_t s) {
  int rc = p->d_cbank.ensure((size_t)cap * 16 * lanes, p->dev);
  const int nb = P0.n_batches;
  if (rc == MC_OK) rc = p->d_pc.ensure((size_t)(nb + 4) * 8, p->dev);
  if (rc != MC_OK) return rc;
  long long* wq = (long long*)p->d_pc.ptr;
  unsigned long long* out_n = (unsigned long long*)(wq + nb);
  unsigned long long* copies = out_n + 1;
  int* status = (int*)(copies + 1);
  std::vector<unsigned long long> cnt(MC_NCOUNTERS, 0ull);
  unsigned long long iterations = 0, log_n = 0;
  RunParams prev = P0;
  const int K = (int)census.size();
  auto harvest = [&](int* st, unsigned long long* banked) -> int {  // the finished launch's counters
    Ctl c;
    CK(cudaMemcpyAsync(&c, p->d_ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < MC_NCOUNTERS; ++i) cnt[i] += c.counters[i];
    iterations += c.iterations;
    log_n = c.log_n;
    *st = c.status;
    *banked = c.pc_n;
    return MC_OK;
  };
  for (int i = 0; i <= K; ++i) {
    NvtxRange interval_range("census interval");
    RunParams Q = P0;
    Q.n_sources = i == 0 ? P0.n_sources : 0;
    set_census(Q, i < K ? census[i] : t_final, i < K);
    char* cb = (char*)p->d_cbank.ptr;
    for (int l = 0; l < lanes; ++l) Q.C[l] = (uint4*)(cb + (size_t)l * cap * 16);
    Q.cap_c = cap;
    if (i > 0) {
      CK(cudaMemsetAsync(p->d_pc.ptr, 0, (size_t)(nb + 4) * 8, s));
      const unsigned long long* pc_n = (const unsigned long long*)((const char*)p->d_ctl.ptr + offsetof(Ctl, pc_n));
      CK(fp64 ? launch_pc<double>(prev, Q, pc_n, wq, out_n, copies, status, false, s)
              : launch_pc<float>(prev, Q, pc_n, wq, out_n, copies, status, false, s));
      int st = 0;
      unsigned long long banked = 0;
      rc = harvest(&st, &banked);
      if (rc != MC_OK) return rc;
      if (comb && st == 0) {
        // the comb sorts the census bank first, so it needs the banked count on the host
        const uint64_t n = banked < cap ? banked : cap;
        const size_t bytes = comb_scratch_bytes(n, nb);
        rc = p->d_comb.ensure(bytes, p->dev);
        if (rc != MC_OK) return rc;
        CK(fp64 ? launch_comb_pc<double>(prev, Q, n, wq, (uint32_t)(i - 1), p->d_comb.ptr, bytes, out_n, copies,
                                         status, s)
                : launch_comb_pc<float>(prev, Q, n, wq, (uint32_t)(i - 1), p->d_comb.ptr, bytes, out_n, copies,
                                        status, s));
      } else if (st == 0) {
        CK(fp64 ? launch_pc<double>(prev, Q, pc_n, wq, out_n, copies, status, true, s)
                : launch_pc<float>(prev, Q, pc_n, wq, out_n, copies, status, true, s));
      }
      unsigned long long pc_state[2] = {0ull, 0ull};  // copies, status word
      CK(cudaMemcpyAsync(pc_state, copies, 16, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      cnt[MC_C_PC_COPIES] += pc_state[0];
      if (st == 0) st = (int)(pc_state[1] & 0xFFFFFFFFu);
      if (st != 0) {
        p->last_status = st;
        return fail(st, "population-control interval %d: device status %d", i - 1, st);
      }
      CK(cudaMemsetAsync(p->d_ctl.ptr, 0, sizeof(Ctl), s));
      CK(cudaMemcpyAsync((char*)p->d_ctl.ptr + offsetof(Ctl, log_n), &log_n, sizeof(log_n), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync((char*)p->d_ctl.ptr + offsetof(Ctl, birth), out_n, 8, cudaMemcpyDeviceToDevice, s));
    }
    CK(fp64 ? launch_transport<double>(Q, grid, block, smem, s, wide, range)
            : launch_transport<float>(Q, grid, block, smem, s, wide, range));
    prev = Q;
  }
  int st = 0;
  unsigned long long banked_last = 0;
  rc = harvest(&st, &banked_last);
  if (rc != MC_OK) return rc;
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  for (int i = 0; i < MC_NCOUNTERS; ++i) c.counters[i] = cnt[i];
  c.iterations = iterations;
  c.log_n = log_n;
  c.status = st;
  CK(cudaMemcpyAsync(p->d_ctl.ptr, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_run(mc_problem* p, uint64_t n_histories, uint64_t seed, const mc_run_opts* opts, void* stream) {
  NvtxRange nvtx_range("mc_run");
  g_err.clear();
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  mc_run_opts o;
  if (opts) o = *opts;
  else mc_run_opts_default(&o);
  if (o.block_size == 0 && o.blocks_per_sm == 0 && p->tuned_block) {
    o.block_size = p->tuned_block;  // the configuration mc_run_tune found for this problem
    o.blocks_per_sm = p->tuned_bps;
    if (o.drain_threshold == 0) o.drain_threshold = p->tuned_drain;
  }
  if (o.algorithm == MC_ALG_AUTO) o.algorithm = p->tuned_alg;  // event-based until tuned
  if (o.precision != MC_FP32 && o.precision != MC_FP64) return fail(MC_ERR_INVALID, "precision");
  if (o.tally_mode != MC_TALLY_FIXED64 && o.tally_mode != MC_TALLY_FP64) return fail(MC_ERR_INVALID, "tally_mode");
  if (o.fixed_bits < 0 || o.fixed_bits > 48) return fail(MC_ERR_INVALID, "fixed_bits outside [0,48]");
  if (o.n_batches < 2 || o.n_batches > 4096) return fail(MC_ERR_INVALID, "n_batches outside [2,4096]");
  if (n_histories < (uint64_t)o.n_batches) return fail(MC_ERR_INVALID, "need at least n_batches histories");
  if (n_histories >= (1ull << 32) || o.first_history + n_histories > (1ull << 32))
    return fail(MC_ERR_INVALID, "history indices must stay below 2^32");
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32))
    return fail(MC_ERR_INVALID, "block_size must be a multiple of 32 in [32,256]");
  if (o.ww_enable && !p->ww_set) return fail(MC_ERR_STATE, "weight windows enabled but no table set");
  if (o.algorithm != MC_ALG_EVENT && o.algorithm != MC_ALG_HISTORY) return fail(MC_ERR_INVALID, "algorithm");
  if (check_implicit_opts(o) != MC_OK) return MC_ERR_INVALID;
  const double t_final = reinterpret_cast<const TableHeader*>(p->blob[1].data())->t_census;
  if (o.pc_method != MC_PC_SPLIT_ROULETTE && o.pc_method != MC_PC_COMB)
    return fail(MC_ERR_INVALID, "pc_method must be MC_PC_SPLIT_ROULETTE or MC_PC_COMB");
  if (o.n_census < 0 || o.n_census > 4096 || (o.n_census > 0 && !o.census_times))
    return fail(MC_ERR_INVALID, "n_census outside [0, 4096] or census_times NULL");
  std::vector<double> census(o.census_times, o.census_times + std::max(0, o.n_census));
  for (int i = 0; i < o.n_census; ++i)
    if (!(census[i] > (i ? census[i - 1] : 0.0)) || !(census[i] < t_final))
      return fail(MC_ERR_INVALID, "census_times must increase, be > 0 and below t_census");
  int dev;
  int rc = current_device(&dev);
  if (rc != MC_OK) return rc;
  if (dev != p->dev) return fail(MC_ERR_STATE, "problem was created on device %d, current is %d", p->dev, dev);
  cudaStream_t s = (cudaStream_t)stream;
  const int fp64 = o.precision == MC_FP64;
  const int lanes = fp64 ? kLanesFP64 : kLanesFP32;
  uint64_t cap = o.bank_capacity;
  if (cap == 0) {
    // in flight a bank is refilled in chunks, so 2^22 suffices; with census times the census bank
    // holds every particle alive at a census and the birth bank all their copies
    const uint64_t limit = o.n_census > 0 ? (1ull << 28) : (1ull << 22);
    cap = 1ull << 16;
    while (cap < 2 * n_histories && cap < limit) cap <<= 1;
  }
  if (cap < 1024) return fail(MC_ERR_INVALID, "bank_capacity must be >= 1024");
  if (cap >= (1ull << 32)) return fail(MC_ERR_INVALID, "bank_capacity must be below 2^32");
  const size_t bank_bytes = (size_t)cap * 16 * lanes;
  rc = p->d_banks.ensure(4 * bank_bytes, p->dev);
  if (rc != MC_OK) return rc;
  const int nb = o.n_batches;
  const uint64_t bins = (uint64_t)p->total_bins;
  // small tallies get up to 16 copies (within a 64 MB budget) to spread same-bin atomics
  uint32_t stripes = o.tally_stripes > 0 ? (uint32_t)o.tally_stripes : 1u;
  const uint64_t row = p->row;  // bins, then the range walk's difference slots
  if (o.tally_stripes <= 0) {
    const double copy_bytes = (double)nb * (double)row * 8.0;
    stripes = (uint32_t)std::max(1.0, std::min(16.0, std::floor(64.0 * 1048576.0 / copy_bytes)));
  }
  if (stripes > 256) return fail(MC_ERR_INVALID, "tally_stripes above 256");
  if ((double)stripes * nb * (double)row >= 4294967296.0)
    return fail(MC_ERR_INVALID, "tally bins x batches x stripes must stay below 2^32");
  rc = p->d_tally.ensure((size_t)stripes * nb * row * 8, p->dev);
  if (rc == MC_OK) rc = p->d_stats.ensure((size_t)3 * bins * 8, p->dev);
  if (rc != MC_OK) return rc;
  uint64_t log_cap = 0;
  if (o.log_count > 0) {
    log_cap = o.log_capacity ? o.log_capacity : 64 * o.log_count;
    rc = p->d_log.ensure(log_cap * sizeof(mc_event), p->dev);
    if (rc != MC_OK) return rc;
  }
  RunParams P;
  std::memset(&P, 0, sizeof(P));
  char* banks = (char*)p->d_banks.ptr;
  for (int side = 0; side < 2; ++side)
    for (int l = 0; l < lanes; ++l) {
      P.S[side][l] = (uint4*)(banks + (size_t)side * bank_bytes + (size_t)l * cap * 16);
      P.B[side][l] = (uint4*)(banks + (size_t)(2 + side) * bank_bytes + (size_t)l * cap * 16);
    }
  P.cap_s = cap;
  P.cap_b = cap;
  P.ctl = (Ctl*)p->d_ctl.ptr;
  P.sticky = (int*)p->d_sticky.ptr;
  fill_run_params(p, o, n_histories, seed, stripes, P);
  P.history_mode = o.algorithm == MC_ALG_HISTORY;
  rc = p->d_trace.ensure((size_t)3 * kTraceCap * 8, p->dev);
  if (rc != MC_OK) return rc;
  P.trace = (unsigned long long*)p->d_trace.ptr;
  P.trace_cap = kTraceCap;
  P.h_first = o.first_history;
  P.spin_limit = 1ull << 22;
  P.log = o.log_count ? (mc_event*)p->d_log.ptr : nullptr;
  P.log_cap = log_cap;
  P.log_first = o.log_first;
  P.log_count = o.log_count;
  CK(cudaMemsetAsync(p->d_ctl.ptr, 0, sizeof(Ctl), s));
  CK(cudaMemsetAsync(p->d_tally.ptr, 0, (size_t)stripes * nb * row * 8, s));
  if (P.log) CK(cudaMemsetAsync(p->d_log.ptr, 0, log_cap * sizeof(mc_event), s));
  // blocks_per_sm == 2 selects the 128-register build of the kernel, any other explicit value the
  // 80-register one (96 registers for a segment build at 128 threads per CTA); 0 takes the
  // 128-register build when a tally is scored by the range walk (that walk needs the registers) and
  // the 80- or 96-register build otherwise
  const bool range = p->range;
  const bool wide = o.blocks_per_sm == 2 || (o.blocks_per_sm == 0 && range);
  // FP32 tracking with plain-walk tallies only: segments are scored apart from their flights
  bool seg = !fp64 && !range && p->n_tally <= 4;
  for (const HostTally& t : p->tallies) seg = seg && t.est == MC_EST_TRACK_LENGTH;
  // default CTA size: 128 threads for the segment build's 96-register budget, else 256
  const int block = o.block_size ? o.block_size : (seg && !wide ? 128 : 256);
  // tables + per-warp flight queues (64 slots) + per-warp tally staging (128 x 12 B, warp-aggregated
  // tally adds only) + per-warp segment regions (64 records of 64 B)
  const size_t smem = P.blob_bytes + (size_t)(block / 32) * (transport_warp_smem(fp64, P.aggregate != 0) +
                                                             (seg ? (size_t)kSegLanes * kSegCap * 16 : 0));
  rc = check_shared_memory(p->dev, smem, "the transport kernel");
  if (rc != MC_OK) return rc;
  int per_sm = 0;
  CK(fp64 ? transport_occupancy<double>(block, smem, &per_sm, wide, range, false)
          : transport_occupancy<float>(block, smem, &per_sm, wide, range, seg));
  if (per_sm < 1) return fail(MC_ERR_CUDA, "transport kernel does not fit on an SM (block %d, smem %zu)", block, smem);
  if (o.blocks_per_sm > 0) per_sm = std::min(per_sm, std::max(1, o.blocks_per_sm * 256 / block));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev));
  const int grid = sms * per_sm;
  P.drain_threshold = o.drain_threshold ? o.drain_threshold : (uint64_t)2 * grid * block;
  P.seg = seg ? 1 : 0;
  if (seg || (range && !fp64)) {
    // split run: the history-style tail flies each warp's secondaries from its own stack of up to
    // 256, carved out of the bank capacity (a bank too small for 32 per warp runs in one launch).
    // Runs with weight windows stay one launch: a stack keeps a lineage on its warp, and lineages
    // that split many times over would hold a few warps busy while the grid waits, where the
    // one-launch tail spreads every generation of copies over all warps.
    const uint64_t nwt = (uint64_t)grid * (uint64_t)(block / 32);
    const uint64_t wcap = std::min<uint64_t>(256, cap / nwt);
    if (o.n_census == 0 && !o.ww_enable && wcap >= 32) {
      rc = p->d_wstack.ensure((size_t)lanes * nwt * wcap * 16, p->dev);
      if (rc != MC_OK) return rc;
      for (int l = 0; l < lanes; ++l) P.WS[l] = (uint4*)p->d_wstack.ptr + (size_t)l * nwt * wcap;
      P.ws_cap = wcap;
    }
  }
  CK(cudaEventRecord(p->ev[0], s));
  p->launches = 0;
  if (o.n_census == 0) {
    CK(fp64 ? launch_transport<double>(P, grid, block, smem, s, wide, range)
            : launch_transport<float>(P, grid, block, smem, s, wide, range));
    // a split run (see launch_transport) is two launches
    const bool split = !fp64 && (seg || range) && P.WS[0] != nullptr;
    p->launches = (split ? 2 : 1) + (p->range ? 1 : 0) + 1;
  } else {
    rc = run_population_controlled(p, P, census, t_final, grid, block, smem, wide, range, fp64, lanes, cap,
                                   o.pc_method == MC_PC_COMB, s);
    if (rc != MC_OK) return rc;
  }
  CK(cudaEventRecord(p->ev[1], s));
  if (p->range)
    CK(launch_reconstruct(P.tally, (const char*)p->d_blob[1].ptr, p->range_rows, row, nb, (int)stripes, P.tally_fp64, s));
  CK(launch_batch_stats(P.tally, P.tally_fp64, bins, row, nb, (int)stripes, n_histories, p->d_stats.ptr, s));
  CK(cudaEventRecord(p->ev[2], s));
  p->has_run = 1;
  p->batched = 0;
  p->n_hist = n_histories;
  p->n_batches = nb;
  p->stream = s;
  p->log_cap = log_cap;
  p->last_status = MC_OK;
  p->tally_fp64 = P.tally_fp64;
  p->stripes = stripes;
  p->fixed_scale = P.fixed_scale;
  return MC_OK;
}

int mc_run_eigen(mc_problem* p, uint64_t n_per_cycle, int n_inactive, int n_active, uint64_t seed,
                 const mc_run_opts* opts, void* stream, double* k_cycle, uint64_t* sites_cycle, double* k_mean,
                 double* k_std_err) {
  NvtxRange nvtx_range("mc_run_eigen");
  g_err.clear();
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  mc_run_opts o;
  if (opts) o = *opts;
  else mc_run_opts_default(&o);
  if (o.block_size == 0 && o.blocks_per_sm == 0 && p->tuned_block) {
    o.block_size = p->tuned_block;
    o.blocks_per_sm = p->tuned_bps;
  }
  if (o.algorithm == MC_ALG_AUTO) o.algorithm = p->tuned_alg;
  const uint64_t N = n_per_cycle;
  const int n_cycles = n_inactive + n_active;
  if (N < 1 || N >= (1ull << 32)) return fail(MC_ERR_INVALID, "n_per_cycle must be in [1, 2^32)");
  if (n_inactive < 0 || n_active < 2 || n_cycles > 65535)
    return fail(MC_ERR_INVALID, "need n_inactive >= 0, n_active >= 2, at most 65535 cycles");
  if (o.precision != MC_FP32 && o.precision != MC_FP64) return fail(MC_ERR_INVALID, "precision");
  if (o.tally_mode != MC_TALLY_FIXED64 && o.tally_mode != MC_TALLY_FP64) return fail(MC_ERR_INVALID, "tally_mode");
  if (o.fixed_bits < 0 || o.fixed_bits > 48) return fail(MC_ERR_INVALID, "fixed_bits outside [0,48]");
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32))
    return fail(MC_ERR_INVALID, "block_size must be a multiple of 32 in [32,256]");
  if (o.algorithm != MC_ALG_EVENT && o.algorithm != MC_ALG_HISTORY) return fail(MC_ERR_INVALID, "algorithm");
  if (o.ww_enable || o.implicit_capture || o.first_history)
    return fail(MC_ERR_INVALID, "k-eigenvalue cycles are analog, without weight windows or a first_history offset");
  const TableHeader* H0 = reinterpret_cast<const TableHeader*>(p->blob[0].data());
  if (H0->has_census) return fail(MC_ERR_INVALID, "k-eigenvalue cycles need a steady-state problem (t_census = inf)");
  if (!(p->nu_max > 0.0)) return fail(MC_ERR_INVALID, "no material has a production cross section");
  int dev;
  int rc = current_device(&dev);
  if (rc != MC_OK) return rc;
  if (dev != p->dev) return fail(MC_ERR_STATE, "problem was created on device %d, current is %d", p->dev, dev);
  cudaStream_t s = (cudaStream_t)stream;
  const int fp64 = o.precision == MC_FP64;
  const int lanes = fp64 ? kLanesFP64 : kLanesFP32;
  const int slanes = fp64 ? kSiteLanesFP64 : kSiteLanesFP32;
  o.n_batches = n_active;  // every active cycle is one statistical batch
  const int nb = n_active;
  uint64_t cap = o.bank_capacity;
  if (cap == 0) {
    cap = 1ull << 16;
    while (cap < 2 * N && cap < (1ull << 22)) cap <<= 1;
  }
  if (cap < 1024) return fail(MC_ERR_INVALID, "bank_capacity must be >= 1024");
  if (cap >= (1ull << 32)) return fail(MC_ERR_INVALID, "bank_capacity must be below 2^32");
  const size_t bank_bytes = (size_t)cap * 16 * lanes;
  rc = p->d_banks.ensure(4 * bank_bytes, p->dev);
  if (rc != MC_OK) return rc;
  const uint64_t bins = (uint64_t)p->total_bins, row = p->row;
  uint32_t stripes = o.tally_stripes > 0 ? (uint32_t)o.tally_stripes : 1u;
  if (o.tally_stripes <= 0) {
    const double copy_bytes = (double)nb * (double)row * 8.0;
    stripes = (uint32_t)std::max(1.0, std::min(16.0, std::floor(64.0 * 1048576.0 / copy_bytes)));
  }
  if ((double)stripes * nb * (double)row >= 4294967296.0)
    return fail(MC_ERR_INVALID, "tally bins x active cycles x stripes must stay below 2^32");
  rc = p->d_tally.ensure((size_t)stripes * nb * row * 8, p->dev);
  if (rc == MC_OK) rc = p->d_stats.ensure((size_t)3 * bins * 8, p->dev);
  if (rc == MC_OK) rc = p->d_counts.ensure((size_t)N * 4, p->dev);
  if (rc == MC_OK) rc = p->d_scan.ensure((size_t)N * 8, p->dev);
  if (rc == MC_OK) rc = p->d_blocksums.ensure((size_t)((N + 1023) / 1024) * 8, p->dev);
  if (rc == MC_OK) rc = p->d_src.ensure((size_t)N * 16 * slanes, p->dev);
  if (rc == MC_OK) rc = p->d_trace.ensure((size_t)3 * kTraceCap * 8, p->dev);
  if (rc != MC_OK) return rc;
  uint64_t log_cap = 0;
  if (o.log_count > 0) {
    log_cap = o.log_capacity ? o.log_capacity : 64 * o.log_count * (uint64_t)n_cycles;
    rc = p->d_log.ensure(log_cap * sizeof(mc_event), p->dev);
    if (rc != MC_OK) return rc;
    CK(cudaMemsetAsync(p->d_log.ptr, 0, log_cap * sizeof(mc_event), s));
  }
  const int block = o.block_size ? o.block_size : 256;
  const size_t smem = p->blob[fp64].size() + (size_t)(block / 32) * transport_warp_smem(fp64, o.aggregate_atomics > 0);
  rc = check_shared_memory(p->dev, smem, "the transport kernel");
  if (rc != MC_OK) return rc;
  const bool range = p->range;
  const bool wide = o.blocks_per_sm == 2 || (o.blocks_per_sm == 0 && range);
  int per_sm = 0;
  CK(fp64 ? transport_occupancy<double>(block, smem, &per_sm, wide, range, false)
          : transport_occupancy<float>(block, smem, &per_sm, wide, range, false));
  if (per_sm < 1) return fail(MC_ERR_CUDA, "transport kernel does not fit on an SM (block %d, smem %zu)", block, smem);
  if (o.blocks_per_sm > 0) per_sm = std::min(per_sm, std::max(1, o.blocks_per_sm * 256 / block));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev));
  const int grid = sms * per_sm;
  CK(cudaMemsetAsync(p->d_tally.ptr, 0, (size_t)stripes * nb * row * 8, s));
  std::vector<double> ks(n_cycles);
  std::vector<unsigned long long> counters(MC_NCOUNTERS, 0ull);
  unsigned long long log_n = 0, iterations = 0;
  double k_prev = 1.0;
  CK(cudaEventRecord(p->ev[0], s));
  for (int c = 0; c < n_cycles; ++c) {
    NvtxRange cycle_range(c < n_inactive ? "inactive cycle" : "active cycle");
    const double nm = std::floor(p->nu_max / k_prev * (1.0 + 1e-9)) + 2.0;
    if (!(nm <= 64.0)) return fail(MC_ERR_INVALID, "cycle %d: k = %g leaves more than 64 sites per history", c, k_prev);
    const uint32_t nmax = (uint32_t)nm;
    rc = p->d_sites.ensure((size_t)N * nmax * 16 * slanes, p->dev);
    if (rc != MC_OK) return rc;
    RunParams P;
    std::memset(&P, 0, sizeof(P));
    char* banks = (char*)p->d_banks.ptr;
    for (int side = 0; side < 2; ++side)
      for (int l = 0; l < lanes; ++l) {
        P.S[side][l] = (uint4*)(banks + (size_t)side * bank_bytes + (size_t)l * cap * 16);
        P.B[side][l] = (uint4*)(banks + (size_t)(2 + side) * bank_bytes + (size_t)l * cap * 16);
      }
    P.cap_s = cap;
    P.cap_b = cap;
    fill_run_params(p, o, N, seed, stripes, P);
    P.history_mode = o.algorithm == MC_ALG_HISTORY;
    P.trace = (unsigned long long*)p->d_trace.ptr;
    P.trace_cap = kTraceCap;
    P.h_first = 0;
    P.spin_limit = 1ull << 22;
    P.log = o.log_count ? (mc_event*)p->d_log.ptr : nullptr;
    P.log_cap = log_cap;
    P.log_first = o.log_first;
    P.log_count = o.log_count;
    // a cycle starts with all its N sources and ends each history at its first production, so the
    // event iterations only pay off for the first generations: drain at 16x the fixed-source default
    // (measured on the 7-group pin cell: 1e6 histories per cycle 4.5 -> 3.6 ms per cycle, results
    // identical; at 1e5 per cycle no change, the longest history sets the time)
    P.drain_threshold = o.drain_threshold ? o.drain_threshold : (uint64_t)32 * grid * block;
    P.eigen = 1;
    P.eigen_score = c >= n_inactive;
    P.cycle = (uint32_t)c;
    P.batch_fixed = c >= n_inactive ? (uint32_t)(c - n_inactive) : 0u;
    P.nmax = nmax;
    P.inv_k = 1.0 / k_prev;
    P.src_site = (const uint4*)p->d_src.ptr;
    P.site_next = (uint4*)p->d_sites.ptr;
    P.count_next = (uint32_t*)p->d_counts.ptr;
    CK(cudaMemsetAsync(p->d_ctl.ptr, 0, sizeof(Ctl), s));
    CK(cudaMemcpyAsync((char*)p->d_ctl.ptr + offsetof(Ctl, log_n), &log_n, sizeof(log_n), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(p->d_counts.ptr, 0, (size_t)N * 4, s));
    CK(fp64 ? launch_transport<double>(P, grid, block, smem, s, wide, range)
            : launch_transport<float>(P, grid, block, smem, s, wide, range));
    CK(launch_scan_sites((const uint32_t*)p->d_counts.ptr, (unsigned long long*)p->d_scan.ptr,
                         (unsigned long long*)p->d_blocksums.ptr, N, s));
    CK(launch_comb((const uint32_t*)p->d_counts.ptr, (const unsigned long long*)p->d_scan.ptr,
                   (const uint4*)p->d_sites.ptr, nmax, N, seed, (uint32_t)(c + 1), (uint4*)p->d_src.ptr, slanes, s));
    Ctl ctl;
    unsigned long long M = 0;
    CK(cudaMemcpyAsync(&ctl, p->d_ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&M, (const char*)p->d_scan.ptr + (N - 1) * 8, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int sticky = 0;
    CK(cudaMemcpy(&sticky, p->d_sticky.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (ctl.status != 0 || sticky != 0) {
      CK(cudaMemset(p->d_sticky.ptr, 0, 16));
      const int st = ctl.status ? ctl.status : sticky;
      p->last_status = st;
      return fail(st == MC_ERR_BANK_FULL || st == MC_ERR_TIMEOUT || st == MC_ERR_LOST || st == MC_ERR_BOUNDS
                      ? st
                      : MC_ERR_CUDA,
                  "cycle %d: device status %d", c, st);
    }
    for (int i = 0; i < MC_NCOUNTERS; ++i) counters[i] += ctl.counters[i];
    iterations += ctl.iterations;
    log_n = ctl.log_n;
    ks[c] = (double)(long long)ctl.k_acc / 4294967296.0 / (double)N;
    if (k_cycle) k_cycle[c] = ks[c];
    if (sites_cycle) sites_cycle[c] = M;
    if (M == 0) return fail(MC_ERR_STATE, "cycle %d banked no fission site", c);
    if (!(ks[c] > 0.0)) return fail(MC_ERR_STATE, "cycle %d: k estimate %g", c, ks[c]);
    k_prev = ks[c];
  }
  CK(cudaEventRecord(p->ev[1], s));
  // the run's counters over all cycles, where mc_counters_get reads them
  {
    Ctl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    for (int i = 0; i < MC_NCOUNTERS; ++i) ctl.counters[i] = counters[i];
    ctl.iterations = iterations;
    ctl.log_n = log_n;
    CK(cudaMemcpyAsync(p->d_ctl.ptr, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  if (p->range)
    CK(launch_reconstruct(p->d_tally.ptr, (const char*)p->d_blob[1].ptr, p->range_rows, row, nb, (int)stripes,
                          o.tally_mode == MC_TALLY_FP64, s));
  CK(launch_batch_stats(p->d_tally.ptr, o.tally_mode == MC_TALLY_FP64, bins, row, nb, (int)stripes, N * (uint64_t)nb,
                        p->d_stats.ptr, s));
  CK(cudaEventRecord(p->ev[2], s));
  double km = 0.0, kv = 0.0;
  for (int c = n_inactive; c < n_cycles; ++c) km += ks[c];
  km /= n_active;
  for (int c = n_inactive; c < n_cycles; ++c) kv += (ks[c] - km) * (ks[c] - km);
  if (k_mean) *k_mean = km;
  if (k_std_err) *k_std_err = std::sqrt(kv / (n_active - 1) / n_active);
  p->has_run = 1;
  p->launches = 0;  // not counted
  p->batched = 0;
  p->n_hist = N * (uint64_t)nb;
  p->n_batches = nb;
  p->stream = s;
  p->log_cap = log_cap;
  p->last_status = MC_OK;
  p->tally_fp64 = o.tally_mode == MC_TALLY_FP64;
  p->stripes = stripes;
  p->fixed_scale = std::ldexp(1.0, o.fixed_bits);
  return MC_OK;
}

int mc_run_tune(mc_problem* p, uint64_t n_histories, uint64_t seed, const mc_run_opts* opts, void* stream,
                mc_run_opts* tuned, double* best_ms) {
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  mc_run_opts o;
  if (opts) o = *opts;
  else mc_run_opts_default(&o);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  int best_block = 0, best_bps = 0, best_alg = MC_ALG_EVENT, rc = MC_OK;
  int ev_block = 0, ev_bps = 0;  // fastest event-based configuration
  float best_t = 0.f, ev_t = 0.f;
  const int cands[4][2] = {{256, 0}, {256, 2}, {128, 0}, {128, 2}};  // 80- / 128-register builds
  p->tuned_block = 0;
  p->tuned_drain = 0;
  // MC_ALG_AUTO: both algorithms are candidates (their results are identical)
  const int n_alg = o.algorithm == MC_ALG_AUTO ? 2 : 1;
  for (int c = 0; c < 4 * n_alg && rc == MC_OK; ++c) {
    mc_run_opts k = o;
    k.algorithm = o.algorithm == MC_ALG_AUTO ? (c < 4 ? MC_ALG_EVENT : MC_ALG_HISTORY) : o.algorithm;
    k.block_size = cands[c % 4][0];
    k.blocks_per_sm = cands[c % 4][1] ? 2 : 3;  // 128-register build at 2 x 256 threads per SM, else 80 at 3
    if (o.precision == MC_FP64 && cands[c % 4][1] == 0) continue;  // FP64 tracking has one build
    rc = mc_run(p, n_histories, seed, &k, stream);  // warm-up
    float t = -1.f;
    for (int rep = 0; rep < 2 && rc == MC_OK; ++rep) {
      ce = cudaEventRecord(e0, s);
      if (ce == cudaSuccess) rc = mc_run(p, n_histories, seed, &k, stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess && rc == MC_OK) rc = cuda_fail(ce, "timing a candidate");
      if (t < 0.f || ms < t) t = ms;
    }
    if (rc == MC_OK) rc = mc_wait(p);  // a candidate that failed on the device fails the tuning
    if (rc == MC_OK && (best_block == 0 || t < best_t)) {
      best_block = k.block_size;
      best_bps = k.blocks_per_sm;
      best_alg = k.algorithm;
      best_t = t;
    }
    if (rc == MC_OK && k.algorithm == MC_ALG_EVENT && (ev_block == 0 || t < ev_t)) {
      ev_block = k.block_size;
      ev_bps = k.blocks_per_sm;
      ev_t = t;
    }
  }
  // Event mode: when the run turns history-style (the drain threshold) is a candidate too, at the
  // fastest event-based configuration.  Turning early saves grid barriers and bank round trips where
  // histories are short and alike, and costs where they are long and uneven (lattices with
  // production, a supercritical medium), so 16x and 64x the default (twice the resident threads) are
  // timed; the result may beat the history-based candidates too.
  uint64_t best_drain = 0;
  int sms = 0;
  if (rc == MC_OK && ev_block != 0 && o.drain_threshold == 0) {
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaDeviceGetAttribute");
  }
  for (int mult : {16, 64}) {
    if (rc != MC_OK || sms == 0) break;
    mc_run_opts k = o;
    k.algorithm = MC_ALG_EVENT;
    k.block_size = ev_block;
    k.blocks_per_sm = ev_bps;
    k.drain_threshold = (uint64_t)mult * 2ull * (uint64_t)sms * (uint64_t)ev_bps * 256ull;
    rc = mc_run(p, n_histories, seed, &k, stream);  // warm-up
    float t = -1.f;
    for (int rep = 0; rep < 2 && rc == MC_OK; ++rep) {
      ce = cudaEventRecord(e0, s);
      if (ce == cudaSuccess) rc = mc_run(p, n_histories, seed, &k, stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess && rc == MC_OK) rc = cuda_fail(ce, "timing a candidate");
      if (t < 0.f || ms < t) t = ms;
    }
    if (rc == MC_OK) rc = mc_wait(p);
    if (rc == MC_OK && t < best_t) {
      best_block = ev_block;
      best_bps = ev_bps;
      best_alg = MC_ALG_EVENT;
      best_drain = k.drain_threshold;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MC_OK) return rc;
  p->tuned_block = best_block;
  p->tuned_bps = best_bps;
  p->tuned_alg = best_alg;
  p->tuned_drain = best_drain;
  if (tuned) {
    *tuned = o;
    tuned->block_size = best_block;
    tuned->blocks_per_sm = best_bps;
    tuned->algorithm = best_alg;
    tuned->drain_threshold = best_drain;
  }
  if (best_ms) *best_ms = best_t;
  return MC_OK;
}

int mc_wait(mc_problem* p) {
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  if (!p->has_run) return fail(MC_ERR_STATE, "no run yet");
  CK(cudaStreamSynchronize(p->stream));
  int status = 0;
  CK(cudaMemcpy(&status, p->d_sticky.ptr, sizeof(int), cudaMemcpyDeviceToHost));
  if (status != 0) CK(cudaMemset(p->d_sticky.ptr, 0, sizeof(int)));
  if (status == 0) status = p->last_status;  // an error already reported stays the run's status
  p->last_status = status;
  if (status == MC_ERR_BANK_FULL) return fail(status, "particle bank overflowed; raise bank_capacity");
  if (status == MC_ERR_TIMEOUT) return fail(status, "device watchdog expired (iteration or barrier budget)");
  if (status == MC_ERR_LOST) return fail(status, "particles left the geometry");
  if (status == MC_ERR_BOUNDS) return fail(status, "an index was out of range (bounds-checked build)");
  if (status != 0) return fail(MC_ERR_CUDA, "device status %d", status);
  return MC_OK;
}

int mc_tally_shape(const mc_problem* p, int tally_id, int64_t shape[5]) {
  if (!p || !shape) return fail(MC_ERR_INVALID, "NULL argument");
  if (tally_id < 0 || tally_id > p->n_tally) return fail(MC_ERR_INVALID, "tally_id %d outside [0,%d]", tally_id, p->n_tally);
  if (tally_id == p->n_tally) {
    shape[0] = 1;
    shape[1] = 1;
    shape[2] = p->n_surf;
    shape[3] = 1;
    shape[4] = 1;
    return MC_OK;
  }
  const HostTally& T = p->tallies[tally_id];
  shape[0] = T.n[2];
  shape[1] = T.n[1];
  shape[2] = T.n[0];
  shape[3] = p->G;
  shape[4] = T.nval;
  return MC_OK;
}

int mc_tally_sums(mc_problem* p, int tally_id, int64_t* sums, size_t n, int* fixed_bits) {
  int64_t shp[5];
  int rc = mc_tally_shape(p, tally_id, shp);
  if (rc != MC_OK) return rc;
  rc = mc_wait(p);
  if (rc != MC_OK) return rc;
  if (p->tally_fp64) return fail(MC_ERR_STATE, "the last run kept FP64 tallies, which have no exact sums");
  const size_t nbins = (size_t)(shp[0] * shp[1] * shp[2] * shp[3] * shp[4]);
  if (!sums || n < nbins) return fail(MC_ERR_INVALID, "output holds %zu of %zu bins", sums ? n : 0, nbins);
  const TableHeader* H = reinterpret_cast<const TableHeader*>(p->blob[0].data());
  const size_t first = tally_id == p->n_tally ? (size_t)H->leak_offset : (size_t)H->tally[tally_id].bin_offset;
  // the batch statistics start with the exact integer sum over batches (and stripes) of every bin
  CK(cudaMemcpy(sums, (const char*)p->d_stats.ptr + 8 * first, nbins * 8, cudaMemcpyDeviceToHost));
  if (fixed_bits) *fixed_bits = (int)std::lround(std::log2(p->fixed_scale));
  return MC_OK;
}

int mc_tally_get(mc_problem* p, int tally_id, double* mean, double* std_err, size_t n) {
  NvtxRange nvtx_range("mc_tally_get");
  int64_t shp[5];
  int rc = mc_tally_shape(p, tally_id, shp);
  if (rc != MC_OK) return rc;
  rc = mc_wait(p);
  if (rc != MC_OK) return rc;
  const size_t nbins = (size_t)(shp[0] * shp[1] * shp[2] * shp[3] * shp[4]);
  if (n < nbins) return fail(MC_ERR_INVALID, "output holds %zu of %zu bins", n, nbins);
  const TableHeader* H = reinterpret_cast<const TableHeader*>(p->blob[0].data());
  const size_t first = tally_id == p->n_tally ? (size_t)H->leak_offset : (size_t)H->tally[tally_id].bin_offset;
  const size_t bins = (size_t)p->total_bins;
  const double B = (double)p->n_batches;
  const double N = (double)p->n_hist;
  const double nbar = N / B;  // mean batch size
  const char* st = (const char*)p->d_stats.ptr;
  std::vector<double> mv(nbins), sv(nbins);
  if (p->tally_fp64) {
    std::vector<double> tot(nbins), s1(nbins), s2(nbins);
    CK(cudaMemcpy(tot.data(), st + 8 * first, nbins * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s1.data(), st + 8 * (bins + first), nbins * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s2.data(), st + 8 * (2 * bins + first), nbins * 8, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < nbins; ++i) {
      mv[i] = tot[i] / N;
      sv[i] = (s2[i] - s1[i] * s1[i] / B) / (B * (B - 1.0));
    }
  } else {
    std::vector<long long> sum(nbins);
    std::vector<unsigned long long> lo(nbins), hi(nbins);
    CK(cudaMemcpy(sum.data(), st + 8 * first, nbins * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(lo.data(), st + 8 * (bins + first), nbins * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hi.data(), st + 8 * (2 * bins + first), nbins * 8, cudaMemcpyDeviceToHost));
    const double q = 1.0 / p->fixed_scale;
    for (size_t i = 0; i < nbins; ++i) {
      // batch means m_b = T_b q / nbar: S1 = sum m_b, S2 = sum m_b^2 (exact integer sums scaled once)
      const double s1 = (double)sum[i] * q / nbar;
      const double sq = ((double)hi[i] * 18446744073709551616.0 + (double)lo[i]) * q * q;
      const double s2 = sq / (nbar * nbar);
      mv[i] = (double)sum[i] * q / N;
      sv[i] = (s2 - s1 * s1 / B) / (B * (B - 1.0));
    }
  }
  const char* blob64 = reinterpret_cast<const char*>(p->blob[1].data());
  for (size_t i = 0; i < nbins; ++i) {
    const double f = bin_value_factor(blob64, first + i);
    if (mean) mean[i] = mv[i] * f;
    if (std_err) std_err[i] = (sv[i] > 0.0 ? std::sqrt(sv[i]) : 0.0) * f;
  }
  return MC_OK;
}

int mc_tally_batches(mc_problem* p, int tally_id, double* out, size_t n, int* n_batches) {
  int64_t shp[5];
  int rc = mc_tally_shape(p, tally_id, shp);
  if (rc != MC_OK) return rc;
  rc = mc_wait(p);
  if (rc != MC_OK) return rc;
  const size_t nbins = (size_t)(shp[0] * shp[1] * shp[2] * shp[3] * shp[4]);
  const int nb = p->n_batches;
  if (n_batches) *n_batches = nb;
  if (!out) return MC_OK;
  if (n < nbins * (size_t)nb) return fail(MC_ERR_INVALID, "output holds %zu of %zu values", n, nbins * (size_t)nb);
  const TableHeader* H = reinterpret_cast<const TableHeader*>(p->blob[0].data());
  const size_t first = tally_id == p->n_tally ? (size_t)H->leak_offset : (size_t)H->tally[tally_id].bin_offset;
  const size_t bins = (size_t)p->total_bins;
  std::vector<int64_t> raw(nbins), part(nbins);
  for (int j = 0; j < nb; ++j) {
    for (uint32_t c = 0; c < p->stripes; ++c) {
      CK(cudaMemcpy(c ? part.data() : raw.data(),
                    (const char*)p->d_tally.ptr + ((size_t)c * nb * p->row + (size_t)j * p->row + first) * 8,
                    nbins * 8, cudaMemcpyDeviceToHost));
      if (c)
        for (size_t i = 0; i < nbins; ++i) {
          if (p->tally_fp64) {
            double a, b;
            std::memcpy(&a, &raw[i], 8);
            std::memcpy(&b, &part[i], 8);
            a += b;
            std::memcpy(&raw[i], &a, 8);
          } else {
            raw[i] += part[i];
          }
        }
    }
    const uint64_t lo = ((uint64_t)j * p->n_hist + nb - 1) / nb, hi = ((uint64_t)(j + 1) * p->n_hist + nb - 1) / nb;
    const double cnt = (double)(hi - lo);
    const char* blob64 = reinterpret_cast<const char*>(p->blob[1].data());
    for (size_t i = 0; i < nbins; ++i) {
      double x;
      if (p->tally_fp64) std::memcpy(&x, &raw[i], 8);
      else x = (double)raw[i] / p->fixed_scale;
      out[(size_t)j * nbins + i] = x / cnt * bin_value_factor(blob64, first + i);
    }
  }
  return MC_OK;
}

int mc_counters_get(mc_problem* p, int64_t* counters, size_t n) {
  if (!p || !counters) return fail(MC_ERR_INVALID, "NULL argument");
  int rc = mc_wait(p);
  if (rc != MC_OK && rc != MC_ERR_BANK_FULL && rc != MC_ERR_TIMEOUT && rc != MC_ERR_LOST && rc != MC_ERR_BOUNDS)
    return rc;
  Ctl c;
  CK(cudaMemcpy(&c, p->d_ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < n && i < (size_t)MC_NCOUNTERS; ++i)
    counters[i] = i == MC_C_ITERATIONS ? (int64_t)c.iterations : (int64_t)c.counters[i];
  return MC_OK;
}

int mc_event_log(mc_problem* p, mc_event* out, size_t cap, size_t* n_out) {
  if (!p || !n_out) return fail(MC_ERR_INVALID, "NULL argument");
  if (!p->has_run) return fail(MC_ERR_STATE, "no run yet");
  // the log is most useful after a failed run, so it is copied whatever the run's status
  CK(cudaStreamSynchronize(p->stream));
  unsigned long long n = 0;
  CK(cudaMemcpy(&n, (char*)p->d_ctl.ptr + offsetof(Ctl, log_n), sizeof(n), cudaMemcpyDeviceToHost));
  size_t m = (size_t)std::min<unsigned long long>(n, p->log_cap);
  if (m > cap) m = cap;
  if (m && out) CK(cudaMemcpy(out, p->d_log.ptr, m * sizeof(mc_event), cudaMemcpyDeviceToHost));
  *n_out = m;
  if (n > p->log_cap) return fail(MC_ERR_BANK_FULL, "event log overflowed (%llu records)", n);
  return MC_OK;
}

int mc_ww_set_table_t(mc_problem* p, int nx, int ny, int nz, int nt, const double* edges, const double* centre) {
  g_err.clear();
  if (!p || !edges || !centre) return fail(MC_ERR_INVALID, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || nt < 1 || (int64_t)nx * ny * nz * nt > (1 << 24))
    return fail(MC_ERR_INVALID, "weight-window mesh size");
  const int n[4] = {nx, ny, nz, nt};
  const double* e = edges;
  for (int d = 0; d < 4; ++d) {
    for (int i = 0; i <= n[d]; ++i)
      if (std::isnan(e[i]) || (i > 0 && !(e[i] > e[i - 1])))
        return fail(MC_ERR_INVALID, "weight-window edges must increase");
    e += n[d] + 1;
  }
  const size_t cells = (size_t)nx * ny * nz * nt * p->G;
  for (size_t i = 0; i < cells; ++i)
    if (!(centre[i] >= 0.0) || !std::isfinite(centre[i]))
      return fail(MC_ERR_INVALID, "weight-window centres must be finite and >= 0 (0 disables a cell)");
  const size_t n_edges = (size_t)(nx + 1) + (ny + 1) + (nz + 1) + (nt + 1);
  if (p->has_run) CK(cudaStreamSynchronize(p->stream));
  int rc = p->d_ww.ensure((n_edges + cells) * sizeof(double), p->dev);
  if (rc != MC_OK) return rc;
  CK(cudaMemcpy(p->d_ww.ptr, edges, n_edges * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy((double*)p->d_ww.ptr + n_edges, centre, cells * sizeof(double), cudaMemcpyHostToDevice));
  for (int d = 0; d < 4; ++d) p->ww_n[d] = n[d];
  p->ww_set = 1;
  return MC_OK;
}

int mc_ww_set_table(mc_problem* p, int nx, int ny, int nz, const double* edges, const double* centre) {
  g_err.clear();
  if (!p || !edges || !centre) return fail(MC_ERR_INVALID, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz > (1 << 24))
    return fail(MC_ERR_INVALID, "weight-window mesh size");
  // one time bin holding every time: [0, +inf)
  std::vector<double> e(edges, edges + (nx + 1) + (ny + 1) + (nz + 1));
  e.push_back(0.0);
  e.push_back(std::numeric_limits<double>::infinity());
  return mc_ww_set_table_t(p, nx, ny, nz, 1, e.data(), centre);
}

size_t mc_problem_table_bytes(const mc_problem* p) {
  return p ? p->blob[0].size() + p->blob[1].size() : 0;
}

int mc_trace_get(mc_problem* p, uint64_t* t_ns, uint64_t* items, uint64_t* sources, size_t cap,
                 size_t* n_out) {
  if (!p || !n_out) return fail(MC_ERR_INVALID, "NULL argument");
  if (!p->has_run) return fail(MC_ERR_STATE, "no run yet");
  CK(cudaStreamSynchronize(p->stream));
  Ctl c;
  CK(cudaMemcpy(&c, p->d_ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost));
  size_t n = (size_t)std::min<unsigned long long>(c.iterations, kTraceCap);
  if (n > cap) n = cap;
  std::vector<unsigned long long> buf(3 * n);
  if (n) CK(cudaMemcpy(buf.data(), p->d_trace.ptr, 3 * n * 8, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < n; ++i) {
    if (t_ns) t_ns[i] = buf[3 * i] - c.t_start;
    if (items) items[i] = buf[3 * i + 1];
    if (sources) sources[i] = buf[3 * i + 2];
  }
  *n_out = n;
  return MC_OK;
}

int mc_run_launches(const mc_problem* p, int* n) {
  if (!p || !n) return fail(MC_ERR_INVALID, "problem or output is NULL");
  if (!p->has_run) return fail(MC_ERR_STATE, "no run yet");
  if (p->batched || p->launches == 0) return fail(MC_ERR_STATE, "the last run's launches are not counted");
  *n = p->launches;
  return MC_OK;
}

int mc_run_timing(mc_problem* p, double* transport_ms, double* stats_ms) {
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  if (!p->has_run) return fail(MC_ERR_STATE, "no run yet");
  if (p->batched) {
    // part of a batched launch: first claimed unit to last finished particle, device clock
    CK(cudaStreamSynchronize(p->stream));
    Ctl c;
    CK(cudaMemcpy(&c, p->d_ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (transport_ms) *transport_ms = c.t_end > c.t_start ? (double)(c.t_end - c.t_start) * 1e-6 : 0.0;
    if (stats_ms) *stats_ms = 0.0;
    return MC_OK;
  }
  CK(cudaEventSynchronize(p->ev[2]));
  float a = 0.f, b = 0.f;
  CK(cudaEventElapsedTime(&a, p->ev[0], p->ev[1]));
  CK(cudaEventElapsedTime(&b, p->ev[1], p->ev[2]));
  if (transport_ms) *transport_ms = a;
  if (stats_ms) *stats_ms = b;
  return MC_OK;
}

int mc_tally_layout(const mc_problem* p, int* stripes, int* n_batches, uint64_t* row) {
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  if (!p->has_run) return fail(MC_ERR_STATE, "no run yet");
  if (stripes) *stripes = (int)p->stripes;
  if (n_batches) *n_batches = p->n_batches;
  if (row) *row = p->row;
  return MC_OK;
}

int mc_atomic_peak(uint64_t span, double* atomics_per_s) {
  g_err.clear();
  if (!atomics_per_s || span < 1 || span > (1ull << 27)) return fail(MC_ERR_INVALID, "span outside [1, 2^27]");
  int dev, sms = 0;
  int rc = current_device(&dev);
  if (rc != MC_OK) return rc;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevBuf buf;
  rc = buf.ensure(span * 8, dev);
  if (rc != MC_OK) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemset(buf.ptr, 0, span * 8);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = sms * 8, iters = 256;
  if (e == cudaSuccess) e = launch_atomic_probe((unsigned long long*)buf.ptr, span, grid, iters, 1u, 0);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r)
    e = launch_atomic_probe((unsigned long long*)buf.ptr, span, grid, iters, 2u + r, 0);
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  buf.release();
  if (e != cudaSuccess) return cuda_fail(e, "atomic probe");
  *atomics_per_s = 3.0 * grid * 256.0 * iters / (ms * 1e-3);
  return MC_OK;
}

int mc_op_rates(double* ops_per_clk_per_sm, int n) {
  g_err.clear();
  if (!ops_per_clk_per_sm || n < 6) return fail(MC_ERR_INVALID, "need room for 6 rates");
  int dev, sms = 0;
  int rc = current_device(&dev);
  if (rc != MC_OK) return rc;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevBuf buf;
  rc = buf.ensure(64, dev);
  if (rc != MC_OK) return rc;
  unsigned long long* sink = (unsigned long long*)buf.ptr;
  unsigned long long* clk = sink + 2;
  const int grid = sms * 8;  // 8 CTAs of 256 threads per SM
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int op = 0; op < 6 && e == cudaSuccess; ++op) {
    // FP64 and the int64 conversion are slow: fewer iterations
    const int iters = (op == 1 || op == 4) ? 512 : 8192;
    e = launch_op_probe(op, grid, iters, sink, clk, 0);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = launch_op_probe(op, grid, iters, sink, clk, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long c[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(c, clk, sizeof(c), cudaMemcpyDeviceToHost);
    // operations / (launch time x SM clock x SMs); the clock is block 0's ticks per nanosecond
    const double ops = (double)grid * 256.0 * 4.0 * iters;
    const double ghz = c[1] > 0 ? (double)c[0] / (double)c[1] : 0.0;
    if (e == cudaSuccess) ops_per_clk_per_sm[op] = (ms > 0.f && ghz > 0.0) ? ops / (ms * 1e6 * ghz * sms) : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  buf.release();
  if (e != cudaSuccess) return cuda_fail(e, "instruction probe");
  return MC_OK;
}

int mc_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, uint64_t n, void* stream) {
  g_err.clear();
  if (n == 0) return MC_OK;
  if (!ctr || !out) return fail(MC_ERR_INVALID, "NULL device pointer");
  if (((uintptr_t)ctr | (uintptr_t)out) & 15) return fail(MC_ERR_INVALID, "arrays must be 16-byte aligned");
  CK(launch_philox(seed, (const uint4*)ctr, (uint4*)out, n, (cudaStream_t)stream));
  return MC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------ static scratch
// Run entry point for callers that cannot allocate device memory (see mc_run_static in mc.h).
// All of its scratch lives in this file-scope array, which the CUDA runtime reserves on every
// device that loads this module and keeps until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[MC_STATIC_SCRATCH_BYTES];

namespace {
constexpr uint64_t kStaticBank = 32768;  // particles in flight per bank
std::mutex g_static_mu;
void* g_static_ptr[64] = {nullptr};

// Device address of g_static_scratch on `dev` (current): looked up once per device.  The host-side
// name of the array is only a stand-in, never a device address.
int static_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return fail(MC_ERR_STATE, "device %d outside the supported range", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = ptr;
  }
  *out = (unsigned char*)g_static_ptr[dev];
  return MC_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Per-bin mean and standard error from the batch statistics, or NaN everywhere if the run failed.
__global__ void k_static_finalize(const Ctl* ctl, const void* stats, int fp64, uint64_t bins, double n_hist,
                                  double nb, double inv_scale, const char* blob64, double* mean, double* std_err) {
  const bool bad = ctl->status != 0;
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const double nbar = n_hist / nb;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins;
       b += (uint64_t)gridDim.x * blockDim.x) {
    double m, var;
    if (fp64) {
      const double* st = reinterpret_cast<const double*>(stats);
      m = st[b] / n_hist;
      var = (st[2 * bins + b] - st[bins + b] * st[bins + b] / nb) / (nb * (nb - 1.0));
    } else {
      const long long* sum = reinterpret_cast<const long long*>(stats);
      const unsigned long long* lo = reinterpret_cast<const unsigned long long*>(sum + bins);
      const unsigned long long* hi = lo + bins;
      const double s1 = (double)sum[b] * inv_scale / nbar;
      const double sq = ((double)hi[b] * 18446744073709551616.0 + (double)lo[b]) * inv_scale * inv_scale;
      m = (double)sum[b] * inv_scale / n_hist;
      var = (sq / (nbar * nbar) - s1 * s1 / nb) / (nb * (nb - 1.0));
    }
    const double f = bin_value_factor(blob64, b);  // v_g for time-crossing bins
    mean[b] = bad ? nan : m * f;
    std_err[b] = bad ? nan : (var > 0.0 ? sqrt(var) : 0.0) * f;
  }
}
}  // namespace

extern "C" int mc_run_static(const mc_problem* p, uint64_t n_histories, uint64_t seed, const mc_run_opts* opts,
                             double* mean, double* std_err, void* stream) {
  g_err.clear();
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  if (!mean || !std_err) return fail(MC_ERR_INVALID, "mean and std_err must be device arrays");
  mc_run_opts o;
  if (opts) o = *opts;
  else mc_run_opts_default(&o);
  if (o.precision != MC_FP32 && o.precision != MC_FP64) return fail(MC_ERR_INVALID, "precision");
  if (o.tally_mode != MC_TALLY_FIXED64 && o.tally_mode != MC_TALLY_FP64) return fail(MC_ERR_INVALID, "tally_mode");
  if (o.fixed_bits < 0 || o.fixed_bits > 48) return fail(MC_ERR_INVALID, "fixed_bits outside [0,48]");
  if (o.n_batches < 2 || o.n_batches > 4096) return fail(MC_ERR_INVALID, "n_batches outside [2,4096]");
  if (n_histories < (uint64_t)o.n_batches) return fail(MC_ERR_INVALID, "need at least n_batches histories");
  if (n_histories >= (1ull << 32) || o.first_history + n_histories > (1ull << 32))
    return fail(MC_ERR_INVALID, "history indices must stay below 2^32");
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32))
    return fail(MC_ERR_INVALID, "block_size must be a multiple of 32 in [32,256]");
  if (o.algorithm == MC_ALG_AUTO) o.algorithm = p->tuned_alg;
  if (o.algorithm != MC_ALG_EVENT && o.algorithm != MC_ALG_HISTORY) return fail(MC_ERR_INVALID, "algorithm");
  if (check_implicit_opts(o) != MC_OK) return MC_ERR_INVALID;
  if (o.log_count > 0) return fail(MC_ERR_INVALID, "mc_run_static keeps no event log");
  if (o.n_census > 0) return fail(MC_ERR_INVALID, "mc_run_static runs no population control");
  if (o.ww_enable && !p->ww_set) return fail(MC_ERR_STATE, "weight windows enabled but no table set");
  if (o.bank_capacity > kStaticBank)
    return fail(MC_ERR_INVALID, "bank_capacity %llu exceeds the static limit of %llu particles",
                (unsigned long long)o.bank_capacity, (unsigned long long)kStaticBank);
  if (o.bank_capacity > 0 && o.bank_capacity < 1024) return fail(MC_ERR_INVALID, "bank_capacity must be >= 1024");
  if (o.tally_stripes > 1) return fail(MC_ERR_INVALID, "mc_run_static keeps a single tally copy");
  int dev;
  int rc = current_device(&dev);
  if (rc != MC_OK) return rc;
  if (dev != p->dev) return fail(MC_ERR_STATE, "problem was created on device %d, current is %d", p->dev, dev);
  // the outputs must be 8-byte aligned device memory of this device (a runtime query, no allocation)
  if (((uintptr_t)mean | (uintptr_t)std_err) & 7u) return fail(MC_ERR_INVALID, "mean and std_err must be 8-byte aligned");
  for (const double* q : {mean, std_err}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
      cudaGetLastError();
      return fail(MC_ERR_INVALID, "mean and std_err must be device arrays");
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
      return fail(MC_ERR_INVALID, "mean and std_err must be device arrays of device %d", dev);
  }
  const int fp64 = o.precision == MC_FP64;
  const int lanes = fp64 ? kLanesFP64 : kLanesFP32;
  const uint64_t cap = kStaticBank;
  const int nb = o.n_batches;
  const uint64_t bins = (uint64_t)p->total_bins;
  // layout: [control block][sticky word][4 particle banks][batch tallies][batch statistics]
  const size_t off_sticky = align256(sizeof(Ctl));
  const size_t off_banks = off_sticky + 256;
  const size_t bank_bytes = (size_t)cap * 16 * lanes;
  const size_t off_tally = align256(off_banks + 4 * bank_bytes);
  const size_t tally_bytes = (size_t)nb * p->row * 8;
  const size_t off_stats = align256(off_tally + tally_bytes);
  const size_t need = off_stats + (size_t)3 * bins * 8;
  if (need > (size_t)MC_STATIC_SCRATCH_BYTES)
    return fail(MC_ERR_INVALID,
                "%d batches x %llu bins need %zu bytes of scratch; the static scratch holds %zu (use mc_run)", nb,
                (unsigned long long)p->row, need, (size_t)MC_STATIC_SCRATCH_BYTES);
  unsigned char* base = nullptr;
  rc = static_scratch(dev, &base);
  if (rc != MC_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  RunParams P;
  std::memset(&P, 0, sizeof(P));
  // the parameters mc_run sets, then the addresses in the static array and the settings of this call
  fill_run_params(p, o, n_histories, seed, 1, P);
  for (int side = 0; side < 2; ++side)
    for (int l = 0; l < lanes; ++l) {
      P.S[side][l] = (uint4*)(base + off_banks + (size_t)side * bank_bytes + (size_t)l * cap * 16);
      P.B[side][l] = (uint4*)(base + off_banks + (size_t)(2 + side) * bank_bytes + (size_t)l * cap * 16);
    }
  P.cap_s = cap;
  P.cap_b = cap;
  P.ctl = (Ctl*)base;
  P.sticky = (int*)(base + off_sticky);
  P.tally = base + off_tally;
  P.history_mode = o.algorithm == MC_ALG_HISTORY;
  P.trace = nullptr;
  P.trace_cap = 0;
  P.h_first = o.first_history;
  P.spin_limit = 1ull << 22;
  // the array keeps the previous call's contents: clear what must start at zero
  CK(cudaMemsetAsync(base, 0, off_banks, s));
  CK(cudaMemsetAsync(base + off_tally, 0, tally_bytes, s));
  const int block = o.block_size ? o.block_size : 256;
  const size_t smem = P.blob_bytes + (size_t)(block / 32) * transport_warp_smem(fp64, P.aggregate != 0);
  rc = check_shared_memory(p->dev, smem, "the transport kernel");
  if (rc != MC_OK) return rc;
  int per_sm = 0;
  const bool range = p->range;
  const bool wide = o.blocks_per_sm == 2 || (o.blocks_per_sm == 0 && range);
  CK(fp64 ? transport_occupancy<double>(block, smem, &per_sm, wide, range, false)
          : transport_occupancy<float>(block, smem, &per_sm, wide, range, false));
  if (per_sm < 1) return fail(MC_ERR_CUDA, "transport kernel does not fit on an SM (block %d, smem %zu)", block, smem);
  if (o.blocks_per_sm > 0) per_sm = std::min(per_sm, std::max(1, o.blocks_per_sm * 256 / block));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * per_sm;
  P.drain_threshold = o.drain_threshold ? o.drain_threshold : (uint64_t)2 * grid * block;
  CK(fp64 ? launch_transport<double>(P, grid, block, smem, s, wide, range)
          : launch_transport<float>(P, grid, block, smem, s, wide, range));
  if (p->range)
    CK(launch_reconstruct(P.tally, (const char*)p->d_blob[1].ptr, p->range_rows, p->row, nb, 1, P.tally_fp64, s));
  CK(launch_batch_stats(P.tally, P.tally_fp64, bins, p->row, nb, 1, n_histories, base + off_stats, s));
  unsigned g = (unsigned)std::min<uint64_t>((bins + 255) / 256, 1024);
  k_static_finalize<<<g ? g : 1, 256, 0, s>>>((const Ctl*)base, base + off_stats, P.tally_fp64, bins,
                                              (double)n_histories, (double)nb, 1.0 / P.fixed_scale,
                                              (const char*)p->d_blob[1].ptr, mean, std_err);
  CK(cudaGetLastError());
  return MC_OK;
}

// ------------------------------------------------------------------------------------------ importance network
namespace mcgb {
size_t mlp_param_count();
size_t mlp_weights_bytes();
cudaError_t mlp_refresh(const float* master, void* Wg, cudaStream_t s);
cudaError_t mlp_forward(const void* Wg, const float* x, float* y, int n, cudaStream_t s);
cudaError_t mlp_loss_grad(const void* Wg, const float* x, const float* tgt, const float* wt, int n, float* grad,
                          float* loss, cudaStream_t s);
size_t mlp_train_scratch_bytes();
cudaError_t mlp_train(float* master, float* m1, float* m2, void* Wg, const float* x, const float* tgt, const float* wt,
                      int n, int epochs, float lr, long long step0, float* last_loss, void* scratch, cudaStream_t s);
cudaError_t mlp_centres(const float* y, int n, double scale, double ymin, double ymax, double ref, double* centre,
                        cudaStream_t s);
}  // namespace mcgb

struct mc_mlp {
  int dev = 0;
  DevBuf master, m1, m2, wg, data, aux;
  DevBuf train;  // the trainer's epoch gradients and grid barrier
  long long steps = 0;
};

extern "C" {

int mc_mlp_param_count(void) { return (int)mlp_param_count(); }

int mc_mlp_create(mc_mlp** out) {
  g_err.clear();
  if (!out) return fail(MC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  mc_mlp* m = new mc_mlp();
  int rc = current_device(&m->dev);
  const size_t np = mlp_param_count();
  if (rc == MC_OK) rc = m->master.ensure(np * 4, m->dev);
  if (rc == MC_OK) rc = m->m1.ensure(np * 4, m->dev);
  if (rc == MC_OK) rc = m->m2.ensure(np * 4, m->dev);
  if (rc == MC_OK) rc = m->wg.ensure(mlp_weights_bytes(), m->dev);
  if (rc == MC_OK) rc = m->train.ensure(mlp_train_scratch_bytes(), m->dev);
  if (rc == MC_OK) {
    cudaError_t e = cudaMemset(m->master.ptr, 0, np * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m1.ptr, 0, np * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m2.ptr, 0, np * 4);
    if (e == cudaSuccess) e = cudaMemset(m->wg.ptr, 0, mlp_weights_bytes());
    if (e == cudaSuccess) e = mlp_refresh((const float*)m->master.ptr, m->wg.ptr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "mc_mlp_create");
  }
  if (rc != MC_OK) {
    mc_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return MC_OK;
}

void mc_mlp_destroy(mc_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  m->master.release();
  m->m1.release();
  m->m2.release();
  m->wg.release();
  m->data.release();
  m->aux.release();
  m->train.release();
  delete m;
}

int mc_mlp_set_params(mc_mlp* m, const double* params, size_t n) {
  g_err.clear();
  const size_t np = mlp_param_count();
  if (!m || !params || n != np) return fail(MC_ERR_INVALID, "expected %zu parameters", np);
  std::vector<float> f(np);
  for (size_t i = 0; i < np; ++i) {
    if (!std::isfinite(params[i])) return fail(MC_ERR_INVALID, "parameter %zu is not finite", i);
    f[i] = (float)params[i];
  }
  CK(cudaMemcpy(m->master.ptr, f.data(), np * 4, cudaMemcpyHostToDevice));
  CK(cudaMemset(m->m1.ptr, 0, np * 4));
  CK(cudaMemset(m->m2.ptr, 0, np * 4));
  CK(mlp_refresh((const float*)m->master.ptr, m->wg.ptr, 0));
  CK(cudaDeviceSynchronize());
  m->steps = 0;
  return MC_OK;
}

int mc_mlp_get_params(mc_mlp* m, double* params, size_t n) {
  g_err.clear();
  const size_t np = mlp_param_count();
  if (!m || !params || n < np) return fail(MC_ERR_INVALID, "expected room for %zu parameters", np);
  std::vector<float> f(np);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(f.data(), m->master.ptr, np * 4, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < np; ++i) params[i] = f[i];
  return MC_OK;
}

int mc_mlp_forward(mc_mlp* m, const float* x, float* y, int n, void* stream) {
  g_err.clear();
  if (!m || !x || !y || n < 0) return fail(MC_ERR_INVALID, "bad argument");
  if (n == 0) return MC_OK;
  CK(mlp_forward(m->wg.ptr, x, y, n, (cudaStream_t)stream));
  return MC_OK;
}

int mc_mlp_loss_grad(mc_mlp* m, const float* x, const float* target, const float* wt, int n, float* grad,
                     float* loss, void* stream) {
  g_err.clear();
  if (!m || !x || !target || !grad || !loss || n < 1) return fail(MC_ERR_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(grad, 0, mlp_param_count() * 4, s));
  CK(cudaMemsetAsync(loss, 0, 4, s));
  CK(mlp_loss_grad(m->wg.ptr, x, target, wt, n, grad, loss, s));
  return MC_OK;
}

int mc_mlp_train(mc_mlp* m, const float* x, const float* target, const float* wt, int n, int epochs, float lr,
                 float* last_loss, void* stream) {
  g_err.clear();
  if (!m || !x || !target || n < 1 || epochs < 0 || !(lr > 0.f)) return fail(MC_ERR_INVALID, "bad argument");
  CK(mlp_train((float*)m->master.ptr, (float*)m->m1.ptr, (float*)m->m2.ptr, m->wg.ptr, x, target, wt, n, epochs, lr,
               m->steps, last_loss, m->train.ptr, (cudaStream_t)stream));
  m->steps += epochs;
  return MC_OK;
}

}  // extern "C"

namespace {
// scaled coordinate in [-1, 1] of bin i of an edge list (0 on axes without finite extent)
double scaled_centre(const std::vector<double>& e, int i) {
  const int n = (int)e.size() - 1;
  double lo = e[0], hi = e[n];
  if (!std::isfinite(lo)) lo = n > 1 ? e[1] : 0.0;
  if (!std::isfinite(hi)) hi = n > 1 ? e[n - 1] : 0.0;
  if (!(hi > lo)) return 0.0;
  double a = e[i], b = e[i + 1];
  if (!std::isfinite(a)) a = b;
  if (!std::isfinite(b)) b = a;
  const double c = 0.5 * (a + b);
  const double v = 2.0 * (c - lo) / (hi - lo) - 1.0;
  return v < -1.0 ? -1.0 : (v > 1.0 ? 1.0 : v);
}

int bin_of_point(const std::vector<double>& e, double v) {
  const int n = (int)e.size() - 1;
  for (int i = 0; i < n; ++i)
    if (v >= e[i] && v < e[i + 1]) return i;
  return v < e[0] ? 0 : n - 1;
}
}  // namespace

extern "C" int mc_ww_learn(mc_problem* p, mc_mlp* m, int tally_id, int epochs, float lr, double extrap_slope,
                           double extrap_efolds, double info[5]) {
  g_err.clear();
  if (!p || !m) return fail(MC_ERR_INVALID, "NULL argument");
  if (tally_id < 0 || tally_id >= p->n_tally) return fail(MC_ERR_INVALID, "tally_id must name a mesh tally");
  if (!(extrap_slope >= 0.0 && extrap_slope <= 1.0)) return fail(MC_ERR_INVALID, "extrap_slope outside [0,1]");
  if (!(extrap_efolds >= 0.0 && extrap_efolds <= 700.0)) return fail(MC_ERR_INVALID, "extrap_efolds outside [0,700]");
  int64_t shp[5];
  int rc = mc_tally_shape(p, tally_id, shp);
  if (rc != MC_OK) return rc;
  const int nz = (int)shp[0], ny = (int)shp[1], nx = (int)shp[2], G = (int)shp[3], nt = (int)shp[4];
  const size_t nbin = (size_t)nz * ny * nx * G * nt;
  std::vector<double> mean(nbin), err(nbin);
  rc = mc_tally_get(p, tally_id, mean.data(), err.data(), nbin);
  if (rc != MC_OK) return rc;
  const HostTally& T = p->tallies[tally_id];
  // Windows resolved in time when the tally has several time bins: the targets are then the flux
  // of each (cell, group, time bin), so that the windows follow the particle population in time as
  // they follow it in space (about the same number of tracks in every bin); otherwise the flux
  // summed over time.
  const bool timed = nt > 1;
  const int ntw = timed ? nt : 1;
  const size_t ncell = (size_t)nz * ny * nx * G;
  std::vector<double> phi(ncell * ntw, 0.0), var(ncell * ntw, 0.0);
  for (size_t c = 0; c < ncell; ++c)
    for (int it = 0; it < nt; ++it) {
      const size_t k = c * ntw + (timed ? it : 0);
      phi[k] += mean[c * nt + it];
      var[k] += err[c * nt + it] * err[c * nt + it];
    }
  const int rx = bin_of_point(T.e[0], p->src_center[0]), ry = bin_of_point(T.e[1], p->src_center[1]),
            rz = bin_of_point(T.e[2], p->src_center[2]);
  const int rt = timed ? bin_of_point(T.e[3], reinterpret_cast<const TableHeader*>(p->blob[1].data())->src_t0) : 0;
  const double phi_ref = phi[((((size_t)rz * ny + ry) * nx + rx) * G + p->src_group) * ntw + rt];
  if (!(phi_ref > 0.0)) return fail(MC_ERR_STATE, "the source cell of tally %d has no flux yet", tally_id);
  std::vector<float> xs, tg, wt, xall;
  double scale = 1.0;
  // network input: the cell centre scaled to [-1, 1] along x, y, z, the group, and the time bin
  // (its index scaled to [-1, 1], which keeps log-spaced bins evenly apart; 0 without time bins)
  auto point = [&](int ix, int iy, int iz, int g, int iw, float* pt) {
    pt[0] = (float)scaled_centre(T.e[0], ix);
    pt[1] = (float)scaled_centre(T.e[1], iy);
    pt[2] = (float)scaled_centre(T.e[2], iz);
    pt[3] = G > 1 ? (float)(2.0 * g / (G - 1) - 1.0) : 0.f;
    pt[4] = ntw > 1 ? (float)(2.0 * iw / (ntw - 1) - 1.0) : 0.f;
  };
  auto add = [&](const float* pt, double target, double w) {
    xs.insert(xs.end(), pt, pt + 5);
    tg.push_back((float)target);
    wt.push_back((float)w);
    scale = std::max(scale, std::fabs(target));
  };
  int n_extra = 0;
  for (int iw = 0; iw < ntw; ++iw)
    for (int iz = 0; iz < nz; ++iz)
      for (int iy = 0; iy < ny; ++iy) {
        // resolved cells of every group's x line; then one common slope per side: the flattest of
        // the groups' fitted slopes (deep in a medium every group decays at the common asymptotic
        // rate, which no group's near-source rate undercuts)
        std::vector<std::vector<int>> rix(G);
        std::vector<std::vector<double>> rtg(G);
        for (int g = 0; g < G; ++g)
          for (int ix = 0; ix < nx; ++ix) {
            float pt[5];
            point(ix, iy, iz, g, iw, pt);
            xall.insert(xall.end(), pt, pt + 5);
            const size_t c = ((((size_t)iz * ny + iy) * nx + ix) * G + g) * ntw + iw;
            if (!(phi[c] > 0.0)) continue;
            const double rel = std::sqrt(var[c]) / phi[c];
            if (!(rel < 0.5)) continue;
            const double target = std::log(phi[c] / phi_ref);
            add(pt, target, std::min(1.0 / std::max(rel * rel, 1e-12), 1e4));
            rix[g].push_back(ix);
            rtg[g].push_back(target);
          }
        if (!(extrap_slope > 0.0)) continue;
        for (int side = 0; side < 2; ++side) {
          // least-squares line through the k outermost resolved cells of each group on this side
          std::vector<double> fa(G, 0.0), fb(G, 0.0);
          std::vector<char> fit(G, 0);
          double common = 0.0;
          bool any = false;
          for (int g = 0; g < G; ++g) {
            const int nr = (int)rix[g].size();
            if (nr < 3) continue;
            const int k = std::max(3, nr / 4);
            double sx = 0, sy = 0, sxx = 0, sxy = 0;
            bool finite = true;
            for (int j = 0; j < k; ++j) {
              const int q = side ? nr - 1 - j : j;
              const double xc = 0.5 * (T.e[0][rix[g][q]] + T.e[0][rix[g][q] + 1]);
              finite = finite && std::isfinite(xc);
              sx += xc;
              sy += rtg[g][q];
              sxx += xc * xc;
              sxy += xc * rtg[g][q];
            }
            const double den = k * sxx - sx * sx;
            if (!finite || !(den > 0.0) || !std::isfinite(den)) continue;
            const double a = (k * sxy - sx * sy) / den;
            if (side ? !(a < 0.0) : !(a > 0.0)) continue;  // not falling away from the resolved cells
            fa[g] = a;
            fb[g] = (sy - a * sx) / k;
            fit[g] = 1;
            common = any ? (side ? std::max(common, a) : std::min(common, a)) : a;
            any = true;
          }
          if (!any) continue;
          // each group continues from its own outermost resolved cell with extrap_slope times the
          // common slope until the windows have fallen by extrap_efolds, then stays constant
          const double slope = extrap_slope * common;
          for (int g = 0; g < G; ++g) {
            if (!fit[g]) continue;
            const int nr = (int)rix[g].size();
            const int edge = side ? rix[g][nr - 1] : rix[g][0];
            const double xe = 0.5 * (T.e[0][edge] + T.e[0][edge + 1]);
            const double ye = fa[g] * xe + fb[g];
            const int from = side ? edge + 1 : 0, to = side ? nx : edge;
            for (int ix = from; ix < to; ++ix) {
              const double xc = 0.5 * (T.e[0][ix] + T.e[0][ix + 1]);
              if (!std::isfinite(xc)) continue;
              const double drop = std::min(std::fabs(slope * (xc - xe)), extrap_efolds);
              float pt[5];
              point(ix, iy, iz, g, iw, pt);
              add(pt, std::max(ye - drop, -700.0), 4.0);  // the weight of a 50% relative error
              ++n_extra;
            }
          }
        }
      }
  // xall is in [t][z][y][g][x] order here; the window table wants [t][z][y][x][g]
  {
    std::vector<float> re(xall.size());
    for (int iw = 0; iw < ntw; ++iw)
      for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
          for (int g = 0; g < G; ++g)
            for (int ix = 0; ix < nx; ++ix) {
              const size_t line = ((size_t)iw * nz + iz) * ny + iy;
              const size_t from = ((line * G + g) * nx + ix) * 5;
              const size_t to = ((line * nx + ix) * G + g) * 5;
              std::copy(xall.begin() + from, xall.begin() + from + 5, re.begin() + to);
            }
    xall.swap(re);
  }
  const int n = (int)tg.size();
  if (n - n_extra < 2) return fail(MC_ERR_STATE, "tally %d resolves fewer than two bins", tally_id);
  if (n > (1 << 20)) return fail(MC_ERR_INVALID, "too many training points");
  double wsum = 0.0;
  for (float w : wt) wsum += w;
  for (int i = 0; i < n; ++i) {
    tg[i] = (float)(tg[i] / scale);
    wt[i] = (float)(wt[i] * n / wsum);
  }
  const int nall = (int)(xall.size() / 5);
  // device: [x n*5][target n][weight n][loss 1] and [all points nall*5][y nall]
  rc = m->data.ensure(((size_t)n * 7 + 4) * 4, m->dev);
  if (rc == MC_OK) rc = m->aux.ensure((size_t)nall * 6 * 4, m->dev);
  if (rc != MC_OK) return rc;
  float* dx = (float*)m->data.ptr;
  float* dt = dx + (size_t)n * 5;
  float* dw = dt + n;
  float* dl = dw + n;
  float* dall = (float*)m->aux.ptr;
  float* dy = dall + (size_t)nall * 5;
  CK(cudaMemcpy(dx, xs.data(), (size_t)n * 5 * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dt, tg.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dw, wt.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dall, xall.data(), (size_t)nall * 5 * 4, cudaMemcpyHostToDevice));
  CK(mlp_train((float*)m->master.ptr, (float*)m->m1.ptr, (float*)m->m2.ptr, m->wg.ptr, dx, dt, dw, n, epochs, lr,
               m->steps, dl, m->train.ptr, 0));
  m->steps += epochs;
  CK(mlp_forward(m->wg.ptr, dall, dy, nall, 0));
  // the window table lives on the tally's spatial mesh and, when resolved in time, its time bins
  std::vector<double> edges;
  for (int d = 0; d < 3; ++d) edges.insert(edges.end(), T.e[d].begin(), T.e[d].end());
  if (timed) {
    edges.insert(edges.end(), T.e[3].begin(), T.e[3].end());
  } else {
    edges.push_back(0.0);
    edges.push_back(std::numeric_limits<double>::infinity());
  }
  const size_t n_edges = edges.size();
  if (p->has_run) CK(cudaStreamSynchronize(p->stream));
  rc = p->d_ww.ensure((n_edges + (size_t)nall) * sizeof(double), p->dev);
  if (rc != MC_OK) return rc;
  CK(cudaMemcpy(p->d_ww.ptr, edges.data(), n_edges * sizeof(double), cudaMemcpyHostToDevice));
  // window centres relative to the source particle's weight 1 at phi_ref
  CK(mlp_centres(dy, nall, scale, -700.0, 50.0, 1.0, (double*)p->d_ww.ptr + n_edges, 0));
  float loss = 0.f;
  CK(cudaMemcpy(&loss, dl, 4, cudaMemcpyDeviceToHost));
  if (std::isnan(loss)) return fail(MC_ERR_TIMEOUT, "the network's training grid barrier timed out");
  p->ww_n[0] = nx;
  p->ww_n[1] = ny;
  p->ww_n[2] = nz;
  p->ww_n[3] = ntw;
  p->ww_set = 1;
  if (info) {
    info[0] = n - n_extra;
    info[1] = loss;
    info[2] = scale;
    info[3] = phi_ref;
    info[4] = n_extra;
  }
  return MC_OK;
}

// The problem's own network, for callers that do not manage an mc_mlp (see mc.h).
extern "C" int mc_ww_set_mlp(mc_problem* p, const uint16_t* bf16_weights, size_t n) {
  g_err.clear();
  if (!p || !bf16_weights) return fail(MC_ERR_INVALID, "NULL argument");
  if (n != (size_t)mc_mlp_param_count())
    return fail(MC_ERR_INVALID, "expected %d BF16 parameters, got %zu", mc_mlp_param_count(), n);
  std::vector<double> params(n);
  for (size_t i = 0; i < n; ++i) {
    const uint32_t bits = (uint32_t)bf16_weights[i] << 16;  // BF16 is the top half of an FP32
    float f;
    std::memcpy(&f, &bits, sizeof(f));
    if (!std::isfinite(f)) return fail(MC_ERR_INVALID, "parameter %zu is not finite", i);
    params[i] = (double)f;
  }
  if (!p->own_mlp) {
    const int rc = mc_mlp_create(&p->own_mlp);
    if (rc != MC_OK) return rc;
  }
  return mc_mlp_set_params(p->own_mlp, params.data(), n);
}

extern "C" int mc_ww_train(mc_problem* p, int tally_id, int epochs, float lr) {
  g_err.clear();
  if (!p) return fail(MC_ERR_INVALID, "problem is NULL");
  if (!p->own_mlp) return fail(MC_ERR_STATE, "no network: load its weights with mc_ww_set_mlp first");
  return mc_ww_learn(p, p->own_mlp, tally_id, epochs, lr, 0.0, 0.0, nullptr);
}
