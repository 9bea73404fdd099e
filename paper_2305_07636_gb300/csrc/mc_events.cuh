// Device-side steps of the random walk shared by the transport kernels (sm_103a): bounded grid
// barrier, event log, per-CTA counters, birth-bank appends, weight windows, the collision and
// surface events, the two halves of a flight, source sampling and the pending-event handler.
// Included by the single-problem persistent kernel and by the batched kernel.
#pragma once
#include <cuda_runtime.h>

#include "mc_device.cuh"

namespace mcgb {

// ------------------------------------------------------------------------------------------ barrier
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

// records a device error in the run's status word and in the problem's sticky error word
__device__ __forceinline__ void set_status(const RunParams& P, int code) {
  atomicCAS(&P.ctl->status, 0, code);
  atomicCAS(P.sticky, 0, code);
}

// Sense-reversing grid barrier for a cooperative (co-resident) grid.  The spin is bounded by
// `limit` polls; on expiry the block records MC_ERR_TIMEOUT and leaves.  A waiting block also
// leaves as soon as any block has posted an error status, so one failing block cannot leave the
// others spinning; every block then stops at the top of its next iteration.
__device__ inline void grid_barrier(const RunParams& P, Ctl* ctl, unsigned long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(&ctl->bar_gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      unsigned long long polls = 0;
      while (ld_acquire(&ctl->bar_gen) == gen) {
        if (ld_volatile_int(&ctl->status) != 0) break;
        if (++polls > limit) {
          set_status(P, MC_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------ logging
// The event-log write is compiled out of line (the log is off in every timed run, and its code
// would otherwise sit inline at each of the walk's event sites); only the test for an open log
// stays inline.
template <typename R>
__device__ __noinline__ void log_event_write(const RunParams& P, const Tab<R>& T, const Part<R>& p, int kind,
                                             int outcome, int n_child) {
  if ((uint64_t)p.root < P.log_first || (uint64_t)p.root >= P.log_first + P.log_count) return;
  const unsigned long long i = atomicAdd(&P.ctl->log_n, 1ull);
  if (i >= P.log_cap) return;
  mc_event e;
  e.tag = (uint64_t)p.tlo | ((uint64_t)p.thi << 32);
  e.root = p.root;
  e.k = p.k;
  e.kind = kind;
  e.outcome = outcome;
  e.n_child = n_child;
  e.cell = (int)pk_cell(p.pk);
  e.elem = T.h->has_lat ? lat_e(p.elem) : 0;
  e.in_pin = (int)pk_pin(p.pk);
  e.g = (int)pk_g(p.pk);
  e.x = p.x; e.y = p.y; e.z = p.z;
  e.ux = p.ux; e.uy = p.uy; e.uz = p.uz;
  e.t = p.time_d(); e.w = p.w;
  P.log[i] = e;
}

template <typename R>
__device__ __forceinline__ void log_event(const RunParams& P, const Tab<R>& T, const Part<R>& p, int kind,
                                          int outcome, int n_child) {
  if (P.log != nullptr) log_event_write(P, T, p, kind, outcome, n_child);
}

// ------------------------------------------------------------------------------------------ counters
// per-CTA (per-warp in the batched kernel) event counters and the weight-window split limit: with
// a split counter (the persistent kernel: the iteration's count of split copies) hold_at is the
// iteration's budget of copies (half the birth store, less the births that wait to be stored
// again); without one, the fill of the warp's stack above which splits wait (the batched kernel)
struct __align__(16) BlockCounters {
  unsigned int c[MC_NCOUNTERS];
  unsigned long long* split_ctr;
  unsigned long long hold_at;
  // the tail launch of a split run: births go to the warp's own stack first (wn[w]: its fill,
  // which runs past P.ws_cap when the stack overflowed into the birth bank)
  unsigned int local;
  unsigned int wn[8];
};
__device__ __forceinline__ void bump(BlockCounters* bc, int i, unsigned v = 1u) { atomicAdd(&bc->c[i], v); }

// ------------------------------------------------------------------------------------------ births
template <typename R>
__device__ __forceinline__ void append_birth(const RunParams& P, uint4* const* Bout, unsigned long long* counter,
                                             BlockCounters* bc, const Part<R>& c) {
  if (bc->local) {
    const unsigned w = threadIdx.x >> 5;
    const unsigned j = atomicAdd(&bc->wn[w], 1u);
    if (j < P.ws_cap) {
      bank_store(c, P.WS, ((uint64_t)blockIdx.x * (blockDim.x >> 5) + w) * P.ws_cap + j);
      return;
    }
  }
  const unsigned long long i = atomicAdd(counter, 1ull);
  if (i >= P.cap_b) {
    set_status(P, MC_ERR_BANK_FULL);
    return;
  }
  bank_store(c, Bout, i);
}

// Weight-window test after a collision or surface event (split above, roulette below).  Where
// MCGB_WW_OUT_OF_LINE is 1 (the batched kernel's translation unit) it is compiled out of line, so
// that the walk's hot loop carries only the test of P.ww_on: that kernel's warps run different
// problems at different points of the walk, and it is bound by instruction fetch.  The persistent
// kernel keeps it inline (a run with windows splits and roulettes at many of its events).
#ifndef MCGB_WW_OUT_OF_LINE
#define MCGB_WW_OUT_OF_LINE 0
#endif
template <typename R>
__device__ __forceinline__ bool weight_window_body(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                                                   unsigned long long* bcount, BlockCounters* bc) {
  const double* ex = P.ww_edges;
  const double* ey = ex + P.ww_nx + 1;
  const double* ez = ey + P.ww_ny + 1;
  const double* et = ez + P.ww_nz + 1;
  // the window of the cell the particle moves into: a particle on a window-mesh edge (e.g. just
  // after crossing a layer plane that is also a mesh plane) is looked up 1e-9 cm ahead; the time
  // bin is the one holding the particle's time
  const double ah = 1e-9;
  const int ix = bin_search(ex, P.ww_nx, (double)p.x + ah * (double)p.ux),
            iy = bin_search(ey, P.ww_ny, (double)p.y + ah * (double)p.uy),
            iz = bin_search(ez, P.ww_nz, (double)p.z + ah * (double)p.uz),
            it = P.ww_nt > 1 ? bin_search(et, P.ww_nt, p.time_d()) : 0;
  if (ix < 0 || ix >= P.ww_nx || iy < 0 || iy >= P.ww_ny || iz < 0 || iz >= P.ww_nz || it < 0 || it >= P.ww_nt)
    return true;
  const double wc =
      __ldg(P.ww_center + ((((size_t)it * P.ww_nz + iz) * P.ww_ny + iy) * P.ww_nx + ix) * T.G + pk_g(p.pk));
  if (!(wc > 0.0)) return true;
  if (p.w > P.ww_upper * wc) {
    int n = (int)ceil(p.w / wc);
    if (n > P.ww_split_max) n = P.ww_split_max;
    // A split is optional: while it would overfill the split budget the particle keeps its weight
    // (unbiased), so that windows far below the flux cannot overflow the birth store.  In the
    // persistent kernel the n - 1 copies are first counted on the iteration's split counter (one
    // atomic add; an attempt that would pass the budget holds, and since its count is not taken
    // back the counter only errs towards holding), so that particles splitting at the same moment
    // cannot overshoot the budget together; in a warp's private stack the stack's fill is compared
    // with the limit.  (Runs with windows are never split, so no copy goes to a tail launch's
    // stack of secondaries.)
    const unsigned long long need = (unsigned long long)(n - 1);
    if (bc->split_ctr != nullptr) {
      if (atomicAdd(bc->split_ctr, need) + need > bc->hold_at) {
        bump(bc, MC_C_WW_HELD);
        return true;
      }
    } else if (*reinterpret_cast<volatile unsigned long long*>(bcount) >= bc->hold_at) {
      bump(bc, MC_C_WW_HELD);
      return true;
    }
    p.w = p.w / n;
    for (int j = 1; j < n; ++j) {
      Part<R> c = p;
      const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)j, kSplitMark);
      c.tlo = t.x;
      c.thi = t.y;
      c.k = 0;
      c.pk = pk_set_pending(c.pk, PEND_NONE, 0, 1, 0);
      append_birth(P, Bout, bcount, bc, c);
      bump(bc, MC_C_WW_SPLIT);
    }
  } else if (p.w < P.ww_lower * wc) {
    const double u = draw<double>(P.seed, p.tlo, p.thi, p.k, 2).b;
    if (u < p.w / wc) {
      p.w = wc;
    } else {
      bump(bc, MC_C_WW_KILL);
      return false;
    }
  }
  return true;
}

template <typename R>
__device__ __noinline__ bool weight_window_apply(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                                                 unsigned long long* bcount, BlockCounters* bc) {
  return weight_window_body(P, T, p, Bout, bcount, bc);
}

template <typename R>
__device__ bool weight_window(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                              unsigned long long* bcount, BlockCounters* bc) {
  if (!P.ww_on) return true;
  if (MCGB_WW_OUT_OF_LINE) return weight_window_apply(P, T, p, Bout, bcount, bc);
  return weight_window_body(P, T, p, Bout, bcount, bc);
}

// ------------------------------------------------------------------------------------------ events
// Channel of a collision of a particle in material m, group g, from u_channel (the second uniform
// of block 0 of the flight that ends in it).  Analog: drawn over Sigma_t (scatter, production,
// capture).  Implicit capture: drawn over Sigma_s + Sigma_f only; a collision whose non-capture
// probability is 0 captures as in the analog walk.
template <typename R>
__device__ __forceinline__ uint32_t collision_channel(const RunParams& P, const Tab<R>& T, int m, int g, R St, R u) {
  const int i = m * T.G + g;
  const R keep = T.ssf[i];  // Sigma_s + Sigma_f: the part of Sigma_t that is not capture
  R xi = u * St;
  if (P.implicit) xi = keep > R(0) ? u * keep : rinf<R>();
  return xi < T.ss[i] ? CHAN_SCATTER : (xi < keep ? CHAN_PRODUCTION : CHAN_CAPTURE);
}

// k-eigenvalue cycle, a production collision in material m: floor(nu / k + xi) fission sites for
// the next cycle, banked in this history's own slots (so their order does not depend on the
// schedule), groups from chi.  Out of line: fixed-source runs never come here.
template <typename R>
__device__ __noinline__ void bank_fission_sites(const RunParams& P, const Tab<R>& T, const Part<R>& p, int m,
                                                BlockCounters* bc) {
  const int G = T.G;
  const int g = (int)pk_g(p.pk);
  bump(bc, MC_C_PRODUCTION);
  const R u = draw<R>(P.seed, p.tlo, p.thi, p.k, 3).a;
  int n = (int)floor(radd(rmul(T.nu[m * G + g], (R)P.inv_k), u));
  if (n > (int)P.nmax) {
    set_status(P, MC_ERR_BANK_FULL);  // cannot happen: nmax covers nu_max / k + 1
    n = (int)P.nmax;
  }
  for (int j = 0; j < n; ++j) {
    const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)j, kChildMark);
    const Pair2<R> c2 = draw<R>(P.seed, t.x, t.y, kSourceEvent, 2);
    const int cg = sample_cdf(T.chi + m * G, G, c2.b);
    site_store(P.site_next, (uint64_t)p.root * P.nmax + (uint64_t)j, p.x, p.y, p.z, cg);
  }
  P.count_next[p.root] = (uint32_t)n;
  if (n > 0) bump(bc, MC_C_SECONDARY, (unsigned)n);
  log_event(P, T, p, 0, 1, n);
}

// Handles the particle's pending collision at the end of flight k (uses the blocks of event k).
// Its channel was drawn with the flight (a capture ends the particle there and never comes here).
template <typename R>
__device__ bool do_collision(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                             unsigned long long* bcount, BlockCounters* bc) {
  const int G = T.G;
  const int g = (int)pk_g(p.pk);
  const int m = material_of(T, p.pk, p.elem);
  const R St = T.st[m * G + g];
  const R keep = T.ssf[m * G + g];
  const uint32_t chan = pk_chan(p.pk);
  // implicit capture: the surviving weight takes the non-capture probability (Sigma_s + Sigma_f) / Sigma_t
  const double wkeep = (P.implicit && keep > R(0)) ? (double)keep / (double)St : 1.0;
  bump(bc, MC_C_COLLISION);
  if (chan == CHAN_SCATTER) {
    bump(bc, MC_C_SCATTER);
    const Pair2<R> b1 = draw<R>(P.seed, p.tlo, p.thi, p.k, 1);
    const Pair2<R> b2 = draw<R>(P.seed, p.tlo, p.thi, p.k, 2);
    const int ng = sample_cdf(T.scdf + (m * G + g) * G, G, b1.a);
    if (!in_range(P, (uint64_t)ng, (uint64_t)G)) return false;
    log_event(P, T, p, 0, 0, 0);
    p.pk = (p.pk & ~0x1Fu) | (uint32_t)ng;
    iso_dir(R(2) * b1.b - R(1), b2.a, p.ux, p.uy, p.uz);
    if (P.implicit) {
      p.w *= wkeep;
      if (p.w < P.wr_cutoff) {
        // weight cutoff: survive with probability w / w_s at weight w_s (unbiased)
        const R u = draw<R>(P.seed, p.tlo, p.thi, p.k, 3).b;
        if ((double)u < p.w / P.wr_survival) {
          p.w = P.wr_survival;
        } else {
          bump(bc, MC_C_WW_KILL);
          return false;
        }
      }
    }
    return weight_window(P, T, p, Bout, bcount, bc);
  }
  if (chan == CHAN_PRODUCTION && P.eigen) {
    bank_fission_sites(P, T, p, m, bc);
    return false;
  }
  if (chan == CHAN_PRODUCTION) {
    bump(bc, MC_C_PRODUCTION);
    const R u = draw<R>(P.seed, p.tlo, p.thi, p.k, 3).a;
    const int n = (int)floor(T.nu[m * G + g] + u);
    for (int j = 0; j < n; ++j) {
      Part<R> c = p;
      c.w = p.w * wkeep;
      const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)j, kChildMark);
      c.tlo = t.x;
      c.thi = t.y;
      c.k = 0;
      const Pair2<R> c1 = draw<R>(P.seed, t.x, t.y, kSourceEvent, 1);
      const Pair2<R> c2 = draw<R>(P.seed, t.x, t.y, kSourceEvent, 2);
      iso_dir(R(2) * c1.b - R(1), c2.a, c.ux, c.uy, c.uz);
      const int cg = sample_cdf(T.chi + m * G, G, c2.b);
      c.pk = pk_set_pending((c.pk & ~0x1Fu) | (uint32_t)cg, PEND_NONE, 0, 1, 0);
      append_birth(P, Bout, bcount, bc, c);
    }
    if (n > 0) bump(bc, MC_C_SECONDARY, (unsigned)n);
    log_event(P, T, p, 0, 1, n);
    return false;
  }
  bump(bc, MC_C_CAPTURE);
  log_event(P, T, p, 0, 2, 0);
  return false;
}

// Handles the particle's pending surface crossing (type and surface stored in its packed word)
template <typename R>
__device__ bool do_surface(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                           unsigned long long* bcount, BlockCounters* bc, uint64_t batch_base) {
  bump(bc, MC_C_SURFACE);
  const uint32_t hit = pk_hit(p.pk);
  if (hit == HIT_CELL) {
    const int s = (int)pk_surf(p.pk);
    const int bcnd = T.sbc[s];
    if (bcnd == MC_BC_VACUUM) {
      if (!P.eigen || P.eigen_score) Scorer<R>(P, p.w)(batch_base + (uint64_t)(T.h->leak_offset + s), R(1));
      bump(bc, MC_C_LEAK);
      log_event(P, T, p, 1, 2, 0);
      return false;
    }
    if (bcnd == MC_BC_REFLECT) {
      bump(bc, MC_C_REFLECT);
      log_event(P, T, p, 1, 1, 0);
      const int kind = T.skind[s];
      if (kind == MC_SURF_PX) p.ux = -p.ux;
      else if (kind == MC_SURF_PY) p.uy = -p.uy;
      else p.uz = -p.uz;
    } else {
      log_event(P, T, p, 1, 0, 0);
      const int c = (int)pk_cell(p.pk);
      int old_sense = 0;
      for (int i = 0; i < T.nhs[c]; ++i) {
        const int e = T.hs[c * MC_MAX_HALFSPACES + i];
        if ((e & 0xFFFF) == s) old_sense = (e >> 16) ? -1 : 1;
      }
      const int nc = locate_cell(T, p.x, p.y, p.z, s, -old_sense, p.ux, p.uy, p.uz);
      if (nc < 0) {
        bump(bc, MC_C_LOST);
        set_status(P, MC_ERR_LOST);
        return false;
      }
      p.pk = (p.pk & ~(0xFFu << 5)) | ((uint32_t)nc << 5);
      if (T.cmat[nc] < 0) lattice_locate(T, p);
    }
  } else if (hit == HIT_PIN) {
    log_event(P, T, p, 1, 4, 0);
    p.pk ^= (1u << 13);
  } else {
    log_event(P, T, p, 1, 3, 0);
    // a lattice wall: the next element along the wall's axis (strides 1, nx, nx ny)
    const uint32_t axis = pk_surf(p.pk);
    const int stride = axis == 0 ? 1 : (axis == 1 ? T.h->lat_nx : T.h->lat_nx * T.h->lat_ny);
    const uint32_t e = (uint32_t)((int)lat_e(p.elem) + pk_dir(p.pk) * stride);
    if (!in_range(P, e, (uint64_t)T.h->lat_nx * T.h->lat_ny * T.h->lat_nz)) return false;
    p.elem = lat_pack(p.elem, e);
    const LatIdx L = lat_split(T, e);
    p.pk = (p.pk & ~(1u << 13)) | (pin_inside(T, p.x, p.y, L.ix, L.iy, e) << 13);
  }
  return weight_window(P, T, p, Bout, bcount, bc);
}

// Flight k, first half: distance to collision, to the nearest surface and to census; chooses the
// event and the flight length l.  Returns false if no event is reachable (the particle is lost).
template <typename R>
__device__ bool flight_plan(const RunParams& P, const Tab<R>& T, Part<R>& p, BlockCounters* bc, R& l,
                            uint32_t& pend, Hit& hit) {
  const int G = T.G;
  const int g = (int)pk_g(p.pk);
  if (kChecked) {
    // the particle's cell, group, lattice element and material index the tables
    const int c = (int)pk_cell(p.pk);
    if (!in_range(P, (uint64_t)c, (uint64_t)T.h->n_cell) || !in_range(P, (uint64_t)g, (uint64_t)G)) return false;
    if (T.cmat[c] < 0 &&
        !in_range(P, lat_e(p.elem), (uint64_t)T.h->lat_nx * T.h->lat_ny * T.h->lat_nz))
      return false;
    if (!in_range(P, (uint64_t)(int64_t)material_of(T, p.pk, p.elem), (uint64_t)T.h->M)) return false;
  }
  const int m = material_of(T, p.pk, p.elem);
  const R St = T.st[m * G + g];
  const Pair2<R> b0 = draw<R>(P.seed, p.tlo, p.thi, p.k, 0);  // (u_dist, u_channel)
  const R dc = St > R(0) ? rdiv(-rlog(b0.a), St) : rinf<R>();
  const R ds = boundary_distance(T, p, hit);
  R dt = rinf<R>();
  if (P.has_census) {
    const R d = sizeof(R) == 4 ? (R)p.census_distance((R)P.tc_hi, (R)P.tc_lo, T.v[g])
                               : (R)p.census_distance((R)P.tc, R(0), T.v[g]);
    dt = d > R(0) ? d : R(0);
  }
  bump(bc, MC_C_FLIGHT);
  if (dc < ds && dc < dt) {
    pend = PEND_COLL;
    l = dc;
    hit.chan = collision_channel(P, T, m, g, St, b0.b);
  } else if (ds <= dt) {
    pend = PEND_SURF;
    l = ds;
  } else {
    pend = PEND_NONE;  // census
    l = dt;
  }
  if (!(l < rinf<R>())) {
    bump(bc, MC_C_LOST);
    log_event(P, T, p, 3, 0, 0);
    set_status(P, MC_ERR_LOST);
    return false;
  }
  return true;
}

// Interior census of population control: banks the particle (event index = its census flight).
// Out of line: runs without census times never come here.
template <typename R>
__device__ __noinline__ void bank_census(const RunParams& P, const Part<R>& p, BlockCounters* bc) {
  const unsigned long long i = atomicAdd(&P.ctl->pc_n, 1ull);
  if (i < P.cap_c) bank_store(p, P.C, i);
  else set_status(P, MC_ERR_BANK_FULL);
  bump(bc, MC_C_PC_BANKED);
}

// Flight k, second half (after the segment was scored): move, advance the clock, set the pending
// event.  Returns false if the particle ends at the census or is captured at the flight's end.
template <typename R>
__device__ bool flight_finish(const RunParams& P, const Tab<R>& T, Part<R>& p, BlockCounters* bc, R l,
                              uint32_t pend, const Hit& hit) {
  const int g = (int)pk_g(p.pk);
  p.x += l * p.ux;
  p.y += l * p.uy;
  p.z += l * p.uz;
  p.advance(l, T.v[g], T.inv_v[g]);
  if (pend == PEND_NONE) {
    log_event(P, T, p, 2, 0, 0);
    if (P.pc_interior) bank_census(P, p, bc);
    else bump(bc, MC_C_CENSUS);
    return false;
  }
  if (pend == PEND_COLL && hit.chan == CHAN_CAPTURE) {
    // a capture ends the particle here: no bank round trip, no second draw of block 0
    bump(bc, MC_C_COLLISION);
    bump(bc, MC_C_CAPTURE);
    log_event(P, T, p, 0, 2, 0);
    return false;
  }
  p.pk = pk_set_pending(p.pk, pend, hit.type, hit.dir, hit.surf);
  if (pend == PEND_COLL) p.pk = pk_set_chan(p.pk, hit.chan);
  return true;
}

// source box and time in the tracking precision (float copies are made on the host)
__device__ __forceinline__ void source_box(const TableHeader* H, float lo[3], float hi[3]) {
  for (int i = 0; i < 3; ++i) {
    lo[i] = H->src_lo_f[i];
    hi[i] = H->src_hi_f[i];
  }
}
__device__ __forceinline__ void source_box(const TableHeader* H, double lo[3], double hi[3]) {
  for (int i = 0; i < 3; ++i) {
    lo[i] = H->src_lo[i];
    hi[i] = H->src_hi[i];
  }
}
__device__ __forceinline__ void source_time(const TableHeader* H, Part<float>& p, float u) {
  p.th = H->src_t0_f + (H->src_t1_f - H->src_t0_f) * u;
  p.tl = 0.0f;
}
__device__ __forceinline__ void source_time(const TableHeader* H, Part<double>& p, double u) {
  p.t = H->src_t0 + (H->src_t1 - H->src_t0) * u;
}

// statistical batch of history h (and of all its descendants): floor(h_rel nb / N), from a
// 32-bit reciprocal estimate corrected by exact 64-bit products (no 64-bit division)
__device__ __forceinline__ uint32_t batch_of(const RunParams& P, uint64_t h) {
  const uint32_t hr = (uint32_t)(h - P.h_first);
  const unsigned long long num = (unsigned long long)hr * (unsigned long long)P.n_batches;
  uint32_t q = __umulhi(hr, P.batch_magic);
  while ((unsigned long long)(q + 1) * P.n_hist <= num) ++q;
  while (q > 0 && (unsigned long long)q * P.n_hist > num) --q;
  return q;
}

// k-eigenvalue: the flight's contribution w l nu Sigma_f to the track-length estimate of k, in fixed
// point at 2^-32 (products rounded as the oracle rounds them, then to the nearest integer)
__device__ __forceinline__ long long eigen_tl_fixed(const Tab<float>& T, const Part<float>& p, float l) {
  const float nusf = T.nusf[material_of(T, p.pk, p.elem) * T.G + (int)pk_g(p.pk)];
  return float_to_fixed(__fmul_rn(__fmul_rn(__fmul_rn(weight_to_float(p.w), l), nusf), 4294967296.0f));
}
__device__ __forceinline__ long long eigen_tl_fixed(const Tab<double>& T, const Part<double>& p, double l) {
  const double nusf = T.nusf[material_of(T, p.pk, p.elem) * T.G + (int)pk_g(p.pk)];
  return __double2ll_rn(__dmul_rn(__dmul_rn(__dmul_rn(p.w, l), nusf), 4294967296.0));
}

// Source particle of history h of a k-eigenvalue cycle >= 1: at its fission site (picked by the
// systematic sampling of the previous cycle's bank), isotropic from its source draws (blocks 1, 2),
// the site's group, t = 0, weight 1, tag (h, cycle)
template <typename R>
__device__ __noinline__ bool make_site_source(const RunParams& P, const Tab<R>& T, uint64_t h, Part<R>& p) {
  const uint32_t tlo = (uint32_t)h, thi = P.cycle;
  const Pair2<R> b1 = draw<R>(P.seed, tlo, thi, kSourceEvent, 1);
  const Pair2<R> b2 = draw<R>(P.seed, tlo, thi, kSourceEvent, 2);
  int g = 0;
  site_load(P.src_site, h, p.x, p.y, p.z, g);
  iso_dir(R(2) * b1.b - R(1), b2.a, p.ux, p.uy, p.uz);
  p.zero_time();
  p.w = 1.0;
  p.tlo = tlo;
  p.thi = thi;
  p.k = 0;
  p.root = (uint32_t)h;
  p.elem = P.batch_fixed << 16;
  const int c = locate_cell(T, p.x, p.y, p.z, -1, 0);
  p.pk = pk_make((uint32_t)g, (uint32_t)(c < 0 ? 0 : c), 0u);
  if (c < 0) return false;
  if (T.cmat[c] < 0) lattice_locate(T, p);
  return true;
}

// Source particle of history h (event index kSourceEvent, blocks 0..3)
template <typename R>
__device__ bool make_source(const RunParams& P, const Tab<R>& T, uint64_t h, Part<R>& p) {
  if (P.eigen && P.cycle > 0) return make_site_source(P, T, h, p);
  const TableHeader* H = T.h;
  const uint32_t tlo = (uint32_t)h, thi = (uint32_t)(h >> 32);
  const Pair2<R> b0 = draw<R>(P.seed, tlo, thi, kSourceEvent, 0);
  const Pair2<R> b1 = draw<R>(P.seed, tlo, thi, kSourceEvent, 1);
  const Pair2<R> b2 = draw<R>(P.seed, tlo, thi, kSourceEvent, 2);
  const Pair2<R> b3 = draw<R>(P.seed, tlo, thi, kSourceEvent, 3);
  R lo[3], hi[3];
  source_box(H, lo, hi);
  if (H->src_pos == MC_SRC_BOX)
    p.x = lo[0] + (hi[0] - lo[0]) * b0.a;
  else
    p.x = lo[0];
  p.y = lo[1] + (hi[1] - lo[1]) * b0.b;
  p.z = lo[2] + (hi[2] - lo[2]) * b1.a;
  if (H->src_dir == MC_DIR_BEAM_X) {
    p.ux = R(1);
    p.uy = R(0);
    p.uz = R(0);
  } else {
    const R mu = H->src_dir == MC_DIR_COS_X ? rsqrt_(b1.b) : R(2) * b1.b - R(1);
    iso_dir(mu, b2.a, p.ux, p.uy, p.uz);
  }
  const int g = sample_cdf(T.src_cdf, T.G, b2.b);
  source_time(H, p, b3.a);
  p.w = 1.0;
  p.tlo = tlo;
  p.thi = thi;
  p.k = 0;
  p.root = (uint32_t)h;
  p.elem = (P.eigen ? P.batch_fixed : batch_of(P, h)) << 16;
  const int c = locate_cell(T, p.x, p.y, p.z, -1, 0);
  p.pk = pk_make((uint32_t)g, (uint32_t)(c < 0 ? 0 : c), 0u);
  if (c < 0) return false;
  if (T.cmat[c] < 0) lattice_locate(T, p);
  return true;
}

// ------------------------------------------------------------------------------------------ kernel
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Handles the pending event of a particle loaded from the bank; on survival it is ready to fly.
template <typename R>
__device__ __forceinline__ bool handle_pending(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                                               unsigned long long* bcount, BlockCounters* bc, uint64_t row,
                                               uint64_t stripe_off) {
  const uint32_t pend = pk_pend(p.pk);
  const uint64_t bbase = stripe_off + (uint64_t)(p.elem >> 16) * row;
  const bool alive = pend == PEND_COLL ? do_collision(P, T, p, Bout, bcount, bc)
                                       : do_surface(P, T, p, Bout, bcount, bc, bbase);
  if (alive) {
    p.k += 1;
    p.pk = pk_set_pending(p.pk, PEND_NONE, 0, 1, 0);
  }
  return alive;
}

// ------------------------------------------------------------------------------------------ stats
// Batch statistics of bin b of a tally laid out [stripes][nb][bins].  Fixed point: the exact
// integer sum over batches of the batch totals T_b and the exact 128-bit sum of T_b^2 (integer
// pipes only; the floating-point arithmetic happens once per bin at readback).  FP64: the sum of
// T_b and of the batch means and their squares (inv_nbar = batches / histories).
__device__ __forceinline__ void stats_bin_fixed(const long long* tally, uint64_t row, int nb, int stripes, uint64_t b,
                                                long long& sum, unsigned long long& sq_lo, unsigned long long& sq_hi) {
  const uint64_t stride = (uint64_t)nb * row;
  long long s = 0;
  unsigned long long lo = 0, hi = 0;
  for (int j = 0; j < nb; ++j) {
    long long x = 0;
    for (int c = 0; c < stripes; ++c) x += __ldcs(tally + c * stride + (uint64_t)j * row + b);
    s += x;
    const unsigned long long ux = (unsigned long long)(x < 0 ? -x : x);
    const unsigned long long plo = ux * ux, phi = __umul64hi(ux, ux);
    const unsigned long long nlo = lo + plo;
    hi += phi + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
  }
  sum = s;
  sq_lo = lo;
  sq_hi = hi;
}

__device__ __forceinline__ void stats_bin_fp64(const double* tally, uint64_t row, int nb, int stripes,
                                               double inv_nbar, uint64_t b, double& tot, double& s1, double& s2) {
  const uint64_t stride = (uint64_t)nb * row;
  double t = 0.0, a = 0.0, q = 0.0;
  for (int j = 0; j < nb; ++j) {
    double x = 0.0;
    for (int c = 0; c < stripes; ++c) x += __ldcs(tally + c * stride + (uint64_t)j * row + b);
    t += x;
    const double m = x * inv_nbar;
    a += m;
    q += m * m;
  }
  tot = t;
  s1 = a;
  s2 = q;
}

// Range-walk reconstruction of (batch j, range row r): a range row is one (tally, mesh cell, group)
// of a tally scored by the range walk.  Its difference slots hold, summed over the stripes, +w
// where a run starts and -w one past where it ends, so the running sum over k is the weight of the
// runs that cover k.  Track length: bin k is crossed in full by those flights, each with the track
// length v_g (t_{k+1} - t_k), and running sum x length is added to bin k (only bins 1 .. nt - 2
// can be crossed in full, so a bin of infinite width never takes part).  Time crossing: point k
// scores the running sum itself.  The warp scans the slots 32 at a time (shuffle scan with a
// carry) and adds to stripe 0; in fixed point the sums are exact integers, so the result does not
// depend on the order of the atomics.
__device__ inline void reconstruct_warp(void* tally, const char* blob64, uint64_t row, int nb, int stripes, int fp64,
                                        int j, uint64_t r) {
  const TableHeader* H = reinterpret_cast<const TableHeader*>(blob64);
  const int lane = threadIdx.x & 31;
  int t = 0;
  for (; t < H->n_tally; ++t) {
    const TallyDesc& D = H->tally[t];
    if (!D.range) continue;
    const uint64_t rows_t = (uint64_t)D.nx * D.ny * D.nz * H->G;
    if (r < rows_t) break;
    r -= rows_t;
  }
  if (t >= H->n_tally) return;
  const TallyDesc& D = H->tally[t];
  const int nt = D.nt;
  const bool crossing = D.est == MC_EST_TIME_CROSSING;
  const int nval = D.nval;                   // nt bins or nt + 1 points
  const int k_lo = crossing ? 0 : 1, k_hi = crossing ? nt : nt - 2;  // values a run can cover
  const int g = (int)(r % (uint64_t)H->G);
  const double v = reinterpret_cast<const double*>(blob64 + H->o_v)[g];
  const double* et = reinterpret_cast<const double*>(blob64 + D.o_et);
  const uint64_t stride = (uint64_t)nb * row;
  const uint64_t dslot = (uint64_t)j * row + (uint64_t)H->total_bins + (uint64_t)D.diff_offset + r * (uint64_t)D.ndiff;
  const uint64_t bslot = (uint64_t)j * row + (uint64_t)D.bin_offset + r * (uint64_t)nval;
  if (fp64) {
    double* T = reinterpret_cast<double*>(tally);
    double carry = 0.0;
    for (int k0 = 0; k0 < nval; k0 += 32) {
      const int k = k0 + lane;
      double d = 0.0;
      if (k < nval)
        for (int c = 0; c < stripes; ++c) d += __ldcg(T + c * stride + dslot + k);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xFFFFFFFFu, d, o);
        if (lane >= o) d += u;
      }
      const double run = carry + d;
      carry += __shfl_sync(0xFFFFFFFFu, d, 31);
      if (k >= k_lo && k <= k_hi && run != 0.0)
        T[bslot + k] += crossing ? run : run * (v * (et[k + 1] - et[k]));
    }
  } else {
    long long* T = reinterpret_cast<long long*>(tally);
    long long carry = 0;
    for (int k0 = 0; k0 < nval; k0 += 32) {
      const int k = k0 + lane;
      long long d = 0;
      if (k < nval)
        for (int c = 0; c < stripes; ++c) d += __ldcg(T + c * stride + dslot + k);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xFFFFFFFFu, d, o);
        if (lane >= o) d += u;
      }
      const long long run = carry + d;
      carry += __shfl_sync(0xFFFFFFFFu, d, 31);
      if (k >= k_lo && k <= k_hi && run != 0)
        T[bslot + k] += crossing ? run : __double2ll_rn((double)run * (v * (et[k + 1] - et[k])));
    }
  }
}


}  // namespace mcgb
