// Persistent event-based transport kernel and its helpers (sm_103a).
//
// One cooperative launch owns the whole run.  Each iteration every live particle performs one
// event and one flight:
//   [handle its pending event: collision or surface]  ->  [flight: distance to collision /
//   surface / census, move, track-length scoring]  ->  [append to the next bank, partitioned by
//   the kind of its new pending event: collisions from the front, surfaces from the back]
// so that in the next iteration the claimed chunks of work are homogeneous (collisions, then
// surfaces, then births, then new sources).  Inside a CTA the two halves are compacted through a
// shared-memory queue: all threads handle claimed events, the survivors are packed into the
// queue, and the queue is flown by the first threads of the CTA, so flights run on full warps
// even though collisions kill particles.  Newly sourced histories fill the room left by particles
// that died; secondaries and weight-window copies go to a birth bank that the next iteration
// transports.  Once every history is sourced and few particles remain, the iteration runs
// history-style (particles stay in the queue until they die) so the tail costs one grid barrier
// per generation instead of one per event.  Iterations are separated by a grid barrier whose wait
// is bounded; the device status word reports overflow, lost particles and watchdog expiry instead
// of hanging or trapping.
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
__device__ void grid_barrier(const RunParams& P, Ctl* ctl, unsigned long long limit) {
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
template <typename R>
__device__ void log_event(const RunParams& P, const Tab<R>& T, const Part<R>& p, int kind,
                          int outcome, int n_child) {
  if (P.log == nullptr) return;
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
  e.elem = T.h->has_lat ? lat_iy(p.elem) * T.h->lat_nx + lat_ix(p.elem) : 0;
  e.in_pin = (int)pk_pin(p.pk);
  e.g = (int)pk_g(p.pk);
  e.x = p.x; e.y = p.y; e.z = p.z;
  e.ux = p.ux; e.uy = p.uy; e.uz = p.uz;
  e.t = p.time_d(); e.w = p.w;
  P.log[i] = e;
}

// ------------------------------------------------------------------------------------------ counters
struct BlockCounters {
  unsigned int c[MC_NCOUNTERS];
};
__device__ __forceinline__ void bump(BlockCounters* bc, int i, unsigned v = 1u) { atomicAdd(&bc->c[i], v); }

// ------------------------------------------------------------------------------------------ births
template <typename R>
__device__ __forceinline__ void append_birth(const RunParams& P, uint4* const* Bout, unsigned long long* counter,
                                             const Part<R>& c) {
  const unsigned long long i = atomicAdd(counter, 1ull);
  if (i >= P.cap_b) {
    set_status(P, MC_ERR_BANK_FULL);
    return;
  }
  bank_store(c, Bout, i);
}

// weight-window test after a collision or surface event (split above, roulette below)
template <typename R>
__device__ bool weight_window(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                              unsigned long long* bcount, BlockCounters* bc) {
  if (!P.ww_on) return true;
  const double* ex = P.ww_edges;
  const double* ey = ex + P.ww_nx + 1;
  const double* ez = ey + P.ww_ny + 1;
  // the window of the cell the particle moves into: a particle on a window-mesh edge (e.g. just
  // after crossing a layer plane that is also a mesh plane) is looked up 1e-9 cm ahead
  const double ah = 1e-9;
  const int ix = bin_search(ex, P.ww_nx, (double)p.x + ah * (double)p.ux),
            iy = bin_search(ey, P.ww_ny, (double)p.y + ah * (double)p.uy),
            iz = bin_search(ez, P.ww_nz, (double)p.z + ah * (double)p.uz);
  if (ix < 0 || ix >= P.ww_nx || iy < 0 || iy >= P.ww_ny || iz < 0 || iz >= P.ww_nz) return true;
  const double wc = __ldg(P.ww_center + ((size_t)(iz * P.ww_ny + iy) * P.ww_nx + ix) * T.G + pk_g(p.pk));
  if (!(wc > 0.0)) return true;
  if (p.w > P.ww_upper * wc) {
    int n = (int)ceil(p.w / wc);
    if (n > P.ww_split_max) n = P.ww_split_max;
    p.w = p.w / n;
    for (int j = 1; j < n; ++j) {
      Part<R> c = p;
      const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)j, kSplitMark);
      c.tlo = t.x;
      c.thi = t.y;
      c.k = 0;
      c.pk = pk_set_pending(c.pk, PEND_NONE, 0, 1, 0);
      append_birth(P, Bout, bcount, c);
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

// ------------------------------------------------------------------------------------------ events
// Handles the particle's pending collision at the end of flight k (uses the blocks of event k)
template <typename R>
__device__ bool do_collision(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                             unsigned long long* bcount, BlockCounters* bc) {
  const int G = T.G;
  const int g = (int)pk_g(p.pk);
  const int m = material_of(T, p.pk, p.elem);
  const R St = T.st[m * G + g];
  const R xi = draw<R>(P.seed, p.tlo, p.thi, p.k, 0).b * St;
  bump(bc, MC_C_COLLISION);
  if (xi < T.ss[m * G + g]) {
    bump(bc, MC_C_SCATTER);
    const Pair2<R> b1 = draw<R>(P.seed, p.tlo, p.thi, p.k, 1);
    const Pair2<R> b2 = draw<R>(P.seed, p.tlo, p.thi, p.k, 2);
    const int ng = sample_cdf(T.scdf + (m * G + g) * G, G, b1.a);
    log_event(P, T, p, 0, 0, 0);
    p.pk = (p.pk & ~0x1Fu) | (uint32_t)ng;
    iso_dir(R(2) * b1.b - R(1), b2.a, p.ux, p.uy, p.uz);
    return weight_window(P, T, p, Bout, bcount, bc);
  }
  if (xi < T.ssf[m * G + g]) {
    bump(bc, MC_C_PRODUCTION);
    const R u = draw<R>(P.seed, p.tlo, p.thi, p.k, 3).a;
    const int n = (int)floor(T.nu[m * G + g] + u);
    for (int j = 0; j < n; ++j) {
      Part<R> c = p;
      const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)j, kChildMark);
      c.tlo = t.x;
      c.thi = t.y;
      c.k = 0;
      const Pair2<R> c1 = draw<R>(P.seed, t.x, t.y, kSourceEvent, 1);
      const Pair2<R> c2 = draw<R>(P.seed, t.x, t.y, kSourceEvent, 2);
      iso_dir(R(2) * c1.b - R(1), c2.a, c.ux, c.uy, c.uz);
      const int cg = sample_cdf(T.chi + m * G, G, c2.b);
      c.pk = pk_set_pending((c.pk & ~0x1Fu) | (uint32_t)cg, PEND_NONE, 0, 1, 0);
      append_birth(P, Bout, bcount, c);
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
      Scorer<R>(P, p.w)(batch_base + (uint64_t)(T.h->leak_offset + s), R(1));
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
      const int nc = locate_cell(T, p.x, p.y, p.z, s, -old_sense);
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
    int ix = lat_ix(p.elem), iy = lat_iy(p.elem);
    if (hit == HIT_LAT_X) ix += pk_dir(p.pk);
    else iy += pk_dir(p.pk);
    p.elem = lat_pack(p.elem, ix, iy);
    p.pk = (p.pk & ~(1u << 13)) | (pin_inside(T, p.x, p.y, ix, iy) << 13);
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
  const int m = material_of(T, p.pk, p.elem);
  const R St = T.st[m * G + g];
  const R u = draw<R>(P.seed, p.tlo, p.thi, p.k, 0).a;
  const R dc = St > R(0) ? -rlog(u) / St : rinf<R>();
  const R ds = boundary_distance(T, p, hit);
  R dt = rinf<R>();
  if (T.h->has_census) {
    const R d = sizeof(R) == 4 ? (R)p.census_distance((R)T.h->tc_hi, (R)T.h->tc_lo, T.v[g])
                               : (R)p.census_distance((R)T.h->t_census, R(0), T.v[g]);
    dt = d > R(0) ? d : R(0);
  }
  bump(bc, MC_C_FLIGHT);
  if (dc < ds && dc < dt) {
    pend = PEND_COLL;
    l = dc;
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

// Flight k, second half (after the segment was scored): move, advance the clock, set the pending
// event.  Returns false if the particle ends at the census.
template <typename R>
__device__ bool flight_finish(const RunParams& P, const Tab<R>& T, Part<R>& p, BlockCounters* bc, R l,
                              uint32_t pend, const Hit& hit) {
  const int g = (int)pk_g(p.pk);
  p.x += l * p.ux;
  p.y += l * p.uy;
  p.z += l * p.uz;
  p.advance(l, T.v[g], T.inv_v[g]);
  if (pend == PEND_NONE) {
    bump(bc, MC_C_CENSUS);
    log_event(P, T, p, 2, 0, 0);
    return false;
  }
  p.pk = pk_set_pending(p.pk, pend, hit.type, hit.dir, hit.surf);
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

// Source particle of history h (event index kSourceEvent, blocks 0..3)
template <typename R>
__device__ bool make_source(const RunParams& P, const Tab<R>& T, uint64_t h, Part<R>& p) {
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
  p.elem = batch_of(P, h) << 16;
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
                                               unsigned long long* bcount, BlockCounters* bc, uint64_t bins,
                                               uint64_t stripe_off) {
  const uint32_t pend = pk_pend(p.pk);
  const uint64_t bbase = stripe_off + (uint64_t)(p.elem >> 16) * bins;
  const bool alive = pend == PEND_COLL ? do_collision(P, T, p, Bout, bcount, bc)
                                       : do_surface(P, T, p, Bout, bcount, bc, bbase);
  if (alive) {
    p.k += 1;
    p.pk = pk_set_pending(p.pk, PEND_NONE, 0, 1, 0);
  }
  return alive;
}

// Items a warp claims per atomic on the iteration's work counter (processed 32 at a time).
constexpr unsigned kClaim = 128;
constexpr unsigned kWarpQ = 64;  // per-warp flight queue slots

// dynamic shared memory: [table blob][per-warp flight queues: warps x Lanes<R>::N x kWarpQ]
template <typename R, int MINB>
__global__ void __launch_bounds__(256, MINB) k_transport(RunParams P) {
  extern __shared__ __align__(16) char smem[];
  __shared__ BlockCounters bc;
  __shared__ int s_status;
  for (int i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = P.blob[i];
  if (threadIdx.x < MC_NCOUNTERS) bc.c[threadIdx.x] = 0u;
  __syncthreads();
  const Tab<R> T(smem);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint4* wq = reinterpret_cast<uint4*>(smem + P.blob_bytes) + warp * (Lanes<R>::N * kWarpQ);
  // per-warp tally staging buffers follow the queues: values (8 B) then slots (4 B)
  char* stage_base = smem + P.blob_bytes + (size_t)nwarp * Lanes<R>::N * kWarpQ * 16;
  const Stage stage{reinterpret_cast<uint32_t*>(stage_base + (size_t)nwarp * kStage * 8) + warp * kStage,
                    reinterpret_cast<unsigned long long*>(stage_base) + warp * kStage};
  Ctl* ctl = P.ctl;
  const unsigned lt = lanemask_lt();
  unsigned scored = 0;  // tally updates issued by this warp
  const uint64_t bins = (uint64_t)T.h->total_bins;
  // small tallies are striped over several copies so that hot bins are not one L2 address
  const uint64_t stripe_off = (uint64_t)(blockIdx.x % P.tally_stripes) * P.stripe_stride;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_start = globaltimer();

  for (uint64_t it = 0;; ++it) {
    const int cur = (int)(it % 3), nxt = (int)((it + 1) % 3), old = (int)((it + 2) % 3);
    // the status word can change at any time (another CTA may post an error): read it once per
    // CTA so that every thread of the CTA takes the same branch
    if (threadIdx.x == 0) s_status = ld_volatile_int(&ctl->status);
    __syncthreads();
    if (s_status != 0) break;
    // the counters cannot exceed the banks (overflow stops the run above); clamp regardless
    uint64_t nF = ld_volatile_u64(&ctl->front[cur]);
    uint64_t nS = ld_volatile_u64(&ctl->back[cur]);
    uint64_t nB = ld_volatile_u64(&ctl->birth[cur]);
    nB = nB < P.cap_b ? nB : P.cap_b;
    nF = nF < P.cap_s ? nF : P.cap_s;
    nS = nS < P.cap_s - nF ? nS : P.cap_s - nF;
    const uint64_t h0 = ld_volatile_u64(&ctl->hstart[cur]);
    const uint64_t left = P.n_hist - h0;
    // history-style iterations never write survivors back, so the transport bank is all room
    const uint64_t room = P.history_mode ? P.cap_s : P.cap_s - nF - nS;
    const uint64_t nBt = nB < room ? nB : room;  // births transported now; the rest wait
    const uint64_t room2 = room - nBt;
    const uint64_t nSrc = left < room2 ? left : room2;
    const uint64_t W = nF + nS + nB + nSrc;
    if (W == 0) break;
    if (it >= P.max_iter) {
      set_status(P, MC_ERR_TIMEOUT);
      break;
    }
    const bool drain = P.history_mode || (nSrc == left && W <= P.drain_threshold);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->front[old] = 0ull;
      ctl->back[old] = 0ull;
      ctl->birth[old] = 0ull;
      ctl->next[old] = 0ull;
      ctl->hstart[nxt] = h0 + nSrc;
      ctl->iterations = it + 1;
      if (P.trace && it < P.trace_cap) {
        P.trace[3 * it] = globaltimer();
        P.trace[3 * it + 1] = W;
        P.trace[3 * it + 2] = nSrc | (drain ? (1ull << 63) : 0ull);
      }
    }
    uint4* const* Sin = P.S[it & 1];
    uint4* const* Sout = P.S[(it + 1) & 1];
    uint4* const* Bin = P.B[it & 1];
    uint4* const* Bout = P.B[(it + 1) & 1];
    unsigned long long* bcount = &ctl->birth[nxt];
    unsigned long long* claim = &ctl->next[cur];

    // Warp loop with a per-warp flight queue in shared memory.  (A) While fewer than 32
    // particles are queued, the warp takes the next 32 items of its claimed range, handles their
    // pending events on all lanes, and packs the survivors into the queue.  (B) The warp flies up
    // to 32 queued particles on full lanes and appends the survivors to the next bank (or, in
    // history-style iterations, handles their next event and queues them again).  The queue
    // count is warp-uniform and lives in a register; only __syncwarp orders the queue accesses.
    unsigned qn = 0;
    uint64_t rbeg = 0, rend = 0;  // the warp's claimed item range
    bool exhausted = false;
    while (true) {
      while (qn < 32u && !(exhausted && rbeg >= rend)) {
        if (rbeg >= rend) {
          unsigned long long b = 0;
          if (lane == 0) b = atomicAdd(claim, (unsigned long long)kClaim);
          b = __shfl_sync(0xFFFFFFFFu, b, 0);
          rbeg = b;
          rend = b + kClaim < W ? b + kClaim : W;
          if (b + kClaim >= W) exhausted = true;
          if (rbeg >= rend) break;
        }
        const uint64_t item = rbeg + lane;
        rbeg = rbeg + 32 < rend ? rbeg + 32 : rend;
        Part<R> p;
        bool ready = false;
        if (item < rend) {
          if (item < nF + nS) {
            bank_load(p, Sin, item < nF ? item : P.cap_s - 1 - (item - nF));
            ready = handle_pending(P, T, p, Bout, bcount, &bc, bins, stripe_off);
          } else if (item < nF + nS + nB) {
            const uint64_t j = item - nF - nS;
            bank_load(p, Bin, j);
            if (j >= nBt) append_birth(P, Bout, bcount, p);  // waits for room
            else ready = true;
          } else {
            const uint64_t h = P.h_first + h0 + (item - nF - nS - nB);
            bump(&bc, MC_C_SOURCE);
            ready = make_source(P, T, h, p);
            if (!ready) {
              bump(&bc, MC_C_LOST);
              set_status(P, MC_ERR_LOST);
            }
          }
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, ready);
        if (ready) queue_store(p, wq, kWarpQ, qn + __popc(m & lt));
        qn += __popc(m);
        __syncwarp();
      }
      if (qn == 0u) break;  // the warp's items are exhausted and nothing is left to fly
      const unsigned nfly = qn < 32u ? qn : 32u;
      Part<R> p;
      const bool have = (unsigned)lane < nfly;
      if (have) queue_load(p, wq, kWarpQ, qn - nfly + lane);
      __syncwarp();
      qn -= nfly;
      bool out = false, again = false;
      R l = R(0);
      uint32_t pend = PEND_NONE;
      Hit hit;
      const bool flies = have && flight_plan(P, T, p, &bc, l, pend, hit);
      score_segment_warp(T, P, p, l, stripe_off + (uint64_t)(p.elem >> 16) * bins, flies, stage, scored);
      if (flies) {
        bool alive = flight_finish(P, T, p, &bc, l, pend, hit);
        if (alive && p.k + 1 >= P.max_iter) {
          // a particle that never ends (e.g. a reflective void without census) cannot keep the
          // warp busy forever in history-style iterations: the same budget as the iteration
          // watchdog ends it with MC_ERR_TIMEOUT
          set_status(P, MC_ERR_TIMEOUT);
          alive = false;
        }
        if (alive) {
          if (drain) again = handle_pending(P, T, p, Bout, bcount, &bc, bins, stripe_off);
          else out = true;
        }
      }
      if (drain) {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, again);
        if (again) queue_store(p, wq, kWarpQ, qn + __popc(m & lt));
        qn += __popc(m);
        __syncwarp();
        continue;
      }
      // append survivors, partitioned by their pending event: one atomic per warp per side
      const bool wF = out && pk_pend(p.pk) == PEND_COLL;
      const bool wS = out && pk_pend(p.pk) == PEND_SURF;
      const unsigned mF = __ballot_sync(0xFFFFFFFFu, wF), mS = __ballot_sync(0xFFFFFFFFu, wS);
      if (mF | mS) {
        unsigned long long bF = 0, bS = 0;
        if (lane == 0) {
          if (mF) bF = atomicAdd(&ctl->front[nxt], (unsigned long long)__popc(mF));
          if (mS) bS = atomicAdd(&ctl->back[nxt], (unsigned long long)__popc(mS));
        }
        bF = __shfl_sync(0xFFFFFFFFu, bF, 0);
        bS = __shfl_sync(0xFFFFFFFFu, bS, 0);
        // front + back <= items transported <= cap_s, so the two regions never meet
        if (wF) {
          const uint64_t i = bF + __popc(mF & lt);
          if (i < P.cap_s) bank_store(p, Sout, i);
          else set_status(P, MC_ERR_BANK_FULL);
        }
        if (wS) {
          const uint64_t i = bS + __popc(mS & lt);
          if (i < P.cap_s) bank_store(p, Sout, P.cap_s - 1 - i);
          else set_status(P, MC_ERR_BANK_FULL);
        }
      }
    }
    grid_barrier(P, ctl, P.spin_limit);
  }
  if ((threadIdx.x & 31) == 0 && scored) atomicAdd(&bc.c[MC_C_SCORES], scored);
  __syncthreads();
  if (threadIdx.x < MC_NCOUNTERS && bc.c[threadIdx.x])
    atomicAdd(&ctl->counters[threadIdx.x], (unsigned long long)bc.c[threadIdx.x]);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_end = globaltimer();
}

// ------------------------------------------------------------------------------------------ stats
// Batch statistics of every bin.  Fixed-point tallies: the exact integer sum over batches of the
// batch totals T_b and the exact 128-bit sum of T_b^2 (integer pipes only; the final
// floating-point arithmetic happens once per bin at readback).  FP64 tallies: sum of T_b and of
// the batch means and their squares, with the mean batch size.
__global__ void k_batch_stats_fixed(const long long* tally, uint64_t bins, int nb, int stripes, long long* sum,
                                    unsigned long long* sq_lo, unsigned long long* sq_hi) {
  const uint64_t stride = (uint64_t)nb * bins;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins;
       b += (uint64_t)gridDim.x * blockDim.x) {
    long long s = 0;
    unsigned long long lo = 0, hi = 0;
    for (int j = 0; j < nb; ++j) {
      long long x = 0;
      for (int c = 0; c < stripes; ++c) x += __ldcs(tally + c * stride + (uint64_t)j * bins + b);
      s += x;
      const unsigned long long ux = (unsigned long long)(x < 0 ? -x : x);
      const unsigned long long plo = ux * ux, phi = __umul64hi(ux, ux);
      const unsigned long long nlo = lo + plo;
      hi += phi + (nlo < lo ? 1ull : 0ull);
      lo = nlo;
    }
    sum[b] = s;
    sq_lo[b] = lo;
    sq_hi[b] = hi;
  }
}

__global__ void k_batch_stats_fp64(const double* tally, uint64_t bins, int nb, int stripes, double inv_nbar,
                                   double* tot, double* s1, double* s2) {
  const uint64_t stride = (uint64_t)nb * bins;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins;
       b += (uint64_t)gridDim.x * blockDim.x) {
    double t = 0.0, a = 0.0, q = 0.0;
    for (int j = 0; j < nb; ++j) {
      double x = 0.0;
      for (int c = 0; c < stripes; ++c) x += __ldcs(tally + c * stride + (uint64_t)j * bins + b);
      t += x;
      const double m = x * inv_nbar;
      a += m;
      q += m * m;
    }
    tot[b] = t;
    s1[b] = a;
    s2[b] = q;
  }
}

// L2 atomic throughput probe: 64-bit adds to pseudo-random slots of an array of `span` elements
// (the access pattern of tally scoring), `iters` per thread.
__global__ void k_atomic_probe(unsigned long long* a, unsigned long long span, int iters, unsigned salt) {
  unsigned long long x = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * 2654435761ull + salt;
  for (int i = 0; i < iters; ++i) {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    atomicAdd(a + ((x >> 20) % span), 1ull);
  }
}

cudaError_t launch_atomic_probe(unsigned long long* a, unsigned long long span, int grid, int iters, unsigned salt,
                                cudaStream_t s) {
  k_atomic_probe<<<grid, 256, 0, s>>>(a, span, iters, salt);
  return cudaGetLastError();
}

__global__ void k_philox(uint64_t seed, const uint4* ctr, uint4* out, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr[i]);
}

// ------------------------------------------------------------------------------------------ launchers
// Two register budgets of the same kernel: 3 CTAs of 256 threads per SM (80 registers) or 2 CTAs
// (128 registers, no spills); `wide` selects the second.
template <typename R>
static const void* transport_fn(bool wide) {
  if (sizeof(R) == 8) return (const void*)k_transport<R, 2>;
  return wide ? (const void*)k_transport<R, 2> : (const void*)k_transport<R, 3>;
}

template <typename R>
cudaError_t launch_transport(const RunParams& P, int grid, int block, size_t smem, cudaStream_t s, bool wide) {
  void* args[] = {const_cast<RunParams*>(&P)};
  return cudaLaunchCooperativeKernel(transport_fn<R>(wide), grid, block, args, smem, s);
}

template <typename R>
cudaError_t transport_occupancy(int block, size_t smem, int* per_sm, bool wide) {
  const void* f = transport_fn<R>(wide);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, f, block, smem);
}

template cudaError_t launch_transport<float>(const RunParams&, int, int, size_t, cudaStream_t, bool);
template cudaError_t launch_transport<double>(const RunParams&, int, int, size_t, cudaStream_t, bool);
template cudaError_t transport_occupancy<float>(int, size_t, int*, bool);
template cudaError_t transport_occupancy<double>(int, size_t, int*, bool);

cudaError_t launch_batch_stats(const void* tally, int fp64, uint64_t bins, int nb, int stripes,
                               uint64_t n_hist, void* out, cudaStream_t s) {
  const int block = 256;
  uint64_t g = (bins + block - 1) / block;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  if (fp64) {
    double* o = reinterpret_cast<double*>(out);
    k_batch_stats_fp64<<<(unsigned)g, block, 0, s>>>(reinterpret_cast<const double*>(tally), bins, nb, stripes,
                                                     (double)nb / (double)n_hist, o, o + bins, o + 2 * bins);
  } else {
    char* o = reinterpret_cast<char*>(out);
    k_batch_stats_fixed<<<(unsigned)g, block, 0, s>>>(
        reinterpret_cast<const long long*>(tally), bins, nb, stripes, reinterpret_cast<long long*>(o),
        reinterpret_cast<unsigned long long*>(o + 8 * bins), reinterpret_cast<unsigned long long*>(o + 16 * bins));
  }
  return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t seed, const uint4* ctr, uint4* out, uint64_t n, cudaStream_t s) {
  const int block = 256;
  uint64_t g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  k_philox<<<(unsigned)g, block, 0, s>>>(seed, ctr, out, n);
  return cudaGetLastError();
}

}  // namespace mcgb
