// Persistent event-based transport kernel and its helpers (sm_103a).
//
// One cooperative launch owns the whole run.  Each iteration every live particle performs one
// event and one flight:
//   [handle its pending event: collision or surface]  ->  [flight: distance to collision /
//   surface / census, move, track-length scoring]  ->  [append to the next bank, partitioned by
//   the kind of its new pending event: collisions from the front, surfaces from the back]
// so that in the next iteration warps take homogeneous work (all collisions, then all surfaces,
// then births).  Newly sourced histories fill the room left by particles that died; secondaries
// and weight-window copies go to a birth bank that the next iteration transports.  Iterations are
// separated by a grid barrier whose wait is bounded; the device status word reports overflow,
// lost particles and watchdog expiry instead of hanging or trapping.
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

__device__ __forceinline__ void set_status(Ctl* ctl, int code) { atomicCAS(&ctl->status, 0, code); }

// Sense-reversing grid barrier for a cooperative (co-resident) grid.  The spin is bounded by
// `limit` polls; on expiry the block records MC_ERR_TIMEOUT and leaves.  A waiting block also
// leaves as soon as any block has posted an error status, so one failing block cannot leave the
// others spinning; every block then stops at the top of its next iteration.
__device__ void grid_barrier(Ctl* ctl, unsigned long long limit) {
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
          set_status(ctl, MC_ERR_TIMEOUT);
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
  e.t = p.t; e.w = p.w;
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
    set_status(P.ctl, MC_ERR_BANK_FULL);
    return;
  }
  Lanes<R>::store(c, Bout, i);
}

// weight-window test after a collision or surface event (split above, roulette below)
template <typename R>
__device__ bool weight_window(const RunParams& P, const Tab<R>& T, Part<R>& p, uint4* const* Bout,
                              unsigned long long* bcount, BlockCounters* bc) {
  if (!P.ww_on) return true;
  const double* ex = P.ww_edges;
  const double* ey = ex + P.ww_nx + 1;
  const double* ez = ey + P.ww_ny + 1;
  const int ix = bin_search(ex, P.ww_nx, (double)p.x), iy = bin_search(ey, P.ww_ny, (double)p.y),
            iz = bin_search(ez, P.ww_nz, (double)p.z);
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
      score(P, batch_base + (uint64_t)(T.h->leak_offset + s), p.w, R(1));
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
        set_status(P.ctl, MC_ERR_LOST);
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

// Flight k: distance to collision, surface and census; move; score; set the pending event.
// Returns false if the particle ends here (census or lost).
template <typename R>
__device__ bool do_flight(const RunParams& P, const Tab<R>& T, Part<R>& p, BlockCounters* bc,
                          uint64_t batch_base) {
  const int G = T.G;
  const int g = (int)pk_g(p.pk);
  const int m = material_of(T, p.pk, p.elem);
  const R St = T.st[m * G + g];
  const R u = draw<R>(P.seed, p.tlo, p.thi, p.k, 0).a;
  const R dc = St > R(0) ? -rlog(u) / St : rinf<R>();
  Hit hit;
  const R ds = boundary_distance(T, p, hit);
  R dt = rinf<R>();
  const double tc = T.h->t_census;
  if (tc < CUDART_INF) {
    const double d = (double)T.v[g] * (tc - p.t);
    dt = d > 0.0 ? (R)d : R(0);
  }
  bump(bc, MC_C_FLIGHT);
  uint32_t pend;
  R l;
  if (dc < ds && dc < dt) {
    pend = PEND_COLL;
    l = dc;
  } else if (ds <= dt) {
    pend = PEND_SURF;
    l = ds;
  } else {
    pend = 0;
    l = dt;
  }
  if (!(l < rinf<R>())) {
    bump(bc, MC_C_LOST);
    log_event(P, T, p, 3, 0, 0);
    set_status(P.ctl, MC_ERR_LOST);
    return false;
  }
  score_segment(T, P, p, l, batch_base);
  p.x += l * p.ux;
  p.y += l * p.uy;
  p.z += l * p.uz;
  if (sizeof(R) == 8)
    p.t += (double)l / (double)T.v[g];
  else
    p.t += (double)(l * T.inv_v[g]);
  if (pend == 0) {
    bump(bc, MC_C_CENSUS);
    log_event(P, T, p, 2, 0, 0);
    return false;
  }
  p.pk = pk_set_pending(p.pk, pend, hit.type, hit.dir, hit.surf);
  return true;
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
  const R lo0 = (R)H->src_lo[0], lo1 = (R)H->src_lo[1], lo2 = (R)H->src_lo[2];
  if (H->src_pos == MC_SRC_BOX)
    p.x = lo0 + ((R)H->src_hi[0] - lo0) * b0.a;
  else
    p.x = lo0;
  p.y = lo1 + ((R)H->src_hi[1] - lo1) * b0.b;
  p.z = lo2 + ((R)H->src_hi[2] - lo2) * b1.a;
  if (H->src_dir == MC_DIR_BEAM_X) {
    p.ux = R(1);
    p.uy = R(0);
    p.uz = R(0);
  } else {
    const R mu = H->src_dir == MC_DIR_COS_X ? rsqrt_(b1.b) : R(2) * b1.b - R(1);
    iso_dir(mu, b2.a, p.ux, p.uy, p.uz);
  }
  const int g = sample_cdf(T.src_cdf, T.G, b2.b);
  p.t = H->src_t0 + (H->src_t1 - H->src_t0) * (double)b3.a;
  p.w = 1.0;
  p.tlo = tlo;
  p.thi = thi;
  p.k = 0;
  p.root = (uint32_t)h;
  p.elem = 0;
  const int c = locate_cell(T, p.x, p.y, p.z, -1, 0);
  p.pk = pk_make((uint32_t)g, (uint32_t)(c < 0 ? 0 : c), 0u);
  if (c < 0) return false;
  if (T.cmat[c] < 0) lattice_locate(T, p);
  return true;
}

// ------------------------------------------------------------------------------------------ kernel
template <typename R>
__global__ void __launch_bounds__(256) k_transport(RunParams P) {
  extern __shared__ __align__(16) char smem[];
  __shared__ BlockCounters bc;
  for (int i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = P.blob[i];
  if (threadIdx.x < MC_NCOUNTERS) bc.c[threadIdx.x] = 0u;
  __syncthreads();
  const Tab<R> T(smem);
  Ctl* ctl = P.ctl;
  const int lane = threadIdx.x & 31;
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t bins = (uint64_t)T.h->total_bins;

  for (uint64_t it = 0;; ++it) {
    const int cur = (int)(it % 3), nxt = (int)((it + 1) % 3), old = (int)((it + 2) % 3);
    if (ld_volatile_int(&ctl->status) != 0) break;
    // the counters cannot exceed the banks (overflow stops the run above); clamp regardless
    uint64_t nF = ld_volatile_u64(&ctl->front[cur]);
    uint64_t nS = ld_volatile_u64(&ctl->back[cur]);
    uint64_t nB = ld_volatile_u64(&ctl->birth[cur]);
    nB = nB < P.cap_b ? nB : P.cap_b;
    nF = nF < P.cap_s ? nF : P.cap_s;
    nS = nS < P.cap_s - nF ? nS : P.cap_s - nF;
    const uint64_t h0 = ld_volatile_u64(&ctl->hstart[cur]);
    const uint64_t room = P.cap_s - nF - nS;
    const uint64_t nBt = nB < room ? nB : room;  // births transported now; the rest wait
    const uint64_t left = P.n_hist - h0;
    const uint64_t room2 = room - nBt;
    const uint64_t nSrc = left < room2 ? left : room2;
    const uint64_t W = nF + nS + nB + nSrc;
    if (W == 0) break;
    if (it >= P.max_iter) {
      set_status(ctl, MC_ERR_TIMEOUT);
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->front[old] = 0ull;
      ctl->back[old] = 0ull;
      ctl->birth[old] = 0ull;
      ctl->hstart[nxt] = h0 + nSrc;
      ctl->iterations = it + 1;
    }
    uint4* const* Sin = P.S[it & 1];
    uint4* const* Sout = P.S[(it + 1) & 1];
    uint4* const* Bin = P.B[it & 1];
    uint4* const* Bout = P.B[(it + 1) & 1];
    unsigned long long* bcount = &ctl->birth[nxt];

    for (uint64_t base = gwarp * 32; base < W; base += nwarps * 32) {
      const uint64_t item = base + lane;
      bool alive = false;
      Part<R> p;
      if (item < W) {
        bool carry = false;
        bool have = true;
        if (item < nF) {
          Lanes<R>::load(p, Sin, item);
        } else if (item < nF + nS) {
          Lanes<R>::load(p, Sin, P.cap_s - 1 - (item - nF));
        } else if (item < nF + nS + nB) {
          const uint64_t j = item - nF - nS;
          Lanes<R>::load(p, Bin, j);
          carry = j >= nBt;
        } else {
          const uint64_t h = P.h_first + h0 + (item - nF - nS - nB);
          bump(&bc, MC_C_SOURCE);
          have = make_source(P, T, h, p);
          if (!have) {
            bump(&bc, MC_C_LOST);
            set_status(ctl, MC_ERR_LOST);
          }
        }
        if (carry) {
          append_birth(P, Bout, bcount, p);
        } else if (have) {
          const uint64_t batch = ((uint64_t)(p.root - (uint32_t)P.h_first) * (uint64_t)P.n_batches) / P.n_hist;
          const uint64_t bbase = batch * bins;
          const uint32_t pend = pk_pend(p.pk);
          alive = true;
          if (pend == PEND_COLL) alive = do_collision(P, T, p, Bout, bcount, &bc);
          else if (pend == PEND_SURF) alive = do_surface(P, T, p, Bout, bcount, &bc, bbase);
          if (alive) {
            if (pend != PEND_NONE) p.k += 1;
            p.pk = pk_set_pending(p.pk, PEND_NONE, 0, 1, 0);
            alive = do_flight(P, T, p, &bc, bbase);
          }
        }
      }
      // append survivors, partitioned by their pending event: one atomic per warp per side
      const bool wF = alive && pk_pend(p.pk) == PEND_COLL;
      const bool wS = alive && pk_pend(p.pk) == PEND_SURF;
      const unsigned mF = __ballot_sync(0xFFFFFFFFu, wF), mS = __ballot_sync(0xFFFFFFFFu, wS);
      unsigned long long bF = 0, bS = 0;
      if (lane == 0) {
        if (mF) bF = atomicAdd(&ctl->front[nxt], (unsigned long long)__popc(mF));
        if (mS) bS = atomicAdd(&ctl->back[nxt], (unsigned long long)__popc(mS));
      }
      bF = __shfl_sync(0xFFFFFFFFu, bF, 0);
      bS = __shfl_sync(0xFFFFFFFFu, bS, 0);
      const unsigned lt = lanemask_lt();
      // front + back <= items transported <= cap_s, so the two regions never meet
      if (wF) {
        const uint64_t i = bF + __popc(mF & lt);
        if (i < P.cap_s) Lanes<R>::store(p, Sout, i);
        else set_status(ctl, MC_ERR_BANK_FULL);
      }
      if (wS) {
        const uint64_t i = bS + __popc(mS & lt);
        if (i < P.cap_s) Lanes<R>::store(p, Sout, P.cap_s - 1 - i);
        else set_status(ctl, MC_ERR_BANK_FULL);
      }
    }
    grid_barrier(ctl, P.spin_limit);
  }
  __syncthreads();
  if (threadIdx.x < MC_NCOUNTERS && bc.c[threadIdx.x])
    atomicAdd(&ctl->counters[threadIdx.x], (unsigned long long)bc.c[threadIdx.x]);
}

// ------------------------------------------------------------------------------------------ stats
// Per bin: total over batches, and sum / sum of squares of the per-history batch means.
// History h belongs to batch floor(h nb / N), so batch j holds ceil((j+1)N/nb) - ceil(jN/nb) >= 1
// histories when N >= nb.
__global__ void k_batch_stats(const void* tally, int fp64, double inv_scale, uint64_t bins, int nb,
                              uint64_t n_hist, double* tot, double* s1, double* s2) {
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins;
       b += (uint64_t)gridDim.x * blockDim.x) {
    double t = 0.0, a = 0.0, q = 0.0;
    for (int j = 0; j < nb; ++j) {
      const uint64_t i = (uint64_t)j * bins + b;
      const double x = fp64 ? reinterpret_cast<const double*>(tally)[i]
                            : (double)reinterpret_cast<const long long*>(tally)[i] * inv_scale;
      t += x;
      const uint64_t lo = ((uint64_t)j * n_hist + nb - 1) / nb, hi = ((uint64_t)(j + 1) * n_hist + nb - 1) / nb;
      const double m = x / (double)(hi - lo);
      a += m;
      q += m * m;
    }
    tot[b] = t;
    s1[b] = a;
    s2[b] = q;
  }
}

__global__ void k_philox(uint64_t seed, const uint4* ctr, uint4* out, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr[i]);
}

// ------------------------------------------------------------------------------------------ launchers
template <typename R>
cudaError_t launch_transport(const RunParams& P, int grid, int block, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<RunParams*>(&P)};
  return cudaLaunchCooperativeKernel((const void*)k_transport<R>, grid, block, args, smem, s);
}

template <typename R>
cudaError_t transport_occupancy(int block, size_t smem, int* per_sm) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_transport<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, (const void*)k_transport<R>, block, smem);
}

template cudaError_t launch_transport<float>(const RunParams&, int, int, size_t, cudaStream_t);
template cudaError_t launch_transport<double>(const RunParams&, int, int, size_t, cudaStream_t);
template cudaError_t transport_occupancy<float>(int, size_t, int*);
template cudaError_t transport_occupancy<double>(int, size_t, int*);

cudaError_t launch_batch_stats(const void* tally, int fp64, double inv_scale, uint64_t bins, int nb,
                               uint64_t n_hist, double* tot, double* s1, double* s2, cudaStream_t s) {
  const int block = 256;
  uint64_t g = (bins + block - 1) / block;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  k_batch_stats<<<(unsigned)g, block, 0, s>>>(tally, fp64, inv_scale, bins, nb, n_hist, tot, s1, s2);
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
