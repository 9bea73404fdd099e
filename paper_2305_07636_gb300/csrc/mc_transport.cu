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

#include "mc_events.cuh"

namespace mcgb {

// Items a warp claims per atomic on the iteration's work counter (processed 32 at a time): kClaim
// while more than kTailWaves claims per warp of the grid remain, kClaimTail after that, so that
// the warps of the grid run out of work at nearly the same time and wait less at the barrier.
#ifndef MCGB_CLAIM
#define MCGB_CLAIM 128
#endif
#ifndef MCGB_CLAIM_TAIL
#define MCGB_CLAIM_TAIL 32
#endif
#ifndef MCGB_TAIL_WAVES
#define MCGB_TAIL_WAVES 2
#endif
constexpr unsigned kClaim = MCGB_CLAIM, kClaimTail = MCGB_CLAIM_TAIL, kTailWaves = MCGB_TAIL_WAVES;

// dynamic shared memory: [table blob][per-warp flight queues: warps x Lanes<R>::N x kWarpQ]
// [per-warp tally staging: warps x kStage x 12 B]
//
// MODE 0 runs the whole transport in one launch: event-based iterations, then history-style ones
// once the work left is below the drain threshold.  A split run launches MODE 1, which stops where
// MODE 0 would turn history-style (and records that iteration in ctl->tail_it), then MODE 2, which
// runs the history-style iterations from there with per-warp stacks of secondaries: a warp flies
// its particles' secondaries before it claims more work, so one history-style iteration ends the
// run instead of one per generation of secondaries, and the event-based launch carries none of
// the tail's code.
template <typename R, int MINB, bool RANGE, bool SEG, int MODE>
__global__ void __launch_bounds__(256, MINB) k_transport(RunParams P) {
  extern __shared__ __align__(16) char smem[];
  __shared__ BlockCounters bc;
  __shared__ int s_status;
  for (int i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = P.blob[i];
  if (threadIdx.x < MC_NCOUNTERS) bc.c[threadIdx.x] = 0u;
  if (threadIdx.x < 8) bc.wn[threadIdx.x] = 0u;
  if (threadIdx.x == 0) bc.local = MODE == 2 && P.WS[0] != nullptr ? 1u : 0u;
  __syncthreads();
  const Tab<R> T(smem);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint4* wq = reinterpret_cast<uint4*>(smem + P.blob_bytes) + warp * (Lanes<R>::N * kWarpQ);
  // per-warp tally staging buffers follow the queues: values (8 B) then slots (4 B)
  char* stage_base = smem + P.blob_bytes + (size_t)nwarp * Lanes<R>::N * kWarpQ * 16;
  const Stage stage{reinterpret_cast<uint32_t*>(stage_base + (size_t)nwarp * kStage * 8) + warp * kStage,
                    reinterpret_cast<unsigned long long*>(stage_base) + warp * kStage};
  // SEG: the warp's region of segments waiting to be scored, ns of them (warp-uniform)
  uint4* const sq = SEG ? P.seg + ((size_t)blockIdx.x * nwarp + warp) * (kSegLanes * kSegCap) : nullptr;
  unsigned ns = 0;
  Ctl* ctl = P.ctl;
  const unsigned lt = lanemask_lt();
  unsigned scored = 0;  // tally updates issued by this warp
  long long ktl = 0;    // k-eigenvalue cycle: this thread's track-length estimate of k (fixed point)
  const uint64_t row = P.row;  // tally elements per batch: bins, then difference slots
  // small tallies are striped over several copies so that hot bins are not one L2 address
  const uint64_t stripe_off = (uint64_t)(blockIdx.x % P.tally_stripes) * P.stripe_stride;
  if (MODE != 2 && blockIdx.x == 0 && threadIdx.x == 0) ctl->t_start = globaltimer();

  for (uint64_t it = MODE == 2 ? ld_volatile_u64(&ctl->tail_it) : 0ull;; ++it) {
    const int cur = (int)(it % 3), nxt = (int)((it + 1) % 3), old = (int)((it + 2) % 3);
    // event-based launch of a split run: whichever way it ends (history-style turn, no work left,
    // an error), the tail launch starts from the iteration recorded here (the counters it reads
    // are those every CTA of this launch read)
    if (MODE == 1 && blockIdx.x == 0 && threadIdx.x == 0) ctl->tail_it = it;
    // the status word can change at any time (another CTA may post an error): read it once per
    // CTA so that every thread of the CTA takes the same branch
    if (threadIdx.x == 0) s_status = ld_volatile_int(&ctl->status);
    __syncthreads();
    if (s_status != 0) break;
    // the counters cannot exceed the banks (overflow stops the run above); clamp regardless
    // the next bank's fill: collision-pending particles in the low half, surface-pending ones in the high half
    const unsigned long long fb = ld_volatile_u64(&ctl->fb[cur]);
    uint64_t nF = fb & 0xFFFFFFFFull;
    uint64_t nS = fb >> 32;
    uint64_t nB = ld_volatile_u64(&ctl->birth[cur]);
    nB = nB < P.cap_b ? nB : P.cap_b;
    nF = nF < P.cap_s ? nF : P.cap_s;
    nS = nS < P.cap_s - nF ? nS : P.cap_s - nF;
    const uint64_t h0 = ld_volatile_u64(&ctl->hstart[cur]);
    const uint64_t left = P.n_sources - h0;
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
    const bool drain = MODE == 2 || P.history_mode || (nSrc == left && W <= P.drain_threshold);
    if (MODE == 1 && drain) break;  // the tail launch takes over from this iteration
    const bool hs = MODE == 2 || (MODE == 0 && drain);  // this iteration runs history-style
    // splits are held once the copies made in this iteration would exceed half the birth store,
    // less the nB - nBt waiting births that are stored again below
    if (threadIdx.x == 0) {
      bc.split_ctr = &ctl->splits[cur];
      bc.hold_at = P.cap_b / 2 > nB - nBt ? P.cap_b / 2 - (nB - nBt) : 0ull;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->fb[old] = 0ull;
      ctl->splits[old] = 0ull;
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
    // the items left when the claims switch to the tail size (the end of the previous claimed
    // range stands for the shared claim counter, which only grows)
    const uint64_t tail = (uint64_t)kTailWaves * kClaim * gridDim.x * nwarp;
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
      while (qn < 32u && ((MODE == 2 && bc.wn[warp] != 0u) || !(exhausted && rbeg >= rend))) {
        if constexpr (MODE == 2) {
          // secondaries of this warp's particles first (depth first keeps the stack shallow)
          const unsigned sn = bc.wn[warp] < (unsigned)P.ws_cap ? bc.wn[warp] : (unsigned)P.ws_cap;
          if (sn != 0u) {
            const unsigned k = sn < 32u - qn ? sn : 32u - qn;
            if ((unsigned)lane < k) {
              Part<R> b;
              bank_load(b, P.WS, ((uint64_t)blockIdx.x * nwarp + warp) * P.ws_cap + sn - k + lane);
              queue_store(b, wq, kWarpQ, qn + lane);
            }
            __syncwarp();
            if (lane == 0) bc.wn[warp] = sn - k;
            __syncwarp();
            qn += k;
            continue;
          }
        }
        if (rbeg >= rend) {
          unsigned long long b = 0;
          const unsigned take = rend + tail < W ? kClaim : kClaimTail;
          if (lane == 0) b = atomicAdd(claim, (unsigned long long)take);
          b = __shfl_sync(0xFFFFFFFFu, b, 0);
          rbeg = b;
          rend = b + take < W ? b + take : W;
          if (b + take >= W) exhausted = true;
          if (rbeg >= rend) break;
        }
        const uint64_t item = rbeg + lane;
        rbeg = rbeg + 32 < rend ? rbeg + 32 : rend;
        Part<R> p;
        bool ready = false;
        if (item < rend) {
          if (item < nF + nS) {
            bank_load(p, Sin, item < nF ? item : P.cap_s - 1 - (item - nF));
            ready = handle_pending(P, T, p, Bout, bcount, &bc, row, stripe_off);
          } else if (item < nF + nS + nB) {
            const uint64_t j = item - nF - nS;
            bank_load(p, Bin, j);
            if (j >= nBt) append_birth(P, Bout, bcount, &bc, p);  // waits for room
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
      if constexpr (SEG) {
        // a full warp of segments whenever 32 wait; fewer stay in the warp's region into the next
        // iteration (a record holds all it needs), and the rest is scored when the run ends
        if (ns >= 32u) score_segments(T, P, sq, ns, false, stripe_off, stage, scored);
      }
      if (qn == 0u) break;  // the warp's items are exhausted and nothing is left to fly
      const unsigned nfly = qn < 32u ? qn : 32u;
      Part<R> p;
      const bool have = (unsigned)lane < nfly;
      if (have) queue_load(p, wq, kWarpQ, qn - nfly + lane);
      __syncwarp();
      qn -= nfly;
      bool again = false;
      R l = R(0);
      uint32_t pend = PEND_NONE;
      Hit hit;
      const bool flies = have && flight_plan(P, T, p, &bc, l, pend, hit);
      // The particles that survive this flight into the next bank are known once it is planned:
      // a collision other than a capture (front of the bank) or a surface crossing (back); only
      // the watchdog below can still end one of them, and it stops the run.  Their slots are
      // reserved now with one atomic per warp on the packed pair of counts (front in the low
      // half, back in the high half), so the atomic's latency hides behind the scoring.
      const bool wF = !hs && flies && pend == PEND_COLL && hit.chan != CHAN_CAPTURE;
      const bool wS = !hs && flies && pend == PEND_SURF;
      const unsigned mF = __ballot_sync(0xFFFFFFFFu, wF), mS = __ballot_sync(0xFFFFFFFFu, wS);
      unsigned long long bFS = 0;
      if (lane == 0 && (mF | mS))
        bFS = atomicAdd(&ctl->fb[nxt], (unsigned long long)__popc(mF) | ((unsigned long long)__popc(mS) << 32));
      if (P.eigen && flies) ktl += eigen_tl_fixed(T, p, l);
      if constexpr (SEG) {
        const bool sc = flies && (!P.eigen || P.eigen_score);
        const unsigned msc = __ballot_sync(0xFFFFFFFFu, sc);
        if (sc) seg_push_flight(sq, ns + __popc(msc & lt), p, l);
        ns += __popc(msc);
      } else {
        score_segment_warp<R, RANGE>(T, P, p, l, stripe_off + (uint64_t)(p.elem >> 16) * row,
                                     flies && (!P.eigen || P.eigen_score), stage, scored);
      }
      if (flies) {
        bool alive = flight_finish(P, T, p, &bc, l, pend, hit);
        if (alive && p.k + 1 >= P.max_iter) {
          // a particle that never ends (e.g. a reflective void without census) cannot keep the
          // warp busy forever in history-style iterations: the same budget as the iteration
          // watchdog ends it with MC_ERR_TIMEOUT
          set_status(P, MC_ERR_TIMEOUT);
          alive = false;
        }
        if (alive && hs) again = handle_pending(P, T, p, Bout, bcount, &bc, row, stripe_off);
      }
      if (hs) {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, again);
        if (again) queue_store(p, wq, kWarpQ, qn + __popc(m & lt));
        qn += __popc(m);
        __syncwarp();
        continue;
      }
      // append the survivors into the reserved slots, partitioned by their pending event
      if (mF | mS) {
        bFS = __shfl_sync(0xFFFFFFFFu, bFS, 0);
        const uint64_t bF = bFS & 0xFFFFFFFFull, bS = bFS >> 32;
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
  if constexpr (SEG) {
    if (ns > 0u) score_segments(T, P, sq, ns, true, stripe_off, stage, scored);
  }
  if (P.eigen) {
    for (int o = 16; o > 0; o >>= 1) ktl += __shfl_xor_sync(0xFFFFFFFFu, ktl, o);
    if ((threadIdx.x & 31) == 0 && ktl) atomicAdd(&ctl->k_acc, (unsigned long long)ktl);
  }
  if ((threadIdx.x & 31) == 0 && scored) atomicAdd(&bc.c[MC_C_SCORES], scored);
  __syncthreads();
  if (threadIdx.x < MC_NCOUNTERS && bc.c[threadIdx.x])
    atomicAdd(&ctl->counters[threadIdx.x], (unsigned long long)bc.c[threadIdx.x]);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_end = globaltimer();
}

// ------------------------------------------------------------------------------------------ stats
// Batch statistics of every bin of one problem (stats_bin_fixed / stats_bin_fp64 per bin); batch
// rows are `row` elements apart.
__global__ void k_batch_stats_fixed(const long long* tally, uint64_t bins, uint64_t row, int nb, int stripes,
                                    long long* sum, unsigned long long* sq_lo, unsigned long long* sq_hi) {
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins;
       b += (uint64_t)gridDim.x * blockDim.x)
    stats_bin_fixed(tally, row, nb, stripes, b, sum[b], sq_lo[b], sq_hi[b]);
}

__global__ void k_batch_stats_fp64(const double* tally, uint64_t bins, uint64_t row, int nb, int stripes,
                                   double inv_nbar, double* tot, double* s1, double* s2) {
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins;
       b += (uint64_t)gridDim.x * blockDim.x)
    stats_bin_fp64(tally, row, nb, stripes, inv_nbar, b, tot[b], s1[b], s2[b]);
}

// Range-walk reconstruction of every batch of one problem (reconstruct_warp per (batch, row)).
__global__ void k_reconstruct(void* tally, const char* blob64, uint64_t rows, uint64_t row, int nb, int stripes,
                              int fp64) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t wi = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < (uint64_t)nb * rows;
       wi += warps)
    reconstruct_warp(tally, blob64, row, nb, stripes, fp64, (int)(wi / rows), wi % rows);
}

// ------------------------------------------------------------------------------------------ k-eigenvalue
// Inclusive scan of the sites banked per history (uint32, n entries) into uint64 offsets: per
// block of 1024 entries (256 threads x 4), then over the block totals, then the block offsets.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* warp_tot,
                                                                   unsigned long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const unsigned long long before = (warp > 0 ? warp_tot[warp - 1] : 0ull) + x - v;
  if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_blocks(const uint32_t* in, unsigned long long* out, unsigned long long* block_sums, uint64_t n) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long tot;
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * 4;
  unsigned long long v[4], s = 0;
  for (int i = 0; i < 4; ++i) {
    v[i] = base + i < n ? (unsigned long long)in[base + i] : 0ull;
    s += v[i];
  }
  unsigned long long run = block_exclusive_scan(s, warp_tot, &tot);
  for (int i = 0; i < 4; ++i) {
    run += v[i];
    if (base + i < n) out[base + i] = run;
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(unsigned long long* block_sums, uint64_t nblocks) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long tot;
  unsigned long long carry = 0;
  for (uint64_t b0 = 0; b0 < nblocks; b0 += blockDim.x) {
    const uint64_t b = b0 + threadIdx.x;
    const unsigned long long v = b < nblocks ? block_sums[b] : 0ull;
    const unsigned long long ex = block_exclusive_scan(v, warp_tot, &tot);
    if (b < nblocks) block_sums[b] = carry + ex + v;  // inclusive
    carry += tot;
  }
}

__global__ void k_scan_add(unsigned long long* out, const unsigned long long* block_sums, uint64_t n) {
  if (blockIdx.x == 0) return;
  const unsigned long long add = block_sums[blockIdx.x - 1];
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock;
  for (uint64_t i = base + threadIdx.x; i < base + kScanBlock && i < n; i += blockDim.x) out[i] += add;
}

// Systematic sampling of the next cycle's N sources from the M sites banked by this cycle's N
// histories: history h of the next cycle takes site floor((h + u0) M / N) (sites ordered by
// producing history, then production order; u0 = the cycle's combing offset).  One thread per
// producing history writes each of its sites to the histories that pick it: the candidates around
// the inverse of that formula, each checked with the formula itself in FP64, so that every new
// history gets exactly the site the formula gives it.
template <int LANES>
__global__ void k_comb(const uint32_t* counts, const unsigned long long* scan, const uint4* sites, uint32_t nmax,
                       uint64_t N, uint64_t seed, uint32_t next_cycle, uint4* src) {
  const unsigned long long M = scan[N - 1];
  if (M == 0) return;
  const double u0 = draw<double>(seed, 0xFFFFFFFFu, next_cycle, kSourceEvent, 4).a;
  const double dN = (double)N, dM = (double)M;
  for (uint64_t hp = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; hp < N; hp += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t n = counts[hp];
    const unsigned long long o = scan[hp] - n;
    for (uint32_t j = 0; j < n; ++j) {
      const unsigned long long g = o + j;
      long long lo = (long long)ceil((double)g * dN / dM - u0) - 1, hi = (long long)ceil((double)(g + 1) * dN / dM - u0);
      if (lo < 0) lo = 0;
      if (hi > (long long)N - 1) hi = (long long)N - 1;
      for (long long h = lo; h <= hi; ++h) {
        unsigned long long idx = (unsigned long long)floor(((double)h + u0) * dM / dN);
        if (idx >= M) idx = M - 1;
        if (idx != g) continue;
        for (int l = 0; l < LANES; ++l) src[(uint64_t)h * LANES + l] = sites[(hp * nmax + j) * LANES + l];
      }
    }
  }
}

cudaError_t launch_scan_sites(const uint32_t* counts, unsigned long long* scan, unsigned long long* block_sums, uint64_t n,
                              cudaStream_t s) {
  const uint64_t nblocks = (n + kScanBlock - 1) / kScanBlock;
  k_scan_blocks<<<(unsigned)nblocks, 256, 0, s>>>(counts, scan, block_sums, n);
  k_scan_sums<<<1, 1024, 0, s>>>(block_sums, nblocks);
  k_scan_add<<<(unsigned)nblocks, 256, 0, s>>>(scan, block_sums, n);
  return cudaGetLastError();
}

cudaError_t launch_comb(const uint32_t* counts, const unsigned long long* scan, const uint4* sites, uint32_t nmax,
                        uint64_t n, uint64_t seed, uint32_t next_cycle, uint4* src, int lanes, cudaStream_t s) {
  uint64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (lanes == 2) k_comb<2><<<(unsigned)g, 256, 0, s>>>(counts, scan, sites, nmax, n, seed, next_cycle, src);
  else k_comb<1><<<(unsigned)g, 256, 0, s>>>(counts, scan, sites, nmax, n, seed, next_cycle, src);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ population control
// Exact total weight of every batch's banked particles: sum of llrint(w 2^40) per batch.
template <typename R>
__global__ void k_pc_weight(const RunParams P, const unsigned long long* pc_n, long long* wq) {
  const unsigned long long n = *pc_n < P.cap_c ? *pc_n : P.cap_c;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    Part<R> p;
    bank_load(p, P.C, i);
    atomicAdd(reinterpret_cast<unsigned long long*>(wq + (p.elem >> 16)),
              (unsigned long long)__double2ll_rn(__dmul_rn(p.w, 1099511627776.0)));
  }
}

// Splitting-roulette of the banked particles to N_b per batch: floor(w / w_t + xi) copies of weight
// w_t = W_b 2^-40 / N_b at the census time, appended to the birth bank that the next interval's
// launch starts from (count in *out_n); FP64 arithmetic rounded as the oracle rounds it.
template <typename R>
__global__ void k_pc_split(const RunParams P, const unsigned long long* pc_n, const long long* wq, const RunParams Q,
                           unsigned long long* out_n, unsigned long long* copies, int* status) {
  const unsigned long long n = *pc_n < P.cap_c ? *pc_n : P.cap_c;
  const uint64_t N = P.n_hist, nb = (uint64_t)P.n_batches;
  unsigned local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    Part<R> p;
    bank_load(p, P.C, i);
    const uint64_t b = p.elem >> 16;
    const uint64_t Nb = ((b + 1) * N + nb - 1) / nb - (b * N + nb - 1) / nb;
    if (wq[b] <= 0 || Nb == 0) continue;
    const double wt = __ddiv_rn(__ddiv_rn((double)wq[b], 1099511627776.0), (double)Nb);
    const double xi = draw<double>(P.seed, p.tlo, p.thi, p.k, 1).a;
    const int c = (int)floor(__dadd_rn(__ddiv_rn(p.w, wt), xi));
    for (int j = 0; j < c; ++j) {
      Part<R> q = p;
      const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)j, 0x40000000u);
      q.tlo = t.x;
      q.thi = t.y;
      q.k = 0;
      q.w = wt;
      q.pk = pk_set_pending(q.pk, PEND_NONE, 0, 1, 0);
      set_census_time(q, P);
      const unsigned long long k = atomicAdd(out_n, 1ull);
      if (k < Q.cap_b) bank_store(q, Q.B[0], k);
      else atomicCAS(status, 0, MC_ERR_BANK_FULL);
    }
    local += (unsigned)c;
  }
  if (local) atomicAdd(copies, (unsigned long long)local);
}

// P: the parameters of the launch that banked the particles; Q: those of the next launch (its
// birth bank B[0] receives the copies)
template <typename R>
cudaError_t launch_pc(const RunParams& P, const RunParams& Q, const unsigned long long* pc_n, long long* wq,
                      unsigned long long* out_n, unsigned long long* copies, int* status, bool split, cudaStream_t s) {
  const unsigned g = 152 * 8;
  if (!split) k_pc_weight<R><<<g, 256, 0, s>>>(P, pc_n, wq);
  else k_pc_split<R><<<g, 256, 0, s>>>(P, pc_n, wq, Q, out_n, copies, status);
  return cudaGetLastError();
}
template cudaError_t launch_pc<float>(const RunParams&, const RunParams&, const unsigned long long*, long long*,
                                      unsigned long long*, unsigned long long*, int*, bool, cudaStream_t);
template cudaError_t launch_pc<double>(const RunParams&, const RunParams&, const unsigned long long*, long long*,
                                       unsigned long long*, unsigned long long*, int*, bool, cudaStream_t);

// L2 atomic throughput probe: 64-bit reductions (adds whose old value is not returned, as the
// tally scoring issues them) to pseudo-random slots of an array of `span` elements, `iters` per
// thread.
__global__ void k_atomic_probe(unsigned long long* a, unsigned long long span, int iters, unsigned salt) {
  unsigned long long x = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * 2654435761ull + salt;
  for (int i = 0; i < iters; ++i) {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    red_add(a + ((x >> 20) % span), 1ull);
  }
}

cudaError_t launch_atomic_probe(unsigned long long* a, unsigned long long span, int grid, int iters, unsigned salt,
                                cudaStream_t s) {
  k_atomic_probe<<<grid, 256, 0, s>>>(a, span, iters, salt);
  return cudaGetLastError();
}

// Instruction throughput probe: every thread runs four independent chains of `iters` operations of
// one kind (op 0 FP32 FMA, 1 FP64 add, 2 32-bit umulhi, 3 int -> float, 4 float -> int64, 5 __logf),
// so that throughput, not latency, bounds it; block 0 records the SM clock ticks and the global
// nanoseconds it took (the clock rate seen by the kernel).  The result feeds a sink so that nothing
// is optimised away.
template <int OP>
__global__ void k_op_probe(int iters, unsigned long long* sink, unsigned long long* clk) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const long long c0 = clock64();
  unsigned long long g0 = 0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  unsigned long long acc = 0;
  if (OP == 0) {
    float a[4] = {1.0f + t * 1e-9f, 1.1f, 1.2f, 1.3f};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = __fmaf_rn(a[c], 0.999999f, 1e-7f);
    acc = __float_as_uint(a[0] + a[1] + a[2] + a[3]);
  } else if (OP == 1) {
    double a[4] = {1.0 + t * 1e-12, 1.1, 1.2, 1.3};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = __dadd_rn(a[c], 1e-9);
    acc = (unsigned long long)__double_as_longlong(a[0] + a[1] + a[2] + a[3]);
  } else if (OP == 2) {
    unsigned a[4] = {t | 1u, 3u, 5u, 7u};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = __umulhi(a[c], 0x9E3779B9u) + 0x6A09E667u;
    acc = a[0] ^ a[1] ^ a[2] ^ a[3];
  } else if (OP == 3) {
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int b[4] = {(int)t, 2, 3, 4};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        a[c] = __int2float_rn(b[c]);
        b[c] = __float_as_int(a[c]) >> 3;
      }
    acc = __float_as_uint(a[0] + a[1] + a[2] + a[3]);
  } else if (OP == 4) {
    float a[4] = {1.5f + t, 2.5f, 3.5f, 4.5f};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = __int_as_float((int)(__float2ll_rn(a[c]) | 0x3F800000ll));
    acc = __float_as_uint(a[0] + a[1] + a[2] + a[3]);
  } else {
    float a[4] = {1.5f + t * 1e-7f, 2.5f, 3.5f, 4.5f};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = __logf(a[c]) + 2.0f;
    acc = __float_as_uint(a[0] + a[1] + a[2] + a[3]);
  }
  if (acc == 0x5EED5EEDull) *sink = acc;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long g1 = 0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    clk[0] = (unsigned long long)(clock64() - c0);
    clk[1] = g1 - g0;
  }
}

cudaError_t launch_op_probe(int op, int grid, int iters, unsigned long long* sink, unsigned long long* clk,
                            cudaStream_t s) {
  switch (op) {
    case 0: k_op_probe<0><<<grid, 256, 0, s>>>(iters, sink, clk); break;
    case 1: k_op_probe<1><<<grid, 256, 0, s>>>(iters, sink, clk); break;
    case 2: k_op_probe<2><<<grid, 256, 0, s>>>(iters, sink, clk); break;
    case 3: k_op_probe<3><<<grid, 256, 0, s>>>(iters, sink, clk); break;
    case 4: k_op_probe<4><<<grid, 256, 0, s>>>(iters, sink, clk); break;
    default: k_op_probe<5><<<grid, 256, 0, s>>>(iters, sink, clk); break;
  }
  return cudaGetLastError();
}

__global__ void k_philox(uint64_t seed, const uint4* ctr, uint4* out, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr[i]);
}

// ------------------------------------------------------------------------------------------ launchers
// Two register budgets of the same kernel: 3 CTAs of 256 threads per SM (80 registers) or 2 CTAs
// (128 registers, no spills); `wide` selects the second.  `range` selects the build with the range
// walk of the scoring (tallies whose time axis is much finer than their mesh), `seg` the build that
// scores segments apart from their flights, `mode` the launch of a split run (1: event-based part,
// 2: history-style tail; only the segment builds are split).
template <typename R>
static const void* transport_fn(bool wide, bool range, bool seg, int mode = 0) {
  if constexpr (sizeof(R) == 8) {
    return range ? (const void*)k_transport<R, 2, true, false, 0> : (const void*)k_transport<R, 2, false, false, 0>;
  } else {
    if (seg) {
      if (mode == 1) return wide ? (const void*)k_transport<R, 2, false, true, 1> : (const void*)k_transport<R, 3, false, true, 1>;
      if (mode == 2) return wide ? (const void*)k_transport<R, 2, false, true, 2> : (const void*)k_transport<R, 3, false, true, 2>;
      return wide ? (const void*)k_transport<R, 2, false, true, 0> : (const void*)k_transport<R, 3, false, true, 0>;
    }
    if (range) return wide ? (const void*)k_transport<R, 2, true, false, 0> : (const void*)k_transport<R, 3, true, false, 0>;
    return wide ? (const void*)k_transport<R, 2, false, false, 0> : (const void*)k_transport<R, 3, false, false, 0>;
  }
}

// A run with per-warp stacks (P.WS) of a segment build is split into the event-based launch and
// the history-style tail launch, back to back on the stream; any other run is one launch.
template <typename R>
cudaError_t launch_transport(const RunParams& P, int grid, int block, size_t smem, cudaStream_t s, bool wide,
                             bool range) {
  void* args[] = {const_cast<RunParams*>(&P)};
  const bool seg = P.seg != nullptr;
  if (sizeof(R) == 4 && seg && P.WS[0] != nullptr) {
    cudaError_t e = cudaLaunchCooperativeKernel(transport_fn<R>(wide, range, true, 1), grid, block, args, smem, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(transport_fn<R>(wide, range, true, 2), grid, block, args, smem, s);
  }
  return cudaLaunchCooperativeKernel(transport_fn<R>(wide, range, seg), grid, block, args, smem, s);
}

template <typename R>
cudaError_t transport_occupancy(int block, size_t smem, int* per_sm, bool wide, bool range, bool seg) {
  // every mode of a build has the same register budget; the split launches need the grid to fit
  // for each of them, so the least occupancy of the modes is taken
  const int n_modes = (sizeof(R) == 4 && seg) ? 3 : 1;
  int best = 1 << 30;
  for (int mode = 0; mode < n_modes; ++mode) {
    const void* f = transport_fn<R>(wide, range, seg, mode);
    // opt in for the exact size: the default limit (48 KB less the kernel's static shared memory)
    // can be exceeded by a dynamic size just under 48 KB
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem);
    if (e != cudaSuccess) return e;
    best = n < best ? n : best;
  }
  *per_sm = best;
  return cudaSuccess;
}

template cudaError_t launch_transport<float>(const RunParams&, int, int, size_t, cudaStream_t, bool, bool);
template cudaError_t launch_transport<double>(const RunParams&, int, int, size_t, cudaStream_t, bool, bool);
template cudaError_t transport_occupancy<float>(int, size_t, int*, bool, bool, bool);
template cudaError_t transport_occupancy<double>(int, size_t, int*, bool, bool, bool);

cudaError_t launch_reconstruct(void* tally, const char* blob64, uint64_t rows, uint64_t row, int nb, int stripes,
                               int fp64, cudaStream_t s) {
  const uint64_t warps = (uint64_t)nb * rows;
  uint64_t g = (warps + 7) / 8;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  k_reconstruct<<<(unsigned)g, 256, 0, s>>>(tally, blob64, rows, row, nb, stripes, fp64);
  return cudaGetLastError();
}

cudaError_t launch_batch_stats(const void* tally, int fp64, uint64_t bins, uint64_t row, int nb, int stripes,
                               uint64_t n_hist, void* out, cudaStream_t s) {
  const int block = 256;
  uint64_t g = (bins + block - 1) / block;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  if (fp64) {
    double* o = reinterpret_cast<double*>(out);
    k_batch_stats_fp64<<<(unsigned)g, block, 0, s>>>(reinterpret_cast<const double*>(tally), bins, row, nb, stripes,
                                                     (double)nb / (double)n_hist, o, o + bins, o + 2 * bins);
  } else {
    char* o = reinterpret_cast<char*>(out);
    k_batch_stats_fixed<<<(unsigned)g, block, 0, s>>>(
        reinterpret_cast<const long long*>(tally), bins, row, nb, stripes, reinterpret_cast<long long*>(o),
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
