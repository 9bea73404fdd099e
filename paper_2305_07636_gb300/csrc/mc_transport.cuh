// The persistent transport kernel k_transport (sm_103a): one template, instantiated per build
// family in its own translation unit (mc_transport.cu: the plain walk and FP64 tracking;
// mc_transport_seg.cu: segments scored apart from their flights; mc_transport_range.cu: the range
// walk), so that the families compile in parallel.
//
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
// transports.  Once every history is sourced and few particles remain, the iterations run
// history-style (particles stay in the queue until they die): in one launch, one grid barrier per
// generation of secondaries instead of one per event; in the tail launch of a split run (below),
// one history-style iteration in all.  Iterations are separated by a grid barrier whose wait
// is bounded; the device status word reports overflow, lost particles and watchdog expiry instead
// of hanging or trapping.
#pragma once
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
// [per-warp tally staging, with warp-aggregated tally adds only: warps x kStage x 12 B][SEG:
// per-warp segment regions: warps x kSegLanes x kSegCap x 16 B]
//
// MODE 0 runs the whole transport in one launch: event-based iterations, then history-style ones
// once the work left is below the drain threshold.  A split run launches MODE 1, which stops where
// MODE 0 would turn history-style (and records that iteration in ctl->tail_it), then MODE 2, which
// runs the history-style iterations from there with per-warp stacks of secondaries: a warp flies
// its particles' secondaries before it claims more work, so one history-style iteration ends the
// run instead of one per generation of secondaries, and the event-based launch carries none of
// the tail's code.
//
// MINB sets the register budget: 2 or 3 CTAs of 256 threads per SM (128 or 80 registers), or 5 CTAs
// of 128 threads (96 registers, the segment builds at 128 threads per CTA).
template <typename R, int MINB, bool RANGE, bool SEG, int MODE>
__global__ void __launch_bounds__(MINB == 5 ? 128 : 256, MINB) k_transport(RunParams P) {
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
  // per-warp tally staging buffers follow the queues: values (8 B) then slots (4 B); only runs
  // that warp-aggregate their tally adds stage scores, the others have no staging region
  const unsigned kst = P.aggregate ? kStage : 0u;
  char* stage_base = smem + P.blob_bytes + (size_t)nwarp * Lanes<R>::N * kWarpQ * 16;
  const Stage stage{reinterpret_cast<uint32_t*>(stage_base + (size_t)nwarp * kst * 8) + warp * kst,
                    reinterpret_cast<unsigned long long*>(stage_base) + warp * kst};
  // SEG: the warp's region of segments waiting to be scored (ns of them, warp-uniform), after the
  // staging buffers
  uint4* const sq = SEG ? reinterpret_cast<uint4*>(stage_base + (size_t)nwarp * kst * 12) + warp * (kSegLanes * kSegCap)
                        : nullptr;
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

// the kernel of one build family: `wide` the 128-register build (else 80, or for the segment
// builds at 128 threads per CTA 96), `mode` 0 for one launch, 1 / 2 for the event-based part and
// the tail of a split run
const void* transport_fn_seg(bool wide, int block, int mode);  // FP32, segments scored apart
const void* transport_fn_range(bool wide, int mode);           // FP32, range walk

}  // namespace mcgb
