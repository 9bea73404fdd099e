// Batched persistent transport (sm_103a): many independent problems of uneven size in one launch.
//
// The histories of every problem are cut into work units of a few dozen to a few hundred
// consecutive histories.  Every warp of a persistent grid claims units with one atomic, stages the
// unit's problem (its run parameters and its table blob) in its own slice of shared memory when
// the problem changes, and carries the unit's particles to completion history-style through a
// per-warp flight queue: all 32 lanes fly, survivors handle their next event and fly again.
// Secondaries and weight-window copies go to a warp-private stack in device memory (depth first,
// so it stays shallow for subcritical problems) and are popped back into the queue before new
// sources.  A warp claims the next unit as soon as its queue runs low, so lanes stay full across
// units of one problem; a unit of another problem waits until the current problem's particles are
// finished.  No warp ever waits for another, so the launch needs neither a grid barrier nor a
// cooperative launch, and uneven problems balance at the granularity of one unit.
//
// Every particle draws the same random numbers and takes the same steps as in the single-problem
// kernel (problem i uses the seed seed + i), so fixed-point tallies equal those of separate runs.
// The launch (clear, transport, statistics) is captured once per launch shape into a CUDA graph;
// each call uploads the problem list and replays the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <vector>

// this kernel's weight-window test out of line (see weight_window), its segment walks started by
// bisection (see bin_find)
#define MCGB_WW_OUT_OF_LINE 1
#define MCGB_BIN_GUESS 0
#include "mc_events.cuh"
#include "mc_host.h"

namespace mcgb {

// one problem of a batch, in claim order (geometry kind, then ascending history count)
struct __align__(16) BatchItem {
  RunParams P;          // the problem's run parameters; births use the claiming warp's stack
  void* stats;          // [3][bins] statistics output (the problem's own buffer)
  uint64_t bins;        // bins of one batch tally
  uint64_t unit_first;  // index of the problem's first work unit
  uint64_t n_units;     // work units of the problem
  int caller_index;     // position in the caller's list
  int pad;
  const char* blob64;   // the problem's FP64 tables on the device (range-walk reconstruction)
  uint64_t range_rows;  // its (tally, cell, group) rows scored by the range walk
};

struct BatchHeader {
  unsigned long long next_unit;  // claim counter (cleared by the graph)
  unsigned long long t0;         // launch start: earliest %globaltimer read by a warp
  unsigned long long n_units;    // total work units
  unsigned long long stack_cap;  // particles per warp stack
  unsigned int n_items, unit;    // problems; histories per unit
  int tally_fp64, pad;
};

constexpr size_t kParamBytes = (sizeof(RunParams) + 15) & ~size_t(15);
static_assert(sizeof(BatchItem) >= kParamBytes && sizeof(BatchItem) % 16 == 0, "BatchItem layout");

// shared memory of one warp: [run parameters][table blob][flight queue][stage values][stage
// slots][counters][stack count]
template <typename R>
__host__ __device__ constexpr size_t batch_warp_bytes(size_t slot_bytes) {
  return kParamBytes + slot_bytes + (size_t)Lanes<R>::N * kWarpQ * 16 + (size_t)kStage * 12 +
         sizeof(BlockCounters) + 16;
}

// the item that owns work unit u (items sorted by unit_first)
__device__ __forceinline__ int item_of_unit(const BatchItem* items, int n, unsigned long long u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&items[mid].unit_first) <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// copies `bytes` (a multiple of 16) from global to shared memory with the 32 lanes of a warp
__device__ __forceinline__ void warp_copy16(void* dst, const void* src, size_t bytes, int lane) {
  uint4* d = reinterpret_cast<uint4*>(dst);
  const uint4* s = reinterpret_cast<const uint4*>(src);
  for (size_t i = lane; i < bytes / 16; i += 32) d[i] = __ldg(s + i);
}

// SEG (FP32, plain-walk tallies only): flown segments are scored apart from their flights, 32 at a
// time, from the warp's segment region in `segs` (score_segments); the region is emptied before
// the warp turns to another problem, whose tables and tallies its records do not address.
template <typename R, int MINB, bool RANGE, bool SEG>
__global__ void __launch_bounds__(256, MINB)
    k_transport_batch(BatchHeader* bh, const BatchItem* items, unsigned long long* t_done, uint4* stacks,
                      int slot_bytes, uint4* segs) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  char* wbase = smem + (size_t)warp * batch_warp_bytes<R>((size_t)slot_bytes);
  RunParams* wP = reinterpret_cast<RunParams*>(wbase);
  char* blob = wbase + kParamBytes;
  uint4* wq = reinterpret_cast<uint4*>(blob + slot_bytes);
  char* st = reinterpret_cast<char*>(wq + Lanes<R>::N * kWarpQ);
  const Stage stage{reinterpret_cast<uint32_t*>(st + kStage * 8), reinterpret_cast<unsigned long long*>(st)};
  BlockCounters* bc = reinterpret_cast<BlockCounters*>(st + kStage * 12);
  unsigned long long* sc = reinterpret_cast<unsigned long long*>(st + kStage * 12 + sizeof(BlockCounters));
  const unsigned lt = lanemask_lt();
  const uint64_t gw = (uint64_t)blockIdx.x * nwarp + warp, nwt = (uint64_t)gridDim.x * nwarp;
  uint4* const sq = SEG ? segs + gw * (kSegLanes * kSegCap) : nullptr;
  unsigned ns = 0;
  const uint64_t cap = bh->stack_cap;
  const unsigned long long n_units = bh->n_units;
  const uint64_t unit = bh->unit;
  const int n_items = (int)bh->n_items;
  if (lane == 0) atomicMin(&bh->t0, globaltimer());
  if (lane < MC_NCOUNTERS) bc->c[lane] = 0u;
  if (lane == 0) {
    *sc = 0ull;
    bc->split_ctr = nullptr;
    bc->local = 0u;
    bc->hold_at = cap / 2;  // weight-window splits are held while the warp's stack is half full
  }

  unsigned long long u0 = 0;
  if (lane == 0) u0 = atomicAdd(&bh->next_unit, 1ull);
  u0 = __shfl_sync(0xFFFFFFFFu, u0, 0);
  unsigned qn = 0;
  while (u0 < n_units) {
    // ---- stage the problem of unit u0 in this warp's slice of shared memory
    const int j = item_of_unit(items, n_items, u0);
    __syncwarp();
    warp_copy16(wP, &items[j].P, kParamBytes, lane);  // items are 16-byte aligned and longer than kParamBytes
    __syncwarp();
    if (lane < Lanes<R>::N) wP->B[0][lane] = stacks + ((uint64_t)lane * nwt + gw) * cap;
    if (lane == 0) wP->cap_b = cap;
    warp_copy16(blob, wP->blob, (size_t)wP->blob_bytes, lane);
    __syncwarp();
    const RunParams& P = *wP;
    const Tab<R> T(blob);
    const uint64_t row = P.row;  // tally elements per batch: bins, then difference slots
    const uint64_t ufirst = __ldg(&items[j].unit_first);
    unsigned scored = 0;
    uint64_t hn = 0, he = 0;  // histories of the claimed units still to start
    // claims unit u of this problem: its history range, unless the problem has failed already
    auto begin_unit = [&](unsigned long long u) {
      hn = (u - ufirst) * unit;
      he = hn + unit < P.n_hist ? hn + unit : P.n_hist;
      int stt = 0;
      if (lane == 0) {
        stt = ld_volatile_int(&P.ctl->status);
        atomicAdd(&P.ctl->iterations, 1ull);
        atomicMin(&P.ctl->t_start, globaltimer());
      }
      if (__shfl_sync(0xFFFFFFFFu, stt, 0) != 0) hn = he;
    };
    begin_unit(u0);
    unsigned long long next = n_units;  // first claimed unit of another problem
    bool can_claim = true;
    while (true) {
      // (A) refill the queue to at least 32: secondaries first (depth first), then new sources,
      // then the next unit of this problem
      while (qn < 32u) {
        __syncwarp();
        unsigned long long ns = *reinterpret_cast<volatile unsigned long long*>(sc);
        ns = ns < cap ? ns : cap;  // pushes past the capacity were dropped with MC_ERR_BANK_FULL
        Part<R> p;
        bool ready = false;
        if (ns > 0) {
          const unsigned n = ns < 32ull ? (unsigned)ns : 32u;
          if ((unsigned)lane < n) {
            bank_load(p, wP->B[0], ns - n + lane);
            ready = true;
          }
          __syncwarp();
          if (lane == 0) *sc = ns - n;
        } else if (hn < he) {
          const uint64_t n = he - hn < 32 ? he - hn : 32;
          if ((uint64_t)lane < n) {
            bump(bc, MC_C_SOURCE);
            ready = make_source(P, T, P.h_first + hn + lane, p);
            if (!ready) {
              bump(bc, MC_C_LOST);
              set_status(P, MC_ERR_LOST);
            }
          }
          hn += n;
        } else if (can_claim) {
          unsigned long long u = 0;
          if (lane == 0) u = atomicAdd(&bh->next_unit, 1ull);
          u = __shfl_sync(0xFFFFFFFFu, u, 0);
          if (u >= n_units) {
            can_claim = false;
          } else if (u < ufirst + __ldg(&items[j].n_units)) {
            begin_unit(u);
          } else {
            next = u;
            can_claim = false;
          }
          continue;
        } else {
          break;
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, ready);
        if (ready) queue_store(p, wq, kWarpQ, qn + __popc(m & lt));
        qn += __popc(m);
      }
      __syncwarp();
      if constexpr (SEG) {
        if (ns >= 32u || (qn == 0u && ns > 0u)) score_segments(T, P, sq, ns, qn == 0u, 0, stage, scored);
      }
      if (qn == 0u) break;
      // (B) fly up to 32 queued particles; survivors handle their next event and queue again
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
      const bool flies = have && flight_plan(P, T, p, bc, l, pend, hit);
      if constexpr (SEG) {
        const unsigned msc = __ballot_sync(0xFFFFFFFFu, flies);
        if (flies) seg_push_flight(sq, ns + __popc(msc & lt), p, l);
        ns += __popc(msc);
      } else {
        score_segment_warp<R, RANGE>(T, P, p, l, (uint64_t)(p.elem >> 16) * row, flies, stage, scored);
      }
      if (flies) {
        bool alive = flight_finish(P, T, p, bc, l, pend, hit);
        if (alive && p.k + 1 >= P.max_iter) {
          set_status(P, MC_ERR_TIMEOUT);  // the per-particle event budget
          alive = false;
        }
        if (alive) again = handle_pending(P, T, p, wP->B[0], sc, bc, row, 0);
      }
      const unsigned m = __ballot_sync(0xFFFFFFFFu, again);
      if (again) queue_store(p, wq, kWarpQ, qn + __popc(m & lt));
      qn += __popc(m);
    }
    // ---- the warp's share of this problem is done: counters and completion time
    __syncwarp();
    if (lane == 0 && scored) atomicAdd(&bc->c[MC_C_SCORES], scored);
    __syncwarp();
    if (lane < MC_NCOUNTERS) {
      const unsigned v = bc->c[lane];
      if (v) atomicAdd(&P.ctl->counters[lane], (unsigned long long)v);
      bc->c[lane] = 0u;
    }
    if (lane == 0) {
      const unsigned long long now = globaltimer();
      atomicMax(&P.ctl->t_end, now);
      atomicMax(&t_done[j], now);
    }
    u0 = next;
  }
}

// Clears what a batched launch accumulates: each problem's batch tallies and control block
// (blockIdx.x = problem), the per-problem completion times and the claim counter.
__global__ void k_batch_clear(BatchHeader* bh, const BatchItem* items, unsigned long long* t_done) {
  const BatchItem& it = items[blockIdx.x];
  const uint64_t words = (uint64_t)it.P.n_batches * it.P.row;
  long long* t = reinterpret_cast<long long*>(it.P.tally);
  for (uint64_t i = (uint64_t)blockIdx.y * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.y * blockDim.x)
    t[i] = 0;
  if (blockIdx.y == 0) {
    unsigned long long* c = reinterpret_cast<unsigned long long*>(it.P.ctl);
    for (unsigned i = threadIdx.x; i < sizeof(Ctl) / 8; i += blockDim.x) c[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
      it.P.ctl->t_start = ~0ull;
      t_done[blockIdx.x] = 0ull;
      if (blockIdx.x == 0) {
        bh->next_unit = 0ull;
        bh->t0 = ~0ull;
      }
    }
  }
}

// Range-walk reconstruction of every problem that has range rows (blockIdx.x = problem,
// blockIdx.y strides over its (batch, row) pairs, one warp each).
__global__ void k_batch_reconstruct_multi(const BatchHeader* bh, const BatchItem* items) {
  const BatchItem& it = items[blockIdx.x];
  const uint64_t rows = it.range_rows;
  if (rows == 0) return;
  const int nb = it.P.n_batches;
  const uint64_t warps = (uint64_t)gridDim.y * (blockDim.x >> 5);
  for (uint64_t wi = (uint64_t)blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < (uint64_t)nb * rows;
       wi += warps)
    reconstruct_warp(it.P.tally, it.blob64, it.P.row, nb, 1, bh->tally_fp64, (int)(wi / rows), wi % rows);
}

// Batch statistics of every problem (blockIdx.x = problem, blockIdx.y strides over its bins).
__global__ void k_batch_stats_multi(const BatchHeader* bh, const BatchItem* items) {
  const BatchItem& it = items[blockIdx.x];
  const uint64_t bins = it.bins;
  const int nb = it.P.n_batches;
  for (uint64_t b = (uint64_t)blockIdx.y * blockDim.x + threadIdx.x; b < bins; b += (uint64_t)gridDim.y * blockDim.x) {
    if (bh->tally_fp64) {
      double* o = reinterpret_cast<double*>(it.stats);
      stats_bin_fp64(reinterpret_cast<const double*>(it.P.tally), it.P.row, nb, 1, (double)nb / (double)it.P.n_hist, b,
                     o[b], o[bins + b], o[2 * bins + b]);
    } else {
      char* o = reinterpret_cast<char*>(it.stats);
      stats_bin_fixed(reinterpret_cast<const long long*>(it.P.tally), it.P.row, nb, 1, b,
                      reinterpret_cast<long long*>(o)[b], reinterpret_cast<unsigned long long*>(o + 8 * bins)[b],
                      reinterpret_cast<unsigned long long*>(o + 16 * bins)[b]);
    }
  }
}

// the two register budgets of the batched kernel (FP64 tracking has only the wide one), each with
// and without the range walk of the scoring
template <typename R>
static const void* batch_fn(bool wide, bool range, bool seg) {
  if constexpr (sizeof(R) == 8) {
    return range ? (const void*)k_transport_batch<R, 2, true, false> : (const void*)k_transport_batch<R, 2, false, false>;
  } else {
    if (seg)
      return wide ? (const void*)k_transport_batch<R, 2, false, true> : (const void*)k_transport_batch<R, 3, false, true>;
    if (range)
      return wide ? (const void*)k_transport_batch<R, 2, true, false> : (const void*)k_transport_batch<R, 3, true, false>;
    return wide ? (const void*)k_transport_batch<R, 2, false, false> : (const void*)k_transport_batch<R, 3, false, false>;
  }
}

}  // namespace mcgb

// ------------------------------------------------------------------------------------------ host
namespace mcgb {
namespace {

struct BatchConfig {
  int block, wide, unit;
};

// Everything one launch shape needs on the device, and the graph that replays it: the problem
// list and header (uploaded by every call from pinned staging), per-problem completion times,
// and the warp stacks.
struct BatchPlan {
  int dev = 0, n = 0, block = 0, wide = 0, fp64 = 0, range = 0, seg = 0, grid = 0;
  size_t slot_bytes = 0, smem = 0;
  uint64_t stack_cap = 0;
  DevBuf d_items, d_head, d_tdone, d_stacks, d_segs;
  BatchItem* h_items = nullptr;
  BatchHeader* h_head = nullptr;
  unsigned long long* h_tdone = nullptr;
  cudaEvent_t uploaded = nullptr;  // recorded after the last upload from the staging buffers
  cudaEvent_t done = nullptr;      // recorded after the last replay (orders calls on other streams)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (uploaded) cudaEventDestroy(uploaded);
    if (done) cudaEventDestroy(done);
    if (h_items) cudaFreeHost(h_items);
    if (h_head) cudaFreeHost(h_head);
    if (h_tdone) cudaFreeHost(h_tdone);
    d_items.release();
    d_head.release();
    d_tdone.release();
    d_stacks.release();
    d_segs.release();
  }
};

std::mutex g_batch_mu;
std::vector<std::unique_ptr<BatchPlan>> g_plans;
uint64_t g_plan_clock = 0;
std::map<uint64_t, BatchConfig> g_tuned;
constexpr size_t kMaxPlans = 4;
constexpr uint64_t kDefaultStack = 2048;

template <typename R>
cudaError_t batch_occupancy(int block, size_t smem, bool wide, bool range, bool seg, int* per_sm) {
  const void* f = batch_fn<R>(wide, range, seg);
  // opt in for the exact size: the default limit (48 KB less the kernel's static shared memory)
  // can be exceeded by a dynamic size just under 48 KB
  {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, f, block, smem);
}

// Captures clear -> transport -> statistics on the plan's own stream (a graph may be launched
// into any stream, including the legacy default one, which cannot be captured).
int capture(BatchPlan* pl) {
  BatchHeader* bh = (BatchHeader*)pl->d_head.ptr;
  const BatchItem* items = (const BatchItem*)pl->d_items.ptr;
  unsigned long long* tdone = (unsigned long long*)pl->d_tdone.ptr;
  uint4* stacks = (uint4*)pl->d_stacks.ptr;
  uint4* segs = (uint4*)pl->d_segs.ptr;
  int slot = (int)pl->slot_bytes;
  const void* f = pl->fp64 ? batch_fn<double>(pl->wide, pl->range, false)
                           : batch_fn<float>(pl->wide, pl->range, pl->seg != 0);
  void* args[] = {&bh, &items, &tdone, &stacks, &slot, &segs};
  CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
  k_batch_clear<<<dim3((unsigned)pl->n, 16), 256, 0, pl->cap_stream>>>(bh, items, tdone);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaLaunchKernel(f, pl->grid, pl->block, args, pl->smem, pl->cap_stream);
  if (e == cudaSuccess && pl->range) {
    k_batch_reconstruct_multi<<<dim3((unsigned)pl->n, 4), 256, 0, pl->cap_stream>>>(bh, items);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_batch_stats_multi<<<dim3((unsigned)pl->n, 8), 256, 0, pl->cap_stream>>>(bh, items);
    e = cudaGetLastError();
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(pl->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "batched launch capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&pl->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return MC_OK;
}

// The plan of a launch shape, created (and its graph captured) on first use.  Caller holds
// g_batch_mu.
int get_plan(int dev, int n, const BatchConfig& c, int fp64, int range, int seg, size_t slot, uint64_t stack_cap,
             BatchPlan** out) {
  for (auto& pl : g_plans)
    if (pl->dev == dev && pl->n == n && pl->block == c.block && pl->wide == c.wide && pl->fp64 == fp64 &&
        pl->range == range && pl->seg == seg && pl->slot_bytes == slot && pl->stack_cap == stack_cap) {
      pl->last_use = ++g_plan_clock;
      *out = pl.get();
      return MC_OK;
    }
  if (g_plans.size() >= kMaxPlans) {
    // the least recently used plan may still be running on some stream
    auto it = std::min_element(g_plans.begin(), g_plans.end(),
                               [](const std::unique_ptr<BatchPlan>& a, const std::unique_ptr<BatchPlan>& b) {
                                 return a->last_use < b->last_use;
                               });
    CK(cudaDeviceSynchronize());
    g_plans.erase(it);
  }
  std::unique_ptr<BatchPlan> pl(new BatchPlan);
  pl->dev = dev;
  pl->n = n;
  pl->block = c.block;
  pl->wide = c.wide;
  pl->fp64 = fp64;
  pl->range = range;
  pl->seg = seg;
  pl->slot_bytes = slot;
  pl->stack_cap = stack_cap;
  const size_t wb = fp64 ? batch_warp_bytes<double>(slot) : batch_warp_bytes<float>(slot);
  pl->smem = (size_t)(c.block / 32) * wb;
  int rc0 = check_shared_memory(dev, pl->smem, "the batched kernel");
  if (rc0 != MC_OK) return rc0;
  int per_sm = 0;
  CK(fp64 ? batch_occupancy<double>(c.block, pl->smem, c.wide, range, false, &per_sm)
          : batch_occupancy<float>(c.block, pl->smem, c.wide, range, seg != 0, &per_sm));
  if (per_sm < 1)
    return fail(MC_ERR_INVALID, "batched kernel does not fit on an SM (block %d, %zu B shared memory)", c.block,
                pl->smem);
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  pl->grid = sms * per_sm;
  const int lanes = fp64 ? kLanesFP64 : kLanesFP32;
  const uint64_t warps = (uint64_t)pl->grid * (c.block / 32);
  int rc = pl->d_stacks.ensure((size_t)lanes * warps * stack_cap * 16, dev);
  if (rc == MC_OK && seg) rc = pl->d_segs.ensure((size_t)warps * kSegLanes * kSegCap * 16, dev);
  if (rc == MC_OK) rc = pl->d_items.ensure((size_t)n * sizeof(BatchItem), dev);
  if (rc == MC_OK) rc = pl->d_head.ensure(sizeof(BatchHeader), dev);
  if (rc == MC_OK) rc = pl->d_tdone.ensure((size_t)n * 8, dev);
  if (rc != MC_OK) return rc;
  CK(cudaMallocHost(&pl->h_items, (size_t)n * sizeof(BatchItem)));
  CK(cudaMallocHost(&pl->h_head, sizeof(BatchHeader)));
  CK(cudaMallocHost(&pl->h_tdone, (size_t)n * 8 + 8));
  CK(cudaEventCreateWithFlags(&pl->uploaded, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
  rc = capture(pl.get());
  if (rc != MC_OK) return rc;
  pl->last_use = ++g_plan_clock;
  *out = pl.get();
  g_plans.push_back(std::move(pl));
  return MC_OK;
}

uint64_t fnv(uint64_t h, uint64_t v) {
  for (int i = 0; i < 8; ++i) {
    h ^= (v >> (8 * i)) & 0xFFu;
    h *= 1099511628211ull;
  }
  return h;
}

// shape of a batch for the autotuner's table
uint64_t batch_signature(mc_problem* const* ps, int n, const uint64_t* n_hist, const mc_run_opts& o) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, (uint64_t)n);
  h = fnv(h, (uint64_t)o.precision | ((uint64_t)o.tally_mode << 8) | ((uint64_t)o.n_batches << 16) |
                 ((uint64_t)o.ww_enable << 40));
  for (int i = 0; i < n; ++i) {
    const TableHeader* H = reinterpret_cast<const TableHeader*>(ps[i]->blob[0].data());
    int lg = 0;
    while ((n_hist[i] >> lg) > 1) ++lg;
    h = fnv(h, (uint64_t)ps[i]->G | ((uint64_t)H->has_lat << 8) | ((uint64_t)ps[i]->n_cell << 16) |
                   ((uint64_t)lg << 32));
    h = fnv(h, (uint64_t)ps[i]->total_bins);
  }
  return h;
}

}  // namespace
}  // namespace mcgb

// ------------------------------------------------------------------------------------------ ABI
using namespace mcgb;

extern "C" {

int mc_run_batch(mc_problem* const* ps, int n, const uint64_t* n_hist, uint64_t seed, const mc_run_opts* opts,
                 void* stream, double* per_problem_wall_s) {
  if (!ps || !n_hist) return fail(MC_ERR_INVALID, "NULL argument");
  if (n < 1 || n > 65536) return fail(MC_ERR_INVALID, "n=%d outside [1,65536]", n);
  mc_run_opts o;
  if (opts) o = *opts;
  else mc_run_opts_default(&o);
  if (o.precision != MC_FP32 && o.precision != MC_FP64) return fail(MC_ERR_INVALID, "precision");
  if (o.tally_mode != MC_TALLY_FIXED64 && o.tally_mode != MC_TALLY_FP64) return fail(MC_ERR_INVALID, "tally_mode");
  if (o.fixed_bits < 0 || o.fixed_bits > 48) return fail(MC_ERR_INVALID, "fixed_bits outside [0,48]");
  if (o.n_batches < 2 || o.n_batches > 4096) return fail(MC_ERR_INVALID, "n_batches outside [2,4096]");
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32))
    return fail(MC_ERR_INVALID, "block_size must be a multiple of 32 in [32,256]");
  if (o.batch_unit < 0 || o.batch_unit > (1 << 20)) return fail(MC_ERR_INVALID, "batch_unit outside [0,2^20]");
  if (o.blocks_per_sm < 0) return fail(MC_ERR_INVALID, "blocks_per_sm < 0");
  if (check_implicit_opts(o) != MC_OK) return MC_ERR_INVALID;
  const uint64_t stack_cap = o.bank_capacity ? o.bank_capacity : kDefaultStack;
  if (stack_cap < 64 || stack_cap > (1ull << 24)) return fail(MC_ERR_INVALID, "bank_capacity outside [64,2^24]");
  int dev;
  int rc = current_device(&dev);
  if (rc != MC_OK) return rc;
  const int nb = o.n_batches;
  const int fp64 = o.precision == MC_FP64;
  {
    std::vector<mc_problem*> seen(ps, ps + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(MC_ERR_INVALID, "a problem appears twice in the batch");
  }
  size_t slot = 0;
  int range = 0;  // some problem has a tally scored by the range walk
  int seg = !fp64;  // every problem's tallies take the plain walk: segments scored apart (FP32)
  for (int i = 0; i < n; ++i) {
    mc_problem* p = ps[i];
    if (!p) return fail(MC_ERR_INVALID, "problem %d is NULL", i);
    range = range || p->range;
    seg = seg && !p->range && p->n_tally <= 4;
    for (const HostTally& t : p->tallies) seg = seg && t.est == MC_EST_TRACK_LENGTH;
    if (p->dev != dev) return fail(MC_ERR_STATE, "problem %d was created on device %d, current is %d", i, p->dev, dev);
    if (n_hist[i] < (uint64_t)nb) return fail(MC_ERR_INVALID, "problem %d: need at least n_batches histories", i);
    if (n_hist[i] >= (1ull << 32)) return fail(MC_ERR_INVALID, "problem %d: history indices must stay below 2^32", i);
    if (o.ww_enable && !p->ww_set) return fail(MC_ERR_STATE, "problem %d: weight windows enabled but no table set", i);
    if ((double)nb * (double)p->row >= 4294967296.0)
      return fail(MC_ERR_INVALID, "problem %d: tally bins x batches must stay below 2^32", i);
    slot = std::max(slot, p->blob[fp64].size());
  }
  // configuration: explicit options, else what the autotuner stored for this shape, else defaults
  BatchConfig c{256, 0, 128};
  if (o.block_size || o.blocks_per_sm || o.batch_unit) {
    if (o.block_size) c.block = o.block_size;
    c.wide = o.blocks_per_sm == 2;
    if (o.batch_unit) c.unit = o.batch_unit;
  } else {
    const uint64_t sig = batch_signature(ps, n, n_hist, o);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_tuned.find(sig);
    if (it != g_tuned.end()) c = it->second;
  }
  if (fp64) c.wide = 0;  // FP64 tracking has one register budget
  for (int i = 0; i < n; ++i) {
    mc_problem* p = ps[i];
    const uint64_t bins = (uint64_t)p->total_bins;
    rc = p->d_tally.ensure((size_t)nb * p->row * 8, dev);
    if (rc == MC_OK) rc = p->d_stats.ensure((size_t)3 * bins * 8, dev);
    if (rc != MC_OK) return rc;
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  // claim order: problems of one geometry kind together (plain cells, then lattices), so that the
  // warps of an SM mostly run the same code (mixing them stalled the kernel on instruction
  // fetch), and shortest first within a kind
  auto kind = [&](int i) { return reinterpret_cast<const TableHeader*>(ps[i]->blob[0].data())->has_lat; };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    if (kind(a) != kind(b)) return kind(a) < kind(b);
    return n_hist[a] < n_hist[b];
  });

  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchPlan* pl = nullptr;
  rc = get_plan(dev, n, c, fp64, range, seg, slot, stack_cap, &pl);
  if (rc != MC_OK) return rc;
  CK(cudaEventSynchronize(pl->uploaded));  // the staging buffers are free again
  uint64_t units = 0;
  for (int k = 0; k < n; ++k) {
    const int i = ord[k];
    BatchItem& it = pl->h_items[k];
    std::memset(&it, 0, sizeof(it));
    fill_run_params(ps[i], o, n_hist[i], seed + (uint64_t)i, 1u, it.P);
    it.P.history_mode = 1;
    it.stats = ps[i]->d_stats.ptr;
    it.bins = (uint64_t)ps[i]->total_bins;
    it.blob64 = (const char*)ps[i]->d_blob[1].ptr;
    it.range_rows = ps[i]->range_rows;
    it.unit_first = units;
    it.n_units = (n_hist[i] + (uint64_t)c.unit - 1) / (uint64_t)c.unit;
    it.caller_index = i;
    units += it.n_units;
  }
  BatchHeader& H = *pl->h_head;
  std::memset(&H, 0, sizeof(H));
  H.n_units = units;
  H.stack_cap = stack_cap;
  H.n_items = (unsigned)n;
  H.unit = (unsigned)c.unit;
  H.tally_fp64 = o.tally_mode == MC_TALLY_FP64;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaStreamWaitEvent(s, pl->done, 0));  // a replay of this plan on another stream has finished
  CK(cudaMemcpyAsync(pl->d_head.ptr, pl->h_head, sizeof(BatchHeader), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl->d_items.ptr, pl->h_items, (size_t)n * sizeof(BatchItem), cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(pl->uploaded, s));
  CK(cudaGraphLaunch(pl->exec, s));
  CK(cudaEventRecord(pl->done, s));
  for (int i = 0; i < n; ++i) {
    mc_problem* p = ps[i];
    p->has_run = 1;
    p->launches = 0;  // not counted
    p->batched = 1;
    p->n_hist = n_hist[i];
    p->n_batches = nb;
    p->stream = s;
    p->log_cap = 0;
    p->last_status = MC_OK;
    p->tally_fp64 = o.tally_mode == MC_TALLY_FP64;
    p->stripes = 1;
    p->fixed_scale = std::ldexp(1.0, o.fixed_bits);
  }
  if (per_problem_wall_s) {
    CK(cudaMemcpyAsync(pl->h_tdone, pl->d_tdone.ptr, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pl->h_tdone + n, (char*)pl->d_head.ptr + offsetof(BatchHeader, t0), 8,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const unsigned long long t0 = pl->h_tdone[n];
    for (int k = 0; k < n; ++k) {
      const unsigned long long t = pl->h_tdone[k];
      per_problem_wall_s[pl->h_items[k].caller_index] = t > t0 ? (double)(t - t0) * 1e-9 : 0.0;
    }
  }
  return MC_OK;
}

int mc_batch_tune(mc_problem* const* ps, int n, const uint64_t* n_hist, uint64_t seed, const mc_run_opts* opts,
                  void* stream, mc_run_opts* tuned, double* best_ms) {
  mc_run_opts o;
  if (opts) o = *opts;
  else mc_run_opts_default(&o);
  const int fp64 = o.precision == MC_FP64;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  // the arguments are checked once, by a run of the default configuration
  int rc = mc_run_batch(ps, n, n_hist, seed, &o, stream, nullptr);
  std::vector<BatchConfig> cands;
  for (int block : {128, 256})
    for (int wide = 0; wide <= (fp64 ? 0 : 1); ++wide)
      for (int unit : {32, 64, 128, 256, 512}) cands.push_back(BatchConfig{block, wide, unit});
  BatchConfig best{0, 0, 0};
  float best_t = 0.f;
  for (size_t ci = 0; ci < cands.size() && rc == MC_OK; ++ci) {
    mc_run_opts c = o;
    c.block_size = cands[ci].block;
    c.blocks_per_sm = cands[ci].wide ? 2 : 0;
    c.batch_unit = cands[ci].unit;
    rc = mc_run_batch(ps, n, n_hist, seed, &c, stream, nullptr);  // warm-up (captures the plan)
    if (rc == MC_ERR_INVALID) {  // this block size does not fit the problems' tables: skip it
      rc = MC_OK;
      continue;
    }
    float t = -1.f;
    for (int rep = 0; rep < 2 && rc == MC_OK; ++rep) {
      ce = cudaEventRecord(e0, s);
      if (ce == cudaSuccess) rc = mc_run_batch(ps, n, n_hist, seed, &c, stream, nullptr);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess && rc == MC_OK) rc = cuda_fail(ce, "timing a candidate");
      if (t < 0.f || ms < t) t = ms;
    }
    if (rc == MC_OK && (best.block == 0 || t < best_t)) {
      best = cands[ci];
      best_t = t;
    }
  }
  if (rc == MC_OK && best.block == 0) rc = fail(MC_ERR_INVALID, "no candidate configuration fits the batch");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MC_OK) return rc;
  for (int i = 0; i < n; ++i) {
    rc = mc_wait(ps[i]);  // a candidate that failed on the device fails the tuning
    if (rc != MC_OK) return rc;
  }
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_tuned[batch_signature(ps, n, n_hist, o)] = best;
  }
  if (tuned) {
    *tuned = o;
    tuned->block_size = best.block;
    tuned->blocks_per_sm = best.wide ? 2 : 0;
    tuned->batch_unit = best.unit;
  }
  if (best_ms) *best_ms = best_t;
  return MC_OK;
}

}  // extern "C"
