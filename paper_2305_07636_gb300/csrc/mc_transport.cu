// Transport helpers and launchers (sm_103a): batch statistics, range-walk reconstruction,
// k-eigenvalue site combing, population control, measurement probes, and the launchers of the
// persistent transport kernel (mc_transport.cuh) with its plain-walk and FP64 builds.
#include <cuda_runtime.h>

#include "mc_transport.cuh"

namespace mcgb {

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
// (128 registers, no spills); `wide` selects the second (the segment builds at 128 threads per CTA
// take a third, 96 registers at 5 CTAs per SM, instead of 80).  `range` selects the build with the
// range walk of the scoring (tallies whose time axis is much finer than their mesh), `seg` the
// build that scores segments apart from their flights, `mode` the launch of a split run (1:
// event-based part, 2: history-style tail; the FP32 segment and range-walk builds are split).
template <typename R>
static const void* transport_fn(bool wide, bool range, bool seg, int block, int mode = 0) {
  if constexpr (sizeof(R) == 8) {
    return range ? (const void*)k_transport<R, 2, true, false, 0> : (const void*)k_transport<R, 2, false, false, 0>;
  } else {
    if (seg) return transport_fn_seg(wide, block, mode);
    if (range) return transport_fn_range(wide, mode);
    return wide ? (const void*)k_transport<R, 2, false, false, 0> : (const void*)k_transport<R, 3, false, false, 0>;
  }
}

// A run with per-warp stacks (P.WS) of a segment or range-walk build is split into the event-based
// launch and the history-style tail launch, back to back on the stream; any other run is one
// launch.
template <typename R>
cudaError_t launch_transport(const RunParams& P, int grid, int block, size_t smem, cudaStream_t s, bool wide,
                             bool range) {
  void* args[] = {const_cast<RunParams*>(&P)};
  const bool seg = P.seg != 0;
  if (sizeof(R) == 4 && (seg || range) && P.WS[0] != nullptr) {
    cudaError_t e = cudaLaunchCooperativeKernel(transport_fn<R>(wide, range, seg, block, 1), grid, block, args, smem, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(transport_fn<R>(wide, range, seg, block, 2), grid, block, args, smem, s);
  }
  return cudaLaunchCooperativeKernel(transport_fn<R>(wide, range, seg, block), grid, block, args, smem, s);
}

template <typename R>
cudaError_t transport_occupancy(int block, size_t smem, int* per_sm, bool wide, bool range, bool seg) {
  // every mode of a build has the same register budget; the split launches need the grid to fit
  // for each of them, so the least occupancy of the modes is taken
  const int n_modes = (sizeof(R) == 4 && (seg || range)) ? 3 : 1;
  int best = 1 << 30;
  for (int mode = 0; mode < n_modes; ++mode) {
    const void* f = transport_fn<R>(wide, range, seg, block, mode);
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
