// Population control by combing (systematic sampling of the census bank), sm_103a.
//
// At an interior census every statistical batch of the run is brought back to N_b particles.  The
// comb needs an order of the banked particles that does not depend on the GPU schedule: the bank
// (filled by atomics) is sorted by 64-bit particle tag and then, stably, by batch, with CUB's device
// radix sort (a library primitive of the CUDA toolkit).  Then per batch the cumulative fixed-point
// weights C_j are an inclusive scan of llrint(w 2^40) in that order, less the batch's start, and
// particle j becomes F(C_j) - F(C_{j-1}) copies, F(C) = min(N_b, max(0, ceil(C N_b / W_b - xi_b)))
// in FP64 (each operation rounded in that order, as the CPU reference does), i.e. the N_b teeth
// (k + xi_b) W_b / N_b that fall in its weight interval.  Copies are tagged and placed as the
// splitting-roulette copies are, so the next interval starts from them alone.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "mc_events.cuh"

namespace mcgb {

constexpr double kW40 = 1099511627776.0;  // 2^40, the fixed-point scale of census weights

// Where the comb's fields sit in a banked particle (16-byte lanes): tag (x, y), batch in the high
// half of elem, weight (FP64 bits).  FP32: tag lane 3, elem lane 1 .z, weight lane 2 (.z, .w).
// FP64: tag lane 4, elem lane 5 .x, weight lane 3 (.z, .w).
template <typename R>
struct CombLanes;
template <>
struct CombLanes<float> {
  static constexpr int kTag = 3, kElem = 1, kW = 2;
  static __device__ __forceinline__ uint32_t elem(const uint4& v) { return v.z; }
};
template <>
struct CombLanes<double> {
  static constexpr int kTag = 4, kElem = 5, kW = 3;
  static __device__ __forceinline__ uint32_t elem(const uint4& v) { return v.x; }
};

// One pass over the census bank, three of its lanes: tag keys, identity indices, and in bank order
// the batch and the fixed-point weight llrint(w 2^40) of every particle.
template <typename R>
__global__ void k_comb_keys(const RunParams P, uint64_t n, unsigned long long* tag, uint32_t* idx, uint32_t* bat0,
                            long long* wq0) {
  using L = CombLanes<R>;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 t = __ldcg(P.C[L::kTag] + i);
    const uint4 e = __ldcg(P.C[L::kElem] + i);
    const uint4 w = __ldcg(P.C[L::kW] + i);
    tag[i] = ((unsigned long long)t.y << 32) | t.x;
    idx[i] = (uint32_t)i;
    bat0[i] = L::elem(e) >> 16;
    const double wd = __longlong_as_double((long long)(((unsigned long long)w.w << 32) | w.z));
    wq0[i] = __double2ll_rn(__dmul_rn(wd, kW40));
  }
}

// batch of each particle, in tag order
__global__ void k_comb_batch(uint64_t n, const uint32_t* idx, const uint32_t* bat0, uint32_t* batch) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x)
    batch[j] = bat0[idx[j]];
}

// fixed-point weights in (batch, tag) order, and the first position of every batch
__global__ void k_comb_weights(uint64_t n, const uint32_t* idx, const uint32_t* batch, const long long* wq0,
                               long long* wq, uint32_t* start) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    wq[j] = wq0[idx[j]];
    if (j == 0 || batch[j - 1] != batch[j]) start[batch[j]] = (uint32_t)j;
  }
}

// #{k in [0, Nb) : (k + xi) W / Nb < C}
__device__ __forceinline__ long long comb_teeth_below(long long C, long long W, uint64_t Nb, double xi) {
  const double x = __dsub_rn(__ddiv_rn(__dmul_rn(__ll2double_rn(C), __ull2double_rn(Nb)), __ll2double_rn(W)), xi);
  const double f = ceil(x);
  if (!(f > 0.0)) return 0;
  return f >= __ull2double_rn(Nb) ? (long long)Nb : (long long)f;
}

template <typename R>
__global__ void k_comb_copies(const RunParams P, uint64_t n, const uint32_t* idx, const uint32_t* batch,
                              const long long* wq, const long long* csum, const uint32_t* start, const long long* wb,
                              uint32_t census, const RunParams Q, unsigned long long* out_n,
                              unsigned long long* copies, int* status) {
  const uint64_t N = P.n_hist, nb = (uint64_t)P.n_batches;
  unsigned local = 0;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = batch[j];
    const uint64_t Nb = (((uint64_t)b + 1) * N + nb - 1) / nb - ((uint64_t)b * N + nb - 1) / nb;
    const long long W = wb[b];
    if (W <= 0 || Nb == 0) continue;
    const uint32_t s = start[b];
    const long long Cj = csum[j] - (s > 0 ? csum[s - 1] : 0ll);
    const long long Cp = Cj - wq[j];
    const double xi = draw<double>(P.seed, 0xFFFFFFFEu, b, census, 5).a;
    const long long c = comb_teeth_below(Cj, W, Nb, xi) - comb_teeth_below(Cp, W, Nb, xi);
    if (c <= 0) continue;
    Part<R> p;
    bank_load(p, P.C, idx[j]);
    const double wt = __ddiv_rn(__ddiv_rn((double)W, kW40), (double)Nb);
    for (long long k = 0; k < c; ++k) {
      Part<R> q = p;
      const uint2 t = child_tag(P.seed, p.tlo, p.thi, p.k, (uint32_t)k, 0x40000000u);
      q.tlo = t.x;
      q.thi = t.y;
      q.k = 0;
      q.w = wt;
      q.pk = pk_set_pending(q.pk, PEND_NONE, 0, 1, 0);
      set_census_time(q, P);
      const unsigned long long o = atomicAdd(out_n, 1ull);
      if (o < Q.cap_b) bank_store(q, Q.B[0], o);
      else atomicCAS(status, 0, MC_ERR_BANK_FULL);
    }
    local += (unsigned)c;
  }
  if (local) atomicAdd(copies, (unsigned long long)local);
}

// Scratch the comb needs for n banked particles and nb batches (bytes), CUB's included.
size_t comb_scratch_bytes(uint64_t n, int nb) {
  size_t sort_tmp = 0, sort2_tmp = 0, scan_tmp = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, sort_tmp, (const unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                  (const uint32_t*)nullptr, (uint32_t*)nullptr, (int64_t)n);
  cub::DeviceRadixSort::SortPairs(nullptr, sort2_tmp, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                  (const uint32_t*)nullptr, (uint32_t*)nullptr, (int64_t)n);
  cub::DeviceScan::InclusiveSum(nullptr, scan_tmp, (const long long*)nullptr, (long long*)nullptr, (int64_t)n);
  const size_t tmp = std::max(sort_tmp, std::max(sort2_tmp, scan_tmp));
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  return up(n * 8) * 2 + up(n * 4) * 5 + up(n * 8) * 3 + up((size_t)nb * 4) + up(tmp);
}

// The comb of the n particles banked by launch P (its census bank P.C), copies into Q's birth bank.
// wb: exact batch weights (from k_pc_weight); census: the interior census index.
template <typename R>
cudaError_t launch_comb_pc(const RunParams& P, const RunParams& Q, uint64_t n, const long long* wb, uint32_t census,
                           void* scratch, size_t scratch_bytes, unsigned long long* out_n, unsigned long long* copies,
                           int* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* c = (char*)scratch;
  unsigned long long* tag_a = (unsigned long long*)c;
  c += up(n * 8);
  unsigned long long* tag_b = (unsigned long long*)c;
  c += up(n * 8);
  uint32_t* idx_a = (uint32_t*)c;
  c += up(n * 4);
  uint32_t* idx_b = (uint32_t*)c;
  c += up(n * 4);
  uint32_t* bat_a = (uint32_t*)c;
  c += up(n * 4);
  uint32_t* bat_b = (uint32_t*)c;
  c += up(n * 4);
  long long* wq = (long long*)c;
  c += up(n * 8);
  long long* csum = (long long*)c;
  c += up(n * 8);
  uint32_t* start = (uint32_t*)c;
  c += up((size_t)P.n_batches * 4);
  uint32_t* bat0 = (uint32_t*)c;
  c += up(n * 4);
  long long* wq0 = (long long*)c;
  c += up(n * 8);
  void* tmp = c;
  size_t tmp_bytes = scratch_bytes - (size_t)(c - (char*)scratch);
  const unsigned g = 152 * 8;
  int end_bit = 1;
  while ((1 << end_bit) < P.n_batches) ++end_bit;
  k_comb_keys<R><<<g, 256, 0, s>>>(P, n, tag_a, idx_a, bat0, wq0);
  cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, tag_a, tag_b, idx_a, idx_b, (int64_t)n, 0, 64, s);
  if (e != cudaSuccess) return e;
  k_comb_batch<<<g, 256, 0, s>>>(n, idx_b, bat0, bat_a);
  e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, bat_a, bat_b, idx_b, idx_a, (int64_t)n, 0, end_bit, s);
  if (e != cudaSuccess) return e;
  k_comb_weights<<<g, 256, 0, s>>>(n, idx_a, bat_b, wq0, wq, start);
  e = cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, wq, csum, (int64_t)n, s);
  if (e != cudaSuccess) return e;
  k_comb_copies<R><<<g, 256, 0, s>>>(P, n, idx_a, bat_b, wq, csum, start, wb, census, Q, out_n, copies, status);
  return cudaGetLastError();
}

template cudaError_t launch_comb_pc<float>(const RunParams&, const RunParams&, uint64_t, const long long*, uint32_t,
                                           void*, size_t, unsigned long long*, unsigned long long*, int*, cudaStream_t);
template cudaError_t launch_comb_pc<double>(const RunParams&, const RunParams&, uint64_t, const long long*, uint32_t,
                                            void*, size_t, unsigned long long*, unsigned long long*, int*, cudaStream_t);

}  // namespace mcgb
