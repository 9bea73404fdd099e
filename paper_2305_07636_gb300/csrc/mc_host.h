// Host-side internals of libmcgb shared by its translation units: error reporting, the device
// memory pool and the problem object behind the opaque mc_problem handle.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <stdint.h>

#include <vector>

#include "mc_internal.h"

namespace mcgb {

// records the message returned by mc_last_error (thread-local) and returns `code`
int fail(int code, const char* fmt, ...);
// maps a CUDA error to MC_ERR_OOM / MC_ERR_CUDA with its message
int cuda_fail(cudaError_t e, const char* what);
int current_device(int* dev);
// MC_ERR_INVALID (with a message naming `what`) when `bytes` of dynamic shared memory per CTA exceed
// the device's opt-in limit: the transport kernels keep the problem's tables in shared memory
int check_shared_memory(int dev, size_t bytes, const char* what);
// validates the implicit-capture fields of run options (MC_OK or MC_ERR_INVALID with a message)
int check_implicit_opts(const mc_run_opts& o);

// device blocks are recycled across problems instead of returned to the driver; a block must be
// returned with the size it was requested with
int pool_alloc(void** out, size_t bytes, int dev);
void pool_free(void* p, size_t bytes, int dev);

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int dev = 0;
  int ensure(size_t want, int device) {
    if (ptr && bytes >= want && dev == device) return MC_OK;
    release();
    int rc = pool_alloc(&ptr, want, device);
    if (rc != MC_OK) {
      ptr = nullptr;
      return rc;
    }
    bytes = want;
    dev = device;
    return MC_OK;
  }
  void release() {
    pool_free(ptr, bytes, dev);
    ptr = nullptr;
    bytes = 0;
  }
};

struct HostTally {
  int n[4];
  int est = MC_EST_TRACK_LENGTH;
  int nval = 0;  // values along time per (cell, group): n[3] bins or n[3] + 1 points
  std::vector<double> e[4];
};

}  // namespace mcgb

struct mc_problem;
namespace mcgb {
// run parameters that mc_run and mc_run_batch share: control block, sticky error, tallies
// (stripes copies), statistics scale, batches, tables of the run's precision, seed, event budget,
// weight windows.  Banks, logging, tracing and the algorithm are the caller's.
void fill_run_params(const mc_problem* p, const mc_run_opts& o, uint64_t n_histories, uint64_t seed,
                     uint32_t stripes, RunParams& P);
}  // namespace mcgb

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return mcgb::cuda_fail(e_, #call); \
  } while (0)

struct mc_problem {
  int dev = 0;
  mc_mlp* own_mlp = nullptr;  // mc_ww_set_mlp / mc_ww_train's network, released with the problem
  int G = 0, M = 0, n_surf = 0, n_cell = 0, n_tally = 0;
  int total_bins = 0, leak_offset = 0;
  bool range = false;  // some mesh tally is scored by the range walk (kernel build)
  uint64_t row = 0;    // elements of one batch row of the tallies: bins, then difference slots
  uint64_t range_rows = 0;  // (tally, cell, group) rows scored by the range walk
  int tuned_block = 0, tuned_bps = 0;  // mc_run_tune's choice (block_size, blocks_per_sm), 0 = none
  int tuned_alg = MC_ALG_EVENT;        // mc_run_tune's algorithm for MC_ALG_AUTO
  uint64_t tuned_drain = 0;            // mc_run_tune's drain threshold (0 = the default)
  std::vector<mcgb::HostTally> tallies;
  std::vector<uint8_t> blob[2];  // [0] FP32 tables, [1] FP64 tables
  mcgb::DevBuf d_blob[2];
  mcgb::DevBuf d_ctl, d_tally, d_stats, d_log, d_banks, d_trace;
  mcgb::DevBuf d_wstack;  // per-warp stacks of secondaries of a split run's tail launch
  mcgb::DevBuf d_sticky;  // first device error of any run since the last mc_wait (not reset by mc_run)
  // last run
  int has_run = 0;
  int launches = 0;  // kernels the last plain mc_run launched (0: not counted)
  int batched = 0;  // the last run was part of mc_run_batch (timing from the device clock)
  uint64_t n_hist = 0;
  int n_batches = 0;
  cudaStream_t stream = nullptr;
  uint64_t log_cap = 0;
  int last_status = MC_OK;
  int tally_fp64 = 0;
  uint32_t stripes = 1;
  double fixed_scale = 1.0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // transport start, transport end, stats end
  // weight windows
  int ww_set = 0, ww_n[4] = {0, 0, 0, 0};  // window mesh: x, y, z and time bins
  double src_center[3] = {0.0, 0.0, 0.0};  // reference point of the source (box centre / surface point)
  int src_group = 0;                        // the source's most likely group
  mcgb::DevBuf d_ww;
  // k-eigenvalue cycles: fission sites [N][nmax], sites per history, their scan and block totals,
  // the next cycle's sources [N]; the last run's per-cycle k and its active-cycle mean and error
  mcgb::DevBuf d_sites, d_counts, d_scan, d_blocksums, d_src;
  // population control: the census bank, per-batch weights and split counters
  mcgb::DevBuf d_cbank, d_pc;
  mcgb::DevBuf d_comb;  // combing: sort keys and indices, fixed-point weights and their scan, CUB scratch
  double nu_max = 0.0;
};
