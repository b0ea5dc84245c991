// noalloc.cu -- gp_eval_population_noalloc: float fitness without any device
// allocation by the library.
//
// gp_eval_population keeps its per-block partial sums and arrival counters in
// a workspace it allocates (and grows) with the stream-ordered allocator.
// Some callers cannot let a library allocate: a host application that hands
// the GPU's memory to its own fixed-size pool and forbids other allocations,
// or an evaluation loop that must not risk an allocation failure or the
// synchronisation cudaMalloc can imply in the middle of a run.  This entry
// point serves them with the same kernel, whose scratch lives in the
// fixed-size device array below instead.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "../../include/gpeval.h"
#include "config.h"
#include "launch.h"
#include "status.h"

using namespace gpdev;

namespace {

// Capacity of the fixed scratch: partial sums of up to this many
// (program, chunk) blocks, and arrival counters of up to this many programs.
constexpr int64_t kMaxPartials = GP_NOALLOC_MAX_PARTIALS;
constexpr int64_t kMaxCounters = GP_NOALLOC_MAX_PARTIALS;

struct NoallocScratch {
  Partial partials[kMaxPartials];
  unsigned counters[kMaxCounters];
  int32_t order[kMaxCounters];  // programs longest first
  int status;
};

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 64;

std::mutex g_mu;
NoallocScratch* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol g_noalloc_scratch is only a stand-in, so the address is asked
// of the runtime once per device (with that device current) and kept until
// gp_shutdown forgets it.
int scratch_on_current_device(NoallocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return gp_fail(GP_ERR_INVALID_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return gp_fail(GP_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
    g_addr[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_addr[dev];
  return GP_OK;
}

}  // namespace

namespace gpdev {
void noalloc_forget_devices() {
  std::lock_guard<std::mutex> lk(g_mu);
  for (NoallocScratch*& p : g_addr) p = nullptr;
}
}  // namespace gpdev

extern "C" int gp_eval_population_noalloc(const uint32_t* programs, const int64_t* offsets,
                                          const int32_t* lengths, int32_t n_progs,
                                          const float* cases, int32_t n_inputs, int64_t n_cases,
                                          const float* targets, double* fitness_out,
                                          gp_stream_t stream) {
  gp_clear_error();
  if (n_progs < 0 || n_inputs < 0 || n_cases < 0) return gp_fail(GP_ERR_INVALID_ARG, "negative size");
  if (!fitness_out) return gp_fail(GP_ERR_INVALID_ARG, "null fitness_out");
  if (n_progs == 0) return GP_OK;
  if (n_progs > kMaxCounters)
    return gp_fail(GP_ERR_INVALID_ARG,
                   "gp_eval_population_noalloc takes at most %lld programs per call (got %d)",
                   (long long)kMaxCounters, n_progs);
  if (!programs || !offsets || !lengths) return gp_fail(GP_ERR_INVALID_ARG, "null program arrays");
  if (!aligned16(programs)) return gp_fail(GP_ERR_INVALID_ARG, "programs must be 16-byte aligned");
  if (n_cases > 0 && n_inputs > 0 && !cases) return gp_fail(GP_ERR_INVALID_ARG, "null cases");
  if (n_cases > 0 && !targets) return gp_fail(GP_ERR_INVALID_ARG, "null targets");
  if (n_cases > kMaxCases) return gp_fail(GP_ERR_INVALID_ARG, "n_cases too large");
  // the configuration gp_eval_population would run: the default, then the
  // autotuner's record for this workload's shape
  gp_config c;
  int rc = resolve_config(nullptr, &c);
  if (rc) return rc;
  apply_tuned(nullptr, &c, n_inputs, n_cases, n_progs);
  const int32_t tile_inputs = (c.tile_inputs > 0 && c.tile_inputs < n_inputs) ? c.tile_inputs : n_inputs;
  size_t smem = 0;
  rc = float_launch_smem(c, tile_inputs, &smem);
  if (rc) return rc;

  NoallocScratch* scratch = nullptr;
  rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  // The same split of the cases as gp_eval_population, unless its partial
  // sums would not fit the scratch: then fewer, larger chunks (whole passes
  // of the block each), and the fitness agrees within the fitness tolerance
  // rather than bit for bit.  (The automatic split never needs that: it aims
  // at kAutoBlocksPerSm blocks per multiprocessor, far below the capacity;
  // a recorded tuning with small chunks of a large case set can.)
  const int per_pass = c.k * c.block;
  int64_t chunk = choose_chunk(n_cases, n_progs, per_pass, c.chunk_cases, kAutoBlocksPerSm);
  int64_t n_chunks = std::max<int64_t>(1, (n_cases + chunk - 1) / chunk);
  if (n_chunks > 1 && n_chunks * n_progs > kMaxPartials) {
    const int64_t fit = std::max<int64_t>(1, kMaxPartials / n_progs);
    chunk = (n_cases + fit - 1) / fit;
    chunk = std::max<int64_t>(per_pass, ((chunk + per_pass - 1) / per_pass) * per_pass);
    n_chunks = std::max<int64_t>(1, (n_cases + chunk - 1) / chunk);
  }
  // (n_chunks <= kMaxPartials / n_progs now, or 1, which uses no partials)

  // the array keeps the previous call's contents: clear the counters this
  // call relies on and the status word
  cudaError_t e = cudaMemsetAsync(scratch->counters, 0, sizeof(unsigned) * (size_t)n_progs, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&scratch->status, 0, sizeof(int), s);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "clearing the scratch: %s", cudaGetErrorString(e));

  FloatArgs a{};
  a.programs = programs;
  a.offsets = offsets;
  a.lengths = lengths;
  a.n_progs = n_progs;
  a.cases = cases;
  a.n_inputs = n_inputs;
  a.n_cases = n_cases;
  a.targets = targets;
  a.fitness_out = fitness_out;
  a.outputs = nullptr;
  a.partials = scratch->partials;
  a.counters = scratch->counters;
  a.status = &scratch->status;
  a.chunk_cases = chunk;
  a.n_chunks = (int32_t)n_chunks;
  a.x_aligned = aligned16(cases) && (n_inputs <= 1 || n_cases % 4 == 0);
  a.y_aligned = aligned16(targets);
  a.o_aligned = 0;
  a.want_fitness = 1;
  a.fitness_kind = c.fitness;
  a.tile_inputs = tile_inputs;
  a.prog_cap = c.max_instructions;
  a.order = nullptr;
  if (order_blocks(n_progs, n_cases, sm_count())) {
    e = launch_order_by_size(lengths, n_progs, scratch->order, s);
    if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "ordering launch: %s", cudaGetErrorString(e));
    a.order = scratch->order;
  }
  e = launch_float_config(a, c, n_inputs == 1, (int)(n_progs * n_chunks), smem, s);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return GP_OK;
}
