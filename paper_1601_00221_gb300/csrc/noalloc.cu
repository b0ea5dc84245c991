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
// of the runtime once per device (with that device current) and cached.
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

int sm_count_current() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
    return v;
  return 148;
}

}  // namespace

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
  if (((uintptr_t)programs & 15u) != 0) return gp_fail(GP_ERR_INVALID_ARG, "programs must be 16-byte aligned");
  if (n_cases > 0 && n_inputs > 0 && !cases) return gp_fail(GP_ERR_INVALID_ARG, "null cases");
  if (n_cases > 0 && !targets) return gp_fail(GP_ERR_INVALID_ARG, "null targets");
  gp_config c;
  int rc = gp_get_config(&c);
  if (rc) return rc;
  if (c.variant != GP_VARIANT_EXTENDED && c.variant != GP_VARIANT_EXTENDED_RPN)
    c.variant = GP_VARIANT_REGISTER;
  c.stack_registers = 0;  // every level in registers

  NoallocScratch* scratch = nullptr;
  rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  // chunks per program: fill the GPU, but never more partial sums than the
  // scratch holds
  const int per_pass = c.k * c.block;
  const int64_t target_blocks = (int64_t)kAutoBlocksPerSm * sm_count_current();
  int64_t want = std::max<int64_t>(1, (target_blocks + n_progs - 1) / n_progs);
  want = std::min<int64_t>(want, std::max<int64_t>(1, kMaxPartials / n_progs));
  int64_t chunk = (n_cases + want - 1) / want;
  chunk = std::max<int64_t>(per_pass, ((chunk + per_pass - 1) / per_pass) * per_pass);
  const int64_t n_chunks = std::max<int64_t>(1, (n_cases + chunk - 1) / chunk);
  if (n_chunks > 1 && n_chunks * n_progs > kMaxPartials)
    return gp_fail(GP_ERR_INVALID_ARG, "%lld partial sums exceed the fixed scratch of %lld",
                   (long long)(n_chunks * n_progs), (long long)kMaxPartials);
  const int32_t tile_inputs = (c.tile_inputs > 0 && c.tile_inputs < n_inputs) ? c.tile_inputs : n_inputs;
  const size_t tile_bytes = float_tile_bytes(c.k, c.block, tile_inputs);
  if (tile_bytes > 200 * 1024)
    return gp_fail(GP_ERR_INVALID_ARG, "a tile of %d inputs needs %zu bytes of shared memory per block",
                   tile_inputs, tile_bytes);
  const int32_t prog_cap = c.max_instructions > 0 ? c.max_instructions : gpisa::MAX_INSTR;
  const size_t smem = prog_buffer_bytes(prog_cap) + tile_bytes;

  // the array keeps the previous call's contents: clear the counters this
  // call relies on and the status word
  cudaError_t e = cudaMemsetAsync(scratch->counters, 0, sizeof(unsigned) * (size_t)n_progs, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&scratch->status, 0, sizeof(int), s);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "clearing the scratch: %s", cudaGetErrorString(e));

  FloatArgs a;
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
  a.x_aligned = (((uintptr_t)cases & 15u) == 0) && (n_inputs <= 1 || n_cases % 4 == 0);
  a.y_aligned = ((uintptr_t)targets & 15u) == 0;
  a.o_aligned = 0;
  a.want_fitness = 1;
  a.fitness_kind = c.fitness;
  a.tile_inputs = tile_inputs;
  a.prog_cap = prog_cap;
  a.order = nullptr;
  if (order_blocks(n_progs, n_cases, sm_count_current())) {
    e = launch_order_by_size(lengths, n_progs, scratch->order, s);
    if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "ordering launch: %s", cudaGetErrorString(e));
    a.order = scratch->order;
  }
  const int grid = (int)(n_progs * n_chunks);
  const bool xreg = (n_inputs == 1);
  if (c.variant == GP_VARIANT_EXTENDED) {
    if (c.k == 1) e = launch_floatx_k1(a, xreg, c.block, grid, smem, s);
    else if (c.k == 2) e = launch_floatx_k2(a, xreg, c.block, grid, smem, s);
    else if (c.k == 4) e = launch_floatx_k4(a, xreg, c.block, grid, smem, s);
    else e = launch_floatx_k8(a, xreg, c.block, grid, smem, s);
  } else if (c.variant == GP_VARIANT_EXTENDED_RPN) {
    if (c.k == 1) e = launch_floatrx_k1(a, xreg, c.block, grid, smem, s);
    else if (c.k == 2) e = launch_floatrx_k2(a, xreg, c.block, grid, smem, s);
    else if (c.k == 4) e = launch_floatrx_k4(a, xreg, c.block, grid, smem, s);
    else e = launch_floatrx_k8(a, xreg, c.block, grid, smem, s);
  } else if (c.k == 1) e = launch_float_k1(a, xreg, c.block, grid, smem, s);
  else if (c.k == 2) e = launch_float_k2(a, xreg, c.block, grid, smem, s);
  else if (c.k == 4) e = launch_float_k4(a, xreg, c.block, grid, smem, s);
  else e = launch_float_k8(a, xreg, c.block, grid, smem, s);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return GP_OK;
}
