// api.cu -- the C ABI of include/gpeval.h: argument checks, the per-stream
// workspace, launch configuration and the evaluation entry points.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/gpeval.h"
#include "eval_bool.cuh"
#include "config.h"
#include "launch.h"
#include "status.h"

using namespace gpdev;

namespace {

std::mutex g_mu;
// the library's own defaults, and the current ones (gp_set_config)
const gp_config kLibraryDefault = {GP_VARIANT_REGISTER, 8, 128, 0, GP_FITNESS_SUM_ABS, 0, 0, 0};
gp_config g_default = kLibraryDefault;
bool g_default_set = false;  // gp_set_config was called: its K and block stand

// Internal workspace of one (device, stream): per-block partial sums, the
// per-program arrival counters of the fused reduction (zero between
// launches) and the program-error status word.
struct Workspace {
  int device;
  cudaStream_t stream;
  Partial* partials = nullptr;
  size_t partial_cap = 0;  // entries
  unsigned* counters = nullptr;
  size_t counter_cap = 0;  // entries
  int32_t* order = nullptr;  // programs longest first (launch_order_by_size)
  size_t order_cap = 0;      // entries
  int* status = nullptr;
};
std::vector<Workspace*> g_ws;

// autotuned configurations by workload shape
using TuneKey = std::tuple<int, int, int>;  // several inputs?, log2 n_cases, log2 n_progs
std::map<TuneKey, gp_config> g_tuned;

int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) { v >>= 1; ++r; }
  return r;
}
TuneKey tune_key(int32_t n_inputs, int64_t n_cases, int32_t n_progs) {
  return TuneKey(n_inputs > 1 ? 1 : 0, ilog2(std::max<int64_t>(n_cases, 1)), ilog2(std::max<int32_t>(n_progs, 1)));
}

int cuda_fail(cudaError_t e, const char* what) {
  return gp_fail(e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

int get_workspace(cudaStream_t s, size_t n_partials, size_t n_counters, Workspace** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace* w = nullptr;
  for (Workspace* x : g_ws)
    if (x->device == dev && x->stream == s) w = x;
  if (!w) {
    w = new Workspace();
    w->device = dev;
    w->stream = s;
    e = cudaMallocAsync((void**)&w->status, sizeof(int), s);
    if (e != cudaSuccess) { delete w; return cuda_fail(e, "workspace allocation"); }
    e = cudaMemsetAsync(w->status, 0, sizeof(int), s);
    if (e != cudaSuccess) { delete w; return cuda_fail(e, "workspace clear"); }
    g_ws.push_back(w);
  }
  if (n_partials > w->partial_cap) {
    size_t cap = std::max(n_partials, 2 * w->partial_cap);
    Partial* p = nullptr;
    e = cudaMallocAsync((void**)&p, cap * sizeof(Partial), s);
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    if (w->partials) cudaFreeAsync(w->partials, s);
    w->partials = p;
    w->partial_cap = cap;
  }
  if (n_counters > w->counter_cap) {
    size_t cap = std::max(n_counters, 2 * w->counter_cap);
    unsigned* c = nullptr;
    e = cudaMallocAsync((void**)&c, cap * sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    e = cudaMemsetAsync(c, 0, cap * sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    if (w->counters) cudaFreeAsync(w->counters, s);
    w->counters = c;
    w->counter_cap = cap;
  }
  *out = w;
  return GP_OK;
}

// the workspace's order array, grown to n entries (same stream and lock
// discipline as get_workspace)
int get_order(Workspace* w, size_t n, cudaStream_t s, int32_t** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (n > w->order_cap) {
    size_t cap = std::max(n, 2 * w->order_cap);
    int32_t* o = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&o, cap * sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    if (w->order) cudaFreeAsync(w->order, s);
    w->order = o;
    w->order_cap = cap;
  }
  *out = w->order;
  return GP_OK;
}

}  // namespace

namespace gpdev {

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n = v;
    if (n <= 0) n = 148;
  }
  return n;
}

// Fills zero fields of `c` from the default configuration and checks it.
int resolve_config(const gp_config* user, gp_config* c) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    *c = g_default;
  }
  if (user) {
    if (user->variant) c->variant = user->variant;
    if (user->k) c->k = user->k;
    if (user->block) c->block = user->block;
    c->chunk_cases = user->chunk_cases;
    if (user->fitness) c->fitness = user->fitness;
    c->tile_inputs = user->tile_inputs;
    c->stack_registers = user->stack_registers;
    c->max_instructions = user->max_instructions;
  }
  if (c->max_instructions < 0 || c->max_instructions > gpisa::MAX_INSTR)
    return gp_fail(GP_ERR_INVALID_ARG, "max_instructions must be 0..%d (got %d)", gpisa::MAX_INSTR,
                   c->max_instructions);
  if (c->max_instructions == 0) c->max_instructions = gpisa::MAX_INSTR;
  if (c->stack_registers == gpisa::R) c->stack_registers = 0;
  if (c->stack_registers != 0 && c->stack_registers != 4)
    return gp_fail(GP_ERR_INVALID_ARG, "stack_registers must be 0, 4 or 8 (got %d)", c->stack_registers);
  if (c->tile_inputs < 0) return gp_fail(GP_ERR_INVALID_ARG, "negative tile_inputs");
  if (c->variant != GP_VARIANT_REGISTER && c->variant != GP_VARIANT_LOCAL &&
      c->variant != GP_VARIANT_AUTO && c->variant != GP_VARIANT_LANES &&
      c->variant != GP_VARIANT_EXTENDED && c->variant != GP_VARIANT_EXTENDED_RPN)
    return gp_fail(GP_ERR_INVALID_ARG, "unknown variant %d", c->variant);
  if (c->fitness != GP_FITNESS_SUM_ABS && c->fitness != GP_FITNESS_MSE && c->fitness != GP_FITNESS_CLASS)
    return gp_fail(GP_ERR_INVALID_ARG, "unknown fitness measure %d", c->fitness);
  if (c->variant == GP_VARIANT_AUTO) c->variant = GP_VARIANT_REGISTER;
  if (c->k != 1 && c->k != 2 && c->k != 4 && c->k != 8)
    return gp_fail(GP_ERR_INVALID_ARG, "k must be 1, 2, 4 or 8 (got %d)", c->k);
  if (c->variant == GP_VARIANT_LOCAL) c->k = 1;
  if (c->block < 32 || c->block > 512 || c->block % 32)
    return gp_fail(GP_ERR_INVALID_ARG, "block must be a multiple of 32 in [32, 512] (got %d)", c->block);
  if (c->block > 256 && c->variant == GP_VARIANT_LOCAL)
    return gp_fail(GP_ERR_INVALID_ARG, "the local-memory variant takes at most 256 threads per block");
  if (c->chunk_cases < 0 || (c->chunk_cases % ((int64_t)c->k * c->block)) != 0)
    return gp_fail(GP_ERR_INVALID_ARG, "chunk_cases must be a multiple of k*block");
  return GP_OK;
}

// The recorded tuned configuration for a float workload, if any, fills the
// k and block fields the caller left at 0.
void apply_tuned(const gp_config* user, gp_config* c, int32_t n_inputs, int64_t n_cases, int32_t n_progs) {
  if (user && user->k && user->block) return;
  if (c->variant != GP_VARIANT_REGISTER) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_tuned.find(tune_key(n_inputs, n_cases, n_progs));
  if (it == g_tuned.end()) return;
  if (!user || !user->k) c->k = it->second.k;
  if (!user || !user->block) c->block = it->second.block;
  if (!user || !user->chunk_cases) c->chunk_cases = it->second.chunk_cases;
}

// Cases (or words) per block: enough blocks to fill the GPU several times
// over, each covering whole passes of the block.  blocks_per_sm: the float
// kernels take the programs longest first and want few long blocks
// (kAutoBlocksPerSm); the Boolean kernel keeps the caller's order and more,
// shorter blocks.
int64_t choose_chunk(int64_t n_units, int32_t n_progs, int per_pass, int64_t user_chunk,
                     int blocks_per_sm) {
  if (user_chunk > 0) return user_chunk;
  const int64_t target_blocks = (int64_t)blocks_per_sm * sm_count();
  int64_t want = (target_blocks + n_progs - 1) / std::max<int32_t>(n_progs, 1);
  want = std::max<int64_t>(want, 1);
  int64_t chunk = (n_units + want - 1) / want;
  chunk = ((chunk + per_pass - 1) / per_pass) * per_pass;
  return std::max<int64_t>(chunk, per_pass);
}

int float_launch_smem(const gp_config& c, int32_t tile_inputs, size_t* smem) {
  const bool rl4 = c.stack_registers == 4;
  if (rl4 && (c.k != 8 || c.variant != GP_VARIANT_REGISTER))
    return gp_fail(GP_ERR_INVALID_ARG, "stack_registers = 4 needs k = 8 and the register variant");
  const size_t tile_bytes = float_tile_bytes(c.k, c.block, tile_inputs) +
                            (rl4 ? (size_t)(c.block / 32) * spill_bytes_per_warp<8, 4>() : 0);
  if (c.variant != GP_VARIANT_LOCAL && tile_bytes > kMaxTileBytes)
    return gp_fail(GP_ERR_INVALID_ARG,
                   "a tile of %d inputs needs %zu bytes of shared memory per block (max %zu): "
                   "lower k, block or tile_inputs",
                   tile_inputs, tile_bytes, kMaxTileBytes);
  *smem = prog_buffer_bytes(c.max_instructions) + tile_bytes;
  return GP_OK;
}

cudaError_t launch_float_config(const FloatArgs& a, const gp_config& c, bool xreg, int grid, size_t smem,
                                cudaStream_t s) {
  if (c.variant == GP_VARIANT_LOCAL) return launch_blockgp(a, c.block, grid, s);
  if (c.stack_registers == 4) return launch_float_k8_rl4(a, xreg, c.block, grid, smem, s);
  if (c.variant == GP_VARIANT_EXTENDED) {
    if (c.k == 1) return launch_floatx_k1(a, xreg, c.block, grid, smem, s);
    if (c.k == 2) return launch_floatx_k2(a, xreg, c.block, grid, smem, s);
    if (c.k == 4) return launch_floatx_k4(a, xreg, c.block, grid, smem, s);
    return launch_floatx_k8(a, xreg, c.block, grid, smem, s);
  }
  if (c.variant == GP_VARIANT_EXTENDED_RPN) {
    if (c.k == 1) return launch_floatrx_k1(a, xreg, c.block, grid, smem, s);
    if (c.k == 2) return launch_floatrx_k2(a, xreg, c.block, grid, smem, s);
    if (c.k == 4) return launch_floatrx_k4(a, xreg, c.block, grid, smem, s);
    return launch_floatrx_k8(a, xreg, c.block, grid, smem, s);
  }
  if (c.k == 1) return launch_float_k1(a, xreg, c.block, grid, smem, s);
  if (c.k == 2) return launch_float_k2(a, xreg, c.block, grid, smem, s);
  if (c.k == 4) return launch_float_k4(a, xreg, c.block, grid, smem, s);
  return launch_float_k8(a, xreg, c.block, grid, smem, s);
}

}  // namespace gpdev

extern "C" int gp_set_config(const gp_config* cfg) {
  gp_clear_error();
  if (!cfg) {  // back to the library's own defaults
    std::lock_guard<std::mutex> lk(g_mu);
    g_default = kLibraryDefault;
    g_default_set = false;
    return GP_OK;
  }
  gp_config c;
  int rc = resolve_config(cfg, &c);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  g_default = c;
  g_default.chunk_cases = 0;
  g_default_set = true;
  return GP_OK;
}

extern "C" int gp_get_config(gp_config* cfg) {
  gp_clear_error();
  if (!cfg) return gp_fail(GP_ERR_INVALID_ARG, "null config");
  std::lock_guard<std::mutex> lk(g_mu);
  *cfg = g_default;
  return GP_OK;
}

extern "C" int gp_eval_population_ex(const uint32_t* programs, const int64_t* offsets,
                                     const int32_t* lengths, int32_t n_progs, const float* cases,
                                     int32_t n_inputs, int64_t n_cases, const float* targets,
                                     double* fitness_out, float* outputs, const gp_config* cfg,
                                     gp_stream_t stream) {
  gp_clear_error();
  if (n_progs < 0 || n_inputs < 0 || n_cases < 0)
    return gp_fail(GP_ERR_INVALID_ARG, "negative size");
  if (!fitness_out && !outputs) return gp_fail(GP_ERR_INVALID_ARG, "no output requested");
  if (n_progs == 0) return GP_OK;
  if (!programs || !offsets || !lengths) return gp_fail(GP_ERR_INVALID_ARG, "null program arrays");
  if (!aligned16(programs)) return gp_fail(GP_ERR_INVALID_ARG, "programs must be 16-byte aligned");
  if (n_cases > 0 && n_inputs > 0 && !cases) return gp_fail(GP_ERR_INVALID_ARG, "null cases");
  if (fitness_out && n_cases > 0 && !targets) return gp_fail(GP_ERR_INVALID_ARG, "null targets");
  if (n_cases > kMaxCases) return gp_fail(GP_ERR_INVALID_ARG, "n_cases too large");
  gp_config c;
  int rc = resolve_config(cfg, &c);
  if (rc) return rc;
  apply_tuned(cfg, &c, n_inputs, n_cases, n_progs);
  if (c.chunk_cases % ((int64_t)c.k * c.block) != 0)
    return gp_fail(GP_ERR_INVALID_ARG, "chunk_cases must be a multiple of k*block");
  cudaStream_t s = (cudaStream_t)stream;

  const int32_t tile_inputs = (c.tile_inputs > 0 && c.tile_inputs < n_inputs) ? c.tile_inputs : n_inputs;
  size_t smem = 0;
  rc = float_launch_smem(c, tile_inputs, &smem);
  if (rc) return rc;
  const int per_pass = c.k * c.block;
  const int64_t chunk = choose_chunk(n_cases, n_progs, per_pass, c.chunk_cases, kAutoBlocksPerSm);
  const int64_t n_chunks64 = std::max<int64_t>(1, (n_cases + chunk - 1) / chunk);
  if (n_chunks64 * n_progs > 0x7fffffffLL) return gp_fail(GP_ERR_INVALID_ARG, "too many blocks");
  const int32_t n_chunks = (int32_t)n_chunks64;

  Workspace* w = nullptr;
  rc = get_workspace(s, n_chunks > 1 ? (size_t)n_chunks * n_progs : 0, n_chunks > 1 ? n_progs : 0, &w);
  if (rc) return rc;

  FloatArgs a;
  a.programs = programs;
  a.offsets = offsets;
  a.lengths = lengths;
  a.n_progs = n_progs;
  a.cases = cases;
  a.n_inputs = n_inputs;
  a.n_cases = n_cases;
  a.targets = fitness_out ? targets : nullptr;
  a.fitness_out = fitness_out;
  a.outputs = outputs;
  a.partials = w->partials;
  a.counters = w->counters;
  a.status = w->status;
  a.chunk_cases = chunk;
  a.n_chunks = n_chunks;
  a.x_aligned = aligned16(cases) && (n_inputs <= 1 || n_cases % 4 == 0);
  a.y_aligned = aligned16(targets);
  a.o_aligned = aligned16(outputs) && (n_progs == 1 || n_cases % 4 == 0);
  a.want_fitness = fitness_out != nullptr;
  a.fitness_kind = c.fitness;
  a.tile_inputs = tile_inputs;
  a.prog_cap = c.max_instructions;
  a.order = nullptr;
  if (order_blocks(n_progs, n_cases, sm_count())) {
    int32_t* order = nullptr;
    rc = get_order(w, (size_t)n_progs, s, &order);
    if (rc) return rc;
    cudaError_t eo = launch_order_by_size(lengths, n_progs, order, s);
    if (eo != cudaSuccess) return cuda_fail(eo, "ordering launch");
    a.order = order;
  }
  const int grid = n_progs * n_chunks;
  const bool xreg = (n_inputs == 1);
  cudaError_t e = launch_float_config(a, c, xreg, grid, smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GP_OK;
}

extern "C" int gp_eval_population(const uint32_t* programs, const int64_t* offsets,
                                  const int32_t* lengths, int32_t n_progs, const float* cases,
                                  int32_t n_inputs, int64_t n_cases, const float* targets,
                                  double* fitness_out, gp_stream_t stream) {
  if (!fitness_out) {
    gp_clear_error();
    return gp_fail(GP_ERR_INVALID_ARG, "null fitness_out");
  }
  return gp_eval_population_ex(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases,
                               targets, fitness_out, nullptr, nullptr, stream);
}

extern "C" int gp_eval_outputs(const uint32_t* programs, const int64_t* offsets,
                               const int32_t* lengths, int32_t n_progs, const float* cases,
                               int32_t n_inputs, int64_t n_cases, float* outputs,
                               const gp_config* cfg, gp_stream_t stream) {
  if (!outputs) {
    gp_clear_error();
    return gp_fail(GP_ERR_INVALID_ARG, "null outputs");
  }
  return gp_eval_population_ex(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases,
                               nullptr, nullptr, outputs, cfg, stream);
}

extern "C" int gp_eval_population_bool_ex(const uint32_t* programs, const int64_t* offsets,
                                          const int32_t* lengths, int32_t n_progs,
                                          const uint32_t* case_bits, int32_t n_inputs,
                                          int64_t n_cases, const uint32_t* target_bits,
                                          uint64_t* hits_out, uint32_t* out_words,
                                          const gp_config* cfg, gp_stream_t stream) {
  gp_clear_error();
  if (n_progs < 0 || n_inputs < 0 || n_cases < 0)
    return gp_fail(GP_ERR_INVALID_ARG, "negative size");
  if (!hits_out && !out_words) return gp_fail(GP_ERR_INVALID_ARG, "no output requested");
  if (n_progs == 0) return GP_OK;
  if (!programs || !offsets || !lengths) return gp_fail(GP_ERR_INVALID_ARG, "null program arrays");
  if (!aligned16(programs)) return gp_fail(GP_ERR_INVALID_ARG, "programs must be 16-byte aligned");
  const int64_t n_words = (n_cases + 31) / 32;
  if (n_words > 0 && n_inputs > 0 && !case_bits) return gp_fail(GP_ERR_INVALID_ARG, "null case_bits");
  if (hits_out && n_words > 0 && !target_bits) return gp_fail(GP_ERR_INVALID_ARG, "null target_bits");
  // program per lane for tiny case sets unless a variant is forced
  const bool lanes = (cfg && cfg->variant == GP_VARIANT_LANES) ||
                     ((!cfg || cfg->variant == GP_VARIANT_AUTO) && n_words > 0 && n_words <= 4);
  if (lanes) {
    if (n_words > 4) return gp_fail(GP_ERR_INVALID_ARG, "the per-lane variant takes at most 4 words (128 cases)");
    Workspace* wl = nullptr;
    int rc0 = get_workspace((cudaStream_t)stream, 0, 0, &wl);
    if (rc0) return rc0;
    const int w = n_words <= 1 ? 1 : (n_words <= 2 ? 2 : 4);
    BoolArgs a;
    a.programs = programs;
    a.offsets = offsets;
    a.lengths = lengths;
    a.n_progs = n_progs;
    a.case_bits = case_bits;
    a.n_inputs = n_inputs;
    a.n_cases = n_cases;
    a.n_words = n_words;
    a.target_bits = hits_out ? target_bits : nullptr;
    a.hits_out = reinterpret_cast<unsigned long long*>(hits_out);
    a.out_words = out_words;
    a.status = wl->status;
    a.chunk_words = 0;
    a.n_chunks = 1;
    a.aligned = 0;
    a.prog_cap = gpisa::MAX_INSTR;  // (programs are read from global memory)
    // the caller's order: a warp's 32 programs then lie side by side in
    // memory, and the lanes' instruction loads share cache lines (taking the
    // programs longest first scattered them: 33-41% slower, measured)
    a.order = nullptr;
    const size_t smem = bool_lanes_smem(w, 32, n_inputs);
    if (smem > 48 * 1024) return gp_fail(GP_ERR_INVALID_ARG, "too many inputs for the per-lane variant");
    cudaError_t el = launch_bool_lanes(a, w, (n_progs + 31) / 32, smem, (cudaStream_t)stream);
    if (el != cudaSuccess) return cuda_fail(el, "kernel launch");
    return GP_OK;
  }
  gp_config c;
  int rc = resolve_config(cfg, &c);
  if (rc) return rc;
  if (c.variant == GP_VARIANT_EXTENDED || c.variant == GP_VARIANT_EXTENDED_RPN)
    c.variant = GP_VARIANT_REGISTER;  // a float-only choice
  if (c.variant != GP_VARIANT_REGISTER) return gp_fail(GP_ERR_INVALID_ARG, "Boolean programs use the register or per-lane variant");
  if (c.block > 256) c.block = 256;  // the Boolean kernel's block limit
  // Defaults for many inputs: the staged tile (inputs x 32 lanes x K words
  // per warp) limits the blocks per SM.  K = 4 and 64-thread blocks, measured
  // on the multiplexers: 20-mux 82.4 T bit-GPop/s against 47.9 at K = 8 with
  // 256-thread blocks (57.9 at K = 8 with 64), 11-mux 5678 against 4502.
  bool user_default;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    user_default = g_default_set;
  }
  if ((!cfg || !cfg->k) && !user_default && n_inputs >= 8) c.k = 4;
  if (!cfg || !cfg->block) {  // small case sets: do not launch idle warps
    int64_t need = (n_words + c.k - 1) / c.k;
    c.block = (int)std::min<int64_t>(c.block, std::max<int64_t>(32, ((need + 31) / 32) * 32));
    if (!user_default && (int64_t)n_inputs * c.k >= 32) c.block = std::min(c.block, 64);
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int per_pass = c.k * c.block;
  const int64_t chunk = choose_chunk(n_words, n_progs, per_pass, c.chunk_cases, 48);
  const int64_t n_chunks64 = std::max<int64_t>(1, (n_words + chunk - 1) / chunk);
  if (n_chunks64 * n_progs > 0x7fffffffLL) return gp_fail(GP_ERR_INVALID_ARG, "too many blocks");
  Workspace* w = nullptr;
  rc = get_workspace(s, 0, 0, &w);
  if (rc) return rc;
  cudaError_t e;
  if (hits_out) {
    e = cudaMemsetAsync(hits_out, 0, sizeof(uint64_t) * (size_t)n_progs, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing hits");
  }
  BoolArgs a;
  a.programs = programs;
  a.offsets = offsets;
  a.lengths = lengths;
  a.n_progs = n_progs;
  a.case_bits = case_bits;
  a.n_inputs = n_inputs;
  a.n_cases = n_cases;
  a.n_words = n_words;
  a.target_bits = hits_out ? target_bits : nullptr;
  a.hits_out = reinterpret_cast<unsigned long long*>(hits_out);
  a.out_words = out_words;
  a.status = w->status;
  a.chunk_words = chunk;
  a.prog_cap = c.max_instructions;
  a.n_chunks = (int32_t)n_chunks64;
  a.aligned = aligned16(case_bits) && aligned16(target_bits) && (n_inputs <= 1 || n_words % 4 == 0);
  a.order = nullptr;
  if (order_blocks(n_progs, n_cases, sm_count())) {
    int32_t* order = nullptr;
    rc = get_order(w, (size_t)n_progs, s, &order);
    if (rc) return rc;
    e = launch_order_by_size(lengths, n_progs, order, s);
    if (e != cudaSuccess) return cuda_fail(e, "ordering launch");
    a.order = order;
  }
  const size_t tile_bytes = bool_tile_bytes(c.k, c.block, n_inputs);
  if (tile_bytes > kMaxTileBytes)
    return gp_fail(GP_ERR_INVALID_ARG, "%d inputs need %zu bytes of staged inputs per block (max %zu)",
                   n_inputs, tile_bytes, kMaxTileBytes);
  const size_t smem = prog_buffer_bytes(c.max_instructions) + tile_bytes;
  e = launch_bool(a, c.k, c.block, (int)(n_progs * n_chunks64), smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GP_OK;
}

extern "C" int gp_eval_population_bool(const uint32_t* programs, const int64_t* offsets,
                                       const int32_t* lengths, int32_t n_progs,
                                       const uint32_t* case_bits, int32_t n_inputs,
                                       int64_t n_cases, const uint32_t* target_bits,
                                       uint64_t* hits_out, gp_stream_t stream) {
  if (!hits_out) {
    gp_clear_error();
    return gp_fail(GP_ERR_INVALID_ARG, "null hits_out");
  }
  return gp_eval_population_bool_ex(programs, offsets, lengths, n_progs, case_bits, n_inputs,
                                    n_cases, target_bits, hits_out, nullptr, nullptr, stream);
}

extern "C" int gp_last_error(gp_stream_t stream, int32_t* status) {
  gp_clear_error();
  if (!status) return gp_fail(GP_ERR_INVALID_ARG, "null status");
  Workspace* w = nullptr;
  int rc = get_workspace((cudaStream_t)stream, 0, 0, &w);
  if (rc) return rc;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, w->status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->status, 0, sizeof(int), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
  *status = v;
  return GP_OK;
}

extern "C" int gp_shutdown(void) {
  gp_clear_error();
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (Workspace* w : g_ws) {
    cudaSetDevice(w->device);
    cudaStreamSynchronize(w->stream);
    if (w->partials) cudaFree(w->partials);
    if (w->counters) cudaFree(w->counters);
    if (w->order) cudaFree(w->order);
    if (w->status) cudaFree(w->status);
    delete w;
  }
  g_ws.clear();
  cudaSetDevice(cur);
  noalloc_forget_devices();
  return GP_OK;
}

extern "C" int gp_autotune_population(const uint32_t* programs, const int64_t* offsets,
                                      const int32_t* lengths, int32_t n_progs, const float* cases,
                                      int32_t n_inputs, int64_t n_cases, const float* targets,
                                      int32_t repeats, gp_config* best, gp_stream_t stream) {
  gp_clear_error();
  if (n_progs <= 0 || n_cases <= 0) return gp_fail(GP_ERR_INVALID_ARG, "nothing to tune on");
  if (repeats <= 0) repeats = 3;
  cudaStream_t s = (cudaStream_t)stream;
  double* fit = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&fit, sizeof(double) * (size_t)n_progs, s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune buffer");
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  gp_config best_c = {GP_VARIANT_REGISTER, 0, 0, 0};
  float best_ms = 1e30f;
  int rc = GP_OK;
  static const int ks[] = {2, 4, 8};
  static const int blocks[] = {64, 128, 256, 512};
  // cases per block: chosen, fixed sizes, or (-1) the whole case set, which
  // with the programs taken longest first often needs the fewest blocks
  static const int chunks[] = {0, 4096, 8192, 16384, 32768, -1};
  for (int k : ks) {
    for (int blk : blocks) {
     for (int ch0 : chunks) {
      int64_t ch = ch0;
      if (ch0 < 0) {
        ch = ((n_cases + k * blk - 1) / (k * blk)) * (k * blk);
        if (ch > 0x7fffffff || ch <= 32768) continue;  // (a 32-bit field; sizes above cover the rest)
      } else if (ch && (ch % (k * blk) || ch >= n_cases)) {
        continue;
      }
      gp_config c = {GP_VARIANT_REGISTER, k, blk, (int32_t)ch};
      rc = gp_eval_population_ex(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases,
                                 targets, fit, nullptr, &c, stream);
      if (rc) break;
      float ms_min = 1e30f;
      for (int r = 0; r < repeats && rc == GP_OK; ++r) {
        cudaEventRecord(t0, s);
        rc = gp_eval_population_ex(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases,
                                   targets, fit, nullptr, &c, stream);
        cudaEventRecord(t1, s);
        e = cudaEventSynchronize(t1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, t0, t1);
        ms_min = std::min(ms_min, ms);
      }
      if (rc) break;
      if (ms_min < best_ms) {
        best_ms = ms_min;
        best_c = c;
      }
     }
     if (rc) break;
    }
    if (rc) break;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFreeAsync(fit, s);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned[tune_key(n_inputs, n_cases, n_progs)] = best_c;
  }
  if (best) *best = best_c;
  return GP_OK;
}

extern "C" int gp_eval_launches(int32_t n_progs, int64_t n_cases, int32_t* launches) {
  gp_clear_error();
  if (!launches || n_progs < 0 || n_cases < 0) return gp_fail(GP_ERR_INVALID_ARG, "bad arguments");
  *launches = n_progs == 0 ? 0 : (order_blocks(n_progs, n_cases, sm_count()) ? 2 : 1);
  return GP_OK;
}

extern "C" int gp_autotune_clear(void) {
  gp_clear_error();
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuned.clear();
  return GP_OK;
}
