// api.cu -- the C ABI of include/gpeval.h: argument checks, the per-stream
// workspace, launch configuration and the evaluation entry points.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
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
// (kernel family, several inputs?, floor(log2 n_cases), floor(log2 n_progs)):
// the family is the configuration's variant before tuning (GP_VARIANT_AUTO
// counts as GP_VARIANT_REGISTER), kTuneBool for Boolean populations
using TuneKey = std::tuple<int, int, int, int>;
std::map<TuneKey, gp_config> g_tuned;
constexpr int kTuneBool = 100;
// width splits the float tuner found faster than one launch, by the same key:
// programs reading at most split_inputs inputs under `narrow`, the rest
// under `wide` (gp_eval_population_split)
struct SplitRec {
  int32_t split_inputs;
  gp_config narrow, wide;
};
std::map<TuneKey, SplitRec> g_split;
// programs the width split takes (its order buffer holds two classes)
constexpr int32_t kSplitMaxProgs = 160000;

int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) { v >>= 1; ++r; }
  return r;
}
TuneKey tune_key(int family, int32_t n_inputs, int64_t n_cases, int32_t n_progs) {
  if (family == GP_VARIANT_AUTO) family = GP_VARIANT_REGISTER;
  return TuneKey(family, n_inputs > 1 ? 1 : 0, ilog2(std::max<int64_t>(n_cases, 1)),
                 ilog2(std::max<int32_t>(n_progs, 1)));
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
      c->variant != GP_VARIANT_EXTENDED && c->variant != GP_VARIANT_EXTENDED_RPN &&
      c->variant != GP_VARIANT_REGISTER_FILE && c->variant != GP_VARIANT_WARPS)
    return gp_fail(GP_ERR_INVALID_ARG, "unknown variant %d", c->variant);
  if (c->fitness != GP_FITNESS_SUM_ABS && c->fitness != GP_FITNESS_MSE && c->fitness != GP_FITNESS_CLASS)
    return gp_fail(GP_ERR_INVALID_ARG, "unknown fitness measure %d", c->fitness);
  if (c->variant == GP_VARIANT_AUTO) c->variant = GP_VARIANT_REGISTER;
  if (c->k != 1 && c->k != 2 && c->k != 4 && c->k != 8)
    return gp_fail(GP_ERR_INVALID_ARG, "k must be 1, 2, 4 or 8 (got %d)", c->k);
  if (c->variant == GP_VARIANT_LOCAL) c->k = 1;
  if (c->block < 32 || c->block > 512 || c->block % 32)
    return gp_fail(GP_ERR_INVALID_ARG, "block must be a multiple of 32 in [32, 512] (got %d)", c->block);
  if (c->block > 256 && (c->variant == GP_VARIANT_LOCAL || c->variant == GP_VARIANT_REGISTER_FILE))
    return gp_fail(GP_ERR_INVALID_ARG, "the local-memory and register-file variants take at most 256 "
                                       "threads per block");
  if (c->chunk_cases < 0 || (c->chunk_cases % ((int64_t)c->k * c->block)) != 0)
    return gp_fail(GP_ERR_INVALID_ARG, "chunk_cases must be a multiple of k*block");
  return GP_OK;
}

// The autotuner's record for the workload, if any, fills the k and block
// fields the caller left at 0, and the chunk; when the caller left the
// variant to the library (no configuration, or GP_VARIANT_AUTO) also the
// variant and the stack levels held in registers the tuner chose.
void apply_tuned(const gp_config* user, gp_config* c, int32_t n_inputs, int64_t n_cases, int32_t n_progs) {
  if (user && user->k && user->block) return;
  const int family = (user && user->variant) ? user->variant : c->variant;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_tuned.find(tune_key(family, n_inputs, n_cases, n_progs));
  if (it == g_tuned.end()) return;
  if (!user || !user->k) c->k = it->second.k;
  if (!user || !user->block) c->block = it->second.block;
  if (!user || !user->chunk_cases) c->chunk_cases = it->second.chunk_cases;
  if (!user || user->variant == GP_VARIANT_AUTO) {
    c->variant = it->second.variant;
    c->stack_registers = it->second.stack_registers;
  }
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
  if (c.variant == GP_VARIANT_REGISTER_FILE) {  // the register files instead of input tiles
    if (c.stack_registers) return gp_fail(GP_ERR_INVALID_ARG, "the register-file variant has no stack");
    *smem = prog_buffer_bytes(c.max_instructions) + linear_rf_bytes(c.k, c.block);
    return GP_OK;
  }
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
  if (c.variant == GP_VARIANT_REGISTER_FILE) return launch_linear_rf(a, c.k, c.block, grid, smem, s);
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
  // a width split the tuner recorded for this shape, when the caller leaves
  // K and block to the library (fitness only; the caller's measure, program
  // buffer and wide tile)
  if (fitness_out && !outputs && (!cfg || (!cfg->k && !cfg->block))) {
    SplitRec rec;
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      auto it = g_split.find(tune_key((cfg && cfg->variant) ? cfg->variant : c.variant, n_inputs, n_cases, n_progs));
      if (it != g_split.end()) {
        rec = it->second;
        have = true;
      }
    }
    // (a population of the same key beyond the split's limits runs one launch)
    if (have && n_inputs > rec.split_inputs && n_inputs <= GP_COMPACT_MAX_INPUTS && n_progs <= kSplitMaxProgs) {
      for (gp_config* x : {&rec.narrow, &rec.wide}) {
        x->fitness = c.fitness;
        x->max_instructions = c.max_instructions;
      }
      rec.narrow.tile_inputs = rec.split_inputs;
      rec.wide.tile_inputs = c.tile_inputs;
      return gp_eval_population_split(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases, targets,
                                      fitness_out, rec.split_inputs, &rec.narrow, &rec.wide, stream);
    }
  }
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

  FloatArgs a{};
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

extern "C" int gp_eval_population_split(const uint32_t* programs, const int64_t* offsets,
                                        const int32_t* lengths, int32_t n_progs, const float* cases,
                                        int32_t n_inputs, int64_t n_cases, const float* targets,
                                        double* fitness_out, int32_t split_inputs, const gp_config* narrow,
                                        const gp_config* wide, gp_stream_t stream) {
  gp_clear_error();
  if (n_progs < 0 || n_inputs < 0 || n_cases < 0 || split_inputs < 0)
    return gp_fail(GP_ERR_INVALID_ARG, "negative size");
  if (!fitness_out) return gp_fail(GP_ERR_INVALID_ARG, "null fitness_out");
  if (n_progs == 0) return GP_OK;
  if (!programs || !offsets || !lengths) return gp_fail(GP_ERR_INVALID_ARG, "null program arrays");
  if (!aligned16(programs)) return gp_fail(GP_ERR_INVALID_ARG, "programs must be 16-byte aligned");
  if (n_cases > 0 && n_inputs > 0 && !cases) return gp_fail(GP_ERR_INVALID_ARG, "null cases");
  if (n_cases > 0 && !targets) return gp_fail(GP_ERR_INVALID_ARG, "null targets");
  if (n_cases > kMaxCases) return gp_fail(GP_ERR_INVALID_ARG, "n_cases too large");
  if (n_inputs > GP_COMPACT_MAX_INPUTS)
    return gp_fail(GP_ERR_INVALID_ARG, "the width split takes at most %d inputs", GP_COMPACT_MAX_INPUTS);
  if (n_progs > kSplitMaxProgs)
    return gp_fail(GP_ERR_INVALID_ARG, "the width split takes at most %d programs", kSplitMaxProgs);
  gp_config cls[2];
  const gp_config* user[2] = {narrow, wide};
  size_t smem[2];
  int64_t chunk[2], n_chunks[2];
  for (int c = 0; c < 2; ++c) {
    int rc = resolve_config(user[c], &cls[c]);
    if (rc) return rc;
    if (cls[c].variant == GP_VARIANT_REGISTER_FILE || cls[c].variant == GP_VARIANT_LOCAL)
      return gp_fail(GP_ERR_INVALID_ARG, "the width split takes the tree interpreters' variants");
    int32_t tile = (cls[c].tile_inputs > 0 && cls[c].tile_inputs < n_inputs) ? cls[c].tile_inputs : n_inputs;
    if (c == 0 && (!user[0] || user[0]->tile_inputs == 0)) tile = std::min(split_inputs, n_inputs);
    if (c == 0 && tile < std::min(split_inputs, n_inputs))
      return gp_fail(GP_ERR_INVALID_ARG, "the narrow class's tile must hold split_inputs inputs");
    cls[c].tile_inputs = tile;
    rc = float_launch_smem(cls[c], tile, &smem[c]);
    if (rc) return rc;
    const int per_pass = cls[c].k * cls[c].block;
    chunk[c] = choose_chunk(n_cases, n_progs, per_pass, cls[c].chunk_cases, kAutoBlocksPerSm);
    n_chunks[c] = std::max<int64_t>(1, (n_cases + chunk[c] - 1) / chunk[c]);
    if (n_chunks[c] * n_progs > 0x7fffffffLL) return gp_fail(GP_ERR_INVALID_ARG, "too many blocks");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t maxch = std::max(n_chunks[0], n_chunks[1]);
  Workspace* w = nullptr;
  int rc = get_workspace(s, maxch > 1 ? (size_t)(maxch * n_progs) : 0, maxch > 1 ? (size_t)n_progs : 0, &w);
  if (rc) return rc;
  int32_t* order = nullptr;
  rc = get_order(w, 2 * (size_t)n_progs + 2, s, &order);  // two classes, then their sizes
  if (rc) return rc;
  int32_t* counts = order + 2 * (size_t)n_progs;
  cudaError_t e = launch_split_by_inputs(programs, offsets, lengths, n_progs, n_inputs, split_inputs, order,
                                         counts, s);
  if (e != cudaSuccess) return cuda_fail(e, "width split launch");
  for (int c = 0; c < 2; ++c) {
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
    a.partials = w->partials;
    a.counters = w->counters;
    a.status = w->status;
    a.chunk_cases = chunk[c];
    a.n_chunks = (int32_t)n_chunks[c];
    a.x_aligned = aligned16(cases) && (n_inputs <= 1 || n_cases % 4 == 0);
    a.y_aligned = aligned16(targets);
    a.o_aligned = 0;
    a.want_fitness = 1;
    a.fitness_kind = cls[c].fitness;
    a.tile_inputs = cls[c].tile_inputs;
    a.prog_cap = cls[c].max_instructions;
    a.order = order + (size_t)c * n_progs;
    a.order_count = counts + c;
    // a grid for every program; the blocks past the class's size return at once
    e = launch_float_config(a, cls[c], n_inputs == 1, (int)(n_progs * n_chunks[c]), smem[c], s);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  }
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

namespace {
// case sets the per-warp variant takes by default (8192 cases)
constexpr int64_t kWarpsAutoWords = 256;

// The per-warp Boolean launch: k words per lane per pass (the caller's, the
// tuner's, else the fewest passes up to k = 8), block / 32 programs per block
// (the caller's, the tuner's, else 128 threads).
int eval_bool_warps(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths, int32_t n_progs,
                    const uint32_t* case_bits, int32_t n_inputs, int64_t n_cases, const uint32_t* target_bits,
                    uint64_t* hits_out, uint32_t* out_words, const gp_config* cfg, const gp_config* tuned,
                    gp_config c, cudaStream_t s) {
  const int64_t n_words = (n_cases + 31) / 32;
  if (n_words == 0) {  // no cases: every program scores 0 hits
    if (hits_out) {
      cudaError_t e = cudaMemsetAsync(hits_out, 0, sizeof(uint64_t) * (size_t)n_progs, s);
      if (e != cudaSuccess) return cuda_fail(e, "clearing hits");
    }
    return GP_OK;
  }
  if (!cfg || !cfg->k) c.k = tuned ? tuned->k : (n_words <= 32 ? 1 : n_words <= 64 ? 2 : n_words <= 128 ? 4 : 8);
  if (!cfg || !cfg->block) c.block = tuned ? tuned->block : 128;
  if (c.block > 256) return gp_fail(GP_ERR_INVALID_ARG, "the per-warp variant takes at most 256 threads per block");
  const size_t smem = bool_warps_smem(c.k, c.block, n_inputs, n_words, c.max_instructions);
  if (smem > kMaxTileBytes)
    return gp_fail(GP_ERR_INVALID_ARG, "%d inputs x %lld words need %zu bytes of shared memory per block (max %zu)",
                   n_inputs, (long long)n_words, smem, kMaxTileBytes);
  Workspace* w = nullptr;
  int rc = get_workspace(s, 0, 0, &w);
  if (rc) return rc;
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
  a.chunk_words = n_words;
  a.n_chunks = 1;
  a.aligned = aligned16(case_bits);
  a.prog_cap = c.max_instructions;
  a.order = nullptr;
  cudaError_t e;
  if (order_blocks(n_progs, n_cases, sm_count())) {
    int32_t* order = nullptr;
    rc = get_order(w, (size_t)n_progs, s, &order);
    if (rc) return rc;
    e = launch_order_by_size(lengths, n_progs, order, s);
    if (e != cudaSuccess) return cuda_fail(e, "ordering launch");
    a.order = order;
  }
  const int per_block = c.block / 32;
  e = launch_bool_warps(a, c.k, c.block, (n_progs + per_block - 1) / per_block, smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GP_OK;
}
}  // namespace

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
  // the autotuner's record for this shape, when the caller leaves k and block
  gp_config tuned{};
  bool have_tuned = false;
  if (!cfg || (!cfg->k && !cfg->block)) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(tune_key(kTuneBool, n_inputs, n_cases, n_progs));
    if (it != g_tuned.end()) {
      tuned = it->second;
      have_tuned = true;
    }
  }
  // program per lane when forced or tuned (a warp per program measured
  // faster by default, even on 2-word case sets: 6-input problems 2352 /
  // 2040 against 2194 / 1523 bit-GPop/s)
  const bool lanes = (cfg && cfg->variant == GP_VARIANT_LANES) ||
                     ((!cfg || cfg->variant == GP_VARIANT_AUTO) && have_tuned && tuned.variant == GP_VARIANT_LANES);
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
  // a warp per program for case sets of a few hundred words, unless a
  // variant is forced
  const bool warps = (cfg && cfg->variant == GP_VARIANT_WARPS) ||
                     ((!cfg || cfg->variant == GP_VARIANT_AUTO) &&
                      (have_tuned ? tuned.variant == GP_VARIANT_WARPS
                                  : (n_words > 0 && n_words <= kWarpsAutoWords)));
  if (warps)
    return eval_bool_warps(programs, offsets, lengths, n_progs, case_bits, n_inputs, n_cases, target_bits,
                           hits_out, out_words, cfg, have_tuned ? &tuned : nullptr, c, (cudaStream_t)stream);
  if (c.variant == GP_VARIANT_EXTENDED || c.variant == GP_VARIANT_EXTENDED_RPN)
    c.variant = GP_VARIANT_REGISTER;  // a float-only choice
  if (c.variant != GP_VARIANT_REGISTER)
    return gp_fail(GP_ERR_INVALID_ARG, "Boolean programs use the register, per-lane or per-warp variant");
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
  if (have_tuned) {
    c.k = tuned.k;
    c.block = tuned.block;
    if (!cfg || !cfg->chunk_cases) c.chunk_cases = tuned.chunk_cases;
  }
  if ((!cfg || !cfg->k) && !user_default && !have_tuned && n_inputs >= 8) c.k = 4;
  if ((!cfg || !cfg->block) && !have_tuned) {  // small case sets: do not launch idle warps
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

static_assert(kMaxSegments == GP_MAX_SEGMENTS, "the kernels' segment table holds GP_MAX_SEGMENTS");

extern "C" int gp_eval_segments(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths,
                                const gp_segment* segments, int32_t n_segments, int32_t kind,
                                const gp_config* cfg, gp_stream_t stream) {
  gp_clear_error();
  if (!segments || n_segments <= 0 || n_segments > GP_MAX_SEGMENTS)
    return gp_fail(GP_ERR_INVALID_ARG, "n_segments must be 1..%d (got %d)", GP_MAX_SEGMENTS, n_segments);
  if (kind != GP_RUN_FLOAT && kind != GP_RUN_BOOL) return gp_fail(GP_ERR_INVALID_ARG, "unknown kind %d", kind);
  const bool fl = kind == GP_RUN_FLOAT;
  gp_config c;
  int rc = resolve_config(cfg, &c);
  if (rc) return rc;
  if (!fl && (c.variant == GP_VARIANT_EXTENDED || c.variant == GP_VARIANT_EXTENDED_RPN)) c.variant = GP_VARIANT_REGISTER;
  if (c.variant != GP_VARIANT_REGISTER || c.stack_registers != 0)
    return gp_fail(GP_ERR_INVALID_ARG, "several populations in one launch run the register variant "
                                       "with every stack level in registers");
  if (!fl && c.block > 256) c.block = 256;  // the Boolean kernel's block limit
  const int per_pass = c.k * c.block;
  // segments in block order: decreasing chunk (the longer blocks first),
  // then the caller's order
  std::vector<int> idx;
  std::vector<int64_t> chunk_of(n_segments, 0);
  int64_t prog_end = 0;
  int32_t max_inputs = 0;
  bool all_single = true;
  for (int i = 0; i < n_segments; ++i) {
    const gp_segment& g = segments[i];
    if (g.prog_begin < 0 || g.n_progs < 0 || g.n_inputs < 0 || g.n_cases < 0 || g.chunk < 0)
      return gp_fail(GP_ERR_INVALID_ARG, "segment %d: negative field", i);
    if (g.n_cases > kMaxCases) return gp_fail(GP_ERR_INVALID_ARG, "segment %d: n_cases too large", i);
    if (g.n_progs == 0) continue;
    if (!g.out) return gp_fail(GP_ERR_INVALID_ARG, "segment %d: null out", i);
    if (g.n_cases > 0 && g.n_inputs > 0 && !g.cases) return gp_fail(GP_ERR_INVALID_ARG, "segment %d: null cases", i);
    if (g.n_cases > 0 && !g.targets) return gp_fail(GP_ERR_INVALID_ARG, "segment %d: null targets", i);
    const int64_t units = fl ? g.n_cases : (g.n_cases + 31) / 32;
    const int64_t ch = choose_chunk(units, g.n_progs, per_pass, g.chunk, fl ? kAutoBlocksPerSm : 48);
    if (ch % per_pass) return gp_fail(GP_ERR_INVALID_ARG, "segment %d: chunk must be a multiple of k*block", i);
    chunk_of[i] = ch;
    prog_end = std::max<int64_t>(prog_end, (int64_t)g.prog_begin + g.n_progs);
    max_inputs = std::max(max_inputs, g.n_inputs);
    all_single = all_single && g.n_inputs == 1;
    idx.push_back(i);
  }
  if (idx.empty()) return GP_OK;
  if (!programs || !offsets || !lengths) return gp_fail(GP_ERR_INVALID_ARG, "null program arrays");
  if (!aligned16(programs)) return gp_fail(GP_ERR_INVALID_ARG, "programs must be 16-byte aligned");
  if (prog_end > 0x7fffffffLL) return gp_fail(GP_ERR_INVALID_ARG, "program index out of range");
  {  // program ranges may not overlap
    std::vector<int> byp(idx);
    std::sort(byp.begin(), byp.end(), [&](int x, int y) { return segments[x].prog_begin < segments[y].prog_begin; });
    for (size_t j = 1; j < byp.size(); ++j)
      if ((int64_t)segments[byp[j - 1]].prog_begin + segments[byp[j - 1]].n_progs > segments[byp[j]].prog_begin)
        return gp_fail(GP_ERR_INVALID_ARG, "segments %d and %d overlap", byp[j - 1], byp[j]);
  }
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return chunk_of[x] > chunk_of[y]; });
  SegTable t;
  memset(&t, 0, sizeof t);
  t.n = (int32_t)idx.size();
  int64_t blocks = 0, partials = 0, progs = 0;
  for (int j = 0; j < t.n; ++j) {
    const gp_segment& g = segments[idx[j]];
    SegDesc& d = t.s[j];
    const int64_t units = fl ? g.n_cases : (g.n_cases + 31) / 32;
    d.cases = g.cases;
    d.targets = g.targets;
    d.out = g.out;
    d.n_cases = g.n_cases;
    d.n_units = units;
    d.chunk = chunk_of[idx[j]];
    d.n_inputs = g.n_inputs;
    d.prog_begin = g.prog_begin;
    d.n_progs = g.n_progs;
    const int64_t nch = std::max<int64_t>(1, (units + d.chunk - 1) / d.chunk);
    d.n_chunks = (int32_t)nch;
    if (blocks + nch * g.n_progs > 0x7fffffffLL) return gp_fail(GP_ERR_INVALID_ARG, "too many blocks");
    d.block_begin = (int32_t)blocks;
    blocks += nch * g.n_progs;
    d.partial_begin = partials;
    if (nch > 1) partials += nch * g.n_progs;
    progs += g.n_progs;
    if (fl)
      d.aligned = ((aligned16(g.cases) && (g.n_inputs <= 1 || g.n_cases % 4 == 0)) ? 1 : 0) |
                  (aligned16(g.targets) ? 2 : 0);
    else
      d.aligned = (aligned16(g.cases) && aligned16(g.targets) && (g.n_inputs <= 1 || units % 4 == 0)) ? 1 : 0;
  }
  size_t smem = 0;
  int32_t tile_inputs = max_inputs;
  if (fl) {
    if (c.tile_inputs > 0 && c.tile_inputs < max_inputs) tile_inputs = c.tile_inputs;
    rc = float_launch_smem(c, tile_inputs, &smem);
    if (rc) return rc;
  } else {
    const size_t tile_bytes = bool_tile_bytes(c.k, c.block, max_inputs);
    if (tile_bytes > kMaxTileBytes)
      return gp_fail(GP_ERR_INVALID_ARG, "%d inputs need %zu bytes of staged inputs per block (max %zu)",
                     max_inputs, tile_bytes, kMaxTileBytes);
    smem = prog_buffer_bytes(c.max_instructions) + tile_bytes;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  rc = get_workspace(s, fl ? (size_t)partials : 0, fl ? (size_t)prog_end : 0, &w);
  if (rc) return rc;
  int32_t* order = nullptr;
  if (progs >= (int64_t)kOrderMinProgsPerSm * sm_count()) {
    rc = get_order(w, (size_t)prog_end, s, &order);
    if (rc) return rc;
  }
  cudaError_t e;
  if (order || !fl) {
    e = launch_segment_prep(t, lengths, order, !fl, s);
    if (e != cudaSuccess) return cuda_fail(e, "segment preparation launch");
  }
  if (fl) {
    FloatArgs a;
    memset(&a, 0, sizeof a);
    a.programs = programs;
    a.offsets = offsets;
    a.lengths = lengths;
    a.n_progs = (int32_t)prog_end;
    a.partials = w->partials;
    a.counters = w->counters;
    a.status = w->status;
    a.n_chunks = 1;
    a.want_fitness = 1;
    a.fitness_kind = c.fitness;
    a.prog_cap = c.max_instructions;
    a.order = order;
    a.tile_inputs = tile_inputs;
    const bool xreg = all_single;
    if (c.k == 1) e = launch_float_seg_k1(a, t, xreg, c.block, (int)blocks, smem, s);
    else if (c.k == 2) e = launch_float_seg_k2(a, t, xreg, c.block, (int)blocks, smem, s);
    else if (c.k == 4) e = launch_float_seg_k4(a, t, xreg, c.block, (int)blocks, smem, s);
    else e = launch_float_seg_k8(a, t, xreg, c.block, (int)blocks, smem, s);
  } else {
    BoolArgs a;
    memset(&a, 0, sizeof a);
    a.programs = programs;
    a.offsets = offsets;
    a.lengths = lengths;
    a.n_progs = (int32_t)prog_end;
    a.n_inputs = max_inputs;
    a.status = w->status;
    a.n_chunks = 1;
    a.prog_cap = c.max_instructions;
    a.order = order;
    e = launch_bool_seg(a, t, c.k, c.block, (int)blocks, smem, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GP_OK;
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

namespace {

// Times `eval(c)` for every candidate (one warm-up launch, `repeats` timed
// launches each, the minimum kept) on `s`; candidates whose launch fails
// argument checks or that report a program error (a kernel that cannot run
// this population's programs) are skipped.  Synchronises `s`.
template <typename Eval>
int tune_over(const std::vector<gp_config>& cands, int repeats, cudaStream_t s, Eval eval, gp_config* best,
              float* best_ms) {
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  *best_ms = 1e30f;
  int rc = GP_OK;
  int32_t st = 0;
  gp_last_error((gp_stream_t)s, &st);  // (clears an earlier status)
  for (const gp_config& c : cands) {
    if (eval(c) != GP_OK) continue;  // this shape does not fit (tile, block limits)
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "autotune"); break; }
    st = 0;
    rc = gp_last_error((gp_stream_t)s, &st);
    if (rc) break;
    if (st != 0) continue;  // programs this kernel does not run
    float ms_min = 1e30f;
    for (int r = 0; r < repeats && rc == GP_OK; ++r) {
      cudaEventRecord(t0, s);
      rc = eval(c);
      cudaEventRecord(t1, s);
      e = cudaEventSynchronize(t1);
      if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, t0, t1);
      ms_min = std::min(ms_min, ms);
    }
    if (rc) break;
    if (ms_min < *best_ms) {
      *best_ms = ms_min;
      *best = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  gp_clear_error();
  if (rc == GP_OK && *best_ms >= 1e30f) rc = gp_fail(GP_ERR_INVALID_ARG, "no candidate configuration runs this population");
  return rc;
}

// cases (or words) per block tried besides the automatic choice: fixed
// sizes, and the whole set in one block when that is large
void add_chunks(std::vector<gp_config>& out, gp_config c, int64_t n_units) {
  static const int chunks[] = {0, 4096, 8192, 16384, 32768, 65536, 131072, -1};
  const int64_t per_pass = (int64_t)c.k * c.block;
  for (int ch0 : chunks) {
    int64_t ch = ch0;
    if (ch0 < 0) {  // the whole set in one block per program
      ch = ((n_units + per_pass - 1) / per_pass) * per_pass;
      if (ch > 0x7fffffff) continue;  // (a 32-bit field)
    } else if (ch && (ch % per_pass || ch >= n_units)) {
      continue;
    }
    c.chunk_cases = (int32_t)ch;
    out.push_back(c);
  }
}

}  // namespace

extern "C" int gp_autotune_population_ex(const uint32_t* programs, const int64_t* offsets,
                                         const int32_t* lengths, int32_t n_progs, const float* cases,
                                         int32_t n_inputs, int64_t n_cases, const float* targets,
                                         const gp_config* base, int32_t repeats, gp_config* best,
                                         gp_stream_t stream) {
  gp_clear_error();
  if (n_progs <= 0 || n_cases <= 0) return gp_fail(GP_ERR_INVALID_ARG, "nothing to tune on");
  if (repeats <= 0) repeats = 3;
  gp_config b;
  int rc = resolve_config(base, &b);
  if (rc) return rc;
  const int family = (base && base->variant) ? base->variant : b.variant;
  cudaStream_t s = (cudaStream_t)stream;
  double* fit = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&fit, sizeof(double) * (size_t)n_progs, s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune buffer");
  // candidates: k x block x chunk within the family; for the register
  // variant also its register-file form (register programs) and, at k = 8,
  // stack levels 4..7 in shared memory (S-form programs); a candidate whose
  // kernel cannot run every program reports a program error and is skipped
  std::vector<gp_config> cands;
  std::vector<int> variants{b.variant};
  if (b.variant == GP_VARIANT_REGISTER) variants.push_back(GP_VARIANT_REGISTER_FILE);
  for (int v : variants) {
    const bool one_case = v == GP_VARIANT_LOCAL;
    const int max_block = (v == GP_VARIANT_LOCAL || v == GP_VARIANT_REGISTER_FILE) ? 256 : 512;
    for (int k : {1, 2, 4, 8}) {
      if (one_case != (k == 1)) continue;
      for (int blk : {64, 128, 256, 512}) {
        if (blk > max_block) continue;
        for (int rl : {0, 4}) {
          if (rl && (v != GP_VARIANT_REGISTER || k != 8)) continue;
          gp_config c = b;
          c.variant = v;
          c.k = k;
          c.block = blk;
          c.stack_registers = rl;
          add_chunks(cands, c, n_cases);
        }
      }
    }
  }
  auto eval = [&](const gp_config& c) {
    return gp_eval_population_ex(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases, targets, fit,
                                 nullptr, &c, stream);
  };
  gp_config best_c = b;
  float best_ms = 0;
  rc = tune_over(cands, repeats, s, eval, &best_c, &best_ms);
  if (rc) {
    cudaFreeAsync(fit, s);
    return rc;
  }
  // Many inputs: also the width split -- programs reading at most `th`
  // inputs with a th-input tile and their own K, block and chunk, the rest
  // under the configuration just found (a split candidate is a gp_config
  // whose tile_inputs holds th and whose k, block and chunk are the narrow
  // class's)
  SplitRec split{0, best_c, best_c};
  const bool tree_family = best_c.variant == GP_VARIANT_REGISTER || best_c.variant == GP_VARIANT_EXTENDED ||
                           best_c.variant == GP_VARIANT_EXTENDED_RPN;
  if (tree_family && n_inputs > 16 && n_inputs <= GP_COMPACT_MAX_INPUTS && n_progs <= kSplitMaxProgs &&
      best_c.stack_registers == 0) {
    std::vector<gp_config> scands;
    for (int th : {6, 8, 12, 16})
      for (int k : {8, 4})
        for (int64_t ch : {(int64_t)0, (int64_t)65536, (int64_t)131072}) {
          if (ch >= n_cases && ch > 0) continue;  // (the automatic chunk covers it)
          gp_config c = best_c;
          c.k = k;
          c.block = 256;
          c.chunk_cases = (int32_t)ch;
          c.tile_inputs = th;
          scands.push_back(c);
        }
    // the wide class holds few programs, so it may want shorter chunks than
    // the single launch (more blocks to fill the GPU): its chunk is tried too
    float split_ms = 1e30f;
    std::vector<int64_t> wchunks{best_c.chunk_cases};
    for (int64_t wch : {(int64_t)65536, (int64_t)32768})
      if (wch != best_c.chunk_cases && wch % ((int64_t)best_c.k * best_c.block) == 0 && wch < n_cases)
        wchunks.push_back(wch);
    for (int64_t wch : wchunks) {
      gp_config wide = best_c;
      wide.chunk_cases = (int32_t)wch;
      auto eval_split = [&](const gp_config& c) {
        return gp_eval_population_split(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases, targets,
                                        fit, c.tile_inputs, &c, &wide, stream);
      };
      gp_config sb = best_c;
      float sms = 0;
      // (a shape that cannot run is skipped; none running leaves the single launch)
      if (tune_over(scands, repeats, s, eval_split, &sb, &sms) == GP_OK && sms < split_ms) {
        split_ms = sms;
        split.split_inputs = sb.tile_inputs;
        split.narrow = sb;
        split.wide = wide;
      }
    }
    if (!(split_ms < 0.98f * best_ms)) split.split_inputs = 0;
    gp_clear_error();
  }
  cudaFreeAsync(fit, s);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const TuneKey key = tune_key(family, n_inputs, n_cases, n_progs);
    g_tuned[key] = best_c;
    if (split.split_inputs > 0) g_split[key] = split;
    else g_split.erase(key);
  }
  if (best) *best = best_c;
  return GP_OK;
}

extern "C" int gp_autotune_split_record(int32_t family, int32_t n_inputs, int64_t n_cases, int32_t n_progs,
                                        int32_t* split_inputs, gp_config* narrow, gp_config* wide) {
  gp_clear_error();
  if (!split_inputs) return gp_fail(GP_ERR_INVALID_ARG, "null split_inputs");
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_split.find(tune_key(family, n_inputs, n_cases, n_progs));
  *split_inputs = it == g_split.end() ? 0 : it->second.split_inputs;
  if (it != g_split.end()) {
    if (narrow) *narrow = it->second.narrow;
    if (wide) *wide = it->second.wide;
  }
  return GP_OK;
}

extern "C" int gp_autotune_population(const uint32_t* programs, const int64_t* offsets,
                                      const int32_t* lengths, int32_t n_progs, const float* cases,
                                      int32_t n_inputs, int64_t n_cases, const float* targets,
                                      int32_t repeats, gp_config* best, gp_stream_t stream) {
  return gp_autotune_population_ex(programs, offsets, lengths, n_progs, cases, n_inputs, n_cases, targets,
                                   nullptr, repeats, best, stream);
}

extern "C" int gp_autotune_population_bool(const uint32_t* programs, const int64_t* offsets,
                                           const int32_t* lengths, int32_t n_progs, const uint32_t* case_bits,
                                           int32_t n_inputs, int64_t n_cases, const uint32_t* target_bits,
                                           const gp_config* base, int32_t repeats, gp_config* best,
                                           gp_stream_t stream) {
  gp_clear_error();
  if (n_progs <= 0 || n_cases <= 0) return gp_fail(GP_ERR_INVALID_ARG, "nothing to tune on");
  if (repeats <= 0) repeats = 3;
  gp_config b;
  int rc = resolve_config(base, &b);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* hits = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&hits, sizeof(uint64_t) * (size_t)n_progs, s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune buffer");
  const int64_t n_words = (n_cases + 31) / 32;
  std::vector<gp_config> cands;
  if (n_words <= 4) {  // one program per lane
    gp_config c = b;
    c.variant = GP_VARIANT_LANES;
    cands.push_back(c);
  }
  for (int k : {1, 2, 4, 8})
    for (int blk : {32, 64, 128, 256}) {
      gp_config c = b;
      c.variant = GP_VARIANT_REGISTER;
      c.k = k;
      c.block = blk;
      c.stack_registers = 0;
      add_chunks(cands, c, n_words);
    }
  for (int k : {1, 2, 4, 8})  // a warp per program, where the case set fits its shared memory
    for (int blk : {64, 128, 256}) {
      if (bool_warps_smem(k, blk, n_inputs, n_words, b.max_instructions) > kMaxTileBytes) continue;
      gp_config c = b;
      c.variant = GP_VARIANT_WARPS;
      c.k = k;
      c.block = blk;
      c.chunk_cases = 0;
      c.stack_registers = 0;
      cands.push_back(c);
    }
  auto eval = [&](const gp_config& c) {
    return gp_eval_population_bool_ex(programs, offsets, lengths, n_progs, case_bits, n_inputs, n_cases,
                                      target_bits, hits, nullptr, &c, stream);
  };
  gp_config best_c = b;
  float best_ms = 0;
  rc = tune_over(cands, repeats, s, eval, &best_c, &best_ms);
  cudaFreeAsync(hits, s);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned[tune_key(kTuneBool, n_inputs, n_cases, n_progs)] = best_c;
  }
  if (best) *best = best_c;
  return GP_OK;
}

extern "C" int gp_autotune_save(const char* path) {
  gp_clear_error();
  if (!path) return gp_fail(GP_ERR_INVALID_ARG, "null path");
  FILE* f = fopen(path, "w");
  if (!f) return gp_fail(GP_ERR_INVALID_ARG, "cannot write %s", path);
  std::lock_guard<std::mutex> lk(g_mu);
  fprintf(f, "# gpeval autotune v1: family several log2_cases log2_progs variant k block chunk_cases "
             "stack_registers\n");
  fprintf(f, "# split family several log2_cases log2_progs split_inputs  narrow: variant k block chunk_cases  "
             "wide: variant k block chunk_cases\n");
  for (const auto& kv : g_tuned) {
    const gp_config& c = kv.second;
    fprintf(f, "%d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
            std::get<2>(kv.first), std::get<3>(kv.first), c.variant, c.k, c.block, c.chunk_cases,
            c.stack_registers);
  }
  for (const auto& kv : g_split) {
    const SplitRec& r = kv.second;
    fprintf(f, "split %d %d %d %d %d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
            std::get<2>(kv.first), std::get<3>(kv.first), r.split_inputs, r.narrow.variant, r.narrow.k,
            r.narrow.block, r.narrow.chunk_cases, r.wide.variant, r.wide.k, r.wide.block, r.wide.chunk_cases);
  }
  const bool ok = fclose(f) == 0;
  return ok ? GP_OK : gp_fail(GP_ERR_INVALID_ARG, "cannot write %s", path);
}

extern "C" int gp_autotune_load(const char* path) {
  gp_clear_error();
  if (!path) return gp_fail(GP_ERR_INVALID_ARG, "null path");
  FILE* f = fopen(path, "r");
  if (!f) return gp_fail(GP_ERR_INVALID_ARG, "cannot read %s", path);
  std::vector<std::pair<TuneKey, gp_config>> recs;
  std::vector<std::pair<TuneKey, SplitRec>> splits;
  char line[512];
  int rc = GP_OK, ln = 0;
  while (fgets(line, sizeof line, f)) {
    ++ln;
    if (line[0] == '#' || line[0] == '\n') continue;
    if (strncmp(line, "split", 5) == 0) {
      int fam, sev, lc, lp, th, nv, nk, nb, nch, wv, wk, wb, wch;
      if (sscanf(line + 5, "%d %d %d %d %d %d %d %d %d %d %d %d %d", &fam, &sev, &lc, &lp, &th, &nv, &nk, &nb,
                 &nch, &wv, &wk, &wb, &wch) != 13 || th <= 0) {
        rc = gp_fail(GP_ERR_INVALID_ARG, "%s line %d: expected 'split' and 13 integers", path, ln);
        break;
      }
      SplitRec r{th, kLibraryDefault, kLibraryDefault};
      r.narrow.variant = nv;
      r.narrow.k = nk;
      r.narrow.block = nb;
      r.narrow.chunk_cases = nch;
      r.wide.variant = wv;
      r.wide.k = wk;
      r.wide.block = wb;
      r.wide.chunk_cases = wch;
      gp_config chk;
      if (resolve_config(&r.narrow, &chk) != GP_OK || resolve_config(&r.wide, &chk) != GP_OK) {
        rc = gp_fail(GP_ERR_INVALID_ARG, "%s line %d: not a valid configuration", path, ln);
        break;
      }
      splits.emplace_back(TuneKey(fam, sev, lc, lp), r);
      continue;
    }
    int fam, sev, lc, lp, var, k, blk, ch, sr;
    if (sscanf(line, "%d %d %d %d %d %d %d %d %d", &fam, &sev, &lc, &lp, &var, &k, &blk, &ch, &sr) != 9) {
      rc = gp_fail(GP_ERR_INVALID_ARG, "%s line %d: expected 9 integers", path, ln);
      break;
    }
    gp_config c = kLibraryDefault;
    c.variant = var;
    c.k = k;
    c.block = blk;
    c.chunk_cases = ch;
    c.stack_registers = sr;
    gp_config chk;
    if (resolve_config(&c, &chk) != GP_OK) {
      rc = gp_fail(GP_ERR_INVALID_ARG, "%s line %d: not a valid configuration", path, ln);
      break;
    }
    recs.emplace_back(TuneKey(fam, sev, lc, lp), c);
  }
  fclose(f);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : recs) g_tuned[r.first] = r.second;
  for (auto& r : splits) g_split[r.first] = r.second;
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
  g_split.clear();
  return GP_OK;
}
