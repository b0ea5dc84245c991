// config.h -- the float evaluation's configuration and launch choices, shared
// by the entry points of api.cu and the allocation-free entry point of
// noalloc.cu, so that both run the same kernel with the same shape.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gpeval.h"
#include "launch.h"

namespace gpdev {

// multiprocessors of the device current at the first call
int sm_count();
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
// dynamic shared memory left for staged input tiles next to the program
// buffer (227 KB per block on sm_103a)
constexpr size_t kMaxTileBytes = 200 * 1024;
// the largest case count an evaluation accepts
constexpr int64_t kMaxCases = (int64_t)1 << 40;

// Fills the zero fields of `user` (may be null) from the default
// configuration and checks the result.
int resolve_config(const gp_config* user, gp_config* c);
// The autotuner's record for the workload, if any, fills the k, block and
// chunk fields the caller left at 0 (register variant only).
void apply_tuned(const gp_config* user, gp_config* c, int32_t n_inputs, int64_t n_cases, int32_t n_progs);
// Cases (or words) per block: user_chunk if set, else enough blocks to fill
// the GPU blocks_per_sm times over, whole passes of the block each.
int64_t choose_chunk(int64_t n_units, int32_t n_progs, int per_pass, int64_t user_chunk, int blocks_per_sm);
// Dynamic shared memory of a float launch under `c` with `tile_inputs`
// staged inputs (program buffer, tiles, shared stack levels); GP_OK or
// GP_ERR_INVALID_ARG when the tile does not fit.
int float_launch_smem(const gp_config& c, int32_t tile_inputs, size_t* smem);
// Launches the float interpreter `c` selects (variant, k, stack levels).
cudaError_t launch_float_config(const FloatArgs& a, const gp_config& c, bool xreg, int grid, size_t smem,
                                cudaStream_t s);
// Forgets the allocation-free entry point's per-device scratch addresses
// (gp_shutdown).
void noalloc_forget_devices();

}  // namespace gpdev
