/*
 * gpeval.h -- C ABI of the GB300 (sm_103a) GP population evaluator.
 *
 * The library evaluates the fitness of whole populations of genetic-programming
 * programs on one GPU with the two-dimensional-stack interpreter of
 * D. M. Chitty, "Faster GPU Based Genetic Programming Using A Two Dimensional
 * Stack" (arXiv:1601.00221): every interpreter pass of a thread runs each
 * program step over K fitness cases at once (Sec. 4, Sec. 4.1), the program is
 * read warp-uniformly so opcode dispatch never diverges, and per-case errors
 * are reduced on the GPU into one fitness value per program.
 *
 * Conventions for every entry point below:
 *   - Return value: GP_OK (0) or one of the gp_status codes.  Argument errors
 *     are detected on the host before anything is launched.
 *   - "device" pointers must point to memory of the current CUDA device;
 *     "host" pointers to ordinary host memory.  The caller owns every buffer it
 *     passes; the library never frees or keeps a caller pointer after return.
 *   - Evaluation calls are asynchronous on `stream` (a cudaStream_t; 0 = the
 *     legacy default stream): results are valid once the stream has reached
 *     the call.  The library owns only an internal workspace per (device,
 *     stream), grown on demand and released by gp_shutdown().  Concurrent
 *     calls on one stream from several host threads are not supported; calls
 *     on different streams are independent.
 *   - A program that is malformed on the device side (an unknown instruction
 *     code, an input index >= n_inputs, a header that does not fit its length)
 *     yields fitness NaN (Boolean: hits UINT64_MAX) for that program only and
 *     sets the status word read by gp_last_error().
 */
#ifndef GPEVAL_H
#define GPEVAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gp_stream_t; /* same type as cudaStream_t */

typedef enum gp_status {
  GP_OK = 0,
  GP_ERR_INVALID_ARG = 1,     /* a null pointer, a negative size, an unknown enum */
  GP_ERR_PROGRAM = 2,         /* malformed program: bad token, missing operand, too deep */
  GP_ERR_CUDA = 3,            /* a CUDA runtime call failed (see gp_error_string) */
  GP_ERR_OOM = 4,             /* workspace or admission memory could not be had */
  GP_ERR_TIMEOUT = 5,         /* a bounded wait gave up */
  GP_ERR_NOT_IMPLEMENTED = 6,
  GP_ERR_BUSY = 7,            /* a serving queue is full, or a request is not finished yet */
  GP_ERR_CANCELLED = 8        /* a serving request was cancelled before it ran */
} gp_status;

/* ------------------------------------------------------------------------
 * User token format of a prefix tree (host memory), Sec. 3 / Sec. 5:
 * one uint32 per token, bits 0..7 opcode, bits 8..31 operand (the input index
 * of GP_OP_VAR).  A GP_OP_CONST token is followed by one word holding the
 * binary32 bit pattern of the constant.  GP_OP_DIV is protected division:
 * a denominator equal to zero (+0 or -0) gives 1.0f, otherwise the IEEE
 * binary32 quotient rounded to nearest even.  SUB(a,b) = a - b and
 * DIV(a,b) = a / b where a is the first child.  Boolean trees use VAR and the
 * bitwise functions AND, OR, NAND, NOR and IF(c,a,b) = (c&a)|(~c&b).
 *
 * Float trees may also use the rest of the function sets of the paper's float
 * problems (Sec. 4.2: sextic regression {*,/,+,-,Sin,Cos,Log,Exp}; Shuttle
 * {*,/,+,-,>,<,==,AND,OR,IF}; KDDcup all of them).  The paper names these
 * functions only; this library defines them as:
 *   SIN, COS, EXP  binary32 sine, cosine (radians), e^a: CUDA's sinf, cosf
 *                  and expf (documented maximum error 2 ulp each).
 *   LOG(a)         0 if a == 0 (either sign), else logf(|a|) (1 ulp).
 *   GT, LT, EQ     1.0f if a > b (a < b, a == b), else 0.0f; IEEE compares,
 *                  so a NaN operand gives 0.0f and -0 == +0.
 *   AND, OR        1.0f if a != 0 and (or) b != 0, else 0.0f; NaN != 0.
 *   IF(c, a, b)    a if c != 0, else b (NaN != 0 selects a).
 * A float tree that uses any of them needs GP_VARIANT_EXTENDED (S-form) or
 * GP_VARIANT_EXTENDED_RPN (RPN form); gp_prog_info.extended tells.
 * ---------------------------------------------------------------------- */
enum {
  GP_OP_ADD = 1, GP_OP_SUB = 2, GP_OP_MUL = 3, GP_OP_DIV = 4,
  GP_OP_VAR = 5, GP_OP_CONST = 6,
  GP_OP_AND = 7, GP_OP_OR = 8, GP_OP_NAND = 9, GP_OP_NOR = 10, GP_OP_IF = 11,
  GP_OP_SIN = 12, GP_OP_COS = 13, GP_OP_EXP = 14, GP_OP_LOG = 15,
  GP_OP_GT = 16, GP_OP_LT = 17, GP_OP_EQ = 18
};

/* Encoded program kinds (the interpreter a program is compiled for). */
typedef enum gp_kind {
  GP_KIND_SFORM = 1,  /* prefix linear "S-form" of a float tree (Sec. 5): one
                         instruction per function, operands input/constant/stack */
  GP_KIND_RPN = 2,    /* postfix reverse-Polish form of a float tree (Sec. 4, 4.1) */
  GP_KIND_LINEAR = 3, /* register linear GP r[d] = r[a] op r[b], 8 registers */
  GP_KIND_BOOL = 4,   /* S-form of a bit-packed Boolean tree (Sec. 4.2) */
  GP_KIND_SFORM_EXT = 5, /* written by the encoder, never requested: the S-form
                            of a float tree that uses the extended functions */
  GP_KIND_RPN_EXT = 6    /* likewise, the RPN form of such a tree */
} gp_kind;

/* Evaluation order of the children of a tree node when it is encoded. */
typedef enum gp_order {
  GP_ORDER_PAPER = 0,     /* children left to right, exactly as the paper's converter */
  GP_ORDER_MIN_DEPTH = 1  /* deeper-needing child first (Sethi-Ullman), fewest stack levels;
                             per-case values are bit-identical to GP_ORDER_PAPER */
} gp_order;

/* Number of stack levels the register interpreters hold (per case) and the
 * longest program (instructions) one interpreter pass accepts. */
#define GP_STACK_LEVELS 8
#define GP_MAX_INSTR 1024
#define GP_HEADER_WORDS 4
#define GP_INSTR_WORDS 4

typedef struct gp_prog_info {
  int32_t n_nodes;      /* tree nodes (functions + terminals): the GPop unit */
  int32_t n_instr;      /* interpreter instructions */
  int32_t max_depth;    /* stack levels used */
  int32_t stack_reads;  /* operands taken from the stack */
  int32_t max_input;    /* largest input index referenced, -1 if none */
  int32_t words;        /* encoded size in uint32 words */
  int32_t extended;     /* 1 if the tree uses SIN..EQ or float AND/OR/IF */
  int32_t inputs_used;  /* distinct input indices the tree reads */
} gp_prog_info;

/* ------------------------------------------------------------------------
 * Host encoder (Sec. 5: symbolic-stack conversion of an RPN tree to the
 * prefix linear form; host memory only, no CUDA calls).
 *
 * gp_encode_tree: encodes one prefix tree `prefix[0..n_words)` into `out`
 * (capacity `cap_words`) as kind `kind` (GP_KIND_SFORM, GP_KIND_RPN or
 * GP_KIND_BOOL) with child order `order`.  `info` (may be NULL) receives the
 * counts.  Returns GP_ERR_PROGRAM for a malformed tree or one that needs more
 * than GP_STACK_LEVELS levels or GP_MAX_INSTR instructions, GP_ERR_INVALID_ARG
 * if `out` is too small (info->words still tells the size needed).
 *
 * Encoded layout (uint32 words, every program a multiple of 4 words):
 *   header {kind | order<<8, n_instr, n_nodes, max_depth | (max_input+1)<<16}
 *   then n_instr instructions of 4 words {code, payload_a, payload_b, payload_c}.
 * ---------------------------------------------------------------------- */
int gp_encode_tree(const uint32_t* prefix, int64_t n_words, int32_t kind, int32_t order,
                   uint32_t* out, int64_t cap_words, gp_prog_info* info);

/* Encodes programs p = 0..n_progs-1, program p being
 * words[offsets[p] .. offsets[p] + lengths[p]).  With out == NULL only the
 * sizes are computed: *total_words receives the encoded size (a program never
 * takes more than 4 + 4 * lengths[p] words, so that bound can size `out` for
 * a single call).  Encoding runs on several host threads; the output is
 * identical to a sequential encoding.  Otherwise
 * out_offsets[p] / out_lengths[p] (host, n_progs entries each) receive the
 * encoded word offset and length of program p, *total_nodes the sum of nodes.
 * `info` (may be NULL) receives n_progs entries.  Stops at the first bad
 * program and reports its index in *bad_prog (may be NULL). */
int gp_encode_population(const uint32_t* words, const int64_t* offsets, const int32_t* lengths,
                         int32_t n_progs, int32_t kind, int32_t order, uint32_t* out,
                         int64_t cap_words, int64_t* out_offsets, int32_t* out_lengths,
                         int64_t* total_words, int64_t* total_nodes, gp_prog_info* info,
                         int32_t* bad_prog);

/* Register linear GP programs: instr[(offsets[p] + i)*4 + {0,1,2,3}] =
 * {dst, op, a, b} (registers 0..7, op GP_OP_ADD..GP_OP_DIV).  Same output
 * conventions as gp_encode_population; nodes = instructions.  An encoded
 * instruction is {code (function and operands), dst, flags, 0}; the flags
 * serve GP_VARIANT_REGISTER_FILE, which holds two values beside the register
 * file (the previous result, and the value its load rules last loaded):
 * bits 0-1 say where operand a is (0 the file, 1 the previous result, 2 the
 * loaded value), bits 2-3 the same for b (at most one of the two held),
 * bit 4 that the result is never read from the file and is not stored.  The
 * kernel checks the flags against the program and reports GP_ERR_PROGRAM for
 * flags that do not match; the register variant ignores them. */
int gp_encode_linear_population(const uint8_t* instr, const int64_t* offsets,
                                const int32_t* lengths, int32_t n_progs, uint32_t* out,
                                int64_t cap_words, int64_t* out_offsets, int32_t* out_lengths,
                                int64_t* total_words, int64_t* total_nodes, int32_t* bad_prog);

/* ------------------------------------------------------------------------
 * Evaluation configuration.  k = fitness cases per thread per interpreter pass
 * (the second dimension of the 2D stack, Sec. 4; 1 = the one-dimensional
 * stack); block = threads per block; chunk_cases = cases one block covers
 * (0 = choose); variant selects the interpreter.
 * ---------------------------------------------------------------------- */
typedef enum gp_variant {
  GP_VARIANT_AUTO = 0,      /* the tuned default for the workload */
  GP_VARIANT_REGISTER = 1,  /* stack levels in registers, K cases per thread */
  GP_VARIANT_LOCAL = 2,     /* BlockGP-style one-case-per-thread stack in local memory
                               (Sec. 3 prior art), GP_KIND_RPN and GP_KIND_RPN_EXT programs */
  GP_VARIANT_LANES = 3,     /* Boolean only: one program per lane over at most 4 words
                               (128 cases); taken when forced or when the tuner picks it */
  GP_VARIANT_EXTENDED = 4,  /* the S-form interpreter with the extended float functions
                               (runs GP_KIND_SFORM and GP_KIND_SFORM_EXT programs) */
  GP_VARIANT_EXTENDED_RPN = 5, /* the RPN interpreter with the extended float functions
                               (runs GP_KIND_RPN and GP_KIND_RPN_EXT programs) */
  GP_VARIANT_REGISTER_FILE = 6, /* GP_KIND_LINEAR programs only, their eight registers in shared
                               memory: one jump per instruction and a kernel of few
                               registers (blocks of at most 256 threads) */
  GP_VARIANT_WARPS = 7      /* Boolean only: one warp per program, block / 32 programs per
                               block sharing one staged copy of the case set (at most 256
                               threads; the case set and the block's programs must fit in
                               200 KB of shared memory); GP_VARIANT_AUTO picks it for 1 to
                               256 words (up to 8192 cases) */
} gp_variant;

/* Fitness measure of a float program (Sec. 4.2 parameter table: mean squared
 * error for regression, the number of incorrect classifications for
 * classification; the default is the sum of absolute errors). */
typedef enum gp_fitness {
  GP_FITNESS_SUM_ABS = 0,  /* sum over cases of |o - y| (binary32 error) */
  GP_FITNESS_MSE = 1,      /* (sum of d*d, d = o - y, binary32) / n_cases */
  GP_FITNESS_CLASS = 2     /* number of cases with rint(o) != y (y holds class labels) */
} gp_fitness;

typedef struct gp_config {
  int32_t variant;
  int32_t k;            /* 1, 2, 4 or 8 (0 = tuned) */
  int32_t block;        /* threads per block: a multiple of 32, at most 512 (256 for the
                           local-memory variant; Boolean launches use at most 256); 0 = tuned */
  int32_t chunk_cases;  /* 0 = choose; else a multiple of k*block */
  int32_t fitness;      /* gp_fitness (0 = GP_FITNESS_SUM_ABS) */
  int32_t tile_inputs;  /* inputs per case the shared-memory tile holds (0 = n_inputs).  A
                           tree stages only the inputs it reads, so the largest
                           gp_prog_info.inputs_used of the population is enough (a tree
                           reading more than 256 distinct inputs, or cases with more than
                           4096 inputs, stage every input; register programs need
                           min(n_inputs, 8)); a program that needs more fails as
                           malformed.  Smaller tiles leave room for more warps. */
  int32_t stack_registers; /* stack levels held in registers: 0 (or 8) = all; 4 = levels 4..7
                              in shared memory, fewer registers per thread (k = 8, the register
                              variant, GP_KIND_SFORM programs only; others fail as malformed) */
  int32_t max_instructions; /* instructions of the longest program (0 = GP_MAX_INSTR): each
                               block holds its program in shared memory, 16 bytes per
                               instruction, so a small buffer leaves room for more blocks; a
                               program with more instructions fails as malformed.  The
                               largest gp_prog_info.n_instr of the population is enough. */
} gp_config;

/* ------------------------------------------------------------------------
 * Float fitness of a population (device pointers).
 *   programs     encoded words (gp_encode_*), GP_KIND_SFORM, GP_KIND_RPN or
 *                GP_KIND_LINEAR, any mix (GP_VARIANT_EXTENDED: the S-form
 *                kinds only, GP_VARIANT_EXTENDED_RPN the RPN ones); offsets[p]
 *                (int64, multiple of
 *                4) and lengths[p] (int32) in words.
 *   cases        binary32 [n_inputs][n_cases], structure of arrays:
 *                input v of case c at cases[v * n_cases + c].
 *   targets      binary32 [n_cases].
 *   fitness_out  binary64 [n_progs]: sum over cases of |o - y| where each
 *                error is binary32 (Sec. 4.1 GetError; the paper leaves the
 *                error unstated, this library fixes the absolute error),
 *                accumulated with compensated binary32 sums per thread and
 *                summed in binary64 across blocks in a fixed order; +inf if any
 *                per-case error is not finite, NaN for a malformed program.
 *                With cfg->fitness = GP_FITNESS_MSE the binary64 sum of the
 *                binary32 squares d*d (d = o - y, binary32) divided by
 *                n_cases; GP_FITNESS_CLASS counts the cases whose output,
 *                rounded to the nearest integer (ties to even), differs from
 *                the target label (NaN never matches; never +inf).
 *                Accuracy: within 1e-5 relative of the same measure summed in
 *                binary64 over the binary32 per-case errors, and equal to it
 *                where that sum is 0 or +inf; classification counts exact.
 *                One case differs: when every per-case error is finite but a
 *                thread's binary32 sum passes the largest binary32 value, the
 *                fitness is +inf although the binary64 sum is finite.
 * The result depends only on (program, cases, config), never on what else
 * runs on the GPU.  n_cases may be 0 (fitness 0).  Sec. 4.1, Listing 1/2.
 * ---------------------------------------------------------------------- */
int gp_eval_population(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths,
                       int32_t n_progs, const float* cases, int32_t n_inputs, int64_t n_cases,
                       const float* targets, double* fitness_out, gp_stream_t stream);

/* As gp_eval_population with an explicit configuration (NULL = default).
 * `fitness_out` may be NULL; `outputs` (may be NULL) receives the per-case
 * program outputs, binary32 [n_progs][n_cases] (row p, column c). */
int gp_eval_population_ex(const uint32_t* programs, const int64_t* offsets,
                          const int32_t* lengths, int32_t n_progs, const float* cases,
                          int32_t n_inputs, int64_t n_cases, const float* targets,
                          double* fitness_out, float* outputs, const gp_config* cfg,
                          gp_stream_t stream);

/* Width split (many-input cases, Sec. 4.2's KDDcup shape): the staged-input
 * tile of a block is sized for the widest program, which limits the blocks
 * per multiprocessor for all.  Programs reading at most `split_inputs`
 * distinct inputs are evaluated under `narrow` (its tile: split_inputs when
 * narrow->tile_inputs is 0, at least split_inputs otherwise), every other
 * program under `wide`, in two launches over the same cases after a small
 * classification kernel on the device (asynchronous: the class sizes never
 * reach the host).  Each program's fitness is what gp_eval_population_ex
 * gives it under its class's configuration.  Tree variants only (register,
 * extended, extended RPN); n_inputs <= 4096 and n_progs <= 160000. */
int gp_eval_population_split(const uint32_t* programs, const int64_t* offsets,
                             const int32_t* lengths, int32_t n_progs, const float* cases,
                             int32_t n_inputs, int64_t n_cases, const float* targets,
                             double* fitness_out, int32_t split_inputs, const gp_config* narrow,
                             const gp_config* wide, gp_stream_t stream);

/* Per-case outputs only (parity testing): outputs[p * n_cases + c]. */
int gp_eval_outputs(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths,
                    int32_t n_progs, const float* cases, int32_t n_inputs, int64_t n_cases,
                    float* outputs, const gp_config* cfg, gp_stream_t stream);

/* ------------------------------------------------------------------------
 * Float fitness without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory -- for instance an application that gives the GPU's memory
 * to its own fixed-size pool, or an evaluation loop that must not meet an
 * allocation failure, or the synchronisation an allocation can imply, in the
 * middle of a run.  It takes gp_eval_population's arguments and runs what
 * gp_eval_population would run for them (the default configuration with its
 * variant and fitness measure, then the autotuner's record for the
 * workload's shape, the same kernel and the same split of the cases), but
 * keeps the kernel's scratch (per-block partial sums, per-program counters,
 * the block order, a status word) in a fixed array of about 1.5 MiB that
 * every device loading the library holds until the process exits; it never
 * calls cudaMalloc or cudaFree.
 *   - n_progs may be at most GP_NOALLOC_MAX_PARTIALS, n_cases at most 2^40;
 *     larger calls return GP_ERR_INVALID_ARG.  When that split of the cases
 *     would need more partial sums than the array holds (possible only with
 *     a recorded tuning of small chunks over many cases), the cases are split
 *     into fewer blocks and the fitness then agrees with gp_eval_population
 *     within the fitness tolerance (1e-5 relative) instead of bit for bit.
 *   - A width split the autotuner recorded for the shape (more than 16
 *     inputs) is not run: this entry point runs the recorded single-launch
 *     configuration, whose fitness agrees with the split's within the
 *     fitness tolerance (bit for bit under the classification measure).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and keeps it; make that
 *     first call before any stream capture.  gp_shutdown forgets the
 *     addresses: call it before a device reset (cudaDeviceReset) and the
 *     next call looks the address up again.
 *   - All calls on a device share the one array, which keeps the previous
 *     call's contents; each call clears the parts it relies on.  Calls whose
 *     work overlaps on the GPU (different streams, or host threads) race on
 *     the array: serialise them.
 *   - Malformed programs give NaN fitness as in gp_eval_population; the
 *     status word is not reported (gp_last_error does not see it).
 * ---------------------------------------------------------------------- */
#define GP_NOALLOC_MAX_PARTIALS 65536
int gp_eval_population_noalloc(const uint32_t* programs, const int64_t* offsets,
                               const int32_t* lengths, int32_t n_progs, const float* cases,
                               int32_t n_inputs, int64_t n_cases, const float* targets,
                               double* fitness_out, gp_stream_t stream);

/* ------------------------------------------------------------------------
 * Bit-packed Boolean fitness (Sec. 4.2: 32 fitness cases per 32-bit word,
 * sub-machine-code GP).  programs: GP_KIND_BOOL.  case_bits uint32
 * [n_inputs][ceil(n_cases/32)]: case c of input v is bit (c & 31) of word
 * case_bits[v * n_words + (c >> 5)].  target_bits uint32 [n_words].
 * hits_out uint64 [n_progs]: cases c < n_cases whose output bit equals the
 * target bit (bits beyond n_cases in the last word are ignored).  Exact.
 * By default case sets of up to 256 words run one warp per program
 * (GP_VARIANT_WARPS), larger ones the register variant's blocks, unless the
 * autotuner's record for the shape says otherwise (it also considers one
 * program per lane, GP_VARIANT_LANES, for up to 4 words).
 * ---------------------------------------------------------------------- */
int gp_eval_population_bool(const uint32_t* programs, const int64_t* offsets,
                            const int32_t* lengths, int32_t n_progs, const uint32_t* case_bits,
                            int32_t n_inputs, int64_t n_cases, const uint32_t* target_bits,
                            uint64_t* hits_out, gp_stream_t stream);

/* As gp_eval_population_bool with a configuration (NULL = default); hits_out
 * may be NULL; out_words (may be NULL) receives the output words
 * [n_progs][n_words] (bits beyond n_cases unspecified). */
int gp_eval_population_bool_ex(const uint32_t* programs, const int64_t* offsets,
                               const int32_t* lengths, int32_t n_progs,
                               const uint32_t* case_bits, int32_t n_inputs, int64_t n_cases,
                               const uint32_t* target_bits, uint64_t* hits_out,
                               uint32_t* out_words, const gp_config* cfg, gp_stream_t stream);

/* ------------------------------------------------------------------------
 * Several populations in one launch (device pointers; the segment table is
 * host memory).  The paper evaluates one population per generation (Sec. 4.2);
 * a service that interleaves the generations of many independent runs wants
 * the programs of all their pending requests -- uneven in number, length,
 * cases and inputs -- in one kernel launch.  Segment i is the programs
 * prog_begin .. prog_begin + n_progs - 1 of the shared programs / offsets /
 * lengths arrays, evaluated on its own cases and targets into its own `out`:
 *   kind GP_RUN_FLOAT  cases binary32 [n_inputs][n_cases], targets binary32
 *                      [n_cases], out binary64 fitness [n_progs] (the measure
 *                      of cfg->fitness); programs GP_KIND_SFORM, GP_KIND_RPN or
 *                      GP_KIND_LINEAR (the register variant's interpreters).
 *   kind GP_RUN_BOOL   cases uint32 [n_inputs][ceil(n_cases/32)], targets
 *                      uint32 [ceil(n_cases/32)], out uint64 hits [n_progs];
 *                      programs GP_KIND_BOOL (a warp per program).
 * `chunk` is the segment's cases (float) or words (Boolean) per block: 0 lets
 * the library choose from the segment alone, otherwise a multiple of
 * k * block.  Every segment uses cfg's k and block (the autotuner's records
 * are not applied).  A float segment's fitness is bit-identical to
 * gp_eval_population_ex on its programs alone with cfg and chunk_cases equal
 * to the segment's chunk, whatever else shares the launch (its cases are
 * split by its own chunk and summed in chunk order); Boolean hits are exact.
 * Blocks take the segments in order of decreasing chunk, and within a
 * segment its programs longest first once the launch fills two blocks per
 * multiprocessor.  At most GP_MAX_SEGMENTS segments; their program ranges
 * may not overlap.  Asynchronous on `stream`; the library's workspace as in
 * gp_eval_population.  Malformed programs: NaN fitness or UINT64_MAX hits.
 * ---------------------------------------------------------------------- */
enum { GP_RUN_FLOAT = 1, GP_RUN_BOOL = 2 };
#define GP_MAX_SEGMENTS 64
typedef struct gp_segment {
  int32_t prog_begin;
  int32_t n_progs;
  const void* cases;
  int32_t n_inputs;
  int32_t chunk;
  int64_t n_cases;
  const void* targets;
  void* out;
} gp_segment;

int gp_eval_segments(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths,
                     const gp_segment* segments, int32_t n_segments, int32_t kind,
                     const gp_config* cfg, gp_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: a continuously batched evaluation service for many independent GP
 * runs (the paper evaluates one population per generation, Sec. 4.2; a
 * server interleaves the generations of many runs).
 *
 * A run registers its fitness cases once; they stay resident on the device.
 * Each submitted request (one population of one run, encoded programs in
 * host memory) is queued, then admitted when an in-flight slot and enough of
 * the server's memory budget are free; consecutive queued requests of the
 * same run are merged into one launch; admitted work is spread over a pool
 * of CUDA streams, so requests of different runs overlap on the GPU.  A
 * host thread owned by the server issues the copies and launches and polls
 * CUDA events for completion: no kernel ever waits on the host.  The case
 * range of a run is split into blocks by its case count alone, so a
 * request's result is bit-identical whether it runs alone or in any mix.
 * All pointers here are host pointers.  Thread-safe: any host thread may
 * submit, poll, wait or cancel.
 * ---------------------------------------------------------------------- */
typedef struct gp_server gp_server;


typedef struct gp_server_opts {
  int32_t n_streams;      /* CUDA streams for admitted work (0 = 4) */
  int32_t max_inflight;   /* admitted launches at once (0 = 16) */
  int32_t max_queued;     /* requests waiting for admission (0 = 65536); more -> GP_ERR_BUSY */
  int32_t max_merge;      /* programs merged into one launch (0 = 65536) */
  int64_t memory_budget;  /* device bytes for admitted requests (0 = 1 GiB) */
  gp_config config;       /* kernel configuration (zero fields = library default) */
} gp_server_opts;

typedef struct gp_request_info {
  int32_t status;         /* GP_OK, or the error that ended the request */
  int32_t n_progs;
  int64_t gpop;           /* tree nodes x cases of the request */
  double t_submit_us;     /* server clock, microseconds since gp_server_create */
  double t_admit_us;
  double t_done_us;
} gp_request_info;

typedef struct gp_server_stats {
  int64_t submitted, completed, failed, cancelled, launches;
  int64_t gpop_completed;
  double p50_latency_us, p99_latency_us, max_latency_us; /* submission to completion */
  double busy_s;          /* wall time between the first admission and the last completion */
  double gpop_per_s;      /* gpop_completed / busy_s */
} gp_server_stats;

int gp_server_create(const gp_server_opts* opts, gp_server** out);

/* Copies a run's cases to the device.  GP_RUN_FLOAT: cases binary32
 * [n_inputs][n_cases], targets binary32 [n_cases].  GP_RUN_BOOL: cases uint32
 * [n_inputs][ceil(n_cases/32)], targets uint32 [ceil(n_cases/32)]. */
int gp_server_register_run(gp_server* srv, int32_t kind, const void* cases, int32_t n_inputs,
                           int64_t n_cases, const void* targets, int32_t* run_id);

/* Queues one population of encoded programs (copied before returning).
 * `result` (host, caller-owned until the request is done, cancelled or failed)
 * receives fitness as double[n_progs] (float runs) or hits as
 * uint64_t[n_progs] (Boolean runs).  `n_nodes` is the request's total tree
 * nodes (its GPop per case).  GP_ERR_BUSY when the queue is full, GP_ERR_OOM
 * when the request alone exceeds the memory budget. */
int gp_server_submit(gp_server* srv, int32_t run_id, const uint32_t* programs,
                     const int64_t* offsets, const int32_t* lengths, int32_t n_progs,
                     int64_t n_nodes, void* result, uint64_t* req_id);

/* GP_OK and *info when the request is finished (done, failed or cancelled);
 * GP_ERR_BUSY while it is queued or running. */
int gp_server_poll(gp_server* srv, uint64_t req_id, gp_request_info* info);

/* Blocks until the request is finished or `timeout_us` passes (GP_ERR_TIMEOUT). */
int gp_server_wait(gp_server* srv, uint64_t req_id, int64_t timeout_us, gp_request_info* info);

/* Cancels a request that is still queued (GP_OK); a request already admitted
 * runs to completion (GP_ERR_BUSY). */
int gp_server_cancel(gp_server* srv, uint64_t req_id);

int gp_server_get_stats(gp_server* srv, gp_server_stats* stats);

/* Waits for admitted work, drops queued requests (cancelled), frees everything. */
int gp_server_destroy(gp_server* srv);

/* ------------------------------------------------------------------------
 * Autotuning.  The best K (the second dimension of the 2D stack) and block
 * size depend on the hardware and the workload (Sec. 4.2: the paper's best K
 * and thread count differ per problem, Tables of Sec. 4.2, 5 and 6; Sec. 6.2
 * picks how many stack levels sit in registers per problem).
 *
 * gp_autotune_population_ex times candidate configurations of one kernel
 * family on the given float population with CUDA events on `stream` (one
 * warm-up launch, `repeats` timed launches each, the minimum kept), writes
 * the fastest to *best (may be NULL) and records it for the workload's shape.
 * `base` (NULL = the default configuration) gives the family -- its variant
 * -- and the fields that stay fixed: fitness measure, staged-input tile,
 * program buffer.  Candidates: k in {2, 4, 8} (k = 1 for the local-memory
 * variant) x block in {64, 128, 256, 512} (at most 256 where the variant
 * allows no more) x cases per block in {chosen, 4096, 8192, 16384, 32768,
 * 65536, 131072, all}; for the register variant also its register-file form
 * (GP_VARIANT_REGISTER_FILE) and, at k = 8, stack levels 4..7 in shared
 * memory (stack_registers = 4).  A candidate whose kernel cannot run every
 * program of the population (it reports a program error) or whose shape does
 * not fit is skipped.  Records are keyed by (family, single vs several
 * inputs, floor(log2 n_cases), floor(log2 n_progs)); a later float
 * evaluation of that family whose configuration leaves k and block at 0 takes
 * the record's k, block and (if 0) chunk, and, when its variant is
 * GP_VARIANT_AUTO or it passes no configuration, the record's variant and
 * stack levels too.  gp_autotune_population is the _ex call with base NULL.
 *
 * For a population of more than 16 inputs the float tuner also times the
 * width split (gp_eval_population_split): programs reading at most 6, 8, 12
 * or 16 inputs with a tile of that many inputs at k = 8 or 4 and block 256,
 * the others under the configuration it found.  When a split is more than
 * 2% faster it is recorded under the same key, and a later
 * gp_eval_population(_ex) of fitness (not outputs) whose configuration
 * leaves k and block at 0 runs it (with the caller's fitness measure,
 * program buffer and tile for the wide class); gp_autotune_split_record
 * reports it (split_inputs 0: none), and gp_eval_population_noalloc never
 * runs it.
 *
 * gp_autotune_population_bool does the same for a Boolean population:
 * k in {1, 2, 4, 8} x block in {32, 64, 128, 256} x cases per block, one
 * program per lane when the cases fit 4 words, and one warp per program
 * (k x block in {64, 128, 256}) when the case set fits the per-warp
 * variant's shared memory; the record applies to Boolean evaluations that
 * leave k and block at 0.
 *
 * The tuners synchronise `stream` and allocate a temporary output buffer.
 * gp_autotune_save writes every record to a text file (one line per record:
 * family, several, log2 n_cases, log2 n_progs, variant, k, block, chunk_cases,
 * stack_registers; a split record: "split", the key's four numbers,
 * split_inputs, then variant, k, block and chunk_cases of the narrow and of
 * the wide class); gp_autotune_load adds the records of such a file
 * (GP_ERR_INVALID_ARG for an unreadable file or a malformed line, which
 * loads nothing).  gp_autotune_clear forgets every record.
 * ---------------------------------------------------------------------- */
int gp_autotune_population(const uint32_t* programs, const int64_t* offsets,
                           const int32_t* lengths, int32_t n_progs, const float* cases,
                           int32_t n_inputs, int64_t n_cases, const float* targets,
                           int32_t repeats, gp_config* best, gp_stream_t stream);
int gp_autotune_population_ex(const uint32_t* programs, const int64_t* offsets,
                              const int32_t* lengths, int32_t n_progs, const float* cases,
                              int32_t n_inputs, int64_t n_cases, const float* targets,
                              const gp_config* base, int32_t repeats, gp_config* best,
                              gp_stream_t stream);
int gp_autotune_population_bool(const uint32_t* programs, const int64_t* offsets,
                                const int32_t* lengths, int32_t n_progs, const uint32_t* case_bits,
                                int32_t n_inputs, int64_t n_cases, const uint32_t* target_bits,
                                const gp_config* base, int32_t repeats, gp_config* best,
                                gp_stream_t stream);
int gp_autotune_split_record(int32_t family, int32_t n_inputs, int64_t n_cases, int32_t n_progs,
                             int32_t* split_inputs, gp_config* narrow, gp_config* wide);
int gp_autotune_save(const char* path);
int gp_autotune_load(const char* path);
int gp_autotune_clear(void);

/* Kernels one evaluation (gp_eval_population*, gp_eval_outputs,
 * gp_eval_population_noalloc, gp_eval_population_bool with the register or
 * per-warp variant) of n_progs programs over n_cases cases launches on the current
 * device: the interpreter, plus the ordering kernel that takes the programs
 * longest first once n_progs fills two blocks per multiprocessor and n_cases
 * is at least 16384.  (The Boolean variant with one program per lane launches
 * the interpreter alone.)  Writes the count to *launches.  Returns
 * GP_ERR_INVALID_ARG for a null pointer or a negative count. */
int gp_eval_launches(int32_t n_progs, int64_t n_cases, int32_t* launches);

/* ------------------------------------------------------------------------
 * Device-side encoder.  The S-form encoding of gp_encode_population (float
 * trees, basic or extended functions; Sec. 5 symbolic stack), run on the GPU
 * with one warp per tree, so that a generation loop needs no host
 * conversion between generations (the paper converts on the host, Sec. 5).
 * Output words are identical to gp_encode_population's for the same trees.
 *   words, offsets, lengths   device: the trees in the user token format.
 *   out, out_offsets          device: program p is written at
 *                             out[out_offsets[p] ..]; the slot must hold
 *                             4 + 4 * lengths[p] words (the same bound as on
 *                             the host) and start on a multiple of 4 words.
 *   out_lengths               device: the encoded length of each program.
 * Trees of at most GP_DEVICE_ENCODE_MAX_NODES nodes.  A malformed tree, a
 * larger one, or one that needs more than GP_STACK_LEVELS levels is written as
 * a 4-word header of kind 0, which every evaluation reports as malformed
 * (fitness NaN).  Asynchronous on `stream`.
 * ---------------------------------------------------------------------- */
#define GP_DEVICE_ENCODE_MAX_NODES 256
int gp_encode_population_device(const uint32_t* words, const int64_t* offsets,
                                const int32_t* lengths, int32_t n_progs, int32_t order,
                                uint32_t* out, const int64_t* out_offsets, int32_t* out_lengths,
                                gp_stream_t stream);

/* Slot offsets for gp_encode_population_device: out_offsets[p] (device) =
 * the sum over q < p of 4 + 4 * max(lengths[q], 0) words, the back-to-back
 * layout in which every program's slot holds its encoding.  lengths
 * (device) are the trees' word counts.  One small kernel, asynchronous on
 * `stream`, so that a captured generation step computes the layout on the
 * device.  Returns GP_ERR_INVALID_ARG for a negative count or a null array. */
int gp_encode_slots_device(const int32_t* lengths, int32_t n_progs, int64_t* out_offsets,
                           gp_stream_t stream);

/* ------------------------------------------------------------------------
 * On-device generation loop.  A GP run (Sec. 4.2 parameter table: population
 * 1000, tournament selection of size 7, crossover 0.95, mutation 0.2) evolves
 * the population on the GPU: each generation is one variation kernel
 * (selection, subtree crossover, subtree mutation; one thread per offspring),
 * the device encoder and the fitness evaluation, captured once as a CUDA
 * graph and replayed, with the cases resident.  The paper names the
 * operators only; this library defines them as:
 *   draws        Philox4x32-10 (Salmon et al., SC'11): offspring i of
 *                generation g reads the output words of the counters
 *                (i, g, 0, 0), (i, g, 1, 0), ... in order under the key
 *                (seed & 0xffffffff, seed >> 32).
 *   uniform(n)   (u * n) >> 32 of a draw u; an event of probability p happens
 *                when u < floor(p * 2^32) (capped at 2^32 - 1).
 *   tournament   `tournament` uniform picks; the first is the provisional
 *                winner and a later pick wins only with a strictly lower
 *                fitness (NaN counts as +inf).
 *   offspring    parent A by tournament; then with p_crossover parent B by
 *                tournament, a node of A and a node of B uniformly (prefix
 *                order) and the child is A with that subtree replaced by B's,
 *                or A if the result has more than max_nodes nodes; then with
 *                p_mutation a node of the child uniformly, replaced by a grown
 *                subtree, unless that exceeds max_nodes.
 *   grow(D)      a node at depth d (the root at 1) is a terminal if d >= D;
 *                otherwise, below the root, one draw makes it a terminal with
 *                probability 1/2; else a function uniformly from `funcs`,
 *                children grown at depth d + 1.  A terminal is a constant with
 *                probability p_const (a second draw u gives
 *                const_lo + (const_hi - const_lo) * ((u >> 8) * 2^-24), each
 *                step one binary32 operation), else an input uniformly.
 * max_nodes is at most 255, which keeps every tree within GP_STACK_LEVELS
 * register levels.  Generation 0 is the population given to
 * gp_evolve_create; each gp_evolve_run generation produces the next one and
 * its fitness.
 * ---------------------------------------------------------------------- */
typedef struct gp_evolve_params {
  int32_t pop_size;
  int32_t max_nodes;       /* tree size cap, 1..255 */
  int32_t tournament;      /* tournament size, >= 1 (the paper: 7) */
  float p_crossover;       /* the paper: 0.95 */
  float p_mutation;        /* the paper: 0.2 */
  int32_t mutation_depth;  /* depth cap D of a grown subtree, 1..4 */
  int32_t n_funcs;         /* 1..16 */
  int32_t funcs[16];       /* float function opcodes (GP_OP_ADD .. GP_OP_EQ, AND, OR, IF) */
  float p_const;           /* probability that a grown terminal is a constant */
  float const_lo, const_hi;
  uint64_t seed;
  gp_config eval;          /* evaluation: variant (GP_VARIANT_AUTO becomes
                              GP_VARIANT_EXTENDED when funcs has an extended
                              function), k, block, fitness, tile_inputs */
} gp_evolve_params;

typedef struct gp_evolver gp_evolver;

/* Creates a run: copies the initial population (host, user token format,
 * pop_size trees of at most max_nodes nodes) to the device, encodes and
 * evaluates it (generation 0) on `stream`.  cases / targets are device
 * arrays ([n_inputs][n_cases] and [n_cases]) that must stay valid and
 * unchanged until gp_evolve_destroy; grown inputs are drawn from
 * 0 .. n_inputs - 1.  The run owns its device buffers and its own stream. */
int gp_evolve_create(const gp_evolve_params* params, const uint32_t* words,
                     const int64_t* offsets, const int32_t* lengths, const float* cases,
                     int32_t n_inputs, int64_t n_cases, const float* targets,
                     gp_evolver** out);
/* Enqueues `generations` generations (graph replays); asynchronous. */
int gp_evolve_run(gp_evolver* ev, int32_t generations);
/* Waits for the run, then copies the current population (host: words with
 * room for pop_size * 2 * max_nodes words, tree p at p * 2 * max_nodes;
 * lengths pop_size), its fitness (pop_size doubles), the generation index and
 * the tree nodes evaluated so far over all generations (generation 0
 * included; times n_cases gives the GP operations).  Any pointer may be NULL. */
int gp_evolve_read(gp_evolver* ev, uint32_t* words, int32_t* lengths, double* fitness,
                   int32_t* generation, int64_t* nodes_evaluated);
int gp_evolve_destroy(gp_evolver* ev);

/* ------------------------------------------------------------------------
 * Configuration, status and lifetime.
 * ---------------------------------------------------------------------- */
/* Default configuration used when cfg is NULL or a field is 0.  Until it is
 * called, Boolean evaluations over 8 or more inputs that leave k or block at
 * 0 use k = 4 and blocks of at most 64 threads (their staged input tile
 * limits the blocks per multiprocessor); after it, its k and block stand.
 * gp_set_config(NULL) restores the library's own defaults (register variant,
 * k = 8, block 128, sum of absolute errors) and that Boolean rule. */
int gp_set_config(const gp_config* cfg);
int gp_get_config(gp_config* cfg);

/* Program-error status of the last evaluations on `stream`: synchronises the
 * stream, writes the status (0 = none, else a GP_ERR_* code) and clears it. */
int gp_last_error(gp_stream_t stream, int32_t* status);

/* Text of the last host-side error of the calling thread (never NULL). */
const char* gp_error_string(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t gp_version(void);

/* Releases every internal workspace of every device (synchronises them). */
int gp_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* GPEVAL_H */
