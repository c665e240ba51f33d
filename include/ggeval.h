/*
 * ggeval: batched fitness evaluation of GP-GOMEA trial solutions on one
 * NVIDIA GB300 (sm_103a).
 *
 * The paper ("GP-GOMEA with GPU-Based Fitness Evaluations") restructures
 * gene-pool optimal mixing so that every offspring changed in one FOS step
 * is evaluated together (Algorithm 1, the GPU-side Evaluate(O[changed])
 * call); it linearises each template tree to RPN with introns dropped
 * (Section 3.2, Fig. 1) and evaluates the batch on the GPU, returning one
 * fitness per trial to the host (Section 3.2, "Evaluation on the GPU").
 * This C ABI is that Evaluate call.  Fitness is linearly scaled MSE
 * (least-squares a, b), with the paper's plain MSE (Eq. 1) returned beside
 * it; a reverse-mode adjoint gives the gradient of either in every ERC.
 *
 * Conventions shared by every entry point
 *  - Every call returns a ggeval_status; on failure ggeval_last_error()
 *    returns a thread-local message.  Argument errors are reported
 *    synchronously and leave every output untouched.
 *  - GPU work is enqueued on the caller's CUDA stream (cudaStream_t passed
 *    as void*; NULL = legacy default stream) and is asynchronous: outputs
 *    are valid once that stream has reached the call's end.  Call
 *    ggeval_sync() to wait and to collect device-side errors.
 *  - Device-side errors (an invalid template in a device-memory batch, a
 *    bounded wait that gave up) are recorded in a per-dataset status word,
 *    reported and cleared by ggeval_sync().  An invalid trial gets NaN in
 *    every output; the other trials are unaffected.
 *  - A non-finite fitness is a value, not an error: a trial whose output
 *    is non-finite, or exceeds 2^50 in magnitude, at any row gets +inf
 *    smse and mse, a = b = 0 and a zero gradient.
 *  - Buffers passed in are borrowed: the caller owns them and keeps them
 *    alive until the stream work completes.  The dataset owns its copies
 *    of X and y and a workspace that grows on demand (the growing call
 *    allocates with cudaMalloc, so call once with the largest batch before
 *    capturing the stream in a CUDA graph).
 *  - A dataset is used from one host thread at a time.
 */
#ifndef GGEVAL_H
#define GGEVAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ggeval_dataset ggeval_dataset;

typedef enum {
  GGEVAL_OK = 0,
  GGEVAL_ERR_ARG = -1,         /* bad argument (null pointer, size, range)   */
  GGEVAL_ERR_TEMPLATE = -2,    /* a trial's template is invalid              */
  GGEVAL_ERR_CUDA = -3,        /* a CUDA runtime call failed                 */
  GGEVAL_ERR_OOM = -4,         /* device allocation failed                   */
  GGEVAL_ERR_TIMEOUT = -5,     /* a bounded device wait gave up              */
  GGEVAL_ERR_CHECKED = -6,     /* bounds check failed (checked build only)   */
  GGEVAL_ERR_UNSUPPORTED = -7  /* size beyond what this build supports       */
} ggeval_status;

/* Template layouts.  A trial of height h has 2^(h+1)-1 nodes of arity 2.
 * HEAP: node i has children 2i+1 and 2i+2.  PREFIX: pre-order of the full
 * template, so a node at position p whose subtree has height s has children
 * p+1 and p+2^s.  (Section 3.1: an individual is a fixed-length string of
 * variables mapped onto a fixed tree template.) */
enum { GGEVAL_LAYOUT_HEAP = 0, GGEVAL_LAYOUT_PREFIX = 1 };

/* Where a batch's arrays live.  HOST batches are copied to the device by
 * the call (inside the stream work); their outputs are host memory written
 * by a device-to-host copy on the stream.  Use pinned host memory for
 * asynchronous copies. */
enum { GGEVAL_MEM_DEVICE = 0, GGEVAL_MEM_HOST = 1 };

/* Template node opcodes (one uint8 per node).
 * Functions: binary operands are (left child, right child); a unary
 * function reads its left child and its right subtree is an intron.
 * AQ(a, b) = a / sqrt(1 + b^2) (analytic quotient).  DIV, SQUARE, LOG,
 * SQRT and POW are the paper's Table 2 operators (plain division, x^2,
 * unprotected log and sqrt, and pow(left, right) = left^right with the C99
 * powf special cases: NaN, so +inf fitness, for a negative base and a
 * non-integer exponent).  Terminals: ERC reads the node's constant from cval;
 * FEATURE0 + k reads feature k (k < n_features).  The root is active; the
 * children of an active function are active (only the left child of a
 * unary one); a terminal's subtree is an intron.  Introns may hold any
 * byte; an active node must be one of the codes below, and an active
 * function must not sit at a leaf position (Fig. 1 shows a multiplication
 * at a leaf as an intron). */
enum {
  GGEVAL_OP_ADD = 0, GGEVAL_OP_SUB = 1, GGEVAL_OP_MUL = 2, GGEVAL_OP_AQ = 3,
  GGEVAL_OP_SIN = 4, GGEVAL_OP_COS = 5, GGEVAL_OP_EXP = 6,
  GGEVAL_OP_LOG_ABS = 7, GGEVAL_OP_SQRT_ABS = 8,
  GGEVAL_OP_DIV = 9, GGEVAL_OP_SQUARE = 10, GGEVAL_OP_LOG = 11, GGEVAL_OP_SQRT = 12,
  GGEVAL_OP_POW = 13,
  GGEVAL_OP_ERC = 31,
  GGEVAL_OP_FEATURE0 = 32,
  GGEVAL_OP_PAD = 255
};

/* Largest template height this build evaluates (511 nodes, the paper's
 * depth-8 templates of Table 2) and the largest feature count. */
#define GGEVAL_MAX_HEIGHT 8
#define GGEVAL_MAX_FEATURES 223

/* One FOS step's trials (the batch O[changed] of Algorithm 1).
 * op and cval are [n][stride] row-major with stride = 2^(max_height+1)-1;
 * trial p of height h_p uses its first 2^(h_p+1)-1 entries.  height is
 * int8 [n] (each 0..max_height) or NULL for "all max_height".  All three
 * live in `memory`. */
typedef struct {
  int32_t n;           /* number of trials, >= 0                          */
  int32_t max_height;  /* 0..GGEVAL_MAX_HEIGHT                            */
  int32_t layout;      /* GGEVAL_LAYOUT_*                                 */
  int32_t memory;      /* GGEVAL_MEM_*                                    */
  const uint8_t* op;
  const float* cval;
  const int8_t* height;
} ggeval_batch;

/* Flags for the evaluation calls. */
enum {
  GGEVAL_F_GRAPH = 1u << 0,   /* replay (or capture once) the call's launch
                                 sequence as a CUDA graph, keyed on every
                                 argument value; needs a device batch      */
  GGEVAL_F_EXACT = 1u << 1,   /* per-row error-free FP32 sums (slower); the
                                 default picks them for small row counts   */
  GGEVAL_F_GRAD_MSE = 1u << 2,/* ggeval_grad_batch: gradient of plain MSE
                                 instead of scaled MSE                     */
  GGEVAL_F_PROFILE = 1u << 3, /* record CUDA events around the batched
                                 forward kernel (not with GGEVAL_F_GRAPH),
                                 or around the adjoint kernel in
                                 ggeval_grad_batch; read them with
                                 ggeval_profile_read                       */
  GGEVAL_F_POW = 1u << 4,     /* the batch may hold active POW nodes: run
                                 the kernel builds that include pow.
                                 Without it an active POW node is an
                                 invalid template (GGEVAL_ERR_TEMPLATE); the
                                 other kernels leave the pow code out
                                 because it costs them registers and speed */
  GGEVAL_F_NO_FOLD = 1u << 5, /* evaluate constant subtrees on every row.
                                 By default the packer folds each active
                                 subtree without a feature into one constant,
                                 computed once per trial with the same FP32
                                 functions, so the outputs are bit-identical
                                 either way; the gradient never folds      */
  GGEVAL_F_TEST_STALL = 1u << 6 /* test hook for failure detection
                                 (ggeval_eval_batch / ggeval_evaluate): the
                                 batched forward kernel issues no tile copy,
                                 so every bounded wait for a tile gives up
                                 after a short limit (milliseconds); nothing
                                 is left in flight, ggeval_sync() then
                                 reports GGEVAL_ERR_TIMEOUT and the call's
                                 outputs are unspecified.  The device stays
                                 usable for the next call.               */
};

/* Create a dataset from X (n_rows x n_features, float32, row-major when
 * x_row_major != 0, else feature-major) and the target y (n_rows float32).
 * X and y may be host or device pointers (unified addressing decides); they
 * are copied, so the caller may free them when the call returns (the call
 * synchronises `stream`).  Section 3.2 evaluates every trial over every
 * dataset row; the dataset is stored once, feature-major, and reused by
 * every batch.  y must be finite with |y| <= 2^50.
 * Errors: ERR_ARG (null, n_rows < 1, n_features outside 1..223, bad y),
 * ERR_CUDA / ERR_OOM. */
ggeval_status ggeval_create_dataset(const float* X, const float* y, int64_t n_rows,
                                    int32_t n_features, int32_t x_row_major,
                                    int32_t device, void* stream,
                                    ggeval_dataset** out);

/* Release a dataset and its workspace (synchronises its device).  NULL is
 * a no-op. */
void ggeval_destroy(ggeval_dataset* ds);

/* Evaluate every trial of the batch over all dataset rows: the batched
 * Evaluate(O[changed]) of Algorithm 1.  Outputs are float [n] in the
 * batch's memory; any of a, b, mse may be NULL.
 *   smse = min_{a,b} (1/N) sum_i (y_i - a - b f_i)^2, a, b the minimisers
 *   mse  = (1/N) sum_i (f_i - y_i)^2                   (Eq. 1)
 * with f_i the trial's active expression at row i (introns are skipped).
 * A trial whose f has population variance <= 1e-12 mean(f)^2 counts as
 * constant: b = 0, a = mean(y), smse = Var(y).
 * Errors: ERR_ARG, ERR_UNSUPPORTED (max_height > 8), ERR_CUDA, ERR_OOM;
 * template errors come back through ggeval_sync(). */
ggeval_status ggeval_eval_batch(ggeval_dataset* ds, const ggeval_batch* batch,
                                uint32_t flags, float* smse, float* a, float* b,
                                float* mse, void* stream);

/* Outputs of ggeval_evaluate, each an array of n values in the batch's
 * memory (device or host, as the batch); every pointer but smse may be
 * NULL.  smse, a, b and mse as for ggeval_eval_batch; nmse = mse / Var(y)
 * (Eq. 2, population variance); size = the number of active nodes of each
 * trial (the size objective of multi-objective GP, which the Conclusion
 * names as future work: error and size come from the same launch
 * sequence, the size from the packer that linearises the trial anyway);
 * size_evaluated = the nodes evaluated on every row after constant
 * subtrees are folded (equal to size with GGEVAL_F_NO_FOLD).  An invalid
 * trial gets NaN in the float outputs and -1 in the sizes. */
typedef struct {
  float* smse;
  float* a;
  float* b;
  float* mse;
  float* nmse;
  int32_t* size;
  int32_t* size_evaluated;
} ggeval_outputs;

/* ggeval_eval_batch with every output: error objectives (scaled MSE, MSE,
 * NMSE) and the size objective of each trial in one launch sequence
 * (pack, batched forward, finalise).  Flags and errors as for
 * ggeval_eval_batch. */
ggeval_status ggeval_evaluate(ggeval_dataset* ds, const ggeval_batch* batch, uint32_t flags,
                              const ggeval_outputs* out, void* stream);

/* Per-row values f_i of every trial (float [n][n_rows], batch memory), the
 * quantity each "sub-evaluation" of Section 3.2 squares.  For checking and
 * for building targets: it runs the launch configuration ggeval_eval_batch
 * would run with the same flags (tuned or default; see
 * ggeval_tile_config), in a build of the same kernel that also stores
 * every row's value, so the per-row values are those the fitness sums
 * take.  flags: GGEVAL_F_POW, GGEVAL_F_NO_FOLD, GGEVAL_F_EXACT as for
 * ggeval_eval_batch (the others are ignored). */
ggeval_status ggeval_eval_rows(ggeval_dataset* ds, const ggeval_batch* batch,
                               uint32_t flags, float* f, void* stream);

/* The same fitness as ggeval_eval_batch computed the plain way: one launch
 * of the row-parallel kernel per trial followed by a second-stage
 * reduction launch (the multi-block-per-individual design of Fig. 2,
 * right).  Device batches only.  For comparison with the batched form. */
ggeval_status ggeval_eval_plain(ggeval_dataset* ds, const ggeval_batch* batch,
                                uint32_t flags, float* smse, float* a, float* b,
                                float* mse, void* stream);

/* Fitness and its gradient with respect to every ERC constant:
 * dcval is float [n][stride] in the batch's memory, d smse / d cval (or
 * d mse / d cval with GGEVAL_F_GRAD_MSE), 0 at every non-ERC or intron
 * position.  Uses the envelope theorem for a, b:
 *   d smse/d c = (2b/N) sum_i (a + b f_i - y_i) d f_i/d c.
 * Node values are recomputed per row on chip, never stored in HBM.
 * smse may be NULL.  Errors as ggeval_eval_batch. */
ggeval_status ggeval_grad_batch(ggeval_dataset* ds, const ggeval_batch* batch,
                                uint32_t flags, float* smse, float* dcval,
                                void* stream);

/* One Adam step on the ERC constants of a device batch, in place:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * c -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps), for every
 * position whose op is ERC.  cval, grad, m, v: float [n][stride] device;
 * t >= 1 is the step number. */
ggeval_status ggeval_adam_step(const ggeval_batch* batch, float* cval, const float* grad,
                               float* m, float* v, int32_t t, float lr, float beta1,
                               float beta2, float eps, void* stream);

/* Time candidate tile shapes (rows per tile, trials per work item, warps per
 * CTA, rows per lane, register budget) on this batch and keep the fastest for batches of
 * the same shape (n, max_height, layout, flags).  Synchronises the stream;
 * runs the evaluation several times.  Device batches only.  With the
 * environment variable GGEVAL_VERBOSE set (not "0") every candidate's time
 * and the choice are printed to stderr. */
ggeval_status ggeval_autotune(ggeval_dataset* ds, const ggeval_batch* batch,
                              uint32_t flags, void* stream);

/* The autotuner's choices as a file: one JSON object per line, keyed by
 * the GPU's name and SM count, the dataset's rows and features, and the
 * batch shape (trials, max_height, layout, flags & (EXACT | POW)), with the
 * chosen {variant, tile_rows, group, warps}.  ggeval_tuning_save writes
 * every choice this dataset holds (replacing the file); ggeval_tuning_load
 * takes the entries that match this dataset's GPU and shape (n_loaded may
 * be NULL; a missing file holds none).  With the environment variable
 * GGEVAL_TUNE_CACHE naming such a file, ggeval_autotune uses a matching
 * entry instead of timing candidates, and appends the choices it makes.
 * Host-side only.  Errors: ERR_ARG (NULL, a file that cannot be opened). */
ggeval_status ggeval_tuning_save(ggeval_dataset* ds, const char* path);
ggeval_status ggeval_tuning_load(ggeval_dataset* ds, const char* path, int32_t* n_loaded);

/* The launch configuration of ggeval_eval_batch for batches of this shape
 * (n, max_height, layout, flags & (EXACT | POW)): int32 [4] = {variant,
 * rows per tile, trials per work item, warps per CTA}.  variant: 0 = 8
 * rows per lane with grouped sums, 1 = 4 rows per lane grouped, 2 = 4 rows
 * per lane with per-row error-free sums, 4..6 = 0..2 built for at most 64
 * registers, 8 and 9 = 0 and 5 running the C++ interpreter instead of the
 * PTX one (the same results).  With `set` non-NULL the given configuration is checked (it
 * must fit in shared memory; rows per tile a multiple of 32 x rows per
 * lane) and kept for such batches, as ggeval_autotune keeps its choice;
 * with `get` non-NULL the configuration in force is written there.  The
 * evaluation results do not depend on the configuration beyond rounding
 * of the fitness sums.  Errors: ERR_ARG (bad configuration, empty batch). */
ggeval_status ggeval_tile_config(ggeval_dataset* ds, const ggeval_batch* batch,
                                 uint32_t flags, const int32_t* set, int32_t* get);

/* Issue-rate microbenchmarks for the roofline denominators (not part of
 * the evaluation): on `device`, long chains of independent operations, 64
 * warps per SM, timed with CUDA events on the legacy default stream.
 * ops_per_s is double [6]: scalar FP32 FMA, packed two-row FMA (counted as
 * two operations), and the SFU's reciprocal square root, base-2
 * exponential, base-2 logarithm and sine.  Divide by the SM count and the
 * SM clock for operations per SM per clock.  `iters` sets the chain length
 * (the FP32 chains; the SFU chains run iters / 8).  Synchronous.
 * Errors: ERR_ARG, ERR_CUDA. */
ggeval_status ggeval_pipe_rates(int32_t device, int32_t iters, double* ops_per_s);

/* Wait for the dataset's work on `stream`, then report and clear the
 * device-side status: GGEVAL_OK, ERR_TEMPLATE, ERR_TIMEOUT or ERR_CHECKED. */
ggeval_status ggeval_sync(ggeval_dataset* ds, void* stream);

/* Sum of the batched forward kernel's durations (ms, from CUDA events on
 * the launching stream) and the number of launches timed since the last
 * read, for calls made with GGEVAL_F_PROFILE; waits for those events and
 * resets the sums.  At most 4096 launches are kept between reads. */
ggeval_status ggeval_profile_read(ggeval_dataset* ds, double* fwd_ms, int64_t* launches);

/* Thread-local message for the last non-OK status (never NULL). */
const char* ggeval_last_error(void);

/* Statistics of a batch for throughput accounting: for each trial, counts
 * of active nodes by class.  out is int64 [n][GGEVAL_NSTAT] host memory:
 * [0] active nodes, [1] terminals, [2] +/-/x, [3] AQ, [4] DIV,
 * [5] sin/cos, [6] exp, [7] log, [8] sqrt, [9] square; [10] interpreter
 * instructions after fusion; [11] stack slots used; [12] pow;
 * [13..23] the counts of [0..9] and pow ([23]) for the nodes evaluated on
 * every row after constant folding (GGEVAL_F_NO_FOLD); [24] interpreter
 * instructions after folding.  An invalid trial has -1 in [0].  Host
 * batches only; runs on the CPU, no dataset needed. */
#define GGEVAL_NSTAT 25
ggeval_status ggeval_batch_stats(const ggeval_batch* batch, int32_t n_features,
                                 int64_t* out);

/* The packer on the CPU, for inspection and tests: linearises trial `index`
 * of a host batch into the interpreter's instruction words (post-order of
 * the active nodes, Section 3.2, with operands of a binary node reordered
 * so the subtree needing more stack goes first).  words: uint32 [cap]
 * opcode | feature << 8; consts: float [cap]; tpos: int32 [cap], template
 * position of each instruction's main node.  Returns the instruction count
 * in *len (ERR_TEMPLATE for an invalid trial). */
ggeval_status ggeval_pack_host(const ggeval_batch* batch, int32_t index, int32_t n_features,
                               uint32_t* words, float* consts, int32_t* tpos, int32_t cap,
                               int32_t* len);

/* The device packer, for inspection and tests: packs a device batch exactly
 * as the evaluation calls do with these flags (GGEVAL_F_POW accepts pow;
 * constant subtrees are folded unless GGEVAL_F_NO_FOLD) and copies the
 * programs to host memory: words uint32 [n][cap] (opcode | feature << 8),
 * consts float [n][cap], len int32 [n] (the instruction count, -1 for an
 * invalid trial, whose template error also reaches ggeval_sync).  Entries
 * past a trial's length are left as they were.  Synchronous on `stream`. */
ggeval_status ggeval_pack_device(ggeval_dataset* ds, const ggeval_batch* batch, uint32_t flags,
                                 uint32_t* words, float* consts, int32_t* len, int32_t cap,
                                 void* stream);

/* Evaluate only the trials whose mask byte is nonzero: Evaluate(O[changed])
 * of Algorithm 1.  mask is uint8 [n] in device memory (device batches only);
 * the outputs of masked-out trials are left untouched.  Otherwise as
 * ggeval_eval_batch (GGEVAL_F_GRAPH replays read the mask's current
 * contents). */
ggeval_status ggeval_eval_batch_masked(ggeval_dataset* ds, const ggeval_batch* batch,
                                       const uint8_t* mask, uint32_t flags, float* smse,
                                       float* a, float* b, float* mse, void* stream);

/* One GOM step over a FOS index on the device (Algorithm 1's inner loop),
 * so that a whole FOS sweep runs without host round trips.  All arrays are
 * device memory, row-major [n][stride] with stride = 2^(max_height+1)-1.
 *
 * ggeval_gom_donate: for every offspring j, copy the nodes (op and constant)
 * of FOS subset subset[j] from population member donor[j]:
 * O_j[FOS[s]] <- P_donor[FOS[s]].  The FOS is given in CSR form: the nodes
 * of subset s are fos_nodes[fos_offsets[s] .. fos_offsets[s+1]).  An
 * out-of-range donor, subset or node leaves the offspring unchanged. */
ggeval_status ggeval_gom_donate(int32_t n, int32_t max_height, uint8_t* op, float* cval,
                                const uint8_t* pop_op, const float* pop_cval, int32_t n_pop,
                                const int32_t* donor, const int32_t* subset,
                                const int32_t* fos_offsets, const int32_t* fos_nodes,
                                int32_t n_fos, void* stream);

/* changed[j] = 1 when offspring j differs from its backup at a node that is
 * active in either (opcode, or the constant of an ERC node): the paper
 * evaluates an offspring only if an actively used part of its template
 * changed (Section 3.1).  The offspring batch gives n, heights and layout;
 * the backup has the same shape. */
ggeval_status ggeval_gom_changed(const ggeval_batch* offspring, const uint8_t* backup_op,
                                 const float* backup_cval, int32_t n_features,
                                 uint8_t* changed, void* stream);

/* Accept or revert (Algorithm 1): offspring j is accepted when it is
 * unchanged, or when f_new[j] <= f_backup[j] (not worse; a NaN never
 * replaces a number and a number always replaces a NaN); then its backup
 * becomes a copy of it and, if changed, f_backup[j] = f_new[j].  Otherwise
 * the offspring is reverted to its backup.  changed may be NULL (all
 * changed); accepted (uint8 [n]) may be NULL. */
ggeval_status ggeval_gom_accept(int32_t n, int32_t max_height, uint8_t* op, float* cval,
                                uint8_t* backup_op, float* backup_cval, const uint8_t* changed,
                                const float* f_new, float* f_backup, uint8_t* accepted,
                                void* stream);

/* Active size of every trial: size[j] = number of active nodes (int32 [n],
 * batch memory must be device), the size objective of an error + size
 * (multi-objective) search.  -1 for a trial whose height is out of range.
 * The active set follows the same rule as the evaluation. */
ggeval_status ggeval_trial_sizes(const ggeval_batch* batch, int32_t n_features, int32_t* size,
                                 void* stream);

/* The dataset's shape and target statistics: rows, features, mean(y) and
 * the population variance Var(y) (1/N), both in FP64 from the stored target.
 * NMSE (Eq. 2) = mse / Var(y).  Any output pointer may be NULL. */
ggeval_status ggeval_dataset_info(const ggeval_dataset* ds, int64_t* n_rows,
                                  int32_t* n_features, double* y_mean, double* y_var);

/* Evaluation that allocates nothing.  Some callers cannot call cudaMalloc
 * while they evaluate: code running inside a CUDA stream capture (the
 * allocator is not allowed there), latency-critical loops that cannot take
 * the device-wide synchronisation cudaMalloc implies, and processes whose
 * device memory is budgeted up front.  ggeval_eval_batch may grow its
 * workspace on such a call; this entry point never does.  It computes the
 * same outputs as ggeval_eval_batch with flags 0 (same definitions, same
 * error rules; so no POW nodes) for a device batch on an existing dataset, using as scratch one static
 * device array of GGEVAL_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until the process exits.  (The paper has no counterpart:
 * it is a deployment form of the batched evaluation, not part of the
 * method.)
 *  - Limits: n <= GGEVAL_NOALLOC_MAX_TRIALS, max_height <=
 *    GGEVAL_NOALLOC_MAX_HEIGHT, and the dataset's rows must fit in at most
 *    GGEVAL_NOALLOC_MAX_TILES row tiles that fit in shared memory; larger
 *    requests return GGEVAL_ERR_UNSUPPORTED with a message and launch
 *    nothing.  Host-memory batches return GGEVAL_ERR_ARG.
 *  - A call made outside a stream capture looks up the array's device
 *    address (cudaGetSymbolAddress) with the dataset's device current, so
 *    after a device reset the new context's address is used; a call made
 *    during a capture uses the address from that device's last call outside
 *    one.  So make the first call on each device (and the first after a
 *    reset) before any stream capture.
 *  - Every call on a device shares the one array and it keeps the previous
 *    call's contents (the call zeroes what must start at zero).  Calls whose
 *    GPU work overlaps (different streams, or different datasets on the
 *    same device without ordering) race on it: order them on one stream. */
#define GGEVAL_NOALLOC_MAX_TRIALS 4096
#define GGEVAL_NOALLOC_MAX_HEIGHT 6
#define GGEVAL_NOALLOC_MAX_TILES 64
#define GGEVAL_NOALLOC_SCRATCH_BYTES (4096u * 128u * 8u + 4096u * 4u + 4096u * 64u * 32u + 256u)
ggeval_status ggeval_eval_batch_noalloc(ggeval_dataset* ds, const ggeval_batch* batch,
                                        float* smse, float* a, float* b, float* mse,
                                        void* stream);

/* Library version string. */
const char* ggeval_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GGEVAL_H */
