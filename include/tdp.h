/*
 * tdp.h -- C ABI of the GB300 tridiagonal partition solver.
 *
 * Method: the parallel partition method for tridiagonal systems (Veneva,
 * "ML-Based Optimum Sub-system Size for the GPU Implementation of the
 * Tridiagonal Partition Method", arXiv 2510.27351, Sec. I): the N unknowns
 * are split into sub-systems of s rows; Stage 1 reduces every sub-system to
 * two interface equations, Stage 2 solves the tridiagonal interface system,
 * Stage 3 substitutes the interface values and solves the interiors.  The
 * sub-system size s is chosen by a 1-nearest-neighbour model over measured
 * timings (Sec. II-E) when the caller passes s = 0.
 *
 * Matrix convention: row i reads  a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i];
 * a[0] and c[n-1] of every system are ignored (need not be zero).
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller and
 * aligned to 16 bytes; the library never frees or retains it.  Inputs are
 * read-only; x must not alias an input.  Scratch memory (the interface
 * system and the per-row coefficients kept between stages) comes from a
 * library-owned workspace per CUDA stream, grown on demand; it cannot grow
 * while the stream is being captured into a CUDA graph, so call tdp_reserve
 * (or run the call once) before capturing.
 *
 * Streams: every call is asynchronous on `stream` (a cudaStream_t, NULL = the
 * legacy default stream) and makes no host synchronisation unless checked
 * mode is on (tdp_set_checked) or the workspace has to grow.
 *
 * Errors: every int-returning call returns one of the TDP_* codes below and
 * records a message retrievable with tdp_last_error() (per host thread).
 * Pivot failures found on the device (a zero or non-finite pivot) are
 * recorded in a per-stream device status word; they are returned as
 * TDP_ESINGULAR by the call itself in checked mode, else by tdp_status().
 */
#ifndef TDP_H
#define TDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Precision of a solve.
 *  TDP_F64        binary64 storage, binary64 arithmetic.
 *  TDP_F32        binary32 storage, binary32 arithmetic for the sub-system
 *                 eliminations and substitutions, binary64 interface solve;
 *                 by default single systems and batches take the windowed
 *                 single pass (TDP_TUNE_WINDOW32, below).
 *  TDP_F32_REFINE binary64 storage; binary32 eliminations/substitutions with a
 *                 binary64 residual r = d - A x and correction x += delta
 *                 (iterative refinement), binary64 interface solve; by
 *                 default single systems and batches take the windowed
 *                 single pass (TDP_TUNE_WINDOW, below).
 *
 * The windowed single pass (not in the paper: for binary32 arithmetic, where
 * GB300's binary64 pipe does not bound the solve) reads the inputs once:
 * every tile of about 1700 rows (up to 3300 for TDP_F32) is solved inside a
 * window with 48 halo rows (32 for TDP_F32) on each side (binary32
 * partition solve of the window, its
 * interface system included, then for TDP_F32_REFINE the binary64 residual
 * and corrections on chip; the binary32 copies of d, x and the residuals
 * carry a power-of-two scale per window, so any scale of d keeps binary64
 * accuracy).  Each tile checks at run time that its window rows are
 * diagonally dominant and that the decay of A^-1 across each halo bounds the
 * windowed solution's distance from x (by 2^-45 ||x|| for TDP_F32_REFINE,
 * 2^-30 ||x|| for TDP_F32); if any tile fails, the exact partition method
 * solves the whole system in binary64 in one further cooperative launch,
 * and the status word gets its informational fallback bit (8).  The size s
 * does not apply to the windowed pass.  The exact TDP_F32_REFINE schedules
 * (TDP_TUNE_WINDOW = 0, or the recursion schedule) narrow d without a scale:
 * a system with a nonzero |d| outside [2^-70, 2^70] or |b| outside
 * [2^-30, 2^30] is solved again by the same binary64 fallback (bit 8). */
typedef enum { TDP_F64 = 0, TDP_F32 = 1, TDP_F32_REFINE = 2 } tdp_dtype;

#define TDP_OK 0
#define TDP_EINVAL 1     /* bad argument: size, s, null or misaligned pointer, offsets */
#define TDP_ECUDA 2      /* a CUDA runtime call or kernel launch failed */
#define TDP_ESINGULAR 3  /* a zero or non-finite pivot was met on the device */
#define TDP_ETIMEOUT 4   /* a bounded device wait ran out */
#define TDP_ENOMEM 5     /* workspace too small and cannot grow (e.g. during capture) */

/* Solve one system of n unknowns (Sec. I, three stages).
 *  a, b, c, d : device arrays of n elements (binary64 for TDP_F64 and
 *               TDP_F32_REFINE, binary32 for TDP_F32).
 *  x          : device array of n elements, same type; receives the solution.
 *  n          : number of unknowns, n >= 1.
 *  s          : sub-system size, 2 <= s <= 1024, or 0 to let tdp_predict_s
 *               choose (Sec. II-E).  s >= n solves the system as one block.
 *  refine_iters: for TDP_F32_REFINE, number of binary64-residual corrections
 *               (0..8); ignored otherwise.
 * Returns TDP_OK or an error code. */
int tdp_solve(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t s,
              tdp_dtype dtype, int32_t refine_iters, void* stream);

/* Solve `batch` independent systems stored back to back.
 *  offsets    : DEVICE array of batch+1 int64, offsets[0] = 0, non-decreasing;
 *               system j occupies rows offsets[j] .. offsets[j+1]-1.
 *  total_n    : offsets[batch] (passed by value so that no copy to the host is
 *               needed; the device checks it and reports TDP_EINVAL through
 *               the status word when it disagrees).
 *  s          : sub-system size for every system (2..1024), or 0 for the
 *               size model's choice: a batch of at least 4096 rows per system
 *               on average is solved as one block-diagonal system of total_n
 *               rows (the couplings between systems are cut on the device;
 *               TDP_TUNE_BATCH_FLAT) and s = 0 takes tdp_predict_s(total_n, 1,
 *               dtype); otherwise blocks never straddle systems and s = 0
 *               takes the size model for the mean system size and the batch
 *               size.  With the tuning key TDP_TUNE_PER_SYSTEM_S = 1, s = 0
 *               gives every system its own size on the device
 *               (tdp_predict_s_batched), capped at the largest size the model
 *               gives for the nearest batch size.
 * Empty systems are allowed; a[offsets[j]] and c[offsets[j+1]-1] are ignored.
 * Other arguments as tdp_solve. */
int tdp_solve_batched(const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                      const void* c, const void* d, void* x, int32_t s, tdp_dtype dtype, int32_t refine_iters,
                      void* stream);

/* Constant-coefficient systems (the implicit step of the heat equation and
 * other alternating-direction schemes; not in the paper): `batch` systems of n
 * unknowns whose rows all read  a x[i-1] + b x[i] + c x[i+1] = d[i]  (a of a
 * system's first row and c of its last row are ignored).  d and x are
 * DEVICE arrays addressed like tdp_solve_strided: element i of system j at
 * j*sys_stride + i*elem_stride (in elements, both >= 1); the systems must not
 * overlap: elem_stride >= batch*sys_stride (interleaved) or
 * sys_stride >= n*elem_stride (one after another).  Pointers aligned to their
 * element; x must not alias d.  The partition method with the coefficient
 * part of Stage 1 (pivots, multipliers, spike and backward coefficients)
 * computed once per call for a block of s rows; s in [2, 512] or 0 for the
 * size model.  Moves 3 words per unknown (d twice, x once); dtype as
 * tdp_solve, except that TDP_F32_REFINE is solved in binary64 arithmetic
 * (with the coefficient part tabulated a row costs 4 binary64 operations,
 * less than binary32 passes with a binary64 residual and update would:
 * the answer meets the refinement's accuracy at lower cost) and
 * refine_iters is then ignored. */
int tdp_solve_const(double a, double b, double c, const void* d, void* x, int64_t n, int32_t batch,
                    int64_t sys_stride, int64_t elem_stride, int32_t s, tdp_dtype dtype, int32_t refine_iters,
                    void* stream);

/* tdp_solve with HOST arrays (a, b, c, d in, x out; n elements each), for
 * callers whose data are not on the device yet.  Pinned host memory
 * (cudaHostAlloc / cudaHostRegister) lets the copies overlap the solve: the
 * binary64 solve (and the binary32 one with TDP_TUNE_WINDOW32 = 0) runs in
 * about eight chunks, Stage 1 of a chunk while the next one is copied in,
 * Stage 3 of a chunk while the previous one is copied out (a second stream
 * that the call creates and releases); the answer is the one tdp_solve
 * gives, bit for bit.  The windowed passes (the refinement and, by default,
 * binary32) stream in about sixteen chunks of whole tiles: a chunk's tiles
 * are solved as soon as it has been copied in, and their x is copied out on a
 * second stream while later chunks are copied in; this needs x in memory the
 * device can address (pinned or registered), where the exact fallback, if a
 * tile fails, writes x directly; with pageable x these passes copy everything
 * in, solve and copy out.  Asynchronous on `stream` like tdp_solve: x is
 * complete when the stream's work is.  The device copies of the arrays live
 * in the workspace (5n elements).  Other arguments and errors as tdp_solve;
 * x must not overlap an input. */
int tdp_solve_host(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t s,
                   tdp_dtype dtype, int32_t refine_iters, void* stream);

/* Many right-hand sides with one matrix (not in the paper): solve A X = D for
 * nrhs columns of n unknowns.  Column j of D starts at element j*ldd of d, column
 * j of X at element j*ldx of x (ldd, ldx >= n; the X and D ranges must not
 * overlap).  The matrix part of the method (reciprocal pivots, multipliers, the
 * spike and backward coefficients of Stage 3 and the interface matrix, Sec. I)
 * is computed once; each column then costs the d-part of Stage 1 and Stage 3
 * (5 operations per row instead of 14) and its share of one interface solve over
 * all columns.  dtype TDP_F64 or TDP_F32 (a, b, c, d, x of that type); s in
 * [2, 1024], or 0 for four times tdp_predict_s(n, 1, dtype) within [16, 64]
 * (a column skips the matrix part, so the interface solve weighs more and a
 * larger s pays); 1 <= nrhs <= 65535.  All
 * pointers 16-byte aligned and every column too (ldd, ldx multiples of 16
 * bytes), else TDP_EINVAL.  Scratch: 5n words for the matrix part plus the
 * interface systems. */
int tdp_solve_multi(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t nrhs,
                    int64_t ldd, int64_t ldx, int32_t s, tdp_dtype dtype, void* stream);

/* Solve `batch` systems of n unknowns each with arbitrary element strides:
 * element i of system j lives at index  j*sys_stride + i*elem_stride  of each
 * array (in elements).  sys_stride = n, elem_stride = 1 is a contiguous batch;
 * sys_stride = 1, elem_stride = batch is the interleaved layout of the column
 * sweep of an alternating-direction implicit step.  The index ranges of
 * different systems must not overlap. */
int tdp_solve_strided(int32_t batch, int64_t n, int64_t sys_stride, int64_t elem_stride, const void* a,
                      const void* b, const void* c, const void* d, void* x, int32_t s, tdp_dtype dtype,
                      int32_t refine_iters, void* stream);

/* Adjoint of the solve (not in the paper).  Given the forward solution x of
 * A x = d and g = dL/dx, computes lambda = A^{-T} g with the same partition
 * kernels and the gradients of L:
 *   grad_d = lambda,  grad_a[i] = -lambda[i] x[i-1] (0 at a system's first row),
 *   grad_b[i] = -lambda[i] x[i],  grad_c[i] = -lambda[i] x[i+1] (0 at its last row).
 *  offsets    : DEVICE array of batch+1 int64 (batch = 1, offsets = {0, n} for
 *               a single system); total_n = offsets[batch].
 *  grad_*     : device arrays of total_n elements; any may be NULL to skip it
 *               (grad_d is lambda and is computed even when NULL is passed
 *               for it, into workspace).
 * The transposed diagonals are written with zeros at every system boundary,
 * so the whole batch is solved as one system of total_n rows; s (0 = the size
 * model for one system of total_n rows) partitions that system.
 * dtype TDP_F64, TDP_F32 or TDP_F32_REFINE (binary64 arrays; the transposed
 * solve in binary32 with one binary64 correction).  TDP_F32 and
 * TDP_F32_REFINE run the windowed passes by default, whose windows read A^T's
 * diagonals straight from a and c: no transposed copies are written and s is
 * not used. */
int tdp_solve_backward(const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                       const void* c, const void* x, const void* g, void* grad_a, void* grad_b, void* grad_c,
                       void* grad_d, int32_t s, tdp_dtype dtype, void* stream);

/* Sub-system size for a solve of `batch` systems of about n unknowns each
 * (Sec. II-E: 1-nearest-neighbour over (log2 n, log2 batch) in the table of
 * the given precision, ties to the larger s).  Uses the table loaded by
 * tdp_load_table, else the built-in table measured on GB300, else the
 * paper's interval rule (Sec. II-D).  Never fails: returns a valid s >= 2. */
int32_t tdp_predict_s(int64_t n, int32_t batch, tdp_dtype dtype);

/* Number R of recursive steps of the partition method (Sec. III-A: a
 * 1-nearest-neighbour model for the optimum number of recursive steps).
 * 1-NN over (log2 n, log2 batch) in the recursion-depth table of the given
 * precision (ties to the larger R): the table loaded by tdp_load_rtable, else
 * the built-in one measured on GB300, else the intervals of the paper's table
 * of optimum R (R = 0 up to 2.2e6 unknowns, 1 up to 4.8e6, 2 up to 9.6e6,
 * 3 above).  Used by the solves when the tuning key TDP_TUNE_RECURSION is 1.
 * Returns -1 for n < 1, batch < 1 or an unknown dtype. */
int32_t tdp_predict_r(int64_t n, int32_t batch, tdp_dtype dtype);

/* Load a recursion-depth table: a text file of rows "dtype n batch R"
 * ('#' starts a comment), R in [0, 12].  The empty string "" restores the
 * built-in table.  TDP_EINVAL for an unreadable file or a bad row (the
 * current table is kept). */
int tdp_load_rtable(const char* path);

/* Sub-system sizes of the R recursive steps the paper's schedule (Sec. III-B)
 * uses for one system of n unknowns partitioned with sub-system size s: step
 * 1 uses 10 when R >= 2, every other step the size model (tdp_predict_s,
 * binary64) applied to the interface system it partitions; steps stop early
 * once the interface system has at most 64 rows or would form one block.
 * R < 0 means the predicted R (tdp_predict_r).  Writes at most cap sizes to
 * the HOST array m_out and returns how many steps there are, or -1 for bad
 * arguments.  Host only. */
int32_t tdp_recursion_plan(int64_t n, int32_t s, int32_t R, tdp_dtype dtype, int32_t* m_out, int32_t cap);

/* The same size model evaluated on the device, one system per thread: s_out[j]
 * (DEVICE array of batch int32) receives the predicted s of system j of
 * the batch described by the DEVICE offsets (batch+1 int64), with the batch
 * size as second feature.  This inference kernel is what tdp_solve_batched
 * runs when called with s = 0.  Asynchronous on `stream`. */
int tdp_predict_s_batched(const int64_t* offsets, int32_t batch, tdp_dtype dtype, int32_t* s_out, void* stream);

/* Replace the predictor's table (text: lines "dtype n batch s", '#' comments;
 * dtype 0/1/2 as tdp_dtype); an empty path "" restores the built-in table.
 * Returns TDP_OK or TDP_EINVAL (unreadable file or bad row; the table is
 * then unchanged). */
int tdp_load_table(const char* path);

/* Grow the workspace of `stream` to what a solve of `total_n` unknowns in
 * `batch` systems with sub-system size s (0 = smallest supported) needs, so
 * that later calls of that size make no allocation (required before CUDA
 * graph capture).  May synchronise the stream. */
int tdp_reserve(int64_t total_n, int32_t batch, int32_t s, tdp_dtype dtype, void* stream);

/* Read and clear the device status word of `stream` (synchronises it).
 * Returns TDP_OK, TDP_ESINGULAR, TDP_ETIMEOUT or TDP_EINVAL. */
int tdp_status(void* stream);

/* Return code that a device status word stands for (host only, no GPU
 * needed): bit 4 (arguments rejected on the device) gives TDP_EINVAL, bit 2
 * (a bounded wait ran out) TDP_ETIMEOUT, bit 1 (zero or non-finite pivot)
 * TDP_ESINGULAR, in that order of precedence when several are set; 0 gives
 * TDP_OK.  tdp_status, checked-mode solves and tdp_solve_noalloc all map
 * the word this way. */
int tdp_status_code(uint32_t bits);

/* The raw device status word that the last checked-mode call or tdp_status
 * call of this host thread read (before clearing it).  Besides the error bits
 * above, bit 8 is informational: the windowed pass of a TDP_F32_REFINE solve
 * found a tile whose checks failed and the exact binary64 fallback produced
 * the answer (tdp_status_code maps it to TDP_OK). */
uint32_t tdp_last_status_bits(void);

/* Checked mode: when on, every solve synchronises its stream and returns the
 * device status.  Default off. */
void tdp_set_checked(int on);

/* Message of the last error on this host thread ("" if none). */
const char* tdp_last_error(void);

/* Number of kernels this library has launched in this process (all
 * streams); lets callers count launches inside a timed region. */
int64_t tdp_launch_count(void);

/* Launch tuning knobs, process-wide (change them between solves, not while
 * another thread is solving).  Start values come from environment variables
 * of the same names.  tdp_set_tuning returns TDP_OK or TDP_EINVAL (unknown
 * key or value out of range); tdp_get_tuning returns the value or -1. */
#define TDP_TUNE_SMEM_BUDGET 0  /* shared memory per CTA of the register-staged tiles, bytes [4096, 232448] */
#define TDP_TUNE_S_REC 1        /* sub-system size inside the interface recursion [3, 1024] */
#define TDP_TUNE_S_TAIL 2       /* sub-system size in the one-launch tail of that recursion [3, 256] */
#define TDP_TUNE_VTILE 3        /* 1: 16-byte cp.async interleaved tiles for single systems */
#define TDP_TUNE_COOP 4         /* 1: the small interface levels in one cooperative launch */
/* keys 5 to 8 are retired (variants measured slower and removed); they are rejected */
#define TDP_TUNE_REFINE3 9      /* 1: TDP_F32_REFINE runs its solve and first correction as three fused passes */
#define TDP_TUNE_RECURSION 10   /* 1: the interface system follows the paper's recursion schedule (Sec. III);
                                   0: s = TDP_TUNE_S_REC levels down to 2^19 rows, then the one-launch tail */
#define TDP_TUNE_R 11           /* number of recursive steps of that schedule, -1 = tdp_predict_r [-1, 12] */
#define TDP_TUNE_SEGMENTED 12   /* 1: batches of >= 32 systems with at most 512 interface rows per system on
                                   average solve them one CTA per system */
#define TDP_TUNE_PER_SYSTEM_S 13 /* 1: tdp_solve_batched with s = 0 gives every system its own s (device model) */
#define TDP_TUNE_IFACE32 14     /* 1: TDP_F32 and TDP_F32_REFINE solve the first level of their interface
                                   recursion (interface systems above 2^19 rows) in binary32 arithmetic
                                   (default 0: every interface level in binary64) */
#define TDP_TUNE_REFINE_KEPT 15 /* 1: the refinement's second pass keeps the correction's Stage-1 coefficients
                                   (binary32) so that its last pass is elementwise (104 instead of 120 B/row) */
#define TDP_TUNE_COOP_REG 16    /* 1: the one-launch interface tail reads its 8-row blocks into registers */
#define TDP_TUNE_BATCH_FLAT 17  /* 1: tdp_solve_batched with at least 4096 rows per system on average solves the
                                   batch as one block-diagonal system on the single-system tiles */
#define TDP_TUNE_VTILE_B 18     /* 1: binary64 Stage 1 at s = 8 or 16 keeps b in registers and a, c, d in the
                                   interleaved tile (a quarter less shared memory per row) */
#define TDP_TUNE_VTILE_L 19     /* 1: binary32 storage runs Stage 1 and Stage 3 on padded block-major tiles
                                   (each block's rows contiguous in shared memory) */
#define TDP_TUNE_WINDOW 20      /* 1: TDP_F32_REFINE single systems and batches take the windowed single pass
                                   (see tdp_solve) */
#define TDP_TUNE_WINDOW_HALO 21 /* halo rows on each side of a tile of the refinement's windowed pass [16, 64],
                                   rounded down to a multiple of 4; default 48 */
#define TDP_TUNE_WAIT_LOG2 22   /* every bounded device wait gives up after 2^value clock cycles [10, 40] */
#define TDP_TUNE_WAIT_NEVER 23  /* 1 (testing only): grid barriers wait for one arrival more than the grid has,
                                   so every such wait runs out and the call reports TDP_ETIMEOUT */
#define TDP_TUNE_WINDOW_SW 24   /* rows per thread in the refinement's windowed pass: 5 or 7 (default; odd,
                                   so that the threads' strided shared-memory reads avoid bank conflicts) */
#define TDP_TUNE_WINDOW32 25    /* 1: TDP_F32 single systems and batches take the windowed single pass too
                                   (binary32 solve of each window, no refinement; exact fallback) */
#define TDP_TUNE_WINDOW_PREFETCH 26 /* the CTA of tile t of the windowed pass asks L2 for the window of tile
                                   t + value before loading its own [0, 4096], default 128; 0 = no prefetch */
#define TDP_TUNE_WINDOW_HALO32 27 /* halo rows on each side of a tile of the binary32 windowed pass [16, 64],
                                   default 32 (its bound, 2^-30, needs a third fewer rows than the
                                   refinement's 2^-46) */
#define TDP_TUNE_WINDOW_SW32 28  /* most rows per thread of the binary32 windowed pass [5, 13], default 13: it
                                   takes the largest odd count up to this that gives every SM three tiles,
                                   else 5 */
int tdp_set_tuning(int key, int value);
int tdp_get_tuning(int key);

/* Measured binary64 FMA rate of the current device (a diagnostic, not part
 * of the method): every thread of four full waves of CTAs runs 8 independent
 * chains of 2048 dependent FMAs.  *fma_per_s receives FMAs per second of the
 * fastest of three timed launches (after one warm-up launch), *ms_out (may be
 * NULL) that launch's duration.  This is the denominator of the binary64
 * kernels' ALU roofline.  Synchronises `stream`; allocates and frees a small
 * device buffer.  TDP_EINVAL for a null fma_per_s, TDP_ECUDA on a CUDA error. */
int tdp_fp64_fma_rate(double* fma_per_s, double* ms_out, void* stream);

/* Per-kernel timing (a tracing aid): when enabled, every kernel the library
 * launches outside stream capture is bracketed by two CUDA events recorded
 * on its launch stream.  Enabling (or disabling) clears earlier records. */
void tdp_profile_enable(int on);

/* Waits for the recorded events and writes one line per kernel name,
 * "name launches total_ms", in first-launch order, into buf (NUL-terminated,
 * truncated to len-1 bytes).  Returns the full text length. */
int64_t tdp_profile_summary(char* buf, int64_t len);

/* Plain GPU Thomas baseline: one thread per system, sequential Thomas.
 * Same arguments as tdp_solve_batched (TDP_F64 or TDP_F32). */
int tdp_thomas_batched(const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                       const void* c, const void* d, void* x, tdp_dtype dtype, void* stream);

/* Diagnostics: run Stage 1 only on one system and write its interface
 * system (2*ceil(n/s) rows, binary64, row 2k for x[k*s], row 2k+1 for the
 * last row of block k; a one-row last block gets an identity row 2k+1).
 * ra..rd are device arrays of at least 2*ceil(n/s) doubles. */
int tdp_stage1(const void* a, const void* b, const void* c, const void* d, int64_t n, int32_t s, tdp_dtype dtype,
               double* ra, double* rb, double* rc, double* rd, void* stream);

/* Allocation-free solve of one system (the paper has no counterpart; this
 * is a service of the library).  For callers that cannot allocate device
 * memory at the moment they solve: latency-critical loops in which a
 * cudaMalloc would synchronise the device, and hosts whose memory pool owns
 * all device memory and forbids other allocations after start-up.
 *
 * Same arguments and results as tdp_solve, for TDP_F64 and TDP_F32 only (no
 * refinement); the tuning keys (tdp_set_tuning) apply as they do to
 * tdp_solve.  Scratch comes from one statically sized 16 MiB __device__ array
 * inside the library, present on every GPU that loads the library until the
 * process exits; the call makes no cudaMalloc, cudaFree or other device
 * allocation.  Binary64 solves re-solve the interiors in Stage 3 instead of
 * keeping per-row coefficients, so only the interface systems use scratch:
 * about 4.3 bytes per unknown at s = 32, i.e. n up to about 3.9 million
 * unknowns at s = 32 (more with larger s).  Larger sizes are rejected with
 * TDP_EINVAL and a message giving the bytes needed.
 *
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress, with that device current), once per device.  Every
 * call shares the one array, which keeps the previous call's contents (the
 * status word is cleared at the start of each call): calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * it and must be serialised by the caller.  In checked mode (tdp_set_checked)
 * the call synchronises its stream and maps the device status word like
 * tdp_status_code; otherwise read it with the array's own status, which the
 * next call clears. */
int tdp_solve_noalloc(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t s,
                      tdp_dtype dtype, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TDP_H */
