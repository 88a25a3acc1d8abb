/*
 * sp2.h -- C ABI of the GB300 SP2 density-matrix purification library.
 *
 * The library turns a symmetric Fock matrix F (N x N) into the density matrix D,
 * the orthogonal projector onto the eigenvectors of the n_occ smallest eigenvalues
 * of F (Kruchinina, Rudberg, Rubensson, arXiv:1507.02087, §1, definition of D).
 * It runs the original SP2 recursive expansion (Alg. 3): X_0 = (lmax I - F) /
 * (lmax - lmin) with Gershgorin bounds, then X_i = X_{i-1}^2 if Tr[X_{i-1}] > n_occ
 * and X_i = 2 X_{i-1} - X_{i-1}^2 otherwise, and stops with the paper's parameterless
 * test on v_i = ||X_i - X_i^2||_F (§2, Frobenius estimate; Alg. 3 stop):
 *   stop at the first i >= 2 with p_i != p_{i-1}, v_{i-2} < 1 and
 *   log(v_i / C) / log(v_{i-2}) < qtilde,  C = (71 + 17 sqrt(17)) / 32, qtilde = 1.8.
 * Two readings where the paper is silent are built in: the order test is only
 * evaluated when v_{i-2} < 1 (§2 assumes it), and a trace guard stops when the trace
 * does not move the way the chosen polynomial must move it in exact arithmetic
 * (reason SP2_STOP_TRACE_GUARD; see sp2_stop_reason).
 *
 * Everything is enqueued on the caller's CUDA stream; the stopping test runs on the
 * device, so a run makes no host synchronisation until sp2_get_info.
 *
 * Conventions for every entry point:
 *  - Matrices are dense, row-major, N x N, leading dimension N, FP64, and F must be
 *    exactly symmetric (both triangles hold the same value).  "_dev" pointers are
 *    device memory of the current CUDA device, "_host" pointers host memory.
 *  - The caller owns F and D.  F is only read.  D may not alias F.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Every function returns an sp2_status; none aborts, traps or prints.  Errors
 *    found on the device (non-finite input, exhausted wait) surface through
 *    sp2_get_info's `status`.
 *  - A handle is not thread-safe: calls on one handle must be serialised by the
 *    caller, and at most one run per handle may be in flight at a time.
 */
#ifndef SP2_H
#define SP2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SP2_OK = 0,
  SP2_ERR_INVALID_ARG = 1,  /* bad size, null pointer, aliasing, bad option */
  SP2_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  SP2_ERR_NONFINITE = 3,    /* F holds a NaN or an infinity (found on the device) */
  SP2_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  SP2_ERR_NOMEM = 5,        /* workspace allocation failed */
  SP2_ERR_NO_GAP = 6,       /* lmax == lmin with 0 < n_occ < N: F = cI has no gap */
  SP2_ERR_UNSUPPORTED = 7,  /* option not supported on this path or handle */
  SP2_ERR_BOUNDS = 8        /* debug library only (libsp2_debug.so, sp2_build_device_checks):
                               a device-side index failed its bounds check and the access it
                               guarded was skipped; the run's results are not valid */
} sp2_status;

/* Why a run stopped (sp2_info.stop_reason). */
typedef enum {
  SP2_STOP_ORDER = 0,        /* the paper's convergence-order test fired (Alg. 3) */
  SP2_STOP_TRACE_GUARD = 1,  /* trace moved the wrong way: rounding dominates */
  SP2_STOP_EXACT = 2,        /* n_occ in {0, N}, or X exactly idempotent */
  SP2_STOP_CAP = 3,          /* max_iter reached (safety net) */
  SP2_STOP_SCHEDULE = 4      /* SP2-ACC: the precomputed schedule ended (n_max, Alg. 4) */
} sp2_stop_reason;

/* Arithmetic of the squaring X -> X^2.  The three tensor-core modes share one scheme: X is
 * held as FP32 values split into 16-bit pieces, squares run on the tcgen05 tensor cores as
 * sums of piece products with FP32 accumulation, bounds, reductions and the stop test are
 * FP64, and the low-precision expansion (which detects its own, earlier rounding floor with
 * the same parameterless test) is followed by a first-order correction of the occupied
 * subspace driven by F (sp2_opts.corrections) and a refinement pair (sp2_opts.refine_steps).
 * The derivative pass of the correction always runs at the mode's low precision.  Workspace
 * of the tensor-core modes: (max_iter + 8) slots of P * E * ld^2 bytes (P pieces of E bytes), ld = N
 * rounded up to a multiple of 128 (256 with CTA-pair tiles); see sp2_opts.history. */
typedef enum {
  SP2_PREC_FP64 = 0,   /* FP64 products and FP64 everything (the plain method) */
  SP2_PREC_MIXED = 1,  /* = SP2_PREC_BF16X6: each FP32 value stored exactly as three bf16
                          pieces (P = 3), products as the six piece products with a + b <= 2
                          (FP32-accurate) */
  SP2_PREC_BF16X6 = 1,
  SP2_PREC_BF16X3 = 2, /* the same three bf16 pieces, every product as the three with a + b <= 1
                          (about 16 significant bits, half the tensor work of BF16X6); a
                          comparison point: its error after the correction stays near 1e-5 */
  SP2_PREC_FP16X3 = 3, /* each value as two fp16 pieces of 2^14 x (P = 2, 22 significant bits;
                          |x| < 4, which every iterate satisfies), products as the three piece
                          products p0 q0 + p0 q1 + p1 q0 (relative error about 2^-21, half the
                          tensor work of BF16X6), derivative steps as p0 q0; the correction's
                          F enters as (F - c I) / w' (c, w' the centre and half-width of the
                          spectral bounds, so its entries fit the fp16 range) */
  SP2_PREC_TF32X3 = 4  /* each value as two tf32 pieces held in FP32 words, hi = tf32(x) and
                          lo = tf32(x - hi) (P = 2, 4-byte pieces, 22 significant bits, FP32's
                          exponent range), products as hi lo' + lo hi' + hi hi' on kind::tf32
                          tensor cores (half the kind::f16 rate), derivative steps as hi hi' */
} sp2_precision;

typedef struct {
  int32_t max_iter;     /* iteration cap, 1..SP2_MAX_ITER (default 200) */
  int32_t guard;        /* 1 = trace guard on (default), 0 = paper's test only */
  double  qtilde;       /* relaxed order, default 1.8 (§2) */
  int32_t corrections;  /* tensor-core precisions: first-order subspace correction, 0 or 1 (default
                           1).  The correction and the refinement assume X_n is near a projector:
                           a run that ends at the cap (SP2_STOP_CAP) gets neither, D = X_n.  A
                           non-finite value in the assembled D is reported as SP2_ERR_NONFINITE */
  int32_t refine_steps; /* SP2_PREC_MIXED: purification steps after the correction, 0 or 2 (default 2):
                           an alternating pair, X^2 and 2X - X^2, which squares the remaining
                           eigenvalue error */
  int32_t refine_fp64;  /* SP2_PREC_MIXED: 0 = refinement pair on the tensor cores like the
                           expansion (default); 1 = the pair in FP64 (two FP64 squares); 2 = one
                           McWeeny step 3D^2 - 2D^3 = D + E - 2DE with E = D^2 - D, the square in
                           FP64 and the small product DE on the tensor cores (one FP64 square;
                           squares the eigenvalue error on both sides of the gap).  1 and 2 need
                           a single problem and two ld x ld FP64 buffers */
  int32_t launch_mode;  /* 0 = the loops run as CUDA-graph conditional WHILE nodes (default);
                           1 = the same kernels launched on the stream up to the iteration cap,
                           each returning at once after the device-side stop (same results and
                           work plus a few microseconds per idle launch; for tools that cannot
                           follow conditional graph nodes, such as kernel profilers) */
  int32_t history;      /* SP2_PREC_MIXED with corrections: 0 = automatic (default), 1 = keep every
                           iterate X_i in HBM for the derivative pass ((max_iter + 8) slots of
                           6 ld^2 bytes), 2 = keep 11 slots and recompute X_i during the derivative
                           pass (one more square per derivative step, bit-identical result);
                           automatic keeps every iterate when that fits in 60% of free memory */
  int32_t tile;         /* SP2_PREC_MIXED tensor-core tiles: 1 = 128 x 128 output tiles, one per
                           SM (ld = N rounded up to a multiple of 128); 2 = 256 x 256 tiles, one
                           per pair of SMs (cta_group::2 MMAs; ld rounded up to a multiple of
                           256); 0 = tuned (default): at create time one tensor-core product of
                           the handle's problems is timed with each choice on scratch memory and
                           the faster one is kept (when the scratch would exceed 2 GiB, a model
                           of the two kernels' measured rates decides instead); the choice is
                           reported in sp2_info.tile */
  int32_t norm;         /* error measure of the stop test: 0 = Frobenius v_i = ||X_i - X_i^2||_F
                           (default); 1 = the mixed norm m_i of §2, the spectral norm of the
                           matrix of Frobenius norms of the square kernel's tiles (64 x 64 on the
                           FP64 path, 128 x 128 on the mixed path), e_i <= m_i <= v_i, which stays
                           below 1 at large N where v_i may not (power iteration on the device,
                           scratch of (ld/b)^2 doubles); 2 = the spectral norm e_i itself, the
                           error the stop is defined on (§2), estimated after every square by 32
                           Lanczos steps on X - X^2 (a lower bound of e_i within about 1e-3
                           relative; X - X^2 scaled and rounded to FP32 once, 35 small launches per
                           square, scratch of 3 ld doubles + ld (ld + 1) floats + 6 KB): FP64
                           handles (SP2, SP2-ACC and McWeeny) and single-problem tensor-core
                           handles (sp2_create with a tensor-core precision; X - X^2 is formed
                           from the stored X_{k-1} and X_k of the square), SP2_ERR_UNSUPPORTED
                           for batches.
                           sp2_info.v holds the measure used.  Block-sparse handles take 0 or 1
                           (the mixed norm with the 32 x 32 blocks; see sp2_create_bsr) */
  int32_t bsr_cuda_cores; /* block-sparse handles: 0 = block products on the tcgen05 tensor cores
                           (default; each block also kept as two fp16 pieces, see sp2_create_bsr);
                           1 = FP32 block products on the CUDA cores (one fused multiply-add per
                           term in increasing K, then k).  Ignored by dense handles */
} sp2_opts;

#define SP2_MAX_ITER 512

typedef struct {
  int32_t status;          /* sp2_status of the last run (device-side errors) */
  int32_t n_iter;          /* n: D = X_n */
  int32_t stop_reason;     /* sp2_stop_reason */
  int32_t hist_len;        /* entries valid in v[] and trace[] (squares performed) */
  double  lambda_min;      /* Gershgorin bounds used for the scaling */
  double  lambda_max;
  double  loop_ms;         /* device time of the iteration loop of the last run, from CUDA
                              events recorded on the run's stream around the loop */
  const double*  v;        /* v[i] = ||X_i - X_i^2||_F, i < hist_len (host memory owned by the handle) */
  const double*  trace;    /* trace[i] = Tr[X_i], i <= n_iter */
  const uint8_t* p;        /* p[i] in {0,1} for 1 <= i <= n_iter: 1 = X^2, 0 = 2X - X^2 */
  int32_t tile;            /* SP2_PREC_MIXED: tensor-core tiles in use, 1 = 128 x 128 per SM,
                              2 = 256 x 256 per SM pair (as chosen by sp2_opts.tile or its
                              tuner); 0 on the other paths */
} sp2_info;

typedef struct sp2_ctx* sp2_handle;

/* ---- SP2-ACC: homo/lumo-based accelerated expansion (Alg. 4 and Alg. 5) -----------------
 * With bounds of the homo and lumo eigenvalues of F, bounds = {homo_out, homo_in, lumo_in,
 * lumo_out} with homo_out <= homo <= homo_in < lumo_in <= lumo <= lumo_out, the handle's
 * following runs use the predefined polynomial sequence of Alg. 4 with scale-and-fold
 * acceleration instead of the trace-based choice: at the start of each run, right after the
 * Gershgorin bounds, one device thread computes p_i and alpha_i (X_i = ((1 - alpha_i) I +
 * alpha_i X)^2 or 2 alpha_i X - (alpha_i X)^2), n_min (the step after the acceleration is
 * switched off, once both lower bounds are below 0.01) and n_max; the order test runs from
 * n_min on, the trace guard too, and a run that reaches n_max ends there with reason
 * SP2_STOP_SCHEDULE.  Outer bounds beyond the Gershgorin bounds are clamped to them.
 * bounds == NULL returns the handle to the trace-based expansion.  SP2_ERR_INVALID_ARG for
 * unordered or non-finite bounds; a schedule longer than SP2_MAX_ITER steps is reported by
 * the run (status SP2_ERR_INVALID_ARG in sp2_get_info).  Synchronous; must not overlap a run
 * of the same handle.  Works for SP2_PREC_FP64 and SP2_PREC_MIXED handles (the mixed path's
 * first-order correction follows the scaled polynomials). */
int32_t sp2_set_homo_lumo(sp2_handle h, const double* bounds);

/* Outer bounds of the spectrum of F for the scaling (§3: the extremal eigenvalues or any bounds
 * with lambda_min <= lambda_1 and lambda_max >= lambda_N serve), in place of the Gershgorin
 * bounds: bounds = {lambda_min, lambda_max}, used by every later run of the handle (SP2, SP2-ACC
 * and McWeeny scaling alike) and reported in sp2_info; NULL returns to the Gershgorin bounds.
 * Bounds that do not contain the spectrum void the method's guarantees (no check is made).
 * Gershgorin bounds are about sqrt(N) too loose on dense matrices with delocalised eigenvectors,
 * so tighter bounds (from a previous run, or a few Lanczos steps) save squares on either path.
 * Synchronous.  SP2_ERR_INVALID_ARG for non-finite or unordered bounds. */
int32_t sp2_set_bounds(sp2_handle h, const double* bounds);

/* ---- McWeeny expansion (§3) on SP2_PREC_FP64 handles -------------------------------------
 * mode 1: McWeeny, X_0 = (mu I - F) / gamma + I/2 with gamma = 2 max(lmax - mu, mu - lmin)
 * (Gershgorin lmin, lmax), X_i = 3 X_{i-1}^2 - 2 X_{i-1}^3 (two FP64 products per step), and
 * the parameterless stop with C_2^mw = 4 on consecutive errors, log(v_i/4)/log(v_{i-1}) < qtilde
 * (evaluated when v_{i-1} < 1).  mode 2: McW-ACC (§3.1) with gap estimate xi > 0 (some
 * eigenvalue of F lies in [mu - xi/2, mu + xi/2]): X_s = alpha (X - I/2) + I/2 before each step,
 * alpha from the beta recursion; the acceleration is switched off once beta < 0.01 and the stop
 * test runs from the step after.  mode 0 returns to SP2.  mu is the chemical potential (between
 * the homo and lumo eigenvalues); n_occ still selects the trivial cases 0 and N.  Allocates one
 * more ld x ld FP64 buffer on first use; synchronous; SP2_ERR_UNSUPPORTED on mixed handles. */
int32_t sp2_set_mcweeny(sp2_handle h, int32_t mode, double mu, double xi);

/* Fill `opts` with the defaults (max_iter 200, guard on, qtilde 1.8, 1 correction,
 * a 2-step refinement pair on the tensor cores). */
void sp2_default_opts(sp2_opts* opts);

/* Create a handle for problems of size N (1 <= N <= 65536) with n_occ occupied
 * orbitals (0 <= n_occ <= N), allocating its device workspace on the current device:
 * for SP2_PREC_FP64 two N x N FP64 ping-pong buffers padded to a multiple of 64; for
 * SP2_PREC_MIXED the piece arena described at SP2_PREC_MIXED.  opts may be NULL for
 * the defaults.  On failure *out is set to NULL. */
sp2_status sp2_create(int64_t N, int64_t n_occ, int32_t precision, const sp2_opts* opts,
                      sp2_handle* out);

/* Enqueue one purification F_dev -> D_dev on `stream` (Alg. 3 with the stop above).
 * Asynchronous: returns after enqueueing; no host synchronisation happens.  On a
 * device-side error D's contents are unspecified and sp2_get_info reports it. */
sp2_status sp2_run(sp2_handle h, const double* F_dev, double* D_dev, void* stream);

/* The same with host buffers: copies F_host to the device, runs, copies D back
 * into D_host and synchronises `stream` before returning.  Pinned host memory gives
 * the fastest copies; pageable memory works. */
sp2_status sp2_run_host(sp2_handle h, const double* F_host, double* D_host, void* stream);

/* Wait for the handle's last run to finish and describe it.  The arrays in *out stay
 * valid until the next run or sp2_destroy. */
sp2_status sp2_get_info(sp2_handle h, sp2_info* out);

/* Free the handle and its workspace (synchronises the device first).  NULL is a no-op. */
void sp2_destroy(sp2_handle h);

/* ---- batches of problems of uneven size ------------------------------------------------
 * A batch handle holds `count` independent problems (1 <= count <= SP2_MAX_BATCH), problem
 * i of size N[i] with n_occ[i] occupied orbitals.  With SP2_PREC_MIXED one run of the
 * batch is one stream-ordered launch sequence: every round of the expansion is a single
 * persistent tensor-core launch over the tiles of all problems still iterating, each
 * problem stops on its own parameterless test (Alg. 3), and the correction, derivative
 * and refinement rounds are batched the same way.  With SP2_PREC_FP64 the problems run one
 * after the other on the FP64 path.  Workspace is the sum of the single-problem workspaces. */
#define SP2_MAX_BATCH 256
typedef struct sp2_batch_ctx* sp2_batch;

/* Create a batch handle; N and n_occ are host arrays of `count` entries.  opts as for
 * sp2_create (refine_fp64 must be 0 for SP2_PREC_MIXED batches with count > 1). */
sp2_status sp2_create_batch(int32_t count, const int64_t* N, const int64_t* n_occ, int32_t precision,
                            const sp2_opts* opts, sp2_batch* out);

/* Enqueue the batch: F_dev[i] -> D_dev[i] (host arrays of `count` device pointers, each
 * buffer as in sp2_run).  Asynchronous; no host synchronisation. */
sp2_status sp2_run_batch(sp2_batch hb, const double* const* F_dev, double* const* D_dev, void* stream);

/* sp2_set_homo_lumo for problem i of a batch (user order). */
int32_t sp2_set_homo_lumo_batch(sp2_batch hb, int32_t i, const double* bounds);

/* As sp2_set_bounds for problem i of a batch (in the order given to sp2_create_batch). */
int32_t sp2_set_bounds_batch(sp2_batch hb, int32_t i, const double* bounds);

/* Wait for the batch's last run and describe problem i (arrays valid until the next run). */
sp2_status sp2_get_info_batch(sp2_batch hb, int32_t i, sp2_info* out);

/* Free a batch handle (synchronises the device first).  NULL is a no-op. */
void sp2_destroy_batch(sp2_batch hb);

/* ---- block-sparse matrices with block truncation ------------------------------------------
 * The recursive expansion with truncation (Alg. 1: X~_i = X_i + E_i) on a symmetric
 * block-sparse F with 32 x 32 blocks: X~_0 and every iterate are kept as BSR with FP32
 * blocks, and E_i drops every off-diagonal block whose Frobenius norm is below tau
 * (||X_IJ||_F^2 < tau^2, evaluated in FP64 in a fixed order: each block row of squares
 * left to right, then the row sums top to bottom); diagonal blocks are always kept.
 * The squares are block-sparse products over the symbolic pattern of X~^2; bounds,
 * traces, norms and the stop test (Alg. 3 with the trace guard) are FP64, on the device. */
typedef struct sp2_bsr_ctx* sp2_bsr;

/* Truncation rules (the E_i of Alg. 1; the paper names thresholded and error-controlled
 * removal of small matrix parts in its numerical sections but fixes no block rule). */
typedef enum {
  SP2_TRUNC_BLOCK = 0,  /* drop each off-diagonal block with ||X_IJ||_F < tau */
  SP2_TRUNC_ERROR = 1,  /* error-controlled, ||E_i||_F <= tau: over the off-diagonal blocks in
                           (||X_IJ||_F^2, I, J) order, drop the longest prefix whose norms,
                           counted twice (a symmetric pair goes together), add up to at most
                           tau^2; the sums are exact integer multiples of 2^(e-40) with
                           2^e <= tau^2 < 2^(e+1) (each 2 ||X_IJ||_F^2 and tau^2 rounded down to
                           a multiple), so the selection does not depend on summation order */
  SP2_TRUNC_MIXED = 2   /* mixed norm, ||E_i||_2 <= ||E_i||_M <= tau (§6 removes small elements
                           with the mixed norm of the removed part bounded): in the same order,
                           drop the longest prefix in which every block row of the matrix of
                           dropped block norms ||E_IJ||_F sums to at most tau (the spectral
                           norm of that nonnegative symmetric matrix is at most its largest row
                           sum); sums in exact integer multiples of 2^(e-40), 2^e <= tau <
                           2^(e+1), each ||X_IJ||_F and tau rounded down to a multiple */
} sp2_trunc_rule;

/* N: a multiple of 32, at most 65536.  tau >= 0 (0 keeps every stored block).  opts as
 * for sp2_create (corrections, refine_steps and refine_fp64 are ignored).  Block products
 * (opts.bsr_cuda_cores = 0, the default): the square is cut into tiles of 4 x 8 blocks
 * (128 x 256) holding an upper pair of its pattern; each tile is the sum over the K blocks its
 * rows and columns hold of tcgen05 products of the blocks kept as two fp16 pieces of 2^14 x
 * (three piece products, FP32 accumulation in chunks of 4 K blocks, the FP32 iterate and its
 * epilogue as before); an absent block within a tile is the zero block.  Workspace: 4 KB more
 * per block of (N/32)^2 + 1 per iterate.  opts.norm 0 (v_i)
 * or 1 (the mixed norm m_i with the 32 x 32 blocks, estimated after every square by 32
 * Lanczos steps on the (N/32) x (N/32) matrix of block norms of X - X^2, the pairing of the
 * paper's §6 calculations with SP2_TRUNC_MIXED); 2 is SP2_ERR_UNSUPPORTED.  Workspace is
 * about 10 KB per block of (N/32)^2, i.e. ~11 GB at N = 32768.  Rule SP2_TRUNC_BLOCK. */
sp2_status sp2_create_bsr(int64_t N, int64_t n_occ, double tau, const sp2_opts* opts, sp2_bsr* out);

/* As sp2_create_bsr with the truncation rule `rule` (an sp2_trunc_rule; anything else is
 * SP2_ERR_INVALID_ARG).  With SP2_TRUNC_MIXED, tau bounds ||E_i||_M (not ||E_i||_F). */
sp2_status sp2_create_bsr_ex(int64_t N, int64_t n_occ, double tau, int32_t rule, const sp2_opts* opts,
                             sp2_bsr* out);

/* SP2-ACC (Alg. 4 / Alg. 5) on a block-sparse handle, as sp2_set_homo_lumo: bounds = {homo_out,
 * homo_in, lumo_in, lumo_out} for the following runs (the schedule is computed on the device from
 * the run's Gershgorin bounds; the numeric square's epilogue forms ca S + cb X + cc I in FP32 and
 * the truncation follows it as in the trace-based expansion); NULL returns to Alg. 3.
 * Synchronous.  SP2_ERR_INVALID_ARG for unordered or non-finite bounds. */
int32_t sp2_set_homo_lumo_bsr(sp2_bsr h, const double* bounds);

/* As sp2_set_bounds on a block-sparse handle: {lambda_min, lambda_max} for the scaling in place
 * of the Gershgorin bounds of the BSR matrix; NULL returns to them.  Synchronous. */
int32_t sp2_set_bounds_bsr(sp2_bsr h, const double* bounds);

/* F as BSR in device memory: row_ptr [N/32 + 1] (int32), col_idx [nnzb] (int32, sorted
 * in each block row, every diagonal block present), vals [nnzb][32][32] (FP64, row-major
 * blocks); F must be exactly symmetric.  D_dev: NULL, or an N x N FP64 device buffer that
 * receives D densely.  Asynchronous. */
sp2_status sp2_run_bsr(sp2_bsr h, const int32_t* row_ptr_dev, const int32_t* col_idx_dev, const double* vals_dev,
                       int64_t nnzb, double* D_dev, void* stream);

/* Wait for the last run and describe it; *nnzb_out (if not NULL) receives the number of
 * stored blocks of D. */
sp2_status sp2_get_info_bsr(sp2_bsr h, sp2_info* out, int64_t* nnzb_out);

/* Free the handle (synchronises the device first).  NULL is a no-op. */
void sp2_destroy_bsr(sp2_bsr h);

/* Work of the last run's squares (waits for the run): *block_products = 32 x 32 block
 * products X_IK X_JK^T executed (each 2 * 32^3 flops; the tensor-core kernel also multiplies
 * the zero blocks that fill its 4 x 8-block tiles), *needed_products = those with both factors
 * stored and output block J >= I (the sparse square's own work; equal to *block_products on
 * FP32 CUDA cores), *square_blocks = upper blocks of the squares computed, *numeric_ms =
 * summed device time of the numeric-square launches from CUDA events around each launch
 * (launch_mode 1 only; 0 with the graph).  All 0 before the first run. */
sp2_status sp2_get_work_bsr(sp2_bsr h, int64_t* block_products, int64_t* needed_products,
                            int64_t* square_blocks, double* numeric_ms);

/* FP64 purification that allocates no memory (the paper has no counterpart; this is a
 * service for callers that cannot call cudaMalloc, e.g. code running under another
 * component's allocator or in loops where entering the allocator is not allowed).
 * Same method and result as an SP2_PREC_FP64 handle with default options
 * (max_iter 200, guard on, qtilde 1.8), for 1 <= N <= SP2_NOALLOC_MAX_N.
 * F_dev, D_dev: N x N device buffers as in sp2_run.  info_dev: NULL or 4 device
 * int32 that receive (status, n_iter, stop_reason, hist_len) when the run ends.
 * Asynchronous on `stream`.  The workspace is one fixed device array inside the
 * library (about 4.2 MB, held on every GPU that loads the library until exit);
 * N > SP2_NOALLOC_MAX_N returns SP2_ERR_INVALID_ARG.  The first call on a device
 * looks up that array's device address and, under CUDA's default lazy module loading,
 * may load the library's device code and so allocate the array: make that first call
 * as a warm-up, outside any region where allocation is not allowed and before any
 * stream capture.  All calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller. */
#define SP2_NOALLOC_MAX_N 512
sp2_status sp2_run_fp64_noalloc(const double* F_dev, double* D_dev, int64_t N, int64_t n_occ,
                                int32_t* info_dev, void* stream);

/* Human-readable name of a status code (static storage). */
const char* sp2_status_string(int32_t status);

#ifdef __cplusplus
}
#endif
#endif /* SP2_H */
