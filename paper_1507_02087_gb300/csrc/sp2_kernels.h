// Internal launchers shared by the C-ABI layer (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2 {

struct DevState;
namespace tc {
struct Instance;
struct Job;
constexpr int kMaxBatchPtrs = 256;
}  // namespace tc

// F and D of every instance of a run, passed to kernels by value.
struct BatchPtrs {
  const double* F[tc::kMaxBatchPtrs];
  double* D[tc::kMaxBatchPtrs];
};

// SP2-ACC set-up shared by the handles: homo/lumo bounds ordered and finite; the SP2-ACC fields of
// a device state (and its host copy) written, bounds NULL switching the acceleration off.
bool acc_bounds_ok(const double* bounds);
// The caller's outer spectral bounds (bounds[0] < bounds[1]) into a device state, NULL: Gershgorin.
int32_t write_bound_fields(DevState* st_dev, DevState* st_host, const double* bounds);
int32_t write_acc_fields(DevState* st_dev, DevState* st_host, const double* bounds);

// ---- FP64 path ----------------------------------------------------------------------------
// a1 + run set-up: Gershgorin partial bounds over `nparts` blocks, then one block
// that combines them, handles the trivial occupations and computes Tr[X_0].
cudaError_t launch_bounds_and_init(DevState* st, const double* F, int64_t ldf, int N,
                                   double* part_lo, double* part_hi, int* part_bad, int nparts,
                                   cudaStream_t s);
// a2: X_0 = (lmax I - F) / (lmax - lmin) into an ld x ld FP64 buffer.
cudaError_t launch_scale_f64(const DevState* st, const double* F, int64_t ldf, int N, double* X0,
                             int ld, cudaStream_t s);
// a3-a5, a7 for the FP64 path: the body of the device-controlled loop (square +
// finalize), added to `body` as kernel nodes.  `mscr` (T^2 + 2T doubles, or null) is the
// scratch of the mixed-norm stop, used when the state asks for it; `lz` (lanczos_scratch_bytes,
// or null) adds the Lanczos estimate of the spectral norm between the square and the finalize.
cudaError_t add_f64_loop_body(cudaGraph_t body, DevState* st, double* buf0, double* buf1, double* part,
                              int T, cudaGraphConditionalHandle cond, double* mscr = nullptr,
                              void* lz = nullptr, int N = 0, const double* E = nullptr, int64_t ecount = 0);
// Alg. 1's prescribed perturbation: E_i (i < count, N x N row-major each) added to X_0 (initial)
// or to the square just written; in the loop bodies it follows the Lanczos nodes.
cudaError_t launch_perturb(DevState* st, double* buf0, double* buf1, const double* E, int64_t count, int N,
                           int initial, cudaStream_t s);
// The McWeeny expansion's loop body (FP64): shifted square into S, finalize (stop test),
// then X_k = (3 - 2c) S - 2 alpha S X_{k-1}; S is an ld x ld FP64 buffer.
cudaError_t add_mcw_loop_body(cudaGraph_t body, DevState* st, double* buf0, double* buf1, double* S, double* part,
                              int T, cudaGraphConditionalHandle cond, double* mscr, void* lz = nullptr, int N = 0);
cudaError_t launch_mcw_step_plain(DevState* st, double* buf0, double* buf1, double* S, double* part, int T,
                                  cudaStream_t s, double* mscr, void* lz = nullptr, int N = 0);
// Spectral-norm estimate e_{k-1} = ||X_{k-1} - X_{k-1}^2||_2 (Lanczos) of the square just written,
// into st->spec_e: graph nodes after `dep` (the last one in *last), or stream launches.  S is the
// McWeeny step's shifted square (null for SP2 / SP2-ACC); part / ntiles are the square's
// (v^2, trace) partial records, whose v^2 sum sets the FP32 scaling of X - X^2.
size_t lanczos_scratch_bytes(int ld);
cudaError_t add_lanczos_nodes(cudaGraph_t g, cudaGraphNode_t dep, DevState* st, const double* buf0,
                              const double* buf1, const double* S, const double* part, int ntiles, void* lz,
                              int N, int ld, cudaGraphNode_t* last);
cudaError_t launch_lanczos(DevState* st, const double* buf0, const double* buf1, const double* S,
                           const double* part, int ntiles, void* lz, int N, int ld, cudaStream_t s);
// The same estimate for the mixed norm of the block-sparse path: the spectral norm of the nb x nb
// matrix of block norms of X - X^2, built from the square's upper-pair records (row[q], col[q],
// part[2q] = ||(X - X^2)_IJ||_F^2, doubled off the diagonal; *nnz_p pairs); ld = nb rounded up
// to a multiple of 64 for lanczos_scratch_bytes.
cudaError_t launch_lanczos_pairs(DevState* st, const int* row, const int* col, const int* nnz_p, const double* part,
                                 void* lz, int nb, int ld, cudaStream_t s);
// The estimate on the tensor-core path, one problem: X_{k-1} and X_k from the instance's piece
// arena (inst: its device record), part / nparts the forward square's records of 4 doubles.
cudaError_t add_lanczos_tc_nodes(cudaGraph_t g, cudaGraphNode_t dep, DevState* st, const tc::Instance* inst,
                                 const double* part, int nparts, void* lz, int N, int ld, cudaGraphNode_t* last);
cudaError_t launch_lanczos_tc(DevState* st, const tc::Instance* inst, const double* part, int nparts, void* lz,
                              int N, int ld, cudaStream_t s);
// Per-iteration reduction + stop test over `nparts` partial records of `stride` doubles.
cudaError_t add_finalize_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, DevState* st,
                              double* part, int nparts, int stride, cudaGraphConditionalHandle cond,
                              cudaGraphNode_t* node, double* mscr = nullptr);
// D = X_n (or 0 / I / NaN for the special outcomes).
cudaError_t launch_copy_out(const DevState* st, const double* buf0, const double* buf1, int ld, int N,
                            double* D, int64_t ldd, cudaStream_t s);
// One FP64 square + stop test launched directly on a stream (no graph); a no-op once
// st->done is set.
cudaError_t launch_f64_step_plain(DevState* st, double* buf0, double* buf1, double* part, int T,
                                  cudaStream_t s, double* mscr = nullptr, void* lz = nullptr, int N = 0,
                                  const double* E = nullptr, int64_t ecount = 0);
// FP64 purification step `step` (0 or 1) on an ld x ld FP64 matrix (mixed-path refinement).
cudaError_t launch_refine_f64(const DevState* st, const double* Xin, double* Xout, int ld, int step, double* part,
                              cudaStream_t s);
cudaError_t launch_copy_f64(const DevState* st, const double* X, int ld, int N, double* D, int64_t ldd,
                            cudaStream_t s);

// ---- tensor-core path ------------------------------------------------------------------------
// TMA tensor maps over a piece arena of `nslots` ld x ld matrices in piece format `fmt`
// (tc::Fmt; boxes of 128 rows).
cudaError_t tc_make_maps(void* arena, int ld, int nslots, int fmt, CUtensorMap* mapA, CUtensorMap* mapB);
int tc_tiles(int ld, int upper, int pair);
int tc_grid_for(int total_tiles, int pair);
cudaError_t tc_launch(const tc::Job& job, cudaStream_t s);
cudaError_t tc_add_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, const tc::Job& job,
                        cudaGraphNode_t* node);

// Batched elementwise kernels and loop tails of the mixed path (all instances at once).
cudaError_t batch_launch_prologue(const tc::Instance* inst, int count, int pb, int sb, const BatchPtrs& ptrs,
                                  double* part_lo, double* part_hi, int* part_bad, cudaStream_t s);
cudaError_t batch_add_forward_tail(cudaGraph_t g, const cudaGraphNode_t* dep, const tc::Instance* inst, int count,
                                   cudaGraphConditionalHandle cond);
cudaError_t batch_add_deriv_tail(cudaGraph_t g, const cudaGraphNode_t* dep, const tc::Instance* inst, int count,
                                 cudaGraphConditionalHandle cond);
cudaError_t batch_add_corrected_to_pieces(cudaGraph_t g, const cudaGraphNode_t* dep, const tc::Instance* inst,
                                          int count, int sb, int use_dx, cudaGraphNode_t* node);
cudaError_t batch_launch_forward_tail(const tc::Instance* inst, int count, cudaStream_t s);
cudaError_t batch_launch_deriv_tail(const tc::Instance* inst, int count, cudaStream_t s);
cudaError_t batch_launch_corrected_to_pieces(const tc::Instance* inst, int count, int sb, int use_dx,
                                             cudaStream_t s);
cudaError_t batch_launch_assemble(const tc::Instance* inst, int count, int sb, int use_dx, int from_r0,
                                  const BatchPtrs& ptrs, double* f64_buf, cudaStream_t s);
// one FP64-accurate McWeeny step on a single problem (D in Dbuf, S = D^2 in Sbuf, ld = the
// instance's ld): split E = S - D and the pieces of D, E; then D + E - 2 D E into ptrs.D[0]
cudaError_t launch_mcw_split(const tc::Instance* inst, const double* Dbuf, double* Sbuf, int sb, cudaStream_t s);
cudaError_t launch_mcw_out(const tc::Instance* inst, const double* Dbuf, const double* Ebuf, const BatchPtrs& ptrs,
                           int sb, cudaStream_t s);

}  // namespace sp2
