// Mixed-precision path: the batched kernels around the tensor-core GEMM.  Every
// kernel here works on all instances of a batch at once (a single problem is a batch
// of one); per-run buffers (F and D of every instance) arrive by value in a Ptrs
// record, so one launch covers the whole batch with no per-instance host work.
//
//  * bounds / init: Gershgorin bounds per instance, special cases, Tr[X_0].
//  * scale_split: X_0 = (lmax I - F)/(lmax - lmin) in FP64, rounded to FP32 and stored
//    as pieces (history slot 0); F as pieces for the correction (FMT_BF16X3: F itself;
//    FMT_FP16X2: F' = (F - c I) / W' with c and W' the centre and half-width of
//    [lmin, lmax], whose entries lie in [-1, 1] and fit the fp16 range; the shift drops out
//    of dF and the scale is undone where dX_0 is formed).
//  * finalize / check: per-instance reduction + stop test after each round of squares;
//    the loop's condition is cleared once every instance has stopped.
//  * deriv_advance: advances every instance's derivative loop.
//  * corrected_to_pieces, assemble: D = X_n + dX_n (then the refinement pair) in FP64.
//
// Correction (a reading for the mixed path; the paper has no precision scheme):
// the low-precision expansion returns X_n close to the projector P of a matrix near
// F.  The part of F that P does not commute with, dF = P F (I - P) + (I - P) F P,
// drives the first-order change of the projector; pushing dX_0 = -dF/(lmax - lmin)
// through the derivative of the same polynomial sequence (X^2 -> X dX + dX X,
// 2X - X^2 -> 2 dX - (X dX + dX X)) gives dX_n and D = X_n + dX_n.
#include <cuda_bf16.h>

#include "sp2_common.cuh"
#include "sp2_kernels.h"
#include "sp2_tc.cuh"

namespace sp2 {

using tc::Instance;

using tc::piece_load;
using tc::piece_store;

// ---- bounds and initialisation ------------------------------------------------------------
constexpr int kGT = 256;

// Blocks [i * pb, (i+1) * pb) handle instance i; warp per row.
__global__ void __launch_bounds__(kGT)
batch_gersh_kernel(const Instance* inst, int count, int pb, BatchPtrs ptrs, double* part_lo, double* part_hi,
                   int* part_bad) {
  __shared__ double s_lo[kGT / 32], s_hi[kGT / 32];
  __shared__ int s_bad[kGT / 32];
  const int i = blockIdx.x / pb, b = blockIdx.x % pb;
  if (i >= count) return;
  const DevState* st = inst[i].st;
  const int N = st->N;
  const double* F = ptrs.F[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double lo = INFINITY, hi = -INFINITY;
  int bad = 0;
  for (int r = b * (kGT / 32) + warp; r < N; r += pb * (kGT / 32)) {
    const double* row = F + (int64_t)r * N;
    double s = 0.0;
    for (int j = lane; j < N; j += 32) {
      const double a = row[j];
      if (j != r) s += fabs(a);
      if (!isfinite(a)) bad = 1;
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double d = row[r];
    lo = fmin(lo, d - s);
    hi = fmax(hi, d + s);
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; s_bad[warp] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kGT / 32; ++w) {
      s_lo[0] = fmin(s_lo[0], s_lo[w]);
      s_hi[0] = fmax(s_hi[0], s_hi[w]);
      s_bad[0] |= s_bad[w];
    }
    part_lo[blockIdx.x] = s_lo[0];
    part_hi[blockIdx.x] = s_hi[0];
    part_bad[blockIdx.x] = s_bad[0];
  }
}

constexpr int kIT = 1024;

__global__ void __launch_bounds__(kIT)
batch_init_kernel(const Instance* inst, int count, int pb, BatchPtrs ptrs, const double* part_lo,
                  const double* part_hi, const int* part_bad) {
  __shared__ double sm[32];
  __shared__ double s_lmin, s_lmax;
  __shared__ int s_bad;
  const int i = blockIdx.x;
  if (i >= count) return;
  DevState* st = inst[i].st;
  const double* F = ptrs.F[i];
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int b = 0; b < pb; ++b) {
      lo = fmin(lo, part_lo[i * pb + b]);
      hi = fmax(hi, part_hi[i * pb + b]);
      bad |= part_bad[i * pb + b];
    }
    if (!isfinite(lo) || !isfinite(hi)) bad = 1;
    if (st->ubounds) {                           // the caller's outer bounds (§3: any serve)
      lo = st->ub_lo;
      hi = st->ub_hi;
    }
    s_lmin = lo; s_lmax = hi; s_bad = bad;
  }
  __syncthreads();
  const double lmin = s_lmin, lmax = s_lmax, w = lmax - lmin;
  const int N = st->N, nocc = st->nocc;
  double t = 0.0;   // Tr[X_0] over the stored (FP32-rounded) diagonal
  for (int r = threadIdx.x; r < N; r += kIT) t += (double)(float)((lmax - F[(int64_t)r * N + r]) / w);
  t = block_sum<kIT>(t, sm);
  if (threadIdx.x == 0) {
    st->lmin = lmin; st->lmax = lmax;
    st->dk = 0;
    st->k = 0; st->done = 0; st->n_out = 0; st->reason = SP2_STOP_EXACT;
    st->status = SP2_OK; st->out_buf = 0; st->out_mode = OUT_COPY; st->hist_len = 0;
    st->tr[0] = 0.0; st->p[0] = 0;
    if (s_bad) {
      st->status = SP2_ERR_NONFINITE; st->done = 1; st->out_mode = OUT_NAN;
    } else if (nocc == 0) {
      st->done = 1; st->out_mode = OUT_ZERO;
    } else if (nocc == N) {
      st->done = 1; st->out_mode = OUT_IDENTITY;
    } else if (!(lmax > lmin)) {
      st->status = SP2_ERR_NO_GAP; st->done = 1; st->out_mode = OUT_NAN;
    } else {
      st->tr[0] = t;
      if (st->acc && !acc_schedule(st)) {   // SP2-ACC: Alg. 4 from the bounds just found
        st->status = SP2_ERR_INVALID_ARG; st->done = 1; st->out_mode = OUT_NAN;
      }
    }
  }
}

// Blocks [i * sb, (i+1) * sb) handle instance i, grid-stride over its N x N elements.
__global__ void batch_scale_split_kernel(const Instance* inst, int count, int sb, BatchPtrs ptrs) {
  const int i = blockIdx.x / sb, b = blockIdx.x % sb;
  if (i >= count) return;
  const Instance& In = inst[i];
  const DevState* st = In.st;
  if (st->done) return;
  const int N = st->N, ld = In.ld;
  const double lmax = st->lmax, w = st->lmax - st->lmin;
  const int fmt = In.fmt;
  const double cmid = 0.5 * (st->lmax + st->lmin), hw = 0.5 * w;
  const int64_t plane = (int64_t)ld * ld;
  __nv_bfloat16* X = In.arena + (int64_t)tc::xslot(In.lowmem, In.hist0, 0) * In.slot_elems;
  __nv_bfloat16* Fp = In.arena + (int64_t)In.f_slot * In.slot_elems;
  const double* F = ptrs.F[i];
  const int64_t total = (int64_t)N * N;
  for (int64_t e = b * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)sb * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    const double f = F[e];
    const float x = (float)(((r == c ? lmax : 0.0) - f) / w);
    const int64_t off = (int64_t)r * ld + c;
    piece_store(fmt, X, plane, off, x);
    const float fv = fmt == tc::FMT_FP16X2 ? (float)((f - (r == c ? cmid : 0.0)) / hw) : (float)f;
    piece_store(fmt, Fp, plane, off, fv);
  }
}

// ---- per-round reduction, stop test and loop conditions ----------------------------------
constexpr int kFT = 1024;

// One block per instance: (v^2, ||X_{k-1}||_F^2, Tr[X_{k-1}]) partials, one record of 4
// doubles per (tile, epilogue warp).
// Tr[X_k] comes from Tr[X^2] = ||X||_F^2 (symmetric X): ||X_{k-1}||_F^2 after X^2,
// 2 Tr[X_{k-1}] - ||X_{k-1}||_F^2 after 2X - X^2, so the polynomial choice does not
// inherit the bias of the tensor cores' accumulation.
__global__ void __launch_bounds__(kFT) batch_finalize_kernel(const Instance* inst, int count) {
  __shared__ double sm[32];
  const int i = blockIdx.x;
  if (i >= count) return;
  const Instance& In = inst[i];
  DevState* st = In.st;
  if (st->done) return;
  const int nparts = In.nparts;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int t = threadIdx.x; t < nparts; t += kFT) {
    a += In.part[4 * (int64_t)t];
    b += In.part[4 * (int64_t)t + 1];
    c += In.part[4 * (int64_t)t + 2];
  }
  a = block_sum<kFT>(a, sm);
  b = block_sum<kFT>(b, sm);
  c = block_sum<kFT>(c, sm);
  double vk = sqrt(a);
  if (st->norm == 2) vk = st->spec_e;   // e_{k-1}, the Lanczos estimate of the 2-norm (one problem)
  if (st->norm == 1 && In.mscr) {
    // mixed norm over 128 x 128 blocks: a 128 x 128 tile holds 4 records (one per epilogue
    // warp, 32 rows each); a 256 x 256 pair tile holds 16, record 8 rank + 4 hc + q covering
    // rows 128 rank + 32 q .., columns 128 hc ..; off-diagonal blocks are counted twice
    const int nb = In.ld / tc::BM;
    const double* pt = In.part;
    const int pair = In.rec_pair;
    vk = mixed_norm_cta<kFT>(nb, In.mscr, sm, [&](int I, int J) {
      int64_t r0;
      if (pair) r0 = 16 * upper_index(I / 2, J / 2, nb / 2) + 8 * (I & 1) + 4 * (J & 1);
      else r0 = 4 * upper_index(I, J, nb);
      double v2 = 0.0;
      for (int q = 0; q < 4; ++q) v2 += pt[4 * (r0 + q)];
      return I == J ? v2 : 0.5 * v2;
    });
  }
  if (threadIdx.x != 0) return;
  const int k = st->k + 1;
  double tr_new;
  int pk;
  if (st->acc) {   // Alg. 5: X_k = a X^2 + b X + c I, so Tr[X_k] = a ||X||_F^2 + b Tr[X] + c N
    double ca, cb, cc;
    pk = acc_step(st, k, ca, cb, cc);
    tr_new = ca * b + cb * c + cc * (double)st->N;
  } else {
    pk = st->tr[k - 1] > (double)st->nocc ? 1 : 0;
    tr_new = pk ? b : 2.0 * c - b;
  }
  record_and_test(st, pk, vk, tr_new, c);
}

// Clears `cond` once no instance needs another round: which = 0 for the expansion
// (every instance done), 1 for the derivative loop (every instance at dk == n_out).
// Only used inside the loop graphs.
__global__ void batch_check_kernel(const Instance* inst, int count, int which, cudaGraphConditionalHandle cond) {
  __shared__ int busy;
  if (threadIdx.x == 0) busy = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const DevState* st = inst[i].st;
    const bool more = which == 0 ? !st->done : (corrects_run(st) && st->dk < st->n_out);
    if (more) atomicOr(&busy, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && !busy) cudaGraphSetConditional(cond, 0);
}

// After a derivative round: every instance still short of n_out has done one more step.
// In the loop graph (use_cond) it also clears the loop condition when none is left.
__global__ void batch_deriv_advance_kernel(const Instance* inst, int count, cudaGraphConditionalHandle cond,
                                           int use_cond) {
  __shared__ int busy;
  if (threadIdx.x == 0) busy = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    DevState* st = inst[i].st;
    if (corrects_run(st) && st->dk < st->n_out) {
      st->dk += 1;
      if (st->dk < st->n_out) atomicOr(&busy, 1);
    }
  }
  __syncthreads();
  if (use_cond && threadIdx.x == 0 && !busy) cudaGraphSetConditional(cond, 0);
}

// ---- corrected result and output ------------------------------------------------------------

// The corrected D = X_n + dX_n rounded to FP32 and split into pieces in slot r0, the
// input of the tensor-core refinement pair.
__global__ void batch_corrected_to_pieces_kernel(const Instance* inst, int count, int sb, int use_dx) {
  const int i = blockIdx.x / sb, b = blockIdx.x % sb;
  if (i >= count) return;
  const Instance& In = inst[i];
  const DevState* st = In.st;
  if (!corrects_run(st)) return;
  const int N = st->N, ld = In.ld;
  const int64_t plane = (int64_t)ld * ld;
  const int n = st->n_out;
  const __nv_bfloat16* X = In.arena + (int64_t)tc::xslot(In.lowmem, In.hist0, n) * In.slot_elems;
  const __nv_bfloat16* dX = In.arena + (int64_t)(In.dx0 + (n & 1)) * In.slot_elems;
  __nv_bfloat16* R = In.arena + (int64_t)In.r0_slot * In.slot_elems;
  const bool corr = use_dx && n > 0 && st->dk == n;
  const int64_t total = (int64_t)N * N;
  for (int64_t e = b * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)sb * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    const int64_t off = (int64_t)r * ld + c;
    double val = (double)piece_load(In.fmt, X, plane, off);
    if (corr) val += (double)piece_load(In.fmt, dX, plane, off);
    piece_store(In.fmt, R, plane, off, (float)val);
  }
}

// D in FP64: from slot r0 (after the tensor-core refinement) when from_r0, else
// X_n (+ dX_n with the correction); 0 / I / NaN for the special outcomes.  A run that reached
// the cap is neither corrected nor refined: D = X_n.  A non-finite value in a D the run
// reported as ok sets SP2_ERR_NONFINITE.
__global__ void batch_assemble_kernel(const Instance* inst, int count, int sb, int use_dx, int from_r0,
                                      BatchPtrs ptrs, int to_f64_buf, double* f64_buf) {
  const int i = blockIdx.x / sb, b = blockIdx.x % sb;
  if (i >= count) return;
  const Instance& In = inst[i];
  DevState* st = In.st;
  if (!corrects_run(st)) {
    from_r0 = 0;
    use_dx = 0;
  }
  const int N = st->N, ld = In.ld;
  const int mode = st->out_mode;
  const int64_t plane = (int64_t)ld * ld;
  const int n = st->n_out;
  const __nv_bfloat16* X =
      In.arena + (int64_t)(from_r0 ? In.r0_slot : tc::xslot(In.lowmem, In.hist0, n)) * In.slot_elems;
  const __nv_bfloat16* dX = In.arena + (int64_t)(In.dx0 + (n & 1)) * In.slot_elems;
  const bool corr = !from_r0 && use_dx && n > 0 && st->dk == n;
  double* D = to_f64_buf ? f64_buf : ptrs.D[i];
  const int64_t ldd = to_f64_buf ? ld : N;
  const int64_t total = (int64_t)N * N;
  for (int64_t e = b * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)sb * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    double val;
    if (mode == OUT_COPY) {
      const int64_t off = (int64_t)r * ld + c;
      val = (double)piece_load(In.fmt, X, plane, off);
      if (corr) val += (double)piece_load(In.fmt, dX, plane, off);
    } else if (mode == OUT_ZERO) {
      val = 0.0;
    } else if (mode == OUT_IDENTITY) {
      val = (r == c) ? 1.0 : 0.0;
    } else {
      val = __longlong_as_double(0x7ff8000000000000ll);
    }
    if (mode == OUT_COPY && !isfinite(val)) atomicCAS(&st->status, (int32_t)SP2_OK, (int32_t)SP2_ERR_NONFINITE);
    D[(int64_t)r * ldd + c] = val;
  }
}

// ---- one FP64-accurate McWeeny step (refinement option 2, single problem) --------------------
// p(D) = 3 D^2 - 2 D^3 = D + E - 2 D E with E = D^2 - D.  D^2 comes from the FP64 square; E is
// tiny next to D, so the product D E runs on the tensor cores (its FP32-level relative error
// lands far below the FP64 error of E).  Each eigenvalue error e of D becomes about 3 e^2, on
// both sides of the gap.
// mcw_split: E = S - D in place of S = D^2 (FP64, both ld x ld), D and E as pieces into the
// refinement slots r0 and r0 + 1.
__global__ void mcw_split_kernel(const Instance* inst, const double* Dbuf, double* Sbuf, int sb) {
  const Instance& In = inst[0];
  const DevState* st = In.st;
  if (!corrects_run(st)) return;
  const int N = st->N, ld = In.ld;
  const int64_t plane = (int64_t)ld * ld;
  __nv_bfloat16* Dp = In.arena + (int64_t)In.r0_slot * In.slot_elems;
  __nv_bfloat16* Ep = In.arena + (int64_t)(In.r0_slot + 1) * In.slot_elems;
  const int64_t total = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)sb * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    const int64_t off = (int64_t)r * ld + c;
    const double d = Dbuf[off];
    const double ev = Sbuf[off] - d;
    Sbuf[off] = ev;
    piece_store(In.fmt, Dp, plane, off, (float)d);
    piece_store(In.fmt, Ep, plane, off, (float)ev);
  }
}

// mcw_out: D_out = D + E - 2 P, P = D E from the pieces in m_slot (the output modes of the
// special cases as in batch_assemble_kernel).
__global__ void mcw_out_kernel(const Instance* inst, const double* Dbuf, const double* Ebuf, BatchPtrs ptrs,
                               int sb) {
  const Instance& In = inst[0];
  const DevState* st = In.st;
  const int N = st->N, ld = In.ld;
  const int mode = st->out_mode;
  const int64_t plane = (int64_t)ld * ld;
  const __nv_bfloat16* Pp = In.arena + (int64_t)In.m_slot * In.slot_elems;
  double* D = ptrs.D[0];
  const int64_t total = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)sb * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    double val;
    if (mode == OUT_COPY && corrects_run(st)) {
      const int64_t off = (int64_t)r * ld + c;
      val = Dbuf[off] + Ebuf[off] - 2.0 * (double)piece_load(In.fmt, Pp, plane, off);
    } else if (mode == OUT_COPY && st->status == SP2_OK) {
      val = Dbuf[(int64_t)r * ld + c];     // a capped run: X_n as assembled, not refined
    } else if (mode == OUT_ZERO) {
      val = 0.0;
    } else if (mode == OUT_IDENTITY) {
      val = (r == c) ? 1.0 : 0.0;
    } else {
      val = __longlong_as_double(0x7ff8000000000000ll);
    }
    D[e] = val;
  }
}

// ---- host-side launchers ------------------------------------------------------------------

static cudaError_t add_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, void* func, dim3 grid,
                            dim3 block, void** args, cudaGraphNode_t* node) {
  cudaKernelNodeParams kp = {};
  kp.func = func;
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

cudaError_t batch_launch_prologue(const Instance* inst, int count, int pb, int sb, const BatchPtrs& ptrs,
                                  double* part_lo, double* part_hi, int* part_bad, cudaStream_t s) {
  batch_gersh_kernel<<<count * pb, kGT, 0, s>>>(inst, count, pb, ptrs, part_lo, part_hi, part_bad);
  batch_init_kernel<<<count, kIT, 0, s>>>(inst, count, pb, ptrs, part_lo, part_hi, part_bad);
  batch_scale_split_kernel<<<count * sb, 256, 0, s>>>(inst, count, sb, ptrs);
  return cudaGetLastError();
}

cudaError_t batch_add_forward_tail(cudaGraph_t g, const cudaGraphNode_t* dep, const Instance* inst, int count,
                                   cudaGraphConditionalHandle cond) {
  cudaGraphNode_t n_fin, n_chk;
  void* a1[] = {&inst, &count};
  cudaError_t e = add_node(g, dep, 1, (void*)batch_finalize_kernel, dim3(count), dim3(kFT), a1, &n_fin);
  if (e != cudaSuccess) return e;
  int which = 0;
  void* a2[] = {&inst, &count, &which, &cond};
  return add_node(g, &n_fin, 1, (void*)batch_check_kernel, dim3(1), dim3(256), a2, &n_chk);
}

cudaError_t batch_add_deriv_tail(cudaGraph_t g, const cudaGraphNode_t* dep, const Instance* inst, int count,
                                 cudaGraphConditionalHandle cond) {
  cudaGraphNode_t n;
  int use_cond = 1;
  void* a[] = {&inst, &count, &cond, &use_cond};
  return add_node(g, dep, 1, (void*)batch_deriv_advance_kernel, dim3(1), dim3(256), a, &n);
}

// Stream-launched forms of the loop tails (launch_mode 1: no graph).
cudaError_t batch_launch_forward_tail(const Instance* inst, int count, cudaStream_t s) {
  batch_finalize_kernel<<<count, kFT, 0, s>>>(inst, count);
  return cudaGetLastError();
}

cudaError_t batch_launch_deriv_tail(const Instance* inst, int count, cudaStream_t s) {
  batch_deriv_advance_kernel<<<1, 256, 0, s>>>(inst, count, 0, 0);
  return cudaGetLastError();
}

cudaError_t batch_launch_corrected_to_pieces(const Instance* inst, int count, int sb, int use_dx, cudaStream_t s) {
  batch_corrected_to_pieces_kernel<<<count * sb, 256, 0, s>>>(inst, count, sb, use_dx);
  return cudaGetLastError();
}

cudaError_t batch_add_corrected_to_pieces(cudaGraph_t g, const cudaGraphNode_t* dep, const Instance* inst, int count,
                                          int sb, int use_dx, cudaGraphNode_t* node) {
  void* a[] = {&inst, &count, &sb, &use_dx};
  return add_node(g, dep, 1, (void*)batch_corrected_to_pieces_kernel, dim3(count * sb), dim3(256), a, node);
}

cudaError_t batch_launch_assemble(const Instance* inst, int count, int sb, int use_dx, int from_r0,
                                  const BatchPtrs& ptrs, double* f64_buf, cudaStream_t s) {
  batch_assemble_kernel<<<count * sb, 256, 0, s>>>(inst, count, sb, use_dx, from_r0, ptrs, f64_buf ? 1 : 0,
                                                   f64_buf);
  return cudaGetLastError();
}

}  // namespace sp2

namespace sp2 {
cudaError_t launch_mcw_split(const tc::Instance* inst, const double* Dbuf, double* Sbuf, int sb, cudaStream_t s) {
  mcw_split_kernel<<<sb, 256, 0, s>>>(inst, Dbuf, Sbuf, sb);
  return cudaGetLastError();
}
cudaError_t launch_mcw_out(const tc::Instance* inst, const double* Dbuf, const double* Ebuf, const BatchPtrs& ptrs,
                           int sb, cudaStream_t s) {
  mcw_out_kernel<<<sb, 256, 0, s>>>(inst, Dbuf, Ebuf, ptrs, sb);
  return cudaGetLastError();
}
}  // namespace sp2
