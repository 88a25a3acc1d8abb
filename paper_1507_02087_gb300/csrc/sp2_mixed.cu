// Mixed-precision path: elementwise kernels around the tensor-core GEMM.
//
//  * scale_split: X_0 = (lmax I - F)/(lmax - lmin) in FP64, rounded to FP32 and stored
//    as three bf16 pieces (history slot 0); F itself as pieces for the correction.
//  * deriv_finalize: advances the derivative loop and clears its condition.
//  * assemble: D = X_n + dX_n in FP64 (the first-order correction), or X_n alone.
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

__device__ __forceinline__ void split3_(float x, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
  p0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ float join3_(const __nv_bfloat16* s, int64_t plane, int64_t off) {
  return (__bfloat162float(s[off]) + __bfloat162float(s[plane + off])) + __bfloat162float(s[2 * plane + off]);
}

__global__ void scale_split_kernel(const DevState* st, const double* __restrict__ F, int64_t ldf,
                                   __nv_bfloat16* __restrict__ arena, int64_t slot_elems, int ld, int x_slot,
                                   int f_slot) {
  if (st->done) return;
  const int N = st->N;
  const double lmax = st->lmax, w = st->lmax - st->lmin;
  const int64_t plane = (int64_t)ld * ld;
  __nv_bfloat16* X = arena + (int64_t)x_slot * slot_elems;
  __nv_bfloat16* Fp = arena + (int64_t)f_slot * slot_elems;
  const int64_t total = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const double f = F[(int64_t)i * ldf + j];
    const float x = (float)(((i == j ? lmax : 0.0) - f) / w);
    const int64_t off = (int64_t)i * ld + j;
    __nv_bfloat16 a, b, c;
    split3_(x, a, b, c);
    X[off] = a; X[plane + off] = b; X[2 * plane + off] = c;
    split3_((float)f, a, b, c);
    Fp[off] = a; Fp[plane + off] = b; Fp[2 * plane + off] = c;
  }
}

__global__ void deriv_finalize_kernel(DevState* st, cudaGraphConditionalHandle cond) {
  const bool ok_run = st->status == SP2_OK && st->out_mode == OUT_COPY;
  if (!ok_run || st->dk >= st->n_out) {
    cudaGraphSetConditional(cond, 0);
    return;
  }
  st->dk += 1;
  if (st->dk >= st->n_out) cudaGraphSetConditional(cond, 0);
}

// The corrected D = X_n + dX_n rounded to FP32 and split into pieces in slot r0, the
// input of the tensor-core refinement pair.
__global__ void corrected_to_pieces_kernel(const DevState* st, __nv_bfloat16* __restrict__ arena, int64_t slot_elems,
                                           int ld, int hist0, int dx0, int use_dx, int r0) {
  if (st->status != SP2_OK || st->out_mode != OUT_COPY) return;
  const int N = st->N;
  const int64_t plane = (int64_t)ld * ld;
  const int n = st->n_out;
  const __nv_bfloat16* X = arena + (int64_t)(hist0 + n) * slot_elems;
  const __nv_bfloat16* dX = arena + (int64_t)(dx0 + (n & 1)) * slot_elems;
  __nv_bfloat16* R = arena + (int64_t)r0 * slot_elems;
  const bool corr = use_dx && n > 0 && st->dk == n;
  const int64_t total = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const int64_t off = (int64_t)i * ld + j;
    double val = (double)join3_(X, plane, off);
    if (corr) val += (double)join3_(dX, plane, off);
    __nv_bfloat16 a, b, c;
    split3_((float)val, a, b, c);
    R[off] = a; R[plane + off] = b; R[2 * plane + off] = c;
  }
}

// D in FP64: from slot r0 (after the tensor-core refinement) when from_r0, else
// X_n (+ dX_n with the correction).
__global__ void assemble_kernel(const DevState* st, const __nv_bfloat16* __restrict__ arena, int64_t slot_elems,
                                int ld, int hist0, int dx0, int use_dx, int r0, int from_r0,
                                double* __restrict__ D, int64_t ldd) {
  const int N = st->N;
  const int mode = st->out_mode;
  const int64_t plane = (int64_t)ld * ld;
  const int n = st->n_out;
  const __nv_bfloat16* X = arena + (int64_t)(from_r0 ? r0 : hist0 + n) * slot_elems;
  const __nv_bfloat16* dX = arena + (int64_t)(dx0 + (n & 1)) * slot_elems;
  const bool corr = !from_r0 && use_dx && n > 0 && st->dk == n;
  const int64_t total = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    double val;
    if (mode == OUT_COPY) {
      const int64_t off = (int64_t)i * ld + j;
      val = (double)join3_(X, plane, off);
      if (corr) val += (double)join3_(dX, plane, off);
    } else if (mode == OUT_ZERO) {
      val = 0.0;
    } else if (mode == OUT_IDENTITY) {
      val = (i == j) ? 1.0 : 0.0;
    } else {
      val = __longlong_as_double(0x7ff8000000000000ll);
    }
    D[(int64_t)i * ldd + j] = val;
  }
}

static int ew_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

cudaError_t launch_scale_split(const DevState* st, const double* F, int64_t ldf, int N, void* arena,
                               int64_t slot_elems, int ld, int x_slot, int f_slot, cudaStream_t s) {
  scale_split_kernel<<<ew_blocks((int64_t)N * N), 256, 0, s>>>(st, F, ldf, (__nv_bfloat16*)arena, slot_elems, ld,
                                                                x_slot, f_slot);
  return cudaGetLastError();
}

cudaError_t add_deriv_finalize_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, DevState* st,
                                    cudaGraphConditionalHandle cond, cudaGraphNode_t* node) {
  void* args[] = {&st, &cond};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)deriv_finalize_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

cudaError_t launch_assemble(const DevState* st, const void* arena, int64_t slot_elems, int ld, int hist0, int dx0,
                            int use_dx, int r0, int from_r0, int N, double* D, int64_t ldd, cudaStream_t s) {
  assemble_kernel<<<ew_blocks((int64_t)N * N), 256, 0, s>>>(st, (const __nv_bfloat16*)arena, slot_elems, ld, hist0,
                                                             dx0, use_dx, r0, from_r0, D, ldd);
  return cudaGetLastError();
}

cudaError_t add_corrected_to_pieces_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, const DevState* st,
                                         void* arena, int64_t slot_elems, int ld, int hist0, int dx0, int use_dx,
                                         int r0, int N, cudaGraphNode_t* node) {
  __nv_bfloat16* a = (__nv_bfloat16*)arena;
  void* args[] = {&st, &a, &slot_elems, &ld, &hist0, &dx0, &use_dx, &r0};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)corrected_to_pieces_kernel;
  kp.gridDim = dim3(ew_blocks((int64_t)N * N));
  kp.blockDim = dim3(256);
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

}  // namespace sp2
