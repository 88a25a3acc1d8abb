// Shared device-side state and helpers of the SP2 purification path.
//
// One Sp2DevState lives in device memory per handle.  The kernels of a run read
// and advance it, so the whole expansion (Alg. 3) -- the polynomial choice, the
// history of v_i and Tr[X_i], and the stop test -- is decided on the device with
// no host round trip per iteration.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sp2.h"

namespace sp2 {

// C_2^sp = (71 + 17 sqrt(17)) / 32 (§4), written as a literal of the closed form.
constexpr double kC2sp = 4.409149863609382;  // the double nearest the closed form

// How the output D is produced once the loop ends.
enum OutMode : int32_t {
  OUT_COPY = 0,      // D = X_n from ping-pong buffer out_buf
  OUT_ZERO = 1,      // n_occ == 0
  OUT_IDENTITY = 2,  // n_occ == N
  OUT_NAN = 3        // an error: D is filled with NaN
};

struct DevState {
  // fixed for a handle
  int32_t N;
  int32_t ld;          // padded leading dimension of the ping-pong buffers
  int32_t nocc;
  int32_t max_iter;
  int32_t guard;
  int32_t _pad0;
  double qtilde;
  // set by the bounds pass
  double lmin, lmax;
  // progress of the current run
  int32_t k;           // squares completed so far
  int32_t done;
  int32_t n_out;       // D = X_{n_out}
  int32_t reason;      // sp2_stop_reason
  int32_t status;      // sp2_status
  int32_t out_buf;     // 0 or 1
  int32_t out_mode;    // OutMode
  int32_t hist_len;
  int32_t dk;          // derivative steps completed (mixed path correction)
  int32_t round_fp32;  // 1: X_0 is rounded to FP32 (mixed path)
  int32_t iter_active; // block-sparse path: the current loop round squares (set at its start)
  int32_t _pad1;
  // block-sparse path, work of the current run's squares: 32 x 32 block products and
  // upper blocks of the squares computed
  unsigned long long bprod;
  unsigned long long sblocks;
  // history
  double v[SP2_MAX_ITER + 2];
  double tr[SP2_MAX_ITER + 2];
  uint8_t p[SP2_MAX_ITER + 2];
};

// The paper's convergence-order test (Alg. 3; §2 relaxed order qtilde), only
// evaluated when v_{i-2} < 1, and in its logarithmic form.
__device__ __forceinline__ bool order_test_stops(double v_i, double v_im2, double qtilde) {
  if (v_im2 == 0.0) return true;
  if (!(v_im2 < 1.0)) return false;
  if (v_i == 0.0) return false;
  return log(v_i / kC2sp) / log(v_im2) < qtilde;
}

// Records square k = st->k + 1 (v_{k-1}, Tr[X_k], p_k) and applies the stop rules in
// the order the iteration meets them: the order test for X_{k-1} (Alg. 3, evaluated
// one square late because v_{k-1} needs X_{k-1}^2), the cap, then the trace guard for
// X_k, which compares Tr[X_k] with `tr_ref` = Tr[X_{k-1}].  Returns true if the run
// stops; single thread.
__device__ __forceinline__ bool record_and_test(DevState* st, int pk, double v_prev, double tr_new,
                                                double tr_ref) {
  const int k = st->k + 1;
  st->v[k - 1] = v_prev;
  st->tr[k] = tr_new;
  st->p[k] = (uint8_t)pk;
  st->k = k;
  st->hist_len = k;
  const int i = k - 1;
  bool stop = true;
  if (!isfinite(v_prev) || !isfinite(tr_new)) {
    st->status = SP2_ERR_NONFINITE; st->out_mode = OUT_NAN; st->n_out = i;
  } else if (k == 1 && v_prev == 0.0) {
    st->reason = SP2_STOP_EXACT; st->n_out = 0; st->out_buf = 0;
  } else if (i >= 2 && st->p[i] != st->p[i - 1] && order_test_stops(st->v[i], st->v[i - 2], st->qtilde)) {
    st->reason = SP2_STOP_ORDER; st->n_out = i; st->out_buf = i & 1;
  } else if (i >= st->max_iter) {
    st->reason = SP2_STOP_CAP; st->n_out = i; st->out_buf = i & 1;
  } else if (st->guard && ((pk == 1 && tr_new >= tr_ref) || (pk == 0 && tr_new <= tr_ref))) {
    st->reason = SP2_STOP_TRACE_GUARD; st->n_out = k; st->out_buf = k & 1;
  } else {
    stop = false;
  }
  if (stop) st->done = 1;
  return stop;
}

// Deterministic block-wide sum (fixed shuffle tree, then warps in index order).
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* smem) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) smem[warp] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) t += smem[w];
    smem[0] = t;
  }
  __syncthreads();
  t = smem[0];
  __syncthreads();
  return t;
}

// Row/column of upper-triangular tile `t` in a T x T tile grid, tiles ordered by row.
__device__ __forceinline__ void upper_tile(int t, int T, int& I, int& J) {
  int i = 0, rem = t;
  while (rem >= T - i) { rem -= T - i; ++i; }
  I = i;
  J = i + rem;
}

}  // namespace sp2
