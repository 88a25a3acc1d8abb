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
