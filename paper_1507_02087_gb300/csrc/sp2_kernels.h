// Internal launchers shared by the C-ABI layer (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2 {

struct DevState;

// a1 + run set-up: Gershgorin partial bounds over `nparts` blocks, then one block
// that combines them, handles the trivial occupations and computes Tr[X_0].
cudaError_t launch_bounds_and_init(DevState* st, const double* F, int64_t ldf, int N,
                                   double* part_lo, double* part_hi, int* part_bad, int nparts,
                                   cudaStream_t s);

// a2: X_0 = (lmax I - F) / (lmax - lmin) into an ld x ld FP64 buffer.
cudaError_t launch_scale_f64(const DevState* st, const double* F, int64_t ldf, int N, double* X0,
                             int ld, cudaStream_t s);

// a3-a5, a7 for the FP64 path: the body of the device-controlled loop (square +
// finalize), added to `body` as kernel nodes.
cudaError_t add_f64_loop_body(cudaGraph_t body, DevState* st, double* buf0, double* buf1, double* part,
                              int T, cudaGraphConditionalHandle cond);

// D = X_n (or 0 / I / NaN for the special outcomes).
cudaError_t launch_copy_out(const DevState* st, const double* buf0, const double* buf1, int ld, int N,
                            double* D, int64_t ldd, cudaStream_t s);

}  // namespace sp2
