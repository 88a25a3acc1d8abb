/*
 * sp2_testing.h -- internal kernels of libsp2 exposed for unit tests.
 *
 * Not part of the purification API.  These entry points let tests check the
 * tensor-core matrix product, the block truncation and the symbolic square on their
 * own, and run Alg. 1 with prescribed perturbations E_i (the noise of the §4.1
 * example).
 */
#ifndef SP2_TESTING_H
#define SP2_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* C = A B^T with the tcgen05 product used by SP2_PREC_MIXED.
 * `arena_dev`: device buffer of `nslots` slots, each three bf16 planes of ld x ld
 * (row-major, plane-major), so slot s piece p element (i, j) sits at
 * ((s * 3 + p) * ld + i) * ld + j.  A is slot a_slot, B is slot b_slot; each
 * matrix is the sum of its three pieces.  ld must be a positive multiple of 128 and
 * arena_dev 16-byte aligned.  With upper = 1 only C's upper triangle is computed and
 * mirrored (meaningful when A B^T is symmetric); with upper = 0 every element is.
 * tile: 1 = 128 x 128 tiles, one per SM; 2 = 256 x 256 tiles, one per pair of SMs
 * (ld a multiple of 256); 0 = 2 when ld is a multiple of 256, else 1.
 * out_dev: ld x ld FP32, row-major.  Synchronises `stream`; returns an sp2_status
 * (SP2_ERR_INVALID_ARG for bad arguments, SP2_ERR_TIMEOUT if a device-side wait gave up). */
int32_t sp2_test_tc_gemm(const void* arena_dev, int32_t ld, int32_t nslots, int32_t a_slot, int32_t b_slot,
                         int32_t upper, int32_t tile, float* out_dev, void* stream);

/* Block truncation decision of the block-sparse path on its own: for every 32 x 32 block
 * (I, J) of the dense, symmetric N x N FP32 device matrix, keep_dev[I * (N/32) + J] = 1 if
 * the block is kept, else 0, under `rule` (an sp2_trunc_rule of sp2.h): SP2_TRUNC_BLOCK
 * keeps I == J or ||block||_F^2 >= tau^2 (FP64, the fixed summation order of
 * sp2_create_bsr); SP2_TRUNC_ERROR runs the error-controlled selection of the device loop
 * over the upper blocks (I, J >= I) in row-major order.  Synchronises `stream`. */
int32_t sp2_test_bsr_keep(const float* dense_dev, int64_t N, double tau, int32_t rule, uint8_t* keep_dev,
                          void* stream);

/* Symbolic square of the block-sparse path on its own: mask_host is an nb x nb 0/1 block
 * pattern (host, row-major); upper_host receives the pattern of its square restricted to
 * J >= I, as computed by the device kernels.  Synchronous. */
int32_t sp2_test_bsr_square_pattern(const uint8_t* mask_host, int32_t nb, uint8_t* upper_host);

/* Alg. 1 with prescribed perturbations on an FP64 handle (SP2 or SP2-ACC expansion): later runs
 * add E_i to X_i as soon as it is formed, X~_i = X_i + E_i (X_0 after the scaling, X_i after
 * square i), before its trace and error are taken; E_i = 0 for i >= count.  E_dev holds `count`
 * consecutive N x N row-major FP64 device matrices, owned by the caller and read by every run
 * until the hook is switched off (E_dev NULL or count 0).  Synchronous; the loop graph is
 * rebuilt.  SP2_ERR_INVALID_ARG for count < 0 or a missing E_dev; SP2_ERR_UNSUPPORTED on mixed
 * handles and with the McWeeny expansion. */
int32_t sp2_test_set_perturbation(struct sp2_ctx* h, const double* E_dev, int64_t count);

#ifdef __cplusplus
}
#endif
#endif /* SP2_TESTING_H */
