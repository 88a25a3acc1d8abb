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

/* As sp2_test_tc_gemm for either piece format of the tensor-core path.  fmt 0: three bf16
 * planes per slot as above; fmt 1: two fp16 planes per slot holding S x split as
 * p0 = fp16(S x), p1 = fp16(S x - p0) with S = 2^14, so slot s piece p element (i, j) sits
 * at ((s * 2 + p) * ld + i) * ld + j and the matrix is (p0 + p1) / S.  lowprec 0 forms the
 * format's full product (bf16: the six piece products with a + b <= 2; fp16: p0 q0 + p0 q1 +
 * p1 q0); lowprec 1 the low-precision one (bf16: the three with a + b <= 1; fp16: p0 q0).
 * out_dev receives C itself (the fp16 scale removed). */
int32_t sp2_test_tc_gemm_ex(const void* arena_dev, int32_t ld, int32_t nslots, int32_t a_slot, int32_t b_slot,
                            int32_t upper, int32_t tile, int32_t fmt, int32_t lowprec, float* out_dev,
                            void* stream);

/* The bounded waits of the tensor-core kernel, made to run out: one launch of the 128 x 128
 * (one SM per tile) bf16 product C = A A^T over slot 0 of a one-slot arena as in
 * sp2_test_tc_gemm (ld a multiple of 128, every element computed), with every mbarrier wait
 * limited to `wait_ms` (1..2000) and CTA 0 leaving the first stage of its copy ring unarmed:
 * its MMA thread's wait for that stage gives up, the CTA's other warps give up or stop, wait
 * (bounded) for the copies they issued, free their tensor memory and return, while the other
 * CTAs finish their tiles.  Returns SP2_ERR_TIMEOUT when the waits gave up as they must, the
 * tiles of the other CTAs are written to out_dev.  Synchronises `stream`.  No GPU fault is
 * involved: the kernel returns normally and the context stays usable. */
int32_t sp2_test_tc_timeout(const void* arena_dev, int32_t ld, int32_t wait_ms, float* out_dev, void* stream);

/* 1 if this library was built with device-side bounds checks (libsp2_debug.so, built with
 * SP2_DEVICE_CHECKS=1), 0 for the release library. */
int32_t sp2_build_device_checks(void);

/* A device-side bounds check made to fail, debug library only: one launch of the bf16 product
 * of sp2_test_tc_gemm over an arena of `nslots` slots (ld a multiple of 128, 128 x 128 tiles)
 * whose A operand is slot `bad_slot`, nslots <= bad_slot < nslots + 1024, which the host does not
 * reject here.  That slot only addresses tensor-map loads, which read zeros outside the map, so
 * the launch is safe even without the check; with it, every tile is skipped and the call returns
 * SP2_ERR_BOUNDS.  The release library returns SP2_ERR_UNSUPPORTED without launching anything.
 * Synchronises `stream`. */
int32_t sp2_test_tc_bounds(const void* arena_dev, int32_t ld, int32_t nslots, int32_t bad_slot, float* out_dev,
                           void* stream);

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
