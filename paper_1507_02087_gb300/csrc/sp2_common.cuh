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

// Debug builds (-DSP2_DEVICE_CHECKS=1, the library libsp2_debug.so) check indices that the
// device computes from its own state against the buffers they address.  A failed check
// records SP2_ERR_BOUNDS in the run's error word and the guarded access is skipped; release
// builds compile the checks away.
#ifndef SP2_DEVICE_CHECKS
#define SP2_DEVICE_CHECKS 0
#endif

namespace sp2 {

// `ok` in release builds; in debug builds a false `ok` also records SP2_ERR_BOUNDS in *err
// (the first error recorded wins).
__device__ __forceinline__ bool dcheck(bool ok, int32_t* err) {
#if SP2_DEVICE_CHECKS
  if (!ok) atomicCAS(err, 0, (int32_t)SP2_ERR_BOUNDS);
  return ok;
#else
  (void)ok;
  (void)err;
  return true;
#endif
}

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
  int32_t norm;        // error measure of the stop: 0 = Frobenius v_i, 1 = mixed norm m_i (§2),
                       // 2 = spectral e_i (Lanczos; FP64 path)
  // block-sparse path, work of the current run's squares: 32 x 32 block products executed,
  // upper blocks of the squares computed, and the block products the squares need (both
  // factors stored, output block J >= I)
  unsigned long long bprod;
  unsigned long long sblocks;
  unsigned long long uprod;
  double spec_e;       // norm = 2: the Lanczos estimate of ||X_{k-1} - X_{k-1}^2||_2 of the last square
  double tr_shift;     // Tr[E_k] of a prescribed perturbation added to the square just written
  int32_t ubounds;     // 1: the caller's outer bounds (ub_lo, ub_hi) replace the Gershgorin bounds
  int32_t _pad4;
  double ub_lo, ub_hi;
  // SP2-ACC (Alg. 4 / Alg. 5): set by sp2_set_homo_lumo, schedule filled by the init kernel
  int32_t acc;         // 1: homo/lumo-based accelerated expansion
  int32_t n_min;       // first step of the stop test (acceleration off)
  int32_t n_max;       // last step of the schedule
  int32_t _pad2;
  double hl[4];        // homo_out, homo_in, lumo_in, lumo_out
  double alpha[SP2_MAX_ITER + 2];
  uint8_t psched[SP2_MAX_ITER + 2];
  // McWeeny expansion (§3; FP64 path): set by sp2_set_mcweeny; alpha[] holds the McW-ACC
  // factors and n_min the first step of the stop test
  int32_t mcw;         // 0: SP2, 1: McWeeny, 2: McW-ACC
  int32_t _pad3;
  double mu, xi;       // chemical potential, gap estimate (McW-ACC)
  // initial scaling X_0 = (scale_a I - F) / scale_w: SP2 (lmax, lmax - lmin); McWeeny
  // (mu + gamma/2, gamma) with gamma = 2 max(lmax - mu, mu - lmin)
  double scale_a, scale_w;
  // history
  double v[SP2_MAX_ITER + 2];
  double tr[SP2_MAX_ITER + 2];
  uint8_t p[SP2_MAX_ITER + 2];
};

// A run whose iterate X_n the tensor-core path corrects and refines: it ran without error to a
// stop rule.  A run that reached the iteration cap did not converge, and the first-order
// correction and the refinement, which assume X_n is near a projector, would only push its
// values out of range; D is then X_n itself.
__host__ __device__ __forceinline__ bool corrects_run(const DevState* st) {
  return st->status == SP2_OK && st->out_mode == OUT_COPY && st->reason != SP2_STOP_CAP;
}

// The paper's convergence-order test (Alg. 3; §2 relaxed order qtilde), only
// evaluated when v_{i-2} < 1, and in its logarithmic form.
__device__ __forceinline__ bool order_test_stops(double v_i, double v_im2, double qtilde, double C = kC2sp) {
  if (v_im2 == 0.0) return true;
  if (!(v_im2 < 1.0)) return false;
  if (v_i == 0.0) return false;
  return log(v_i / C) / log(v_im2) < qtilde;
}

// McWeeny (§3): C_2^mw = 4, the maximum of (p(x) - p(x)^2) / (x - x^2)^2 = 3 + 4x - 4x^2.
constexpr double kC2mw = 4.0;

// ---- SP2-ACC ---------------------------------------------------------------------------
// Alg. 4 on the device (one thread): the polynomial p_i and scale-and-fold factor alpha_i of
// every step, n_min (the step after the acceleration is switched off, once both lower
// bounds are below delta = 0.01) and n_max (bounds converged to machine epsilon and the
// last two polynomials different; the printed loop condition joins its two parts with
// "and", read as "or").  Outer bounds beyond [lmin, lmax] are clamped to it.  Every value
// is one correctly rounded double operation in the order of the algorithm (no fused
// multiply-add), so the schedule equals a host evaluation of the same formulas bit for
// bit.  Returns false if the schedule does not converge within SP2_MAX_ITER steps.
__device__ __forceinline__ double acc_fold(double a, double x) {   // ((1 - a) + a x)^2
  const double y = __dadd_rn(__dsub_rn(1.0, a), __dmul_rn(a, x));
  return __dmul_rn(y, y);
}
__device__ __forceinline__ double acc_lift(double a, double x) {   // 2 a x - (a x)^2
  const double y = __dmul_rn(a, x);
  return __dsub_rn(__dmul_rn(__dmul_rn(2.0, a), x), __dmul_rn(y, y));
}

__device__ inline bool acc_schedule(DevState* st) {
  const double lmin = st->lmin, lmax = st->lmax;
  const double homo_out = fmax(st->hl[0], lmin), homo_in = st->hl[1];
  const double lumo_in = st->hl[2], lumo_out = fmin(st->hl[3], lmax);
  const double W = __dsub_rn(lmax, lmin);
  double bu = __dsub_rn(1.0, __ddiv_rn(__dsub_rn(lmax, homo_in), W));
  double bl = __dsub_rn(1.0, __ddiv_rn(__dsub_rn(lmax, homo_out), W));
  double gu = __ddiv_rn(__dsub_rn(lmax, lumo_in), W);
  double gl = __ddiv_rn(__dsub_rn(lmax, lumo_out), W);
  const double eps = 2.220446049250313e-16;   // 2^-52
  double delta = 0.01;
  int i = 0, nmin = -1;
  st->psched[0] = 0;
  st->alpha[0] = 1.0;
  while ((__dsub_rn(bu, __dmul_rn(bu, bu)) > eps || __dsub_rn(gu, __dmul_rn(gu, gu)) > eps) || i < 2 ||
         st->psched[i] == st->psched[i - 1]) {
    if (i >= SP2_MAX_ITER) return false;
    ++i;
    if (delta > 0.0 && bl < delta && gl < delta) {
      bl = 0.0; gl = 0.0;
      nmin = i + 1;
      delta = 0.0;
    }
    double a;
    if (gu >= bu) {
      a = __ddiv_rn(2.0, __dsub_rn(2.0, gl));
      gl = acc_fold(a, gl); gu = acc_fold(a, gu);
      bl = acc_lift(a, bl); bu = acc_lift(a, bu);
      st->psched[i] = 1;
    } else {
      a = __ddiv_rn(2.0, __dsub_rn(2.0, bl));
      gl = acc_lift(a, gl); gu = acc_lift(a, gu);
      bl = acc_fold(a, bl); bu = acc_fold(a, bu);
      st->psched[i] = 0;
    }
    st->alpha[i] = a;
  }
  st->n_min = nmin < 0 ? i + 1 : nmin;
  st->n_max = i;
  return true;
}

// Polynomial of square j (X_j from X_{j-1}) on the accelerated path:
// X_j = a X^2 + b X + c I, from p_j and alpha_j (Alg. 5); past n_max, p = 1 with alpha = 1.
__device__ __forceinline__ int acc_step(const DevState* st, int j, double& a, double& b, double& c) {
  const bool in = j >= 1 && j <= st->n_max;
  const int p = in ? st->psched[j] : 1;
  const double al = in ? st->alpha[j] : 1.0;
  if (p) {
    a = al * al;
    b = 2.0 * al * (1.0 - al);
    c = (1.0 - al) * (1.0 - al);
  } else {
    a = -al * al;
    b = 2.0 * al;
    c = 0.0;
  }
  return p;
}

// McW-ACC schedule (§3.1) for steps 1..max_iter: alpha_i = 3 / sqrt(12 beta^2 - 18 beta + 9)
// while the acceleration is on, beta_0 = (1 - xi / gamma) / 2, beta <- p(alpha (beta - 1/2) + 1/2);
// the acceleration is switched off for good once beta < 0.01 (n_min = the step after), as
// the Frobenius estimate may stop the accelerated scheme early.  McWeeny: alpha = 1, n_min = 1.
__device__ inline void mcw_schedule(DevState* st, double gamma) {
  double beta = __dmul_rn(0.5, __dsub_rn(1.0, __ddiv_rn(st->xi, gamma)));
  bool on = st->mcw == 2;
  int nmin = on ? -1 : 1;
  st->alpha[0] = 1.0;
  for (int i = 1; i <= st->max_iter; ++i) {
    if (on && beta < 0.01) {
      on = false;
      nmin = i + 1;
    }
    const double a = on ? __ddiv_rn(3.0, __dsqrt_rn(__dadd_rn(__dsub_rn(__dmul_rn(__dmul_rn(12.0, beta), beta),
                                                                       __dmul_rn(18.0, beta)), 9.0)))
                        : 1.0;
    const double bs = __dadd_rn(__dmul_rn(a, __dsub_rn(beta, 0.5)), 0.5);
    const double bs2 = __dmul_rn(bs, bs);
    beta = __dsub_rn(__dmul_rn(3.0, bs2), __dmul_rn(__dmul_rn(2.0, bs2), bs));
    st->alpha[i] = a;
  }
  st->n_min = nmin < 0 ? st->max_iter + 1 : nmin;
}

// Records square k = st->k + 1 (v_{k-1}, Tr[X_k], p_k) and applies the stop rules in
// the order the iteration meets them: the order test for X_{k-1} (Alg. 3, evaluated
// one square late because v_{k-1} needs X_{k-1}^2; on the accelerated path from n_min
// on, Alg. 5), the end of the schedule (accelerated path), the cap, then the trace guard
// for X_k, which compares Tr[X_k] with `tr_ref` = Tr[X_{k-1}] (accelerated path: only
// from n_min on, where the polynomials are the plain ones) and fires only when the order test
// on the last pair (v_{k-1}, v_{k-3}, without the alternation it needs) says the convergence
// order has fallen below qtilde.  Returns true if the run stops; single thread.
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
  if (st->mcw) {   // McWeeny: consecutive errors, C = 4, from n_min on; no trace rule
    if (!isfinite(v_prev)) {
      st->status = SP2_ERR_NONFINITE; st->out_mode = OUT_NAN; st->n_out = i;
    } else if (k == 1 && v_prev == 0.0) {
      st->reason = SP2_STOP_EXACT; st->n_out = 0; st->out_buf = 0;
    } else if (i >= max(1, st->n_min) && order_test_stops(st->v[i], st->v[i - 1], st->qtilde, kC2mw)) {
      st->reason = SP2_STOP_ORDER; st->n_out = i; st->out_buf = i & 1;
    } else if (i >= st->max_iter) {
      st->reason = SP2_STOP_CAP; st->n_out = i; st->out_buf = i & 1;
    } else {
      stop = false;
    }
    if (stop) st->done = 1;
    return stop;
  }
  if (!isfinite(v_prev) || !isfinite(tr_new)) {
    st->status = SP2_ERR_NONFINITE; st->out_mode = OUT_NAN; st->n_out = i;
  } else if (k == 1 && v_prev == 0.0) {
    st->reason = SP2_STOP_EXACT; st->n_out = 0; st->out_buf = 0;
  } else if (i >= (st->acc ? max(2, st->n_min) : 2) && st->p[i] != st->p[i - 1] &&
             order_test_stops(st->v[i], st->v[i - 2], st->qtilde)) {
    st->reason = SP2_STOP_ORDER; st->n_out = i; st->out_buf = i & 1;
  } else if (st->acc && i >= st->n_max) {
    st->reason = SP2_STOP_SCHEDULE; st->n_out = i; st->out_buf = i & 1;
  } else if (i >= st->max_iter) {
    st->reason = SP2_STOP_CAP; st->n_out = i; st->out_buf = i & 1;
  } else if (st->guard && (!st->acc || k >= st->n_min) &&
             ((pk == 1 && tr_new >= tr_ref) || (pk == 0 && tr_new <= tr_ref)) &&
             k >= 3 && order_test_stops(st->v[k - 1], st->v[k - 3], st->qtilde)) {
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

// Index of upper tile (I, J), I <= J, in a T x T grid whose upper tiles are numbered by rows.
__host__ __device__ __forceinline__ int64_t upper_index(int I, int J, int T) {
  return (int64_t)I * T - (int64_t)I * (I - 1) / 2 + (J - I);
}

// Mixed norm (§2): the spectral norm of the nb x nb matrix of block Frobenius norms, from
// `block_n2(I, J)` = ||block (I, J)||_F^2 for I <= J (the matrix is symmetric).  One CTA of
// NT threads: the matrix goes to `scr` (nb^2 doubles, then two vectors of nb), and its
// largest eigenvalue comes from kMixedIters power steps from the all-ones vector, the last
// one as a Rayleigh quotient; every sum in a fixed order.
constexpr int kMixedIters = 200;

template <int NT, class BlockN2>
__device__ double mixed_norm_cta(int nb, double* scr, double* sm, BlockN2 block_n2) {
  double* M = scr;
  double* x = scr + (int64_t)nb * nb;
  double* y = x + nb;
  const int tid = threadIdx.x;
  for (int64_t e = tid; e < (int64_t)nb * nb; e += NT) {
    const int I = (int)(e / nb), J = (int)(e % nb);
    M[e] = sqrt(fmax(block_n2(min(I, J), max(I, J)), 0.0));
  }
  for (int i = tid; i < nb; i += NT) x[i] = 1.0 / sqrt((double)nb);
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < kMixedIters; ++it) {
    for (int i = tid; i < nb; i += NT) {
      double acc = 0.0;
      for (int j = 0; j < nb; ++j) acc += M[(int64_t)i * nb + j] * x[j];
      y[i] = acc;
    }
    __syncthreads();
    double ss = 0.0, xy = 0.0;
    for (int i = tid; i < nb; i += NT) {
      ss += y[i] * y[i];
      xy += x[i] * y[i];
    }
    ss = block_sum<NT>(ss, sm);
    xy = block_sum<NT>(xy, sm);
    lam = xy;                                  // x has unit norm: Rayleigh quotient
    if (!(ss > 0.0)) { lam = 0.0; break; }
    const double inv = 1.0 / sqrt(ss);
    for (int i = tid; i < nb; i += NT) x[i] = y[i] * inv;
    __syncthreads();
  }
  return lam;
}

// Row/column of upper-triangular tile `t` in a T x T tile grid, tiles ordered by row.
__device__ __forceinline__ void upper_tile(int t, int T, int& I, int& J) {
  int i = 0, rem = t;
  while (rem >= T - i) { rem -= T - i; ++i; }
  I = i;
  J = i + rem;
}

}  // namespace sp2
