// Spectral-norm stop of the FP64 path (§2: the stop is defined on e_i = ||X_i - X_i^2||_2;
// the Frobenius v_i and the mixed norm m_i are its upper bounds).
//
// After square k the buffers hold X_{k-1} and the stored product Y = a X_{k-1}^2 + b X_{k-1} + c I
// of this step: X_k itself (SP2: (a, b, c) = (1, 0, 0) or (-1, 2, 0); SP2-ACC: the scheduled
// coefficients) or the McWeeny step's shifted square S_s (alpha^2, 2 alpha c, c^2).  So
//     A = X_{k-1} - X_{k-1}^2 = ((a + b) X_{k-1} - Y + c I) / a
// is available without forming X^2, and e_{k-1} = ||A||_2 = max |lambda(A)| is estimated by
// kLzSteps steps of the symmetric Lanczos recurrence (three-term, no reorthogonalisation: lost
// orthogonality only repeats converged extreme Ritz values) from a fixed start vector.  The
// extreme eigenvalues of the tridiagonal matrix come from multisection with Sturm counts (one
// warp, 32 points a round).  The Ritz values are inside the spectrum, so the estimate is a lower
// bound of e that approaches it from below; the stop test only needs its logarithm.
//
// Kernels per estimate: start (1 CTA), kLzSteps x {matvec (one warp per row over the grid),
// update (1 CTA)}, eig (1 warp): 2 kLzSteps + 2 launches, added to the loop graph between the
// square and the stop test.  Traffic: two ld x ld FP64 matrices per matvec.
#include <math.h>

#include "sp2_common.cuh"
#include "sp2_kernels.h"

namespace sp2 {
namespace {

constexpr int kLzSteps = 32;          // Lanczos steps per estimate
constexpr int kLzThreads = 1024;      // start / update: one CTA
constexpr int kLzMvThreads = 256;     // matvec: 8 warps, one row per warp at a time
constexpr int kLzMvBlocks = 152 * 4;  // matvec grid cap = number of partial sums
constexpr int kSturmRounds = 14;      // 33^14 > 2^70: far below FP64 resolution

struct LzScratch {
  const double* Xa;           // X_{k-1}
  const double* Y;            // the stored product of this step
  double ab;                  // a + b
  double c;                   // identity coefficient of Y
  double inv_a;               // 1 / a
  int32_t m;                  // completed steps
  int32_t live;               // 0 once the Krylov space is invariant (beta = 0) or not finite
  double alpha[kLzSteps];     // diagonal of the tridiagonal matrix
  double beta[kLzSteps + 1];  // beta[j] couples q_{j-1} and q_j; beta[0] = 0
  double part[kLzMvBlocks];   // per-CTA partials of q_j . A q_j
};

constexpr size_t kVecOff = (sizeof(LzScratch) + 255) / 256 * 256;

__device__ __forceinline__ double* lz_vec(LzScratch* lz, int ld, int which) {
  return reinterpret_cast<double*>(reinterpret_cast<char*>(lz) + kVecOff) + (size_t)which * ld;
}

// Start vector entry i: SplitMix64 (Steele, Lea, Flood 2014) of the index, mapped to [-1, 1).
__device__ __forceinline__ double start_entry(int i) {
  unsigned long long z = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}

__global__ void __launch_bounds__(kLzThreads)
lz_start_kernel(const DevState* st, const double* buf0, const double* buf1, const double* S, LzScratch* lz) {
  __shared__ double sm[32];
  if (st->done) return;
  const int N = st->N, ld = st->ld, k = st->k;    // the square k + 1 has just been written
  double* qp = lz_vec(lz, ld, 0);
  double* q = lz_vec(lz, ld, 1);
  if (threadIdx.x == 0) {
    const double* Xprev = (k & 1) ? buf1 : buf0;
    double a, b, c;
    const double* Y;
    if (st->mcw) {                               // S_s = (alpha X + c0 I)^2, c0 = (1 - alpha) / 2
      const double al = st->alpha[k + 1], c0 = 0.5 * (1.0 - al);
      a = al * al; b = 2.0 * al * c0; c = c0 * c0;
      Y = S;
    } else {
      if (st->acc) {
        acc_step(st, k + 1, a, b, c);
      } else {
        const int pk = st->tr[k] > (double)st->nocc ? 1 : 0;
        a = pk ? 1.0 : -1.0; b = pk ? 0.0 : 2.0; c = 0.0;
      }
      Y = (k & 1) ? buf0 : buf1;
    }
    lz->Xa = Xprev;
    lz->Y = Y;
    lz->ab = a + b;
    lz->c = c;
    lz->inv_a = 1.0 / a;
    lz->m = 0;
    lz->live = 1;
    lz->beta[0] = 0.0;
  }
  double ss = 0.0;
  for (int i = threadIdx.x; i < ld; i += kLzThreads) {
    const double u = i < N ? start_entry(i) : 0.0;
    q[i] = u;
    qp[i] = 0.0;
    ss = fma(u, u, ss);
  }
  ss = block_sum<kLzThreads>(ss, sm);
  const double inv = 1.0 / sqrt(ss);
  for (int i = threadIdx.x; i < N; i += kLzThreads) q[i] *= inv;
}

// w = A q_j, one warp per row (16-byte loads along the row), and the CTA's share of q_j . w.
__global__ void __launch_bounds__(kLzMvThreads)
lz_matvec_kernel(const DevState* st, LzScratch* lz) {
  __shared__ double sm[32];
  if (st->done || !lz->live) return;
  const int N = st->N, ld = st->ld;
  const double2* __restrict__ X = reinterpret_cast<const double2*>(lz->Xa);
  const double2* __restrict__ Y = reinterpret_cast<const double2*>(lz->Y);
  const double ab = lz->ab, c = lz->c, inv_a = lz->inv_a;
  const double* __restrict__ q = lz_vec(lz, ld, 1);
  const double2* __restrict__ q2 = reinterpret_cast<const double2*>(q);
  double* w = lz_vec(lz, ld, 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = ld / 2;
  double pa = 0.0;
  for (int r = blockIdx.x * (kLzMvThreads / 32) + warp; r < N; r += gridDim.x * (kLzMvThreads / 32)) {
    const double2* xr = X + (int64_t)r * h;
    const double2* yr = Y + (int64_t)r * h;
    double s = 0.0;
    for (int j = lane; j < h; j += 32) {
      const double2 x = xr[j], y = yr[j], v = q2[j];
      s = fma(fma(ab, x.x, -y.x), v.x, s);
      s = fma(fma(ab, x.y, -y.y), v.y, s);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double wr = fma(c, q[r], s) * inv_a;
    if (lane == 0) {
      w[r] = wr;
      pa = fma(q[r], wr, pa);
    }
  }
  pa = block_sum<kLzMvThreads>(pa, sm);
  if (threadIdx.x == 0) lz->part[blockIdx.x] = pa;
}

// alpha_j = q_j . w; r = w - alpha_j q_j - beta_j q_{j-1}; beta_{j+1} = ||r||; q_{j+1} = r / beta_{j+1}.
__global__ void __launch_bounds__(kLzThreads)
lz_update_kernel(const DevState* st, LzScratch* lz, int j, int nblk) {
  __shared__ double sm[32];
  if (st->done || !lz->live) return;
  const int N = st->N, ld = st->ld;
  double* qp = lz_vec(lz, ld, 0);
  double* q = lz_vec(lz, ld, 1);
  double* w = lz_vec(lz, ld, 2);
  double a = 0.0;
  for (int t = threadIdx.x; t < nblk; t += kLzThreads) a += lz->part[t];
  a = block_sum<kLzThreads>(a, sm);
  const double bj = lz->beta[j];
  double ss = 0.0;
  for (int i = threadIdx.x; i < N; i += kLzThreads) {
    const double r = w[i] - a * q[i] - bj * qp[i];
    w[i] = r;
    ss = fma(r, r, ss);
  }
  ss = block_sum<kLzThreads>(ss, sm);
  const double b = sqrt(ss);
  const bool finite = isfinite(a) && isfinite(b);
  if (threadIdx.x == 0) {
    lz->alpha[j] = finite ? a : __longlong_as_double(0x7ff8000000000000ll);
    lz->m = j + 1;
    if (j + 1 < kLzSteps) lz->beta[j + 1] = b;
    if (!finite || !(b > 1e-300)) lz->live = 0;
  }
  if (j + 1 == kLzSteps || !finite || !(b > 1e-300)) return;
  const double ib = 1.0 / b;
  for (int i = threadIdx.x; i < N; i += kLzThreads) {
    qp[i] = q[i];
    q[i] = w[i] * ib;
  }
}

// Number of eigenvalues of the m x m tridiagonal (alpha, beta) below x: the count of negative
// pivots of the LDL^T factorisation of T - x I (Sturm sequence), tiny pivots pushed to -pivmin.
__device__ __forceinline__ int sturm_count(const double* al, const double* be, int m, double x) {
  constexpr double kPivMin = 1e-300;
  double d = al[0] - x;
  if (fabs(d) < kPivMin) d = -kPivMin;
  int cnt = d < 0.0;
  for (int i = 1; i < m; ++i) {
    d = (al[i] - x) - be[i] * be[i] / d;
    if (fabs(d) < kPivMin) d = -kPivMin;
    cnt += d < 0.0;
  }
  return cnt;
}

__global__ void __launch_bounds__(32)
lz_eig_kernel(DevState* st, const LzScratch* lz) {
  __shared__ double al[kLzSteps], be[kLzSteps];
  if (st->done) return;
  const int lane = threadIdx.x;
  const int m = lz->m;
  if (lane < m) {
    al[lane] = lz->alpha[lane];
    be[lane] = lane ? lz->beta[lane] : 0.0;
  }
  __syncwarp();
  double lo = INFINITY, hi = -INFINITY;
  bool bad = m < 1;
  for (int i = 0; i < m; ++i) {                  // Gershgorin interval of T
    const double rad = fabs(be[i]) + (i + 1 < m ? fabs(be[i + 1]) : 0.0);
    lo = fmin(lo, al[i] - rad);
    hi = fmax(hi, al[i] + rad);
    bad = bad || !isfinite(al[i]) || !isfinite(be[i]);
  }
  if (bad) {
    if (lane == 0) st->spec_e = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const double pad = 1e-300 + 0x1p-50 * fmax(fabs(lo), fabs(hi));
  lo -= pad;
  hi += pad;
  double lo1 = lo, hi1 = hi, lo2 = lo, hi2 = hi;  // brackets of the largest and the smallest
  for (int round = 0; round < kSturmRounds; ++round) {
    const double f = (double)(lane + 1) / 33.0;
    const double x1 = lo1 + (hi1 - lo1) * f;
    const double x2 = lo2 + (hi2 - lo2) * f;
    // largest: the points with fewer than m eigenvalues below them form a prefix
    const int L = __popc(__ballot_sync(0xffffffffu, sturm_count(al, be, m, x1) <= m - 1));
    // smallest: the points with no eigenvalue below them form a prefix
    const int S = __popc(__ballot_sync(0xffffffffu, sturm_count(al, be, m, x2) == 0));
    const double xl1 = __shfl_sync(0xffffffffu, x1, L > 0 ? L - 1 : 0);
    const double xh1 = __shfl_sync(0xffffffffu, x1, L < 32 ? L : 31);
    const double xl2 = __shfl_sync(0xffffffffu, x2, S > 0 ? S - 1 : 0);
    const double xh2 = __shfl_sync(0xffffffffu, x2, S < 32 ? S : 31);
    if (L > 0) lo1 = xl1;
    if (L < 32) hi1 = xh1;
    if (S > 0) lo2 = xl2;
    if (S < 32) hi2 = xh2;
  }
  if (lane == 0) st->spec_e = fmax(fabs(0.5 * (lo1 + hi1)), fabs(0.5 * (lo2 + hi2)));
}

int matvec_blocks(int N) {
  const int b = (N + kLzMvThreads / 32 - 1) / (kLzMvThreads / 32);
  return b < kLzMvBlocks ? (b < 1 ? 1 : b) : kLzMvBlocks;
}

}  // namespace

size_t lanczos_scratch_bytes(int ld) { return kVecOff + 3 * sizeof(double) * (size_t)ld; }

cudaError_t add_lanczos_nodes(cudaGraph_t g, cudaGraphNode_t dep, DevState* st, const double* buf0,
                              const double* buf1, const double* S, void* scratch, int N, cudaGraphNode_t* last) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  const DevState* cst = st;
  cudaKernelNodeParams kp = {};
  cudaGraphNode_t prev = dep, node;
  void* a0[] = {&cst, &buf0, &buf1, &S, &lz};
  kp.func = (void*)lz_start_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(kLzThreads);
  kp.kernelParams = a0;
  cudaError_t e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp);
  if (e != cudaSuccess) return e;
  prev = node;
  int nblk = matvec_blocks(N);
  for (int j = 0; j < kLzSteps; ++j) {
    void* a1[] = {&cst, &lz};
    kp.func = (void*)lz_matvec_kernel;
    kp.gridDim = dim3(nblk);
    kp.blockDim = dim3(kLzMvThreads);
    kp.kernelParams = a1;
    if ((e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp)) != cudaSuccess) return e;
    prev = node;
    int jj = j;
    void* a2[] = {&cst, &lz, &jj, &nblk};
    kp.func = (void*)lz_update_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kLzThreads);
    kp.kernelParams = a2;
    if ((e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp)) != cudaSuccess) return e;
    prev = node;
  }
  const LzScratch* clz = lz;
  void* a3[] = {&st, &clz};
  kp.func = (void*)lz_eig_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(32);
  kp.kernelParams = a3;
  e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp);
  *last = node;
  return e;
}

cudaError_t launch_lanczos(DevState* st, const double* buf0, const double* buf1, const double* S, void* scratch,
                           int N, cudaStream_t s) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  const int nblk = matvec_blocks(N);
  lz_start_kernel<<<1, kLzThreads, 0, s>>>(st, buf0, buf1, S, lz);
  for (int j = 0; j < kLzSteps; ++j) {
    lz_matvec_kernel<<<nblk, kLzMvThreads, 0, s>>>(st, lz);
    lz_update_kernel<<<1, kLzThreads, 0, s>>>(st, lz, j, nblk);
  }
  lz_eig_kernel<<<1, 32, 0, s>>>(st, lz);
  return cudaGetLastError();
}

}  // namespace sp2
