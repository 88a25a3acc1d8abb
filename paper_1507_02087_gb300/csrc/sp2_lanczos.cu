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
// warp, 32 points a round, in FP32: the tridiagonal of the scaled A is O(1) and the estimate only
// needs a few digits).  The Ritz values are inside the spectrum, so the estimate is a lower
// bound of e that approaches it from below; the stop test only needs its logarithm.
//
// Per estimate: start (1 CTA: coefficients, start vector, a power-of-two scale 2^-s with 2^s near
// v_{k-1} from the square's Frobenius partials), form (A 2^-s rounded to FP32 once: the ld x ld
// FP32 matrix, half the bytes of one FP64 iterate, is then read kLzSteps times, from L2 where it
// fits), kLzSteps x step (w = A q_j, one warp per row, FP32 products summed in FP32 per lane and
// FP64 across lanes; the last CTA to finish, found by an atomic ticket after a fence, runs the
// FP64 three-term update, so no CTA waits on another), eig (1 warp).  The FP32 rounding of A and
// of the products perturbs A by about 1e-7 of its norm, far below the Lanczos truncation error.
#include <math.h>

#include "sp2_common.cuh"
#include "sp2_kernels.h"
#include "sp2_tc.cuh"

namespace sp2 {
namespace {

constexpr int kLzSteps = 32;          // Lanczos steps per estimate
constexpr int kLzThreads = 1024;      // start: one CTA
constexpr int kLzMvThreads = 512;     // step: 16 warps, one row per warp at a time
constexpr int kLzMvBlocks = 152 * 2;  // step grid cap = number of partial sums
constexpr int kSturmRounds = 6;       // 33^6 > 2^30: below FP32 resolution of the interval

struct LzScratch {
  double scale;               // 2^-s applied before rounding A to FP32
  int32_t m;                  // completed steps
  int32_t live;               // 0 once the Krylov space is invariant (beta = 0) or not finite
  uint32_t ticket;            // CTAs of the current step that have finished their rows
  int32_t _pad;
  double alpha[kLzSteps];     // diagonal of the tridiagonal matrix
  double beta[kLzSteps + 1];  // beta[j] couples q_{j-1} and q_j; beta[0] = 0
  double part[kLzMvBlocks];   // per-CTA partials of q_j . A q_j
};
// followed by q_{j-1}, q_j, w (FP64, ld each), q_j in FP32 (ld) and A 2^-s in FP32 (ld x ld)

constexpr size_t kVecOff = (sizeof(LzScratch) + 255) / 256 * 256;

__device__ __forceinline__ double* lz_vec(LzScratch* lz, int ld, int which) {
  return reinterpret_cast<double*>(reinterpret_cast<char*>(lz) + kVecOff) + (size_t)which * ld;
}
__device__ __forceinline__ float* lz_q32(LzScratch* lz, int ld) {
  return reinterpret_cast<float*>(lz_vec(lz, ld, 3));
}
__device__ __forceinline__ float* lz_a32(LzScratch* lz, int ld) { return lz_q32(lz, ld) + ld; }

// Start vector entry i: SplitMix64 (Steele, Lea, Flood 2014) of the index, mapped to [-1, 1).
__device__ __forceinline__ double start_entry(int i) {
  unsigned long long z = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}

// X_{k-1}, the stored product Y and its coefficients (a, b, c) for the square just written.
__device__ __forceinline__ void lz_operands(const DevState* st, const double* buf0, const double* buf1,
                                            const double* S, const double*& Xa, const double*& Y, double& a,
                                            double& b, double& c) {
  const int k = st->k;
  Xa = (k & 1) ? buf1 : buf0;
  if (st->mcw) {                                 // S_s = (alpha X + c0 I)^2, c0 = (1 - alpha) / 2
    const double al = st->alpha[k + 1], c0 = 0.5 * (1.0 - al);
    a = al * al; b = 2.0 * al * c0; c = c0 * c0;
    Y = S;
    return;
  }
  if (st->acc) {
    acc_step(st, k + 1, a, b, c);
  } else {
    const int pk = st->tr[k] > (double)st->nocc ? 1 : 0;
    a = pk ? 1.0 : -1.0; b = pk ? 0.0 : 2.0; c = 0.0;
  }
  Y = (k & 1) ? buf0 : buf1;
}

// n x n operator stored with leading dimension ld; the square's partial records (v^2 first, `rec`
// doubles each), ntiles of them (or *ntiles_dev when given), set the scale.
__global__ void __launch_bounds__(kLzThreads)
lz_start_kernel(const DevState* st, const double* __restrict__ part, int ntiles, const int* ntiles_dev, int rec,
                LzScratch* lz, int N, int ld) {
  __shared__ double sm[32];
  if (st->done) return;
  const int cnt = ntiles_dev ? *ntiles_dev : ntiles;
  double v2 = 0.0;                               // v_{k-1}^2 from the square's partials
  for (int t = threadIdx.x; t < cnt; t += kLzThreads) v2 += part[rec * (int64_t)t];
  v2 = block_sum<kLzThreads>(v2, sm);
  double* qp = lz_vec(lz, ld, 0);
  double* q = lz_vec(lz, ld, 1);
  float* q32 = lz_q32(lz, ld);
  if (threadIdx.x == 0) {
    const double v = sqrt(v2);
    int e = (v > 0.0 && isfinite(v)) ? ilogb(v) : 0;
    e = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
    lz->scale = ldexp(1.0, -e);
    lz->m = 0;
    lz->live = 1;
    lz->ticket = 0;
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
  for (int i = threadIdx.x; i < ld; i += kLzThreads) {
    const double u = q[i] * inv;
    q[i] = u;
    q32[i] = (float)u;
  }
}

// A 2^-s = ((a + b) X_{k-1} - Y + c I) (2^-s / a), rounded to FP32, over the whole ld x ld
// buffer (the zero border stays zero; the identity term on the N true diagonal entries).
__global__ void lz_form_kernel(const DevState* st, const double* buf0, const double* buf1, const double* S,
                               LzScratch* lz) {
  if (st->done) return;
  const int N = st->N, ld = st->ld;
  const double* Xa;
  const double* Y;
  double a, b, c;
  lz_operands(st, buf0, buf1, S, Xa, Y, a, b, c);
  const double ab = a + b, f = lz->scale / a;
  const double2* __restrict__ X2 = reinterpret_cast<const double2*>(Xa);
  const double2* __restrict__ Y2 = reinterpret_cast<const double2*>(Y);
  float2* __restrict__ A2 = reinterpret_cast<float2*>(lz_a32(lz, ld));
  const int h = ld / 2;
  const int64_t total = (int64_t)ld * h;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / h), c2 = 2 * (int)(e % h);
    const double2 x = X2[e], y = Y2[e];
    double d0 = fma(ab, x.x, -y.x), d1 = fma(ab, x.y, -y.y);
    if (r < N && r == c2) d0 += c;
    if (r < N && r == c2 + 1) d1 += c;
    A2[e] = make_float2((float)(d0 * f), (float)(d1 * f));
  }
}

// The same operator on the tensor-core path (one problem): X_{k-1} and X_k are slots of the
// instance's piece arena, each element the exact FP32 value of its pieces, so
//     A 2^-s = ((a + b) X_{k-1} - X_k + c I) (2^-s / a), rounded to FP32,
// with the step's coefficients (SP2: (1, 0, 0) after X^2, (-1, 2, 0) after 2X - X^2).
__global__ void lz_form_tc_kernel(const DevState* st, const tc::Instance* inst, LzScratch* lz) {
  if (st->done) return;
  const tc::Instance& In = inst[0];
  const int N = st->N, ld = In.ld, k = st->k;
  double a, b, c;
  if (st->acc) {
    acc_step(st, k + 1, a, b, c);
  } else {
    const int pk = st->tr[k] > (double)st->nocc ? 1 : 0;
    a = pk ? 1.0 : -1.0; b = pk ? 0.0 : 2.0; c = 0.0;
  }
  const double ab = a + b, f = lz->scale / a;
  const int64_t plane = (int64_t)ld * ld;
  const __nv_bfloat16* xs = In.arena + (int64_t)tc::xslot(In.lowmem, In.hist0, k) * In.slot_elems;
  const __nv_bfloat16* ys = In.arena + (int64_t)tc::xslot(In.lowmem, In.hist0, k + 1) * In.slot_elems;
  float* A = lz_a32(lz, ld);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), col = (int)(e % ld);
    const double x = (double)tc::piece_load(In.fmt, xs, plane, e);
    const double y = (double)tc::piece_load(In.fmt, ys, plane, e);
    double d = fma(ab, x, -y);
    if (r < N && r == col) d += c;
    A[e] = (float)(d * f);
  }
}

// One Lanczos step: w = A q_j (one warp per row, FP32 products, 16-byte loads) and the CTA's
// share of q_j . w; the last CTA to finish its rows then computes alpha_j = q_j . w,
// r = w - alpha_j q_j - beta_j q_{j-1}, beta_{j+1} = ||r|| and q_{j+1} = r / beta_{j+1} in FP64.
__global__ void __launch_bounds__(kLzMvThreads)
lz_step_kernel(const DevState* st, LzScratch* lz, int j, int N, int ld) {
  __shared__ double sm[32];
  __shared__ int s_last;
  if (st->done || !lz->live) return;
  const float4* __restrict__ A = reinterpret_cast<const float4*>(lz_a32(lz, ld));
  const float4* __restrict__ q4 = reinterpret_cast<const float4*>(lz_q32(lz, ld));
  double* qp = lz_vec(lz, ld, 0);
  double* q = lz_vec(lz, ld, 1);
  double* w = lz_vec(lz, ld, 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = ld / 4;
  double pa = 0.0;
  for (int r = blockIdx.x * (kLzMvThreads / 32) + warp; r < N; r += gridDim.x * (kLzMvThreads / 32)) {
    const float4* ar = A + (int64_t)r * h;
    float s0 = 0.f, s1 = 0.f;
    int i = lane;
    for (; i + 32 < h; i += 64) {
      const float4 x0 = ar[i], v0 = q4[i], x1 = ar[i + 32], v1 = q4[i + 32];
      s0 = fmaf(x0.x, v0.x, s0); s0 = fmaf(x0.y, v0.y, s0); s0 = fmaf(x0.z, v0.z, s0); s0 = fmaf(x0.w, v0.w, s0);
      s1 = fmaf(x1.x, v1.x, s1); s1 = fmaf(x1.y, v1.y, s1); s1 = fmaf(x1.z, v1.z, s1); s1 = fmaf(x1.w, v1.w, s1);
    }
    if (i < h) {
      const float4 x0 = ar[i], v0 = q4[i];
      s0 = fmaf(x0.x, v0.x, s0); s0 = fmaf(x0.y, v0.y, s0); s0 = fmaf(x0.z, v0.z, s0); s0 = fmaf(x0.w, v0.w, s0);
    }
    double s = (double)s0 + (double)s1;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      w[r] = s;
      pa = fma(q[r], s, pa);
    }
  }
  if (lane == 0) __threadfence();                // this warp's w rows, before the ticket
  pa = block_sum<kLzMvThreads>(pa, sm);
  if (threadIdx.x == 0) {
    lz->part[blockIdx.x] = pa;
    __threadfence();
    s_last = atomicAdd(&lz->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // the last CTA: every row of w and every partial is written
  double a = 0.0;
  for (int t = threadIdx.x; t < (int)gridDim.x; t += kLzMvThreads) a += __ldcg(&lz->part[t]);
  a = block_sum<kLzMvThreads>(a, sm);
  const double bj = lz->beta[j];
  double ss = 0.0;
  for (int i = threadIdx.x; i < N; i += kLzMvThreads) {
    const double r = __ldcg(&w[i]) - a * q[i] - bj * qp[i];
    w[i] = r;
    ss = fma(r, r, ss);
  }
  ss = block_sum<kLzMvThreads>(ss, sm);
  const double b = sqrt(ss);
  const bool finite = isfinite(a) && isfinite(b);
  const bool more = j + 1 < kLzSteps && finite && b > 1e-300;
  if (threadIdx.x == 0) {
    lz->alpha[j] = finite ? a : __longlong_as_double(0x7ff8000000000000ll);
    lz->m = j + 1;
    if (j + 1 < kLzSteps) lz->beta[j + 1] = b;
    if (!more) lz->live = 0;
    lz->ticket = 0;
  }
  if (!more) return;
  const double ib = 1.0 / b;
  float* q32 = lz_q32(lz, ld);
  for (int i = threadIdx.x; i < N; i += kLzMvThreads) {
    const double u = w[i] * ib;
    qp[i] = q[i];
    q[i] = u;
    q32[i] = (float)u;
  }
}

// Number of eigenvalues of the m x m tridiagonal (alpha, beta) below x: the count of negative
// pivots of the LDL^T factorisation of T - x I (Sturm sequence), tiny pivots pushed to -pivmin.
__device__ __forceinline__ int sturm_count(const float* al, const float* be2, int m, float x) {
  constexpr float kPivMin = 1e-30f;
  float d = al[0] - x;
  if (fabsf(d) < kPivMin) d = -kPivMin;
  int cnt = d < 0.0f;
  for (int i = 1; i < m; ++i) {
    d = (al[i] - x) - be2[i] / d;
    if (fabsf(d) < kPivMin) d = -kPivMin;
    cnt += d < 0.0f;
  }
  return cnt;
}

__global__ void __launch_bounds__(32)
lz_eig_kernel(DevState* st, const LzScratch* lz) {
  __shared__ float al[kLzSteps], be2[kLzSteps];
  if (st->done) return;
  const int lane = threadIdx.x;
  const int m = lz->m;
  bool bad = m < 1;
  if (lane < m) {
    const double a = lz->alpha[lane], b = lane ? lz->beta[lane] : 0.0;
    bad = bad || !isfinite(a) || !isfinite(b) || fabs(a) > 1e30 || fabs(b) > 1e15;
    al[lane] = (float)a;
    be2[lane] = (float)(b * b);
  }
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  if (bad) {
    if (lane == 0) st->spec_e = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  float lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < m; ++i) {                  // Gershgorin interval of T
    const float rad = sqrtf(be2[i]) + (i + 1 < m ? sqrtf(be2[i + 1]) : 0.0f);
    lo = fminf(lo, al[i] - rad);
    hi = fmaxf(hi, al[i] + rad);
  }
  const float pad = 1e-30f + 0x1p-20f * fmaxf(fabsf(lo), fabsf(hi));
  lo -= pad;
  hi += pad;
  float lo1 = lo, hi1 = hi, lo2 = lo, hi2 = hi;  // brackets of the largest and the smallest
  for (int round = 0; round < kSturmRounds; ++round) {
    const float f = (float)(lane + 1) / 33.0f;
    const float x1 = lo1 + (hi1 - lo1) * f;
    const float x2 = lo2 + (hi2 - lo2) * f;
    // largest: the points with fewer than m eigenvalues below them form a prefix
    const int L = __popc(__ballot_sync(0xffffffffu, sturm_count(al, be2, m, x1) <= m - 1));
    // smallest: the points with no eigenvalue below them form a prefix
    const int S = __popc(__ballot_sync(0xffffffffu, sturm_count(al, be2, m, x2) == 0));
    const float xl1 = __shfl_sync(0xffffffffu, x1, L > 0 ? L - 1 : 0);
    const float xh1 = __shfl_sync(0xffffffffu, x1, L < 32 ? L : 31);
    const float xl2 = __shfl_sync(0xffffffffu, x2, S > 0 ? S - 1 : 0);
    const float xh2 = __shfl_sync(0xffffffffu, x2, S < 32 ? S : 31);
    if (L > 0) lo1 = xl1;
    if (L < 32) hi1 = xh1;
    if (S > 0) lo2 = xl2;
    if (S < 32) hi2 = xh2;
  }
  if (lane == 0) {
    const double top = 0.5 * ((double)lo1 + (double)hi1), bot = 0.5 * ((double)lo2 + (double)hi2);
    st->spec_e = fmax(fabs(top), fabs(bot)) / lz->scale;
  }
}

// Block-sparse path: the mixed norm's matrix of block norms M_IJ = ||(X - X^2)_IJ||_F (nb x nb,
// both triangles) from the square's upper-pair records (v^2 part counted twice off the
// diagonal), scaled and rounded to FP32 after a zero fill.
__global__ void lz_zero_kernel(const DevState* st, LzScratch* lz, int ld) {
  if (st->done) return;
  float4* A = reinterpret_cast<float4*>(lz_a32(lz, ld));
  const int64_t total = (int64_t)ld * ld / 4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    A[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void lz_form_pairs_kernel(const DevState* st, const int* __restrict__ row, const int* __restrict__ col,
                                     const int* nnz_p, const double* __restrict__ part, LzScratch* lz, int ld) {
  if (st->done) return;
  const int nnz = *nnz_p;
  const double sc = lz->scale;
  float* A = lz_a32(lz, ld);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
    const int I = row[q], J = col[q];
    const double v2 = part[2 * (int64_t)q] * (I == J ? 1.0 : 0.5);
    const float w = (float)(sqrt(v2) * sc);
    A[(int64_t)I * ld + J] = w;
    A[(int64_t)J * ld + I] = w;
  }
}

int step_blocks(int N) {
  const int b = (N + kLzMvThreads / 32 - 1) / (kLzMvThreads / 32);
  return b < kLzMvBlocks ? (b < 1 ? 1 : b) : kLzMvBlocks;
}

int form_blocks(int ld) {
  const int64_t b = ((int64_t)ld * (ld / 2) + 255) / 256;
  return (int)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

size_t lanczos_scratch_bytes(int ld) {
  return kVecOff + 3 * sizeof(double) * (size_t)ld + sizeof(float) * ((size_t)ld + (size_t)ld * ld);
}

cudaError_t add_lanczos_nodes(cudaGraph_t g, cudaGraphNode_t dep, DevState* st, const double* buf0,
                              const double* buf1, const double* S, const double* part, int ntiles, void* scratch,
                              int N, int ld, cudaGraphNode_t* last) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  const DevState* cst = st;
  cudaKernelNodeParams kp = {};
  cudaGraphNode_t prev = dep, node;
  const int* no_count = nullptr;
  int rec = 2;
  void* a0[] = {&cst, &part, &ntiles, &no_count, &rec, &lz, &N, &ld};
  kp.func = (void*)lz_start_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(kLzThreads);
  kp.kernelParams = a0;
  cudaError_t e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp);
  if (e != cudaSuccess) return e;
  prev = node;
  void* a1[] = {&cst, &buf0, &buf1, &S, &lz};
  kp.func = (void*)lz_form_kernel;
  kp.gridDim = dim3(form_blocks(ld));
  kp.blockDim = dim3(256);
  kp.kernelParams = a1;
  if ((e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp)) != cudaSuccess) return e;
  prev = node;
  for (int j = 0; j < kLzSteps; ++j) {
    int jj = j;
    void* a2[] = {&cst, &lz, &jj, &N, &ld};
    kp.func = (void*)lz_step_kernel;
    kp.gridDim = dim3(step_blocks(N));
    kp.blockDim = dim3(kLzMvThreads);
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

cudaError_t launch_lanczos(DevState* st, const double* buf0, const double* buf1, const double* S,
                           const double* part, int ntiles, void* scratch, int N, int ld, cudaStream_t s) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  lz_start_kernel<<<1, kLzThreads, 0, s>>>(st, part, ntiles, nullptr, 2, lz, N, ld);
  lz_form_kernel<<<form_blocks(ld), 256, 0, s>>>(st, buf0, buf1, S, lz);
  for (int j = 0; j < kLzSteps; ++j) lz_step_kernel<<<step_blocks(N), kLzMvThreads, 0, s>>>(st, lz, j, N, ld);
  lz_eig_kernel<<<1, 32, 0, s>>>(st, lz);
  return cudaGetLastError();
}

// Tensor-core path, one problem: the estimate for the square just written into `inst`'s arena;
// `part` holds its nparts records of 4 doubles (v^2 first).
cudaError_t add_lanczos_tc_nodes(cudaGraph_t g, cudaGraphNode_t dep, DevState* st, const tc::Instance* inst,
                                 const double* part, int nparts, void* scratch, int N, int ld,
                                 cudaGraphNode_t* last) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  const DevState* cst = st;
  cudaKernelNodeParams kp = {};
  cudaGraphNode_t prev = dep, node;
  const int* no_count = nullptr;
  int rec = 4;
  void* a0[] = {&cst, &part, &nparts, &no_count, &rec, &lz, &N, &ld};
  kp.func = (void*)lz_start_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(kLzThreads);
  kp.kernelParams = a0;
  cudaError_t e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp);
  if (e != cudaSuccess) return e;
  prev = node;
  void* a1[] = {&cst, &inst, &lz};
  kp.func = (void*)lz_form_tc_kernel;
  kp.gridDim = dim3(form_blocks(ld));
  kp.blockDim = dim3(256);
  kp.kernelParams = a1;
  if ((e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp)) != cudaSuccess) return e;
  prev = node;
  for (int j = 0; j < kLzSteps; ++j) {
    int jj = j;
    void* a2[] = {&cst, &lz, &jj, &N, &ld};
    kp.func = (void*)lz_step_kernel;
    kp.gridDim = dim3(step_blocks(N));
    kp.blockDim = dim3(kLzMvThreads);
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

cudaError_t launch_lanczos_tc(DevState* st, const tc::Instance* inst, const double* part, int nparts, void* scratch,
                              int N, int ld, cudaStream_t s) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  lz_start_kernel<<<1, kLzThreads, 0, s>>>(st, part, nparts, nullptr, 4, lz, N, ld);
  lz_form_tc_kernel<<<form_blocks(ld), 256, 0, s>>>(st, inst, lz);
  for (int j = 0; j < kLzSteps; ++j) lz_step_kernel<<<step_blocks(N), kLzMvThreads, 0, s>>>(st, lz, j, N, ld);
  lz_eig_kernel<<<1, 32, 0, s>>>(st, lz);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_pairs(DevState* st, const int* row, const int* col, const int* nnz_p, const double* part,
                                 void* scratch, int nb, int ld, cudaStream_t s) {
  LzScratch* lz = static_cast<LzScratch*>(scratch);
  lz_start_kernel<<<1, kLzThreads, 0, s>>>(st, part, 0, nnz_p, 2, lz, nb, ld);
  lz_zero_kernel<<<form_blocks(ld), 256, 0, s>>>(st, lz, ld);
  lz_form_pairs_kernel<<<form_blocks(ld), 256, 0, s>>>(st, row, col, nnz_p, part, lz, ld);
  for (int j = 0; j < kLzSteps; ++j) lz_step_kernel<<<step_blocks(nb), kLzMvThreads, 0, s>>>(st, lz, j, nb, ld);
  lz_eig_kernel<<<1, 32, 0, s>>>(st, lz);
  return cudaGetLastError();
}

}  // namespace sp2
