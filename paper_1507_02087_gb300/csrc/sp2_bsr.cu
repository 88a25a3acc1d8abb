// Block-sparse SP2 with Frobenius block truncation (the E_i of Alg. 1).
//
// X~_i is a symmetric block-sparse matrix with 32 x 32 FP32 blocks, stored with both
// triangles as BSR (row_ptr, sorted col_idx, values) plus one bitmap row per block
// row (bit J of row I set iff block (I, J) is stored) and a popcount rank table, so
// "where is block (I, J)" is an O(1) integer computation.  One loop round (square k):
//
//   1. symbolic square: the upper block pattern of S = X~_{k-1}^2 (row I of S is the
//      OR of the bitmap rows K in row I of X~_{k-1}), listed as (I, J >= I) pairs;
//   2. numeric square + SP2 epilogue for each pair: S_IJ = sum_K X_IK X_JK^T over
//      the K both rows hold (increasing K), X_IJ <- S_IJ or 2 X_IJ - S_IJ (Alg. 3),
//      the FP64 partials of ||X~_{k-1} - S||_F^2 and Tr[X_k], and ||X_IJ||_F^2 of the
//      new block in a fixed order (row sums left to right, rows top to bottom);
//   3. stop test on the device (Alg. 3, with the trace guard) on v_{k-1}, or on the mixed
//      norm m_{k-1} with the 32 x 32 blocks (§2; the spectral norm of the matrix of block
//      norms of X~ - X~^2, by the Lanczos kernels);
//   4. truncation: off-diagonal blocks with ||X_IJ||_F^2 < tau^2 are dropped (rule 0),
//      or the longest prefix in (||X_IJ||_F^2, I, J) order whose doubled norms add up to
//      at most tau^2 (rule 1, error-controlled: ||E||_F <= tau, sums in exact integer
//      units), or the longest prefix in that order in which every block row's sum of
//      dropped block norms stays within tau (rule 2, mixed norm: ||E||_M <= tau, §6);
//      the kept bitmap is set for (I, J) and (J, I), and X~_k is written as BSR (each
//      kept upper block and its transpose at the rank of its column in its row).
//
// All index work is integer and fixed-order, so the pattern of every iterate is
// reproducible bit for bit (and equals the host's, given the same stored blocks).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sp2.h"
#include "sp2_common.cuh"
#include "sp2_kernels.h"

#include "sp2_bsr.cuh"
#include "sp2_tc.cuh"

namespace sp2 {
namespace bsr {

constexpr int NT = 256;            // threads of the block kernels
constexpr int MAX_NB = 2048;       // block rows (N <= 65536)

// ---- generic bitmap / pattern kernels ----------------------------------------------------
__global__ void clear_words_kernel(uint32_t* bits, int64_t n, const DevState* st) {
  if (st && !st->iter_active) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bits[i] = 0u;
}

// per row: number of set bits (J >= I only with `upper`)
__global__ void row_counts_kernel(const uint32_t* bits, int nb, int W, int upper, int* counts, const DevState* st) {
  if (st && !st->iter_active) return;
  const int I = blockIdx.x;
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int c = 0;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    uint32_t x = bits[(int64_t)I * W + w];
    if (upper) {
      const int lo = w * 32;
      if (lo + 31 < I) x = 0u;
      else if (lo < I) x &= ~((1u << (I - lo)) - 1u);
    }
    c += popc(x);
  }
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) counts[I] = s;
}

// exclusive scan of counts[0..nb) into ptr[0..nb], total in *total (one block)
__global__ void scan_kernel(const int* counts, int nb, int* ptr, int* total, const DevState* st) {
  if (st && !st->iter_active) return;
  __shared__ int sm[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? counts[i] : 0;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
      __syncthreads();
      sm[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) ptr[i] = carry + sm[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sm[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ptr[nb] = carry;
    if (total) *total = carry;
  }
}

// rank[I][w] = set bits of row I in words < w (one block per row, W <= 64)
__global__ void rank_kernel(const uint32_t* bits, int nb, int W, int* rank, const DevState* st) {
  if (st && !st->iter_active) return;
  const int I = blockIdx.x;
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < W; ++w) {
      rank[(int64_t)I * W + w] = acc;
      acc += popc(bits[(int64_t)I * W + w]);
    }
  }
}

// list the set bits of every row (J >= I with `upper`) as pairs, in increasing J
__global__ void fill_pairs_kernel(const uint32_t* bits, int nb, int W, int upper, Pairs P, const DevState* st) {
  if (st && !st->iter_active) return;
  const int I = blockIdx.x;
  if (threadIdx.x == 0) {
    int pos = P.ptr[I];
    for (int w = 0; w < W; ++w) {
      uint32_t x = bits[(int64_t)I * W + w];
      const int lo = w * 32;
      if (upper) {
        if (lo + 31 < I) continue;
        if (lo < I) x &= ~((1u << (I - lo)) - 1u);
      }
      while (x) {
        const int b = __ffs(x) - 1;
        x &= x - 1u;
        P.col[pos] = lo + b;
        P.row[pos] = I;
        ++pos;
      }
    }
  }
}

__global__ void csr_to_bits_kernel(const int* rp, const int* ci, int nb, int W, uint32_t* bits) {
  const int I = blockIdx.x;
  for (int e = rp[I] + threadIdx.x; e < rp[I + 1]; e += blockDim.x) {
    const int J = ci[e];
    atomicOr(&bits[(int64_t)I * W + (J >> 5)], 1u << (J & 31));
  }
}

// ---- initialisation: Gershgorin bounds of the BSR input, X_0 on F's upper pattern --------
// One block per block row; thread r < 32 sums |F| over row r of the block row.
__global__ void bsr_gersh_kernel(const int* rp, const int* ci, const double* vals, int nb, double* lo_out,
                                 double* hi_out, int* bad_out) {
  const int I = blockIdx.x;
  __shared__ double slo[B], shi[B];
  __shared__ int sbad[B];
  const int r = threadIdx.x;
  double s = 0.0, d = 0.0;
  int bad = 0;
  if (r < B) {
    for (int e = rp[I]; e < rp[I + 1]; ++e) {
      const int J = ci[e];
      const double* blk = vals + (int64_t)e * BE + r * B;
      for (int c = 0; c < B; ++c) {
        const double a = blk[c];
        if (!isfinite(a)) bad = 1;
        if (J == I && c == r) d = a;
        else s += fabs(a);
      }
    }
    slo[r] = d - s;
    shi[r] = d + s;
    sbad[r] = bad;
  }
  __syncthreads();
  if (r == 0) {
    double lo = slo[0], hi = shi[0];
    int b = sbad[0];
    for (int k = 1; k < B; ++k) { lo = fmin(lo, slo[k]); hi = fmax(hi, shi[k]); b |= sbad[k]; }
    lo_out[I] = lo; hi_out[I] = hi; bad_out[I] = b;
  }
}

constexpr int kIT = 1024;

__global__ void __launch_bounds__(kIT)
bsr_init_kernel(DevState* st, const int* rp, const int* ci, const double* vals, int nb, const double* lo_in,
                const double* hi_in, const int* bad_in) {
  __shared__ double sm[32];
  __shared__ double s_lmin, s_lmax;
  __shared__ int s_bad;
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int I = 0; I < nb; ++I) { lo = fmin(lo, lo_in[I]); hi = fmax(hi, hi_in[I]); bad |= bad_in[I]; }
    if (!isfinite(lo) || !isfinite(hi)) bad = 1;
    if (st->ubounds) {                           // the caller's outer bounds (§3: any serve)
      lo = st->ub_lo;
      hi = st->ub_hi;
    }
    s_lmin = lo; s_lmax = hi; s_bad = bad;
  }
  __syncthreads();
  const double lmin = s_lmin, lmax = s_lmax, w = lmax - lmin;
  // Tr[X_0] over the stored (FP32) diagonal; the diagonal block of row I is found by search
  double t = 0.0;
  for (int i = threadIdx.x; i < nb * B; i += kIT) {
    const int I = i / B, r = i % B;
    double f = 0.0;
    for (int e = rp[I]; e < rp[I + 1]; ++e)
      if (ci[e] == I) { f = vals[(int64_t)e * BE + r * B + r]; break; }
    t += (double)(float)((lmax - f) / w);
  }
  t = block_sum<kIT>(t, sm);
  if (threadIdx.x == 0) {
    const int N = st->N, nocc = st->nocc;
    st->lmin = lmin; st->lmax = lmax;
    st->dk = 0; st->k = 0; st->done = 0; st->n_out = 0; st->reason = SP2_STOP_EXACT;
    st->status = SP2_OK; st->out_buf = 0; st->out_mode = OUT_COPY; st->hist_len = 0;
    st->tr[0] = 0.0; st->p[0] = 0; st->iter_active = 1;
    st->bprod = 0ull; st->sblocks = 0ull; st->uprod = 0ull;
    if (s_bad) { st->status = SP2_ERR_NONFINITE; st->done = 1; st->out_mode = OUT_NAN; }
    else if (nocc == 0) { st->done = 1; st->out_mode = OUT_ZERO; }
    else if (nocc == N) { st->done = 1; st->out_mode = OUT_IDENTITY; }
    else if (!(lmax > lmin)) { st->status = SP2_ERR_NO_GAP; st->done = 1; st->out_mode = OUT_NAN; }
    else {
      st->tr[0] = t;
      if (st->acc && !acc_schedule(st)) {        // SP2-ACC: Alg. 4 from the bounds just found
        st->status = SP2_ERR_INVALID_ARG; st->done = 1; st->out_mode = OUT_NAN;
      }
    }
  }
}

// ||blk||_F^2 in the fixed order (rows left to right, then rows top to bottom) by warp 0;
// blk in shared memory with row stride B + 1.
__device__ __forceinline__ double block_norm2_fixed(const float* blk) {
  const int lane = threadIdx.x & 31;
  double rs = 0.0;
  for (int c = 0; c < B; ++c) {
    const double x = (double)blk[lane * (B + 1) + c];
    rs = __dadd_rn(rs, __dmul_rn(x, x));
  }
  double tot = 0.0;
  for (int r = 0; r < B; ++r) tot = __dadd_rn(tot, __shfl_sync(0xffffffffu, rs, r));
  return tot;
}

// X_0 = (lmax I - F)/(lmax - lmin) on the upper pairs of F's pattern, with the
// truncation decision (Alg. 1: X~_0 = X_0 + E_0).
__global__ void __launch_bounds__(NT)
bsr_scale_pairs_kernel(const DevState* st, const int* frp, const uint32_t* fbits, const int* frank,
                       const double* fvals, int W, Pairs P, float* svals, uint8_t* skeep, double* sn2,
                       double tau2) {
  __shared__ float blk[B * (B + 1)];
  if (st->done) return;
  const int nnz = *P.nnz;
  const double lmax = st->lmax, w = st->lmax - st->lmin;
  for (int q = blockIdx.x; q < nnz; q += gridDim.x) {
    const int I = P.row[q], J = P.col[q];
    const uint32_t word = fbits[(int64_t)I * W + (J >> 5)];
    const int pos = frp[I] + frank[(int64_t)I * W + (J >> 5)] + popc(word & ((1u << (J & 31)) - 1u));
    for (int e = threadIdx.x; e < BE; e += NT) {
      const int r = e / B, c = e % B;
      const double f = fvals[(int64_t)pos * BE + e];
      const float x = (float)((((I == J && r == c) ? lmax : 0.0) - f) / w);
      blk[r * (B + 1) + c] = x;
      svals[(int64_t)q * BE + e] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const double n2 = block_norm2_fixed(blk);
      if (threadIdx.x == 0) {
        skeep[q] = (I == J || n2 >= tau2) ? 1 : 0;
        sn2[q] = n2;
      }
    }
    __syncthreads();
  }
}

// ---- symbolic square -----------------------------------------------------------------------
// S row I (upper part) = OR over K in row I of X of bitmap row K.
__global__ void bsr_sym_kernel(DevState* st, Mat X, int nb, int W, uint32_t* sbits) {
  const int I = blockIdx.x;
  if (I == 0 && threadIdx.x == 0) st->iter_active = st->done ? 0 : 1;
  if (st->done) return;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    uint32_t acc = 0u;
    for (int e = X.rp[I]; e < X.rp[I + 1]; ++e) acc |= X.bits[(int64_t)X.ci[e] * W + w];
    const int lo = w * 32;
    if (lo + 31 < I) acc = 0u;
    else if (lo < I) acc &= ~((1u << (I - lo)) - 1u);
    sbits[(int64_t)I * W + w] = acc;
  }
}

// ---- numeric square + SP2 epilogue + truncation decision -----------------------------------
// One warp per upper pair (I, J) of the square; a CTA holds NUM_WARPS warps.  The products
// S_IJ = sum_K X_IK X_JK^T run over the K of row I (increasing) that row J also holds.  Both
// triangles are stored and X_KI is the exact transpose of X_IK, so the operands come from
// block row K as X_KI and X_KJ: read row-major they give X_IK[r][k] = X_KI[k][r] and
// X_JK[c][k] = X_KJ[k][c], k-major, without a transpose.  Each product is staged as two
// halves (k rows 0..15, then 16..31 of both blocks) through a per-warp double buffer with
// cp.async while the previous half is computed (8 KB per warp, so six 4-warp CTAs fit an SM);
// each lane accumulates a 4 x 8 tile (rows 4 rg .. 4 rg + 3, columns 8 cg .. 8 cg + 7,
// lane = 4 rg + cg) with one fused multiply-add per term in increasing K, then k.
constexpr int NUM_WARPS = 4;
constexpr int NUM_THREADS = 32 * NUM_WARPS;
constexpr int HK = B / 2;                         // k rows per staged half
constexpr int HBE = HK * B;                       // floats of one half block
constexpr int WARP_FLOATS = 2 * 2 * HBE;          // two stages of (X_KI, X_KJ) halves
constexpr int NUM_SMEM = NUM_WARPS * WARP_FLOATS * 4;
static_assert(WARP_FLOATS >= B * (B + 1), "the epilogue stages a block with row stride B + 1");

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// half h (k rows 16 h .. 16 h + 15) of blocks pa (X_KI) and pb (X_KJ) into stage `stg`
__device__ __forceinline__ void issue_half(float* wbuf, int stg, const float* vals, int pa, int pb, int h,
                                           int lane) {
  float* dA = wbuf + stg * 2 * HBE;
  float* dB = dA + HBE;
  const float* sA = vals + (int64_t)pa * BE + h * HBE;
  const float* sB = vals + (int64_t)pb * BE + h * HBE;
  #pragma unroll
  for (int i = 0; i < HBE / 128; ++i) {
    const int off = (i * 32 + lane) * 4;
    cp_async16(dA + off, sA + off);
    cp_async16(dB + off, sB + off);
  }
  cp_async_commit();
}

// Packed FP32 pairs: fma.rn.f32x2 rounds each lane once, exactly as fmaf, and halves the FMA
// instruction count of the issue-bound inner loop.  acc[i][jp] holds columns (2 jp, 2 jp + 1)
// of row i (low word first), so the B pairs come straight from the 16-byte shared loads and
// each A value is broadcast into a pair once per k.
__device__ __forceinline__ unsigned long long pair_bcast(float x) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void ffma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

__device__ __forceinline__ void product_tile(const float* wbuf, int stg, int rg, int cg,
                                             unsigned long long (&acc)[4][4]) {
  const float* At = wbuf + stg * 2 * HBE;
  const float* Bt = At + HBE;
  #pragma unroll 8
  for (int k = 0; k < HK; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(At + k * B + 4 * rg);
    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(Bt + k * B + 8 * cg);
    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(Bt + k * B + 8 * cg + 4);
    const unsigned long long av[4] = {pair_bcast(a.x), pair_bcast(a.y), pair_bcast(a.z), pair_bcast(a.w)};
    const unsigned long long bv[4] = {b0.x, b0.y, b1.x, b1.y};
    #pragma unroll
    for (int i = 0; i < 4; ++i)
      #pragma unroll
      for (int jp = 0; jp < 4; ++jp) ffma2(acc[i][jp], av[i], bv[jp]);
  }
}

__global__ void __launch_bounds__(NUM_THREADS)
bsr_numeric_kernel(DevState* st, Mat X, int W, Pairs P, float* svals, uint8_t* skeep, double* spart,
                   double* sn2, double tau2) {
  extern __shared__ __align__(16) float num_smem[];
  if (!st->iter_active) return;
  const int nnz = *P.nnz;
  const int kprev = st->k;
  // Alg. 3 trace test, or the scheduled polynomial of SP2-ACC (Alg. 5): X_k = ca S + cb X + cc I
  double ca = 0.0, cb = 0.0, cc = 0.0;
  const int gen = st->acc;
  const int pk = gen ? acc_step(st, kprev + 1, ca, cb, cc) : (st->tr[kprev] > (double)st->nocc ? 1 : 0);
  const float fa = (float)ca, fb = (float)cb, fc = (float)cc;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rg = lane >> 2, cg = lane & 3;
  float* wbuf = num_smem + wid * WARP_FLOATS;
  const int gw = blockIdx.x * NUM_WARPS + wid, nw = gridDim.x * NUM_WARPS;
  for (int q = gw; q < nnz; q += nw) {
    const int I = P.row[q], J = P.col[q];
    unsigned long long acc2[4][4];
    #pragma unroll
    for (int i = 0; i < 4; ++i)
      #pragma unroll
      for (int jp = 0; jp < 4; ++jp) acc2[i][jp] = 0ull;     // +0.0f in both words
    int items = 0;
    const int b0 = X.rp[I], b1 = X.rp[I + 1];
    for (int e0 = b0; e0 < b1; e0 += 32) {
      const int e = e0 + lane;
      int pa = -1, pb = -1;
      if (e < b1) {
        const int K = X.ci[e];
        pb = find_block(X, W, K, J);
        if (pb >= 0) pa = find_block(X, W, K, I);
      }
      // (K, I) is present whenever (I, K) is (symmetric patterns); both are checked anyway
      unsigned mask = __ballot_sync(0xffffffffu, pa >= 0 && pb >= 0);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1u;
        const int a = __shfl_sync(0xffffffffu, pa, src);
        const int b = __shfl_sync(0xffffffffu, pb, src);
        #pragma unroll
        for (int h = 0; h < 2; ++h) {
          issue_half(wbuf, items & 1, X.vals, a, b, h, lane);
          if (items > 0) {
            cp_async_wait<1>();
            __syncwarp();
            product_tile(wbuf, (items - 1) & 1, rg, cg, acc2);
            __syncwarp();
          }
          ++items;
        }
      }
    }
    if (items > 0) {
      cp_async_wait<0>();
      __syncwarp();
      product_tile(wbuf, (items - 1) & 1, rg, cg, acc2);
      __syncwarp();
    }
    if (lane == 0) {
      atomicAdd(&st->bprod, (unsigned long long)(items / 2));
      atomicAdd(&st->uprod, (unsigned long long)(items / 2));   // every product formed is needed
    }
    float acc[4][8];
    #pragma unroll
    for (int i = 0; i < 4; ++i)
      #pragma unroll
      for (int jp = 0; jp < 4; ++jp)
        asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[i][2 * jp]), "=f"(acc[i][2 * jp + 1]) : "l"(acc2[i][jp]));
    // epilogue: X_old (I, J) of X~_{k-1} if stored; the new block is staged in the warp's
    // buffer (row stride B + 1) for the fixed-order norm
    const int po = find_block(X, W, I, J);
    float* blk = wbuf;
    float vloc = 0.f;
    double trloc = 0.0;
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = 4 * rg + i;
      float old[8];
      if (po >= 0) {
        const float4 o0 = *reinterpret_cast<const float4*>(X.vals + (int64_t)po * BE + r * B + 8 * cg);
        const float4 o1 = *reinterpret_cast<const float4*>(X.vals + (int64_t)po * BE + r * B + 8 * cg + 4);
        old[0] = o0.x; old[1] = o0.y; old[2] = o0.z; old[3] = o0.w;
        old[4] = o1.x; old[5] = o1.y; old[6] = o1.z; old[7] = o1.w;
      } else {
        #pragma unroll
        for (int j = 0; j < 8; ++j) old[j] = 0.f;
      }
      float nwv[8];
      #pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float sv = acc[i][j];
        nwv[j] = gen ? fmaf(fa, sv, fmaf(fb, old[j], (I == J && r == 8 * cg + j) ? fc : 0.f))
                     : (pk ? sv : fmaf(2.0f, old[j], -sv));
        const float d = old[j] - sv;
        vloc = fmaf(d, d, vloc);
        if (I == J && r == 8 * cg + j) trloc += (double)nwv[j];
        blk[r * (B + 1) + 8 * cg + j] = nwv[j];
      }
      float* dst = svals + (int64_t)q * BE + r * B + 8 * cg;
      *reinterpret_cast<float4*>(dst) = make_float4(nwv[0], nwv[1], nwv[2], nwv[3]);
      *reinterpret_cast<float4*>(dst + 4) = make_float4(nwv[4], nwv[5], nwv[6], nwv[7]);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vloc += __shfl_xor_sync(0xffffffffu, vloc, o);
      trloc += __shfl_xor_sync(0xffffffffu, trloc, o);
    }
    __syncwarp();
    const double n2 = block_norm2_fixed(blk);
    __syncwarp();
    if (lane == 0) {
      spart[2 * (int64_t)q] = (I == J ? 1.0 : 2.0) * (double)vloc;
      spart[2 * (int64_t)q + 1] = trloc;
      skeep[q] = (I == J || n2 >= tau2) ? 1 : 0;
      sn2[q] = n2;
    }
  }
}

// ---- error-controlled truncation (rule 1) ------------------------------------------------
// Candidates are the off-diagonal pairs with 2 n2 <= tau^2; the candidate of pair q weighs
// u_q = floor(2 n2_q / 2^(e-40)) units (2^e <= tau^2 < 2^(e+1)), the budget is
// floor(tau^2 / 2^(e-40)).  The pairs with key (n2 bits, q) <= K* are dropped, K* the
// largest key whose prefix sum is within the budget.  Integer sums do not depend on the
// summation order, so one CTA finds K* by a radix select: eight passes over the bytes of
// the n2 bit pattern (non-negative doubles order like their bit patterns), each a
// 256-bucket histogram of units over the candidates that share the digits chosen so far,
// find the value G whose candidates no longer all fit; they all weigh u(G), so the first
// m = (budget - units below G) / u(G) of them in q order are dropped.  The pair list is
// in (I, J) order, so q breaks ties as (I, J) does.  `cbits` (nnz entries of scratch)
// caches each pair's candidate bits (~0 if none).
constexpr int kEC = 512;

__device__ __forceinline__ uint64_t ec_units(uint64_t bits, int e) {
  return (uint64_t)floor(ldexp(__longlong_as_double((long long)bits), 41 - e));
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kEC)
bsr_errctl_kernel(const DevState* st, const double* n2, const int* row, const int* col, const int* nnz_p,
                  uint64_t* cbits, uint8_t* keep, double tau2) {
  __shared__ unsigned long long hist[256];
  __shared__ unsigned long long s_u64[2];
  __shared__ int s_int[kEC + 1];
  if (st && !st->iter_active) return;
  const int nnz = *nnz_p;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr uint64_t kNone = ~0ull;
  if (!(tau2 > 0.0)) {
    for (int q = tid; q < nnz; q += kEC) keep[q] = 1;
    return;
  }
  const int e = ilogb(tau2);     // 2^e <= tau^2 < 2^(e+1)
  const uint64_t budget = (uint64_t)floor(ldexp(tau2, 40 - e));
  // candidate bits and the total of their units
  if (tid == 0) s_u64[0] = 0ull;
  __syncthreads();
  uint64_t acc = 0;
  for (int q = tid; q < nnz; q += kEC) {
    const double v = n2[q];
    const bool c = row[q] != col[q] && 2.0 * v <= tau2;
    const uint64_t b = c ? (uint64_t)__double_as_longlong(v) : kNone;
    cbits[q] = b;
    if (c) acc += ec_units(b, e);
  }
  acc = warp_sum_u64(acc);
  if (lane == 0) atomicAdd(&s_u64[0], (unsigned long long)acc);
  __syncthreads();
  const uint64_t total = s_u64[0];
  uint64_t gbits = kNone;   // candidates with bits < gbits are dropped ...
  int qstar = -1;           // ... and those with bits == gbits and q <= qstar
  if (total > budget) {
    uint64_t prefix = 0, pmask = 0, below = 0;
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int d = tid; d < 256; d += kEC) hist[d] = 0ull;
      __syncthreads();
      for (int q0 = 0; q0 < nnz; q0 += kEC) {
        const int q = q0 + tid;
        const uint64_t b = q < nnz ? cbits[q] : kNone;
        const bool in = b != kNone && (b & pmask) == prefix;
        const int dig = in ? (int)((b >> shift) & 255u) : -1;
        const uint64_t u = in ? ec_units(b, e) : 0ull;
        const unsigned vm = __ballot_sync(0xffffffffu, in);
        if (!vm) continue;
        const int d0 = __shfl_sync(0xffffffffu, dig, __ffs(vm) - 1);
        if (__all_sync(0xffffffffu, !in || dig == d0)) {
          const uint64_t sum = warp_sum_u64(u);     // one atomic for the warp's common digit
          if (lane == 0) atomicAdd(&hist[d0], (unsigned long long)sum);
        } else if (in) {
          atomicAdd(&hist[dig], (unsigned long long)u);
        }
      }
      __syncthreads();
      if (tid == 0) {
        uint64_t run = below;
        int d = 0;
        for (; d < 255; ++d) {
          if (run + hist[d] > budget) break;
          run += hist[d];
        }
        s_u64[0] = run;
        s_u64[1] = (uint64_t)d;
      }
      __syncthreads();
      below = s_u64[0];
      prefix |= s_u64[1] << shift;
      pmask |= 255ull << shift;
      __syncthreads();
    }
    gbits = prefix;
    // every candidate with bits == gbits weighs u(gbits) > 0; m of them fit
    const uint64_t ug = ec_units(gbits, e);
    const uint64_t m = (budget - below) / ug;
    // the m-th member in q order: counts over contiguous q ranges, then a scan
    const int chunk = (nnz + kEC - 1) / kEC;
    const int lo = tid * chunk, hi = min(nnz, lo + chunk);
    int c = 0;
    for (int q = lo; q < hi; ++q) c += cbits[q] == gbits ? 1 : 0;
    s_int[tid + 1] = c;
    if (tid == 0) s_int[0] = 0;
    __syncthreads();
    if (tid == 0) {
      for (int t = 1; t <= kEC; ++t) s_int[t] += s_int[t - 1];
      s_u64[0] = ~0ull;
    }
    __syncthreads();
    if (m > 0 && (uint64_t)s_int[tid] < m && m <= (uint64_t)s_int[tid + 1]) {
      int seen = s_int[tid];
      for (int q = lo; q < hi; ++q)
        if (cbits[q] == gbits && (uint64_t)(++seen) == m) { s_u64[0] = (unsigned long long)q; break; }
    }
    __syncthreads();
    qstar = m > 0 ? (int)s_u64[0] : -1;
  }
  for (int q = tid; q < nnz; q += kEC) {
    const uint64_t b = cbits[q];
    const bool drop = b != kNone && (b < gbits || (b == gbits && q <= qstar));
    keep[q] = drop ? 0 : 1;
  }
}

// ---- mixed-norm truncation (rule 2) ------------------------------------------------------
// Candidates are the off-diagonal pairs with ||X_IJ||_F = sqrt(n2) <= tau, weighing
// u_q = floor(||X_IJ||_F / 2^(e-40)) units (2^e <= tau < 2^(e+1)); every block row may take
// floor(tau / 2^(e-40)) units, and dropping pair q = (I, J) adds u_q to rows I and J.  Dropped:
// the longest prefix of the key order (n2 bits, q) in which every row stays within the budget.
// Walking that order, the first candidate that does not fit is the earliest of the rows' own
// first overflows: restricted to the candidates touching row r the global order is r's own
// sorted order, and r's sum at a candidate counts exactly r's earlier candidates.  So one CTA
// per row sorts the row's candidates by key, scans their units and reports the key at which
// its sum first exceeds the budget; the cut is the smallest reported key and every candidate
// below it is dropped: the decision of the sequential walk, without a global sort.
constexpr int kMR = 256;                 // threads of the per-row kernel
constexpr int kMRMax = MAX_NB;           // candidates of one row: fewer than nb <= MAX_NB

__device__ __forceinline__ void mr_push(double v, int q, double tau, int e, unsigned long long* kb, int* kq,
                                        unsigned long long* ku, int* n) {
  const double w = sqrt(v);
  if (!(w <= tau)) return;
  const int pos = atomicAdd(n, 1);
  kb[pos] = (unsigned long long)__double_as_longlong(v);
  kq[pos] = q;
  ku[pos] = (unsigned long long)floor(ldexp(w, 40 - e));
}

__global__ void __launch_bounds__(kMR)
mix_row_kernel(const DevState* st, const double* __restrict__ n2, const int* __restrict__ ptr,
               const int* __restrict__ col, int nb, double tau, uint64_t* key_bits, int* key_q) {
  __shared__ unsigned long long kb[kMRMax];
  __shared__ unsigned long long ku[kMRMax];
  __shared__ int kq[kMRMax];
  __shared__ unsigned long long s_part[kMR + 1];
  __shared__ int s_n, s_first;
  if (st && !st->iter_active) return;
  const int r = blockIdx.x, tid = threadIdx.x;
  if (!(tau > 0.0)) {
    if (tid == 0) { key_bits[r] = ~0ull; key_q[r] = INT_MAX; }
    return;
  }
  const int e = ilogb(tau);
  const unsigned long long budget = (unsigned long long)floor(ldexp(tau, 40 - e));
  if (tid == 0) { s_n = 0; s_first = INT_MAX; }
  __syncthreads();
  for (int q = ptr[r] + tid; q < ptr[r + 1]; q += kMR)          // (r, J > r)
    if (col[q] != r) mr_push(n2[q], q, tau, e, kb, kq, ku, &s_n);
  for (int I = tid; I < r; I += kMR) {                          // (I < r, r): search row I
    int lo = ptr[I], hi = ptr[I + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (col[mid] < r) lo = mid + 1;
      else hi = mid;
    }
    if (lo < ptr[I + 1] && col[lo] == r) mr_push(n2[lo], lo, tau, e, kb, kq, ku, &s_n);
  }
  __syncthreads();
  const int n = s_n;
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = n + tid; i < P; i += kMR) { kb[i] = ~0ull; kq[i] = INT_MAX; ku[i] = 0ull; }
  __syncthreads();
  // bitonic sort by (bits, q), ascending
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += kMR) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const bool gt = kb[i] > kb[l] || (kb[i] == kb[l] && kq[i] > kq[l]);
          if (gt == up) {
            const unsigned long long tb = kb[i], tu = ku[i];
            const int tq = kq[i];
            kb[i] = kb[l]; ku[i] = ku[l]; kq[i] = kq[l];
            kb[l] = tb; ku[l] = tu; kq[l] = tq;
          }
        }
      }
      __syncthreads();
    }
  }
  // running sum of units in that order: segments per thread, an exclusive scan of their sums,
  // then each thread finds the first overflow inside its segment
  const int seg = (P + kMR - 1) / kMR;
  const int a = tid * seg, z = min(P, a + seg);
  unsigned long long loc = 0ull;
  for (int i = a; i < z; ++i) loc += ku[i];
  s_part[tid + 1] = loc;
  if (tid == 0) s_part[0] = 0ull;
  __syncthreads();
  if (tid == 0)
    for (int t = 1; t <= kMR; ++t) s_part[t] += s_part[t - 1];
  __syncthreads();
  unsigned long long run = s_part[tid];
  for (int i = a; i < z; ++i) {
    run += ku[i];
    if (run > budget) { atomicMin(&s_first, i); break; }
  }
  __syncthreads();
  if (tid == 0) {
    const int f = s_first;
    key_bits[r] = f < n ? (uint64_t)kb[f] : ~0ull;
    key_q[r] = f < n ? kq[f] : INT_MAX;
  }
}

// the cut: the smallest (bits, q) the rows reported, into cut[0] (bits) and cut[1] (q)
__global__ void __launch_bounds__(1024)
mix_cut_kernel(const DevState* st, const uint64_t* key_bits, const int* key_q, int nb, uint64_t* cut) {
  __shared__ unsigned long long sb[1024];
  __shared__ int sq[1024];
  if (st && !st->iter_active) return;
  const int tid = threadIdx.x;
  unsigned long long b = ~0ull;
  int q = INT_MAX;
  for (int r = tid; r < nb; r += 1024) {
    const unsigned long long rb = key_bits[r];
    const int rq = key_q[r];
    if (rb < b || (rb == b && rq < q)) { b = rb; q = rq; }
  }
  sb[tid] = b;
  sq[tid] = q;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (tid < o && (sb[tid + o] < sb[tid] || (sb[tid + o] == sb[tid] && sq[tid + o] < sq[tid]))) {
      sb[tid] = sb[tid + o];
      sq[tid] = sq[tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    cut[0] = sb[0];
    cut[1] = (uint64_t)(uint32_t)sq[0];
  }
}

__global__ void mix_keep_kernel(const DevState* st, const double* n2, const int* row, const int* col, const int* nnz_p,
                                double tau, const uint64_t* cut, uint8_t* keep) {
  if (st && !st->iter_active) return;
  const int nnz = *nnz_p;
  const uint64_t cb = cut[0];
  const int cq = (int)(uint32_t)cut[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
    const double v = n2[q];
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const bool cand = tau > 0.0 && row[q] != col[q] && sqrt(v) <= tau;
    keep[q] = cand && (b < cb || (b == cb && q < cq)) ? 0 : 1;
  }
}

// scratch: key bits [nb] (8 B), cut [2] (8 B), key q [nb] (4 B)
size_t mixctl_scratch_bytes(int nb) { return sizeof(uint64_t) * (nb + 2) + sizeof(int) * nb; }

void launch_mixctl(const DevState* st, const double* n2, const int* ptr, const int* row, const int* col,
                   const int* nnz_p, int nb, double tau, void* scratch, uint8_t* keep, int grid, cudaStream_t s) {
  uint64_t* kbits = static_cast<uint64_t*>(scratch);
  uint64_t* cut = kbits + nb;
  int* kq = reinterpret_cast<int*>(cut + 2);
  mix_row_kernel<<<nb, kMR, 0, s>>>(st, n2, ptr, col, nb, tau, kbits, kq);
  mix_cut_kernel<<<1, 1024, 0, s>>>(st, kbits, kq, nb, cut);
  mix_keep_kernel<<<grid, 256, 0, s>>>(st, n2, row, col, nnz_p, tau, cut, keep);
}

// per-round reduction over the pairs and the stop test (stored-diagonal trace)
__global__ void __launch_bounds__(1024)
bsr_finalize_kernel(DevState* st, const double* spart, const int* nnz_p, cudaGraphConditionalHandle cond,
                    int use_cond) {
  __shared__ double sm[32];
  if (!st->iter_active) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  const int nnz = *nnz_p;
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nnz; t += 1024) { a += spart[2 * (int64_t)t]; b += spart[2 * (int64_t)t + 1]; }
  a = block_sum<1024>(a, sm);
  b = block_sum<1024>(b, sm);
  if (threadIdx.x != 0) return;
  const int k = st->k + 1;
  double ca, cb, cc;
  const int pk = st->acc ? acc_step(st, k, ca, cb, cc) : (st->tr[k - 1] > (double)st->nocc ? 1 : 0);
  st->sblocks += (unsigned long long)nnz;
  // v_{k-1}, or m_{k-1}: the Lanczos estimate of the mixed norm with the 32 x 32 blocks
  record_and_test(st, pk, st->norm == 1 ? st->spec_e : sqrt(a), b, st->tr[k - 1]);
  // the loop stops after this round's truncation (the kernels below still run)
  if (use_cond && st->done) cudaGraphSetConditional(cond, 0);
}

// ---- truncation and the next iterate ------------------------------------------------------------
__global__ void set_kept_bits_kernel(const DevState* st, Pairs P, const uint8_t* skeep, int W, uint32_t* bits) {
  if (st && !st->iter_active) return;
  const int nnz = *P.nnz;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
    if (!skeep[q]) continue;
    const int I = P.row[q], J = P.col[q];
    atomicOr(&bits[(int64_t)I * W + (J >> 5)], 1u << (J & 31));
    atomicOr(&bits[(int64_t)J * W + (I >> 5)], 1u << (I & 31));
  }
}

// kept upper block q -> row I at the rank of J, its transpose -> row J at the rank of I
__global__ void __launch_bounds__(NT)
fill_next_kernel(const DevState* st, Pairs P, const uint8_t* skeep, const float* svals, Mat Y, int W) {
  if (st && !st->iter_active) return;
  const int nnz = *P.nnz;
  for (int q = blockIdx.x; q < nnz; q += gridDim.x) {
    if (!skeep[q]) continue;
    const int I = P.row[q], J = P.col[q];
    const int pij = find_block(Y, W, I, J);
    const int pji = find_block(Y, W, J, I);
    if (threadIdx.x == 0) {
      Y.ci[pij] = J;
      Y.ci[pji] = I;
    }
    const float* src = svals + (int64_t)q * BE;
    for (int e = threadIdx.x; e < BE; e += NT) {
      const float v = src[e];
      const int64_t et = (e % B) * B + e / B;
      Y.vals[(int64_t)pij * BE + e] = v;
      if (I != J) Y.vals[(int64_t)pji * BE + et] = v;
      if (Y.pvals) {   // the fp16 pieces of 2^14 v, the tensor-core operands
        __half p0, p1;
        tc::split_fp16x2(v, p0, p1);
        Y.pvals[(int64_t)pij * 2 * BE + e] = p0;
        Y.pvals[(int64_t)pij * 2 * BE + BE + e] = p1;
        if (I != J) {
          Y.pvals[(int64_t)pji * 2 * BE + et] = p0;
          Y.pvals[(int64_t)pji * 2 * BE + BE + et] = p1;
        }
      }
    }
  }
}

// ---- tile list of the tensor-core square ------------------------------------------------------
// Tile (g, c) = block rows 4 g .. 4 g + 3, block columns 8 c .. 8 c + 7; listed when one of its
// rows holds an upper pair of the square's pattern in its columns.
__device__ __forceinline__ bool tile_active(const uint32_t* sbits, int nb, int W, int g, int c) {
  bool act = false;
  for (int r = 0; r < TTR; ++r) {
    const int I = g * TTR + r;
    if (I >= nb) break;
    const uint32_t word = sbits[(int64_t)I * W + ((c * TTC) >> 5)];
    act |= ((word >> ((c * TTC) & 31)) & 0xFFu) != 0u;
  }
  return act;
}

__global__ void tile_count_kernel(const DevState* st, const uint32_t* sbits, int nb, int W, int ncg, int* counts) {
  if (!st->iter_active) return;
  const int g = blockIdx.x;
  int n = 0;
  for (int c = threadIdx.x; c < ncg; c += 32) n += tile_active(sbits, nb, W, g, c) ? 1 : 0;
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if (threadIdx.x == 0) counts[g] = n;
}

__global__ void tile_fill_kernel(const DevState* st, const uint32_t* sbits, int nb, int W, int ncg, const int* tptr,
                                 int* tiles) {
  if (!st->iter_active) return;
  const int g = blockIdx.x, lane = threadIdx.x;
  int pos = tptr[g];
  for (int c0 = 0; c0 < ncg; c0 += 32) {
    const int c = c0 + lane;
    const bool act = c < ncg && tile_active(sbits, nb, W, g, c);
    const uint32_t m = __ballot_sync(0xffffffffu, act);
    if (act) tiles[pos + __popc(m & ((1u << lane) - 1u))] = g * ncg + c;
    pos += __popc(m);
  }
}

// Per listed tile (one warp): the K-block count (the K some tile row and some tile column both
// hold, from the OR of the rows' bitmap words), and for block pair (r, c) = lane / 8, lane % 8 the
// pair index and the old block's position.
__global__ void tile_meta_kernel(const DevState* st, Mat X, Pairs P, const uint32_t* sbits, int nb, int W, int ncg,
                                 const int* tiles, const int* tnnz, int* meta) {
  if (!st->iter_active) return;
  const int lane = threadIdx.x & 31;
  const int nt = *tnnz;
  for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt; t += gridDim.x * (blockDim.x >> 5)) {
    const int code = tiles[t];
    const int I0 = (code / ncg) * TTR, J0 = (code % ncg) * TTC;
    const int rowj = lane < TTR ? I0 + lane : J0 + (lane - TTR);
    const bool vj = lane < TTR + TTC && rowj < nb;
    int nk = 0;
    for (int w = 0; w < W; ++w) {
      const uint32_t bj = vj ? X.bits[(int64_t)rowj * W + w] : 0u;
      const uint32_t a = __reduce_or_sync(0xffffffffu, lane < TTR ? bj : 0u);
      const uint32_t b = __reduce_or_sync(0xffffffffu, lane >= TTR && lane < TTR + TTC ? bj : 0u);
      nk += __popc(a & b);
    }
    const int I = I0 + lane / TTC, J = J0 + lane % TTC;
    // block products the pair (I, J) needs: K blocks both rows hold (upper pairs only)
    int need = 0;
    if (I < nb && J < nb && J >= I)
      for (int w = 0; w < W; ++w) need += __popc(X.bits[(int64_t)I * W + w] & X.bits[(int64_t)J * W + w]);
    need = __reduce_add_sync(0xffffffffu, need);
    int qi = -1, po = -1;
    if (I < nb && J < nb) {
      po = find_block(X, W, I, J);
      if (J >= I) {
        const uint32_t sw = sbits[(int64_t)I * W + (J >> 5)];
        if ((sw >> (J & 31)) & 1u) {
          int cnt = P.ptr[I] + __popc(sw & ((1u << (J & 31)) - 1u));
          for (int w = 0; w < (J >> 5); ++w) cnt += __popc(sbits[(int64_t)I * W + w]);
          qi = cnt;
        }
      }
    }
    int* m = meta + (int64_t)t * TMETA;
    if (lane == 0) { m[0] = nk; m[65] = need; }
    m[1 + lane] = qi;
    m[33 + lane] = po;
  }
}

// SMs of the current device (queried once, before any stream capture; see build_graph)
static int meta_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  return sms;
}

cudaError_t tc_tiles_launch(const DevState* st, const Mat& X, const Pairs& P, const uint32_t* sbits, int nb, int W,
                            int* counts, int* tptr, int* tnnz, int* tiles, int* meta, cudaStream_t s) {
  const int ng = (nb + TTR - 1) / TTR, ncg = (nb + TTC - 1) / TTC;
  tile_count_kernel<<<ng, 32, 0, s>>>(st, sbits, nb, W, ncg, counts);
  scan_kernel<<<1, 1024, 0, s>>>(counts, ng, tptr, tnnz, st);
  tile_fill_kernel<<<ng, 32, 0, s>>>(st, sbits, nb, W, ncg, tptr, tiles);
  tile_meta_kernel<<<4 * meta_sms(), 256, 0, s>>>(st, X, P, sbits, nb, W, ncg, tiles, tnnz, meta);
  return cudaGetLastError();
}

// dense FP64 output (N x N, leading dimension N) from the iterate the stop test chose
__global__ void bsr_to_dense_kernel(const DevState* st, Mat X0, Mat X1, int nb, double* D) {
  const int N = nb * B;
  const int mode = st->out_mode;
  const Mat X = st->out_buf ? X1 : X0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    double val = 0.0;
    if (mode == OUT_COPY) {
      const int W = (nb + 31) / 32;
      const int p = find_block(X, W, i / B, j / B);
      if (p >= 0) val = (double)X.vals[(int64_t)p * BE + (i % B) * B + j % B];
    } else if (mode == OUT_IDENTITY) {
      val = (i == j) ? 1.0 : 0.0;
    } else if (mode == OUT_NAN) {
      val = __longlong_as_double(0x7ff8000000000000ll);
    }
    D[e] = val;
  }
}

}  // namespace bsr
}  // namespace sp2

// =================================================================================================
// Host side: handle and C ABI
// =================================================================================================
using namespace sp2;
using namespace sp2::bsr;

struct sp2_bsr_ctx {
  int64_t N = 0, nocc = 0;
  int nb = 0, W = 0;
  double tau = 0.0;
  int rule = 0;                  // sp2_trunc_rule
  sp2_opts opts{};
  int device = 0;
  int64_t cap = 0, cap_s = 0;
  Mat X[2];
  Pairs S{}, FP{};
  uint32_t* sbits = nullptr;
  float* svals = nullptr;
  uint8_t* skeep = nullptr;
  double* spart = nullptr;       // per-pair partials; also the candidate scratch of rule 1
  double* sn2 = nullptr;         // per-pair ||X_IJ||_F^2 of the newest blocks
  void* mixscr = nullptr;        // rule 2: per-row overflow keys and the cut
  void* lz = nullptr;            // norm = 1: Lanczos scratch for the mixed norm (nb x nb)
  int lzld = 0;
  int* counts = nullptr;
  uint32_t* fbits = nullptr;
  int* frank = nullptr;
  int* fnnz_scratch = nullptr;
  double *glo = nullptr, *ghi = nullptr;
  int* gbad = nullptr;
  DevState* st_dev = nullptr;
  DevState* st_host = nullptr;
  int* xnnz_host = nullptr;      // pinned: rp[nb] of the output iterate
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaEvent_t* nev = nullptr;    // launch mode 1: events around each numeric-square launch
  int nrounds = 0;               // numeric launches recorded in the last run
  cudaStream_t last = nullptr;
  bool ran = false;
  // tensor-core block products (opts.bsr_cuda_cores == 0)
  bool tc = false;
  TcMaps* maps_dev = nullptr;    // TMA maps over X[0].pvals and X[1].pvals
  int* tiles = nullptr;          // [ceil(nb/4) * ceil(nb/8)]
  int* tptr = nullptr;           // [ceil(nb/4) + 1]
  int* tnnz = nullptr;
  int* meta = nullptr;           // [ceil(nb/4) * ceil(nb/8)][TMETA]
};

#define BSR_TRY(expr)                              \
  do {                                             \
    if ((expr) != cudaSuccess) {                   \
      (void)cudaGetLastError();                    \
      return SP2_ERR_CUDA;                         \
    }                                              \
  } while (0)

static void bsr_free(sp2_bsr_ctx* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (int p = 0; p < 2; ++p) {
    cudaFree(h->X[p].rp); cudaFree(h->X[p].ci); cudaFree(h->X[p].vals); cudaFree(h->X[p].bits);
    cudaFree(h->X[p].rank); cudaFree(h->X[p].pvals);
  }
  cudaFree(h->maps_dev); cudaFree(h->tiles); cudaFree(h->tptr); cudaFree(h->tnnz); cudaFree(h->meta);
  cudaFree(h->S.ptr); cudaFree(h->S.col); cudaFree(h->S.row); cudaFree(h->S.nnz);
  cudaFree(h->FP.ptr); cudaFree(h->FP.col); cudaFree(h->FP.row); cudaFree(h->FP.nnz);
  cudaFree(h->sbits); cudaFree(h->svals); cudaFree(h->skeep); cudaFree(h->spart); cudaFree(h->sn2);
  cudaFree(h->mixscr); cudaFree(h->lz);
  cudaFree(h->counts);
  cudaFree(h->fbits); cudaFree(h->frank); cudaFree(h->glo); cudaFree(h->ghi); cudaFree(h->gbad);
  cudaFree(h->st_dev);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->xnnz_host) cudaFreeHost(h->xnnz_host);
  if (h->ev[0]) cudaEventDestroy(h->ev[0]);
  if (h->ev[1]) cudaEventDestroy(h->ev[1]);
  if (h->nev) {
    for (int i = 0; i < 2 * (h->opts.max_iter + 4); ++i)
      if (h->nev[i]) cudaEventDestroy(h->nev[i]);
    delete[] h->nev;
  }
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  delete h;
}

// Persistent grid of the numeric square: the resident CTAs of the whole GPU.
static int numeric_grid() {
  static int n = 0;
  if (!n) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(bsr_numeric_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, NUM_SMEM) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bsr_numeric_kernel, NUM_THREADS, NUM_SMEM) !=
            cudaSuccess ||
        per < 1) {
      (void)cudaGetLastError();
      per = 1;
    }
    n = std::max(1, sms) * per;
  }
  return n;
}

static int grid_persistent() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n * 4;
}

// One loop round (the body of the WHILE node, or one unrolled round in launch mode 1).
// The buffers alternate by round: round k reads X[(k-1)&1] and writes X[k&1]; a graph
// body is fixed, so two bodies are recorded and the loop runs them in pairs.
static cudaError_t add_round(sp2_bsr_ctx* h, cudaGraph_t g, cudaStream_t s, int parity, int use_cond) {
  // parity: 0 = X[0] -> X[1], 1 = X[1] -> X[0]
  Mat Xc = h->X[parity], Xn = h->X[1 - parity];
  const int nb = h->nb, W = h->W;
  const double tau2 = h->tau * h->tau;
  const int up = 1;
  DevState* st = h->st_dev;
  int* sn = h->S.nnz;
  (void)g;
  // 1. symbolic
  bsr_sym_kernel<<<nb, 64, 0, s>>>(st, Xc, nb, W, h->sbits);
  row_counts_kernel<<<nb, 64, 0, s>>>(h->sbits, nb, W, up, h->counts, st);
  scan_kernel<<<1, 1024, 0, s>>>(h->counts, nb, h->S.ptr, sn, st);
  fill_pairs_kernel<<<nb, 32, 0, s>>>(h->sbits, nb, W, up, h->S, st);
  // 2. numeric + 3. stop test
  if (h->tc) tc_tiles_launch(st, Xc, h->S, h->sbits, nb, W, h->counts, h->tptr, h->tnnz, h->tiles, h->meta, s);
  const bool timed = !use_cond && h->nev && h->nrounds < h->opts.max_iter + 4;
  if (timed) cudaEventRecord(h->nev[2 * h->nrounds], s);
  if (h->tc) {
    TcRound r;
    r.sbits = h->sbits;
    r.P = h->S;
    r.svals = h->svals;
    r.skeep = h->skeep;
    r.spart = h->spart;
    r.sn2 = h->sn2;
    r.tau2 = tau2;
    r.tiles = h->tiles;
    r.tnnz = h->tnnz;
    r.meta = h->meta;
    tc_numeric_launch(st, Xc, h->maps_dev, parity, nb, W, r, s);
  } else {
    bsr_numeric_kernel<<<numeric_grid(), NUM_THREADS, NUM_SMEM, s>>>(st, Xc, W, h->S, h->svals, h->skeep,
                                                                    h->spart, h->sn2, tau2);
  }
  if (timed) cudaEventRecord(h->nev[2 * h->nrounds++ + 1], s);
  if (h->lz) launch_lanczos_pairs(st, h->S.row, h->S.col, sn, h->spart, h->lz, nb, h->lzld, s);
  bsr_finalize_kernel<<<1, 1024, 0, s>>>(st, h->spart, sn, h->cond, use_cond);
  if (h->rule == SP2_TRUNC_ERROR)
    bsr_errctl_kernel<<<1, kEC, 0, s>>>(st, h->sn2, h->S.row, h->S.col, sn, reinterpret_cast<uint64_t*>(h->spart),
                                        h->skeep, tau2);
  else if (h->rule == SP2_TRUNC_MIXED)
    launch_mixctl(st, h->sn2, h->S.ptr, h->S.row, h->S.col, sn, nb, h->tau, h->mixscr, h->skeep, grid_persistent(), s);
  // 4. truncation -> next iterate
  clear_words_kernel<<<256, 256, 0, s>>>(Xn.bits, (int64_t)nb * W, st);
  set_kept_bits_kernel<<<grid_persistent(), 256, 0, s>>>(st, h->S, h->skeep, W, Xn.bits);
  rank_kernel<<<nb, 32, 0, s>>>(Xn.bits, nb, W, Xn.rank, st);
  row_counts_kernel<<<nb, 64, 0, s>>>(Xn.bits, nb, W, 0, h->counts, st);
  scan_kernel<<<1, 1024, 0, s>>>(h->counts, nb, Xn.rp, nullptr, st);
  fill_next_kernel<<<grid_persistent(), NT, 0, s>>>(st, h->S, h->skeep, h->svals, Xn, W);
  return cudaGetLastError();
}

static sp2_status build_graph(sp2_bsr_ctx* h) {
  // The loop body holds two rounds (X[0] -> X[1] -> X[0]); it is recorded by stream
  // capture into the WHILE node's body graph.
  BSR_TRY(cudaGraphCreate(&h->graph, 0));
  BSR_TRY(cudaGraphConditionalHandleCreate(&h->cond, h->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h->cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  BSR_TRY(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  (void)grid_persistent();   // device queries before capture
  (void)numeric_grid();
  (void)meta_sms();
  tc_prepare();
  cudaStream_t cs;
  BSR_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    add_round(h, body, cs, 0, 1);
    add_round(h, body, cs, 1, 1);
    cudaGraph_t out = body;
    e = cudaStreamEndCapture(cs, &out);
  }
  cudaStreamDestroy(cs);
  BSR_TRY(e);
  BSR_TRY(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return SP2_OK;
}

extern "C" sp2_status sp2_create_bsr(int64_t N, int64_t n_occ, double tau, const sp2_opts* opts, sp2_bsr* out) {
  return sp2_create_bsr_ex(N, n_occ, tau, SP2_TRUNC_BLOCK, opts, out);
}

extern "C" sp2_status sp2_create_bsr_ex(int64_t N, int64_t n_occ, double tau, int32_t rule, const sp2_opts* opts,
                                        sp2_bsr* out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < B || N % B != 0 || N / B > MAX_NB || n_occ < 0 || n_occ > N || !(tau >= 0.0) ||
      (rule != SP2_TRUNC_BLOCK && rule != SP2_TRUNC_ERROR && rule != SP2_TRUNC_MIXED))
    return SP2_ERR_INVALID_ARG;
  sp2_opts o;
  sp2_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.max_iter > SP2_MAX_ITER || !(o.qtilde > 0.0) || (o.guard != 0 && o.guard != 1) ||
      (o.launch_mode != 0 && o.launch_mode != 1))
    return SP2_ERR_INVALID_ARG;
  if (o.norm < 0 || o.norm > 2 || (o.bsr_cuda_cores != 0 && o.bsr_cuda_cores != 1)) return SP2_ERR_INVALID_ARG;
  if (o.norm == 2) return SP2_ERR_UNSUPPORTED;       // v_i or the mixed norm m_i (32 x 32 blocks)
  sp2_bsr_ctx* h = new (std::nothrow) sp2_bsr_ctx();
  if (!h) return SP2_ERR_NOMEM;
  h->N = N; h->nocc = n_occ; h->tau = tau; h->rule = rule; h->opts = o;
  h->nb = (int)(N / B);
  h->W = (h->nb + 31) / 32;
  h->cap = (int64_t)h->nb * h->nb;
  h->cap_s = (int64_t)h->nb * (h->nb + 1) / 2;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return SP2_ERR_CUDA; }
  const int nb = h->nb, W = h->W;
  bool ok = true;
  for (int p = 0; p < 2 && ok; ++p) {
    ok = cudaMalloc(&h->X[p].rp, sizeof(int) * (nb + 1)) == cudaSuccess &&
         cudaMalloc(&h->X[p].ci, sizeof(int) * h->cap) == cudaSuccess &&
         cudaMalloc(&h->X[p].vals, sizeof(float) * BE * h->cap) == cudaSuccess &&
         cudaMalloc(&h->X[p].bits, sizeof(uint32_t) * nb * W) == cudaSuccess &&
         cudaMalloc(&h->X[p].rank, sizeof(int) * nb * W) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&h->S.ptr, sizeof(int) * (nb + 1)) == cudaSuccess &&
       cudaMalloc(&h->S.col, sizeof(int) * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->S.row, sizeof(int) * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->S.nnz, sizeof(int)) == cudaSuccess &&
       cudaMalloc(&h->FP.ptr, sizeof(int) * (nb + 1)) == cudaSuccess &&
       cudaMalloc(&h->FP.col, sizeof(int) * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->FP.row, sizeof(int) * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->FP.nnz, sizeof(int)) == cudaSuccess &&
       cudaMalloc(&h->sbits, sizeof(uint32_t) * nb * W) == cudaSuccess &&
       cudaMalloc(&h->svals, sizeof(float) * BE * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->skeep, h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->spart, sizeof(double) * 2 * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->sn2, sizeof(double) * h->cap_s) == cudaSuccess &&
       cudaMalloc(&h->counts, sizeof(int) * nb) == cudaSuccess &&
       cudaMalloc(&h->fbits, sizeof(uint32_t) * nb * W) == cudaSuccess &&
       cudaMalloc(&h->frank, sizeof(int) * nb * W) == cudaSuccess &&
       cudaMalloc(&h->glo, sizeof(double) * nb) == cudaSuccess &&
       cudaMalloc(&h->ghi, sizeof(double) * nb) == cudaSuccess &&
       cudaMalloc(&h->gbad, sizeof(int) * nb) == cudaSuccess &&
       cudaMalloc(&h->st_dev, sizeof(DevState)) == cudaSuccess &&
       cudaMallocHost(&h->st_host, sizeof(DevState)) == cudaSuccess &&
       cudaMallocHost(&h->xnnz_host, sizeof(int)) == cudaSuccess &&
       cudaEventCreate(&h->ev[0]) == cudaSuccess && cudaEventCreate(&h->ev[1]) == cudaSuccess;
  h->tc = o.bsr_cuda_cores == 0;
  if (ok && h->tc) {
    const int ng = (nb + TTR - 1) / TTR, ncg = (nb + TTC - 1) / TTC;
    const size_t pbytes = sizeof(__half) * 2 * BE * (size_t)(h->cap + 1);
    for (int p = 0; p < 2 && ok; ++p)
      ok = cudaMalloc(&h->X[p].pvals, pbytes) == cudaSuccess &&
           cudaMemset(h->X[p].pvals, 0, pbytes) == cudaSuccess;   // block `cap` stays zero
    ok = ok && cudaMalloc(&h->maps_dev, sizeof(TcMaps)) == cudaSuccess &&
         cudaMalloc(&h->tiles, sizeof(int) * (size_t)ng * ncg) == cudaSuccess &&
         cudaMalloc(&h->tptr, sizeof(int) * (ng + 1)) == cudaSuccess &&
         cudaMalloc(&h->tnnz, sizeof(int)) == cudaSuccess &&
         cudaMalloc(&h->meta, sizeof(int) * TMETA * (size_t)ng * ncg) == cudaSuccess;
    if (ok) {
      TcMaps m;
      std::memset(&m, 0, sizeof(m));
      ok = tc_piece_map(h->X[0].pvals, h->cap, &m.map[0]) == cudaSuccess &&
           tc_piece_map(h->X[1].pvals, h->cap, &m.map[1]) == cudaSuccess &&
           cudaMemcpy(h->maps_dev, &m, sizeof(m), cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (ok && rule == SP2_TRUNC_MIXED) ok = cudaMalloc(&h->mixscr, mixctl_scratch_bytes(nb)) == cudaSuccess;
  if (ok && o.norm == 1) {
    h->lzld = (nb + 63) / 64 * 64;
    ok = cudaMalloc(&h->lz, lanczos_scratch_bytes(h->lzld)) == cudaSuccess;
  }
  if (!ok) { (void)cudaGetLastError(); bsr_free(h); return SP2_ERR_NOMEM; }
  DevState init;
  std::memset(&init, 0, sizeof(init));
  init.N = (int32_t)N; init.ld = (int32_t)N; init.nocc = (int32_t)n_occ;
  init.max_iter = o.max_iter; init.guard = o.guard; init.qtilde = o.qtilde; init.round_fp32 = 1;
  init.norm = o.norm;
  *h->st_host = init;
  *h->xnnz_host = 0;
  if (cudaMemcpy(h->st_dev, &init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) {
    (void)cudaGetLastError(); bsr_free(h); return SP2_ERR_CUDA;
  }
  if (o.launch_mode == 1) {
    const int ne = 2 * (o.max_iter + 4);
    h->nev = new (std::nothrow) cudaEvent_t[ne]();
    bool eok = h->nev != nullptr;
    for (int i = 0; i < ne && eok; ++i) eok = cudaEventCreate(&h->nev[i]) == cudaSuccess;
    if (!eok) { (void)cudaGetLastError(); bsr_free(h); return SP2_ERR_NOMEM; }
  }
  sp2_status s = o.launch_mode == 0 ? build_graph(h) : SP2_OK;
  if (s == SP2_OK && cudaDeviceSynchronize() != cudaSuccess) { (void)cudaGetLastError(); s = SP2_ERR_CUDA; }
  if (s != SP2_OK) { bsr_free(h); return s; }
  *out = h;
  return SP2_OK;
}

extern "C" void sp2_destroy_bsr(sp2_bsr h) { bsr_free(h); }

extern "C" int32_t sp2_set_bounds_bsr(sp2_bsr h, const double* bounds) {
  if (!h || (bounds && !(std::isfinite(bounds[0]) && std::isfinite(bounds[1]) && bounds[0] < bounds[1])))
    return SP2_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  const int32_t r = sp2::write_bound_fields(h->st_dev, h->st_host, bounds);
  cudaSetDevice(cur);
  return r;
}

extern "C" int32_t sp2_set_homo_lumo_bsr(sp2_bsr h, const double* bounds) {
  if (!h || (bounds && !sp2::acc_bounds_ok(bounds))) return SP2_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  const int32_t r = sp2::write_acc_fields(h->st_dev, h->st_host, bounds);
  cudaSetDevice(cur);
  return r;
}

extern "C" sp2_status sp2_get_work_bsr(sp2_bsr h, int64_t* block_products, int64_t* needed_products,
                                       int64_t* square_blocks, double* numeric_ms) {
  if (!h || !block_products || !needed_products || !square_blocks || !numeric_ms) return SP2_ERR_INVALID_ARG;
  if (h->ran) BSR_TRY(cudaStreamSynchronize(h->last));
  *block_products = h->ran ? (int64_t)h->st_host->bprod : 0;
  *needed_products = h->ran ? (int64_t)h->st_host->uprod : 0;
  *square_blocks = h->ran ? (int64_t)h->st_host->sblocks : 0;
  double tot = 0.0;
  for (int r = 0; h->ran && h->nev && r < h->nrounds; ++r) {
    float ms = 0.f;
    BSR_TRY(cudaEventElapsedTime(&ms, h->nev[2 * r], h->nev[2 * r + 1]));
    tot += ms;
  }
  *numeric_ms = tot;
  return SP2_OK;
}

extern "C" sp2_status sp2_run_bsr(sp2_bsr h, const int32_t* row_ptr_dev, const int32_t* col_idx_dev,
                                  const double* vals_dev, int64_t nnzb, double* D_dev, void* stream) {
  nvtxRangePushA("sp2_run_bsr");                  // host-side range over the enqueue
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  if (!h || !row_ptr_dev || !col_idx_dev || !vals_dev || nnzb < h->nb || nnzb > h->cap) return SP2_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = h->nb, W = h->W;
  DevState* st = h->st_dev;
  const double tau2 = h->tau * h->tau;
  // bounds, special cases, Tr[X_0]
  bsr_gersh_kernel<<<nb, B, 0, s>>>(row_ptr_dev, col_idx_dev, vals_dev, nb, h->glo, h->ghi, h->gbad);
  bsr_init_kernel<<<1, kIT, 0, s>>>(st, row_ptr_dev, col_idx_dev, vals_dev, nb, h->glo, h->ghi, h->gbad);
  // X_0 on F's upper pattern, truncated into X[0]
  BSR_TRY(cudaMemsetAsync(h->fbits, 0, sizeof(uint32_t) * nb * W, s));
  csr_to_bits_kernel<<<nb, 64, 0, s>>>(row_ptr_dev, col_idx_dev, nb, W, h->fbits);
  rank_kernel<<<nb, 32, 0, s>>>(h->fbits, nb, W, h->frank, nullptr);
  row_counts_kernel<<<nb, 64, 0, s>>>(h->fbits, nb, W, 1, h->counts, nullptr);
  scan_kernel<<<1, 1024, 0, s>>>(h->counts, nb, h->FP.ptr, h->FP.nnz, nullptr);
  fill_pairs_kernel<<<nb, 32, 0, s>>>(h->fbits, nb, W, 1, h->FP, nullptr);
  bsr_scale_pairs_kernel<<<grid_persistent(), NT, 0, s>>>(st, row_ptr_dev, h->fbits, h->frank, vals_dev, W, h->FP,
                                                           h->svals, h->skeep, h->sn2, tau2);
  if (h->rule == SP2_TRUNC_ERROR)
    bsr_errctl_kernel<<<1, kEC, 0, s>>>(nullptr, h->sn2, h->FP.row, h->FP.col, h->FP.nnz,
                                        reinterpret_cast<uint64_t*>(h->spart), h->skeep, tau2);
  else if (h->rule == SP2_TRUNC_MIXED)
    launch_mixctl(nullptr, h->sn2, h->FP.ptr, h->FP.row, h->FP.col, h->FP.nnz, nb, h->tau, h->mixscr, h->skeep,
                  grid_persistent(), s);
  Mat X0 = h->X[0];
  BSR_TRY(cudaMemsetAsync(X0.bits, 0, sizeof(uint32_t) * nb * W, s));
  set_kept_bits_kernel<<<grid_persistent(), 256, 0, s>>>(nullptr, h->FP, h->skeep, W, X0.bits);
  rank_kernel<<<nb, 32, 0, s>>>(X0.bits, nb, W, X0.rank, nullptr);
  row_counts_kernel<<<nb, 64, 0, s>>>(X0.bits, nb, W, 0, h->counts, nullptr);
  scan_kernel<<<1, 1024, 0, s>>>(h->counts, nb, X0.rp, nullptr, nullptr);
  fill_next_kernel<<<grid_persistent(), NT, 0, s>>>(nullptr, h->FP, h->skeep, h->svals, X0, W);
  BSR_TRY(cudaGetLastError());
  // the loop: rounds in pairs (X[0] -> X[1] -> X[0]) until the device-side stop
  BSR_TRY(cudaEventRecord(h->ev[0], s));
  if (h->opts.launch_mode == 0) {
    BSR_TRY(cudaGraphLaunch(h->exec, s));
  } else {
    h->nrounds = 0;
    for (int it = 0; it <= h->opts.max_iter + 1; it += 2) {
      BSR_TRY(add_round(h, nullptr, s, 0, 0));
      BSR_TRY(add_round(h, nullptr, s, 1, 0));
    }
  }
  BSR_TRY(cudaEventRecord(h->ev[1], s));
  if (D_dev) {
    bsr_to_dense_kernel<<<grid_persistent() * 2, 256, 0, s>>>(st, h->X[0], h->X[1], nb, D_dev);
    BSR_TRY(cudaGetLastError());
  }
  BSR_TRY(cudaMemcpyAsync(h->st_host, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  h->last = s;
  h->ran = true;
  return SP2_OK;
}

extern "C" sp2_status sp2_get_info_bsr(sp2_bsr h, sp2_info* out, int64_t* nnzb_out) {
  if (!h || !out) return SP2_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (h->ran) BSR_TRY(cudaStreamSynchronize(h->last));
  const DevState* s = h->st_host;
  out->status = h->ran ? s->status : SP2_OK;
  out->n_iter = s->n_out;
  out->stop_reason = s->reason;
  out->hist_len = s->hist_len;
  out->lambda_min = s->lmin;
  out->lambda_max = s->lmax;
  float ms = 0.f;
  if (h->ran && cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) == cudaSuccess) out->loop_ms = ms;
  (void)cudaGetLastError();
  out->v = s->v;
  out->trace = s->tr;
  out->p = s->p;
  if (nnzb_out) {
    int nz = 0;
    if (h->ran) {
      if (cudaMemcpy(&nz, h->X[s->out_buf].rp + h->nb, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return SP2_ERR_CUDA;
      }
    }
    *nnzb_out = nz;
  }
  return SP2_OK;
}

// ---- test hooks: the index work on its own ----------------------------------------------------
namespace sp2 {
namespace bsr {
__global__ void test_keep_kernel(const float* dense, int nb, double tau2, uint8_t* keep, double* n2_out) {
  __shared__ float blk[B * (B + 1)];
  const int I = blockIdx.x / nb, J = blockIdx.x % nb;
  const int N = nb * B;
  for (int e = threadIdx.x; e < BE; e += blockDim.x)
    blk[(e / B) * (B + 1) + e % B] = dense[(int64_t)(I * B + e / B) * N + J * B + e % B];
  __syncthreads();
  if (threadIdx.x < 32) {
    const double n2 = block_norm2_fixed(blk);
    if (threadIdx.x == 0) {
      keep[blockIdx.x] = (I == J || n2 >= tau2) ? 1 : 0;
      n2_out[blockIdx.x] = n2;
    }
  }
}

// upper pairs (row-major) of an nb x nb block matrix: gather their norms, scatter decisions
__global__ void test_pairs_gather_kernel(const double* n2_full, int nb, const int* row, const int* col, int npairs,
                                         double* n2p) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += gridDim.x * blockDim.x)
    n2p[q] = n2_full[(int64_t)row[q] * nb + col[q]];
}

__global__ void test_pairs_scatter_kernel(const uint8_t* keepp, int nb, const int* row, const int* col, int npairs,
                                          uint8_t* keep) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += gridDim.x * blockDim.x) {
    keep[(int64_t)row[q] * nb + col[q]] = keepp[q];
    keep[(int64_t)col[q] * nb + row[q]] = keepp[q];
  }
}
}  // namespace bsr
}  // namespace sp2

#include <vector>

#include "../../include/sp2_testing.h"

extern "C" int32_t sp2_test_bsr_keep(const float* dense_dev, int64_t N, double tau, int32_t rule, uint8_t* keep_dev,
                                     void* stream) {
  if (!dense_dev || !keep_dev || N < B || N % B || N / B > MAX_NB || !(tau >= 0.0) ||
      (rule != SP2_TRUNC_BLOCK && rule != SP2_TRUNC_ERROR && rule != SP2_TRUNC_MIXED))
    return SP2_ERR_INVALID_ARG;
  const int nb = (int)(N / B);
  cudaStream_t s = (cudaStream_t)stream;
  const int npairs = nb * (nb + 1) / 2;
  std::vector<int> row(npairs), col(npairs);
  for (int I = 0, q = 0; I < nb; ++I)
    for (int J = I; J < nb; ++J, ++q) { row[q] = I; col[q] = J; }
  double *n2_full = nullptr, *n2p = nullptr;
  uint64_t* scratch = nullptr;
  void* mscr = nullptr;
  int *drow = nullptr, *dcol = nullptr, *dnp = nullptr, *dptr = nullptr;
  uint8_t* keepp = nullptr;
  bool ok = cudaMalloc(&n2_full, sizeof(double) * nb * nb) == cudaSuccess &&
            cudaMalloc(&n2p, sizeof(double) * npairs) == cudaSuccess &&
            cudaMalloc(&scratch, sizeof(uint64_t) * npairs) == cudaSuccess &&
            cudaMalloc(&drow, sizeof(int) * npairs) == cudaSuccess &&
            cudaMalloc(&dcol, sizeof(int) * npairs) == cudaSuccess && cudaMalloc(&dnp, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&keepp, npairs) == cudaSuccess && cudaMalloc(&mscr, mixctl_scratch_bytes(nb)) == cudaSuccess &&
            cudaMalloc(&dptr, sizeof(int) * (nb + 1)) == cudaSuccess;
  std::vector<int> ptr(nb + 1, 0);
  for (int I = 0; I < nb; ++I) ptr[I + 1] = ptr[I] + (nb - I);
  if (ok) {
    test_keep_kernel<<<nb * nb, 64, 0, s>>>(dense_dev, nb, tau * tau, keep_dev, n2_full);
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (ok && (rule == SP2_TRUNC_ERROR || rule == SP2_TRUNC_MIXED)) {
    ok = cudaMemcpyAsync(drow, row.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(dcol, col.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(dnp, &npairs, sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(dptr, ptr.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (ok) {
      test_pairs_gather_kernel<<<256, 256, 0, s>>>(n2_full, nb, drow, dcol, npairs, n2p);
      if (rule == SP2_TRUNC_ERROR)
        bsr_errctl_kernel<<<1, kEC, 0, s>>>(nullptr, n2p, drow, dcol, dnp, scratch, keepp, tau * tau);
      else
        launch_mixctl(nullptr, n2p, dptr, drow, dcol, dnp, nb, tau, mscr, keepp, 256, s);
      test_pairs_scatter_kernel<<<256, 256, 0, s>>>(keepp, nb, drow, dcol, npairs, keep_dev);
      ok = cudaGetLastError() == cudaSuccess;
    }
  }
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  cudaFree(n2_full); cudaFree(n2p); cudaFree(scratch); cudaFree(drow); cudaFree(dcol); cudaFree(dnp); cudaFree(keepp);
  cudaFree(mscr); cudaFree(dptr);
  if (!ok) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  return SP2_OK;
}

extern "C" int32_t sp2_test_bsr_square_pattern(const uint8_t* mask_host, int32_t nb, uint8_t* upper_host) {
  if (!mask_host || !upper_host || nb < 1 || nb > MAX_NB) return SP2_ERR_INVALID_ARG;
  const int W = (nb + 31) / 32;
  std::vector<int> rp(nb + 1, 0), ci;
  for (int I = 0; I < nb; ++I) {
    for (int J = 0; J < nb; ++J)
      if (mask_host[(int64_t)I * nb + J]) ci.push_back(J);
    rp[I + 1] = (int)ci.size();
  }
  const int64_t cap_s = (int64_t)nb * (nb + 1) / 2;
  Mat X{};
  Pairs P{};
  uint32_t* sbits = nullptr;
  int* counts = nullptr;
  DevState* st = nullptr;
  bool ok = cudaMalloc(&X.rp, sizeof(int) * (nb + 1)) == cudaSuccess &&
            cudaMalloc(&X.ci, sizeof(int) * (ci.size() + 1)) == cudaSuccess &&
            cudaMalloc(&X.bits, sizeof(uint32_t) * nb * W) == cudaSuccess &&
            cudaMalloc(&X.rank, sizeof(int) * nb * W) == cudaSuccess &&
            cudaMalloc(&P.ptr, sizeof(int) * (nb + 1)) == cudaSuccess &&
            cudaMalloc(&P.col, sizeof(int) * cap_s) == cudaSuccess &&
            cudaMalloc(&P.row, sizeof(int) * cap_s) == cudaSuccess && cudaMalloc(&P.nnz, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&sbits, sizeof(uint32_t) * nb * W) == cudaSuccess &&
            cudaMalloc(&counts, sizeof(int) * nb) == cudaSuccess && cudaMalloc(&st, sizeof(DevState)) == cudaSuccess;
  int nnz = 0;
  std::vector<int> prow, pcol;
  if (ok) {
    DevState d;
    std::memset(&d, 0, sizeof(d));
    ok = cudaMemcpy(st, &d, sizeof(d), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(X.rp, rp.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
         (ci.empty() || cudaMemcpy(X.ci, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice) == cudaSuccess) &&
         cudaMemset(X.bits, 0, sizeof(uint32_t) * nb * W) == cudaSuccess;
  }
  if (ok) {
    csr_to_bits_kernel<<<nb, 64>>>(X.rp, X.ci, nb, W, X.bits);
    rank_kernel<<<nb, 32>>>(X.bits, nb, W, X.rank, nullptr);
    bsr_sym_kernel<<<nb, 64>>>(st, X, nb, W, sbits);
    row_counts_kernel<<<nb, 64>>>(sbits, nb, W, 1, counts, nullptr);
    scan_kernel<<<1, 1024>>>(counts, nb, P.ptr, P.nnz, nullptr);
    fill_pairs_kernel<<<nb, 32>>>(sbits, nb, W, 1, P, nullptr);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
         cudaMemcpy(&nnz, P.nnz, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  if (ok) {
    prow.resize(nnz > 0 ? nnz : 1);
    pcol.resize(nnz > 0 ? nnz : 1);
    ok = nnz == 0 || (cudaMemcpy(prow.data(), P.row, sizeof(int) * nnz, cudaMemcpyDeviceToHost) == cudaSuccess &&
                      cudaMemcpy(pcol.data(), P.col, sizeof(int) * nnz, cudaMemcpyDeviceToHost) == cudaSuccess);
  }
  if (ok) {
    std::memset(upper_host, 0, (size_t)nb * nb);
    for (int q = 0; q < nnz; ++q) upper_host[(int64_t)prow[q] * nb + pcol[q]] = 1;
  }
  cudaFree(X.rp); cudaFree(X.ci); cudaFree(X.bits); cudaFree(X.rank);
  cudaFree(P.ptr); cudaFree(P.col); cudaFree(P.row); cudaFree(P.nnz);
  cudaFree(sbits); cudaFree(counts); cudaFree(st);
  (void)cudaGetLastError();
  return ok ? SP2_OK : SP2_ERR_CUDA;
}
