// Persistent tcgen05 GEMM over piece operands (FMT_BF16X3, FMT_FP16X2 or FMT_TF32X2) with the
// SP2 epilogues, for a batch of problems of uneven size.
//
// C[I-tile, J-tile] = sum_k A[rows I, k] B[rows J, k] (both operands K-major row
// panels; X symmetric makes X X^T = X^2), as the format's piece products.
// One CTA per SM walks the global tile list (the tiles of every instance, largest
// instances first); tiles of instances that have already stopped are skipped.
// Warp 0 feeds a TMA ring (128-byte swizzle, 64-wide k-blocks; 32-wide blocks with 64-byte
// swizzle in twice as many stages ran 18 % slower) from the instance's tensor maps, whose stages
// hold the pieces the job loads (ring_stages: 2 to 6 stages); warp 1 issues the MMAs (128 x 128 x 16) and closes a
// tensor-memory chunk buffer every CHUNK_TERMS k-terms; warps 2-5 add each closed chunk
// into FP32 registers (round to nearest) and, after the last chunk of a tile, run the
// epilogue.  Four chunk buffers let the MMAs run ahead of the draining.
//
// With `upper` set only tiles with J >= I are computed; element (r, c) with c >= r is
// written at (r, c) and, if c > r, at (c, r), so the result is exactly symmetric.
// Every mbarrier wait is bounded (2 s); a wait that gives up sets *err =
// SP2_ERR_TIMEOUT and the kernel winds down, waiting (bounded) for its own copies and
// MMAs before it frees tensor memory.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "../../include/sp2_testing.h"
#include "sp2_kernels.h"
#include "sp2_tc.cuh"
#include "tc_ptx.cuh"

namespace sp2 {
namespace tc {

using namespace sp2::ptx;

constexpr uint64_t kWaitNs = 2000000000ull;
static_assert(BM == BN, "square tiles");

struct Resolved {
  int a[2], b[2], in, out, pk;
  bool active;
  // accelerated path (gen = 1): new = ca C + cb in + cc I (identity on the N true diagonal
  // entries; cc = 0 for derivative steps)
  int gen;
  float ca, cb, cc;
};

// coefficients of step j of the accelerated schedule into R (derivative steps: no c)
__device__ __forceinline__ void acc_coefs(const DevState* st, int j, bool deriv, Resolved& r) {
  double a, b, c;
  r.pk = acc_step(st, j, a, b, c);
  r.gen = 1;
  r.ca = (float)a;
  r.cb = (float)b;
  r.cc = deriv ? 0.f : (float)c;
}

__device__ __forceinline__ Resolved resolve_slots(const Job& j, const Instance& I) {
  Resolved r;
  r.a[0] = j.a_slot[0]; r.a[1] = j.a_slot[1];
  r.b[0] = j.b_slot[0]; r.b[1] = j.b_slot[1];
  r.in = j.a_slot[0]; r.out = j.out_slot; r.pk = 1; r.active = true;
  r.gen = 0; r.ca = r.cb = r.cc = 0.f;
  if (j.rule == SLOTS_FIXED) return r;
  const DevState* st = I.st;
  const bool ok_run = corrects_run(st);   // correction, recompute and refinement jobs
  switch (j.rule) {
    case SLOTS_FORWARD: {
      const int k = st->k;
      r.a[0] = r.b[0] = r.in = xslot(I.lowmem, I.hist0, k);
      r.out = xslot(I.lowmem, I.hist0, k + 1);
      r.pk = st->tr[k] > (double)st->nocc ? 1 : 0;   // Alg. 3 trace test
      if (st->acc) acc_coefs(st, k + 1, false, r);   // Alg. 5: the scheduled polynomial
      r.active = !st->done;
      break;
    }
    case SLOTS_RECOMPUTE: {
      const int jj = st->dk + 1;
      r.a[0] = r.b[0] = r.in = rslot(1, I.hist0, jj - 1);
      r.out = rslot(1, I.hist0, jj);
      r.pk = st->p[jj];
      if (st->acc) acc_coefs(st, jj, false, r);
      r.active = I.lowmem && ok_run && jj < st->n_out;
      break;
    }
    case SLOTS_DERIV: {
      const int jj = st->dk + 1;
      const int xs = rslot(I.lowmem, I.hist0, jj - 1);
      const int di = I.dx0 + ((jj - 1) & 1);
      r.a[0] = xs; r.b[0] = di;
      r.a[1] = di; r.b[1] = xs;
      r.in = di; r.out = I.dx0 + (jj & 1);
      r.pk = st->p[jj];
      if (st->acc) acc_coefs(st, jj, true, r);   // d(a X^2 + b X) = a (X dX + dX X) + b dX
      r.active = ok_run && st->dk < st->n_out;
      break;
    }
    case SLOTS_CORR_M: {
      r.a[0] = xslot(I.lowmem, I.hist0, st->n_out); r.b[0] = I.f_slot; r.out = I.m_slot;
      r.active = ok_run && st->n_out > 0;
      break;
    }
    case SLOTS_CORR_DF: {
      r.a[0] = I.m_slot; r.b[0] = xslot(I.lowmem, I.hist0, st->n_out); r.in = I.m_slot; r.out = I.dx0;
      r.active = ok_run && st->n_out > 0;
      break;
    }
    case SLOTS_REFINE: {
      const int s = j.a_slot[0];
      const int plast = st->p[st->n_out];
      r.a[0] = r.b[0] = r.in = I.r0_slot + s;
      r.out = I.r0_slot + (1 - s);
      r.pk = s == 0 ? 1 - plast : plast;
      r.active = ok_run;
      break;
    }
    default: break;
  }
  return r;
}

// The slots of tile (I, J) of instance I.  Debug builds also check the tile and every slot the
// job's mode touches against the instance (and the history index against the device state's
// arrays); a tile that fails is skipped by every warp role alike.
__device__ __forceinline__ Resolved resolve(const Job& j, const Instance& I, int ti, int tj) {
#if SP2_DEVICE_CHECKS
  // the history indices first: resolve_slots reads the state's arrays at them
  if (j.rule != SLOTS_FIXED &&
      !dcheck(I.st->k >= 0 && I.st->k < SP2_MAX_ITER + 1 && I.st->dk >= 0 && I.st->dk < SP2_MAX_ITER + 1 &&
                  I.st->n_out >= 0 && I.st->n_out < SP2_MAX_ITER + 2, j.err)) {
    Resolved z = {};
    z.active = false;
    return z;
  }
#endif
  Resolved r = resolve_slots(j, I);
#if SP2_DEVICE_CHECKS
  const int ns = I.nslots, T = j.pair ? PT : BM;
  bool ok = ti >= 0 && tj >= 0 && (ti + 1) * T <= I.ld && (tj + 1) * T <= I.ld;
  for (int t = 0; t < j.nterms; ++t) ok = ok && r.a[t] >= 0 && r.a[t] < ns && r.b[t] >= 0 && r.b[t] < ns;
  if (j.mode != MODE_STORE_F32) ok = ok && r.out >= 0 && r.out < ns;
  if (j.mode == MODE_SP2_STEP || j.mode == MODE_DERIV_STEP || j.mode == MODE_DF_COMBINE)
    ok = ok && r.in >= 0 && r.in < ns;
  if (!dcheck(ok, j.err)) r.active = false;
#else
  (void)ti;
  (void)tj;
#endif
  return r;
}

// k-blocks per tensor-memory chunk: CHUNK_TERMS (64 terms) for full products.  (Full fp16 products
// with 128-term chunks ran 7-15 % faster at N = 8192 but raised the error after the correction
// from 6.3e-7 to 9.2e-7, too close to the 1e-6 target.)  Low-precision jobs, whose 16-bit (bf16)
// or 11-bit (fp16) target tolerates a larger bias, take twice (bf16: 3 products per k-step) or
// four times (fp16, tf32: 1) CHUNK_TERMS.  Halved until the chunks divide the k-blocks of a tile.
// The derivative steps (whole_k) take the tile's whole k range in one chunk: they form a
// first-order correction, whose own truncation bias (at most K 2^-25 of dX_j) is far below
// the error it corrects; measured at N = 8192, the error after the correction is the same to
// three digits (5.44e-7) and the derivative pass takes 61 ms instead of 87 ms.
// FMT_TF32X2 counts as fp16 (one low-precision product), in its 32-wide k-blocks.
__device__ __forceinline__ int chunk_kb(const Job& job, int ld) {
  const int bk = bk_of(job.fmt);
  const int total = job.nterms * (ld / bk);
  if (job.whole_k) return total;
  const int terms = !job.lowprec ? CHUNK_TERMS : (job.fmt == FMT_BF16X3 ? 2 * CHUNK_TERMS : 4 * CHUNK_TERMS);
  int ck = terms / bk;
  while (ck > 1 && total % ck != 0) ck >>= 1;
  return ck;
}

// Piece products of one k-step, smallest first: (piece of A, piece of B).  The low-precision
// product is the tail of the list from lp_first.
template <int FMT>
struct Products;
template <>
struct Products<FMT_BF16X3> {
  static constexpr int n = 6, lp_first = 3;
  __device__ static constexpr int a(int q) { return q == 0 ? 2 : (q == 1 || q == 3) ? 1 : 0; }   // 2,1,0,1,0,0
  __device__ static constexpr int b(int q) { return q == 2 ? 2 : (q == 1 || q == 4) ? 1 : 0; }   // 0,1,2,0,1,0
};
template <>
struct Products<FMT_FP16X2> {
  static constexpr int n = 3, lp_first = 2;
  __device__ static constexpr int a(int q) { return q == 0 ? 1 : 0; }                              // 1,0,0
  __device__ static constexpr int b(int q) { return q == 1 ? 1 : 0; }                              // 0,1,0
};
template <>
struct Products<FMT_TF32X2> : Products<FMT_FP16X2> {};   // lo hi', hi lo', hi hi'

template <int FMT>
__host__ __device__ constexpr uint32_t idesc_of(int M, int N) {
  return FMT == FMT_TF32X2 ? idesc_tf32_f32(M, N) : (FMT == FMT_FP16X2 ? idesc_f16_f32(M, N) : idesc_bf16_f32(M, N));
}

// One MMA of the format's kind (kind::tf32 for FMT_TF32X2, kind::f16 otherwise).
template <int FMT, bool PAIR>
__device__ __forceinline__ void mma_fmt(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if constexpr (FMT == FMT_TF32X2) {
    if constexpr (PAIR) mma_tf32_pair(dt, ad, bd, idesc, acc); else mma_tf32(dt, ad, bd, idesc, acc);
  } else {
    if constexpr (PAIR) mma_bf16_pair(dt, ad, bd, idesc, acc); else mma_bf16(dt, ad, bd, idesc, acc);
  }
}

// Pieces loaded per operand by one job.
template <int FMT>
__device__ __forceinline__ int pieces_loaded(const Job& job) {
  return job.lowprec ? (FMT == FMT_BF16X3 ? 2 : 1) : np_of(FMT);
}

__device__ __forceinline__ int tile_off(const Job& job, const Instance& in) {
  if (job.pair) return job.upper ? in.tile_off_upper2 : in.tile_off_full2;
  return job.upper ? in.tile_off_upper : in.tile_off_full;
}

// Global tile t -> (instance, tile row I, tile column J), in units of the launch's tile
// (128 x 128, or 256 x 256 for CTA pairs): row-major within an instance, over the upper
// triangle (J >= I) or all tiles.  A banded walk (column by column within bands of 2..16 tile
// rows, so that co-resident CTAs share B panels in L2) was measured slower at N = 8192
// (1.84-1.93 ms against 1.81 ms per forward square) and is not used.
__device__ __forceinline__ int locate(const Job& job, int t, int& I, int& J) {
  int i = 0;
  for (; i + 1 < job.count; ++i)
    if (t < tile_off(job, job.inst[i + 1])) break;
  const Instance& in = job.inst[i];
  t -= tile_off(job, in);
  const int R = in.ld / (job.pair ? PT : BM);
  if (!job.upper) {
    I = t / R;
    J = t % R;
  } else {
    int r = 0;
    while (t >= R - r) { t -= R - r; ++r; }
    I = r;
    J = r + t;
  }
  return i;
}

// 8 consecutive values (16-byte aligned) from / to the planes of a slot.
template <int FMT>
__device__ __forceinline__ void load8(const __nv_bfloat16* slot, int64_t plane, int64_t off, float (&x)[8]) {
  if constexpr (FMT == FMT_TF32X2) {   // 32-byte aligned: off is a multiple of 8 values
    const float4* hi = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(slot) + off);
    const float4* lo = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(slot) + plane + off);
    const float4 h0 = hi[0], h1 = hi[1], l0 = lo[0], l1 = lo[1];
    x[0] = h0.x + l0.x; x[1] = h0.y + l0.y; x[2] = h0.z + l0.z; x[3] = h0.w + l0.w;
    x[4] = h1.x + l1.x; x[5] = h1.y + l1.y; x[6] = h1.z + l1.z; x[7] = h1.w + l1.w;
  } else if constexpr (FMT == FMT_FP16X2) {
    const uint4 a = *reinterpret_cast<const uint4*>(slot + off);
    const uint4 b = *reinterpret_cast<const uint4*>(slot + plane + off);
    const __half* pa = reinterpret_cast<const __half*>(&a);
    const __half* pb = reinterpret_cast<const __half*>(&b);
    #pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = (__half2float(pa[e]) + __half2float(pb[e])) * kF16InvScale;
  } else {
    const uint4 a = *reinterpret_cast<const uint4*>(slot + off);
    const uint4 b = *reinterpret_cast<const uint4*>(slot + plane + off);
    const uint4 c = *reinterpret_cast<const uint4*>(slot + 2 * plane + off);
    const __nv_bfloat16* pa = reinterpret_cast<const __nv_bfloat16*>(&a);
    const __nv_bfloat16* pb = reinterpret_cast<const __nv_bfloat16*>(&b);
    const __nv_bfloat16* pc = reinterpret_cast<const __nv_bfloat16*>(&c);
    #pragma unroll
    for (int e = 0; e < 8; ++e)
      x[e] = (__bfloat162float(pa[e]) + __bfloat162float(pb[e])) + __bfloat162float(pc[e]);
  }
}

template <int FMT>
__device__ __forceinline__ void store8(__nv_bfloat16* slot, int64_t plane, int64_t off, const float (&x)[8]) {
  if constexpr (FMT == FMT_TF32X2) {
    float h[8], l[8];
    #pragma unroll
    for (int e = 0; e < 8; ++e) split_tf32x2(x[e], h[e], l[e]);
    float4* hi = reinterpret_cast<float4*>(reinterpret_cast<float*>(slot) + off);
    float4* lo = reinterpret_cast<float4*>(reinterpret_cast<float*>(slot) + plane + off);
    hi[0] = make_float4(h[0], h[1], h[2], h[3]);
    hi[1] = make_float4(h[4], h[5], h[6], h[7]);
    lo[0] = make_float4(l[0], l[1], l[2], l[3]);
    lo[1] = make_float4(l[4], l[5], l[6], l[7]);
  } else if constexpr (FMT == FMT_FP16X2) {
    uint4 a, b;
    __half* pa = reinterpret_cast<__half*>(&a);
    __half* pb = reinterpret_cast<__half*>(&b);
    #pragma unroll
    for (int e = 0; e < 8; ++e) split_fp16x2(x[e], pa[e], pb[e]);
    *reinterpret_cast<uint4*>(slot + off) = a;
    *reinterpret_cast<uint4*>(slot + plane + off) = b;
  } else {
    uint4 a, b, c;
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(&a);
    __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(&b);
    __nv_bfloat16* pc = reinterpret_cast<__nv_bfloat16*>(&c);
    #pragma unroll
    for (int e = 0; e < 8; ++e) split_bf16x3(x[e], pa[e], pb[e], pc[e]);
    *reinterpret_cast<uint4*>(slot + off) = a;
    *reinterpret_cast<uint4*>(slot + plane + off) = b;
    *reinterpret_cast<uint4*>(slot + 2 * plane + off) = c;
  }
}

struct Partials {
  double v2;    // sum of w (x - c)^2   (w = 2 off the diagonal, 1 on it)
  double fro2;  // sum of w x^2
  double trd;   // sum of the diagonal x
};

// Epilogue for row r, columns c0 .. c0+31 of the tile, with the accumulated product s
// (FMT_FP16X2: S^2 times the product, removed here); worked in groups of 8 columns (one
// 16-byte access per plane).  The Frobenius partials of the 32 columns are summed in FP32 in
// column order, then added to P in FP64.
template <int FMT>
__device__ __forceinline__ void epilogue_chunk(const Job& job, const Instance& In, const Resolved& R, int r,
                                               int c0, const float (&s_raw)[32], Partials& P) {
  const int ld = In.ld;
  const int64_t plane = (int64_t)ld * ld;
  const bool upper = job.upper != 0;
  if (upper && c0 + 31 < r) return;
  const int64_t row_off = (int64_t)r * ld + c0;
  float s[32];
  #pragma unroll
  for (int j = 0; j < 32; ++j) s[j] = FMT == FMT_FP16X2 ? s_raw[j] * kF16InvScale2 : s_raw[j];

  if (job.mode == MODE_STORE_F32) {
    const bool all_keep = !upper || c0 >= r;
    #pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = c0 + j;
      if (all_keep || c >= r) job.out32[row_off + j] = s[j];
      if (upper && c > r) job.out32[(int64_t)c * ld + r] = s[j];
    }
    return;
  }

  __nv_bfloat16* out = In.arena + (int64_t)R.out * In.slot_elems;
  const __nv_bfloat16* in = In.arena + (int64_t)R.in * In.slot_elems;
  float vacc = 0.f, facc = 0.f;
  #pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int cb = c0 + 8 * h;
    if (upper && cb + 7 < r) continue;
    float xn[8];
    if (job.mode == MODE_STORE_PIECES) {
      #pragma unroll
      for (int j = 0; j < 8; ++j) xn[j] = s[8 * h + j];
    } else {
      float x[8];
      load8<FMT>(in, plane, row_off + 8 * h, x);
      if (job.mode == MODE_DF_COMBINE) {
        // dX_0 = -dF / (lmax - lmin): the F slot holds F (FMT_BF16X3, FMT_TF32X2), or F' =
        // (F - c I) / W' with c, W' the centre and half-width of [lmin, lmax] (FMT_FP16X2),
        // whose dF' is dF / W'
        const double w = In.st->lmax - In.st->lmin;
        const float sc = FMT == FMT_FP16X2 ? -0.5f : (float)(-1.0 / w);
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t toff = (int64_t)(cb + j) * ld + r;
          const float mt = piece_load(FMT, in, plane, toff);
          xn[j] = sc * ((x[j] + mt) - 2.0f * s[8 * h + j]);
        }
      } else {
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float sj = s[8 * h + j];
          if (R.gen) {
            const float id = (cb + j == r && r < In.st->N) ? R.cc : 0.f;
            xn[j] = fmaf(R.ca, sj, fmaf(R.cb, x[j], id));
          } else {
            xn[j] = R.pk ? sj : fmaf(2.0f, x[j], -sj);
          }
          if (job.mode == MODE_SP2_STEP) {
            const int c = cb + j;
            const float d = x[j] - sj;
            const float wgt = !upper ? 1.f : (c > r ? 2.f : (c == r ? 1.f : 0.f));
            vacc = fmaf(wgt * d, d, vacc);
            facc = fmaf(wgt * x[j], x[j], facc);
            if (c == r) P.trd += (double)x[j];
          }
        }
      }
    }
    if (!upper || cb >= r) {
      store8<FMT>(out, plane, row_off + 8 * h, xn);
    } else {
      #pragma unroll
      for (int j = 0; j < 8; ++j)
        if (cb + j >= r) piece_store(FMT, out, plane, row_off + 8 * h + j, xn[j]);
    }
    if (upper) {
      #pragma unroll
      for (int j = 0; j < 8; ++j)
        if (cb + j > r) piece_store(FMT, out, plane, (int64_t)(cb + j) * ld + r, xn[j]);
    }
  }
  if (job.mode == MODE_SP2_STEP) {
    P.v2 += (double)vacc;
    P.fro2 += (double)facc;
  }
}

template <int FMT>
__global__ void __launch_bounds__(THREADS, 1) tc_gemm_kernel(const Job job) {
  // the job's ring: stages of the pieces it loads (ring_stages in sp2_tc.cuh)
  const int npl = pieces_loaded<FMT>(job);
  const int stg = ring_stages(npl), sbytes = ring_stage_bytes(npl);
  using PR = Products<FMT>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t accf_bar[NBUF];
  __shared__ __align__(8) uint64_t acce_bar[NBUF];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wait_ns = job.wait_ms > 0 ? (uint64_t)job.wait_ms * 1000000ull : kWaitNs;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAX_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < NBUF; ++a) { mbar_init(&accf_bar[a], 1); mbar_init(&acce_bar[a], 4); }
    mbar_init(&drain_bar, 1);
    abort_s = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base_s, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_s;
  const int ntiles = job.total_tiles;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int armed[MAX_STAGES];
      uint32_t armed_par[MAX_STAGES];
      for (int s = 0; s < MAX_STAGES; ++s) { armed[s] = 0; armed_par[s] = 0; }
      bool skip_first = job.test_skip != 0 && blockIdx.x == 0;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int I, J;
        const int ii = locate(job, t, I, J);
        const Instance& In = job.inst[ii];
        const Resolved R = resolve(job, In, I, J);
        if (!R.active) continue;
        const CUtensorMap* mA = &In.mapA;
        const CUtensorMap* mB = &In.mapB;
        const int nkb = In.ld / bk_of(FMT);
        for (int term = 0; term < job.nterms && ok; ++term) {
          for (int kb = 0; kb < nkb; ++kb) {
            if (abort_s || !mbar_wait(&empty_bar[stage], phase ^ 1, globaltimer_ns() + wait_ns)) {
              ok = false;
              break;
            }
            if (skip_first) {   // testing hook: this stage stays unarmed, the MMA thread's wait gives up
              skip_first = false;
              armed[stage] = 0;
              if (++stage == stg) { stage = 0; phase ^= 1; }
              continue;
            }
            uint8_t* sA = smem + stage * sbytes;
            uint8_t* sB = sA + npl * A_PIECE_BYTES;
            mbar_arrive_expect_tx(&full_bar[stage], npl * (A_PIECE_BYTES + B_PIECE_BYTES));
            for (int p = 0; p < npl; ++p)
              tma_load_4d(sA + p * A_PIECE_BYTES, mA, kb * bk_of(FMT), I * BM, p, R.a[term], &full_bar[stage]);
            for (int p = 0; p < npl; ++p)
              tma_load_4d(sB + p * B_PIECE_BYTES, mB, kb * bk_of(FMT), J * BN, p, R.b[term], &full_bar[stage]);
            armed[stage] = 1;
            armed_par[stage] = phase;
            if (++stage == stg) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (!ok) { abort_s = 1; atomicExch(job.err, (int)SP2_ERR_TIMEOUT); }
      // wait (bounded) until every copy issued here has landed
      for (int s = 0; s < stg; ++s)
        if (armed[s]) mbar_wait(&full_bar[s], armed_par[s], globaltimer_ns() + wait_ns);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_of<FMT>(BM, BN);
      // the format's piece products, smallest first; low-precision jobs take the tail
      const int q0 = job.lowprec ? PR::lp_first : 0;
      int stage = 0, buf = 0;
      uint32_t phase = 0, bphase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int I, J;
        const int ii = locate(job, t, I, J);
        const Instance& In = job.inst[ii];
        if (!resolve(job, In, I, J).active) continue;
        const int nchunks = job.nterms * (In.ld / bk_of(FMT)) / chunk_kb(job, In.ld);
        for (int ch = 0; ch < nchunks && ok; ++ch) {
          const uint32_t dt = tmem_base + (uint32_t)(buf * BN);
          uint32_t accumulate = 0;
          for (int kc = 0; kc < chunk_kb(job, In.ld); ++kc) {
            // the ring stage first, then (on the chunk's first stage) the free chunk buffer, as in
            // the pair kernel (2-3 % faster here at N = 8192)
            if (abort_s || !mbar_wait(&full_bar[stage], phase, globaltimer_ns() + wait_ns) ||
                (kc == 0 && !mbar_wait(&acce_bar[buf], bphase ^ 1, globaltimer_ns() + wait_ns))) { ok = false; break; }
            tc_fence_after();
            const uint32_t sA = smem_u32(smem + stage * sbytes);
            const uint32_t sB = sA + npl * A_PIECE_BYTES;
            // the stage's smaller piece products first, then the leading one (p0 q0, the last)
            #pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
              #pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk) {
                #pragma unroll
                for (int q = 0; q < PR::n; ++q) {
                  if (q < q0 || (q == PR::n - 1) != (pass == 1)) continue;
                  const uint64_t ad = smem_desc_sw128(sA + PR::a(q) * A_PIECE_BYTES + kk * 32);
                  const uint64_t bd = smem_desc_sw128(sB + PR::b(q) * B_PIECE_BYTES + kk * 32);
                  mma_fmt<FMT, false>(dt, ad, bd, idesc, accumulate);
                  accumulate = 1;
                }
              }
            }
            mma_commit(&empty_bar[stage]);
            if (++stage == stg) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&accf_bar[buf]);
          if (++buf == NBUF) { buf = 0; bphase ^= 1; }
        }
      }
      if (!ok) { abort_s = 1; atomicExch(job.err, (int)SP2_ERR_TIMEOUT); }
      mma_commit(&drain_bar);
      mbar_wait(&drain_bar, 0, globaltimer_ns() + wait_ns);
    }
  } else {
    // ---------------- chunk draining + epilogue (warps 2..5) ----------------
    const int q = warp & 3;      // TMEM lanes 32q .. 32q+31
    int buf = 0;
    uint32_t bphase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int I, J;
      const int ii = locate(job, t, I, J);
      const Instance& In = job.inst[ii];
      const Resolved R = resolve(job, In, I, J);
      if (!R.active) continue;
      const int nchunks = job.nterms * (In.ld / bk_of(FMT)) / chunk_kb(job, In.ld);
      float acc[BN / 32][32];
      #pragma unroll
      for (int g = 0; g < BN / 32; ++g)
        #pragma unroll
        for (int j = 0; j < 32; ++j) acc[g][j] = 0.f;
      for (int ch = 0; ch < nchunks; ++ch) {
        int got = 0;
        if (lane == 0) got = !abort_s && mbar_wait(&accf_bar[buf], bphase, globaltimer_ns() + wait_ns);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          if (lane == 0) { abort_s = 1; atomicExch(job.err, (int)SP2_ERR_TIMEOUT); }
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t trow = tmem_base + (uint32_t)(buf * BN) + ((uint32_t)(32 * q) << 16);
        #pragma unroll
        for (int g = 0; g < BN / 32; ++g) {
          uint32_t raw[32];
          tmem_ld32(trow + g * 32, raw);
          tmem_wait_ld();
          #pragma unroll
          for (int j = 0; j < 32; ++j) acc[g][j] += __uint_as_float(raw[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[buf]);
        if (++buf == NBUF) { buf = 0; bphase ^= 1; }
      }
      if (!ok) break;
      const int r = I * BM + 32 * q + lane;
      Partials P = {0.0, 0.0, 0.0};
      #pragma unroll
      for (int g = 0; g < BN / 32; ++g) epilogue_chunk<FMT>(job, In, R, r, J * BN + g * 32, acc[g], P);
      if (job.mode == MODE_SP2_STEP) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          P.v2 += __shfl_xor_sync(0xffffffffu, P.v2, o);
          P.fro2 += __shfl_xor_sync(0xffffffffu, P.fro2, o);
          P.trd += __shfl_xor_sync(0xffffffffu, P.trd, o);
        }
        if (lane == 0) {
          const int lt = t - In.tile_off_upper;        // tile index within the instance
          double* dst = In.part + 4 * (4 * (int64_t)lt + q);
          dst[0] = P.v2;
          dst[1] = P.fro2;
          dst[2] = P.trd;
          dst[3] = 0.0;
        }
      }
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---- CTA-pair kernel ------------------------------------------------------------------------
// The same product and epilogues on 256 x 256 tiles, one tile per cluster of two CTAs
// (even CTA: rows 0..127 of the tile, odd CTA: rows 128..255).  Each CTA's TMA warp
// stages its own 128 rows of A and of B (B rows are the output columns: the even CTA
// holds columns 0..127, the odd one 128..255) and counts the bytes on the even CTA's
// `full` barrier, which the even CTA arms for both.  The even CTA's MMA thread issues
// 256 x 256 x 16 pair MMAs and multicasts each commit to both CTAs (`empty` stage
// barriers, `accf` chunk barriers); every epilogue warp of both CTAs arrives on the even
// CTA's `acce` barrier once it has drained a chunk buffer.  Every poll of a barrier is a
// CTA-scope try_wait: what a phase orders is either counted by the barrier itself (TMA bytes,
// MMA commits) or tensor memory, which the tcgen05 fences around the remote arrive order; the
// cluster-scope acquire form cost 3 % of the run at N = 8192 in memory-barrier stalls.  For the
// same reason the epilogue warps hand a drained chunk buffer back with a relaxed arrive (its
// tensor-memory reads are complete): 4 % off the forward square against the release form.
constexpr int P_SMEM_BYTES = STAGES * STAGE_BYTES + 8192 + 1024;   // + alignment and read slack

template <int FMT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P_THREADS, 1) tc_gemm_pair_kernel(const Job job) {
  // the job's ring: stages of the pieces it loads (ring_stages in sp2_tc.cuh)
  const int npl = pieces_loaded<FMT>(job);
  const int stg = ring_stages(npl), sbytes = ring_stage_bytes(npl);
  using PR = Products<FMT>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t accf_bar[P_NBUF];
  __shared__ __align__(8) uint64_t acce_bar[P_NBUF];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wait_ns = job.wait_ms > 0 ? (uint64_t)job.wait_ms * 1000000ull : kWaitNs;
  const uint32_t rank = cluster_ctarank();
  const int pair_id = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAX_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < P_NBUF; ++a) { mbar_init(&accf_bar[a], 1); mbar_init(&acce_bar[a], 2 * P_EPI_WARPS); }
    mbar_init(&drain_bar, 1);
    abort_s = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(&tmem_base_s, P_NBUF * PT);
  tc_fence_before();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_s;
  const int ntiles = job.total_tiles;
  if (warp < 4) {
   setmaxnreg_dec<P_REG_CTRL>();
   if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int armed[MAX_STAGES];
      uint32_t armed_par[MAX_STAGES];
      for (int s = 0; s < MAX_STAGES; ++s) { armed[s] = 0; armed_par[s] = 0; }
      for (int t = pair_id; t < ntiles && ok; t += npairs) {
        int I, J;
        const int ii = locate(job, t, I, J);
        const Instance& In = job.inst[ii];
        const Resolved R = resolve(job, In, I, J);
        if (!R.active) continue;
        const CUtensorMap* mA = &In.mapA;
        const CUtensorMap* mB = &In.mapB;
        const int nkb = In.ld / bk_of(FMT);
        const int rowA = I * PT + (int)rank * BM;
        const int rowB = J * PT + (int)rank * BN;
        for (int term = 0; term < job.nterms && ok; ++term) {
          for (int kb = 0; kb < nkb; ++kb) {
            if (abort_s || !mbar_wait(&empty_bar[stage], phase ^ 1, globaltimer_ns() + wait_ns)) {
              ok = false;
              break;
            }
            uint8_t* sA = smem + stage * sbytes;
            uint8_t* sB = sA + npl * A_PIECE_BYTES;
            const uint32_t fb = mapa_shared(smem_u32(&full_bar[stage]), 0);
            if (rank == 0) mbar_arrive_expect_tx(&full_bar[stage], 2 * npl * (A_PIECE_BYTES + B_PIECE_BYTES));
            for (int p = 0; p < npl; ++p)
              tma_load_4d_pair(sA + p * A_PIECE_BYTES, mA, kb * bk_of(FMT), rowA, p, R.a[term], fb);
            for (int p = 0; p < npl; ++p)
              tma_load_4d_pair(sB + p * B_PIECE_BYTES, mB, kb * bk_of(FMT), rowB, p, R.b[term], fb);
            armed[stage] = 1;
            armed_par[stage] = phase;
            if (++stage == stg) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (!ok) {
        abort_s = 1;
        atomicExch(job.err, (int)SP2_ERR_TIMEOUT);
        // copies of the odd CTA complete on the even CTA's barriers, which it cannot
        // observe: give copies still in flight a fixed 1 ms to land
        const uint64_t until = globaltimer_ns() + 1000000ull;
        while (globaltimer_ns() < until) {}
      }
      if (rank == 0)
        for (int s = 0; s < stg; ++s)
          if (armed[s]) mbar_wait(&full_bar[s], armed_par[s], globaltimer_ns() + wait_ns);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (even CTA) ----------------
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc = idesc_of<FMT>(2 * BM, PT);
      const int q0 = job.lowprec ? PR::lp_first : 0;
      int stage = 0, buf = 0;
      uint32_t phase = 0, bphase = 0;
      bool ok = true;
      for (int t = pair_id; t < ntiles && ok; t += npairs) {
        int I, J;
        const int ii = locate(job, t, I, J);
        const Instance& In = job.inst[ii];
        if (!resolve(job, In, I, J).active) continue;
        const int ckb = chunk_kb(job, In.ld);
        const int nchunks = job.nterms * (In.ld / bk_of(FMT)) / ckb;
        for (int ch = 0; ch < nchunks && ok; ++ch) {
          const uint32_t dt = tmem_base + (uint32_t)(buf * PT);
          uint32_t accumulate = 0;
          for (int kc = 0; kc < ckb; ++kc) {
            // the ring stage first, then (on the chunk's first stage) the free chunk buffer: at
            // N = 8192 the forward square took 1.51 ms with the chunk buffer waited for first
            // and 1.32 ms in this order, the same products bit for bit
            if (abort_s || !mbar_wait(&full_bar[stage], phase, globaltimer_ns() + wait_ns) ||
                (kc == 0 && !mbar_wait(&acce_bar[buf], bphase ^ 1, globaltimer_ns() + wait_ns))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sA = smem_u32(smem + stage * sbytes);
            const uint32_t sB = sA + npl * A_PIECE_BYTES;
            // the stage's smaller piece products first, then the leading one (p0 q0, the last)
            #pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
              #pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk) {
                #pragma unroll
                for (int q = 0; q < PR::n; ++q) {
                  if (q < q0 || (q == PR::n - 1) != (pass == 1)) continue;
                  const uint64_t ad = smem_desc_sw128(sA + PR::a(q) * A_PIECE_BYTES + kk * 32);
                  const uint64_t bd = smem_desc_sw128(sB + PR::b(q) * B_PIECE_BYTES + kk * 32);
                  mma_fmt<FMT, true>(dt, ad, bd, idesc, accumulate);
                  accumulate = 1;
                }
              }
            }
            mma_commit_pair_mc(&empty_bar[stage], 0x3);
            if (++stage == stg) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit_pair_mc(&accf_bar[buf], 0x3);
          if (++buf == P_NBUF) { buf = 0; bphase ^= 1; }
        }
      }
      if (!ok) { abort_s = 1; atomicExch(job.err, (int)SP2_ERR_TIMEOUT); }
      mma_commit_pair_mc(&drain_bar, 0x1);
      mbar_wait(&drain_bar, 0, globaltimer_ns() + wait_ns);
    }
   }
  } else {
    setmaxnreg_inc<P_REG_EPI>();
    // ---------------- chunk draining + epilogue (warps 4..11 of both CTAs) ----------------
    const int ew = warp - 4;       // 0..7
    const int q = warp & 3;        // TMEM lanes 32q .. 32q+31 (the quadrant this warp may access)
    const int hc = ew >> 2;        // columns 128 hc .. 128 hc + 127 of the tile
    int buf = 0;
    uint32_t bphase = 0;
    bool ok = true;
    for (int t = pair_id; t < ntiles && ok; t += npairs) {
      int I, J;
      const int ii = locate(job, t, I, J);
      const Instance& In = job.inst[ii];
      const Resolved R = resolve(job, In, I, J);
      if (!R.active) continue;
      const int nchunks = job.nterms * (In.ld / bk_of(FMT)) / chunk_kb(job, In.ld);
      float acc[BN / 32][32];
      #pragma unroll
      for (int g = 0; g < BN / 32; ++g)
        #pragma unroll
        for (int j = 0; j < 32; ++j) acc[g][j] = 0.f;
      for (int ch = 0; ch < nchunks; ++ch) {
        int got = 0;
        if (lane == 0) got = !abort_s && mbar_wait(&accf_bar[buf], bphase, globaltimer_ns() + wait_ns);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          if (lane == 0) { abort_s = 1; atomicExch(job.err, (int)SP2_ERR_TIMEOUT); }
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t trow = tmem_base + (uint32_t)(buf * PT + hc * BN) + ((uint32_t)(32 * q) << 16);
        #pragma unroll
        for (int g = 0; g < BN / 32; ++g) {
          uint32_t raw[32];
          tmem_ld32(trow + g * 32, raw);
          tmem_wait_ld();
          #pragma unroll
          for (int j = 0; j < 32; ++j) acc[g][j] += __uint_as_float(raw[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster_relaxed(mapa_shared(smem_u32(&acce_bar[buf]), 0));
        if (++buf == P_NBUF) { buf = 0; bphase ^= 1; }
      }
      if (!ok) break;
      const int r = I * PT + (int)rank * BM + 32 * q + lane;
      Partials P = {0.0, 0.0, 0.0};
      #pragma unroll
      for (int g = 0; g < BN / 32; ++g) epilogue_chunk<FMT>(job, In, R, r, J * PT + hc * BN + g * 32, acc[g], P);
      if (job.mode == MODE_SP2_STEP) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          P.v2 += __shfl_xor_sync(0xffffffffu, P.v2, o);
          P.fro2 += __shfl_xor_sync(0xffffffffu, P.fro2, o);
          P.trd += __shfl_xor_sync(0xffffffffu, P.trd, o);
        }
        if (lane == 0) {
          const int lt = t - In.tile_off_upper2;       // pair tile index within the instance
          double* dst = In.part + 4 * (2 * P_EPI_WARPS * (int64_t)lt + P_EPI_WARPS * rank + ew);
          dst[0] = P.v2;
          dst[1] = P.fro2;
          dst[2] = P.trd;
          dst[3] = 0.0;
        }
      }
    }
  }

  // both CTAs stay resident until the pair's MMAs, copies and drains are over
  __syncwarp();
  tc_fence_before();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, P_NBUF * PT);
  }
}

}  // namespace tc

// ---- host side ----------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

cudaError_t tc_make_maps(void* arena, int ld, int nslots, int fmt, CUtensorMap* mapA, CUtensorMap* mapB) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  if (ld % tc::LD_ALIGN != 0 || (reinterpret_cast<uintptr_t>(arena) & 15) != 0) return cudaErrorInvalidValue;
  const int np = tc::np_of(fmt);
  const cuuint64_t es = (cuuint64_t)tc::esize_of(fmt);
  const CUtensorMapDataType dt = fmt == tc::FMT_TF32X2   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : fmt == tc::FMT_FP16X2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[4] = {(cuuint64_t)ld, (cuuint64_t)ld, (cuuint64_t)np, (cuuint64_t)nslots};
  cuuint64_t strides[3] = {(cuuint64_t)ld * es, (cuuint64_t)ld * ld * es, (cuuint64_t)np * ld * ld * es};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t bk = (cuuint32_t)tc::bk_of(fmt);   // 128-byte rows in every format
  cuuint32_t boxA[4] = {bk, (cuuint32_t)tc::BM, 1, 1};
  cuuint32_t boxB[4] = {bk, (cuuint32_t)tc::BN, 1, 1};
  CUresult r1 = enc(mapA, dt, 4, arena, dims, strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(mapB, dt, 4, arena, dims, strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// The kernel instance for a job: tile kind x piece format.
static void* kernel_of(int pair, int fmt) {
  if (pair) return fmt == tc::FMT_TF32X2   ? (void*)tc::tc_gemm_pair_kernel<tc::FMT_TF32X2>
                   : fmt == tc::FMT_FP16X2 ? (void*)tc::tc_gemm_pair_kernel<tc::FMT_FP16X2>
                                           : (void*)tc::tc_gemm_pair_kernel<tc::FMT_BF16X3>;
  return fmt == tc::FMT_TF32X2   ? (void*)tc::tc_gemm_kernel<tc::FMT_TF32X2>
         : fmt == tc::FMT_FP16X2 ? (void*)tc::tc_gemm_kernel<tc::FMT_FP16X2>
                                 : (void*)tc::tc_gemm_kernel<tc::FMT_BF16X3>;
}

static cudaError_t tc_prepare() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int pair = 0; pair < 2 && e == cudaSuccess; ++pair)
    for (int fmt = 0; fmt < 3 && e == cudaSuccess; ++fmt)
      e = cudaFuncSetAttribute(kernel_of(pair, fmt), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               pair ? tc::P_SMEM_BYTES : tc::SMEM_BYTES);
  if (e == cudaSuccess) done = true;
  return e;
}

// Clusters of two that fit on the GPU at once (one CTA per SM); 0 if the query fails.
static int pair_slots() {
  static int n = -1;
  if (n < 0) {
    if (tc_prepare() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * sm_count());
    cfg.blockDim = dim3(tc::P_THREADS);
    cfg.dynamicSmemBytes = tc::P_SMEM_BYTES;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, kernel_of(1, tc::FMT_BF16X3), &cfg) != cudaSuccess || c <= 0) {
      (void)cudaGetLastError();
      c = sm_count() / 2;
    }
    n = c;
  }
  return n;
}

// Persistent grid: one CTA (or one CTA pair) per tile up to what the GPU holds at once.
int tc_grid_for(int total_tiles, int pair) {
  const int t = total_tiles < 1 ? 1 : total_tiles;
  if (pair) {
    const int slots = pair_slots() > 0 ? pair_slots() : 1;
    return 2 * (t < slots ? t : slots);
  }
  const int s = sm_count();
  return t < s ? t : s;
}

int tc_tiles(int ld, int upper, int pair) { return pair ? tc::pair_tiles_of(ld, upper) : tc::tiles_of(ld, upper); }

cudaError_t tc_launch(const tc::Job& job, cudaStream_t s) {
  cudaError_t e = tc_prepare();
  if (e != cudaSuccess) return e;
  if (job.pair) {
    const dim3 g(tc_grid_for(job.total_tiles, 1));
    if (job.fmt == tc::FMT_TF32X2) tc::tc_gemm_pair_kernel<tc::FMT_TF32X2><<<g, tc::P_THREADS, tc::P_SMEM_BYTES, s>>>(job);
    else if (job.fmt == tc::FMT_FP16X2) tc::tc_gemm_pair_kernel<tc::FMT_FP16X2><<<g, tc::P_THREADS, tc::P_SMEM_BYTES, s>>>(job);
    else tc::tc_gemm_pair_kernel<tc::FMT_BF16X3><<<g, tc::P_THREADS, tc::P_SMEM_BYTES, s>>>(job);
  } else {
    const dim3 g(tc_grid_for(job.total_tiles, 0));
    if (job.fmt == tc::FMT_TF32X2) tc::tc_gemm_kernel<tc::FMT_TF32X2><<<g, tc::THREADS, tc::SMEM_BYTES, s>>>(job);
    else if (job.fmt == tc::FMT_FP16X2) tc::tc_gemm_kernel<tc::FMT_FP16X2><<<g, tc::THREADS, tc::SMEM_BYTES, s>>>(job);
    else tc::tc_gemm_kernel<tc::FMT_BF16X3><<<g, tc::THREADS, tc::SMEM_BYTES, s>>>(job);
  }
  return cudaGetLastError();
}

cudaError_t tc_add_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, const tc::Job& job,
                        cudaGraphNode_t* node) {
  cudaError_t e = tc_prepare();
  if (e != cudaSuccess) return e;
  tc::Job j = job;
  void* args[] = {&j};
  cudaKernelNodeParams kp = {};
  kp.func = kernel_of(job.pair, job.fmt);
  kp.gridDim = dim3(tc_grid_for(job.total_tiles, job.pair));
  kp.blockDim = dim3(job.pair ? tc::P_THREADS : tc::THREADS);
  kp.sharedMemBytes = job.pair ? tc::P_SMEM_BYTES : tc::SMEM_BYTES;
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

}  // namespace sp2

extern "C" int32_t sp2_test_tc_gemm(const void* arena_dev, int32_t ld, int32_t nslots, int32_t a_slot,
                                    int32_t b_slot, int32_t upper, int32_t tile, float* out_dev, void* stream) {
  return sp2_test_tc_gemm_ex(arena_dev, ld, nslots, a_slot, b_slot, upper, tile, 0, 0, out_dev, stream);
}

// Shared by the product test entries: one launch of the product of slots a and b, status back.
static int32_t run_test_product(const void* arena_dev, int32_t ld, int32_t nslots, int32_t a_slot, int32_t b_slot,
                                int32_t upper, int pair, int32_t fmt, int32_t lowprec, int32_t wait_ms,
                                int32_t test_skip, float* out_dev, cudaStream_t s);

extern "C" int32_t sp2_test_tc_timeout(const void* arena_dev, int32_t ld, int32_t wait_ms, float* out_dev,
                                       void* stream) {
  if (!arena_dev || !out_dev || ld <= 0 || ld % sp2::tc::LD_ALIGN != 0 || wait_ms < 1 || wait_ms > 2000)
    return SP2_ERR_INVALID_ARG;
  return run_test_product(arena_dev, ld, 1, 0, 0, 0, 0, 0, 0, wait_ms, 1, out_dev, (cudaStream_t)stream);
}

extern "C" int32_t sp2_build_device_checks(void) { return SP2_DEVICE_CHECKS ? 1 : 0; }

extern "C" int32_t sp2_test_tc_bounds(const void* arena_dev, int32_t ld, int32_t nslots, int32_t bad_slot,
                                      float* out_dev, void* stream) {
  if (!arena_dev || !out_dev || ld <= 0 || ld % sp2::tc::LD_ALIGN != 0 || nslots <= 0 || bad_slot < nslots ||
      bad_slot >= nslots + 1024)
    return SP2_ERR_INVALID_ARG;
  if (!SP2_DEVICE_CHECKS) return SP2_ERR_UNSUPPORTED;
  return run_test_product(arena_dev, ld, nslots, bad_slot, 0, 0, 0, 0, 0, 0, 0, out_dev, (cudaStream_t)stream);
}

extern "C" int32_t sp2_test_tc_gemm_ex(const void* arena_dev, int32_t ld, int32_t nslots, int32_t a_slot,
                                       int32_t b_slot, int32_t upper, int32_t tile, int32_t fmt, int32_t lowprec,
                                       float* out_dev, void* stream) {
  if (!arena_dev || !out_dev || ld <= 0 || ld % sp2::tc::LD_ALIGN != 0 || nslots <= 0 || a_slot < 0 ||
      b_slot < 0 || a_slot >= nslots || b_slot >= nslots || (upper != 0 && upper != 1) || tile < 0 || tile > 2 ||
      (tile == 2 && ld % sp2::tc::PT != 0) || fmt < 0 || fmt > 2 || (lowprec != 0 && lowprec != 1))
    return SP2_ERR_INVALID_ARG;
  const int pair = tile == 2 || (tile == 0 && ld % sp2::tc::PT == 0);
  return run_test_product(arena_dev, ld, nslots, a_slot, b_slot, upper, pair, fmt, lowprec, 0, 0, out_dev,
                          (cudaStream_t)stream);
}

static int32_t run_test_product(const void* arena_dev, int32_t ld, int32_t nslots, int32_t a_slot, int32_t b_slot,
                                int32_t upper, int pair, int32_t fmt, int32_t lowprec, int32_t wait_ms,
                                int32_t test_skip, float* out_dev, cudaStream_t s) {
  sp2::tc::Instance hinst;
  std::memset(&hinst, 0, sizeof(hinst));
  if (sp2::tc_make_maps(const_cast<void*>(arena_dev), ld, nslots, fmt, &hinst.mapA, &hinst.mapB) != cudaSuccess) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  hinst.arena = (__nv_bfloat16*)const_cast<void*>(arena_dev);
  hinst.fmt = fmt;
  hinst.np = sp2::tc::np_of(fmt);
  hinst.nslots = nslots;
  hinst.slot_elems = sp2::tc::slot_units_of(fmt, ld);
  hinst.ld = ld;
  // device copies of the instance record and the error word (test entry point only)
  sp2::tc::Instance* dinst = nullptr;
  int32_t* err = nullptr;
  if (cudaMallocAsync((void**)&dinst, sizeof(hinst), s) != cudaSuccess ||
      cudaMallocAsync((void**)&err, sizeof(int32_t), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return SP2_ERR_NOMEM;
  }
  int32_t herr = 0;
  sp2::tc::Job j;
  std::memset(&j, 0, sizeof(j));
  j.mode = sp2::tc::MODE_STORE_F32;
  j.upper = upper;
  j.nterms = 1;
  j.rule = sp2::tc::SLOTS_FIXED;
  j.count = 1;
  j.pair = pair;
  j.fmt = fmt;
  j.lowprec = lowprec;
  j.wait_ms = wait_ms;
  j.test_skip = test_skip;
  j.total_tiles = sp2::tc_tiles(ld, upper, pair);
  j.inst = dinst;
  j.a_slot[0] = a_slot;
  j.b_slot[0] = b_slot;
  j.out32 = out_dev;
  j.err = err;
  bool ok = cudaMemcpyAsync(dinst, &hinst, sizeof(hinst), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemsetAsync(err, 0, sizeof(int32_t), s) == cudaSuccess && sp2::tc_launch(j, s) == cudaSuccess &&
            cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaFreeAsync(err, s) == cudaSuccess && cudaFreeAsync(dinst, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  return herr;
}
