// Tensor-core block products of the block-truncated expansion: the numeric square of one round
// (S = X~_{k-1}^2 on the upper pairs of its pattern, the SP2 epilogue, the per-pair partials of
// ||X~_{k-1} - S||_F^2 and Tr[X_k], the fixed-order block norms and the keep flags of the
// per-block truncation rule), on tcgen05 tensor cores.
//
// The square is cut into tiles of 4 block rows x 8 block columns (M = 128, N = 256); a tile is
// computed when it holds at least one upper pair of the square's pattern.  For tile (I0, J0),
// S[I0.., J0..] = sum over K of X[I0.., K] X[J0.., K]^T (X symmetric), the sum over the K blocks
// that one of the tile's 4 rows and one of its 8 columns both hold; a block a row lacks is the
// all-zero block.  Each iterate keeps, beside its FP32 blocks, every block as two fp16 pieces of
// 2^14 x (the FMT_FP16X2 format of the dense path), so a K block is 12 TMA boxes of 32 x 32 per
// piece into one ring stage, and a tile's product is the three piece products p0 q0 + p0 q1 +
// p1 q0 per 16-wide k-step, accumulated in tensor memory in chunks of 4 K blocks (24 truncating
// FP32 additions, as on the dense path) and added into registers with round-to-nearest additions.
//
// Warp roles (one CTA per SM, persistent over the tile list): warp 0 finds the K blocks (OR of the
// tile rows' bitmap words, AND of the two ORs) and the 12 block positions of each from the words'
// popcounts, and issues the TMA copies; warp 1 issues the MMAs; warps 4..11 drain the chunks (two
// warps per tensor-memory lane quadrant = block row, 128 columns = 4 blocks each) and run the
// epilogue of the tile's pairs.  Every wait is bounded (2 s); a wait that gives up records
// SP2_ERR_TIMEOUT in the run's state, ends the run and winds the kernel down.
#include <cudaTypedefs.h>

#include <cstring>

#include "../../include/sp2.h"
#include "sp2_bsr.cuh"
#include "sp2_tc.cuh"
#include "tc_ptx.cuh"

namespace sp2 {
namespace bsr {

using namespace sp2::ptx;

constexpr int TSTG = 4;                            // ring stages, one K block each
constexpr int PIECE_BYTES = B * B * 2;             // one 32 x 32 fp16 piece
constexpr int A_PLANE = TTR * PIECE_BYTES;         // the 128 rows of one piece of A
constexpr int B_PLANE = TTC * PIECE_BYTES;         // the 256 rows of one piece of B
constexpr int TSTAGE = 2 * (A_PLANE + B_PLANE);    // 48 KB
constexpr int TSMEM = TSTG * TSTAGE + 1024;        // + alignment slack
constexpr int TCHK = 4;                            // K blocks per tensor-memory chunk
constexpr int TN = TTC * B;                        // 256 accumulator columns per chunk buffer
constexpr int TTHREADS = 384;                      // warpgroup 0: TMA, MMA, 2 idle; 8 epilogue warps
constexpr int T_REG_CTRL = 40, T_REG_EPI = 232;    // 40 + 2 x 232 <= 3 x 168 launch registers
constexpr uint64_t kTcWaitNs = 2000000000ull;
static_assert(T_REG_CTRL + 2 * T_REG_EPI <= 3 * 168, "register split exceeds the launch budget");
static_assert(2 * TN <= 512, "tensor memory columns");

__device__ __forceinline__ void tc_give_up(DevState* st, volatile int* abort_s) {
  *abort_s = 1;
  atomicExch(&st->status, (int)SP2_ERR_TIMEOUT);
  st->out_mode = OUT_NAN;
  st->done = 1;
}

constexpr int TMAXW = 64;                          // bitmap words per row (nb <= 2048)

struct TcArgs {
  DevState* st;
  Mat X;
  const TcMaps* maps;
  int parity;
  int nb, W, ncg;                                  // ncg: column groups of 8 blocks
  int zero_blk;                                    // index of the all-zero block
  int64_t pair_cap;                                // capacity of the square's pair arrays
  TcRound r;
};

__global__ void __launch_bounds__(TTHREADS, 1) bsr_tc_kernel(const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TSTG];
  __shared__ __align__(8) uint64_t empty_bar[TSTG];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ uint32_t rbits_s[TTR + TTC][TMAXW];     // producer: the tile rows' bitmap words
  __shared__ int rrank_s[TTR + TTC][TMAXW];          // and their rank-table entries

  DevState* st = a.st;
  if (!st->iter_active) return;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = *a.r.tnnz;
  const Mat& X = a.X;
  const int nb = a.nb, W = a.W;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTG; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf_bar[b], 1); mbar_init(&acce_bar[b], 8); }
    mbar_init(&drain_bar, 1);
    abort_s = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base_s, 2 * TN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_s;

  if (warp < 4) {
    setmaxnreg_dec<T_REG_CTRL>();
    if (warp == 0) {
      // ---------------- K-block discovery + TMA producer ----------------
      const CUtensorMap* map = &a.maps->map[a.parity];
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int armed[TSTG];
      uint32_t armed_par[TSTG];
      for (int s = 0; s < TSTG; ++s) { armed[s] = 0; armed_par[s] = 0; }
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int code = a.r.tiles[t];
        const int I0 = (code / a.ncg) * TTR, J0 = (code % a.ncg) * TTC;
        const int rowj = lane < TTR ? I0 + lane : J0 + (lane - TTR);
        const bool vj = lane < TTR + TTC && rowj < nb;
        const int rpj = vj ? X.rp[rowj] : 0;
        // the 12 rows' bitmap words and ranks, all loads in flight at once
        __syncwarp();
        for (int e = lane; e < (TTR + TTC) * W; e += 32) {
          const int j = e / W, w = e % W;
          const int row = j < TTR ? I0 + j : J0 + (j - TTR);
          const bool v = row < nb;
          rbits_s[j][w] = v ? X.bits[(int64_t)row * W + w] : 0u;
          rrank_s[j][w] = v ? X.rank[(int64_t)row * W + w] : 0;
        }
        __syncwarp();
        for (int w = 0; w < W && ok; ++w) {
          const uint32_t bj = lane < TTR + TTC ? rbits_s[lane][w] : 0u;
          const int rkj = lane < TTR + TTC ? rrank_s[lane][w] : 0;
          const uint32_t am = __reduce_or_sync(0xffffffffu, lane < TTR ? bj : 0u);
          const uint32_t bm = __reduce_or_sync(0xffffffffu, lane >= TTR && lane < TTR + TTC ? bj : 0u);
          uint32_t m = am & bm;
          while (m && ok) {
            const int bit = __ffs(m) - 1;
            m &= m - 1u;
            const bool has = vj && ((bj >> bit) & 1u);
            int posj = has ? rpj + rkj + __popc(bj & ((1u << bit) - 1u)) : a.zero_blk;
            if (!dcheck(posj >= 0 && posj <= a.zero_blk, &st->status)) posj = a.zero_blk;
            int go = 1;
            if (lane == 0) go = !abort_s && mbar_wait(&empty_bar[stage], phase ^ 1, globaltimer_ns() + kTcWaitNs);
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) {
              ok = false;
              break;
            }
            // lane j < 12 copies its own block's two pieces: row j of A (j < 4) or row j - 4 of B;
            // the expected bytes are armed first, so no copy can complete the phase early
            if (lane == 0) {
              mbar_arrive_expect_tx(&full_bar[stage], TSTAGE);
              armed[stage] = 1;
              armed_par[stage] = phase;
            }
            __syncwarp();
            if (lane < TTR + TTC) {
              uint8_t* dst = smem + stage * TSTAGE +
                             (lane < TTR ? lane * PIECE_BYTES : 2 * A_PLANE + (lane - TTR) * PIECE_BYTES);
              const int plane = lane < TTR ? A_PLANE : B_PLANE;
              tma_load_3d(dst, map, 0, 0, 2 * posj, &full_bar[stage]);
              tma_load_3d(dst + plane, map, 0, 0, 2 * posj + 1, &full_bar[stage]);
            }
            if (++stage == TSTG) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (lane == 0) {
        if (!ok) tc_give_up(st, &abort_s);
        for (int s = 0; s < TSTG; ++s)   // wait (bounded) until every copy issued here has landed
          if (armed[s]) mbar_wait(&full_bar[s], armed_par[s], globaltimer_ns() + kTcWaitNs);
      }
    } else if (warp == 1) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = idesc_f16_f32(TTR * B, TN);
      int stage = 0, buf = 0;
      uint32_t phase = 0, bphase = 0;
      bool ok = true;
      unsigned long long kblocks = 0ull, needed = 0ull;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int nk = a.r.meta[(int64_t)t * TMETA];
        kblocks += (unsigned long long)nk;
        needed += (unsigned long long)a.r.meta[(int64_t)t * TMETA + 65];
        if (lane == 0) {
          for (int k0 = 0; k0 < nk && ok; k0 += TCHK) {
            if (abort_s || !mbar_wait(&acce_bar[buf], bphase ^ 1, globaltimer_ns() + kTcWaitNs)) { ok = false; break; }
            tc_fence_after();
            const uint32_t dt = tmem_base + (uint32_t)(buf * TN);
            uint32_t accumulate = 0;
            const int kend = min(nk, k0 + TCHK);
            for (int k = k0; k < kend; ++k) {
              if (abort_s || !mbar_wait(&full_bar[stage], phase, globaltimer_ns() + kTcWaitNs)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sA = smem_u32(smem + stage * TSTAGE);
              const uint32_t sB = sA + 2 * A_PLANE;
              #pragma unroll
              for (int kk = 0; kk < B / 16; ++kk) {
                // p1 q0 and p0 q1 of the whole K block first, then p0 q0: the small products are
                // added while the accumulator is still small
                mma_bf16(dt, smem_desc_sw64(sA + 1 * A_PLANE + kk * 32), smem_desc_sw64(sB + kk * 32), idesc,
                         accumulate);
                accumulate = 1;
                mma_bf16(dt, smem_desc_sw64(sA + kk * 32), smem_desc_sw64(sB + 1 * B_PLANE + kk * 32), idesc, 1);
              }
              #pragma unroll
              for (int kk = 0; kk < B / 16; ++kk)
                mma_bf16(dt, smem_desc_sw64(sA + kk * 32), smem_desc_sw64(sB + kk * 32), idesc, 1);
              mma_commit(&empty_bar[stage]);
              if (++stage == TSTG) { stage = 0; phase ^= 1; }
            }
            if (!ok) break;
            mma_commit(&accf_bar[buf]);
            if (++buf == 2) { buf = 0; bphase ^= 1; }
          }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (lane == 0) {
        // executed 32 x 32 x 32 block products: the tile's 32 block pairs times its K blocks
        atomicAdd(&st->bprod, kblocks * (unsigned long long)(TTR * TTC));
        atomicAdd(&st->uprod, needed);   // the tiles' needed products (tile metadata)
        if (!ok) tc_give_up(st, &abort_s);
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0, globaltimer_ns() + kTcWaitNs);
      }
    }
  } else {
    setmaxnreg_inc<T_REG_EPI>();
    // ---------------- chunk draining + epilogue (warps 4..11) ----------------
    const int ew = warp - 4;
    const int q = warp & 3;        // tensor-memory lanes 32 q .. 32 q + 31 = block row q of the tile
    const int hc = ew >> 2;        // columns 128 hc .. 128 hc + 127 = block columns 4 hc .. 4 hc + 3
    const int kprev = st->k;
    double ca = 0.0, cb = 0.0, cc = 0.0;
    const int gen = st->acc;
    const int pk = gen ? acc_step(st, kprev + 1, ca, cb, cc) : (st->tr[kprev] > (double)st->nocc ? 1 : 0);
    const float fa = (float)ca, fb = (float)cb, fc = (float)cc;
    int buf = 0;
    uint32_t bphase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int code = a.r.tiles[t];
      const int I0 = (code / a.ncg) * TTR, J0 = (code % a.ncg) * TTC;
      const int* meta = a.r.meta + (int64_t)t * TMETA;
      const int nk = meta[0];
      int qis[4], pos[4];
      #pragma unroll
      for (int g = 0; g < 4; ++g) {
        qis[g] = meta[1 + TTC * q + 4 * hc + g];
        pos[g] = meta[33 + TTC * q + 4 * hc + g];
      }
      float acc[4][32];
      #pragma unroll
      for (int g = 0; g < 4; ++g)
        #pragma unroll
        for (int j = 0; j < 32; ++j) acc[g][j] = 0.f;
      for (int k0 = 0; k0 < nk; k0 += TCHK) {
        int got = 0;
        if (lane == 0) got = !abort_s && mbar_wait(&accf_bar[buf], bphase, globaltimer_ns() + kTcWaitNs);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          if (lane == 0) tc_give_up(st, &abort_s);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t trow = tmem_base + (uint32_t)(buf * TN + hc * 128) + ((uint32_t)(32 * q) << 16);
        #pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t raw[32];
          tmem_ld32(trow + g * 32, raw);
          tmem_wait_ld();
          #pragma unroll
          for (int j = 0; j < 32; ++j) acc[g][j] += __uint_as_float(raw[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[buf]);
        if (++buf == 2) { buf = 0; bphase ^= 1; }
      }
      if (!ok) break;
      // epilogue of the tile's upper pairs in this warp's four blocks; lane = row of the block
      const int I = I0 + q;
      #pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int J = J0 + 4 * hc + g;
        const int qi = qis[g];               // -1: not an upper pair of the square's pattern
        if (qi < 0 || !dcheck(qi < a.pair_cap, &st->status)) continue;
        int po = pos[g];
        if (po >= 0 && !dcheck(po < a.zero_blk, &st->status)) po = -1;
        float old[32];
        if (po >= 0) {
          const float4* src = reinterpret_cast<const float4*>(X.vals + (int64_t)po * BE + lane * B);
          #pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float4 o4 = src[v];
            old[4 * v] = o4.x; old[4 * v + 1] = o4.y; old[4 * v + 2] = o4.z; old[4 * v + 3] = o4.w;
          }
        } else {
          #pragma unroll
          for (int j = 0; j < 32; ++j) old[j] = 0.f;
        }
        float sv32[32];
        #pragma unroll
        for (int j = 0; j < 32; ++j) sv32[j] = acc[g][j] * tc::kF16InvScale2;
        float4* dst = reinterpret_cast<float4*>(a.r.svals + (int64_t)qi * BE + lane * B);
        if (I == J) {
          // a diagonal block of the square: the tensor cores sum (r, c) and (c, r) in different
          // orders, so the upper triangle is mirrored (staged through the pair's output block)
          #pragma unroll
          for (int v = 0; v < 8; ++v)
            dst[v] = make_float4(sv32[4 * v], sv32[4 * v + 1], sv32[4 * v + 2], sv32[4 * v + 3]);
          __syncwarp();
          const float* blk = a.r.svals + (int64_t)qi * BE;
          #pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < lane) sv32[j] = blk[j * B + lane];
          __syncwarp();
        }
        float vloc = 0.f;
        double trloc = 0.0, rs = 0.0;
        float nwv[32];
        #pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float sv = sv32[j];
          nwv[j] = gen ? fmaf(fa, sv, fmaf(fb, old[j], (I == J && lane == j) ? fc : 0.f))
                       : (pk ? sv : fmaf(2.0f, old[j], -sv));
          const float d = old[j] - sv;
          vloc = fmaf(d, d, vloc);
          if (I == J && lane == j) trloc += (double)nwv[j];
          const double x = (double)nwv[j];
          rs = __dadd_rn(rs, __dmul_rn(x, x));          // row `lane`, left to right
        }
        #pragma unroll
        for (int v = 0; v < 8; ++v) dst[v] = make_float4(nwv[4 * v], nwv[4 * v + 1], nwv[4 * v + 2], nwv[4 * v + 3]);
        double n2 = 0.0;                                  // then the rows top to bottom
        for (int rr = 0; rr < 32; ++rr) n2 = __dadd_rn(n2, __shfl_sync(0xffffffffu, rs, rr));
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          vloc += __shfl_xor_sync(0xffffffffu, vloc, o);
          trloc += __shfl_xor_sync(0xffffffffu, trloc, o);
        }
        if (lane == 0) {
          a.r.spart[2 * (int64_t)qi] = (I == J ? 1.0 : 2.0) * (double)vloc;
          a.r.spart[2 * (int64_t)qi + 1] = trloc;
          a.r.skeep[qi] = (I == J || n2 >= a.r.tau2) ? 1 : 0;
          a.r.sn2[qi] = n2;
        }
      }
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * TN);
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

cudaError_t tc_piece_map(const __half* pvals, int64_t cap, CUtensorMap* map) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(pvals) & 15) != 0) return cudaErrorInvalidValue;
  // (column, row, piece block): piece p of block q is plane 2 q + p
  cuuint64_t dims[3] = {(cuuint64_t)B, (cuuint64_t)B, (cuuint64_t)(2 * (cap + 1))};
  cuuint64_t strides[2] = {(cuuint64_t)B * 2, (cuuint64_t)B * B * 2};
  cuuint32_t box[3] = {(cuuint32_t)B, (cuuint32_t)B, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(pvals), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int tc_grid() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    if (cudaFuncSetAttribute(bsr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM) != cudaSuccess)
      (void)cudaGetLastError();
  }
  return n;
}

void tc_prepare() { (void)tc_grid(); }

cudaError_t tc_numeric_launch(DevState* st, const Mat& X, const TcMaps* maps, int parity, int nb, int W,
                              const TcRound& r, cudaStream_t s) {
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.st = st;
  a.X = X;
  a.maps = maps;
  a.parity = parity;
  a.nb = nb;
  a.W = W;
  a.ncg = (nb + TTC - 1) / TTC;
  a.zero_blk = nb * nb;
  a.pair_cap = (int64_t)nb * (nb + 1) / 2;
  a.r = r;
  bsr_tc_kernel<<<tc_grid(), TTHREADS, TSMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bsr
}  // namespace sp2
