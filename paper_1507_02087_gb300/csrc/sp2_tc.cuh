// Tensor-core (tcgen05) path: definitions shared by the GEMM kernel, the batched
// elementwise kernels and the host side.
//
// Matrices on this path are FP32 values stored as "pieces", in one of three formats:
//  * FMT_BF16X3: three bf16 pieces x = (p0 + p1) + p2 (p0 = bf16(x), p1 = bf16(x - p0),
//    p2 = x - p0 - p1; each difference is exact in FP32 and the last one fits in bf16),
//    so the FP32 value is stored exactly.  A full product X Y^T is the sum of the six
//    piece products p_a q_b with a + b <= 2 (FP32-accurate); a low-precision product
//    takes the three with a + b <= 1 (about 16 significant bits).
//  * FMT_FP16X2: two fp16 pieces of the scaled value S x, S = 2^14 (p0 = fp16(S x),
//    p1 = fp16(S x - p0)): 22 significant bits, and fp16's exponent range holds every
//    |x| < 4 (the iterates have |x| <= 1).  A full product is the three piece products
//    p0 q0 + p0 q1 + p1 q0 (relative error about 2^-21); a low-precision product is p0 q0
//    alone (11 bits).  Each piece product is exact in FP32, the accumulated sum carries
//    S^2, which the epilogue removes.
//  * FMT_TF32X2: two tf32 pieces stored as FP32 values, hi = tf32(x) (round to nearest) and
//    lo = tf32(x - hi): 22 significant bits like FMT_FP16X2, with FP32's exponent range (no
//    scaling).  A full product is the three piece products hi lo' + lo hi' + hi hi' (relative
//    error about 2^-21); a low-precision product is hi hi' (11 bits).
// The 16-bit formats run as kind::f16 MMAs (fp16 and bf16 inputs at the same tensor-core rate),
// FMT_TF32X2 as kind::tf32 MMAs (half that rate, K = 8 per MMA), all with FP32 accumulation.
//
// Every problem ("instance") owns a piece arena: slot s holds the planes of one ld x ld
// matrix, plane-major ([slot][piece][row][col]; 16-bit or, for FMT_TF32X2, 32-bit elements; the
// arena is addressed in 16-bit units).  A 4-D TMA tensor map (col, row,
// piece, slot) per instance covers its arena, so a kernel selects operands by instance and
// slot.  A launch works on the tiles of all live instances of a batch (a single problem is
// a batch of one).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "sp2_common.cuh"

namespace sp2 {
namespace tc {

// Piece formats (sp2_tc.cuh header comment).
enum Fmt : int32_t { FMT_BF16X3 = 0, FMT_FP16X2 = 1, FMT_TF32X2 = 2 };
constexpr float kF16Scale = 16384.f;                 // S = 2^14
constexpr float kF16InvScale = 1.f / 16384.f;
constexpr float kF16InvScale2 = 1.f / (16384.f * 16384.f);

constexpr int BM = 128;          // tile rows (MMA M)
constexpr int BN = 128;          // tile cols (MMA N)
constexpr int BK = 64;           // k-block of the 16-bit formats: 64 values = 128 B rows, 128-byte swizzle
constexpr int ROW_BYTES = 128;   // one k-block row of any format (FMT_TF32X2: 32 values)
constexpr int KSTEPS = 4;        // MMAs per k-block row and product: 32 B each (16 16-bit or 8 tf32 values)
constexpr int NP = 3;            // pieces per matrix (FMT_BF16X3; the two-piece formats have 2)
constexpr int STAGES = 2;        // ring of full FMT_BF16X3 products (its bytes bound every job's ring: ring_stages)
__host__ __device__ constexpr int np_of(int fmt) { return fmt == FMT_BF16X3 ? 3 : 2; }
__host__ __device__ constexpr int stages_of(int fmt) { return fmt == FMT_BF16X3 ? 2 : 3; }
__host__ __device__ constexpr int esize_of(int fmt) { return fmt == FMT_TF32X2 ? 4 : 2; }   // bytes per value
__host__ __device__ constexpr int bk_of(int fmt) { return ROW_BYTES / esize_of(fmt); }    // values per k-block
// 16-bit units of one slot (np planes of ld x ld values)
__host__ __device__ constexpr int64_t slot_units_of(int fmt, int64_t ld) {
  return (int64_t)np_of(fmt) * ld * ld * (esize_of(fmt) / 2);
}
// The tensor cores' FP32 accumulation drops the bits an addend loses in alignment
// (it rounds toward zero), so a long sum of same-sign products drifts low by about
// K * 2^-25 of its value.  The MMAs therefore accumulate a chunk of k-terms (CHUNK_TERMS,
// 64 terms, for full products; see chunk_kb for the others) at a time into one of the
// tensor-memory buffers, and the epilogue adds the chunk sums into registers with
// round-to-nearest FP32 additions.  Within a ring stage the smaller piece products are
// issued before the leading one (p0 q0), so that they are added while the accumulator is
// still small and lose less to the truncation.
constexpr int CHUNK_TERMS = 64;  // one 16-bit k-block, two FMT_TF32X2 k-blocks
constexpr int NBUF = 4;
constexpr int A_PIECE_BYTES = BM * ROW_BYTES;
constexpr int B_PIECE_BYTES = BN * ROW_BYTES;
constexpr int STAGE_BYTES = NP * (A_PIECE_BYTES + B_PIECE_BYTES);
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;   // + alignment slack
__host__ __device__ constexpr int stage_bytes_of(int fmt) { return np_of(fmt) * (A_PIECE_BYTES + B_PIECE_BYTES); }
static_assert(stages_of(FMT_FP16X2) * stage_bytes_of(FMT_FP16X2) == STAGES * STAGE_BYTES,
              "both formats use the same shared-memory ring size");
// Ring geometry of one job: a stage holds the pieces the job loads of each operand (npl: all of
// them for full products, fewer for low-precision ones), and the ring takes as many such stages
// as fit in its bytes, up to MAX_STAGES (full products: 2 bf16 or 3 fp16 / tf32 stages; one-piece
// low-precision products: 6).
constexpr int MAX_STAGES = 6;
__host__ __device__ constexpr int ring_stage_bytes(int npl) { return npl * (A_PIECE_BYTES + B_PIECE_BYTES); }
__host__ __device__ constexpr int ring_stages(int npl) {
  return STAGES * STAGE_BYTES / ring_stage_bytes(npl) < MAX_STAGES ? STAGES * STAGE_BYTES / ring_stage_bytes(npl)
                                                                   : MAX_STAGES;
}
static_assert(ring_stages(1) == MAX_STAGES && ring_stages(2) == 3 && ring_stages(3) == 2, "ring geometry");
constexpr int THREADS = 192;     // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
constexpr int TMEM_COLS = NBUF * BN;   // four 128 x 128 fp32 chunk accumulators
constexpr int LD_ALIGN = 128;    // ld is a multiple of the tile size
constexpr int MAX_BATCH = 256;   // instances per batch

// CTA-pair tiles (cluster of two SMs, tcgen05 cta_group::2): the pair computes a 256 x 256
// output tile with 256 x 256 x 16 MMAs issued by the even CTA.  Each CTA stages its own
// 128 rows of A and its own 128 rows of B (half of the N dimension), so shared memory
// carries half the bytes per flop of a 128 x 128 tile; each CTA's tensor memory holds
// its 128 rows x 256 columns in two chunk buffers, drained by eight epilogue warps
// (two per lane quadrant, 128 columns each).  Three warpgroups: the first holds the TMA
// and MMA warps and gives registers back (P_REG_CTRL), the other two are the epilogue
// and take them (P_REG_EPI); 3 x 168 launch registers = P_REG_CTRL + 2 P_REG_EPI.
constexpr int PT = 256;              // pair tile edge
constexpr int P_NBUF = 2;
constexpr int P_EPI_WARPS = 8;
constexpr int P_THREADS = 128 + 32 * P_EPI_WARPS;  // warpgroup 0: TMA, MMA, two idle warps
constexpr int P_REG_LAUNCH = 168;    // 65536 / 384, rounded down to a multiple of 8
constexpr int P_REG_CTRL = 40;
constexpr int P_REG_EPI = 232;
static_assert(P_NBUF * PT <= 512, "tensor memory columns");
static_assert(P_REG_CTRL + 2 * P_REG_EPI <= 3 * P_REG_LAUNCH, "register split exceeds the launch budget");
static_assert(P_REG_LAUNCH * P_THREADS <= 65536, "launch registers");

enum Mode : int32_t {
  MODE_STORE_F32 = 0,   // C -> fp32 buffer (tests)
  MODE_SP2_STEP = 1,    // X_k = C or 2 X_{k-1} - C, with ||X_{k-1} - C||_F^2, ||X_{k-1}||_F^2 and
                        // Tr X_{k-1} partials
  MODE_DERIV_STEP = 2,  // dX_j = C or 2 dX_{j-1} - C (also one plain SP2 step with C = in^2)
  MODE_STORE_PIECES = 3,// C -> pieces (full tiles)
  MODE_DF_COMBINE = 4   // dX_0 = s (M + M^T - 2 C) with s = -1/(lmax - lmin)
};

// Where the operands come from.  Slot indices are computed from the instance's device
// state, so one captured launch serves every iteration of a loop.
enum SlotRule : int32_t {
  SLOTS_FIXED = 0,      // a_slot / b_slot / out as given (tests)
  SLOTS_FORWARD = 1,    // A = B = in = hist0 + k, out = hist0 + k + 1      (k = st->k)
  SLOTS_DERIV = 2,      // j = st->dk + 1: (X_{j-1}, dX_{j-1}) + (dX_{j-1}, X_{j-1}) -> dX_j
  SLOTS_CORR_M = 3,     // M = P F with P = X_n:  A = hist0 + n, B = f_slot, out = m_slot
  SLOTS_CORR_DF = 4,    // W = M P:  A = m_slot, B = hist0 + n, in = m_slot, out = dx0
  SLOTS_REFINE = 5,     // purification step s = a_slot[0] on the corrected D: s = 0 maps
                        // r0_slot -> r0_slot + 1 with the polynomial other than p_n, s = 1
                        // maps back with p_n (an alternating pair, §4)
  SLOTS_RECOMPUTE = 6   // low-memory instances: X_j = p_j(X_{j-1}) again during the
                        // derivative pass (j = st->dk + 1), into a two-slot ring
};

// Slot of the forward iterate X_k.  Full history: hist0 + k.  Low memory: X_0 in slot 0,
// X_k (k >= 1) alternating in slots 1 and 2; the derivative pass recomputes the iterates
// into slots 3 and 4 (X_0 from slot 0).
__host__ __device__ __forceinline__ int xslot(int lowmem, int hist0, int k) {
  return lowmem ? (k == 0 ? 0 : 1 + (k & 1)) : hist0 + k;
}
__host__ __device__ __forceinline__ int rslot(int lowmem, int hist0, int j) {
  return lowmem ? (j == 0 ? 0 : 3 + (j & 1)) : hist0 + j;
}

// One problem of a batch (device memory; the tensor maps are read by TMA from here and
// keep the alignment CUtensorMap requires).
struct Instance {
  CUtensorMap mapA;     // box 64 x 128 (A operand; k innermost)
  CUtensorMap mapB;     // box 64 x 128 (B operand)
  __nv_bfloat16* arena;
  int64_t slot_elems;   // 3 * ld * ld
  DevState* st;
  double* part;         // forward-square partials: 4 doubles per (tile, epilogue warp)
  int32_t ld;
  int32_t tile_off_upper;   // first global tile index of this instance (upper schedule)
  int32_t tile_off_full;    // first global tile index (full schedule)
  int32_t hist0, dx0, m_slot, f_slot, r0_slot;
  int32_t lowmem;           // 1: iterates in rings, recomputed in the derivative pass
  int32_t tile_off_upper2;  // first global pair-tile index (upper schedule)
  int32_t tile_off_full2;   // first global pair-tile index (full schedule)
  int32_t nparts;           // forward-square partial records (4 doubles each) per launch
  int32_t rec_pair;         // 1: the records come from CTA-pair tiles (16 per 256 x 256 tile)
  double* mscr;             // mixed-norm scratch ((ld/128)^2 + 2 ld/128 doubles), or null
  int32_t fmt;              // Fmt of the arena
  int32_t np;               // pieces (planes) per slot: np_of(fmt)
  int32_t nslots;           // slots of the arena (the tensor maps' outermost extent)
};

struct Job {
  int32_t mode;
  int32_t upper;        // 1: symmetric result from upper tiles, mirror written
  int32_t nterms;       // 1 or 2 (sum of two products, same accumulator)
  int32_t rule;
  int32_t count;        // instances in the batch
  int32_t total_tiles;  // over all instances, for this schedule
  const Instance* inst;
  int32_t a_slot[2], b_slot[2];   // SLOTS_FIXED operands; SLOTS_REFINE step in a_slot[0]
  int32_t out_slot;
  int32_t pair;         // 1: 256 x 256 CTA-pair tiles (every instance's ld a multiple of 256)
  int32_t lowprec;      // 1: the low-precision product of the format (FMT_BF16X3: pieces 0 and 1,
                        // the three products with a + b <= 1, about 16 bits; FMT_FP16X2: p0 q0,
                        // 11 bits); the derivative pass, and every product of SP2_PREC_BF16X3
  int32_t fmt;          // Fmt of every instance of the batch
  int32_t wait_ms;      // limit of every mbarrier wait in ms (0: the default, 2 s)
  int32_t whole_k;      // 1: one tensor-memory chunk per tile, the whole k range (derivative steps)
  int32_t test_skip;    // testing hook (128 x 128 kernel): 1 = CTA 0 leaves its first ring stage
                        // unarmed, so that the waits on it give up (see sp2_test_tc_timeout)
  float* out32;         // MODE_STORE_F32
  int32_t* err;         // set to SP2_ERR_TIMEOUT if a wait gave up
};

// ---- pieces of one value -------------------------------------------------------------------
// `slot` points at plane 0 of a slot, planes `plane` elements apart.
__device__ __forceinline__ void split_bf16x3(float x, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
  p0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ void split_fp16x2(float x, __half& p0, __half& p1) {
  const float y = x * kF16Scale;                  // exact: a power of two
  p0 = __float2half_rn(y);
  p1 = __float2half_rn(y - __half2float(p0));     // the difference is exact in FP32
}

// The tf32 value nearest x (ties away from zero), as an FP32 value with the low 13 bits zero.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_tf32x2(float x, float& hi, float& lo) {
  hi = round_tf32(x);
  lo = round_tf32(x - hi);                        // the difference is exact in FP32
}

__device__ __forceinline__ float piece_load(int fmt, const __nv_bfloat16* slot, int64_t plane, int64_t off) {
  if (fmt == FMT_TF32X2) {
    const float* f = reinterpret_cast<const float*>(slot);
    return f[off] + f[plane + off];               // exact: 22 significant bits in all
  }
  if (fmt == FMT_FP16X2) {
    const __half* h = reinterpret_cast<const __half*>(slot);
    return (__half2float(h[off]) + __half2float(h[plane + off])) * kF16InvScale;   // exact sum
  }
  return (__bfloat162float(slot[off]) + __bfloat162float(slot[plane + off])) + __bfloat162float(slot[2 * plane + off]);
}

__device__ __forceinline__ void piece_store(int fmt, __nv_bfloat16* slot, int64_t plane, int64_t off, float x) {
  if (fmt == FMT_TF32X2) {
    float* f = reinterpret_cast<float*>(slot);
    float a, b;
    split_tf32x2(x, a, b);
    f[off] = a;
    f[plane + off] = b;
    return;
  }
  if (fmt == FMT_FP16X2) {
    __half* h = reinterpret_cast<__half*>(slot);
    __half a, b;
    split_fp16x2(x, a, b);
    h[off] = a;
    h[plane + off] = b;
    return;
  }
  __nv_bfloat16 a, b, c;
  split_bf16x3(x, a, b, c);
  slot[off] = a;
  slot[plane + off] = b;
  slot[2 * plane + off] = c;
}

__host__ __device__ __forceinline__ int tiles_of(int ld, int upper) {
  const int R = ld / BM;
  return upper ? R * (R + 1) / 2 : R * R;
}

__host__ __device__ __forceinline__ int pair_tiles_of(int ld, int upper) {
  const int R = ld / PT;
  return upper ? R * (R + 1) / 2 : R * R;
}

// Partial records one forward square writes: one per (tile, epilogue warp).
__host__ __device__ __forceinline__ int nparts_of(int ld, int pair) {
  return pair ? 2 * P_EPI_WARPS * pair_tiles_of(ld, 1) : 4 * tiles_of(ld, 1);
}

}  // namespace tc
}  // namespace sp2
