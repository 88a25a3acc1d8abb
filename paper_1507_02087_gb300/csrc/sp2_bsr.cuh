// Block-sparse iterates of the block-truncated expansion: structures shared by the kernels of
// sp2_bsr.cu (index work, CUDA-core block products, truncation) and sp2_bsr_tc.cu (tensor-core
// block products).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sp2_common.cuh"

namespace sp2 {
namespace bsr {

constexpr int B = 32;              // block size
constexpr int BE = B * B;          // elements per block

__device__ __forceinline__ int popc(uint32_t x) { return __popc(x); }

struct Mat {          // one block-sparse iterate
  int* rp;            // [nb + 1]
  int* ci;            // [cap]
  float* vals;        // [cap][32][32]
  uint32_t* bits;     // [nb][W]
  int* rank;          // [nb][W]: set bits of the row in words before w
  __half* pvals;      // [cap + 1][2][32][32]: each block as two fp16 pieces of 2^14 x (the operands of
                      // the tensor-core products); block `cap` is all zero and stands for absent blocks
};

struct Pairs {        // upper (I, J >= I) block pairs of a pattern
  int* ptr;           // [nb + 1]
  int* col;           // [cap]
  int* row;           // [cap]
  int* nnz;           // device count
};

// Position of block (I, K) in `m`, or -1 if absent.
__device__ __forceinline__ int find_block(const Mat& m, int W, int I, int K) {
  const uint32_t w = m.bits[(int64_t)I * W + (K >> 5)];
  const uint32_t bit = 1u << (K & 31);
  if (!(w & bit)) return -1;
  return m.rp[I] + m.rank[(int64_t)I * W + (K >> 5)] + popc(w & (bit - 1u));
}

// Tensor-core block products (sp2_bsr_tc.cu).  A tile is 4 block rows x 8 block columns of the
// square (M = 128, N = 256); the tiles that hold an upper pair of the square's pattern are listed
// per round in row-major tile order.
constexpr int TTR = 4;             // block rows per tile
constexpr int TTC = 8;             // block columns per tile

struct TcMaps {                    // TMA maps over the piece planes of the two ping-pong iterates
  CUtensorMap map[2];
};

// The inputs of one round's tensor-core square besides the iterate: the square's pattern bits
// (upper part, one row per block row), its pair list, and the per-pair outputs the truncation and
// the stop test read, as for the CUDA-core kernel.
struct TcRound {
  const uint32_t* sbits;
  Pairs P;
  float* svals;
  uint8_t* skeep;
  double* spart;
  double* sn2;
  double tau2;
  int* tiles;                      // [cap_t]: g * (nb_cols_groups) + c
  int* tnnz;                       // device count of listed tiles
  int* meta;                       // [cap_t][TMETA]: per tile its K-block count, then for the 32
                                   // block pairs (r, c) (index 8 r + c) the pair index in P (-1: not
                                   // an upper pair of the square) and the position of the old block
                                   // X~_{k-1}(I0 + r, J0 + c) (-1: absent), then (entry 65) the
                                   // block products the tile's upper pairs need
};
constexpr int TMETA = 68;          // 1 + 32 + 32 + 1, padded

// Tile list of the round (count, scan, fill) and the tiles' metadata; `counts` has nb entries.
cudaError_t tc_tiles_launch(const DevState* st, const Mat& X, const Pairs& P, const uint32_t* sbits, int nb, int W,
                            int* counts, int* tptr, int* tnnz, int* tiles, int* meta, cudaStream_t s);
// The numeric square of the round on the tensor cores: X_k = p_k(X~_{k-1}) for every upper pair
// of the square's pattern, with the per-pair partials, block norms and keep flags.
cudaError_t tc_numeric_launch(DevState* st, const Mat& X, const TcMaps* maps, int parity, int nb, int W,
                              const TcRound& r, cudaStream_t s);
// Device queries and kernel attributes of the tensor-core square (before any stream capture).
void tc_prepare();
// TMA map over the piece planes of an iterate with `cap` blocks (+ the zero block).
cudaError_t tc_piece_map(const __half* pvals, int64_t cap, CUtensorMap* map);

}  // namespace bsr
}  // namespace sp2
