// Parameter blocks and entry points of the kernels defined in misc.cu and
// adjoint.cu (the packer, the fitness finaliser, the adjoint, Adam and the
// dataset transpose).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace gg {

struct AdjParams {
  const float* X;      // [F + 1][ldx], row F = centred target
  const float* ylo;    // [ldx]: (y - mean(y)) - the stored centred target (FP32)
  int N, F, ldx;
  const uint2* prog;   // [P][lstride]
  const Aux* aux;      // [P][lstride]
  const int* len;      // [P]
  int lstride, P, stride;
  int slots;           // stack slots per warp
  const double* ab;    // [P][4]: a* - mean(y), b*, finite flag, unused
  int mse_mode;        // 0: d smse / d c, 1: d mse / d c
  double ybar;
  int chunk_rows, n_chunks, n_items;
  int* counter;        // zero at launch
  double* gacc;        // [P][stride], zero at launch
};

struct GradOutParams {
  const double* gacc;
  const int* len;
  int P, stride;
  float* dcval;        // [P][stride]
};

struct AdamParams {
  const uint8_t* op;
  float* cval;
  const float* grad;
  float* m;
  float* v;
  long long count;     // P * stride
  float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
};

struct TransposeParams {
  const float* src;    // [N][F] row-major
  float* dst;          // [F][ldx]
  int N, F, ldx;
};

// per warp: for each program instruction its word, side information, an
// (hi, lo) gradient accumulator (indexed by ERC ordinal) and two 16-bit
// ERC maps (instruction -> ordinal, ordinal -> instruction), padded to 16
// bytes; one value or adjoint per instruction for each of 32 lanes x R
// rows; the stack of `slots` x 32 x R floats; and the per-pass ERC partial
// sums, 33 floats (32 lanes, padded) for each of at most lstride / 2 ERCs
// (a tree of height h has at most 2^h active terminals)
__host__ __device__ inline size_t adj_head_bytes(int lstride) {
  return ((size_t)lstride * (8 + 8 + 8 + 2 + 2) + 15) & ~(size_t)15;
}
// With ftile > 0 (the PTX forward recompute) also the program in the
// interpreter's staged form (lstride + 1 words) and a tile of ftile
// feature rows x 32 lanes x R rows.
__host__ __device__ inline size_t adj_warp_bytes(int lstride, int slots, int rows, int ftile = 0) {
  size_t b = adj_head_bytes(lstride) + (size_t)lstride * 32 * 4 * rows +
             (size_t)slots * 32 * 4 * rows + (size_t)(lstride / 2) * 33 * 4;
  b = (b + 15) & ~(size_t)15;
  if (ftile > 0) b += (((size_t)(lstride + 1) * 8 + 15) & ~(size_t)15) +
                     (size_t)ftile * 32 * 4 * rows;
  return (b + 15) & ~(size_t)15;  // the next warp's value array stays 16-byte aligned
}
inline size_t adj_smem_bytes(int warps, int lstride, int slots, int rows, int ftile = 0) {
  return (size_t)warps * adj_warp_bytes(lstride, slots, rows, ftile) + 16;
}
// feature counts up to which the 4-rows-per-lane adjoint stages a feature
// tile and runs its forward recompute with the PTX interpreter
constexpr int ADJ_FTILE_MAX = 16;

const void* pack_ptr();
const void* fin_ptr();
const void* compact_ptr();
const void* adj_ptr(int rows, bool pow, bool fast);
const void* gradout_ptr();
const void* adam_ptr();
const void* transpose_ptr();

}  // namespace gg
