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

// per warp and program instruction: word, side information, (hi, lo)
// gradient accumulator, and one value or adjoint for each of 32 lanes x R
// rows; then the warp's stack of `slots` x 32 x R floats
__host__ __device__ inline size_t adj_warp_bytes(int lstride, int slots, int rows) {
  return (size_t)lstride * (8 + 8 + 8 + 32 * 4 * (size_t)rows) + (size_t)slots * 32 * 4 * rows;
}
inline size_t adj_smem_bytes(int warps, int lstride, int slots, int rows) {
  return (size_t)warps * adj_warp_bytes(lstride, slots, rows) + 16;
}

const void* pack_ptr();
const void* fin_ptr();
const void* compact_ptr();
const void* adj_ptr(int rows, bool pow);
const void* gradout_ptr();
const void* adam_ptr();
const void* transpose_ptr();

}  // namespace gg
