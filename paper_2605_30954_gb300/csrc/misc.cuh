// Parameter blocks and entry points of the kernels defined in misc.cu and
// adjoint.cu (the packer, the fitness finaliser, the adjoint, Adam and the
// dataset transpose).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace gg {

// The adjoint runs once per length class: the trials whose programs fit in
// lcap - 1 instructions (lcap words with the terminating NOP), binned by
// adj_bin_kernel; each launch sizes its shared memory for its class.
struct AdjParams {
  const float* X;      // [F + 1][ldx], row F = centred target
  const float* ylo;    // [ldx]: (y - mean(y)) - the stored centred target (FP32)
  int N, F, ldx;
  const uint2* prog;   // [P][lstride]
  const Aux* aux;      // [P][lstride]
  const int* len;      // [P]
  int lstride, P, stride;
  int lcap, ecap;      // this class's program words and ERC capacity per warp
  int slots;           // stack slots per warp
  const double* ab;    // [P][4]: a* - mean(y), b*, finite flag, unused
  int mse_mode;        // 0: d smse / d c, 1: d mse / d c
  double ybar;
  const int* list;     // this class's trials (count of them at *count)
  const int* count;
  int target_items;    // work items to aim for (chunks of rows x trials)
  int* counter;        // zero at launch
  double* gacc;        // [P][stride], zero at launch
};

// Length classes: program capacities (words, with the NOP) in increasing
// order; a batch uses the ones below its lstride and lstride itself.
constexpr int ADJ_NCLS_MAX = 16;
constexpr int ADJ_CAPS[] = {16, 24, 32, 40, 48, 56, 64, 80, 96, 128, 192, 256, 384, 512};

struct AdjBinParams {
  const int* len;      // [P]
  const double* ab;    // [P][4]
  int P, mse_mode, ncls;
  int caps[ADJ_NCLS_MAX];
  int* count;          // [ncls], zero at launch
  int* list;           // [ncls][P]
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

// Per-warp shared memory of the adjoint for a class of capacity lcap
// (program words) and ecap (ERCs; a tree of height h has at most 2^h active
// terminals, and every instruction carries at most one), R rows per lane:
//   prog  uint2 [lcap + 1]  the program (the generic kernel: packed words;
//                           the staged kernel: the PTX interpreter's form,
//                           with a NOP read ahead)
//   aux   Aux   [lcap]      operand producers and template positions
//                           (generic kernel)
//   rins  uint4 [lcap]      reverse-sweep descriptors (staged kernel)
//   wg    float2 [ecap]     (hi, lo) gradient accumulator per ERC ordinal
//   eord  u16   [lcap]      instruction -> ERC ordinal (generic kernel)
//   ek    u16   [ecap]      ERC ordinal -> instruction (generic) or
//                           template position (staged)
//   V     [lcap][32][R]     one value or adjoint per instruction and row
//   stk   [slots][32][R]    the forward stack
//   part  [ecap][33]        per-pass ERC partial sums (32 lanes, padded)
//   xt    [ftile][32][R]    the staged feature rows (staged kernel)
// Every array starts on a 16-byte boundary.  In the staged kernel stk and
// part share their bytes: the forward recompute alone uses the stack, the
// reverse sweep writes every ERC ordinal's partial of the pass before the
// reduction reads it, and warp barriers separate the three phases.
struct AdjLayout {
  size_t prog, aux, rins, wg, eord, ek, V, stk, part, xt, total;
};
__host__ __device__ inline size_t adj_round16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline AdjLayout adj_layout(int lcap, int ecap, int slots, int rows,
                                                bool fast, int ftile) {
  AdjLayout l{};
  size_t o = 0;
  l.prog = o;
  o = adj_round16(o + (size_t)(lcap + 1) * 8);
  l.aux = o;
  if (!fast) o = adj_round16(o + (size_t)lcap * 8);
  l.rins = o;
  if (fast) o = adj_round16(o + (size_t)lcap * 16);
  l.wg = o;
  o = adj_round16(o + (size_t)ecap * 8);
  l.eord = o;
  if (!fast) o = adj_round16(o + (size_t)lcap * 2);
  l.ek = o;
  o = adj_round16(o + (size_t)ecap * 2);
  l.V = o;
  o = adj_round16(o + (size_t)lcap * 32 * 4 * rows);
  l.stk = o;
  const size_t stk_bytes = (size_t)slots * 32 * 4 * rows, part_bytes = (size_t)ecap * 33 * 4;
  if (fast) {
    l.part = o;
    o = adj_round16(o + (stk_bytes > part_bytes ? stk_bytes : part_bytes));
  } else {
    o = adj_round16(o + stk_bytes);
    l.part = o;
    o = adj_round16(o + part_bytes);
  }
  l.xt = o;
  if (fast) o = adj_round16(o + (size_t)ftile * 32 * 4 * rows);
  l.total = o;
  return l;
}
inline size_t adj_smem_bytes(int warps, const AdjLayout& l) { return (size_t)warps * l.total + 16; }
// feature counts up to which the adjoint runs the staged 4-rows-per-lane
// kernel (feature tile in shared memory, PTX forward recompute)
constexpr int ADJ_FTILE_MAX = 16;

const void* pack_ptr();
const void* fin_ptr();
const void* compact_ptr();
const void* adj_ptr(int rows, bool pow, bool fast);
const void* adj_bin_ptr();
const void* gradout_ptr();
const void* adam_ptr();
const void* transpose_ptr();

}  // namespace gg
