// Device-side building blocks shared by the kernels: the operators, the
// stack-machine interpreter (top of stack in registers, the rest in shared
// memory), error-free FP32 summation, and the PTX of programmatic launch,
// mbarriers and bulk copies.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gmath.cuh"
#include "isa.h"

namespace gg {

// ------------------------------------------------------------- status word
enum : unsigned { ST_TEMPLATE = 1u, ST_TIMEOUT = 2u, ST_CHECKED = 4u };

// Magnitude above which a trial's output makes its fitness +inf (2^50).
constexpr float OUT_BIG = 1125899906842624.0f;

// ------------------------------------------------------------ the operators
// AQ(a, b) = a / sqrt(1 + b^2): one FMA, one reciprocal square root (SFU),
// one multiply.  Division is IEEE (no fast-math).  pow(a, b) = a^b with the
// C99 special cases (NaN for a negative base and a non-integer exponent).
template <int K>
__device__ __forceinline__ float binop(float a, float b) {
  if constexpr (K == K_ADD) return a + b;
  if constexpr (K == K_SUB) return a - b;
  if constexpr (K == K_MUL) return a * b;
  if constexpr (K == K_AQ) return a * rsqrt_approx(fmaf(b, b, 1.0f));
  if constexpr (K == K_DIV) return a / b;
  if constexpr (K == K_POW) return powf(a, b);
  return 0.f;
}

// The R rows of a lane through one binary operator.  +, -, x and AQ run on
// row pairs as packed FP32 instructions (FADD2 / FMUL2 / FFMA2 of sm_100 and
// later, each half rounded exactly as the scalar instruction, so every row
// is bit-identical to binop); division and pow stay scalar.  `o` may alias
// `a` or `b`.
template <int K, int R>
__device__ __forceinline__ void binop_rows(const float (&a)[R], const float (&b)[R],
                                           float (&o)[R]) {
  if constexpr (R % 2 == 0 && (K == K_ADD || K == K_SUB || K == K_MUL || K == K_AQ)) {
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const float2 x = make_float2(a[2 * i], a[2 * i + 1]);
      const float2 y = make_float2(b[2 * i], b[2 * i + 1]);
      float2 v;
      if constexpr (K == K_ADD) v = __fadd2_rn(x, y);
      if constexpr (K == K_SUB) v = __ffma2_rn(y, make_float2(-1.0f, -1.0f), x);  // exact -y
      if constexpr (K == K_MUL) v = __fmul2_rn(x, y);
      if constexpr (K == K_AQ) {
        const float2 q = __ffma2_rn(y, y, make_float2(1.0f, 1.0f));
        v = __fmul2_rn(x, make_float2(rsqrt_approx(q.x), rsqrt_approx(q.y)));
      }
      o[2 * i] = v.x;
      o[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) o[r] = binop<K>(a[r], b[r]);
  }
}

template <int U>
__device__ __forceinline__ float unop(float a) {
  if constexpr (U == U_SIN) return sinf(a);
  if constexpr (U == U_COS) return cosf(a);
  if constexpr (U == U_EXP) return expf(a);
  if constexpr (U == U_LOG_ABS) return logf(fabsf(a));
  if constexpr (U == U_SQRT_ABS) return sqrtf(fabsf(a));
  if constexpr (U == U_SQUARE) return a * a;
  if constexpr (U == U_LOG) return logf(a);
  if constexpr (U == U_SQRT) return sqrtf(a);
  return 0.f;
}

// The cold path of a unary operator: the CUDA library function on the R
// rows of a lane, kept out of line.  Inlined into every case (R copies of
// the library's range handling each), it spread the interpreter's hot code
// over more instruction-cache lines: 3 to 5 % slower per step.  The rows go
// by value in a struct, so the caller's registers are not forced to memory.
template <int R>
struct ColdRows {
  float v[R];
};
template <int U, int R>
__device__ __noinline__ ColdRows<R> unop_cold(ColdRows<R> a) {
#pragma unroll
  for (int r = 0; r < R; ++r) a.v[r] = unop<U>(a.v[r]);
  return a;
}
template <int U, int R>
__device__ __forceinline__ void unop_cold_rows(float (&A)[R]) {
  ColdRows<R> t;
#pragma unroll
  for (int r = 0; r < R; ++r) t.v[r] = A[r];
  t = unop_cold<U, R>(t);
#pragma unroll
  for (int r = 0; r < R; ++r) A[r] = t.v[r];
}

// The CUDA library's sin (shift 0) or cos (shift 1), out of line.
static __device__ __noinline__ float sincos_library(float x, int shift) {
  return shift ? cosf(x) : sinf(x);
}

// The row-by-row forms for a group of rows of which some lie outside the
// own-math forms' common domain: out of line, with rolled loops, so that the
// interpreter's switch stays compact and this cold code holds few registers
// (the caller saves the ones it clobbers around the call).  The rows go in
// and out by value (ColdRows): passed by reference, the caller's row array
// had its address taken and could no longer live in registers, which made
// the C++ interpreter 1.3x (FOS-step) to 1.7x (largest workload) slower.
template <int R>
__device__ __noinline__ ColdRows<R> sincos_special_v(ColdRows<R> a, int shift) {
#pragma unroll 1
  for (int r = 0; r < R; ++r) {
    const float x = a.v[r];
    a.v[r] = fabsf(x) <= TRIG_RANGE ? sin_or_cos_reduced(x, shift) : sincos_library(x, shift);
  }
  return a;
}
template <int R, bool LOG>
__device__ __noinline__ ColdRows<R> logsqrt_special_v(ColdRows<R> a) {
#pragma unroll 1
  for (int r = 0; r < R; ++r)
    a.v[r] = LOG ? log_total(__float_as_uint(a.v[r])) : sqrt_total(a.v[r]);
  return a;
}
template <int R>
__device__ __noinline__ ColdRows<R> exp_special_v(ColdRows<R> a) {
#pragma unroll 1
  for (int r = 0; r < R; ++r) a.v[r] = exp_total(a.v[r]);
  return a;
}
template <int R>
__device__ __forceinline__ ColdRows<R> to_cold(const float (&A)[R]) {
  ColdRows<R> t;
#pragma unroll
  for (int r = 0; r < R; ++r) t.v[r] = A[r];
  return t;
}
template <int R>
__device__ __forceinline__ void from_cold(float (&A)[R], const ColdRows<R>& t) {
#pragma unroll
  for (int r = 0; r < R; ++r) A[r] = t.v[r];
}
template <int R>
__device__ __forceinline__ void sincos_special(float (&A)[R], int shift) {
  from_cold(A, sincos_special_v<R>(to_cold(A), shift));
}
template <int R, bool LOG>
__device__ __forceinline__ void logsqrt_special(float (&A)[R]) {
  from_cold(A, logsqrt_special_v<R, LOG>(to_cold(A)));
}
template <int R>
__device__ __forceinline__ void exp_special(float (&A)[R]) {
  from_cold(A, exp_special_v<R>(to_cold(A)));
}

// sin and cos on the R rows of a lane: the branch-free form of gmath.cuh,
// on row pairs as packed instructions when R is even.  One test of the
// rows' largest magnitude sends a group with an argument beyond the
// reduction's range (|x| > 2^17 or inf, or NaN in every row) to the cold
// path, which takes the library function for exactly those rows (a row's
// value depends only on its own argument).  `shift` is 0 for sin and 1 for
// cos (a run-time value in the interpreter: both share one body).
template <int R>
__device__ __forceinline__ void sincos_rows(float (&A)[R], int shift) {
  float mx = fabsf(A[0]);
#pragma unroll
  for (int r = 1; r < R; ++r) mx = fmaxf(mx, fabsf(A[r]));
  if (__builtin_expect(!(mx <= TRIG_RANGE), 0)) {
    sincos_special<R>(A, shift);
  } else if constexpr (R % 2 == 0) {
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const float2 v = sin_or_cos_reduced2(make_float2(A[2 * i], A[2 * i + 1]), shift);
      A[2 * i] = v.x;
      A[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) A[r] = sin_or_cos_reduced(A[r], shift);
  }
}

// log (LOG) or sqrt on the R rows of a lane, after `mask` is applied to the
// bits (0x7fffffff for log|x| and sqrt|x|, all ones for the unprotected
// forms): the branch-free forms of gmath.cuh on row pairs when every row is
// a positive normal number, else log_total / sqrt_total row by row.
template <int R, bool LOG>
__device__ __forceinline__ void logsqrt_rows(float (&A)[R], uint32_t mask) {
  bool special = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t b = __float_as_uint(A[r]) & mask;
    A[r] = __uint_as_float(b);
    special |= outside_positive_normal(b);
  }
  if (__builtin_expect(special, 0)) {
    logsqrt_special<R, LOG>(A);
  } else if constexpr (R % 2 == 0) {
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const float2 x = make_float2(A[2 * i], A[2 * i + 1]);
      const float2 v = LOG ? log_normal2(x) : sqrt_newton2(x);
      A[2 * i] = v.x;
      A[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) A[r] = LOG ? log_normal(A[r]) : sqrt_newton(A[r]);
  }
}

constexpr uint32_t ABS_MASK = 0x7fffffffu;

// exp on the R rows of a lane: the own form of gmath.cuh (exp_ex2), on row
// pairs as packed instructions when every |x| <= 87, else exp_total row by
// row.
template <int R>
__device__ __forceinline__ void exp_rows(float (&A)[R]) {
  float mx = fabsf(A[0]);
#pragma unroll
  for (int r = 1; r < R; ++r) mx = fmaxf(mx, fabsf(A[r]));
  if (__builtin_expect(!(mx <= EXP_RANGE), 0)) {
    exp_special<R>(A);
  } else if constexpr (R % 2 == 0) {
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const float2 v = exp_ex2_2(make_float2(A[2 * i], A[2 * i + 1]));
      A[2 * i] = v.x;
      A[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) A[r] = exp_ex2(A[r]);
  }
}

// A unary operator on the R rows of a lane (compile-time operator; the
// interpreter's switch calls the shared bodies above directly).
template <int U, int R>
__device__ __forceinline__ void unop_rows(float (&A)[R]) {
  if constexpr (U == U_SIN || U == U_COS) {
    sincos_rows<R>(A, U == U_COS);
  } else if constexpr (U == U_LOG_ABS || U == U_LOG) {
    logsqrt_rows<R, true>(A, U == U_LOG_ABS ? ABS_MASK : ~0u);
  } else if constexpr (U == U_SQRT_ABS || U == U_SQRT) {
    logsqrt_rows<R, false>(A, U == U_SQRT_ABS ? ABS_MASK : ~0u);
  } else if constexpr (U == U_SQUARE) {
    binop_rows<K_MUL, R>(A, A, A);
  } else if constexpr (U == U_EXP) {
    exp_rows<R>(A);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) A[r] = unop<U>(A[r]);
  }
}

// ------------------------------------------------------------ interpreter
// Load R consecutive rows of one feature row of the shared-memory tile.
template <int R>
__device__ __forceinline__ void load_rows(const float* __restrict__ p, float (&v)[R]) {
  static_assert(R == 1 || R == 2 || R % 4 == 0, "R must be 1, 2 or a multiple of 4");
  if constexpr (R == 1) {
    v[0] = *p;
    return;
  }
  if constexpr (R == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
    return;
  }
#pragma unroll
  for (int q = 0; q < R / 4; ++q) {
    const float4 t = reinterpret_cast<const float4*>(p)[q];
    v[4 * q + 0] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
}

// Store R consecutive rows of a lane (the counterpart of load_rows).
template <int R>
__device__ __forceinline__ void store_rows(float* __restrict__ p, const float (&v)[R]) {
  static_assert(R == 1 || R == 2 || R % 4 == 0, "R must be 1, 2 or a multiple of 4");
  if constexpr (R == 1) {
    *p = v[0];
    return;
  }
  if constexpr (R == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    return;
  }
#pragma unroll
  for (int q = 0; q < R / 4; ++q)
    reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// A lane's R rows in a shared-memory row array (a tile's feature row, a
// stack slot): R consecutive rows for R <= 4; for R = 8 two runs of 4
// consecutive rows, 128 rows apart, the lanes 4 rows apart.  A warp's
// 16-byte access then covers 512 contiguous bytes without bank conflicts
// (8 consecutive rows per lane put the lanes 32 bytes apart, and every
// access conflicted two ways: 44 % of the forward kernel's shared-memory
// wavefronts on 4,096 x h4 over 100,000 rows).
template <int R>
constexpr int LANE_STRIDE = R == 8 ? 4 : R;  // rows between neighbouring lanes
template <int R>
__host__ __device__ constexpr int row_of(int r) {  // row offset of the lane's r-th row
  return R == 8 ? (r >> 2) * 128 + (r & 3) : r;
}
template <int R>
constexpr int LANE_EXTENT = row_of<R>(R - 1) + 1;  // rows spanned from the lane's first

template <int R>
__device__ __forceinline__ void load_lane(const float* __restrict__ p, float (&v)[R]) {
  if constexpr (R == 8) {
    float a[4], b[4];
    load_rows<4>(p, a);
    load_rows<4>(p + 128, b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[r] = a[r];
      v[4 + r] = b[r];
    }
  } else {
    load_rows<R>(p, v);
  }
}
template <int R>
__device__ __forceinline__ void store_lane(float* __restrict__ p, const float (&v)[R]) {
  if constexpr (R == 8) {
    float a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a[r] = v[r];
      b[r] = v[4 + r];
    }
    store_rows<4>(p, a);
    store_rows<4>(p + 128, b);
  } else {
    store_rows<R>(p, v);
  }
}

// Bounds of the checked build (GGEVAL_CHECKED): a lane's stack slots and
// the tile's feature rows.  Every stack and feature access of the C++
// interpreter is tested first; an access outside records ST_CHECKED in the
// status word and reads or writes the region's first entry instead (no
// trap, no access out of bounds).
struct Checks {
  const float* stk_lo;
  const float* stk_hi;
  const float* feat_lo;
  const float* feat_hi;
  unsigned* status;
};
static __device__ __noinline__ void record_violation(unsigned* status) {
  atomicOr(status, 4u);  // ST_CHECKED
}
#ifdef GGEVAL_CHECKED
#define GG_IN(ptr, lo, hi)                                                          \
  (cb && !((ptr) >= cb->lo && (ptr) + LANE_EXTENT<R> <= cb->hi) ? (record_violation(cb->status), \
                                                      const_cast<float*>(cb->lo))  \
                                                   : (ptr))
#else
#define GG_IN(ptr, lo, hi) (ptr)
#endif

// The feature row `byte_off` bytes past xs (the staged words' offsets).
__device__ __forceinline__ const float* feature_at(const float* xs, uint32_t byte_off) {
  return reinterpret_cast<const float*>(reinterpret_cast<const char*>(xs) + byte_off);
}

// Run one packed program on R rows per lane.  `prog` is the warp's copy of
// the program in shared memory (word, const bits) with a NOP at [L];
// `xs` points at row r0 of feature 0 of the tile, features `ts` floats
// apart.  Every lane of the warp executes the same instruction sequence, so
// the switch below is warp-uniform (Section 3.2: all threads interpret the
// same individual, avoiding divergence).  The top of the stack is A (the
// caller's registers); the values below it live in the warp's stack in
// shared memory: `stk` is this lane's entry in slot 0 (slot j at
// stk + 32 R j), so a push or a pop is one R-float shared-memory access per
// lane.  The first instruction of every program loads A without a push.
// With PRESCALED the words are in the staged form the batched kernel
// writes: .x holds the opcode alone and, for an instruction that reads a
// feature, .y holds the feature's offset in bytes (4 x feature x ts) in
// place of the unused constant, so the decode needs neither a mask nor a
// shift.  With TAPE the R values of A after
// instruction k are stored at tape[32 R k] (the caller offsets `tape` by its
// lane's R rows): the forward half of the adjoint.  POW adds the pow
// instructions; without it the program must not contain them.
template <int R, bool TAPE = false, bool PRESCALED = false, bool POW = false>
__device__ __forceinline__ void run_program(const uint2* __restrict__ prog, int L,
                                            const float* __restrict__ xs, int ts,
                                            float (&A)[R], float* __restrict__ stk,
                                            float* __restrict__ tape = nullptr,
                                            const Checks* cb = nullptr) {
  constexpr int SLOT = 32 * R;  // floats per stack slot
  float* sp = stk;              // next free slot of this lane
  {
    // the first instruction is always I_LDF0 or I_LDC0 (the packers emit a
    // load without a push exactly there), so it is peeled off the switch
    const uint2 first = prog[0];
    if ((PRESCALED ? first.x : first.x & 0xffu) == I_LDF0) {
      load_lane<R>(GG_IN(PRESCALED ? feature_at(xs, first.y) : xs + (first.x >> 8) * ts,
                         feat_lo, feat_hi), A);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) A[r] = __uint_as_float(first.y);
    }
    if constexpr (TAPE) store_lane<R>(tape, A);
  }
  uint2 ins = prog[1];
  for (int k = 1; k < L; ++k) {
    const uint2 nxt = prog[k + 1];
    const uint32_t opc = PRESCALED ? ins.x : ins.x & 0xffu;
    const float c = __uint_as_float(ins.y);
    const float* xf = PRESCALED ? feature_at(xs, ins.y) : xs + (ins.x >> 8) * ts;
    float t[R];

#define GG_ROWS _Pragma("unroll") for (int r = 0; r < R; ++r)
#define GG_UN(u)                                   \
  case I_UN + u:                                   \
    unop_rows<u, R>(A);                            \
    break;
#define GG_BIN_AT(kd, off)                                                  \
  case I_BF + kd + (off):                                                \
    load_lane<R>(GG_IN(xf, feat_lo, feat_hi), t);                     \
    binop_rows<kd, R>(A, t, A);                                       \
    break;                                                            \
  case I_BC + kd + (off):                                                \
    GG_ROWS t[r] = c;                                                 \
    binop_rows<kd, R>(A, t, A);                                       \
    break;                                                            \
  case I_LF + kd + (off):                                                \
    load_lane<R>(GG_IN(xf, feat_lo, feat_hi), t);                     \
    binop_rows<kd, R>(t, A, A);                                       \
    break;                                                            \
  case I_LC + kd + (off):                                                \
    GG_ROWS t[r] = c;                                                 \
    binop_rows<kd, R>(t, A, A);                                       \
    break;                                                            \
  case I_BS + kd + (off):                                                \
    sp -= SLOT;                                                       \
    load_lane<R>(GG_IN(sp, stk_lo, stk_hi), t);                       \
    binop_rows<kd, R>(t, A, A);                                       \
    break;                                                            \
  case I_RS + kd + (off):                                                \
    sp -= SLOT;                                                       \
    load_lane<R>(GG_IN(sp, stk_lo, stk_hi), t);                       \
    binop_rows<kd, R>(A, t, A);                                       \
    break;

#define GG_BIN(kd) GG_BIN_AT(kd, 0u)
    switch (opc) {
      case I_PSF:
        store_lane<R>(GG_IN(sp, stk_lo, stk_hi), A);
        sp += SLOT;
        load_lane<R>(GG_IN(xf, feat_lo, feat_hi), A);
        break;
      case I_PSC:
        store_lane<R>(GG_IN(sp, stk_lo, stk_hi), A);
        sp += SLOT;
        GG_ROWS A[r] = c;
        break;
      // each pair of related operators shares one body (a run-time quadrant
      // shift or sign mask): half the code in the switch, which is bound by
      // instruction fetch as much as by issue (measured 1 to 9 % per step)
      case I_UN + U_SIN:
      case I_UN + U_COS:
        sincos_rows<R>(A, (int)(opc - (I_UN + U_SIN)));
        break;
      case I_UN + U_LOG_ABS:
      case I_UN + U_LOG:
        logsqrt_rows<R, true>(A, opc == I_UN + U_LOG ? ~0u : ABS_MASK);
        break;
      case I_UN + U_SQRT_ABS:
      case I_UN + U_SQRT:
        logsqrt_rows<R, false>(A, opc == I_UN + U_SQRT ? ~0u : ABS_MASK);
        break;
      GG_UN(U_EXP)
      GG_UN(U_SQUARE)
      GG_BIN(K_ADD)
      GG_BIN(K_SUB)
      GG_BIN(K_MUL)
      GG_BIN(K_AQ)
      // POW kernels take division through the shared operand fetch below
      // (its labels here are moved out of the opcode range): one copy of the
      // division code instead of six, 11 % faster per step on the Table 2
      // set.  The kernels without pow keep the six division cases: there
      // the change reshaped the switch and cost 1 to 5 % on workloads that
      // never divide.
      GG_BIN_AT(K_DIV, POW ? 0x1000u : 0u)
      default:
        if constexpr (POW) {
          // every pow and division form moves its operands into
          // (A, t) = (left, right) and one body per operator follows, so the
          // library pow and the division are each expanded once
          switch (opc) {
            case I_PW + 0:
            case I_BF + K_DIV:
              load_lane<R>(GG_IN(xf, feat_lo, feat_hi), t);
              break;
            case I_PW + 1:
            case I_BC + K_DIV:
              GG_ROWS t[r] = c;
              break;
            case I_PW + 2:
            case I_LF + K_DIV:
              GG_ROWS t[r] = A[r];
              load_lane<R>(GG_IN(xf, feat_lo, feat_hi), A);
              break;
            case I_PW + 3:
            case I_LC + K_DIV:
              GG_ROWS {
                t[r] = A[r];
                A[r] = c;
              }
              break;
            case I_PWS:
            case I_BS + K_DIV:
              sp -= SLOT;
              GG_ROWS t[r] = A[r];
              load_lane<R>(GG_IN(sp, stk_lo, stk_hi), A);
              break;
            case I_PWR:
            case I_RS + K_DIV:
              sp -= SLOT;
              load_lane<R>(GG_IN(sp, stk_lo, stk_hi), t);
              break;
            default:  // the packer emits only the opcodes above
              __builtin_unreachable();
          }
          if (opc >= I_PW) {
            GG_ROWS A[r] = binop<K_POW>(A[r], t[r]);
          } else {
            GG_ROWS A[r] = binop<K_DIV>(A[r], t[r]);
          }
        } else {
          // the packer emits only the opcodes above (pow only for POW kernels)
          __builtin_unreachable();
        }
    }
#undef GG_ROWS
#undef GG_UN
#undef GG_BIN
#undef GG_BIN_AT
    if constexpr (TAPE) store_lane<R>(tape + 32 * R * k, A);
    ins = nxt;
  }
}

// ------------------------------------------------- error-free FP32 sums
// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// (hi, lo) += x with the rounding error of the high part kept in lo.
__device__ __forceinline__ void acc_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo += e;
}

// (hi, lo) += a * b with the product's rounding error (via FMA) kept too.
__device__ __forceinline__ void acc_dot(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo += e + pe;
}

// Sum of two double-float values (hi1, lo1) + (hi2, lo2), renormalised.
__device__ __forceinline__ void dd_add(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  e += lo + l2;
  hi = s + e;
  lo = e - (hi - s);
}

// Sum (hi, lo) over the warp: TwoSum on the high parts at every level, the
// low parts and the TwoSum errors added plainly (their size is ~2^-24 of
// the high part, so no renormalisation is needed over 5 levels).
__device__ __forceinline__ void warp_dd_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = lo + l2 + e;
  }
}

// ------------------------------------------ programmatic dependent launch
// A kernel launched with the programmatic-serialisation attribute may start
// while the kernel ahead of it in the stream is still running.
// grid_dependency_wait() blocks until that kernel has completed and its
// writes are visible (a no-op for a kernel launched without the attribute);
// allow_dependents() lets the kernel behind this one start launching.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// -------------------------------------------------- mbarrier and bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// One TMA bulk copy global -> shared (both 16-byte aligned, bytes % 16 == 0),
// completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
      "[%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`.  Gives up after `limit` polls
// (each poll may suspend the thread for a hardware-defined time) and
// records ST_TIMEOUT instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned* status, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(status, ST_TIMEOUT);
  return false;
}

constexpr uint32_t WAIT_LIMIT = 1u << 22;

// ---------------------------------------- the PTX interpreter (fast path)
// interp_asm<R> (generated by interp_gen.py, included from the build
// folder) runs a staged program from the instruction at shared address pc
// on R rows per lane: the same operations as run_program<R, false, true>,
// dispatched through an indexed branch instead of a compare tree.  It
// returns at the program's NOP, and at an instruction it leaves to the C++
// code below: pow, or a unary operator whose rows fall outside the domain
// of its own-math form (the CUDA library function then takes the group of
// rows, as run_program decides).  pc then addresses the next instruction,
// sp the lane's next free stack slot.
#include "interp_asm.inc"

// One instruction the PTX interpreter left (opcode `code`, operand word
// `arg`), run by the C++ bodies of run_program: a group of rows of sin, cos,
// exp, log or sqrt of which some lie outside the own-math forms' common
// domain (row by row; the 4-row PTX finishes exp, log and sqrt itself), and
// pow.  Out of line: the rare cases stay off the hot loop's instruction
// stream.
template <int R>
struct ColdState {
  float a[R];
  uint32_t sp;
};
template <int R, bool POW>
__device__ __noinline__ ColdState<R> exec_cold_v(uint32_t code, uint32_t arg, ColdState<R> st,
                                                 const float* xs) {
  float (&A)[R] = st.a;
  uint32_t& sp = st.sp;
  constexpr uint32_t SLOTB = 32 * R * 4;
  switch (code) {
    case I_UN + U_SIN:
    case I_UN + U_COS:
      sincos_special<R>(A, (int)(code - (I_UN + U_SIN)));
      break;
    case I_UN + U_EXP:
      exp_special<R>(A);
      break;
    case I_UN + U_LOG_ABS:
    case I_UN + U_LOG:
    case I_UN + U_SQRT_ABS:
    case I_UN + U_SQRT: {
      const uint32_t mask = (code == I_UN + U_LOG || code == I_UN + U_SQRT) ? ~0u : ABS_MASK;
#pragma unroll 1
      for (int r = 0; r < R; ++r) A[r] = __uint_as_float(__float_as_uint(A[r]) & mask);
      if (code == I_UN + U_LOG_ABS || code == I_UN + U_LOG) logsqrt_special<R, true>(A);
      else logsqrt_special<R, false>(A);
      break;
    }
    default:
      if constexpr (POW) {
        // pow(left, right): the operands into (A, t) = (left, right)
        float t[R];
        const float c = __uint_as_float(arg);
        const float* xf = feature_at(xs, arg);
        switch (code) {
          case I_PW + 0:  // A = pow(A, X[f])
            load_lane<R>(xf, t);
            break;
          case I_PW + 1:  // A = pow(A, c)
#pragma unroll
            for (int r = 0; r < R; ++r) t[r] = c;
            break;
          case I_PW + 2:  // A = pow(X[f], A)
#pragma unroll
            for (int r = 0; r < R; ++r) t[r] = A[r];
            load_lane<R>(xf, A);
            break;
          case I_PW + 3:  // A = pow(c, A)
#pragma unroll
            for (int r = 0; r < R; ++r) {
              t[r] = A[r];
              A[r] = c;
            }
            break;
          case I_PWS:  // A = pow(pop, A)
            sp -= SLOTB;
#pragma unroll
            for (int r = 0; r < R; ++r) t[r] = A[r];
            load_lane<R>(static_cast<const float*>(__cvta_shared_to_generic(sp)), A);
            break;
          default:  // I_PWR: A = pow(A, pop)
            sp -= SLOTB;
            load_lane<R>(static_cast<const float*>(__cvta_shared_to_generic(sp)), t);
            break;
        }
#pragma unroll 1
        for (int r = 0; r < R; ++r) A[r] = binop<K_POW>(A[r], t[r]);
      }
      break;
  }
  return st;
}
// exec_cold_v with the rows and the stack pointer copied in and out by value
// (the caller's registers keep them; see the row-by-row forms above)
template <int R, bool POW>
__device__ __forceinline__ void exec_cold(uint32_t code, uint32_t arg, float (&A)[R],
                                          uint32_t& sp, const float* xs) {
  ColdState<R> st;
#pragma unroll
  for (int r = 0; r < R; ++r) st.a[r] = A[r];
  st.sp = sp;
  st = exec_cold_v<R, POW>(code, arg, st, xs);
#pragma unroll
  for (int r = 0; r < R; ++r) A[r] = st.a[r];
  sp = st.sp;
}

// Run a staged program (words as run_program's PRESCALED form, a NOP after
// the last instruction and one readable word after that) on R rows per lane:
// `xs` is this lane's first row of feature 0 in the tile, `stk` this lane's
// entry in stack slot 0.
template <int R, bool POW>
__device__ __forceinline__ void run_program_fast(const uint2* __restrict__ prog,
                                                 const float* __restrict__ xs, float (&A)[R],
                                                 float* __restrict__ stk) {
  uint32_t pc = smem_u32(prog), sp = smem_u32(stk), code = 0, arg = 0;
  const uint32_t xb = smem_u32(xs);
  for (;;) {
    interp_asm<R>(A, pc, sp, xb, code, arg);
    if (code == I_NOP || code >= I_COUNT) break;
    exec_cold<R, POW>(code, arg, A, sp, xs);
  }
}

}  // namespace gg
