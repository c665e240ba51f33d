// Kernel templates: packer, batched forward interpreter, fitness finaliser.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "isa.h"

namespace gg {

// ----------------------------------------------------------------- packing
struct PackParams {
  const uint8_t* op;
  const float* cval;
  const int8_t* height;  // nullable: every trial has height h_max
  int n, h_max, stride, layout, n_features, max_slots, lstride;
  uint2* prog;           // [n][lstride] (word, const bits)
  Aux* aux;              // nullable, [n][lstride]
  int* len;              // [n] per slot: instruction count, -1 for an invalid trial
  unsigned* status;
  const int* count;      // null, or the number of slots to pack (set on the device)
  const int* idx;        // with count: the trial packed into each slot
  int allow_pow;         // 0: an active pow node makes the trial invalid
  int fold;              // fold constant subtrees (ignored when aux is set)
  int* size_active;      // [n] by trial, or null: active nodes (-1 if invalid)
  int* size_eval;        // [n] by trial, or null: nodes evaluated per row after
                         // folding (a folded subtree counts as one constant)
};

// pack_kernel (pack.cu): one warp per trial, PACK_WARPS warps per block.
// Shared scratch per warp and template node: folded value, constant (floats),
// subtree size, first instruction, template position (int16), class, kind,
// flags, stack need (bytes).
constexpr int PACK_WARPS = 4;
__host__ __device__ inline size_t pack_warp_bytes(int stride) {
  return ((size_t)stride * 18 + 15) & ~(size_t)15;
}


// ------------------------------------------------------- batched forward
// Work item = (group of `group` trials, row tile of `tile_rows` rows).  A
// persistent CTA claims items from a global counter; for each it stages the
// tile's feature rows and centred target (feature-major, row F = y - mean y)
// into shared memory with TMA bulk copies, then its warps claim the group's
// trials one at a time.  A warp runs its trial over every row of the tile,
// R rows per lane per pass, and accumulates per-lane error-free FP32 sums of
// d = f - c, d^2 and d * yc, where c is the mean of f over the tile's first
// pass (a shift that keeps the sums well conditioned).  The warp combines
// its lanes' sums in double-float arithmetic and writes one partial record
// {c, S_d, S_dd, S_dy, max|f|} per (trial, tile), the sums as FP32 (hi, lo)
// pairs; fin_kernel merges them in double-float arithmetic and forms the
// fitness from the merged sums in FP64.  (Section 3.2 accumulates squared
// errors per thread in registers and reduces them per block; here the tile
// of rows is shared by many trials so X is read from HBM once per group
// instead of once per trial.)
struct FwdParams {
  const float* X;      // [F + 1][ldx]: features, then centred target
  int N, F, ldx;
  const uint2* prog;   // [P][lstride]
  const int* len;      // [P]
  int lstride, P;
  int tile_rows, n_tiles, group, n_items;
  int slots;           // stack slots per warp (at least the deepest program's)
  float* part;         // [P][n_tiles][NPART]
  int* counter;        // work-item counter, zero at launch
  unsigned* status;
  float* rows_out;     // [P][N] per-row values (ROWS variant only)
  int* dead;           // [P] zero at launch, or null: 1 once a tile of the trial
                       // is non-finite or exceeds 2^50 (its fitness is +inf)
  const int* count;    // null, or the number of trials (slots) to evaluate, set
                       // on the device (masked evaluation; at most P)
  uint32_t wait_limit; // polls before a tile wait gives up (ST_TIMEOUT)
  int stall;           // test hook: issue no tile copy, so every wait gives up
};

// partial record of one (trial, tile): the shift c, (hi, lo) of S_d, S_dd and
// S_dy, and max |f|, all FP32; the finaliser merges them in double-float
// arithmetic
constexpr int NPART = 8;

// two tile buffers, one stack of `slots` x 32 lanes x R floats per warp, one
// program buffer of lstride + 1 words per warp (the interpreter reads one
// word past the NOP that ends a program), two mbarriers, two 4-int control
// blocks
__host__ __device__ inline size_t fwd_smem_bytes(int F, int tile_rows, int warps, int lstride,
                                                 int slots, int R) {
  return 2 * (size_t)(F + 1) * tile_rows * 4 + (size_t)warps * slots * 32 * R * 4 +
         (size_t)warps * (lstride + 1) * 8 + 16 + 32;
}

template <int R, bool MASK>
__device__ __forceinline__ void accumulate_exact(const float (&A)[R], const float (&yv)[R], float cs,
                                                 int valid, float& s1h, float& s1l, float& s2h,
                                                 float& s2l, float& s3h, float& s3l, float& fm) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const bool ok = !MASK || row_of<R>(r) < valid;
    const float d = ok ? A[r] - cs : 0.f;
    fm = fmaxf(fm, ok ? fabsf(A[r]) : 0.f);
    acc_add(s1h, s1l, d);
    acc_dot(s2h, s2l, d, d);
    acc_dot(s3h, s3l, d, yv[r]);
  }
}

// Plain FP32 group sums: the pass's R rows, two at a time as packed
// FP32 instructions, are added to the lane's group sums m1..m3 (one per
// half of a row pair); the caller folds the group sums into the error-free
// (hi, lo) accumulators every GROUP passes (fold_group).  A group sum adds
// at most GROUP x R / 2 terms per half before it is folded.
template <int R, bool MASK>
__device__ __forceinline__ void accumulate_grouped(const float (&A)[R], const float (&yv)[R],
                                                   float cs, int valid, float2& m1, float2& m2,
                                                   float2& m3, float& fm) {
  if constexpr (R % 2 == 0) {
    const float2 nc = make_float2(-cs, -cs);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      float2 d = __fadd2_rn(make_float2(A[2 * i], A[2 * i + 1]), nc);
      const bool ok0 = !MASK || row_of<R>(2 * i) < valid,
                 ok1 = !MASK || row_of<R>(2 * i + 1) < valid;
      if constexpr (MASK) {
        d.x = ok0 ? d.x : 0.f;
        d.y = ok1 ? d.y : 0.f;
      }
      fm = fmaxf(fm, ok0 ? fabsf(A[2 * i]) : 0.f);
      fm = fmaxf(fm, ok1 ? fabsf(A[2 * i + 1]) : 0.f);
      m1 = __fadd2_rn(m1, d);
      m2 = __ffma2_rn(d, d, m2);
      m3 = __ffma2_rn(d, make_float2(yv[2 * i], yv[2 * i + 1]), m3);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const bool ok = !MASK || row_of<R>(r) < valid;
      const float d = ok ? A[r] - cs : 0.f;
      fm = fmaxf(fm, ok ? fabsf(A[r]) : 0.f);
      m1.x += d;
      m2.x = fmaf(d, d, m2.x);
      m3.x = fmaf(d, yv[r], m3.x);
    }
  }
}

constexpr int GROUP = 4;  // passes per plain FP32 group sum

__device__ __forceinline__ void fold_group(float2& m1, float2& m2, float2& m3, float& s1h,
                                           float& s1l, float& s2h, float& s2l, float& s3h,
                                           float& s3l) {
  acc_add(s1h, s1l, m1.x + m1.y);
  acc_add(s2h, s2l, m2.x + m2.y);
  acc_add(s3h, s3l, m3.x + m3.y);
  m1 = m2 = m3 = make_float2(0.f, 0.f);
}

// Claim the next work item for tile buffer `s` and start loading it: run by
// one whole warp.  The X tile and the centred target rows go to shared
// memory with one TMA bulk copy per feature row, completing on bar[s]; a
// ragged last tile has its tail zeroed first.  Past the last item the
// barrier is completed without a copy so that waiting warps see the end.
__device__ __forceinline__ void produce_tile(const FwdParams& p, int n_items, int s, float* xs,
                                             uint64_t* bar, int* ctl, int lane) {
  int item = 0;
  if (lane == 0) item = atomicAdd(p.counter, 1);
  item = __shfl_sync(0xffffffffu, item, 0);
  if (item < n_items) {
    const int tile = item % p.n_tiles;
    const int row0 = tile * p.tile_rows;
    const int nrows = min(p.tile_rows, p.N - row0);
    const int ncopy = (nrows + 3) & ~3;
    if (ncopy < p.tile_rows) {
      const int tail = p.tile_rows - ncopy;
      for (int i = lane; i < (p.F + 1) * tail; i += 32) {
        const int f = i / tail;
        xs[(size_t)f * p.tile_rows + ncopy + (i - f * tail)] = 0.f;
      }
    }
    __syncwarp();
#ifdef GGEVAL_CHECKED
    // the copy must stay inside the dataset and the tile buffer: otherwise
    // record the violation and complete the barrier without copying
    const bool copy_ok = row0 + ncopy <= p.ldx && ncopy <= p.tile_rows;
    if (!copy_ok) {
      if (lane == 0) {
        record_violation(p.status);
        ctl[0] = item;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
      }
      return;
    }
#endif
    if (lane == 0) {
      ctl[0] = item;
      if (!p.stall) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (uint32_t)((p.F + 1) * ncopy * 4));
        for (int f = 0; f <= p.F; ++f)
          bulk_g2s(xs + (size_t)f * p.tile_rows, p.X + (size_t)f * p.ldx + row0,
                   (uint32_t)(ncopy * 4), bar);
      }
    }
  } else if (lane == 0) {
    ctl[0] = item;
    if (!p.stall)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
  }
}

// Two tile buffers form a pipeline: while the warps work on one tile, the
// other is being loaded.  Each buffer s has a control block ctl[4 s ..]:
// [0] its work item, [1] the next trial of the item's group to hand out,
// [2] how many warps are done with it.  The warp that finishes a buffer
// last resets [1], [2] and refills the buffer with the next item; no warp
// ever waits for the others except for the tile it is about to use.
// MINB is the launch-bounds occupancy target: 1 allows CTAs of up to 28
// warps and the compiler up to 72 registers per thread (the register file
// holds 28 warps at 72), 2 caps it at 64 (two 512-thread CTAs per SM).
// Measured with the autotuner on the 8-rows-per-lane kernel: 16 -> 20 -> 24
// -> 28 warps per SM each gained 1 to 8 % per step, the register caps cost
// nothing measurable.
constexpr int fwd_max_threads(int minb) { return minb == 1 ? 896 : 512; }
template <int R, bool EXACT, bool ROWS, int MINB, bool POW, bool CXXI = false>
__global__ void __launch_bounds__(fwd_max_threads(MINB), MINB) fwd_kernel(const FwdParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const size_t tile_floats = (size_t)(p.F + 1) * p.tile_rows;
  // trials (slots) to evaluate and the work items they make: a masked
  // evaluation sets the count on the device (compacted changed trials)
  const int P = p.count ? min(*p.count, p.P) : p.P;
  // a masked evaluation has fewer trials than the plan was sized for: its
  // groups shrink so that the work items still cover every CTA 16 times,
  // but keep three trials per warp (with fewer, warps that finish early
  // wait for the slowest before the tile buffer is refilled)
  int group = p.group;
  if (p.count) {
    const long long target = 16LL * gridDim.x;
    const int want = (int)(((long long)P * p.n_tiles + target - 1) / target);
    group = min(p.group, max(3 * nw, want));
  }
  const int n_items = p.count ? p.n_tiles * ((P + group - 1) / group) : p.n_items;
  float* xsb = reinterpret_cast<float*>(smem);  // two tile buffers
  float* stacks = xsb + 2 * tile_floats;
  float* stk = stacks + (size_t)warp * p.slots * 32 * R + lane * LANE_STRIDE<R>;  // slot 0
  uint2* progs = reinterpret_cast<uint2*>(stacks + (size_t)nw * p.slots * 32 * R);
  uint2* wprog = progs + (size_t)warp * (p.lstride + 1);
  uint64_t* bar = reinterpret_cast<uint64_t*>(progs + (size_t)nw * (p.lstride + 1));
  int* ctl = reinterpret_cast<int*>(bar + 2);

  // the finaliser behind this kernel may launch now: it waits for this
  // grid to complete before it reads anything
  allow_dependents();
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    for (int i = 0; i < 8; ++i) ctl[i] = 0;
  }
  __syncthreads();
  // the first two tiles read only the dataset and the work counter (zeroed
  // before the packer ran), so they load while the packer may still run
  if (warp == 0) {
    produce_tile(p, n_items, 0, xsb, &bar[0], ctl, lane);
    produce_tile(p, n_items, 1, xsb + tile_floats, &bar[1], ctl + 4, lane);
  }
  grid_dependency_wait();  // the packer's programs and lengths

  float A[R];
#pragma unroll
  for (int r = 0; r < R; ++r) A[r] = 0.f;

  constexpr int RPP = 32 * R;  // rows per pass of a warp
  uint32_t parity = 0;         // bit s: phase parity of bar[s] this warp waits for next
  for (int s = 0;; s ^= 1) {
    if (!mbar_wait_bounded(&bar[s], (parity >> s) & 1u, p.status, p.wait_limit)) {
      // the wait gave up (ST_TIMEOUT is set): before this warp leaves, give
      // a copy still in flight into either buffer time to land (bounded
      // too), so that no bulk copy outlives the CTA's shared memory
      mbar_wait_bounded(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u, p.status, p.wait_limit);
      mbar_wait_bounded(&bar[s], (parity >> s) & 1u, p.status, p.wait_limit);
      return;
    }
    parity ^= 1u << s;
    int* c = ctl + 4 * s;
    const int item = *reinterpret_cast<volatile int*>(&c[0]);
    if (item >= n_items) break;
    const float* xs = xsb + s * tile_floats;
    const int g = item / p.n_tiles;
    const int tile = item - g * p.n_tiles;
    const int row0 = tile * p.tile_rows;
    const int nrows = min(p.tile_rows, p.N - row0);
    const int npass = (nrows + RPP - 1) / RPP;
    for (;;) {
      int t = 0;
      if (lane == 0) t = atomicAdd(&c[1], 1);
      t = __shfl_sync(0xffffffffu, t, 0);
      const int trial = g * group + t;
      if (t >= group || trial >= P) break;
      // stage the program: the opcode alone in .x and, for an instruction
      // that reads a feature, the feature's byte offset in the tile in .y;
      // a trial another tile has already found non-finite is skipped (its
      // fitness is +inf whatever the other tiles hold).  The first 32 words
      // of the program slot are loaded together with the length and the
      // flag, so that a program of up to 31 instructions costs one memory
      // round trip; the rest of a longer one follows once L is known.
      const uint2* src = p.prog + (size_t)trial * p.lstride;
      const uint2 w0 = lane < p.lstride ? src[lane] : make_uint2(0u, 0u);
      const int L = p.len[trial];
      const int dead = p.dead && lane == 0 ? p.dead[trial] : 0;
      if (L <= 0 || __shfl_sync(0xffffffffu, dead, 0)) continue;
      for (int k = lane; k <= L; k += 32) {
        uint2 w = k < 32 ? w0 : src[k];
        const uint32_t op = w.x & 0xffu;
        if (reads_feature(op)) w.y = (w.x >> 8) * (uint32_t)p.tile_rows * 4u;
        w.x = op;
        wprog[k] = w;
      }
      __syncwarp();

      float s1h = 0.f, s1l = 0.f, s2h = 0.f, s2l = 0.f, s3h = 0.f, s3l = 0.f, fm = 0.f;
      float2 m1 = make_float2(0.f, 0.f), m2 = m1, m3 = m1;
      float cs = 0.f;
      for (int ps = 0; ps < npass; ++ps) {
        const int r0 = ps * RPP + lane * LANE_STRIDE<R>;  // the lane's first row (row_of)
        // The C++ interpreter runs in the CXXI variants (the autotuner
        // weighs them against the PTX ones: the compare tree costs more
        // instructions per dispatch, the indirect branch more stalls, and
        // short programs favour the tree) and in the kernels built with pow:
        // pow is a library call, and the PTX interpreter leaves its
        // statement for every pow instruction (on the Table 2 set 0.3 exits
        // per trial and pass, 1.75 ms per step against 1.54 ms with the
        // C++ switch).  The checked build runs it everywhere (its bounds
        // checks are C++).
#ifdef GG_INTERP_CXX
        constexpr bool CXX = true;
#else
        constexpr bool CXX = POW || CXXI;
#endif
        if constexpr (CXX) {
          const Checks cb{stk, stk + (size_t)p.slots * 32 * R, xs + r0,
                          xs + r0 + (size_t)p.F * p.tile_rows, p.status};
          run_program<R, false, true, POW>(wprog, L, xs + r0, p.tile_rows, A, stk, nullptr, &cb);
        } else {
          run_program_fast<R, POW>(wprog, xs + r0, A, stk);
        }
        const int valid = nrows - r0;  // the lane's row r is inside the tile if row_of(r) < valid
        if constexpr (ROWS) {
          float* out = p.rows_out + (size_t)trial * p.N + row0 + r0;
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (row_of<R>(r) < valid) out[row_of<R>(r)] = A[r];
        }
        if (ps == 0) {  // shift: mean of f over the first pass's rows
          float sm = 0.f;
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (row_of<R>(r) < valid) sm += A[r];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
          cs = sm / (float)min(nrows, RPP);
        }
        float yv[R];
        load_lane<R>(xs + (size_t)p.F * p.tile_rows + r0, yv);
        const bool full = (ps + 1) * RPP <= nrows;
        if constexpr (EXACT) {
          if (full)
            accumulate_exact<R, false>(A, yv, cs, valid, s1h, s1l, s2h, s2l, s3h, s3l, fm);
          else
            accumulate_exact<R, true>(A, yv, cs, valid, s1h, s1l, s2h, s2l, s3h, s3l, fm);
        } else {
          if (full)
            accumulate_grouped<R, false>(A, yv, cs, valid, m1, m2, m3, fm);
          else
            accumulate_grouped<R, true>(A, yv, cs, valid, m1, m2, m3, fm);
          if ((ps & (GROUP - 1)) == GROUP - 1 || ps == npass - 1)
            fold_group(m1, m2, m3, s1h, s1l, s2h, s2l, s3h, s3l);
        }
      }
      warp_dd_sum(s1h, s1l);
      warp_dd_sum(s2h, s2l);
      warp_dd_sum(s3h, s3l);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o));
      if (lane == 0) {
        float4* q = reinterpret_cast<float4*>(p.part + ((size_t)trial * p.n_tiles + tile) * NPART);
        q[0] = make_float4(cs, s1h, s1l, s2h);
        q[1] = make_float4(s2l, s3h, s3l, fm);
        // the finaliser's test, per tile: this trial's fitness is +inf
        if (p.dead && !(fm <= OUT_BIG && isfinite(s1h + s2h + s3h) && isfinite(cs)))
          p.dead[trial] = 1;
      }
      __syncwarp();
    }
    // this warp is done with buffer s; the last one refills it
    __threadfence_block();
    int last = 0;
    if (lane == 0) last = atomicAdd(&c[2], 1) == nw - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      if (lane == 0) {
        c[1] = 0;
        c[2] = 0;
      }
      __syncwarp();
      produce_tile(p, n_items, s, xsb + s * tile_floats, &bar[s], c, lane);
    }
  }
}

// ------------------------------------------------------------- finaliser
// Merge the per-tile partial sums of every trial in double-float arithmetic
// (fixed order, so the result is deterministic) and turn the merged sums,
// in FP64, into a*, b*, smse and mse.
// With d = f - c* (c* the first tile's shift) and yc = y - mean(y):
//   var_N = S_dd - S_d^2/N,  cov_N = S_dy - S_d S_yc/N,  b* = cov_N/var_N,
//   smse  = (Syy_N - b* cov_N)/N   (the least-squares residual, Eq. 1 with
//   the optimal affine map), mse = (1/N) sum (d - yc + c* - ybar)^2.
struct FinParams {
  const float* part;
  const int* len;
  int P, n_tiles, tile_rows;
  long long N;
  const float2* pref;  // [N + 1] prefix sums of the stored centred target (FP32 hi, lo)
  double ybar, syc, sycyc;
  float* smse;
  float* a;
  float* b;
  float* mse;
  float* nmse;         // nullable: mse / Var(y) (Eq. 2)
  double* ab;          // [P][4]: a* - ybar, b*, finite flag, 0 (adjoint), nullable
  const int* dead;     // [P] or null: 1 for a trial the forward kernel found
                       // non-finite (some of its tile records were skipped)
  const int* count;    // null, or the number of slots evaluated (masked evaluation)
  const int* idx;      // with count: the trial index of every slot (its outputs)
};

constexpr double VAR_TOL = 1e-12;
constexpr int FIN_WARPS = 16;  // trials per finaliser block

// fin_kernel is defined in misc.cu.

// Kernel pointers: variant 0 = 8 rows/lane grouped sums, 1 = 4 rows/lane
// grouped sums, 2 = 4 rows/lane exact sums, 3 = variant 2 writing per-row values;
// variants 4, 5, 6 = variants 0, 1, 2 compiled for at most 64 registers;
// 7 = variant 0 writing per-row values; 8, 9 = variants 0 and 5 with the C++
// interpreter instead of the PTX one, 10, 11 = their per-row builds (in the
// kernels with pow, which run the C++ interpreter throughout, 8..11 are
// 0, 5, 7, 3).  The per-row variants run the same interpreter code as the
// variants with the same rows per lane.
// fwd.cu holds the table of the kernels without pow, fwd_pow.cu the kernels
// that also run pow instructions (kept apart because the pow code costs the
// other kernels registers and instruction-cache locality).
constexpr int NVARIANT = 12;
template <bool P>
const void* fwd_table(int variant) {
  switch (variant) {
    case 0: return reinterpret_cast<const void*>(&fwd_kernel<8, false, false, 1, P>);
    case 1: return reinterpret_cast<const void*>(&fwd_kernel<4, false, false, 1, P>);
    case 2: return reinterpret_cast<const void*>(&fwd_kernel<4, true, false, 1, P>);
    case 3: return reinterpret_cast<const void*>(&fwd_kernel<4, true, true, 1, P>);
    case 4: return reinterpret_cast<const void*>(&fwd_kernel<8, false, false, 2, P>);
    case 5: return reinterpret_cast<const void*>(&fwd_kernel<4, false, false, 2, P>);
    case 6: return reinterpret_cast<const void*>(&fwd_kernel<4, true, false, 2, P>);
    case 7: return reinterpret_cast<const void*>(&fwd_kernel<8, false, true, 1, P>);
    case 8: return reinterpret_cast<const void*>(&fwd_kernel<8, false, false, 1, P, !P>);
    case 9: return reinterpret_cast<const void*>(&fwd_kernel<4, false, false, 2, P, !P>);
    case 10: return reinterpret_cast<const void*>(&fwd_kernel<8, false, true, 1, P, !P>);
    case 11: return reinterpret_cast<const void*>(&fwd_kernel<4, true, true, 1, P, !P>);
    default: return nullptr;
  }
}
const void* fwd_ptr_plain(int variant);
const void* fwd_ptr_pow(int variant);
inline int variant_rows(int v) { return (v == 0 || v == 4 || v == 7 || v == 8 || v == 10) ? 8 : 4; }
// the variant that also writes per-row values, with v's rows per lane and
// interpreter
inline int rows_variant(int v) {
  if (v == 8 || v == 10) return 10;
  if (v == 9 || v == 11) return 11;
  return variant_rows(v) == 8 ? 7 : 3;
}
// variants a caller may choose for the fitness path (no per-row output)
inline bool fitness_variant(int v) { return (v >= 0 && v < 7 && v != 3) || v == 8 || v == 9; }
inline int variant_max_warps(int v) {
  return fwd_max_threads((v >= 4 && v <= 6) || v == 9 ? 2 : 1) / 32;
}
inline bool variant_exact(int v) { return v == 2 || v == 3 || v == 6 || v == 11; }

}  // namespace gg
