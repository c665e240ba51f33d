// Reverse-mode adjoint: d(scaled MSE)/d(constant) for every ERC leaf of
// every trial.
//
// The trials are binned by program length (adj_bin_kernel); one launch per
// length class sizes its per-warp shared memory for the class.  Work item
// = (trial, chunk of rows); warps claim items from the class's counter.
// For 32 R rows at a time (R per lane) a warp re-runs the trial's program
// forward, storing the value of every instruction in a shared-memory array
// V, seeds the output adjoint with
//   w_i = (2 b*/N) (a* + b* f_i - y_i)          (scaled MSE; envelope theorem)
//   w_i = (2/N) (f_i - y_i)                     (plain MSE)
// and sweeps the program backwards.  Every instruction's value has exactly
// one consumer (the program is a tree), so when the sweep reaches an
// instruction it reads its operands' values from V and overwrites them with
// their adjoints; by the time an operand instruction is reached, V holds its
// adjoint while its own operands still hold values.  The operators whose
// derivative uses their own output (exp, sqrt, division) recompute it from
// the operands.  The contribution of an ERC (pushed, or fused into its
// parent) is summed over the lane's rows into a per-pass partial; after
// the sweep the 32 lanes' partials are summed per ERC and added into a
// per-warp error-free FP32 (hi, lo) accumulator; at the end of the item the
// accumulators go to the trial's FP64 gradient row with atomics.  Node
// values live only in shared memory for 32 R rows at a time: nothing of
// size rows x nodes is stored in HBM, so any dataset size works
// (recomputation instead of storage).  The paper evaluates fitness only;
// this kernel is an addition.
#include "misc.cuh"

namespace gg {

// d op(a, b) / da and / db for R rows: the switch on the (warp-uniform)
// kind is taken once per instruction.
template <int R>
__device__ __forceinline__ void dbin_rows(int kind, const float (&a)[R], const float (&b)[R],
                                          float (&da)[R], float (&db)[R]) {
  switch (kind) {
    case K_ADD:
#pragma unroll
      for (int r = 0; r < R; ++r) da[r] = 1.f, db[r] = 1.f;
      break;
    case K_SUB:
#pragma unroll
      for (int r = 0; r < R; ++r) da[r] = 1.f, db[r] = -1.f;
      break;
    case K_MUL:
#pragma unroll
      for (int r = 0; r < R; ++r) da[r] = b[r], db[r] = a[r];
      break;
    case K_AQ:
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float q = rsqrt_approx(fmaf(b[r], b[r], 1.f));
        da[r] = q;
        db[r] = -a[r] * b[r] * q * q * q;
      }
      break;
    case K_POW:  // d/da = b a^(b-1); d/db = a^b ln|a| (0 where a^b = 0)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float out = powf(a[r], b[r]);
        da[r] = b[r] * powf(a[r], b[r] - 1.f);
        db[r] = out == 0.f ? 0.f : out * logf(fabsf(a[r]));
      }
      break;
    default:  // K_DIV: d/da = 1/b, d/db = -(a/b)/b
#pragma unroll
      for (int r = 0; r < R; ++r) {
        da[r] = 1.f / b[r];
        db[r] = -(a[r] / b[r]) / b[r];
      }
      break;
  }
}

// x <- g * d u(x) / dx for R rows.
template <int R>
__device__ __forceinline__ void dun_rows(int u, const float (&g)[R], float (&x)[R]) {
  switch (u) {
    case U_SIN:
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = g[r] * cosf(x[r]);
      break;
    case U_COS:
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = g[r] * -sinf(x[r]);
      break;
    case U_EXP:
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = g[r] * expf(x[r]);
      break;
    case U_LOG_ABS:
    case U_LOG:
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = g[r] * (1.f / x[r]);
      break;
    case U_SQRT_ABS:
#pragma unroll
      for (int r = 0; r < R; ++r)
        x[r] = g[r] * (x[r] == 0.f ? 0.f : copysignf(0.5f / sqrtf(fabsf(x[r])), x[r]));
      break;
    case U_SQUARE:
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = g[r] * (2.f * x[r]);
      break;
    default:  // U_SQRT
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = g[r] * (0.5f / sqrtf(x[r]));
      break;
  }
}

// Whether an instruction carries an ERC: a constant load, or a constant
// fused into a binary instruction.
template <bool POW>
__device__ __forceinline__ bool carries_erc(uint32_t opc) {
  return opc == I_LDC0 || opc == I_PSC || (opc >= I_BC && opc < I_BC + NKIND) ||
         (opc >= I_LC && opc < I_LC + NKIND) || (POW && (opc == I_PW + 1 || opc == I_PW + 3));
}

// Work items of one length class: about target_items of them (trial x
// chunk of rows), a chunk a multiple of the rows a warp runs per pass.
struct Chunking {
  int chunk_rows, n_chunks, n_items;
};
__device__ __forceinline__ Chunking chunking(const AdjParams& p, int count, int group) {
  Chunking c;
  const int max_chunks = (p.N + group - 1) / group;
  int n = count > 0 ? (p.target_items + count - 1) / count : 1;
  n = max(1, min(n, max_chunks));
  c.chunk_rows = ((p.N + n - 1) / n + group - 1) / group * group;
  c.n_chunks = (p.N + c.chunk_rows - 1) / c.chunk_rows;
  c.n_items = count * c.n_chunks;
  return c;
}

// The output adjoint of R rows: (2 b*/N) (a* + b* f - y) (scaled MSE) or
// (2/N) (f - y) (plain MSE), 0 for rows past the chunk's end.  The
// residual is formed in double-float: TwoProd / TwoSum keep the rounding of
// every term, so only f's own FP32 error remains (y = mean(y) + yc + yl
// exactly to FP64 accuracy).
template <int R>
__device__ __forceinline__ void seed_rows(const AdjParams& p, const double* ab,
                                          const float (&A)[R], const float (&yc)[R],
                                          const float (&yl)[R], const bool (&valid)[R],
                                          float (&w)[R]) {
  // a* - mean(y), b* and mean(y) as FP32 (hi, lo) pairs of their FP64 values
  const float a_hi = (float)ab[0], a_lo = (float)(ab[0] - (double)a_hi);
  const float b_hi = (float)ab[1], b_lo = (float)(ab[1] - (double)b_hi);
  const float yb_hi = (float)p.ybar, yb_lo = (float)(p.ybar - (double)yb_hi);
  const float two_n = (float)(2.0 / (double)p.N);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float s, e1, e2, t, lo;
    if (p.mse_mode) {
      two_sum(A[r], -yb_hi, s, e1);
      lo = -yb_lo;
    } else {
      const float pr = __fmul_rn(b_hi, A[r]);  // never contracted into an FMA
      lo = fmaf(b_hi, A[r], -pr) + fmaf(b_lo, A[r], a_lo);
      two_sum(a_hi, pr, s, e1);
    }
    two_sum(s, -yc[r], t, e2);
    const float res = t + ((e1 + e2) + (lo - yl[r]));
    w[r] = two_n * (p.mse_mode ? res : b_hi * res);
    w[r] = valid[r] ? w[r] : 0.f;
  }
}

// The pass's ERC sums: lane o adds up the 32 lane partials of the ERCs
// o, o + 32, ... (rows padded to 33 floats: no bank conflicts) into its
// error-free accumulators (one transposed reduction per pass instead of a
// shuffle reduction per ERC instruction).  Four running sums over every
// fourth partial keep the chain of dependent additions short.
__device__ __forceinline__ void reduce_erc(const float* part, float2* wg, int n_erc, int lane) {
  for (int o = lane; o < n_erc; o += 32) {
    const float* q = part + (size_t)o * 33;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      s0 += q[j];
      s1 += q[j + 1];
      s2 += q[j + 2];
      s3 += q[j + 3];
    }
    const float sm = (s0 + s1) + (s2 + s3);
    float2 acc = wg[o];
    acc_add(acc.x, acc.y, sm);
    wg[o] = acc;
  }
}

// The item's gradient: ERC ordinal o goes to template position ek[o].
__device__ __forceinline__ void write_grad(const AdjParams& p, int trial, const float2* wg,
                                           const uint16_t* ek, int n_erc, int lane) {
  for (int o = lane; o < n_erc; o += 32) {
    const int tp = ek[o];
    const double gk = (double)wg[o].x + (double)wg[o].y;
    if (tp != NONE16 && gk != 0.0) atomicAdd(p.gacc + (size_t)trial * p.stride + tp, gk);
  }
}

__device__ __forceinline__ bool adj_skip(const AdjParams& p, int trial) {
  const double* ab = p.ab + 4 * (size_t)trial;
  return p.len[trial] <= 0 || ab[2] == 0.0 || (!p.mse_mode && ab[1] == 0.0);
}

// Generic form, R rows per lane: each lane runs rows row0 .. row0 + R - 1
// of a 32 R-row group (feature-major X, so a lane's rows are one aligned
// R-wide load); the forward recompute is the C++ interpreter reading the
// features from global memory.  Values and adjoints live at
// V[instruction][lane][row], private to the lane; rows past the chunk's end
// are evaluated on in-bounds data and left out of every sum.
template <int R, bool POW>
__global__ void __launch_bounds__(256) adjoint_kernel(const AdjParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int SLOT = 32 * R;
  const AdjLayout lay = adj_layout(p.lcap, p.ecap, p.slots, R, false, 0);
  unsigned char* base = smem + (size_t)warp * lay.total;
  uint2* wprog = reinterpret_cast<uint2*>(base + lay.prog);
  Aux* waux = reinterpret_cast<Aux*>(base + lay.aux);
  float2* wg = reinterpret_cast<float2*>(base + lay.wg);        // (hi, lo) per ERC ordinal
  uint16_t* eord = reinterpret_cast<uint16_t*>(base + lay.eord);  // instruction -> ordinal
  uint16_t* ek = reinterpret_cast<uint16_t*>(base + lay.ek);      // ordinal -> template position
  float* V = reinterpret_cast<float*>(base + lay.V) + lane * R;   // [lcap][32][R]
  float* stk = reinterpret_cast<float*>(base + lay.stk) + lane * R;
  float* part = reinterpret_cast<float*>(base + lay.part);        // [ecap][33]
  const Chunking ch = chunking(p, *p.count, SLOT);

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(p.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= ch.n_items) break;
    const int trial = p.list[item / ch.n_chunks];
    const int chunk = item % ch.n_chunks;
    if (adj_skip(p, trial)) continue;
    const int L = p.len[trial];
    const double* ab = p.ab + 4 * (size_t)trial;
    const uint2* src = p.prog + (size_t)trial * p.lstride;
    const Aux* asrc = p.aux + (size_t)trial * p.lstride;
    // the program and, in program order, the ordinals of the instructions
    // that carry an ERC
    int n_erc = 0;
    for (int k0 = 0; k0 <= L; k0 += 32) {
      const int k = k0 + lane;
      bool has = false;
      if (k <= L) {
        const uint2 w = src[k];
        wprog[k] = w;
        if (k < L) {
          const Aux ax = asrc[k];
          waux[k] = ax;
          const uint32_t opc = w.x & 0xffu;
          has = carries_erc<POW>(opc);
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, has);
      if (has) {
        const int o = n_erc + __popc(m & ((1u << lane) - 1u));
        const uint32_t opc = wprog[k].x & 0xffu;
        eord[k] = (uint16_t)o;
        ek[o] = (opc == I_LDC0 || opc == I_PSC) ? waux[k].tpos : waux[k].tpos_fused;
        wg[o] = make_float2(0.f, 0.f);
      }
      n_erc += __popc(m);
    }
    __syncwarp();

    const int r_beg = chunk * ch.chunk_rows;
    const int r_end = min(p.N, r_beg + ch.chunk_rows);
    for (int rb = r_beg; rb < r_end; rb += SLOT) {
      // this lane's first row, kept in bounds (and R-aligned) past the end
      const int row0 = min(rb + lane * R, (r_end - 1) & ~(R - 1));
      bool valid[R];
#pragma unroll
      for (int r = 0; r < R; ++r) valid[r] = rb + lane * R + r < r_end;
      float A[R];
#pragma unroll
      for (int r = 0; r < R; ++r) A[r] = 0.f;
      run_program<R, true, false, POW>(wprog, L, p.X + row0, p.ldx, A, stk, V);
      float yc[R], yl[R], w[R];
      load_rows<R>(p.X + (size_t)p.F * p.ldx + row0, yc);
      load_rows<R>(p.ylo + row0, yl);
      seed_rows<R>(p, ab, A, yc, yl, valid, w);
      store_rows<R>(V + (size_t)SLOT * (L - 1), w);  // the output's value becomes its adjoint
      for (int k = L - 1; k >= 0; --k) {
        const uint2 ins = wprog[k];
        const Aux ax = waux[k];
        const uint32_t opc = ins.x & 0xffu;
        const int feat = (int)(ins.x >> 8);
        const float c = __uint_as_float(ins.y);
        float g[R];  // adjoint of instruction k
        load_rows<R>(V + (size_t)SLOT * k, g);
        float ge[R];  // contribution to this instruction's ERC
        bool has_erc = false;
        if (opc == I_LDF0 || opc == I_PSF) {
          // feature load: nothing to propagate
        } else if (opc == I_LDC0 || opc == I_PSC) {
#pragma unroll
          for (int r = 0; r < R; ++r) ge[r] = g[r];
          has_erc = true;
        } else if (opc >= I_UN && opc < I_UN + NUNARY) {
          float* vx = V + (size_t)SLOT * ax.src_l;
          float x[R];
          load_rows<R>(vx, x);
          dun_rows<R>((int)(opc - I_UN), g, x);
          store_rows<R>(vx, x);
        } else if ((opc >= I_BF && opc < I_BS) || (POW && opc >= I_PW && opc < I_PWS)) {
          const bool pw = POW && opc >= I_PW;
          const int grp = pw ? (int)(opc - I_PW) : (int)(opc - I_BF) / NKIND;  // 0 BF, 1 BC, 2 LF, 3 LC
          const int kind = pw ? K_POW : (int)(opc - I_BF) % NKIND;
          float t[R], da[R], db[R];
          if (grp == 0 || grp == 2) {
            load_rows<R>(p.X + (size_t)feat * p.ldx + row0, t);
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r) t[r] = c;
          }
          float* vs = V + (size_t)SLOT * (grp <= 1 ? ax.src_l : ax.src_r);
          float v[R];
          load_rows<R>(vs, v);
          if (grp <= 1) {
            dbin_rows<R>(kind, v, t, da, db);
#pragma unroll
            for (int r = 0; r < R; ++r) {
              v[r] = g[r] * da[r];
              ge[r] = g[r] * db[r];
            }
          } else {
            dbin_rows<R>(kind, t, v, da, db);
#pragma unroll
            for (int r = 0; r < R; ++r) {
              v[r] = g[r] * db[r];
              ge[r] = g[r] * da[r];
            }
          }
          store_rows<R>(vs, v);
          has_erc = grp == 1 || grp == 3;
        } else if ((opc >= I_BS && opc < I_NOP) || (POW && opc >= I_PWS && opc < I_COUNT)) {
          const int kind = POW && opc >= I_PWS ? K_POW : (int)(opc - (opc < I_RS ? I_BS : I_RS));
          float* va = V + (size_t)SLOT * ax.src_l;
          float* vb = V + (size_t)SLOT * ax.src_r;
          float a[R], b[R], da[R], db[R];
          load_rows<R>(va, a);
          load_rows<R>(vb, b);
          dbin_rows<R>(kind, a, b, da, db);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            a[r] = g[r] * da[r];
            b[r] = g[r] * db[r];
          }
          store_rows<R>(va, a);
          store_rows<R>(vb, b);
        }
        if (has_erc) {  // warp-uniform: the same instruction on every lane
          // this lane's rows summed; the 32 lanes are summed after the sweep
          float sm = 0.f;
#pragma unroll
          for (int r = 0; r < R; ++r) sm += valid[r] ? ge[r] : 0.f;
          part[(size_t)eord[k] * 33 + lane] = sm;
        }
      }
      __syncwarp();
      reduce_erc(part, wg, n_erc, lane);
      __syncwarp();
    }
    write_grad(p, trial, wg, ek, n_erc, lane);
    __syncwarp();
  }
}

// ---- the staged kernel: 4 rows per lane, feature tile in shared memory ----

// The forward half as the PTX interpreter with a value tape: the
// instruction the PTX leaves is run and taped here.
template <int R, bool POW>
__device__ __forceinline__ void run_program_tape(const uint2* prog, const float* xs,
                                                 float (&A)[R], float* stk, float* tape) {
  uint32_t pc = smem_u32(prog), sp = smem_u32(stk), code = 0, arg = 0, tp = smem_u32(tape);
  const uint32_t xb = smem_u32(xs);
  for (;;) {
    interp_tape_asm<R>(A, pc, sp, xb, code, arg, tp);
    if (code == I_NOP || code >= I_COUNT) break;
    exec_cold<R, POW>(code, arg, A, sp, xs);
    store_rows<R>(static_cast<float*>(__cvta_shared_to_generic(tp)), A);
    tp += 32 * R * 4;
  }
}

// Reverse sweep of the staged kernel.  The accumulator discipline of the
// programs gives the sweep its shape: an instruction that reads A reads the
// value of the instruction just before it, so the adjoint of instruction
// k - 1 is produced by instruction k and is the next one the sweep needs.
// It stays in registers (G).  Only a value that was pushed (the instruction
// after it is PSF or PSC) is consumed later by a pop; its adjoint goes
// through V, and the descriptor says so (GSM).  A value has one consumer,
// so the operand values of the next instruction are never written by the
// current one: the sweep loads them one instruction ahead.
//
// Descriptors (only the instructions with work: a feature load propagates
// nothing): x = form | GSM | ERC ordinal << 7 | instruction << 16; y, z =
// byte offsets from the warp's shared-memory base of the two operand rows
// the form reads (a V entry or the feature's row in the tile; unused ones
// point at V's first entry); w = the constant's bits.  The PTX sweep
// (interp_rev_asm, generated by interp_gen.py) runs the forms of +, -, *,
// AQ, the pushed ERC and every unary operator (sin, cos and exp for a group
// within their range); rev_cold_v runs every form (the PTX leaves it
// division, pow and out-of-range groups).
enum : uint32_t {
  RV_CONST = 0,       // a pushed ERC: its adjoint is the ERC's contribution
  RV_UN = 1,          // + u (1..8)
  RV_BIN = 9,         // + group * 6 + kind: group 0 BF, 1 BC, 2 LF, 3 LC, 4 BS, 5 RS
  RV_COUNT = 45,
  RV_GSM = 64
};

// G <- g * d u(x) / dx: the forward kernels' own FP32 forms (the gradient
// is checked to 1e-3, far above their few-ulp error).
template <int R, int U>
__device__ __forceinline__ void rev_un(const float (&g)[R], const float (&xv)[R], float (&G)[R]) {
  float x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = xv[r];
  if constexpr (U == U_SIN || U == U_COS) {
    sincos_rows<R>(x, U == U_SIN ? 1 : 0);  // sin' = cos, cos' = -sin
#pragma unroll
    for (int r = 0; r < R; ++r) G[r] = U == U_SIN ? g[r] * x[r] : -(g[r] * x[r]);
  } else if constexpr (U == U_EXP) {
    exp_rows<R>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) G[r] = g[r] * x[r];
  } else if constexpr (U == U_LOG_ABS || U == U_LOG) {
#pragma unroll
    for (int r = 0; r < R; ++r) G[r] = g[r] * __frcp_rn(x[r]);
  } else if constexpr (U == U_SQRT_ABS) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      G[r] = x[r] == 0.f ? 0.f : g[r] * copysignf(0.5f * rsqrt_approx(fabsf(x[r])), x[r]);
  } else if constexpr (U == U_SQUARE) {
#pragma unroll
    for (int r = 0; r < R; ++r) G[r] = g[r] * (2.f * x[r]);
  } else {  // U_SQRT
#pragma unroll
    for (int r = 0; r < R; ++r) G[r] = g[r] * (0.5f * rsqrt_approx(x[r]));
  }
}

// A binary node kind(a, b) of group GR with operand rows u (at y) and v (at
// z): G <- the adjoint of its A operand; a popped operand's adjoint goes to
// its V entry; (BC / LC) its ERC's contribution summed over the lane's valid
// rows goes to *pe.
template <int R, int GR, int K>
__device__ __forceinline__ void rev_bin(const float (&g)[R], const float (&u)[R],
                                        const float (&v)[R], unsigned char* wl, const uint4 d,
                                        float* pe, const bool (&valid)[R], float (&G)[R]) {
  const float c = __uint_as_float(d.w);
  float a[R], b[R], da[R], db[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    // BF: (A, x)  BC: (A, c)  LF: (x, A)  LC: (c, A)  BS: (pop, A)  RS: (A, pop)
    a[r] = GR == 2 ? v[r] : GR == 3 ? c : u[r];
    b[r] = GR == 0 || GR == 4 || GR == 5 ? v[r] : GR == 1 ? c : u[r];
  }
  dbin_rows<R>(K, a, b, da, db);
  constexpr bool a_is_A = GR == 0 || GR == 1 || GR == 5;
#pragma unroll
  for (int r = 0; r < R; ++r) G[r] = g[r] * (a_is_A ? da[r] : db[r]);
  if constexpr (GR == 4 || GR == 5) {  // the popped operand
    float o[R];
#pragma unroll
    for (int r = 0; r < R; ++r) o[r] = g[r] * (GR == 4 ? da[r] : db[r]);
    store_rows<R>(reinterpret_cast<float*>(wl + (GR == 4 ? d.y : d.z)), o);
  }
  if constexpr (GR == 1 || GR == 3) {
    float sm = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) sm += valid[r] ? g[r] * (GR == 1 ? db[r] : da[r]) : 0.f;
    *pe = sm;
  }
}

// One descriptor in C++: every form (the PTX sweep leaves it the forms it
// does not run).  g is the carried adjoint G, or V's entry (GSM).  G goes
// in and out by value and the valid rows as a bit mask, so the caller's
// arrays keep their registers (nothing of theirs has its address taken).
template <bool POW>
__device__ __noinline__ ColdRows<4> rev_cold_v(const uint4 d, ColdRows<4> gin, unsigned char* wl,
                                               const float* V, float* pel, uint32_t vmask) {
  constexpr int R = 4;
  float G[R];
  bool valid[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    G[r] = gin.v[r];
    valid[r] = (vmask >> r) & 1u;
  }
  float g[R], u[R], v[R];
  if (d.x & RV_GSM) {
    load_rows<R>(V + (size_t)(d.x >> 16) * 32 * R, g);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) g[r] = G[r];
  }
  load_rows<R>(reinterpret_cast<const float*>(wl + d.y), u);
  load_rows<R>(reinterpret_cast<const float*>(wl + d.z), v);
  float* pe = pel + (size_t)((d.x >> 7) & 0x1ffu) * 33;
  switch (d.x & 0x3fu) {
    case RV_CONST: {
      float sm = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) sm += valid[r] ? g[r] : 0.f;
      *pe = sm;
      break;
    }
#define GG_RV_UN(U) \
  case RV_UN + U: rev_un<R, U>(g, u, G); break;
    GG_RV_UN(U_SIN) GG_RV_UN(U_COS) GG_RV_UN(U_EXP) GG_RV_UN(U_LOG_ABS)
    GG_RV_UN(U_SQRT_ABS) GG_RV_UN(U_SQUARE) GG_RV_UN(U_LOG) GG_RV_UN(U_SQRT)
#undef GG_RV_UN
#define GG_RV_BIN(GR, K) \
  case RV_BIN + GR * 6 + K: rev_bin<R, GR, K>(g, u, v, wl, d, pe, valid, G); break;
#define GG_RV_GRP(GR) \
  GG_RV_BIN(GR, K_ADD) GG_RV_BIN(GR, K_SUB) GG_RV_BIN(GR, K_MUL) GG_RV_BIN(GR, K_AQ) \
  GG_RV_BIN(GR, K_DIV)
    GG_RV_GRP(0) GG_RV_GRP(1) GG_RV_GRP(2) GG_RV_GRP(3) GG_RV_GRP(4) GG_RV_GRP(5)
#undef GG_RV_GRP
#undef GG_RV_BIN
    default:
      if constexpr (POW) {  // the pow forms
        switch ((d.x & 0x3fu) - RV_BIN) {
          case 0 * 6 + K_POW: rev_bin<R, 0, K_POW>(g, u, v, wl, d, pe, valid, G); break;
          case 1 * 6 + K_POW: rev_bin<R, 1, K_POW>(g, u, v, wl, d, pe, valid, G); break;
          case 2 * 6 + K_POW: rev_bin<R, 2, K_POW>(g, u, v, wl, d, pe, valid, G); break;
          case 3 * 6 + K_POW: rev_bin<R, 3, K_POW>(g, u, v, wl, d, pe, valid, G); break;
          case 4 * 6 + K_POW: rev_bin<R, 4, K_POW>(g, u, v, wl, d, pe, valid, G); break;
          case 5 * 6 + K_POW: rev_bin<R, 5, K_POW>(g, u, v, wl, d, pe, valid, G); break;
          default: break;
        }
      }
      break;
  }
  ColdRows<4> gout;
#pragma unroll
  for (int r = 0; r < R; ++r) gout.v[r] = G[r];
  return gout;
}

// The staged kernel (at most ADJ_FTILE_MAX features): per pass the lanes'
// rows of every feature go to a shared-memory tile, the forward recompute
// is the PTX interpreter with a value tape, and the reverse sweep walks
// precomputed descriptors.  Everything a lane touches during the sweep is
// its own, so the sweep needs no warp barrier.
template <bool POW>
__global__ void __launch_bounds__(256) adjoint_fast_kernel(const AdjParams p) {
  constexpr int R = 4;
  constexpr int SLOT = 32 * R;
  constexpr uint32_t SLOTB = SLOT * 4;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const AdjLayout lay = adj_layout(p.lcap, p.ecap, p.slots, R, true, p.F);
  unsigned char* base = smem + (size_t)warp * lay.total;
  uint2* sprog = reinterpret_cast<uint2*>(base + lay.prog);
  uint4* rins = reinterpret_cast<uint4*>(base + lay.rins);
  float2* wg = reinterpret_cast<float2*>(base + lay.wg);
  uint16_t* ek = reinterpret_cast<uint16_t*>(base + lay.ek);
  unsigned char* wl = base + (size_t)lane * R * 4;  // the warp's base + this lane's row offset
  float* V = reinterpret_cast<float*>(wl + lay.V);
  float* stk = reinterpret_cast<float*>(wl + lay.stk);
  float* part = reinterpret_cast<float*>(base + lay.part);
  float* partl = part + lane;
  float* xt = reinterpret_cast<float*>(wl + lay.xt);
  const uint32_t oV = (uint32_t)lay.V, oX = (uint32_t)lay.xt;
  const uint32_t wl32 = smem_u32(wl), pe32 = smem_u32(partl), rbase = smem_u32(rins);
  const Chunking ch = chunking(p, *p.count, SLOT);

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(p.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= ch.n_items) break;
    const int trial = p.list[item / ch.n_chunks];
    const int chunk = item % ch.n_chunks;
    if (adj_skip(p, trial)) continue;
    const int L = p.len[trial];
    const double* ab = p.ab + 4 * (size_t)trial;
    const uint2* src = p.prog + (size_t)trial * p.lstride;
    const Aux* asrc = p.aux + (size_t)trial * p.lstride;
    // stage: the interpreter's form of the program, and in program order
    // the ERC ordinals and the descriptors of the instructions with work
    int n_erc = 0, n_rev = 0;
    uint32_t fmask = 0;  // the features the program reads (at most ADJ_FTILE_MAX)
    for (int k0 = 0; k0 <= L; k0 += 32) {
      const int k = k0 + lane;
      bool has = false, work = false;
      uint4 d = make_uint4(0u, oV, oV, 0u);
      uint16_t tpos = NONE16;
      if (k <= L) {
        const uint2 w = src[k];
        const uint32_t opc = w.x & 0xffu;
        if (k < L && reads_feature(opc)) fmask |= 1u << (w.x >> 8);
        const uint32_t f = w.x >> 8;
        sprog[k] = make_uint2(opc, reads_feature(opc) ? f * SLOTB : w.y);
        if (k < L) {
          const Aux ax = asrc[k];
          const uint32_t next = src[k + 1].x & 0xffu;
          has = carries_erc<POW>(opc);
          tpos = (opc == I_LDC0 || opc == I_PSC) ? ax.tpos : ax.tpos_fused;
          const uint32_t sl = oV + (uint32_t)ax.src_l * SLOTB, sr = oV + (uint32_t)ax.src_r * SLOTB;
          const uint32_t fo = oX + f * SLOTB;
          uint32_t rop = RV_COUNT;
          if (opc == I_LDC0 || opc == I_PSC) {
            rop = RV_CONST;
          } else if (opc >= I_UN && opc < I_UN + NUNARY) {
            rop = RV_UN + (opc - I_UN);
            d.y = sl;
          } else if ((opc >= I_BF && opc < I_BS) || (POW && opc >= I_PW && opc < I_PWS)) {
            const bool pw = POW && opc >= I_PW;
            const uint32_t grp = pw ? opc - I_PW : (opc - I_BF) / NKIND;
            const uint32_t kind = pw ? (uint32_t)K_POW : (opc - I_BF) % NKIND;
            rop = RV_BIN + grp * 6 + kind;
            d.y = grp <= 1 ? sl : sr;  // the A operand
            if (grp == 0 || grp == 2) d.z = fo;
            d.w = w.y;
          } else if ((opc >= I_BS && opc < I_NOP) || (POW && opc >= I_PWS && opc < I_COUNT)) {
            const bool rs = POW && opc >= I_PWS ? opc == I_PWR : opc >= I_RS;
            const uint32_t kind =
                POW && opc >= I_PWS ? (uint32_t)K_POW : opc - (opc < I_RS ? I_BS : I_RS);
            rop = RV_BIN + (rs ? 5u : 4u) * 6 + kind;
            d.y = sl;
            d.z = sr;
          }
          work = rop != RV_COUNT;
          d.x = rop | ((next == I_PSF || next == I_PSC) ? RV_GSM : 0u) | ((uint32_t)k << 16);
        }
      }
      const unsigned me = __ballot_sync(0xffffffffu, has);
      const unsigned mw = __ballot_sync(0xffffffffu, work);
      const unsigned below = (1u << lane) - 1u;
      if (has) {
        const int o = n_erc + __popc(me & below);
        ek[o] = tpos;
        wg[o] = make_float2(0.f, 0.f);
        d.x |= (uint32_t)o << 7;
      }
      if (work) rins[n_rev + __popc(mw & below)] = d;
      n_erc += __popc(me);
      n_rev += __popc(mw);
    }
    if (lane == 0) sprog[L + 1] = make_uint2(I_NOP, 0u);  // read ahead, never run
    fmask = __reduce_or_sync(0xffffffffu, fmask);
    __syncwarp();

    const int r_beg = chunk * ch.chunk_rows;
    const int r_end = min(p.N, r_beg + ch.chunk_rows);
    for (int rb = r_beg; rb < r_end; rb += SLOT) {
      const int row0 = min(rb + lane * R, (r_end - 1) & ~(R - 1));
      bool valid[R];
#pragma unroll
      for (int r = 0; r < R; ++r) valid[r] = rb + lane * R + r < r_end;
      // only the feature rows the program reads (a short program reads a
      // few of them; the others' tile rows are never addressed)
      for (uint32_t m = fmask; m != 0; m &= m - 1) {
        const int f = __ffs(m) - 1;
        float v[R];
        load_rows<R>(p.X + (size_t)f * p.ldx + row0, v);
        store_rows<R>(xt + (size_t)f * SLOT, v);
      }
      float yc[R], yl[R], G[R];
      load_rows<R>(p.X + (size_t)p.F * p.ldx + row0, yc);
      load_rows<R>(p.ylo + row0, yl);
      float A[R];
#pragma unroll
      for (int r = 0; r < R; ++r) A[r] = 0.f;
      run_program_tape<R, POW>(sprog, xt, A, stk, V);
      // the stack's bytes are also the ERC partials, which the sweep writes
      // across lanes: every lane leaves the forward recompute first
      __syncwarp();
      seed_rows<R>(p, ab, A, yc, yl, valid, G);  // the root's adjoint, in registers
      if (n_rev > 0) {
        uint32_t vmask = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) vmask |= valid[r] ? 1u << r : 0u;
        uint32_t rp = smem_u32(rins + (n_rev - 1)), cnt = (uint32_t)n_rev;
        for (;;) {
          uint32_t code, dx, dy, dz, dw;
          interp_rev_asm(G, rp, cnt, code, dx, dy, dz, dw, wl32, wl32 + oV, pe32, rbase, vmask);
          if (code == 0) break;
          ColdRows<4> gc;
#pragma unroll
          for (int r = 0; r < R; ++r) gc.v[r] = G[r];
          gc = rev_cold_v<POW>(make_uint4(dx, dy, dz, dw), gc, wl, V, partl, vmask);
#pragma unroll
          for (int r = 0; r < R; ++r) G[r] = gc.v[r];
        }
      }
      __syncwarp();
      reduce_erc(part, wg, n_erc, lane);
      __syncwarp();
    }
    write_grad(p, trial, wg, ek, n_erc, lane);
    __syncwarp();
  }
}

// Bins the trials of a batch by program length into the length classes.
__global__ void __launch_bounds__(256) adj_bin_kernel(const AdjBinParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.P) return;
  const int L = p.len[t];
  if (L <= 0) return;
  const double* ab = p.ab + 4 * (size_t)t;
  if (ab[2] == 0.0 || (!p.mse_mode && ab[1] == 0.0)) return;
  int c = 0;
  while (c < p.ncls - 1 && L + 1 > p.caps[c]) ++c;
  const int pos = atomicAdd(p.count + c, 1);
  p.list[(size_t)c * p.P + pos] = t;
}

const void* adj_ptr(int rows, bool pow, bool fast) {
  if (fast) return pow ? reinterpret_cast<const void*>(&adjoint_fast_kernel<true>)
                       : reinterpret_cast<const void*>(&adjoint_fast_kernel<false>);
  switch (rows) {
    case 4: return pow ? reinterpret_cast<const void*>(&adjoint_kernel<4, true>)
                       : reinterpret_cast<const void*>(&adjoint_kernel<4, false>);
    case 2: return pow ? reinterpret_cast<const void*>(&adjoint_kernel<2, true>)
                       : reinterpret_cast<const void*>(&adjoint_kernel<2, false>);
    default: return pow ? reinterpret_cast<const void*>(&adjoint_kernel<1, true>)
                        : reinterpret_cast<const void*>(&adjoint_kernel<1, false>);
  }
}

const void* adj_bin_ptr() { return reinterpret_cast<const void*>(&adj_bin_kernel); }

}  // namespace gg
