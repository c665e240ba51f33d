// Reverse-mode adjoint: d(scaled MSE)/d(constant) for every ERC leaf of
// every trial.
//
// Work item = (trial, chunk of rows); warps claim items from a global
// counter.  For 32 rows at a time (one per lane) a warp re-runs the trial's
// program forward, storing the value of every instruction in a shared-memory
// array V, seeds the output adjoint with
//   w_i = (2 b*/N) (a* + b* f_i - y_i)          (scaled MSE; envelope theorem)
//   w_i = (2/N) (f_i - y_i)                     (plain MSE)
// and sweeps the program backwards.  Every instruction's value has exactly
// one consumer (the program is a tree), so when the sweep reaches an
// instruction it reads its operands' values from V and overwrites them with
// their adjoints; by the time an operand instruction is reached, V holds its
// adjoint while its own operands still hold values.  The operators whose
// derivative uses their own output (exp, sqrt, division) recompute it from
// the operands.  The contribution of an ERC (pushed, or fused into its
// parent) is summed over the warp's 32 rows with shuffles and added into a
// per-warp error-free FP32 (hi, lo) accumulator; at the end of the item the
// accumulators go to the trial's FP64 gradient row with atomics.  Node
// values live only in shared memory for 32 rows at a time: nothing of size
// rows x nodes is stored in HBM, so any dataset size works (recomputation
// instead of storage).  The paper evaluates fitness only; this kernel is an
// addition.
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
        const float q = rsqrtf(fmaf(b[r], b[r], 1.f));
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

// R rows per lane: each lane runs rows row0 .. row0 + R - 1 of a 32 R-row
// group (feature-major X, so a lane's rows are one aligned R-wide load).
// Values and adjoints live at V[instruction][lane][row]; rows past the
// chunk's end are evaluated on in-bounds data and left out of every sum.
// The forward half as the PTX interpreter with a value tape (4 rows per
// lane): the instruction the PTX leaves is run and taped here.
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

// FAST (4 rows per lane, at most ADJ_FTILE_MAX features): each pass stages
// the lanes' rows of every feature into a shared-memory tile and runs the
// forward half with the PTX interpreter (run_program_tape); otherwise the
// C++ interpreter reads the features from global memory.
template <int R, bool POW, bool FAST>
__global__ void __launch_bounds__(256) adjoint_kernel(const AdjParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int SLOT = 32 * R;
  const int ftile = FAST ? p.F : 0;
  unsigned char* base = smem + (size_t)warp * adj_warp_bytes(p.lstride, p.slots, R, ftile);
  uint2* wprog = reinterpret_cast<uint2*>(base);
  Aux* waux = reinterpret_cast<Aux*>(wprog + p.lstride);
  float2* wg = reinterpret_cast<float2*>(waux + p.lstride);  // (hi, lo) per ERC ordinal
  uint16_t* eord = reinterpret_cast<uint16_t*>(wg + p.lstride);  // instruction -> ordinal
  uint16_t* ek = eord + p.lstride;                                // ordinal -> instruction
  float* V0 = reinterpret_cast<float*>(base + adj_head_bytes(p.lstride));
  float* V = V0 + lane * R;                                  // [lstride][32][R]
  float* stk = V + (size_t)p.lstride * SLOT;                 // [slots][32][R]
  float* part = V0 + (size_t)(p.lstride + p.slots) * SLOT;   // [lstride / 2][33]
  // FAST: the staged program and the feature tile [F][32][R], after the above
  unsigned char* fast_base =
      base + ((adj_head_bytes(p.lstride) + (size_t)p.lstride * 32 * 4 * R +
               (size_t)p.slots * 32 * 4 * R + (size_t)(p.lstride / 2) * 33 * 4 + 15) &
              ~(size_t)15);
  uint2* sprog = reinterpret_cast<uint2*>(fast_base);
  float* xt = reinterpret_cast<float*>(fast_base + (((size_t)(p.lstride + 1) * 8 + 15) &
                                                    ~(size_t)15));  // 16-byte aligned

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(p.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= p.n_items) break;
    const int trial = item / p.n_chunks;
    const int chunk = item - trial * p.n_chunks;
    const int L = p.len[trial];
    if (L <= 0) continue;
    const double* ab = p.ab + 4 * (size_t)trial;
    if (ab[2] == 0.0 || (!p.mse_mode && ab[1] == 0.0)) continue;
    // a* - mean(y), b* and mean(y) as FP32 (hi, lo) pairs of their FP64 values
    const float a_hi = (float)ab[0], a_lo = (float)(ab[0] - (double)a_hi);
    const float b_hi = (float)ab[1], b_lo = (float)(ab[1] - (double)b_hi);
    const float yb_hi = (float)p.ybar, yb_lo = (float)(p.ybar - (double)yb_hi);
    const float two_n = (float)(2.0 / (double)p.N);
    const uint2* src = p.prog + (size_t)trial * p.lstride;
    const Aux* asrc = p.aux + (size_t)trial * p.lstride;
    for (int k = lane; k <= L; k += 32) {
      const uint2 w = src[k];
      wprog[k] = w;
      waux[k] = asrc[k];
      wg[k] = make_float2(0.f, 0.f);
      if constexpr (FAST) {  // the interpreter's staged form: bare opcode, feature byte offset
        const uint32_t op = w.x & 0xffu;
        sprog[k] = make_uint2(op, reads_feature(op) ? (w.x >> 8) * (uint32_t)(SLOT * 4) : w.y);
      }
    }
    if (FAST && lane == 0) sprog[L + 1] = make_uint2(I_NOP, 0u);  // read ahead, never run
    __syncwarp();
    // ordinals of the instructions that carry an ERC, in program order
    int n_erc = 0;
    for (int k0 = 0; k0 < L; k0 += 32) {
      const int k = k0 + lane;
      const bool has = k < L && carries_erc<POW>(wprog[k].x & 0xffu);
      const unsigned m = __ballot_sync(0xffffffffu, has);
      if (has) {
        const int o = n_erc + __popc(m & ((1u << lane) - 1u));
        eord[k] = (uint16_t)o;
        ek[o] = (uint16_t)k;
      }
      n_erc += __popc(m);
    }
    __syncwarp();

    const int r_beg = chunk * p.chunk_rows;
    const int r_end = min(p.N, r_beg + p.chunk_rows);
    for (int rb = r_beg; rb < r_end; rb += SLOT) {
      // this lane's first row, kept in bounds (and R-aligned) past the end
      const int row0 = min(rb + lane * R, (r_end - 1) & ~(R - 1));
      bool valid[R];
#pragma unroll
      for (int r = 0; r < R; ++r) valid[r] = rb + lane * R + r < r_end;
      float A[R];
#pragma unroll
      for (int r = 0; r < R; ++r) A[r] = 0.f;
      if constexpr (FAST) {
        for (int f = 0; f < p.F; ++f) {
          float v[R];
          load_rows<R>(p.X + (size_t)f * p.ldx + row0, v);
          store_rows<R>(xt + (size_t)f * SLOT + lane * R, v);
        }
        __syncwarp();
        run_program_tape<R, POW>(sprog, xt + lane * R, A, stk, V);
      } else {
        run_program<R, true, false, POW>(wprog, L, p.X + row0, p.ldx, A, stk, V);
      }
      float yc[R], yl[R];
      load_rows<R>(p.X + (size_t)p.F * p.ldx + row0, yc);
      load_rows<R>(p.ylo + row0, yl);
      float w[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // the residual a* + b* f - y (smse) or f - y (mse) in double-float:
        // TwoProd / TwoSum keep the rounding of every term, so only f's own
        // FP32 error remains (y = mean(y) + yc + yl exactly to FP64 accuracy)
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
      store_rows<R>(V + (size_t)SLOT * (L - 1), w);  // the output's value becomes its adjoint
      __syncwarp();
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
        __syncwarp();
      }
      // the pass's ERC sums: lane o adds up the 32 lane partials of the ERCs
      // o, o + 32, ... (rows padded to 33 floats: no bank conflicts) into
      // its error-free accumulators (one transposed reduction per pass
      // instead of a shuffle reduction per ERC instruction)
      for (int o = lane; o < n_erc; o += 32) {
        const float* q = part + (size_t)o * 33;
        float sm = 0.f;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) sm += q[j];
        float2 acc = wg[o];
        acc_add(acc.x, acc.y, sm);
        wg[o] = acc;
      }
      __syncwarp();
    }
    __syncwarp();
    for (int o = lane; o < n_erc; o += 32) {
      const int k = ek[o];
      const uint32_t opc = wprog[k].x & 0xffu;
      const int tp = (opc == I_LDC0 || opc == I_PSC) ? waux[k].tpos : waux[k].tpos_fused;
      const double gk = (double)wg[o].x + (double)wg[o].y;
      if (tp != NONE16 && gk != 0.0) atomicAdd(p.gacc + (size_t)trial * p.stride + tp, gk);
    }
    __syncwarp();
  }
}

const void* adj_ptr(int rows, bool pow, bool fast) {
  switch (rows) {
    case 4:
      if (fast)
        return pow ? reinterpret_cast<const void*>(&adjoint_kernel<4, true, true>)
                   : reinterpret_cast<const void*>(&adjoint_kernel<4, false, true>);
      return pow ? reinterpret_cast<const void*>(&adjoint_kernel<4, true, false>)
                 : reinterpret_cast<const void*>(&adjoint_kernel<4, false, false>);
    case 2: return pow ? reinterpret_cast<const void*>(&adjoint_kernel<2, true, false>)
                       : reinterpret_cast<const void*>(&adjoint_kernel<2, false, false>);
    default: return pow ? reinterpret_cast<const void*>(&adjoint_kernel<1, true, false>)
                        : reinterpret_cast<const void*>(&adjoint_kernel<1, false, false>);
  }
}

}  // namespace gg
