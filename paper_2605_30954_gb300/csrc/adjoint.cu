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

__device__ __forceinline__ void dbin(int kind, float a, float b, float& da, float& db) {
  switch (kind) {
    case K_ADD: da = 1.f; db = 1.f; break;
    case K_SUB: da = 1.f; db = -1.f; break;
    case K_MUL: da = b; db = a; break;
    case K_AQ: {
      const float q = rsqrtf(fmaf(b, b, 1.f));
      da = q;
      db = -a * b * q * q * q;
      break;
    }
    case K_POW: {  // d/da = b a^(b-1); d/db = a^b ln|a| (0 where a^b = 0)
      const float out = powf(a, b);
      da = b * powf(a, b - 1.f);
      db = out == 0.f ? 0.f : out * logf(fabsf(a));
      break;
    }
    default: {  // K_DIV: d/da = 1/b, d/db = -(a/b)/b
      da = 1.f / b;
      db = -(a / b) / b;
      break;
    }
  }
}

__device__ __forceinline__ float dun(int u, float x) {
  switch (u) {
    case U_SIN: return cosf(x);
    case U_COS: return -sinf(x);
    case U_EXP: return expf(x);
    case U_LOG_ABS:
    case U_LOG: return 1.f / x;
    case U_SQRT_ABS: return x == 0.f ? 0.f : copysignf(0.5f / sqrtf(fabsf(x)), x);
    case U_SQUARE: return 2.f * x;
    default: return 0.5f / sqrtf(x);  // U_SQRT
  }
}

template <bool POW>
__global__ void __launch_bounds__(256) adjoint_kernel(const AdjParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* base = smem + (size_t)warp * adj_warp_bytes(p.lstride, p.slots);
  uint2* wprog = reinterpret_cast<uint2*>(base);
  Aux* waux = reinterpret_cast<Aux*>(wprog + p.lstride);
  float2* wg = reinterpret_cast<float2*>(waux + p.lstride);  // (hi, lo) per instruction
  float* V = reinterpret_cast<float*>(wg + p.lstride);      // [lstride][32]
  float* stk = V + (size_t)p.lstride * 32 + lane;            // [slots][32], this lane

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
    const float a_c = (float)ab[0];
    const float bb = (float)ab[1];
    const float two_n = (float)(2.0 / (double)p.N);
    const float ybar = (float)p.ybar;
    const uint2* src = p.prog + (size_t)trial * p.lstride;
    const Aux* asrc = p.aux + (size_t)trial * p.lstride;
    for (int k = lane; k <= L; k += 32) {
      wprog[k] = src[k];
      waux[k] = asrc[k];
      wg[k] = make_float2(0.f, 0.f);
    }
    __syncwarp();

    const int r_beg = chunk * p.chunk_rows;
    const int r_end = min(p.N, r_beg + p.chunk_rows);
    for (int rb = r_beg; rb < r_end; rb += 32) {
      const int row = rb + lane;
      const bool valid = row < r_end;
      const int rr = valid ? row : r_end - 1;
      float A[1] = {0.f};
      run_program<1, true, false, POW>(wprog, L, p.X + rr, p.ldx, A, stk, V + lane);
      const float f = A[0];
      const float yc = p.X[(size_t)p.F * p.ldx + rr];
      float w = p.mse_mode ? two_n * (f - ybar - yc) : two_n * bb * (a_c + bb * f - yc);
      V[32 * (L - 1) + lane] = valid ? w : 0.f;  // the output's value becomes its adjoint
      __syncwarp();
      for (int k = L - 1; k >= 0; --k) {
        const uint2 ins = wprog[k];
        const Aux ax = waux[k];
        const uint32_t opc = ins.x & 0xffu;
        const int feat = (int)(ins.x >> 8);
        const float c = __uint_as_float(ins.y);
        const float g = V[32 * k + lane];  // adjoint of instruction k
        float ge = 0.f;                    // contribution to this instruction's ERC
        bool has_erc = false;
        if (opc == I_LDF0 || opc == I_PSF) {
          // feature load: nothing to propagate
        } else if (opc == I_LDC0 || opc == I_PSC) {
          ge = g;
          has_erc = true;
        } else if (opc >= I_UN && opc < I_UN + NUNARY) {
          float* vx = &V[32 * ax.src_l + lane];
          *vx = g * dun((int)(opc - I_UN), *vx);
        } else if ((opc >= I_BF && opc < I_BS) || (POW && opc >= I_PW && opc < I_PWS)) {
          const bool pw = POW && opc >= I_PW;
          const int grp = pw ? (int)(opc - I_PW) : (int)(opc - I_BF) / NKIND;  // 0 BF, 1 BC, 2 LF, 3 LC
          const int kind = pw ? K_POW : (int)(opc - I_BF) % NKIND;
          float da, db;
          if (grp <= 1) {
            float* va = &V[32 * ax.src_l + lane];
            const float b = grp == 0 ? p.X[(size_t)feat * p.ldx + rr] : c;
            dbin(kind, *va, b, da, db);
            *va = g * da;
            if (grp == 1) {
              ge = g * db;
              has_erc = true;
            }
          } else {
            float* vb = &V[32 * ax.src_r + lane];
            const float a = grp == 2 ? p.X[(size_t)feat * p.ldx + rr] : c;
            dbin(kind, a, *vb, da, db);
            *vb = g * db;
            if (grp == 3) {
              ge = g * da;
              has_erc = true;
            }
          }
        } else if ((opc >= I_BS && opc < I_NOP) || (POW && opc >= I_PWS && opc < I_COUNT)) {
          const int kind = POW && opc >= I_PWS ? K_POW : (int)(opc - (opc < I_RS ? I_BS : I_RS));
          float* va = &V[32 * ax.src_l + lane];
          float* vb = &V[32 * ax.src_r + lane];
          float da, db;
          dbin(kind, *va, *vb, da, db);
          *va = g * da;
          *vb = g * db;
        }
        if (has_erc) {  // warp-uniform: the same instruction on every lane
          float sm = valid ? ge : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
          if (lane == 0) {
            float2 acc = wg[k];
            acc_add(acc.x, acc.y, sm);
            wg[k] = acc;
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();
    for (int k = lane; k < L; k += 32) {
      const uint32_t opc = wprog[k].x & 0xffu;
      int tp = -1;
      if (opc == I_LDC0 || opc == I_PSC) tp = waux[k].tpos;
      else if ((opc >= I_BC && opc < I_BC + NKIND) || (opc >= I_LC && opc < I_LC + NKIND) ||
               (POW && (opc == I_PW + 1 || opc == I_PW + 3)))
        tp = waux[k].tpos_fused;
      const double gk = (double)wg[k].x + (double)wg[k].y;
      if (tp >= 0 && tp != NONE16 && gk != 0.0)
        atomicAdd(p.gacc + (size_t)trial * p.stride + tp, gk);
    }
    __syncwarp();
  }
}

const void* adj_ptr(bool pow) {
  return pow ? reinterpret_cast<const void*>(&adjoint_kernel<true>)
             : reinterpret_cast<const void*>(&adjoint_kernel<false>);
}

}  // namespace gg
