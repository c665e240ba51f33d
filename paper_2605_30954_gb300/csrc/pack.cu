// The device packer: one warp per trial turns a template into the
// interpreter's program (Section 3.2 linearises a tree to RPN with the
// introns skipped; Fig. 1).  It computes, level by level with the lanes
// spread over the nodes of a level, exactly the program the sequential
// packer pack_tree (isa.h) emits:
//   A  top-down: the active set (Section 3.1: the root is active; both
//      children of an active binary function, the left child of an active
//      unary one), with the validation of active nodes;
//   B  bottom-up: constant subtrees and their folded values, whether a node
//      is emitted as a terminal, which terminal child a binary node fuses
//      (the right one if it is a terminal, else the left one), the
//      Sethi-Ullman stack need and the instruction count of each subtree;
//   C  top-down: the index of each subtree's first instruction (post-order,
//      the child needing more stack first), and the nodes below a folded
//      subtree's root;
//   D  every emitted node writes its own instruction at the index where its
//      subtree ends.
// A terminal load pushes A exactly when it is not the program's first
// instruction: in post-order every earlier result is still waiting for its
// consumer.  Nodes are addressed in heap order; for the prefix layout each
// node's template position is computed from its path.
#include "misc.cuh"

namespace gg {

// The interpreter's own operator functions for constant folding: unop_rows
// with one row picks the same code path as R equal rows do, and binop is
// the interpreter's binary operator, so a folded constant is bit-identical
// to the value the interpreter would compute on every row.
struct DevFold {
  __device__ float un(int u, float a) const {
    float v[1] = {a};
    switch (u) {
      case U_SIN: unop_rows<U_SIN, 1>(v); break;
      case U_COS: unop_rows<U_COS, 1>(v); break;
      case U_EXP: unop_rows<U_EXP, 1>(v); break;
      case U_LOG_ABS: unop_rows<U_LOG_ABS, 1>(v); break;
      case U_SQRT_ABS: unop_rows<U_SQRT_ABS, 1>(v); break;
      case U_SQUARE: unop_rows<U_SQUARE, 1>(v); break;
      case U_LOG: unop_rows<U_LOG, 1>(v); break;
      default: unop_rows<U_SQRT, 1>(v); break;
    }
    return v[0];
  }
  __device__ float bin(int k, float a, float b) const {
    switch (k) {
      case K_ADD: return binop<K_ADD>(a, b);
      case K_SUB: return binop<K_SUB>(a, b);
      case K_MUL: return binop<K_MUL>(a, b);
      case K_AQ: return binop<K_AQ>(a, b);
      case K_DIV: return binop<K_DIV>(a, b);
      default: return binop<K_POW>(a, b);
    }
  }
};

// per-node flags
constexpr uint8_t N_ACT = 1;      // active
constexpr uint8_t N_CONST = 2;    // constant subtree (folded when emitted)
constexpr uint8_t N_TERM = 4;     // emitted as a terminal (incl. a folded subtree)
constexpr uint8_t N_INSIDE = 8;   // below a folded subtree's root: not emitted
constexpr uint8_t N_RFIRST = 16;  // two subtrees, the right one evaluated first
constexpr uint8_t N_FUSED = 32;   // terminal fused into its parent's instruction

__global__ void __launch_bounds__(PACK_WARPS * 32) pack_kernel(const PackParams p) {
  extern __shared__ __align__(16) unsigned char pk_smem[];
  allow_dependents();  // the forward kernel's prologue needs nothing from here
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = blockIdx.x * PACK_WARPS + warp;  // the program slot
  if (t >= p.n || (p.count && t >= *p.count)) return;  // the whole warp
  const int trial = p.count ? p.idx[t] : t;
  const int S = p.stride;
  unsigned char* base = pk_smem + (size_t)warp * pack_warp_bytes(S);
  float* fv = reinterpret_cast<float*>(base);
  float* cv = fv + S;
  int16_t* size = reinterpret_cast<int16_t*>(cv + S);
  int16_t* start = size + S;
  int16_t* orig = start + S;
  uint8_t* cls = reinterpret_cast<uint8_t*>(orig + S);
  uint8_t* kind = cls + S;
  uint8_t* fl = kind + S;
  uint8_t* need = fl + S;

  const int h = p.height ? (int)p.height[trial] : p.h_max;
  auto invalid = [&]() {
    if (lane == 0) {
      p.len[t] = -1;
      if (p.size_active) p.size_active[trial] = -1;
      if (p.size_eval) p.size_eval[trial] = -1;
      atomicOr(p.status, ST_TEMPLATE);
    }
  };
  if (h < 0 || h > p.h_max) {
    invalid();
    return;
  }
  const int n = (1 << (h + 1)) - 1;
  const bool fold = p.fold && !p.aux;
  const uint8_t* gop = p.op + (size_t)trial * S;
  const float* gcv = p.cval + (size_t)trial * S;
  for (int i = lane; i < n; i += 32) {
    const int o = p.layout ? prefix_position(i, h) : i;
    int k;
    const int c = classify(gop[o], p.n_features, &k);
    orig[i] = (int16_t)o;
    cls[i] = (uint8_t)c;
    kind[i] = (uint8_t)k;
    cv[i] = gcv[o];
    fl[i] = i == 0 ? N_ACT : 0;
    need[i] = 0;
    size[i] = 0;
    start[i] = 0;
  }
  __syncwarp();

  // A: active set and validation, top-down
  bool bad = false;
  for (int d = 0; d <= h; ++d) {
    for (int i = (1 << d) - 1 + lane; i < (1 << (d + 1)) - 1; i += 32) {
      if (!(fl[i] & N_ACT)) continue;
      const int c = cls[i];
      if (c == C_BAD || ((c == C_UNARY || c == C_BINARY) && d >= h) ||
          (c == C_BINARY && kind[i] == K_POW && !p.allow_pow)) {
        bad = true;
        continue;
      }
      if (c == C_UNARY || c == C_BINARY) {
        fl[2 * i + 1] = N_ACT;
        if (c == C_BINARY) fl[2 * i + 2] = N_ACT;
      }
    }
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, bad)) {
    invalid();
    return;
  }
  if (p.size_active) {  // the trial's size: its active node count
    int cnt = 0;
    for (int i = lane; i < n; i += 32) cnt += (fl[i] & N_ACT) != 0;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) p.size_active[trial] = cnt;
  }

  // B: constants, fusion, stack need and instruction counts, bottom-up
  const DevFold ev;
  for (int d = h; d >= 0; --d) {
    for (int i = (1 << d) - 1 + lane; i < (1 << (d + 1)) - 1; i += 32) {
      uint8_t f = fl[i];
      if (!(f & N_ACT)) continue;
      const int c = cls[i];
      int sz = 1, nd = 0;
      if (c == C_TERM_F) {
        f |= N_TERM;
      } else if (c == C_TERM_C) {
        f |= N_TERM | N_CONST;
        fv[i] = cv[i];
      } else {
        const int l = 2 * i + 1, r = 2 * i + 2;
        const uint8_t fll = fl[l];
        if (c == C_UNARY) {
          if (fold && (fll & N_CONST)) {
            f |= N_TERM | N_CONST;
            fv[i] = ev.un(kind[i], fv[l]);
          } else {
            nd = need[l];
            sz = size[l] + 1;
          }
        } else {
          const uint8_t flr = fl[r];
          if (fold && (fll & N_CONST) && (flr & N_CONST)) {
            f |= N_TERM | N_CONST;
            fv[i] = ev.bin(kind[i], fv[l], fv[r]);
          } else if ((flr & N_TERM) || (fll & N_TERM)) {
            const bool rt = (flr & N_TERM) != 0;
            const int sub = rt ? l : r;
            fl[rt ? r : l] = (rt ? flr : fll) | N_FUSED;
            nd = need[sub];
            sz = size[sub] + 1;
          } else {
            const int a = need[l], b = need[r];
            if (a < b) f |= N_RFIRST;
            nd = a >= b ? (a > b + 1 ? a : b + 1) : (b > a + 1 ? b : a + 1);
            sz = size[l] + size[r] + 1;
          }
        }
      }
      fl[i] = f;
      need[i] = (uint8_t)nd;
      size[i] = (int16_t)sz;
    }
    __syncwarp();
  }
  const int L = size[0];
  if (L > p.lstride - 1 || need[0] > p.max_slots) {
    invalid();
    return;
  }

  // C: first instruction of every emitted subtree, top-down
  if (lane == 0) start[0] = 0;
  __syncwarp();
  for (int d = 0; d < h; ++d) {
    for (int i = (1 << d) - 1 + lane; i < (1 << (d + 1)) - 1; i += 32) {
      const uint8_t f = fl[i];
      const int c = cls[i];
      if (!(f & N_ACT) || (c != C_UNARY && c != C_BINARY)) continue;
      const int l = 2 * i + 1, r = 2 * i + 2;
      if (f & (N_TERM | N_INSIDE)) {  // a folded subtree: nothing below is emitted
        fl[l] |= N_INSIDE;
        if (c == C_BINARY) fl[r] |= N_INSIDE;
        continue;
      }
      const int s = start[i];
      if (c == C_UNARY) {
        start[l] = (int16_t)s;
      } else if (fl[r] & N_FUSED) {
        start[l] = (int16_t)s;
      } else if (fl[l] & N_FUSED) {
        start[r] = (int16_t)s;
      } else {
        const int first = (f & N_RFIRST) ? r : l;
        const int second = (f & N_RFIRST) ? l : r;
        start[first] = (int16_t)s;
        start[second] = (int16_t)(s + size[first]);
      }
    }
    __syncwarp();
  }

  if (p.size_eval) {  // nodes evaluated per row: active ones not inside a folded subtree
    int cnt = 0;
    for (int i = lane; i < n; i += 32) cnt += (fl[i] & N_ACT) && !(fl[i] & N_INSIDE);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) p.size_eval[trial] = cnt;
  }

  // D: emission
  uint32_t* words = reinterpret_cast<uint32_t*>(p.prog + (size_t)t * p.lstride);
  float* consts = reinterpret_cast<float*>(words) + 1;
  Aux* aux = p.aux ? p.aux + (size_t)t * p.lstride : nullptr;
  for (int i = lane; i < n; i += 32) {
    const uint8_t f = fl[i];
    if (!(f & N_ACT) || (f & (N_INSIDE | N_FUSED))) continue;
    const int idx = start[i] + size[i] - 1;
    const int c = cls[i];
    uint32_t opc;
    int feat = 0, sl = -1, sr = -1, tf = -1;
    float val = 0.f;
    if (f & N_TERM) {
      const bool isf = c == C_TERM_F;
      opc = idx == 0 ? (isf ? I_LDF0 : I_LDC0) : (isf ? I_PSF : I_PSC);
      if (isf) feat = kind[i];
      else val = c == C_TERM_C ? cv[i] : fv[i];
    } else {
      const int l = 2 * i + 1, r = 2 * i + 2;
      const int il = start[l] + size[l] - 1;
      if (c == C_UNARY) {
        opc = I_UN + (uint32_t)kind[i];
        sl = il;
      } else {
        const bool rfused = (fl[r] & N_FUSED) != 0;
        const bool lfused = !rfused && (fl[l] & N_FUSED);
        if (rfused || lfused) {
          const int term = rfused ? r : l;
          const bool isf = cls[term] == C_TERM_F;
          const int group = rfused ? (isf ? 0 : 1) : (isf ? 2 : 3);
          opc = fused_opcode(group, kind[i]);
          if (isf) feat = kind[term];
          else val = cls[term] == C_TERM_C ? cv[term] : fv[term];
          if (rfused) sl = il;
          else sr = start[r] + size[r] - 1;
          tf = orig[term];
        } else {
          opc = stack_opcode((f & N_RFIRST) != 0, kind[i]);
          sl = il;
          sr = start[r] + size[r] - 1;
        }
      }
    }
    words[2 * idx] = opc | ((uint32_t)feat << 8);
    consts[2 * idx] = val;
    if (aux) {
      aux[idx].src_l = sl < 0 ? NONE16 : (uint16_t)sl;
      aux[idx].src_r = sr < 0 ? NONE16 : (uint16_t)sr;
      aux[idx].tpos = (uint16_t)orig[i];
      aux[idx].tpos_fused = tf < 0 ? NONE16 : (uint16_t)tf;
    }
  }
  if (lane == 0) {
    words[2 * L] = I_NOP;
    consts[2 * L] = 0.f;
    p.len[t] = L;
  }
}

const void* pack_ptr() { return reinterpret_cast<const void*>(&pack_kernel); }

}  // namespace gg
