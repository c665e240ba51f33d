// Interpreter instruction set and the template packer (host + device).
//
// The packer turns one template tree into the program the interpreter runs.
// Section 3.2 of the paper linearises a tree by post-order traversal (RPN)
// with introns skipped and evaluates it with a stack in one forward pass.
// Here the top of the stack lives in an accumulator A (R rows per lane, in
// registers) and the values below it in a per-warp stack in shared memory
// (one slot = R rows of each of the 32 lanes).
//
// Instruction forms (kind = binary op, u = unary op):
//   LDF0 / LDC0        A = X[f] / A = c                  (A holds nothing)
//   PSF / PSC          push A; A = X[f] / c
//   UN(u)              A = u(A)
//   BF/BC(kind)        A = kind(A, X[f] / c)     right child a terminal
//   LF/LC(kind)        A = kind(X[f] / c, A)     left child a terminal
//   BS(kind)           A = kind(pop, A)          left subtree evaluated first
//   RS(kind)           A = kind(A, pop)          right subtree evaluated first
// A binary node whose children are both subtrees evaluates first the child
// that needs more stack (Sethi-Ullman order); a tree of height h then needs
// at most h-1 slots.  Every RPN node of the paper's linearisation appears
// exactly once: terminals either as a load or fused into their parent.
// pow (Table 2) has the same forms in opcodes of its own (PW + BF/BC/LF/LC
// group, PWS, PWR), run only by the kernels built with pow.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define GG_HD __host__ __device__ __forceinline__
#else
#define GG_HD inline
#endif

namespace gg {

// template opcodes (the ABI values of ggeval.h)
enum : int {
  T_ADD = 0, T_SUB = 1, T_MUL = 2, T_AQ = 3, T_SIN = 4, T_COS = 5, T_EXP = 6,
  T_LOG_ABS = 7, T_SQRT_ABS = 8, T_DIV = 9, T_SQUARE = 10, T_LOG = 11, T_SQRT = 12,
  T_POW = 13, T_ERC = 31, T_FEAT0 = 32, T_PAD = 255
};

// binary kinds and unary kinds used by the interpreter
// NKIND counts the kinds of the regular BF..RS opcode groups; K_POW has
// the appended PW/PWS/PWR opcodes.
enum : int { K_ADD = 0, K_SUB = 1, K_MUL = 2, K_AQ = 3, K_DIV = 4, NKIND = 5, K_POW = 5 };
enum : int {
  U_SIN = 0, U_COS = 1, U_EXP = 2, U_LOG_ABS = 3, U_SQRT_ABS = 4, U_SQUARE = 5,
  U_LOG = 6, U_SQRT = 7, NUNARY = 8
};

constexpr int MAX_SLOTS = 8;      // stack slots of the deepest template
constexpr int MAX_HEIGHT = 8;     // 511 template nodes
constexpr int MAX_NODES = 511;

enum : uint32_t {
  I_LDF0 = 0,
  I_LDC0 = 1,
  I_PSF = 2,
  I_PSC = 3,
  I_UN = 4,                        // + u          (4..11)
  I_BF = 12,                       // + kind       (12..16)
  I_BC = 17,                       // + kind       (17..21)
  I_LF = 22,                       // + kind       (22..26)
  I_LC = 27,                       // + kind       (27..31)
  I_BS = 32,                       // + kind       (32..36)
  I_RS = 37,                       // + kind       (37..41)
  I_NOP = 42,
  I_PW = 43,                       // + group BF/BC/LF/LC (43..46)
  I_PWS = 47,                      // A = pow(pop, A)
  I_PWR = 48,                      // A = pow(A, pop)
  I_COUNT = 49
};

// The instructions that read a feature (all opcodes are below 64).
constexpr uint64_t FEATURE_OPS =
    (1ull << I_LDF0) | (1ull << I_PSF) | (0x1full << I_BF) | (0x1full << I_LF) |
    (1ull << (I_PW + 0)) | (1ull << (I_PW + 2));
GG_HD bool reads_feature(uint32_t opc) { return opc < 64 && ((FEATURE_OPS >> opc) & 1u); }

// Opcode of a binary node with a fused terminal: group 0 BF, 1 BC, 2 LF, 3 LC.
GG_HD uint32_t fused_opcode(int group, int kind) {
  return kind == K_POW ? I_PW + (uint32_t)group : I_BF + (uint32_t)(group * NKIND + kind);
}

// Opcode of a binary node over two subtrees: the left one evaluated first
// (BS, the left value is popped) or the right one (RS).
GG_HD uint32_t stack_opcode(bool right_first, int kind) {
  if (kind == K_POW) return right_first ? I_PWR : I_PWS;
  return (right_first ? I_RS : I_BS) + (uint32_t)kind;
}

// node classes
enum : int { C_BAD = 0, C_TERM_F = 1, C_TERM_C = 2, C_UNARY = 3, C_BINARY = 4 };

GG_HD int classify(int op, int n_features, int* kind) {
  switch (op) {
    case T_ADD: *kind = K_ADD; return C_BINARY;
    case T_SUB: *kind = K_SUB; return C_BINARY;
    case T_MUL: *kind = K_MUL; return C_BINARY;
    case T_AQ: *kind = K_AQ; return C_BINARY;
    case T_DIV: *kind = K_DIV; return C_BINARY;
    case T_POW: *kind = K_POW; return C_BINARY;
    case T_SIN: *kind = U_SIN; return C_UNARY;
    case T_COS: *kind = U_COS; return C_UNARY;
    case T_EXP: *kind = U_EXP; return C_UNARY;
    case T_LOG_ABS: *kind = U_LOG_ABS; return C_UNARY;
    case T_SQRT_ABS: *kind = U_SQRT_ABS; return C_UNARY;
    case T_SQUARE: *kind = U_SQUARE; return C_UNARY;
    case T_LOG: *kind = U_LOG; return C_UNARY;
    case T_SQRT: *kind = U_SQRT; return C_UNARY;
    case T_ERC: *kind = 0; return C_TERM_C;
    default:
      if (op >= T_FEAT0 && op < T_PAD && op - T_FEAT0 < n_features) {
        *kind = op - T_FEAT0;
        return C_TERM_F;
      }
      *kind = 0;
      return C_BAD;
  }
}

// Per-instruction side information for the reverse sweep of the adjoint:
// which instructions produced the operands (0xFFFF = a fused terminal or
// none) and the template positions of the main node and of a fused
// terminal (0xFFFF = none).
struct Aux {
  uint16_t src_l, src_r, tpos, tpos_fused;
};
constexpr uint16_t NONE16 = 0xFFFFu;

struct PackResult {
  int len;        // instructions emitted (> 0) or 0 on error
  int slots;      // stack slots used
  int status;     // 0 ok, 1 invalid template, 2 needs more slots than allowed
  int counts[11]; // active nodes by class, see ggeval_batch_stats ([10]: pow)
  int exec[11];   // the same for the nodes evaluated per row after constant
                  // folding (equal to counts when folding is off)
};

// Constant folding (an addition; the paper evaluates every node on every
// row): an active function node with no feature among its active
// descendants has the same value on every row.  An evaluator with `on`
// true computes such a subtree once per trial with the interpreter's own
// FP32 operator functions, so each row gets exactly the value it would have
// computed itself, and the packer emits the largest such subtrees as
// constant terminals.  NoFold leaves programs unchanged.
struct NoFold {
  static constexpr bool on = false;
  GG_HD float un(int, float) const { return 0.f; }
  GG_HD float bin(int, float, float) const { return 0.f; }
};
// depth1[] flag bits used by the packer next to depth + 1 (at most 9)
constexpr uint8_t PK_CONST = 0x40;   // active subtree without a feature
constexpr uint8_t PK_INSIDE = 0x80;  // below the root of a folded subtree
constexpr uint8_t PK_DEPTH = 0x1F;

// Template position of the node with heap index i (children 2i+1, 2i+2) in
// the prefix layout of a template of height h: the path from the root is
// the bits of i + 1 below its leading one (0 = left, 1 = right), and in the
// prefix layout the left child of a node at depth e is the next position,
// the right child 2^(h - e) further.
GG_HD int prefix_position(int i, int h) {
  int d = 0;
  while (((i + 1) >> (d + 1)) != 0) ++d;
  int pos = 0;
  for (int e = 0; e < d; ++e) pos += (((i + 1) >> (d - 1 - e)) & 1) ? (1 << (h - e)) : 1;
  return pos;
}

// Children of the node at `pos` (depth `depth`) in a template of height h.
GG_HD void children(int layout, int h, int pos, int depth, int* l, int* r) {
  if (layout == 0) {
    *l = 2 * pos + 1;
    *r = 2 * pos + 2;
  } else {
    *l = pos + 1;
    *r = pos + (1 << (h - depth));
  }
}

// Linearise one template (heap or prefix layout, height h <= MAX_HEIGHT)
// into at most `cap` instructions.  Iterative (no recursion, so the device
// version needs no call stack): pass 1 marks active nodes top-down and
// validates them, pass 2 computes each active subtree's slot need
// bottom-up (both rely on a parent's position preceding its children's in
// either layout), pass 3 emits the program by an explicit-stack post-order
// walk.  words/consts have room for cap+1 entries at stride `ws`; entry
// [len] is set to NOP so the interpreter may prefetch one instruction ahead.
// `depth1` and `need` are caller scratch of at least 2^(h+1)-1 bytes each
// (shared memory in the packing kernel).  With allow_pow false an active
// pow node makes the template invalid (for interpreters built without pow).
// Folding: with `fv` (caller scratch of 2^(h+1)-1 floats) and an evaluator
// whose `on` is true, constant subtrees are folded (never together with
// `aux`: the adjoint needs every ERC); `fold_stats` alone marks the
// constant subtrees and fills res.exec without changing the program.
template <class Ev = NoFold>
GG_HD PackResult pack_tree(const uint8_t* op, const float* cval, int h, int layout,
                           int n_features, int max_slots, uint32_t* words, float* consts,
                           int ws, Aux* aux, int cap, uint8_t* depth1, uint8_t* need,
                           bool allow_pow = true, const Ev& ev = Ev(), float* fv = nullptr,
                           bool fold_stats = false) {
  PackResult res;
  res.len = 0;
  res.slots = 0;
  res.status = 0;
  for (int i = 0; i < 11; ++i) res.counts[i] = res.exec[i] = 0;
  const bool fold = Ev::on && fv != nullptr && aux == nullptr;
  const bool marks = fold || fold_stats;
  const int n = (1 << (h + 1)) - 1;
  // depth1[i]: depth + 1 of an active node, 0 for an intron;
  // need[i]: slots the active subtree at i needs
  for (int i = 0; i < n; ++i) depth1[i] = 0;
  depth1[0] = 1;
  // pass 1: active set + validation (Section 3.1 / Fig. 1)
  for (int pos = 0; pos < n; ++pos) {
    if (!depth1[pos]) continue;
    const int d = depth1[pos] - 1;
    int kind;
    const int cls = classify(op[pos], n_features, &kind);
    if (cls == C_BAD || ((cls == C_UNARY || cls == C_BINARY) && d >= h) ||
        (cls == C_BINARY && kind == K_POW && !allow_pow)) {
      res.status = 1;
      return res;
    }
    res.counts[0]++;
    if (cls == C_TERM_F || cls == C_TERM_C) {
      res.counts[1]++;
      continue;
    }
    int l, r;
    children(layout, h, pos, d, &l, &r);
    depth1[l] = (uint8_t)(d + 2);
    if (cls == C_BINARY) {
      depth1[r] = (uint8_t)(d + 2);
      res.counts[kind == K_AQ ? 3 : kind == K_DIV ? 4 : kind == K_POW ? 10 : 2]++;
    } else {
      res.counts[kind == U_SIN || kind == U_COS ? 5
                 : kind == U_EXP                 ? 6
                 : (kind == U_LOG_ABS || kind == U_LOG) ? 7
                 : (kind == U_SQRT_ABS || kind == U_SQRT) ? 8
                                                        : 9]++;
    }
  }
  // pass 2: constant subtrees (and their values when folding) and the slot
  // need of every active subtree, bottom-up; a folded subtree is a terminal
  for (int pos = n - 1; pos >= 0; --pos) {
    if (!depth1[pos]) continue;
    const int d = (depth1[pos] & PK_DEPTH) - 1;
    int kind;
    const int cls = classify(op[pos], n_features, &kind);
    need[pos] = 0;
    if (cls == C_TERM_F) continue;
    if (cls == C_TERM_C) {
      if (marks) depth1[pos] |= PK_CONST;
      if (fold) fv[pos] = cval[pos];
      continue;
    }
    int l, r;
    children(layout, h, pos, d, &l, &r);
    if (cls == C_UNARY) {
      if (marks && (depth1[l] & PK_CONST)) {
        depth1[pos] |= PK_CONST;
        if (fold) fv[pos] = ev.un(kind, fv[l]);
      }
      if (!(fold && (depth1[pos] & PK_CONST))) need[pos] = need[l];
      continue;
    }
    if (marks && (depth1[l] & PK_CONST) && (depth1[r] & PK_CONST)) {
      depth1[pos] |= PK_CONST;
      if (fold) fv[pos] = ev.bin(kind, fv[l], fv[r]);
    }
    if (fold && (depth1[pos] & PK_CONST)) continue;
    int kl, kr;
    const int cl = classify(op[l], n_features, &kl);
    const int cr = classify(op[r], n_features, &kr);
    const bool lt = cl == C_TERM_F || cl == C_TERM_C || (fold && (depth1[l] & PK_CONST));
    const bool rt = cr == C_TERM_F || cr == C_TERM_C || (fold && (depth1[r] & PK_CONST));
    if (rt) need[pos] = need[l];
    else if (lt) need[pos] = need[r];
    else {
      const int a = need[l], b = need[r];
      need[pos] = (uint8_t)(a >= b ? (a > b + 1 ? a : b + 1) : (b > a + 1 ? b : a + 1));
    }
  }
  // node counts of the folded program: a folded subtree's root becomes one
  // constant terminal and the nodes below it disappear (top-down)
  for (int i = 0; i < 11; ++i) res.exec[i] = res.counts[i];
  if (marks) {
    for (int pos = 0; pos < n; ++pos) {
      if (!depth1[pos]) continue;
      int kind;
      const int cls = classify(op[pos], n_features, &kind);
      const bool inside = (depth1[pos] & PK_INSIDE) != 0;
      const bool root = !inside && (depth1[pos] & PK_CONST) && (cls == C_UNARY || cls == C_BINARY);
      if (!inside && !root) continue;
      int slot = 1;  // terminal
      if (cls == C_BINARY) slot = kind == K_AQ ? 3 : kind == K_DIV ? 4 : kind == K_POW ? 10 : 2;
      if (cls == C_UNARY)
        slot = kind == U_SIN || kind == U_COS ? 5
               : kind == U_EXP ? 6
               : (kind == U_LOG_ABS || kind == U_LOG) ? 7
               : (kind == U_SQRT_ABS || kind == U_SQRT) ? 8 : 9;
      res.exec[slot]--;
      if (inside) res.exec[0]--;
      else res.exec[1]++;  // the root is now a constant terminal
      if (cls == C_UNARY || cls == C_BINARY) {
        const int d = (depth1[pos] & PK_DEPTH) - 1;
        int l, r;
        children(layout, h, pos, d, &l, &r);
        depth1[l] |= PK_INSIDE;
        if (cls == C_BINARY) depth1[r] |= PK_INSIDE;
      }
    }
  }
  // pass 3: emission
  struct Frame {
    int16_t pos;
    int8_t depth, occ, live, phase, order;
    int16_t c1;
  };
  Frame st[MAX_HEIGHT + 2];
  int sp = 0;
  int k = 0;
  int ret = -1;
  int max_slot = -1;
  st[0].pos = 0; st[0].depth = 0; st[0].occ = 0; st[0].live = 0; st[0].phase = 0;
  st[0].order = 0; st[0].c1 = -1;
  sp = 1;
  auto emit = [&](uint32_t opc, int feat, float c, int sl, int sr, int tp, int tf) -> int {
    if (k >= cap) return -1;
    words[k * ws] = opc | ((uint32_t)feat << 8);
    consts[k * ws] = c;
    if (aux) {
      aux[k].src_l = sl < 0 ? NONE16 : (uint16_t)sl;
      aux[k].src_r = sr < 0 ? NONE16 : (uint16_t)sr;
      aux[k].tpos = tp < 0 ? NONE16 : (uint16_t)tp;
      aux[k].tpos_fused = tf < 0 ? NONE16 : (uint16_t)tf;
    }
    return k++;
  };
  // class and constant of a node as emitted: a folded subtree is a constant
  auto eclass = [&](int pos, int* kind) -> int {
    if (fold && (depth1[pos] & PK_CONST)) {
      *kind = 0;
      return C_TERM_C;
    }
    return classify(op[pos], n_features, kind);
  };
  auto evalue = [&](int pos) -> float {
    return fold && (depth1[pos] & PK_CONST) ? fv[pos] : cval[pos];
  };
  while (sp > 0) {
    Frame& f = st[sp - 1];
    int kind;
    const int cls = eclass(f.pos, &kind);
    if (cls == C_TERM_F || cls == C_TERM_C) {
      const bool feat = cls == C_TERM_F;
      uint32_t opc;
      if (f.live) {
        if (f.occ >= max_slots) { res.status = 2; return res; }
        if (f.occ > max_slot) max_slot = f.occ;
        opc = feat ? I_PSF : I_PSC;
      } else {
        opc = feat ? I_LDF0 : I_LDC0;
      }
      ret = emit(opc, feat ? kind : 0, feat ? 0.f : evalue(f.pos), -1, -1, f.pos, -1);
      if (ret < 0) { res.status = 2; return res; }
      --sp;
      continue;
    }
    int l, r;
    children(layout, h, f.pos, f.depth, &l, &r);
    if (cls == C_UNARY) {
      if (f.phase == 0) {
        f.phase = 1;
        Frame& c = st[sp++];
        c.pos = (int16_t)l; c.depth = (int8_t)(f.depth + 1); c.occ = f.occ; c.live = f.live;
        c.phase = 0; c.order = 0; c.c1 = -1;
      } else {
        ret = emit(I_UN + (uint32_t)kind, 0, 0.f, ret, -1, f.pos, -1);
        if (ret < 0) { res.status = 2; return res; }
        --sp;
      }
      continue;
    }
    int kl, kr;
    const int cl = eclass(l, &kl);
    const int cr = eclass(r, &kr);
    const bool lt = cl == C_TERM_F || cl == C_TERM_C;
    const bool rt = cr == C_TERM_F || cr == C_TERM_C;
    if (rt || lt) {
      // one terminal child is fused into this instruction; the other child
      // (the left one when both are terminals) is evaluated into A first
      const int sub = rt ? l : r;
      const int term = rt ? r : l;
      const int ct = rt ? cr : cl;
      const int kt = rt ? kr : kl;
      if (f.phase == 0) {
        f.phase = 1;
        Frame& c = st[sp++];
        c.pos = (int16_t)sub; c.depth = (int8_t)(f.depth + 1); c.occ = f.occ; c.live = f.live;
        c.phase = 0; c.order = 0; c.c1 = -1;
      } else {
        const bool feat = ct == C_TERM_F;
        const int group = rt ? (feat ? 0 : 1) : (feat ? 2 : 3);
        ret = emit(fused_opcode(group, kind), feat ? kt : 0, feat ? 0.f : evalue(term),
                   rt ? ret : -1, rt ? -1 : ret, f.pos, term);
        if (ret < 0) { res.status = 2; return res; }
        --sp;
      }
      continue;
    }
    const int basis = f.occ + (f.live ? 1 : 0);
    if (f.phase == 0) {
      f.order = (int8_t)(need[l] >= need[r] ? 0 : 1);
      f.phase = 1;
      Frame& c = st[sp++];
      c.pos = (int16_t)(f.order ? r : l); c.depth = (int8_t)(f.depth + 1); c.occ = f.occ;
      c.live = f.live; c.phase = 0; c.order = 0; c.c1 = -1;
    } else if (f.phase == 1) {
      f.c1 = (int16_t)ret;
      f.phase = 2;
      Frame& c = st[sp++];
      c.pos = (int16_t)(f.order ? l : r); c.depth = (int8_t)(f.depth + 1); c.occ = (int8_t)basis;
      c.live = 1; c.phase = 0; c.order = 0; c.c1 = -1;
    } else {
      if (basis >= max_slots) { res.status = 2; return res; }
      const uint32_t opc = stack_opcode(f.order != 0, kind);
      const int sl = f.order ? ret : f.c1;
      const int sr = f.order ? f.c1 : ret;
      ret = emit(opc, 0, 0.f, sl, sr, f.pos, -1);
      if (ret < 0) { res.status = 2; return res; }
      --sp;
    }
  }
  words[k * ws] = I_NOP;
  consts[k * ws] = 0.f;
  res.len = k;
  res.slots = max_slot + 1;
  return res;
}

}  // namespace gg
