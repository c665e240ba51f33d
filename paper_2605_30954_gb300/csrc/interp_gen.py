"""Generate the interpreter's dispatch loop as inline PTX (interp_asm.inc).

The batched forward kernel spends most of its instructions interpreting
programs (Section 3.2: one forward stack pass over each trial's RPN program
per dataset row).  A C++ switch over the instruction set compiles to a tree
of compares and branches, about 27 warp instructions per interpreted
instruction.  PTX has an indexed branch (``brx.idx`` over a
``.branchtargets`` list), so this generator writes the whole loop as one
inline-PTX statement: every case ends by fetching the next instruction word
(prefetched one instruction ahead) and branching through the table.

Semantics are those of ``run_program`` in device.cuh, bit for bit: the same
FP32 operations in the same order, two rows at a time as packed
``.f32x2`` instructions, and (4 rows per lane) row by row (gmath.cuh's
``*_total`` forms) for a group of rows in which some argument lies outside
the common domain of exp, log or sqrt.  Instructions the PTX does not finish
leave the statement with their opcode, and the C++ caller runs them
(``exec_cold``) and re-enters: the end of the program (NOP), pow, sin or cos
with an argument beyond the reduction's range (the CUDA library function
then takes those rows) and, with 8 rows per lane, such groups of exp, log or
sqrt.  The file also generates the staged adjoint's reverse sweep
(``RevGen``).

Run by build.py before the CUDA sources are compiled; writes
``_build/gen/interp_asm.inc``.
"""
from __future__ import annotations

import os
import struct
import sys
from fractions import Fraction

# instruction set (isa.h)
I_LDF0, I_LDC0, I_PSF, I_PSC, I_UN = 0, 1, 2, 3, 4
I_BF, I_BC, I_LF, I_LC, I_BS, I_RS = 12, 17, 22, 27, 32, 37
I_NOP, I_PW, I_COUNT = 42, 43, 49
K_ADD, K_SUB, K_MUL, K_AQ, K_DIV = range(5)
U_SIN, U_COS, U_EXP, U_LOG_ABS, U_SQRT_ABS, U_SQUARE, U_LOG, U_SQRT = range(8)

# FP32 constants of gmath.cuh, as written there (decimal literals; SIN_C and
# COS_C in Horner order, highest power first)
TWO_OVER_PI = "0.636619746685028076"
MAGIC = "12582912.0"
PIO2_1 = "-1.57079637050628662"
PIO2_2 = "4.37113882867379e-08"
PIO2_3 = "1.71512451000588e-15"
SIN_C = ("-0.00019515285", "0.008332158", "-0.16666654")
COS_C = ("2.4433153e-05", "-0.0013887319", "0.04166665", "-0.5")
TRIG_RANGE = "131072.0"
LN2_HI = "0.693147182464599609375"
LN2_LO = "-1.9046542121259336e-09"
ATANH_C = ("0.2222222238779068", "0.2857142984867096", "0.4000000059604645",
           "0.6666666865348816")
SQRT_HALF_BITS = 0x3F3504F3
LOG2E_HI = "1.44269502162933349609375"
LOG2E_LO = "1.925962991126617468e-08"  # log2(e) - LOG2E_HI
EXP_RANGE = "87.0"


def f32_bits(s: str) -> int:
    """Bits of the FP32 value nearest to the decimal s (ties to even), as a
    C++ compiler rounds a float literal."""
    fr = Fraction(s)
    x = float(fr)
    b = struct.unpack("<I", struct.pack("<f", x))[0]
    best = None
    for cand in (b - 1, b, b + 1):
        v = struct.unpack("<f", struct.pack("<I", cand & 0xFFFFFFFF))[0]
        d = abs(Fraction(v) - fr)
        key = (d, cand & 1)
        if best is None or key < best[0]:
            best = (key, cand & 0xFFFFFFFF)
    return best[1]


def f(s: str) -> str:
    """FP32 immediate."""
    return "0f%08X" % f32_bits(s)


def f2(s: str) -> str:
    """The same FP32 value in both halves of a 64-bit immediate."""
    b = f32_bits(s)
    return "0x%08X%08X" % (b, b)


def sincos_pair(o, x, dst):
    """gmath.cuh sin_or_cos_reduced2 on the pair x into dst (x is read
    before dst is written): the quadrant shift in sh (0 sin, 1 cos);
    registers v0..v5, c1, c2, q0, q1, z0..z3, k, ks, p."""
    o(f"mov.b64 c1, {f2(TWO_OVER_PI)};")
    o(f"mov.b64 c2, {f2(MAGIC)};")
    o(f"fma.rn.f32x2 v0, {x}, c1, c2;")               # t
    o(f"mov.b64 c1, {f2('-' + MAGIC)};")
    o("add.rn.f32x2 v1, v0, c1;")                      # j
    o("mov.b64 {q0, q1}, v0;")
    o("add.u32 q0, q0, sh;")
    o("add.u32 q1, q1, sh;")
    o(f"mov.b64 c1, {f2(PIO2_1)};")
    o(f"fma.rn.f32x2 v2, v1, c1, {x};")                # r
    o(f"mov.b64 c1, {f2(PIO2_2)};")
    o("fma.rn.f32x2 v2, v1, c1, v2;")
    o(f"mov.b64 c1, {f2(PIO2_3)};")
    o("fma.rn.f32x2 v2, v1, c1, v2;")
    o("mul.rn.f32x2 v3, v2, v2;")                      # s
    o(f"mov.b64 c1, {f2(SIN_C[0])};")
    o(f"mov.b64 c2, {f2(SIN_C[1])};")
    o("fma.rn.f32x2 v4, v3, c1, c2;")                  # ps
    for k in range(2, len(SIN_C)):
        o(f"mov.b64 c1, {f2(SIN_C[k])};")
        o("fma.rn.f32x2 v4, v3, v4, c1;")
    o("mul.rn.f32x2 v5, v2, v3;")                      # r s
    o("fma.rn.f32x2 v4, v5, v4, v2;")                  # sr
    o(f"mov.b64 c1, {f2(COS_C[0])};")
    o(f"mov.b64 c2, {f2(COS_C[1])};")
    o("fma.rn.f32x2 v5, v3, c1, c2;")                  # pc
    for k in range(2, len(COS_C)):
        o(f"mov.b64 c1, {f2(COS_C[k])};")
        o("fma.rn.f32x2 v5, v3, v5, c1;")
    o(f"mov.b64 c1, {f2('1.0')};")
    o("fma.rn.f32x2 v5, v3, v5, c1;")                  # cr
    o("mov.b64 {z0, z1}, v4;")
    o("mov.b64 {z2, z3}, v5;")
    for e in (0, 1):
        # the quadrant's bit 0 picks cos over sin (bit 0 moved to the sign
        # for slct), bit 1 flips the sign (lop3: z ^ (k & 0x80000000))
        o(f"shl.b32 ks, q{e}, 31;")
        o(f"slct.b32.s32 z{e}, z{e}, z{2 + e}, ks;")
        o(f"shl.b32 k, q{e}, 30;")
        o(f"lop3.b32 z{e}, z{e}, k, 0x80000000, 0x78;")
    o(f"mov.b64 {dst}, {{z0, z1}};")


def exp_pair(o, x, dst):
    """gmath.cuh exp_ex2_2 on the pair x into dst (x is read before dst is
    written); registers v0, v1, c1, c2, z0, z1."""
    o(f"mov.b64 c1, {f2(LOG2E_HI)};")
    o(f"mul.rn.f32x2 v0, {x}, c1;")                   # hi
    o(f"mov.b64 c2, {f2('-1.0')};")
    o("mul.rn.f32x2 v1, v0, c2;")                      # -hi
    o(f"fma.rn.f32x2 v1, {x}, c1, v1;")               # x L - hi (exact)
    o(f"mov.b64 c2, {f2(LOG2E_LO)};")
    o(f"fma.rn.f32x2 v1, {x}, c2, v1;")               # lo
    o("mov.b64 {z0, z1}, v0;")
    o("ex2.approx.f32 z0, z0;")
    o("ex2.approx.f32 z1, z1;")
    o("mov.b64 v0, {z0, z1};")                         # 2^hi
    o(f"mov.b64 c1, {f2(LN2_HI)};")
    o("mul.rn.f32x2 v1, v1, c1;")                      # lo ln2
    o(f"fma.rn.f32x2 {dst}, v0, v1, v0;")


class Gen:
    def __init__(self, R: int, special: bool = True, tape: bool = False):
        """special: finish the row-by-row forms of exp, log and sqrt inside
        the PTX (else their groups leave it for the C++ cold path).  tape:
        store the accumulator after every instruction at the tape address
        (advanced by one slot each time): the forward half of the adjoint."""
        assert R in (4, 8)
        self.R = R
        self.special = special
        self.tape = tape
        self.NP = R // 2          # row pairs per lane
        self.NQ = R // 4          # 16-byte shared-memory accesses per row group
        self.SLOTB = 32 * R * 4   # bytes per stack slot (32 lanes x R rows)
        # a lane's rows (device.cuh row_of): 8 rows as two runs of 4, 128
        # rows (512 bytes) apart
        self.QOFF = 512 if R == 8 else 16
        self.lines = []
        # asm operands: %0 pc, %1 sp, %2 code, %3 arg, %4.. A[0..R-1], then
        # (with tape) the tape address, then xs
        self.A = [f"%{4 + r}" for r in range(R)]
        self.TP = f"%{4 + R}" if tape else None
        self.XS = f"%{5 + R}" if tape else f"%{4 + R}"

    def o(self, s):
        self.lines.append(s)

    def label(self, name):
        self.lines.append(f"{name}:")

    # -- shared-memory row groups -------------------------------------------
    def load(self, dst, addr):
        for q in range(self.NQ):
            self.o(f"ld.shared.v2.b64 {{{dst}{2 * q}, {dst}{2 * q + 1}}}, "
                   f"[{addr}+{self.QOFF * q}];")

    def store(self, src, addr):
        for q in range(self.NQ):
            self.o(f"st.shared.v2.b64 [{addr}+{self.QOFF * q}], "
                   f"{{{src}{2 * q}, {src}{2 * q + 1}}};")

    def const_pairs(self, dst):
        self.o(f"mov.b64 {dst}0, {{arg, arg}};")
        for i in range(1, self.NP):
            self.o(f"mov.b64 {dst}{i}, {dst}0;")

    def next(self):
        """(With tape: store the finished instruction's rows.)  Fetch the
        prefetched instruction, prefetch the one after it and branch through
        the table (an out-of-range opcode goes to BAD)."""
        if self.tape:
            self.store("a", self.TP)
            self.o(f"add.u32 {self.TP}, {self.TP}, {self.SLOTB};")
        self.o("min.u32 opc, nopc, %d;" % I_COUNT)
        self.o("mov.u32 arg, narg;")
        self.o("add.u32 %0, %0, 8;")
        self.o("ld.shared.v2.u32 {nopc, narg}, [%0];")
        self.o("brx.idx.uni opc, GG_TBL;")

    # -- binary operators on pairs: a_i = kind(l_i, r_i) ---------------------
    def binop(self, kind, l, r, const_r=False):
        NP = self.NP
        if kind in (K_ADD, K_SUB, K_MUL):
            ins = {K_ADD: "add", K_SUB: "sub", K_MUL: "mul"}[kind]
            for i in range(NP):
                self.o(f"{ins}.rn.f32x2 a{i}, {l(i)}, {r(i)};")
            return
        if kind == K_AQ:
            if const_r:
                # rsqrt(1 + c^2) is the same for every row: computed once
                self.o("mov.b32 y0, arg;")
                self.o(f"fma.rn.f32 y0, y0, y0, {f('1.0')};")
                self.o("rsqrt.approx.f32 y0, y0;")
                self.o("mov.b64 u0, {y0, y0};")
                for i in range(NP):
                    self.o(f"mul.rn.f32x2 a{i}, {l(i)}, u0;")
                return
            self.o(f"mov.b64 c1, {f2('1.0')};")
            for i in range(NP):
                self.o(f"fma.rn.f32x2 u{i}, {r(i)}, {r(i)}, c1;")
                self.o(f"mov.b64 {{y{2 * i}, y{2 * i + 1}}}, u{i};")
                self.o(f"rsqrt.approx.f32 y{2 * i}, y{2 * i};")
                self.o(f"rsqrt.approx.f32 y{2 * i + 1}, y{2 * i + 1};")
                self.o(f"mov.b64 u{i}, {{y{2 * i}, y{2 * i + 1}}};")
                self.o(f"mul.rn.f32x2 a{i}, {l(i)}, u{i};")
            return
        raise ValueError(kind)

    # -- the cases -----------------------------------------------------------
    def operand_fetch(self, form):
        """Right-hand operand rows into t (or the constant into t0); returns
        (left, right) operand getters and whether the right one is the
        constant."""
        a = lambda i: f"a{i}"
        t = lambda i: f"t{i}"
        c = lambda i: "t0"
        if form == "BF":
            self.o(f"add.u32 ad, {self.XS}, arg;")
            self.load("t", "ad")
            return a, t, False
        if form == "BC":
            self.const_pairs("t")
            return a, c, True
        if form == "LF":
            self.o(f"add.u32 ad, {self.XS}, arg;")
            self.load("t", "ad")
            return t, a, False
        if form == "LC":
            self.const_pairs("t")
            return c, a, False
        if form == "BS":
            self.o(f"sub.u32 %1, %1, {self.SLOTB};")
            self.load("t", "%1")
            return t, a, False
        if form == "RS":
            self.o(f"sub.u32 %1, %1, {self.SLOTB};")
            self.load("t", "%1")
            return a, t, False
        raise ValueError(form)

    def div_body(self, name, left_is_a):
        """a = l / r per row (IEEE division), l and r from a and t."""
        self.label(name)
        for i in range(self.NP):
            self.o(f"mov.b64 {{x{2 * i}, x{2 * i + 1}}}, a{i};")
            self.o(f"mov.b64 {{y{2 * i}, y{2 * i + 1}}}, t{i};")
        for r in range(self.R):
            if left_is_a:
                self.o(f"div.rn.f32 x{r}, x{r}, y{r};")
            else:
                self.o(f"div.rn.f32 x{r}, y{r}, x{r};")
        for i in range(self.NP):
            self.o(f"mov.b64 a{i}, {{x{2 * i}, x{2 * i + 1}}};")
        self.next()

    def unpack_a(self, dst="x"):
        for i in range(self.NP):
            self.o(f"mov.b64 {{{dst}{2 * i}, {dst}{2 * i + 1}}}, a{i};")

    def sincos_body(self):
        """sin (sh = 0) or cos (sh = 1): gmath.cuh sin_or_cos_reduced2 on
        every pair; a group with max |x| beyond 2^17 (or all NaN) goes to
        the library function (cold)."""
        R, NP = self.R, self.NP
        self.label("GG_SINCOS")
        self.unpack_a("x")
        for r in range(R):
            self.o(f"abs.f32 s0, x{r};")
            self.o("mov.f32 m, s0;" if r == 0 else "max.f32 m, m, s0;")
        self.o(f"setp.gtu.f32 p, m, {f(TRIG_RANGE)};")
        self.o("@p bra GG_EXIT;")
        for i in range(NP):
            sincos_pair(self.o, f"a{i}", f"a{i}")
        self.next()

    def logsqrt_check(self, special):
        """Apply the mask (|x| or x) to every row's bits into b0..; go to the
        row-by-row body `special` unless every row is a positive normal
        finite number."""
        R = self.R
        self.unpack_a("x")
        for r in range(R):
            self.o(f"mov.b32 b{r}, x{r};")
            self.o(f"and.b32 b{r}, b{r}, msk;")
            self.o(f"sub.u32 k, b{r}, 0x00800000;")
            self.o("mov.u32 mm, k;" if r == 0 else "max.u32 mm, mm, k;")
        self.o("setp.ge.u32 p, mm, 0x7F000000;")
        self.o(f"@p bra {special};")

    def repack_x(self):
        for i in range(self.NP):
            self.o(f"mov.b64 a{i}, {{x{2 * i}, x{2 * i + 1}}};")

    def log_special_body(self):
        """gmath.cuh log_total row by row, on row pairs (each half of a packed
        operation rounds as the scalar one): a zero or subnormal argument is
        scaled by 2^24 with the exponent corrected, then the special values
        replace the results of zeros, infinities, NaN and negatives."""
        self.label("GG_LOG_SP")
        o = self.o
        for i in range(self.NP):
            for e in (0, 1):
                r = 2 * i + e
                o(f"setp.lt.u32 p, b{r}, 0x00800000;")         # subnormal or zero
                o(f"mov.b32 s0, b{r};")
                o(f"mul.rn.f32 s1, s0, {f('16777216.0')};")
                o(f"selp.f32 s0, s1, s0, p;")                   # x, scaled by 2^24
                o("selp.s32 ea, -24, 0, p;")
                o("mov.b32 k, s0;")
                o(f"sub.s32 kk, k, {SQRT_HALF_BITS};")
                o(f"shr.s32 e{e}, kk, 23;")
                o(f"shl.b32 kk, e{e}, 23;")
                o("sub.s32 kk, k, kk;")
                o(f"mov.b32 z{e}, kk;")                         # m
                o(f"add.s32 ee, e{e}, ea;")
                o(f"cvt.rn.f32.s32 w{e}, ee;")
            self.log_pair(i)
            o(f"mov.b64 {{s0, s1}}, a{i};")
            for e in (0, 1):  # the last select wins: -0 (above +inf as bits) is a zero
                r = 2 * i + e
                o(f"setp.gt.u32 p, b{r}, 0x7F800000;")
                o(f"selp.f32 s{e}, 0f7FFFFFFF, s{e}, p;")       # NaN, negatives: NaN
                o(f"setp.eq.u32 p, b{r}, 0x7F800000;")
                o(f"selp.f32 s{e}, 0f7F800000, s{e}, p;")       # log(inf) = inf
                o(f"and.b32 k, b{r}, 0x7FFFFFFF;")
                o("setp.eq.u32 p, k, 0;")
                o(f"selp.f32 s{e}, 0fFF800000, s{e}, p;")       # log(+-0) = -inf
            o(f"mov.b64 a{i}, {{s0, s1}};")
        self.next()

    def sqrt_special_body(self):
        """gmath.cuh sqrt_total row by row: the Newton form on positive
        normal rows, the IEEE square root on the others."""
        self.label("GG_SQRT_SP")
        o = self.o
        for i in range(self.NP):
            self.sqrt_pair(i)
            o(f"mov.b64 {{s0, s1}}, a{i};")
            for e in (0, 1):
                r = 2 * i + e
                o(f"mov.b32 s2, b{r};")
                o("sqrt.rn.f32 s2, s2;")                       # IEEE
                o(f"sub.u32 k, b{r}, 0x00800000;")
                o("setp.lt.u32 p, k, 0x7F000000;")             # positive normal
                o(f"selp.f32 s{e}, s{e}, s2, p;")
            o(f"mov.b64 a{i}, {{s0, s1}};")
        self.next()

    def exp_special_body(self):
        """gmath.cuh exp_total row by row, on row pairs."""
        self.label("GG_EXP_SP")
        o = self.o
        for i in range(self.NP):
            o(f"mov.b64 {{x0, x1}}, a{i};")                     # the arguments
            o(f"mov.b64 c1, {f2(LOG2E_HI)};")
            o(f"mul.rn.f32x2 v0, a{i}, c1;")                   # hi
            o(f"mov.b64 c2, {f2('-1.0')};")
            o("mul.rn.f32x2 v1, v0, c2;")
            o(f"fma.rn.f32x2 v1, a{i}, c1, v1;")
            o(f"mov.b64 c2, {f2(LOG2E_LO)};")
            o(f"fma.rn.f32x2 v1, a{i}, c2, v1;")               # lo
            o(f"mov.b64 c2, {f2('0.5')};")
            o("mul.rn.f32x2 v2, v0, c2;")                      # hi / 2
            o("mov.b64 {z0, z1}, v0;")
            o("mov.b64 {z2, z3}, v2;")
            for e in (0, 1):
                o(f"ex2.approx.f32 s{e}, z{e};")               # 2^hi
                o(f"ex2.approx.f32 s{2 + e}, z{2 + e};")
                o(f"mul.rn.f32 s{2 + e}, s{2 + e}, s{2 + e};")   # (2^(hi/2))^2
                o(f"abs.f32 s4, x{e};")
                o(f"setp.le.f32 p, s4, {f(EXP_RANGE)};")
                o(f"selp.f32 s{e}, s{e}, s{2 + e}, p;")
            o("mov.b64 v0, {s0, s1};")                         # e
            o(f"mov.b64 c1, {f2(LN2_HI)};")
            o("mul.rn.f32x2 v1, v1, c1;")
            o("fma.rn.f32x2 v2, v0, v1, v0;")
            o("mov.b64 {s2, s3}, v2;")
            for e in (0, 1):
                o(f"setp.eq.f32 p, s{e}, 0f7F800000;")
                o(f"selp.f32 s{2 + e}, 0f7F800000, s{2 + e}, p;")  # overflow stays inf
                o(f"setp.eq.f32 p, x{e}, 0fFF800000;")
                o(f"selp.f32 s{2 + e}, 0f00000000, s{2 + e}, p;")  # exp(-inf) = 0
            o(f"mov.b64 a{i}, {{s2, s3}};")
        self.next()

    def log_pair(self, i):
        """log_normal2 of pair i from m in (z0, z1) and the exponents as
        floats in (w0, w1); the result into a{i}."""
        o = self.o
        o("mov.b64 v0, {z0, z1};")                         # m
        o(f"mov.b64 c1, {f2('-1.0')};")
        o("add.rn.f32x2 v1, v0, c1;")                      # f = m - 1
        o(f"mov.b64 c2, {f2('1.0')};")
        o("add.rn.f32x2 v2, v0, c2;")                      # d = m + 1
        o("mov.b64 {z0, z1}, v2;")
        o("rcp.approx.ftz.f32 z0, z0;")
        o("rcp.approx.ftz.f32 z1, z1;")
        o("mov.b64 v2, {z0, z1};")                         # rc
        o("mul.rn.f32x2 v3, v1, v2;")                      # s
        o(f"mov.b64 c2, {f2('-2.0')};")
        o("fma.rn.f32x2 v4, v3, c2, v1;")                  # t = fma(s, -2, f)
        o("mul.rn.f32x2 v5, v3, c1;")                      # -s
        o("fma.rn.f32x2 v4, v5, v1, v4;")                  # fma(-s, f, t)
        o("fma.rn.f32x2 v3, v4, v2, v3;")                  # s
        o("mul.rn.f32x2 v4, v3, v3;")                      # z
        o(f"mov.b64 c1, {f2(ATANH_C[0])};")
        o(f"mov.b64 c2, {f2(ATANH_C[1])};")
        o("fma.rn.f32x2 v5, v4, c1, c2;")                  # p
        for k in (2, 3):
            o(f"mov.b64 c1, {f2(ATANH_C[k])};")
            o("fma.rn.f32x2 v5, v4, v5, c1;")
        o("mul.rn.f32x2 v0, v3, v4;")                      # s z
        o("add.rn.f32x2 v1, v3, v3;")                      # s + s
        o("fma.rn.f32x2 v0, v0, v5, v1;")                  # u
        o("mov.b64 v1, {w0, w1};")                         # e as float
        o(f"mov.b64 c1, {f2(LN2_LO)};")
        o("fma.rn.f32x2 v0, v1, c1, v0;")
        o(f"mov.b64 c1, {f2(LN2_HI)};")
        o(f"fma.rn.f32x2 a{i}, v1, c1, v0;")

    def log_body(self):
        """gmath.cuh log_normal2 on every pair of the masked rows."""
        self.label("GG_LOG")
        self.logsqrt_check("GG_LOG_SP" if self.special else "GG_EXIT")
        o = self.o
        for i in range(self.NP):
            for e in (0, 1):
                r = 2 * i + e
                o(f"sub.s32 kk, b{r}, {SQRT_HALF_BITS};")
                o(f"shr.s32 e{e}, kk, 23;")
                o(f"shl.b32 kk, e{e}, 23;")
                o(f"sub.s32 kk, b{r}, kk;")
                o(f"mov.b32 z{e}, kk;")
                o(f"cvt.rn.f32.s32 w{e}, e{e};")
            self.log_pair(i)
        self.next()

    def sqrt_pair(self, i):
        """sqrt_newton2 of the masked rows of pair i into a{i}."""
        o = self.o
        o(f"mov.b64 v0, {{b{2 * i}, b{2 * i + 1}}};")      # x (masked)
        o(f"rsqrt.approx.f32 z0, b{2 * i};")
        o(f"rsqrt.approx.f32 z1, b{2 * i + 1};")
        o("mov.b64 v1, {z0, z1};")                         # rs
        o("mul.rn.f32x2 v2, v0, v1;")                      # s
        o(f"mov.b64 c1, {f2('-1.0')};")
        o("mul.rn.f32x2 v3, v2, c1;")                      # -s
        o("fma.rn.f32x2 v3, v3, v2, v0;")                  # e
        o(f"mov.b64 c1, {f2('0.5')};")
        o("mul.rn.f32x2 v1, c1, v1;")                      # 0.5 rs
        o(f"fma.rn.f32x2 a{i}, v3, v1, v2;")

    def sqrt_body(self):
        """gmath.cuh sqrt_newton2 on every pair of the masked rows."""
        self.label("GG_SQRT")
        self.logsqrt_check("GG_SQRT_SP" if self.special else "GG_EXIT")
        for i in range(self.NP):
            self.sqrt_pair(i)
        self.next()

    def exp_body(self):
        """gmath.cuh exp_ex2_2 on every pair; a group with max |x| above 87
        (or all NaN) goes to the library function (cold)."""
        R = self.R
        self.label("GG_EXP")
        self.unpack_a("x")
        for r in range(R):
            self.o(f"abs.f32 s0, x{r};")
            self.o("mov.f32 m, s0;" if r == 0 else "max.f32 m, m, s0;")
        self.o(f"setp.gtu.f32 p, m, {f(EXP_RANGE)};")
        self.o("@p bra GG_EXP_SP;" if self.special else "@p bra GG_EXIT;")
        for i in range(self.NP):
            exp_pair(self.o, f"a{i}", f"a{i}")
        self.next()

    def build(self):
        R, NP = self.R, self.NP
        o = self.o
        o("{")
        o(f".reg .b64 a<{NP}>, t<{NP}>, u<{NP}>, v<6>, c1, c2;")
        o(f".reg .f32 x<{R}>, y<{R}>, w<2>, m;")
        o(f".reg .b32 z<4>, b<{R}>;")
        o(".reg .u32 opc, arg, nopc, narg, ad, sh, msk, k, q<2>, mm;")
        o(".reg .s32 e<2>, ea, ee, kk, ks;")
        o(".reg .f32 s<5>;")
        o(".reg .pred p;")
        for i in range(NP):
            o(f"mov.b64 a{i}, {{{self.A[2 * i]}, {self.A[2 * i + 1]}}};")
        o("ld.shared.v2.u32 {opc, arg}, [%0];")
        o("add.u32 %0, %0, 8;")
        o("min.u32 opc, opc, %d;" % I_COUNT)
        o("ld.shared.v2.u32 {nopc, narg}, [%0];")
        targets = []
        cases = {}  # opcode -> label
        # loads and pushes
        cases[I_LDF0] = "GG_LDF0"
        cases[I_LDC0] = "GG_LDC0"
        cases[I_PSF] = "GG_PSF"
        cases[I_PSC] = "GG_PSC"
        unary = {U_SIN: "GG_SIN", U_COS: "GG_COS", U_EXP: "GG_EXP", U_LOG_ABS: "GG_LOGA",
                 U_SQRT_ABS: "GG_SQRTA", U_SQUARE: "GG_SQUARE", U_LOG: "GG_LOGP",
                 U_SQRT: "GG_SQRTP"}
        for u, lab in unary.items():
            cases[I_UN + u] = lab
        forms = [("BF", I_BF), ("BC", I_BC), ("LF", I_LF), ("LC", I_LC), ("BS", I_BS),
                 ("RS", I_RS)]
        for name, base in forms:
            for k in range(5):
                cases[base + k] = f"GG_{name}{k}"
        cases[I_NOP] = "GG_EXIT"
        for op in range(I_PW, I_COUNT + 1):
            cases[op] = "GG_EXIT"  # pow (cold) and out-of-range opcodes
        for op in range(I_COUNT + 1):
            targets.append(cases[op])
        o("GG_TBL: .branchtargets " + ", ".join(targets) + ";")
        o("brx.idx.uni opc, GG_TBL;")
        # loads and pushes
        self.label("GG_LDF0")
        o(f"add.u32 ad, {self.XS}, arg;")
        self.load("a", "ad")
        self.next()
        self.label("GG_LDC0")
        self.const_pairs("a")
        self.next()
        self.label("GG_PSF")
        self.store("a", "%1")
        o(f"add.u32 %1, %1, {self.SLOTB};")
        o(f"add.u32 ad, {self.XS}, arg;")
        self.load("a", "ad")
        self.next()
        self.label("GG_PSC")
        self.store("a", "%1")
        o(f"add.u32 %1, %1, {self.SLOTB};")
        self.const_pairs("a")
        self.next()
        # unary entry points
        self.label("GG_SIN")
        o("mov.u32 sh, 0;")
        o("bra.uni GG_SINCOS;")
        self.label("GG_COS")
        o("mov.u32 sh, 1;")
        o("bra.uni GG_SINCOS;")
        self.label("GG_LOGA")
        o("mov.u32 msk, 0x7FFFFFFF;")
        o("bra.uni GG_LOG;")
        self.label("GG_LOGP")
        o("mov.u32 msk, 0xFFFFFFFF;")
        o("bra.uni GG_LOG;")
        self.label("GG_SQRTA")
        o("mov.u32 msk, 0x7FFFFFFF;")
        o("bra.uni GG_SQRT;")
        self.label("GG_SQRTP")
        o("mov.u32 msk, 0xFFFFFFFF;")
        o("bra.uni GG_SQRT;")
        self.label("GG_SQUARE")
        for i in range(NP):
            o(f"mul.rn.f32x2 a{i}, a{i}, a{i};")
        self.next()
        # binary forms
        for name, base in forms:
            for k in range(5):
                self.label(f"GG_{name}{k}")
                l, r, const_r = self.operand_fetch(name)
                if k == K_DIV:
                    if name in ("BC", "LC"):
                        pass  # t0 already holds the constant in every pair
                    left_is_a = name in ("BF", "BC", "RS")
                    o("bra.uni %s;" % ("GG_DIVB" if left_is_a else "GG_DIVL"))
                    continue
                self.binop(k, l, r, const_r=const_r)
                self.next()
        self.div_body("GG_DIVB", True)
        self.div_body("GG_DIVL", False)
        self.sincos_body()
        self.log_body()
        self.sqrt_body()
        self.exp_body()
        if self.special:
            self.log_special_body()
            self.sqrt_special_body()
            self.exp_special_body()
        # exit: the opcode that stopped and its operand word; pc already
        # points at the next instruction
        self.label("GG_EXIT")
        o("mov.u32 %2, opc;")
        o("mov.u32 %3, arg;")
        for i in range(NP):
            o(f"mov.b64 {{{self.A[2 * i]}, {self.A[2 * i + 1]}}}, a{i};")
        o("}")
        return self.lines


# reverse-sweep descriptor forms of the staged adjoint (adjoint.cu)
RV_CONST, RV_UN, RV_BIN, RV_COUNT = 0, 1, 9, 45
RV_GSM = 64
G_BF, G_BC, G_LF, G_LC, G_BS, G_RS = range(6)


class RevGen:
    """The staged adjoint's reverse sweep for 4 rows per lane (two .f32x2
    pairs): a loop over the descriptors from the last to the first, the
    next descriptor and its two operand rows loaded one step ahead, and an
    indexed branch on the form (table entries 64 + form first load the
    adjoint of a pushed value from V).  The forms of +, -, *, AQ, the
    pushed ERC and every unary operator run here (sin, cos and exp with the
    forward's own forms, for a group within their range); division, pow
    and out-of-range groups leave the statement with the descriptor and the
    C++ caller runs them (rev_cold) and re-enters.

    Operands: %0 rp (next descriptor's address), %1 count left, %2 code
    (1: a form for the caller, 0: done), %3..%6 the descriptor left with,
    %7..%10 G (the adjoint carried in registers), %11 the lane's base, %12
    the lane's base + V, %13 the lane's ERC partial column, %14 the first
    descriptor's address, %15 the valid-row mask.  Same operations in the
    same order as adjoint.cu's C++ forms."""

    def __init__(self):
        self.lines = []

    def o(self, s):
        self.lines.append(s)

    def label(self, s):
        self.lines.append(s + ":")

    # -- helpers on the current adjoint g (pairs g0, g1) and operand rows --
    def rows(self, pair, dst):
        """Unpack a pair register set into 4 f32 registers dst0..dst3."""
        self.o(f"mov.b64 {{{dst}0, {dst}1}}, {pair}0;")
        self.o(f"mov.b64 {{{dst}2, {dst}3}}, {pair}1;")

    def pack(self, src, pair):
        self.o(f"mov.b64 {pair}0, {{{src}0, {src}1}};")
        self.o(f"mov.b64 {pair}1, {{{src}2, {src}3}};")

    def neg(self, dst, src):
        for i in range(2):
            self.o(f"xor.b64 {dst}{i}, {src}{i}, 0x8000000080000000;")

    def mul(self, dst, a, b):
        for i in range(2):
            self.o(f"mul.rn.f32x2 {dst}{i}, {a}{i}, {b}{i};")

    def store(self, src, off):
        """Store pairs src at the lane's row of the operand at offset off."""
        self.o(f"add.u32 ad, %11, {off};")
        self.o(f"st.shared.v2.b64 [ad], {{{src}0, {src}1}};")

    def erc(self, src):
        """Sum the valid rows of pairs src (in row order from zero, as the
        C++ does) and store the sum at the descriptor's ERC ordinal."""
        self.rows(src, "h")
        for r in range(4):
            self.o(f"selp.f32 h{r}, h{r}, 0f00000000, pv{r};")
        self.o("add.rn.f32 s, h0, h1;")
        self.o("add.rn.f32 s, s, h2;")
        self.o("add.rn.f32 s, s, h3;")
        self.o("bfe.u32 kk, x, 7, 9;")
        self.o("mad.lo.u32 ad, kk, 132, %13;")
        self.o("st.shared.f32 [ad], s;")

    def cpair(self):
        self.o("mov.b64 cc0, {w, w};")
        self.o("mov.b64 cc1, cc0;")

    def aq_q(self, b, q):
        """q = rsqrt(1 + b^2) row by row (rsqrt.approx, as rsqrt_approx)."""
        self.rows(b, "r")
        for r in range(4):
            self.o(f"fma.rn.f32 r{r}, r{r}, r{r}, 0f3F800000;")
            self.o(f"rsqrt.approx.f32 r{r}, r{r};")
        self.pack("r", q)

    def aq_db(self, a, b, q, dst):
        """dst = ((((-a) b) q) q) q, the C++ order."""
        self.neg(dst, a)
        self.mul(dst, dst, b)
        for _ in range(3):
            self.mul(dst, dst, q)

    def nxt(self):
        self.o("bra.uni RV_NEXT;")

    # -- the forms ------------------------------------------------------------
    def bin_form(self, grp, kind):
        o = self.o
        # operands: BF (A=u, x=v)  BC (A=u, c)  LF (x=v, A=u)  LC (c, A=u)
        #           BS (pop=u, A=v)  RS (A=u, pop=v)
        if kind == K_ADD:
            if grp in (G_BC, G_LC):
                self.erc("g")
            elif grp == G_BS:
                self.store("g", "y")
            elif grp == G_RS:
                self.store("g", "z")
        elif kind == K_SUB:
            if grp == G_BC:
                self.neg("e", "g")
                self.erc("e")
            elif grp == G_LF:
                self.neg("g", "g")
            elif grp == G_LC:
                self.erc("g")
                self.neg("g", "g")
            elif grp == G_BS:
                self.store("g", "y")
                self.neg("g", "g")
            elif grp == G_RS:
                self.neg("e", "g")
                self.store("e", "z")
        elif kind == K_MUL:
            if grp in (G_BF, G_LF):
                self.mul("g", "g", "vb")
            elif grp in (G_BC, G_LC):
                self.mul("e", "g", "ua")
                self.erc("e")
                self.cpair()
                self.mul("g", "g", "cc")
            elif grp == G_BS:
                self.mul("e", "g", "vb")
                self.store("e", "y")
                self.mul("g", "g", "ua")
            else:  # RS
                self.mul("e", "g", "ua")
                self.store("e", "z")
                self.mul("g", "g", "vb")
        else:  # K_AQ: da = q(b), db = -a b q^3
            if grp == G_BF:
                self.aq_q("vb", "aq")
                self.mul("g", "g", "aq")
            elif grp == G_BC:
                o("fma.rn.f32 s, cf, cf, 0f3F800000;")
                o("rsqrt.approx.f32 s, s;")
                o("mov.b64 aq0, {s, s};")
                o("mov.b64 aq1, aq0;")
                self.cpair()
                self.aq_db("ua", "cc", "aq", "e")
                self.mul("e", "g", "e")
                self.erc("e")
                self.mul("g", "g", "aq")
            elif grp == G_LF:
                self.aq_q("ua", "aq")
                self.aq_db("vb", "ua", "aq", "e")
                self.mul("g", "g", "e")
            elif grp == G_LC:
                self.aq_q("ua", "aq")
                self.mul("e", "g", "aq")
                self.erc("e")
                self.cpair()
                self.aq_db("cc", "ua", "aq", "e")
                self.mul("g", "g", "e")
            elif grp == G_BS:
                self.aq_q("vb", "aq")
                self.mul("e", "g", "aq")
                self.store("e", "y")
                self.aq_db("ua", "vb", "aq", "e")
                self.mul("g", "g", "e")
            else:  # RS
                self.aq_q("vb", "aq")
                self.aq_db("ua", "vb", "aq", "e")
                self.mul("e", "g", "e")
                self.store("e", "z")
                self.mul("g", "g", "aq")
        self.nxt()

    def range_check(self, bound):
        """Leave for the C++ form (which takes the library's path) unless
        max |x| over the rows is within bound, as the forward's check."""
        o = self.o
        self.rows("ua", "r")
        for r in range(4):
            o(f"abs.f32 s, r{r};")
            o("mov.f32 m, s;" if r == 0 else "max.f32 m, m, s;")
        o(f"setp.gtu.f32 p, m, {f(bound)};")
        o("@p bra RV_COLD;")

    def un_form(self, u):
        o = self.o
        if u in (U_SIN, U_COS):  # sin' = cos, cos' = -sin
            self.range_check(TRIG_RANGE)
            o("mov.u32 sh, %d;" % (1 if u == U_SIN else 0))
            for i in range(2):
                sincos_pair(o, f"ua{i}", f"e{i}")
            self.mul("g", "g", "e")
            if u == U_COS:
                self.neg("g", "g")
        elif u == U_EXP:
            self.range_check(EXP_RANGE)
            for i in range(2):
                exp_pair(o, f"ua{i}", f"e{i}")
            self.mul("g", "g", "e")
        elif u == U_SQUARE:
            for i in range(2):
                o(f"add.rn.f32x2 e{i}, ua{i}, ua{i};")
            self.mul("g", "g", "e")
        elif u in (U_LOG_ABS, U_LOG):
            self.rows("ua", "r")
            for r in range(4):
                o(f"rcp.rn.f32 r{r}, r{r};")
            self.pack("r", "e")
            self.mul("g", "g", "e")
        elif u == U_SQRT:
            self.rows("ua", "r")
            for r in range(4):
                o(f"rsqrt.approx.f32 r{r}, r{r};")
                o(f"mul.rn.f32 r{r}, r{r}, 0f3F000000;")
            self.pack("r", "e")
            self.mul("g", "g", "e")
        else:  # U_SQRT_ABS: x == 0 ? 0 : g copysign(0.5 rsqrt|x|, x)
            self.rows("ua", "r")
            self.rows("g", "h")
            for r in range(4):
                o(f"abs.f32 s, r{r};")
                o(f"rsqrt.approx.f32 s, s;")
                o(f"mul.rn.f32 s, s, 0f3F000000;")
                o(f"copysign.f32 s, r{r}, s;")
                o(f"mul.rn.f32 h{r}, h{r}, s;")
                o(f"setp.eq.f32 p, r{r}, 0f00000000;")
                o(f"selp.f32 h{r}, 0f00000000, h{r}, p;")
            self.pack("h", "g")
        self.nxt()

    def build(self):
        o = self.o
        o("{")
        o(".reg .b64 g<2>, ua<2>, vb<2>, uan<2>, vbn<2>, e<2>, aq<2>, cc<2>, v<6>, c1, c2;")
        o(".reg .f32 r<4>, h<4>, s, cf, m;")
        o(".reg .u32 x, y, z, w, nx, ny, nz, nw, opc, ad, pa, kk, k, sh, q<2>;")
        o(".reg .b32 z<4>;")
        o(".reg .s32 ks;")
        o(".reg .pred p, pv<4>;")
        o("mov.b64 g0, {%7, %8};")
        o("mov.b64 g1, {%9, %10};")
        for r in range(4):
            o(f"and.b32 kk, %15, {1 << r};")
            o(f"setp.ne.u32 pv{r}, kk, 0;")
        o("setp.eq.u32 p, %1, 0;")
        o("@p bra RV_DONE;")
        o("ld.shared.v4.u32 {x, y, z, w}, [%0];")
        o("sub.u32 %0, %0, 16;")
        o("sub.u32 %1, %1, 1;")
        o("add.u32 ad, %11, y;")
        o("ld.shared.v2.b64 {ua0, ua1}, [ad];")
        o("add.u32 ad, %11, z;")
        o("ld.shared.v2.b64 {vb0, vb1}, [ad];")
        # the table: forms 0..63, then the same forms after loading g from V
        hot = {RV_CONST: "RV_CONST"}
        for u in (U_SIN, U_COS, U_EXP, U_SQUARE, U_LOG_ABS, U_LOG, U_SQRT, U_SQRT_ABS):
            hot[RV_UN + u] = f"RV_U{u}"
        for grp in range(6):
            for kind in (K_ADD, K_SUB, K_MUL, K_AQ):
                hot[RV_BIN + grp * 6 + kind] = f"RV_B{grp}_{kind}"
        targets = [hot.get(i, "RV_COLD") for i in range(RV_GSM)]
        targets += [f"RV_G{i}" if i in hot else "RV_COLD" for i in range(RV_GSM)]
        o("RV_TBL: .branchtargets " + ", ".join(targets) + ";")
        self.label("RV_LOOP")
        o("setp.eq.u32 p, %1, 0;")
        o("selp.b32 pa, %14, %0, p;")  # nothing left: a harmless in-range read
        o("ld.shared.v4.u32 {nx, ny, nz, nw}, [pa];")
        o("add.u32 ad, %11, ny;")
        o("ld.shared.v2.b64 {uan0, uan1}, [ad];")
        o("add.u32 ad, %11, nz;")
        o("ld.shared.v2.b64 {vbn0, vbn1}, [ad];")
        o("mov.b32 cf, w;")
        o("and.b32 opc, x, 127;")
        o("brx.idx.uni opc, RV_TBL;")
        # GSM entries: the adjoint of a pushed value, from its V entry
        for i in sorted(hot):
            self.label(f"RV_G{i}")
            o("shr.u32 kk, x, 16;")
            o("mad.lo.u32 ad, kk, 512, %12;")
            o("ld.shared.v2.b64 {g0, g1}, [ad];")
            o(f"bra.uni {hot[i]};")
        self.label("RV_CONST")
        self.erc("g")
        self.nxt()
        for u in (U_SIN, U_COS, U_EXP, U_SQUARE, U_LOG_ABS, U_LOG, U_SQRT, U_SQRT_ABS):
            self.label(f"RV_U{u}")
            self.un_form(u)
        for grp in range(6):
            for kind in (K_ADD, K_SUB, K_MUL, K_AQ):
                self.label(f"RV_B{grp}_{kind}")
                self.bin_form(grp, kind)
        self.label("RV_NEXT")
        o("setp.eq.u32 p, %1, 0;")
        o("@p bra RV_DONE;")
        o("mov.u32 x, nx;")
        o("mov.u32 y, ny;")
        o("mov.u32 z, nz;")
        o("mov.u32 w, nw;")
        for i in range(2):
            o(f"mov.b64 ua{i}, uan{i};")
            o(f"mov.b64 vb{i}, vbn{i};")
        o("sub.u32 %0, %0, 16;")
        o("sub.u32 %1, %1, 1;")
        o("bra.uni RV_LOOP;")
        self.label("RV_COLD")
        o("mov.u32 %2, 1;")
        o("mov.u32 %3, x;")
        o("mov.u32 %4, y;")
        o("mov.u32 %5, z;")
        o("mov.u32 %6, w;")
        o("bra.uni RV_OUT;")
        self.label("RV_DONE")
        o("mov.u32 %2, 0;")
        self.label("RV_OUT")
        o("mov.b64 {%7, %8}, g0;")
        o("mov.b64 {%9, %10}, g1;")
        o("}")
        return self.lines


def emit_rev() -> str:
    lines = RevGen().build()
    body = "\n".join('      "' + ln + '\\n\\t"' for ln in lines)
    return ("__device__ __forceinline__ void interp_rev_asm(float (&G)[4], uint32_t& rp,\n"
            "    uint32_t& cnt, uint32_t& code, uint32_t& dx, uint32_t& dy, uint32_t& dz,\n"
            "    uint32_t& dw, uint32_t wl, uint32_t wlv, uint32_t wpe, uint32_t rbase,\n"
            "    uint32_t vmask) {\n"
            "  asm volatile(\n" + body + "\n"
            '      : "+r"(rp), "+r"(cnt), "=r"(code), "=r"(dx), "=r"(dy), "=r"(dz), "=r"(dw),\n'
            '        "+f"(G[0]), "+f"(G[1]), "+f"(G[2]), "+f"(G[3])\n'
            '      : "r"(wl), "r"(wlv), "r"(wpe), "r"(rbase), "r"(vmask)\n'
            '      : "memory");\n'
            "}\n")


def emit(R: int, special: bool, tape: bool = False) -> str:
    g = Gen(R, special, tape)
    lines = g.build()
    body = "\n".join('      "' + ln + '\\n\\t"' for ln in lines)
    outs = ", ".join(f'"+f"(A[{r}])' for r in range(R))
    name, extra_param, extra_op = "interp_asm", "", ""
    if tape:
        name, extra_param, extra_op = "interp_tape_asm", ", uint32_t& tp", ', "+r"(tp)'
    return (f"template <>\n"
            f"__device__ __forceinline__ void {name}<{R}>(float (&A)[{R}], uint32_t& pc,\n"
            f"    uint32_t& sp, uint32_t xs, uint32_t& code, uint32_t& arg{extra_param}) {{\n"
            f"  asm volatile(\n{body}\n"
            f'      : "+r"(pc), "+r"(sp), "+r"(code), "+r"(arg), {outs}{extra_op}\n'
            f'      : "r"(xs)\n'
            f'      : "memory");\n'
            f"}}\n")


def generate() -> str:
    head = ("// Generated by interp_gen.py (run by build.py); do not edit.\n"
            "// The interpreter's dispatch loop as inline PTX for 8 and 4 rows per lane,\n"
            "// and with a value tape (the adjoint's forward half) for 4 rows per lane;\n"
            "// the staged adjoint's reverse sweep (4 rows per lane).\n"
            "template <int R>\n"
            "__device__ __forceinline__ void interp_asm(float (&A)[R], uint32_t& pc,\n"
            "    uint32_t& sp, uint32_t xs, uint32_t& code, uint32_t& arg);\n"
            "template <int R>\n"
            "__device__ __forceinline__ void interp_tape_asm(float (&A)[R], uint32_t& pc,\n"
            "    uint32_t& sp, uint32_t xs, uint32_t& code, uint32_t& arg, uint32_t& tp);\n\n")
    # The 8-row PTX leaves the rare row-by-row groups of exp, log and sqrt to
    # the C++ cold path: their bodies, four row pairs long, made the hot
    # code larger than the instruction cache serves well (measured on the
    # largest workload: 53.0 ms per step without them, 66.9 ms with).  The
    # 4-row PTX, half the size, keeps them (the autotuner picks it for the
    # operator sets whose unprotected log and sqrt often meet negatives).
    return (head + emit(8, special=False) + "\n" + emit(4, special=True) + "\n" +
            emit(4, special=True, tape=True) + "\n" + emit_rev())


def main(out_path: str) -> None:
    text = generate()
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    old = None
    if os.path.exists(out_path):
        with open(out_path) as fh:
            old = fh.read()
    if old != text:  # keep the timestamp (and the build's up-to-date check) otherwise
        with open(out_path, "w") as fh:
            fh.write(text)


if __name__ == "__main__":
    main(sys.argv[1])
