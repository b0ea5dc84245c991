"""Generates the inline-PTX interpreter loops of the CUDA library.

Each interpreter is one PTX block: every body loads the next 16-byte
instruction from shared memory (one broadcast load per warp) as soon as it has
read its own payloads, then returns to a single ``brx.idx.uni`` jump through a
table straight to the body of the next (function, operand forms, stack level)
combination; a sentinel instruction written after the program jumps out.  The stack levels live in
registers whose names are fixed in each body, so no body indexes a register
at run time (Sec. 6.2 of the paper keeps low stack levels in registers behind
a switch on the stack pointer; here the level is resolved by the encoder and
the switch disappears into the jump).  Pairs of fitness cases are packed
``.b64`` registers operated on by the f32x2 instructions of sm_100+
(add/sub/mul.rn.f32x2), so a K-case body issues K/2 arithmetic instructions
(Sec. 6.1's float2/float4 idea, with a wide ALU behind it on this GPU).
Protected division shares one block per interpreter: operands are copied to
temporaries, divided (emit_pdiv: a correctly rounded reciprocal-and-remainder
sequence on case pairs, with ``div.rn.f32`` as the slow path for extreme
operands) and stored back through a second jump table on the level.

The instruction codes follow ``csrc/isa.h``.  Output: ``gen_interp.h`` with
one string macro per (interpreter, K, input mode), used by
``csrc/eval_float.cuh`` and ``csrc/eval_bool.cuh``.

Operand conventions of the generated asm (documented again in the header).
H = K/2 register units per stack level (one f32 when K == 1, else b64 case
pairs), RH = 8 * H:
  float S-form / RPN / register GP, K >= 2: in-out %0..%{RH-1} the stack
     levels (or registers), level l at %{l*H}..%{l*H+H-1}; the caller keeps
     them between entries, so they are defined once, not at every entry;
     output %{RH} bad flag (u32);
     inputs  %{RH+1} program address (shared, u32), %{RH+2} instruction count,
     then XREG (single input in registers): the K input values (f32);
          XSMEM (inputs staged in shared memory): this lane's tile address
          (u32), input v of this lane's K cases at tile + v*128*K bytes;
          register GP: the tile address, then the number of staged inputs
          (registers beyond start at 0)
  the same with K = 1, and the S-form with levels 4..7 in shared memory
     (K = 8): outputs %0..%{K-1} level-0 values (f32), %K bad; inputs
     %{K+1} program address, %{K+2} count, then the inputs as above (the
     study kernel then this lane's spill address)
  Boolean (words): outputs %0..%{K-1} level-0 words (u32), %K bad;
     inputs  %{K+1} program address, %{K+2} count, %{K+3} tile address
"""
from __future__ import annotations

import os

R = 8
NREG = 8
# csrc/isa.h
SF_FORMS = ["XX", "XC", "CX", "CC", "SX", "XS", "SC", "CS", "SS", "SSR", "MOVX", "MOVC", "XI", "SI", "CI"]
# division by a constant with its reciprocal in payload c (numerator X, S or C)
SF_RECIP = ("XI", "SI", "CI")
RF_FORMS = ["PUSHX", "PUSHC", "OP", "OPR"]
BF_FORMS = ["XX", "XS", "SX", "SS", "SSR"]
BOOL_IF_BASE = len(BF_FORMS) * R * 4
BOOL_MOVX = BOOL_IF_BASE + 16 * R
F32X2 = {0: "add.rn.f32x2", 1: "sub.rn.f32x2", 2: "mul.rn.f32x2"}
F32 = {0: "add.rn.f32", 1: "sub.rn.f32", 2: "mul.rn.f32"}
# lop3 truth tables with a = 0xF0, b = 0xCC, c = 0xAA
LUT = {0: 0xC0, 1: 0xFC, 2: 0x3F, 3: 0x03}  # AND, OR, NAND, NOR of (a, b)
LUT_IF = 0xCA                                 # (a & b) | (~a & c)


def sform_code(form, level, op):
    return (form * R + level) * 4 + op


def rpn_code(form, level, op):
    return (form * R + level) * 4 + op


def lin_code(op, a, b):
    return (op * NREG + a) * NREG + b


def if_descs():
    out = []
    for t in range(64):
        d = (t // 16, (t // 4) % 4, t % 4)
        m = sum(1 for v in d if v > 0)
        used, ok = [], True
        for v in d:
            if v > 0:
                if v - 1 >= m or (v - 1) in used:
                    ok = False
                used.append(v - 1)
        if ok:
            out.append(d)
    assert len(out) == 16
    return out


# bounds of the fast division path on both operands: 2^-50 and 2^50 as binary32
# bit patterns
DIV_LO = "0f26800000"
DIV_HI = "0f58800000"


def _reduce3(b, op, vals, out):
    """out = op over vals (NaN-propagating), three operands per instruction."""
    vals = list(vals)
    n = 0
    while len(vals) > 1:
        nxt = []
        for j in range(0, len(vals), 3):
            g = vals[j:j + 3]
            if len(g) == 1:
                nxt.append(g[0])
                continue
            d = out if len(vals) <= 3 else f"{out}_{n}"
            n += 1
            b(f"{op}.NaN.f32 {d}, {', '.join(g)};")
            nxt.append(d)
        vals = nxt
    if vals[0] != out:
        b(f"mov.f32 {out}, {vals[0]};")


def emit_pdiv(b, K, A, B, Q, tag, group=2, fold=None):
    """Protected division Q = (B == 0) ? 1 : A / B, correctly rounded, for the
    register units A, B, Q (K == 1: one f32 each; else b64 case pairs).

    Fast path (no branch): reciprocal seed y0 = rcp.approx(b), one
    Newton-Raphson step y1 = y0 + y0 (1 - b y0), the quotient q0 = a y1, the
    exact remainder r = a - b q0 (one FMA) and Markstein's correction
    q1 = q0 + r y1 (P. Markstein, IBM J. Res. Dev. 34(1), 1990), in
    fma/mul.rn.f32x2, `group` pairs interleaved at a time.  The fast result
    of a lane is kept when every operand of the lane lies in
    2^-50 <= |a|, |b| <= 2^50 (three-input NaN-propagating min and max, so a
    NaN anywhere fails).  Inside that box every intermediate value is normal,
    the remainder is exact and the quotient lies in [2^-100, 2^100], so the
    sequence is a power-of-two scaling of the same sequence on the
    significands in [1, 2), which is checked exhaustively.  The test reads
    only the operands, so it runs beside the division chain rather than
    after it, and the branch finds its predicate ready.  Any other lane (a
    zero, subnormal, huge or non-finite operand, a zero denominator) takes
    the slow path: div.rn.f32 and the protection select for each element.

    Without `fold` the slow path is a per-lane branch to the emit_pdiv_slow
    block, which must follow in the same asm block; Q may then name the same
    registers as A (quotients stay in dQ until the end).  With `fold` the
    decision is made once per warp: a vote sets `dall` when every lane passed,
    the fast quotients are written to Q, and fold() emits what the caller does
    when `dall` is false (the interpreters redirect their dispatch to an
    emit_pdiv_slow_body block, which recomputes every element exactly, so no
    branch sits in the division's own path).  Q must then not overlap A or B.
    Scratch registers come from pdiv_regs()."""
    H = len(A)
    if K == 1:
        b(f"abs.f32 dt, {A[0]};")
        b(f"abs.f32 dt2, {B[0]};")
        b("min.NaN.f32 dlo, dt, dt2;")
        b("max.NaN.f32 dhi, dt, dt2;")
        b(f"rcp.approx.ftz.f32 dY0, {B[0]};")
        b(f"neg.f32 dN0, {B[0]};")
        b("fma.rn.f32 dE0, dN0, dY0, 0f3F800000;")
        b("fma.rn.f32 dY0, dY0, dE0, dY0;")
        b(f"mul.rn.f32 dQ0, {A[0]}, dY0;")
        b(f"fma.rn.f32 dE0, dN0, dQ0, {A[0]};")
        b("fma.rn.f32 dQ0, dE0, dY0, dQ0;")
    else:
        # the operand test: |a| and |b| of every element, min and max trees
        mags = []
        for i in range(H):
            for src, nm in ((A[i], "dma"), (B[i], "dmb")):
                b(f"mov.b64 {{{nm}{2 * i}, {nm}{2 * i + 1}}}, {src};")
                b(f"abs.f32 {nm}{2 * i}, {nm}{2 * i};")
                b(f"abs.f32 {nm}{2 * i + 1}, {nm}{2 * i + 1};")
                mags += [f"{nm}{2 * i}", f"{nm}{2 * i + 1}"]
        _reduce3(b, "min", mags, "dlo")
        _reduce3(b, "max", mags, "dhi")
        for g0 in range(0, H, group):
            idx = list(range(g0, min(H, g0 + group)))
            # the reciprocal of -b: every step below is the scalar sequence's
            # value negated (rounding to nearest is symmetric), so no
            # negation of b is needed; one multiplication by -1 at the end
            for i in idx:
                b(f"mov.b64 {{dt, dt2}}, {B[i]};")
                b("neg.f32 dt, dt;")
                b("neg.f32 dt2, dt2;")
                b("rcp.approx.ftz.f32 dt, dt;")
                b("rcp.approx.ftz.f32 dt2, dt2;")
                b(f"mov.b64 dY{i}, {{dt, dt2}};")             # -y0
            for i in idx:
                b(f"fma.rn.f32x2 dE{i}, {B[i]}, dY{i}, one2;")  # e = 1 - b y0
            for i in idx:
                b(f"fma.rn.f32x2 dY{i}, dY{i}, dE{i}, dY{i};")  # -y1
            for i in idx:
                b(f"mul.rn.f32x2 dQ{i}, {A[i]}, dY{i};")        # -q0
            for i in idx:
                b(f"fma.rn.f32x2 dE{i}, {B[i]}, dQ{i}, {A[i]};")  # r = a - b q0
            for i in idx:
                b(f"fma.rn.f32x2 dQ{i}, dE{i}, dY{i}, dQ{i};")  # -q1
    b(f"setp.ge.f32 dok, dlo, {DIV_LO};")
    b(f"setp.le.and.f32 dok, dhi, {DIV_HI}, dok;")
    if fold is None:
        if K > 1:  # (the slow path leaves the quotients in dQ with their signs)
            for i in range(H):
                b(f"mul.rn.f32x2 dQ{i}, dQ{i}, mone2;")
        b(f"@!dok bra {tag}SLOW;")
        b(f"{tag}RET:")
        if K == 1:
            b(f"mov.f32 {Q[0]}, dQ0;")
        else:
            for i in range(H):
                b(f"mov.b64 {Q[i]}, dQ{i};")
    else:
        b("vote.sync.all.pred dall, dok, 0xffffffff;")
        if K == 1:
            b(f"mov.f32 {Q[0]}, dQ0;")
        else:  # the sign restored straight into the destination
            for i in range(H):
                b(f"mul.rn.f32x2 {Q[i]}, dQ{i}, mone2;")
    if fold is not None:
        fold()


def emit_pdiv_slow(b, K, A, B, tag):
    """Out-of-line slow path of emit_pdiv: IEEE division and the protection
    select (zero denominator -> 1) of every element into dQ, then back."""
    b(f"{tag}SLOW:")
    if K == 1:
        b(f"div.rn.f32 dQ0, {A[0]}, {B[0]};")
        b(f"setp.eq.f32 dz, {B[0]}, 0f00000000;")
        b("selp.f32 dQ0, 0f3F800000, dQ0, dz;")
    else:
        for i in range(len(A)):
            b(f"mov.b64 {{dlo, dhi}}, {A[i]};")
            b(f"mov.b64 {{dt, dt2}}, {B[i]};")
            b("div.rn.f32 dlo, dlo, dt;")
            b("setp.eq.f32 dz, dt, 0f00000000;")
            b("selp.f32 dlo, 0f3F800000, dlo, dz;")
            b("div.rn.f32 dhi, dhi, dt2;")
            b("setp.eq.f32 dz, dt2, 0f00000000;")
            b("selp.f32 dhi, 0f3F800000, dhi, dz;")
            b(f"mov.b64 dQ{i}, {{dlo, dhi}};")
    b(f"bra {tag}RET;")


def emit_pdiv_slow_body(b, K, A, B, Q, tag):
    """The slow path of a folded emit_pdiv as a block of its own (label
    {tag}SLOW): IEEE division and the protection select of every element of
    A / B, written into Q.  The caller continues the dispatch after it."""
    b(f"{tag}SLOW:")
    if K == 1:
        b(f"div.rn.f32 {Q[0]}, {A[0]}, {B[0]};")
        b(f"setp.eq.f32 dz, {B[0]}, 0f00000000;")
        b(f"selp.f32 {Q[0]}, 0f3F800000, {Q[0]}, dz;")
        return
    for i in range(len(A)):
        b(f"mov.b64 {{dlo, dhi}}, {A[i]};")
        b(f"mov.b64 {{dt, dt2}}, {B[i]};")
        b("div.rn.f32 dlo, dlo, dt;")
        b("setp.eq.f32 dz, dt, 0f00000000;")
        b("selp.f32 dlo, 0f3F800000, dlo, dz;")
        b("div.rn.f32 dhi, dhi, dt2;")
        b("setp.eq.f32 dz, dt2, 0f00000000;")
        b("selp.f32 dhi, 0f3F800000, dhi, dz;")
        b(f"mov.b64 {Q[i]}, {{dlo, dhi}};")


def emit_pdivi(b, K, A, Nb, Yc, Q, fold=None):
    """Protected division Q = A / b by a constant b in the fast range whose
    reciprocal y = RN(1/b) the encoder supplies (the SF_XI / SF_SI / SF_CI
    forms): the register units A (K == 1: f32; else b64 case pairs), and the
    registers Nb holding b (one value, or the pair {b, b}), turned into -b
    here, and Yc holding y (or {y, y}).

    With y correctly rounded the reciprocal needs no seed and no
    Newton-Raphson step: the quotient q0 = a y, the exact remainder
    r = a - b q0 (one FMA with -b) and Markstein's correction q1 = q0 + r y
    (P. Markstein, IBM J. Res. Dev. 34(1), 1990), checked equal to correctly
    rounded division over every pair of significands.  b lies in the fast
    range (the encoder's choice), so only the numerators are tested: every
    |a| in [2^-50, 2^50] (NaN-propagating min and max).  With `fold` the
    decision is once per warp (a vote into `dall`, the quotients written to
    Q, fold() redirecting the dispatch to a slow body, which takes its
    divisor from Nb = -b, when `dall` is false); without it (fold is None)
    there is no test at all, for a constant numerator the encoder has
    checked.  Q must not overlap A.  Each case pair runs its three steps in
    turn, which keeps two temporaries live instead of 2 K."""
    H = len(A)
    if K == 1:
        b(f"neg.f32 {Nb}, {Nb};")
        if fold is not None:
            b(f"abs.f32 dt, {A[0]};")
            b(f"setp.ge.f32 dok, dt, {DIV_LO};")
            b(f"setp.le.and.f32 dok, dt, {DIV_HI}, dok;")
        b(f"mul.rn.f32 dQ0, {A[0]}, {Yc};")
        b(f"fma.rn.f32 dE0, {Nb}, dQ0, {A[0]};")
        b(f"fma.rn.f32 {Q[0]}, dE0, {Yc}, dQ0;")
    else:
        b(f"mul.rn.f32x2 {Nb}, {Nb}, mone2;")  # -b, exact
        if fold is not None:  # a running min and max, two temporaries
            for i in range(H):
                b(f"mov.b64 {{dma0, dma1}}, {A[i]};")
                b("abs.f32 dma0, dma0;")
                b("abs.f32 dma1, dma1;")
                if i == 0:
                    b("min.NaN.f32 dlo, dma0, dma1;")
                    b("max.NaN.f32 dhi, dma0, dma1;")
                else:
                    b("min.NaN.f32 dlo, dlo, dma0, dma1;")
                    b("max.NaN.f32 dhi, dhi, dma0, dma1;")
            b(f"setp.ge.f32 dok, dlo, {DIV_LO};")
            b(f"setp.le.and.f32 dok, dhi, {DIV_HI}, dok;")
        for i in range(H):
            b(f"mul.rn.f32x2 dQ0, {A[i]}, {Yc};")          # q0 = a y
            b(f"fma.rn.f32x2 dE0, {Nb}, dQ0, {A[i]};")     # r = a - b q0
            b(f"fma.rn.f32x2 {Q[i]}, dE0, {Yc}, dQ0;")      # q1 = q0 + r y
    if fold is not None:
        b("vote.sync.all.pred dall, dok, 0xffffffff;")
        fold()


def emit_pdivi_slow_body(b, K, A, Nb, Q, tag):
    """The slow path of a folded emit_pdivi as a block of its own (label
    {tag}SLOW): IEEE division of every element of A by b = -Nb (negated back
    exactly) and the protection select, written into Q."""
    b(f"{tag}SLOW:")
    if K == 1:
        b(f"neg.f32 dt, {Nb};")
        b(f"div.rn.f32 {Q[0]}, {A[0]}, dt;")
        b("setp.eq.f32 dz, dt, 0f00000000;")
        b(f"selp.f32 {Q[0]}, 0f3F800000, {Q[0]}, dz;")
        return
    b(f"mov.b64 {{dt, dt2}}, {Nb};")
    b("neg.f32 dt, dt;")
    b("neg.f32 dt2, dt2;")
    for i in range(len(A)):
        b(f"mov.b64 {{dlo, dhi}}, {A[i]};")
        b("div.rn.f32 dlo, dlo, dt;")
        b("setp.eq.f32 dz, dt, 0f00000000;")
        b("selp.f32 dlo, 0f3F800000, dlo, dz;")
        b("div.rn.f32 dhi, dhi, dt2;")
        b("setp.eq.f32 dz, dt2, 0f00000000;")
        b("selp.f32 dhi, 0f3F800000, dhi, dz;")
        b(f"mov.b64 {Q[i]}, {{dlo, dhi}};")


def pdiv_regs(K, H):
    ty = "f32" if K == 1 else "b64"
    n = 2 * H
    return (f".reg .{ty} dY<{H}>, dE<{H}>, dN<{H}>, dQ<{H}>, one2, mone2, cY, cN;\n"
            f".reg .f32 dlo, dhi, dt, dt2, dma<{n}>, dmb<{n}>, dlo_<{n}>, dhi_<{n}>;\n"
            f".reg .pred dok, dz, dall;")



class Block:
    def __init__(self):
        self.lines = []

    def __call__(self, s):
        self.lines.append(s)

    def macro(self, name, doc):
        body = "".join(f'  "{ln}\\n\\t" \\\n' for ln in self.lines)
        return f"// {doc}\n#define {name} \\\n{body}  \"\"\n"


# ---------------------------------------------------------------------------
# float interpreters
# ---------------------------------------------------------------------------
class FloatGen:
    """One dispatch site (LOOP: brx on the current code).  Every body loads
    the next instruction right after reading its own payloads, so the
    shared-memory load overlaps the body's arithmetic, and branches back to
    LOOP.  (Ending each body with its own brx -- direct threading -- was
    measured to be slower: several hundred indirect-branch sites.)  The kernel
    writes a sentinel instruction (code n_codes) after the last one; its table
    entry is DONE, so the loop needs no bound check.  Codes are validated when
    the program is staged, so no code is clamped."""

    def __init__(self, K, xmode, rl=R):
        assert K in (1, 2, 4, 8) and xmode in ("reg", "smem") and 1 <= rl <= R
        self.K, self.xmode = K, xmode
        self.H = 1 if K == 1 else K // 2   # register units per stack level
        # all levels in registers, K >= 2: they are asm operands the caller
        # keeps across entries (no zeroing at each entry, no copy of level 0
        # out); else level-0 outputs and block-local stack registers.  (At
        # K = 1 the operand form costs the 1D kernel 16 registers and an
        # occupancy step: measured 3% slower.)
        self.stack_ops = rl == R and K >= 2
        base = R * self.H if self.stack_ops else K
        self.o_bad, self.o_prog, self.o_cnt, self.o_x = base, base + 1, base + 2, base + 3
        self.b = Block()
        self.stride = 128 * K              # bytes between inputs in a lane's tile
        # levels rl .. R-1 live in shared memory: per warp [level][chunk][lane]
        # with 16-byte chunks (K >= 4), so a warp's access is conflict-free
        self.rl = rl
        self.chunk = min(16, 4 * K)        # bytes of one lane's chunk
        self.nchunk = 4 * K // self.chunk  # chunks per lane per level
        # division's slow path: decided once per warp and taken through the
        # dispatch (fold_to_slow), or a per-lane branch
        self.fold_div = True

    # register unit names
    def lev(self, l, i):
        if self.stack_ops:
            return f"%{l * self.H + i}"
        return f"s{l * self.H + i}"

    def xreg(self, i):
        return f"x{i}"

    @property
    def ty(self):
        return "f32" if self.K == 1 else "b64"

    def header(self, extra_regs=""):
        K, H, b = self.K, self.H, self.b
        b("{")
        b(f".reg .{self.ty} ta<{H}>, tb<{H}>, xA<{H}>, xB<{H}>, cA, cB;")
        if not self.stack_ops:
            b(f".reg .{self.ty} s<{self.rl * H}>;")
        if self.rl < R:
            b(f".reg .{self.ty} sA<{H}>, sB<{H}>;")
            b(".reg .b32 sbase;")
        if self.xmode == "reg":
            b(f".reg .{self.ty} x<{H}>;")
        b(".reg .b32 code, pa, pb, pc, adr, dl, xa, xbase;")
        b(".reg .pred p;")
        for ln in pdiv_regs(K, H).split("\n"):
            b(ln)
        if K > 1:
            b("mov.b64 one2, 0x3F8000003F800000;")
            b("mov.b64 mone2, 0xBF800000BF800000;")
        if extra_regs:
            b(extra_regs)
        # Block-local stack registers are defined before the first jump: the
        # jump table makes any of them readable at every body, so an undefined
        # one would be live from the kernel's entry and could not share a
        # physical register with the other interpreters of the same kernel.
        # (Operand levels are defined once by the caller instead.)
        if not self.stack_ops:
            zero = "0f00000000" if K == 1 else "0"
            for r in range(self.rl * H):
                b(f"mov.{self.ty} s{r}, {zero};")

    # levels in shared memory (rl <= l < R)
    def spill_off(self, l, q):
        return ((l - self.rl) * self.nchunk + q) * 32 * self.chunk

    def spill_load(self, l, dst):
        b, K = self.b, self.K
        for q in range(self.nchunk):
            off = self.spill_off(l, q)
            if K == 1:
                b(f"ld.shared.f32 {dst[0]}, [sbase+{off}];")
            elif K == 2:
                b(f"ld.shared.b64 {dst[0]}, [sbase+{off}];")
            else:
                b(f"ld.shared.v2.b64 {{{dst[2 * q]}, {dst[2 * q + 1]}}}, [sbase+{off}];")
        return dst

    def spill_store(self, l, src):
        b, K = self.b, self.K
        for q in range(self.nchunk):
            off = self.spill_off(l, q)
            if K == 1:
                b(f"st.shared.f32 [sbase+{off}], {src[0]};")
            elif K == 2:
                b(f"st.shared.b64 [sbase+{off}], {src[0]};")
            else:
                b(f"st.shared.v2.b64 [sbase+{off}], {{{src[2 * q]}, {src[2 * q + 1]}}};")

    def load_x(self, dst, payload):
        """Loads input `payload` (a b32 register) for this lane's K cases into
        the register units `dst` (list of H names)."""
        K, b = self.K, self.b
        if self.xmode == "reg":
            return [self.xreg(i) for i in range(self.H)]
        b(f"mad.lo.u32 xa, {payload}, {self.stride}, xbase;")
        if K == 1:
            b(f"ld.shared.f32 {dst[0]}, [xa];")
        elif K == 2:
            b(f"ld.shared.b64 {dst[0]}, [xa];")
        elif K == 4:
            b(f"ld.shared.v2.b64 {{{dst[0]}, {dst[1]}}}, [xa];")
        else:
            b(f"ld.shared.v2.b64 {{{dst[0]}, {dst[1]}}}, [xa];")
            b(f"ld.shared.v2.b64 {{{dst[2]}, {dst[3]}}}, [xa+16];")
        return dst

    def const(self, reg, payload):
        if self.K == 1:
            self.b(f"mov.b32 {reg}, {payload};")
        else:
            self.b(f"mov.b64 {reg}, {{{payload}, {payload}}};")
        return [reg] * self.H

    def vop(self, op, d, a, c):
        for i in range(self.H):
            if self.K == 1:
                self.b(f"{F32[op]} {d[i]}, {a[i]}, {c[i]};")
            else:
                self.b(f"{F32X2[op]} {d[i]}, {a[i]}, {c[i]};")

    def copy(self, d, a):
        for i in range(self.H):
            self.b(f"mov.{self.ty} {d[i]}, {a[i]};")

    # dispatch pieces
    def fetch(self):
        """Loads the next instruction (call after the payloads are consumed)."""
        self.b("ld.shared.v4.u32 {code, pa, pb, pc}, [adr];")
        self.b("add.u32 adr, adr, 16;")

    def jump(self):
        self.b("bra.uni LOOP;")

    def table(self, n_codes, table, slow_levels=(), slow_levels_i=()):
        """The dispatch table TBL: the codes, then the sentinel (n_codes,
        DONE).  With slow_levels, a second table TBLD for the DIV blocks' own
        dispatch adds one entry per stack level, the folded division's slow
        body (n_codes + 1 + l), and with slow_levels_i one more per level for
        the division by a constant with its reciprocal (n_codes + 1 + R + l).
        A separate dispatch site keeps the division operands live only from a
        DIV block to its slow body: through the common site they would be
        live across every body of the loop."""
        self.n_codes = n_codes
        labels = [table.get(c, "CBAD") for c in range(n_codes)] + ["DONE"]
        self.b("TBL: .branchtargets " + ", ".join(labels) + ";")
        if slow_levels:
            labels += [f"D{l}_SLOW" if l in slow_levels else "CBAD" for l in range(R)]
            if slow_levels_i:
                labels += [f"DI{l}_SLOW" if l in slow_levels_i else "CBAD" for l in range(R)]
            self.b("TBLD: .branchtargets " + ", ".join(labels) + ";")

    def div_jump(self):
        """Dispatch after a folded division (the table with slow bodies)."""
        self.b("brx.idx.uni code, TBLD;")

    def fold_to_slow(self, l, recip=False):
        """fold() of a level-l division: when not every lane took the fast
        path, dispatch to the level's slow body instead of the next code
        (recip: the slow body of the division by a constant with its
        reciprocal)."""
        def emit():
            self.b(f"@!dall mov.u32 code, {self.n_codes + 1 + (R if recip else 0) + l};")
        return emit

    def slow_bodies(self, ta, tb, units_of_level, levels, tag="D"):
        """The slow bodies reload the next code from the instruction just
        fetched (adr was advanced past it) and dispatch it."""
        for l in levels:
            emit_pdiv_slow_body(self.b, self.K, ta, tb, units_of_level(l), f"{tag}{l}_")
            self.b("ld.shared.u32 code, [adr+-16];")
            self.jump()

    def prologue(self):
        b = self.b
        b(f"mov.u32 adr, %{self.o_prog};")
        b(f"mov.u32 %{self.o_bad}, 0;")

    def start(self):
        self.fetch()
        self.b("LOOP:")
        self.b("brx.idx.uni code, TBL;")

    def epilogue(self, out_units):
        b, K = self.b, self.K
        b("CBAD:")
        b(f"mov.u32 %{self.o_bad}, 1;")
        b("DONE:")
        if not self.stack_ops:  # (operand levels: level 0 is the output already)
            if K == 1:
                b(f"mov.f32 %0, {out_units[0]};")
            else:
                for i in range(self.H):
                    b(f"mov.b64 {{%{2 * i}, %{2 * i + 1}}}, {out_units[i]};")
        b("}")

    def setup_inputs(self):
        b, K = self.b, self.K
        if self.xmode == "reg":
            for i in range(self.H):
                if K == 1:
                    b(f"mov.f32 x0, %{self.o_x};")
                else:
                    b(f"mov.b64 x{i}, {{%{self.o_x + 2 * i}, %{self.o_x + 2 * i + 1}}};")
        else:
            b(f"mov.u32 xbase, %{self.o_x};")

    def store_table(self):
        self.b("STTBL: .branchtargets " + ", ".join(f"ST{l}" for l in range(R)) + ";")

    def store_bodies(self, units_of_level, src):
        for l in range(R):
            self.b(f"ST{l}:")
            self.copy(units_of_level(l), src)
            self.jump()

    def div_block(self, ta, tb, then_store=True):
        """DIV: ta <- ta / tb (protected), then jump on `dl` to a store body."""
        b = self.b
        b("DIV:")
        emit_pdiv(b, self.K, ta, tb, ta, "D")
        b("STORE:")
        b("brx.idx.uni dl, STTBL;")
        emit_pdiv_slow(b, self.K, ta, tb, "D")

    def div_blocks_per_level(self, ta, tb, units_of_level):
        """DIV_l, one per stack level: level l <- ta / tb (protected), written
        straight into the level's registers (no store jump, no copy back)."""
        for l in range(R):
            self.b(f"DIV{l}:")
            if self.fold_div:
                emit_pdiv(self.b, self.K, ta, tb, units_of_level(l), f"D{l}_", fold=self.fold_to_slow(l))
                self.div_jump()
            else:
                emit_pdiv(self.b, self.K, ta, tb, units_of_level(l), f"D{l}_")
                self.jump()
                emit_pdiv_slow(self.b, self.K, ta, tb, f"D{l}_")
        if self.fold_div:
            self.slow_bodies(ta, tb, units_of_level, range(R))

    # ------------------------------------------------------------------
    def sform(self):
        """S-form interpreter.  With rl < R the levels rl.. are in shared
        memory: a body loads a spilled operand into sA/sB and stores a spilled
        result back (one more asm operand, the lane's spill address)."""
        K, H, b = self.K, self.H, self.b
        self.header()
        rl = self.rl
        L = lambda l: [self.lev(l, i) for i in range(H)]
        ta = [f"ta{i}" for i in range(H)]
        tb = [f"tb{i}" for i in range(H)]
        xA = [f"xA{i}" for i in range(H)]
        xB = [f"xB{i}" for i in range(H)]
        sA = [f"sA{i}" for i in range(H)]
        sB = [f"sB{i}" for i in range(H)]
        n_codes = len(SF_FORMS) * R * 4
        table, bodies = {}, []
        for f, name in enumerate(SF_FORMS):
            for l in range(R):
                for op in range(4):
                    if name in ("SS", "SSR") and l + 1 >= R:
                        continue
                    if name in ("MOVX", "MOVC") and (l != 0 or op != 0):
                        continue
                    if name in SF_RECIP and op != 3:
                        continue
                    code = sform_code(f, l, op)
                    table[code] = f"C{code}"
                    bodies.append((code, name, l, op))
        self.table(n_codes, table, slow_levels=range(rl), slow_levels_i=range(rl))
        self.prologue()
        self.setup_inputs()
        if rl < R:
            b(f"mov.u32 sbase, %{self.sbase_operand()};")
        self.start()
        opnd = lambda l, tmp: L(l) if l < rl else self.spill_load(l, tmp)
        for code, name, l, op in bodies:
            b(f"C{code}:")
            if name == "MOVX":
                src = self.load_x(xA, "pa")
                self.fetch()
                self.copy(L(0), src)
                self.jump()
                continue
            if name == "MOVC":
                src = self.const("cA", "pa")
                self.fetch()
                self.copy(L(0), src)
                self.jump()
                continue
            if name in SF_RECIP:
                ka = name[0]
                a = opnd(l, sA) if ka == "S" else (self.load_x(xA, "pa") if ka == "X" else self.const("cA", "pa"))
                cb = self.const("cN" if l < rl else "cB", "pb")
                if l >= rl:  # a level in shared memory: the general division
                    self.copy(ta, a)
                    self.copy(tb, cb)
                    self.fetch()
                    b(f"bra.uni DIV{l};")
                    continue
                cy = self.const("cY", "pc")
                if name == "CI":  # both constants in the fast range: no test
                    self.fetch()
                    emit_pdivi(b, K, a, cb[0], cy[0], L(l))
                    self.jump()
                    continue
                self.copy(ta, a)
                self.fetch()
                b(f"bra.uni DIVI{l};")
                continue
            if name == "SS":
                a, c = opnd(l, sA), opnd(l + 1, sB)
            elif name == "SSR":
                a, c = opnd(l + 1, sA), opnd(l, sB)
            else:
                ka, kb = name[0], name[1]
                a = opnd(l, sA) if ka == "S" else (self.load_x(xA, "pa") if ka == "X" else self.const("cA", "pa"))
                c = opnd(l, sB) if kb == "S" else (self.load_x(xB, "pb") if kb == "X" else self.const("cB", "pb"))
            if op == 3:
                self.copy(ta, a)
                self.copy(tb, c)
                self.fetch()
                b(f"bra.uni DIV{l};")
            else:
                self.fetch()
                d = L(l) if l < rl else sA
                self.vop(op, d, a, c)
                if l >= rl:
                    self.spill_store(l, d)
                self.jump()
        for l in range(R):  # level l <- ta / tb (protected)
            b(f"DIV{l}:")
            if l < rl:
                emit_pdiv(b, K, ta, tb, L(l), f"D{l}_", fold=self.fold_to_slow(l))
                self.div_jump()
                continue
            emit_pdiv(b, K, ta, tb, ta, f"D{l}_")
            self.spill_store(l, ta)
            self.jump()
            emit_pdiv_slow(b, K, ta, tb, f"D{l}_")
        for l in range(rl):  # level l <- ta / b by its reciprocal (cN = b, cY)
            b(f"DIVI{l}:")
            emit_pdivi(b, K, ta, "cN", "cY", L(l), fold=self.fold_to_slow(l, recip=True))
            self.div_jump()
        self.slow_bodies(ta, tb, L, range(rl))
        for l in range(rl):
            emit_pdivi_slow_body(b, K, ta, "cN", L(l), f"DI{l}_")
            b("ld.shared.u32 code, [adr+-16];")
            self.jump()

        self.epilogue(L(0))
        return b

    def sbase_operand(self):
        """Operand index of the lane's spill address (after the inputs)."""
        return self.o_x + (self.K if self.xmode == "reg" else 1)

    def rpn(self):
        K, H, b = self.K, self.H, self.b
        self.header()
        L = lambda l: [self.lev(l, i) for i in range(H)]
        ta = [f"ta{i}" for i in range(H)]
        tb = [f"tb{i}" for i in range(H)]
        n_codes = len(RF_FORMS) * R * 4
        table, bodies = {}, []
        for f, name in enumerate(RF_FORMS):
            for l in range(R):
                for op in range(4):
                    if name in ("PUSHX", "PUSHC") and op != 0:
                        continue
                    if name in ("OP", "OPR") and l + 1 >= R:
                        continue
                    code = rpn_code(f, l, op)
                    table[code] = f"C{code}"
                    bodies.append((code, name, l, op))
        self.table(n_codes, table, slow_levels=range(R))
        self.prologue()
        self.setup_inputs()
        self.start()
        for code, name, l, op in bodies:
            b(f"C{code}:")
            if name == "PUSHX":
                if self.xmode == "reg":
                    self.fetch()
                    self.copy(L(l), [self.xreg(i) for i in range(H)])
                else:
                    self.load_x(L(l), "pa")
                    self.fetch()
                self.jump()
                continue
            if name == "PUSHC":
                src = self.const("cA", "pa")
                self.fetch()
                self.copy(L(l), src)
                self.jump()
                continue
            a, c = (L(l), L(l + 1)) if name == "OP" else (L(l + 1), L(l))
            self.fetch()
            if op == 3:
                self.copy(ta, a)
                self.copy(tb, c)
                b(f"bra.uni DIV{l};")
            else:
                self.vop(op, L(l), a, c)
                self.jump()
        self.div_blocks_per_level(ta, tb, L)
        self.epilogue(L(0))
        return b

    def linear(self):
        """Register machine r[d] = r[a] op r[b]; registers start from the staged
        inputs (register v < nin) or 0.  The body computes into ta, then jumps
        on d (the first payload) to the store of register d."""
        K, H, b = self.K, self.H, self.b
        assert self.xmode == "smem"
        self.header(".reg .b32 nin;")
        Rg = lambda r: [self.lev(r, i) for i in range(H)]
        ta = [f"ta{i}" for i in range(H)]
        tb = [f"tb{i}" for i in range(H)]
        n_codes = 4 * NREG * NREG
        table = {lin_code(op, a, c): f"C{lin_code(op, a, c)}"
                 for op in range(4) for a in range(NREG) for c in range(NREG)}
        self.store_table()
        self.table(n_codes, table)
        self.prologue()
        b(f"mov.u32 xbase, %{self.o_x};")
        b(f"mov.u32 nin, %{self.o_x + 1};")
        zero = "0f00000000" if K == 1 else "0"
        for r in range(NREG):
            b(f"setp.lt.u32 p, {r}, nin;")
            b(f"mov.u32 pa, {r};")
            units = Rg(r)
            b(f"@!p bra.uni Z{r};")
            self.load_x(units, "pa")
            b(f"bra.uni I{r};")
            b(f"Z{r}:")
            for u in units:
                b(f"mov.{self.ty} {u}, {zero};")
            b(f"I{r}:")
        self.start()
        for op in range(4):
            for a in range(NREG):
                for c in range(NREG):
                    code = lin_code(op, a, c)
                    b(f"C{code}:")
                    b("mov.u32 dl, pa;")
                    self.fetch()
                    if op == 3:
                        self.copy(ta, Rg(a))
                        self.copy(tb, Rg(c))
                        b("bra.uni DIV;")
                    else:
                        self.vop(op, ta, Rg(a), Rg(c))
                        b("bra.uni STORE;")
        self.div_block(ta, tb)
        self.store_bodies(Rg, ta)
        self.epilogue(Rg(0))
        return b


class FloatGenLoop(FloatGen):
    """The K = 8 S-form interpreter with its input in registers and the pass
    loop inside: each pass loads the lane's 8 inputs, runs the program, and at
    DONE adds the pass's errors to the fitness sum -- the fitness measure's
    error per case (%42: 0 |o - y|, 1 (o - y)^2, 2 the misclassification
    rint(o) != y; chosen once per pass), their pairwise sum and the
    compensated add, in the binary32 steps and order of the kernel's own pass
    code -- then takes the next pass.  No exit from the asm between passes.
    Operands: the stack (%0..%31), bad (%32), the sum and its compensation
    (%33, %34), the fitness flags (%35); the program's shared address (%36),
    its instruction count (%37, unused), the lane's first inputs and targets
    (%38, %39: global addresses), the passes (%40, at least 1), the bytes
    from one pass to the next (%41) and the fitness measure (%42)."""

    FLAG_NONFINITE = 1  # the kernel's fitness flag for a non-finite error
    FIT_MSE, FIT_CLASS = 1, 2  # the kernel's fitness measures (0: sum of |o - y|)

    def __init__(self):
        super().__init__(8, "reg")
        assert self.stack_ops
        self.o_bad, self.o_sum, self.o_comp, self.o_flags = 32, 33, 34, 35
        self.o_prog, self.o_cnt = 36, 37
        self.o_xp, self.o_yp, self.o_np, self.o_st, self.o_fit = 38, 39, 40, 41, 42

    def header(self, extra_regs=""):
        super().header(extra_regs)
        for decl in (".reg .b64 xp, yp, stp;", ".reg .b32 npl;", ".reg .f32 e<8>, ey<8>, csa, csb;",
                     ".reg .pred pnf, pmore, pmse, pcls;"):
            self.b(decl)

    def prologue(self):
        b = self.b
        b(f"mov.u32 %{self.o_bad}, 0;")
        b(f"cvta.to.global.u64 xp, %{self.o_xp};")
        b(f"cvta.to.global.u64 yp, %{self.o_yp};")
        b(f"mov.u32 npl, %{self.o_np};")
        b(f"mov.b64 stp, %{self.o_st};")
        b("PASS:")
        b("ld.global.nc.v4.f32 {e0, e1, e2, e3}, [xp];")
        b("ld.global.nc.v4.f32 {e4, e5, e6, e7}, [xp+16];")
        for i in range(self.H):
            b(f"mov.b64 x{i}, {{e{2 * i}, e{2 * i + 1}}};")
        b(f"mov.u32 adr, %{self.o_prog};")

    def setup_inputs(self):
        pass  # loaded at each pass (prologue)

    def epilogue(self, out_units):
        b = self.b
        b("CBAD:")
        b(f"mov.u32 %{self.o_bad}, 1;")
        b("bra.uni EXIT;")
        b("DONE:")
        b("ld.global.nc.v4.f32 {ey0, ey1, ey2, ey3}, [yp];")
        b("ld.global.nc.v4.f32 {ey4, ey5, ey6, ey7}, [yp+16];")
        for i in range(self.H):
            b(f"mov.b64 {{e{2 * i}, e{2 * i + 1}}}, {out_units[i]};")
        b(f"setp.eq.u32 pmse, %{self.o_fit}, {self.FIT_MSE};")
        b(f"setp.eq.u32 pcls, %{self.o_fit}, {self.FIT_CLASS};")
        b("@pmse bra.uni EMSE;")
        b("@pcls bra.uni ECLS;")
        for j in range(8):  # |o - y|
            b(f"sub.rn.f32 e{j}, e{j}, ey{j};")
            b(f"abs.f32 e{j}, e{j};")
        b("bra.uni ESUM;")
        b("EMSE:")
        for j in range(8):  # (o - y)^2
            b(f"sub.rn.f32 e{j}, e{j}, ey{j};")
            b(f"mul.rn.f32 e{j}, e{j}, e{j};")
        b("bra.uni ESUM;")
        b("ECLS:")
        for j in range(8):  # rint(o) != y
            b(f"cvt.rni.f32.f32 e{j}, e{j};")
            b(f"setp.eq.f32 pnf, e{j}, ey{j};")
            b(f"selp.f32 e{j}, 0f00000000, 0f3F800000, pnf;")
        b("ESUM:")
        for w in (1, 2, 4):
            for j in range(0, 8, 2 * w):
                b(f"add.rn.f32 e{j}, e{j}, e{j + w};")
        # a non-finite pass sum (errors are >= 0) flags the fitness
        b("setp.le.f32 pnf, e0, 0f7F7FFFFF;")
        b(f"@!pnf or.b32 %{self.o_flags}, %{self.o_flags}, {self.FLAG_NONFINITE};")
        # compensated add: t = s + e; c += (max(s, e) - t) + min(s, e); s = t
        b(f"add.rn.f32 csa, %{self.o_sum}, e0;")
        b(f"max.f32 csb, %{self.o_sum}, e0;")
        b(f"min.f32 e1, %{self.o_sum}, e0;")
        b("sub.rn.f32 csb, csb, csa;")
        b("add.rn.f32 csb, csb, e1;")
        b(f"add.rn.f32 %{self.o_comp}, %{self.o_comp}, csb;")
        b(f"mov.f32 %{self.o_sum}, csa;")
        b("add.u64 xp, xp, stp;")
        b("add.u64 yp, yp, stp;")
        b("sub.u32 npl, npl, 1;")
        b("setp.ne.u32 pmore, npl, 0;")
        b("@pmore bra.uni PASS;")
        b("EXIT:")
        b("}")


# ---------------------------------------------------------------------------
# register linear GP with the register file in shared memory
# ---------------------------------------------------------------------------
class LinearRFGen:
    """Register machine r[d] = r[a] op r[b] whose eight registers live in
    shared memory, this lane's K values of register r at
    base + r * RSTRIDE + q * 32 * CB (chunk q of CB bytes; the lanes of a warp
    side by side, so a warp's access to one chunk is conflict-free).  One
    dispatch per instruction, on (flags, function): index = flags * 4 +
    function, where the encoder's flags (second payload) are -- bits 0-1:
    where operand a is (0 the register file, 1 A, 2 B), bits 2-3: operand b
    likewise (at most one of the two held), bit 4: the result is overwritten before anything reads it from
    the file (and is not register 0 at the end) -- and the sentinel after the
    program has index 128 (DONE).  Two values stay in machine
    registers: A, the previous result, and B, which holds what the body's
    rules last loaded into it (operand a from the file is loaded into A, or
    into B when b is A; operand b from the file into B, or into A when a is
    B); the encoder tracks what each holds, so an operand found there is not
    loaded, and a dead result is not stored.  The kernel rewrites its staged
    copy of each instruction as (index, byte offsets of the destination,
    operand a and operand b in the warp's register file), so a body adds
    the lane's file address to offsets and the loop jumps on the index.  Few
    registers: the kernel's warps are bounded by shared memory alone.
    Operands: %0 bad (out, u32); %1 program address, %2 this lane's register
    file address (shared, u32)."""

    def __init__(self, K):
        assert K in (1, 2, 4, 8)
        self.K = K
        self.H = 1 if K == 1 else K // 2
        self.cb = min(16, 4 * K)           # bytes of one chunk
        self.nchunk = 4 * K // self.cb
        self.rstride = self.nchunk * 32 * self.cb
        self.b = Block()

    @property
    def ty(self):
        return "f32" if self.K == 1 else "b64"

    def load(self, dst, adr):
        b, K = self.b, self.K
        for q in range(self.nchunk):
            off = f"+{q * 32 * self.cb}" if q else ""
            if K == 1:
                b(f"ld.shared.f32 {dst[0]}, [{adr}{off}];")
            elif K == 2:
                b(f"ld.shared.b64 {dst[0]}, [{adr}{off}];")
            else:
                b(f"ld.shared.v2.b64 {{{dst[2 * q]}, {dst[2 * q + 1]}}}, [{adr}{off}];")

    def store(self, adr, src):
        b, K = self.b, self.K
        for q in range(self.nchunk):
            off = f"+{q * 32 * self.cb}" if q else ""
            if K == 1:
                b(f"st.shared.f32 [{adr}{off}], {src[0]};")
            elif K == 2:
                b(f"st.shared.b64 [{adr}{off}], {src[0]};")
            else:
                b(f"st.shared.v2.b64 [{adr}{off}], {{{src[2 * q]}, {src[2 * q + 1]}}};")

    def gen(self):
        K, H, b = self.K, self.H, self.b
        A = [f"rA{i}" for i in range(H)]
        B = [f"rB{i}" for i in range(H)]
        b("{")
        b(f".reg .{self.ty} rA<{H}>, rB<{H}>;")
        b(".reg .b32 code, pa, pb, pc, adr, base, aa, ab, ad;")
        for ln in pdiv_regs(K, H).split("\n"):
            b(ln)
        if K > 1:
            b("mov.b64 one2, 0x3F8000003F800000;")
            b("mov.b64 mone2, 0xBF800000BF800000;")
        # dispatch index = flags * 4 + function, flags = (source of a) |
        # (source of b) << 2 | dead << 4, a source 0 the file, 1 A, 2 B, at
        # most one of them held (the rest CBAD); the sentinel's flags are 32
        # (index 128, DONE)
        held = lambda sa, sb: sa == 3 or sb == 3 or (sa and sb)
        labels = []
        for idx in range(128):
            sa, sb = (idx >> 2) & 3, (idx >> 4) & 3
            labels.append("CBAD" if held(sa, sb) else f"OP{idx}")
        b("TBL: .branchtargets " + ", ".join(labels) + ", DONE;")
        b("mov.u32 adr, %1;")
        b("mov.u32 base, %2;")
        b("mov.u32 %0, 0;")
        zero = "0f00000000" if K == 1 else "0"
        for u in A + B:  # (defined before the first jump; the flags never read them unset)
            b(f"mov.{self.ty} {u}, {zero};")
        b("ld.shared.v4.u32 {code, pa, pb, pc}, [adr];")
        b("add.u32 adr, adr, 16;")
        b("LOOP:")
        b("brx.idx.uni code, TBL;")
        for idx in range(128):
            op, sa, sb, dead = idx & 3, (idx >> 2) & 3, (idx >> 4) & 3, (idx >> 6) & 1
            if held(sa, sb):
                continue
            b(f"OP{idx}:")
            # where each operand is: a loaded operand a goes to A (to B when b
            # is A), a loaded b to B (to A when a is B) -- the encoder's rules
            la = A if sa == 0 and sb != 1 else (B if sa == 0 else None)
            lb = B if sb == 0 and sa != 2 else (A if sb == 0 else None)
            xa = la if sa == 0 else (A if sa == 1 else B)
            xb = lb if sb == 0 else (A if sb == 1 else B)
            if sa == 0:
                b("add.u32 aa, pb, base;")
            if sb == 0:
                b("add.u32 ab, pc, base;")
            if not dead:
                b("add.u32 ad, pa, base;")
            if sb == 0:
                self.load(lb, "ab")
            if sa == 0:
                self.load(la, "aa")
            b("ld.shared.v4.u32 {code, pa, pb, pc}, [adr];")
            b("add.u32 adr, adr, 16;")
            if op == 3:  # the division blocks below, one per operand placement
                b(f"bra.uni DIV_{'A' if xa is A else 'B'}{'A' if xb is A else 'B'}{dead};")
            else:
                for i in range(H):
                    b(f"{F32[op] if K == 1 else F32X2[op]} {A[i]}, {xa[i]}, {xb[i]};")
                if not dead:
                    self.store("ad", A)
                b("bra.uni LOOP;")
        # A <- a / b (protected) with a, b in A or B (not both held, so
        # never the same register), then the store unless dead: shared blocks
        # instead of the division in each division body (their code in every
        # body cost the instruction cache)
        for na, xa in (("A", A), ("B", B)):
            for nb, xb in (("A", A), ("B", B)):
                if na == nb:
                    continue
                for dead in (0, 1):
                    tag = f"DIV_{na}{nb}{dead}"
                    b(f"{tag}:")
                    emit_pdiv(b, K, xa, xb, A, f"{tag}_")
                    if not dead:
                        self.store("ad", A)
                    b("bra.uni LOOP;")
                    emit_pdiv_slow(b, K, xa, xb, f"{tag}_")
        b("CBAD:")
        b("mov.u32 %0, 1;")
        b("DONE:")
        b("}")
        return b


# ---------------------------------------------------------------------------
# extended float S-form (the full function sets of Sec. 4.2)
# ---------------------------------------------------------------------------
SFX_BIN_BASE = len(SF_FORMS) * R * 4              # 384
XB_OPS = ["GT", "LT", "EQ", "AND", "OR"]
SFX_UN_BASE = SFX_BIN_BASE + 10 * R * len(XB_OPS)  # 784
UF_FORMS = ["X", "C", "S"]
SFX_IF_BASE = SFX_UN_BASE + len(UF_FORMS) * R * 4  # 880


def xif_descs():
    """IF operand descriptors (c, a, b), each 0 = input, 1 = constant,
    2 + j = stack level l + j, numbered as in csrc/isa.h."""
    out = []
    for t in range(125):
        d = (t // 25, (t // 5) % 5, t % 5)
        m = sum(1 for v in d if v >= 2)
        used, ok = set(), True
        for v in d:
            if v >= 2:
                if v - 2 >= m or (v - 2) in used:
                    ok = False
                used.add(v - 2)
        if ok:
            out.append(d)
    assert len(out) == 38
    return out


SFX_NCODES = SFX_IF_BASE + 38 * R                  # 1184
# extended RPN (csrc/isa.h)
RPX_BIN_BASE = len(RF_FORMS) * R * 4               # 128
RPX_UN_BASE = RPX_BIN_BASE + 2 * R * 5             # 208
RPX_IF_BASE = RPX_UN_BASE + R * 4                  # 240
RPX_NCODES = RPX_IF_BASE + 6 * R                   # 288
# IF permutation index -> levels (relative to l) of c, a, b
RPX_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
# exit status of the extended interpreter: 0 done, 1 bad code, else
# XEXIT + fn * 8 + level (apply unary function fn to t, store to level)
XEXIT = 16


class FloatGenX(FloatGen):
    """S-form interpreter over the full float function sets.  The stack
    registers, the unary-function operand t, the instruction address and the
    status are asm in/out operands, so the loop can leave the PTX block: a
    SIN, COS, EXP or LOG instruction copies its operand into t, records the
    function and the destination level in the status and exits; the caller
    applies CUDA's binary32 function to the K values and enters again, and the
    block first stores t into the level, then goes on with the next
    instruction.  Operands:
        %0 .. %{RH-1}       stack units (f32 for K = 1, b64 case pairs else)
        %{RH} .. %{RH+H-1}  t units
        %{RH+H}             shared address of the next instruction (u32)
        %{RH+H+1}           status: 0 on the first entry, as above on exit
        %{RH+H+2} ..        the K input values (f32, single input in
                            registers) or this lane's tile address (u32)"""

    def __init__(self, K, xmode):
        super().__init__(K, xmode)
        # division's slow path: decided once per warp (the basic
        # interpreters' folded form) except at K = 8 with the input in
        # registers, where the folded form costs spills and the per-lane
        # branch stays (measured: the KDDcup-shaped set at K = 2 +16%,
        # the sextic set at K = 8 -3% folded)
        self.fold_div = not (K == 8 and xmode == "reg")
        self.RH = R * self.H
        self.o_adr = self.RH + self.H
        self.o_st = self.RH + self.H + 1
        self.o_in = self.RH + self.H + 2

    def lev(self, l, i):
        return f"%{l * self.H + i}"

    def t(self):
        return [f"%{self.RH + i}" for i in range(self.H)]

    def setup_inputs(self):
        b, K = self.b, self.K
        if self.xmode == "reg":
            for i in range(self.H):
                if K == 1:
                    b(f"mov.f32 x0, %{self.o_in};")
                else:
                    b(f"mov.b64 x{i}, {{%{self.o_in + 2 * i}, %{self.o_in + 2 * i + 1}}};")
        else:
            b(f"mov.u32 xbase, %{self.o_in};")

    def elementwise(self, d, srcs, emit):
        """d[i] <- emit(elements of srcs[*][i]) one binary32 element at a time."""
        b = self.b
        if self.K == 1:
            for i in range(self.H):
                emit(d[i], [s_[i] for s_ in srcs])
            return
        for i in range(self.H):
            names = []
            for j, s_ in enumerate(srcs):
                b(f"mov.b64 {{e{2 * j}, e{2 * j + 1}}}, {s_[i]};")
                names.append((f"e{2 * j}", f"e{2 * j + 1}"))
            emit("e6", [n[0] for n in names])
            emit("e7", [n[1] for n in names])
            b(f"mov.b64 {d[i]}, {{e6, e7}};")

    def cmp_emit(self, op):
        b = self.b

        def emit(dst, ops):
            a, c = ops
            if op == "GT":
                b(f"setp.gt.f32 q, {a}, {c};")
            elif op == "LT":
                b(f"setp.lt.f32 q, {a}, {c};")
            elif op == "EQ":
                b(f"setp.eq.f32 q, {a}, {c};")
            elif op == "AND":   # NaN != 0 counts as true: unordered compare
                b(f"setp.neu.f32 q, {a}, 0f00000000;")
                b(f"setp.neu.and.f32 q, {c}, 0f00000000, q;")
            else:
                b(f"setp.neu.f32 q, {a}, 0f00000000;")
                b(f"setp.neu.or.f32 q, {c}, 0f00000000, q;")
            b(f"selp.f32 {dst}, 0f3F800000, 0f00000000, q;")
        return emit

    def if_emit(self):
        b = self.b

        def emit(dst, ops):
            c, a, e = ops
            b(f"setp.neu.f32 q, {c}, 0f00000000;")
            b(f"selp.f32 {dst}, {a}, {e}, q;")
        return emit

    def operand(self, kind, l, payload, xreg_units, creg):
        """Register units of an operand: 'X' input, 'C' constant, or a level."""
        if kind == "X":
            return self.load_x(xreg_units, payload)
        if kind == "C":
            return self.const(creg, payload)
        return [self.lev(kind, i) for i in range(self.H)]

    def sform_ext(self):
        K, H, b = self.K, self.H, self.b
        ty = self.ty
        b("{")
        b(f".reg .{ty} ta<{H}>, tb<{H}>, xA<{H}>, xB<{H}>, xC<{H}>, cA, cB, cC;")
        if self.xmode == "reg":
            b(f".reg .{ty} x<{H}>;")
        b(".reg .b32 code, pa, pb, pc, adr, dl, xa, xbase;")
        b(".reg .f32 e<8>;")
        b(".reg .pred p, q;")
        for ln in pdiv_regs(K, H).split("\n"):
            b(ln)
        if K > 1:
            b("mov.b64 one2, 0x3F8000003F800000;")
            b("mov.b64 mone2, 0xBF800000BF800000;")
        L = lambda l: [self.lev(l, i) for i in range(H)]
        ta = [f"ta{i}" for i in range(H)]
        tb = [f"tb{i}" for i in range(H)]
        xA = [f"xA{i}" for i in range(H)]
        xB = [f"xB{i}" for i in range(H)]
        xC = [f"xC{i}" for i in range(H)]
        T = self.t()
        table, bodies = {}, []
        # basic S-form codes (same numbers as the basic interpreter; the
        # divisions by a constant with its reciprocal take the general path)
        for f, name in enumerate(SF_FORMS):
            for l in range(R):
                for op in range(4):
                    if name in ("SS", "SSR") and l + 1 >= R:
                        continue
                    if name in ("MOVX", "MOVC") and (l != 0 or op != 0):
                        continue
                    if name in SF_RECIP and op != 3:
                        continue
                    code = sform_code(f, l, op)
                    table[code] = f"C{code}"
                    bodies.append((code, "basic", name, l, op))
        for f, name in enumerate(SF_FORMS[:10]):
            for l in range(R):
                for op in range(len(XB_OPS)):
                    if name in ("SS", "SSR") and l + 1 >= R:
                        continue
                    code = SFX_BIN_BASE + (f * R + l) * len(XB_OPS) + op
                    table[code] = f"C{code}"
                    bodies.append((code, "cmp", name, l, op))
        for uf, name in enumerate(UF_FORMS):
            for l in range(R):
                for fn in range(4):
                    code = SFX_UN_BASE + (uf * R + l) * 4 + fn
                    table[code] = f"C{code}"
                    bodies.append((code, "un", name, l, fn))
        for fi, d in enumerate(xif_descs()):
            m = sum(1 for v in d if v >= 2)
            for l in range(R):
                if l + max(m - 1, 0) >= R:
                    continue
                code = SFX_IF_BASE + fi * R + l
                table[code] = f"C{code}"
                bodies.append((code, "if", d, l, None))
        assert max(table) < SFX_NCODES
        self.table(SFX_NCODES, table, slow_levels=range(R) if self.fold_div else ())
        b("RSTBL: .branchtargets " + ", ".join(f"RS{l}" for l in range(R)) + ";")
        b(f"mov.u32 adr, %{self.o_adr};")
        self.setup_inputs()
        # resume: store t (the function's result) into its level
        b(f"setp.lt.u32 p, %{self.o_st}, {XEXIT};")
        b("@p bra.uni START;")
        b(f"and.b32 dl, %{self.o_st}, 7;")
        b("brx.idx.uni dl, RSTBL;")
        for l in range(R):
            b(f"RS{l}:")
            self.copy(L(l), T)
            b("bra.uni START;")
        b("START:")
        self.fetch()
        b("LOOP:")
        b("brx.idx.uni code, TBL;")
        for code, kind, name, l, op in bodies:
            b(f"C{code}:")
            if kind == "un":
                if name == "S":
                    self.copy(T, L(l))
                elif name == "X":
                    src = self.load_x(xA, "pa")
                    self.copy(T, src)
                else:
                    self.copy(T, self.const("cA", "pa"))
                b(f"mov.u32 %{self.o_st}, {XEXIT + op * 8 + l};")
                b("bra.uni EXIT;")
                continue
            if kind == "if":
                ops = []
                for dsc, pay, xr, cr in zip(name, ("pa", "pb", "pc"), (xA, xB, xC), ("cA", "cB", "cC")):
                    if dsc == 0:
                        ops.append(self.load_x(xr, pay))
                    elif dsc == 1:
                        ops.append(self.const(cr, pay))
                    else:
                        ops.append(L(l + dsc - 2))
                self.fetch()
                self.elementwise(L(l), ops, self.if_emit())
                self.jump()
                continue
            if name == "MOVX":
                src = self.load_x(xA, "pa")
                self.fetch()
                self.copy(L(0), src)
                self.jump()
                continue
            if name == "MOVC":
                src = self.const("cA", "pa")
                self.fetch()
                self.copy(L(0), src)
                self.jump()
                continue
            if name == "SS":
                a, c = L(l), L(l + 1)
            elif name == "SSR":
                a, c = L(l + 1), L(l)
            else:
                ka, kb = name[0], name[1]
                a = L(l) if ka == "S" else (self.load_x(xA, "pa") if ka == "X" else self.const("cA", "pa"))
                c = L(l) if kb == "S" else (self.load_x(xB, "pb") if kb == "X" else self.const("cB", "pb"))
            if kind == "cmp":
                self.fetch()
                self.elementwise(L(l), [a, c], self.cmp_emit(XB_OPS[op]))
                self.jump()
            elif op == 3:
                self.copy(ta, a)
                self.copy(tb, c)
                self.fetch()
                b(f"bra.uni DIV{l};")
            else:
                self.fetch()
                self.vop(op, L(l), a, c)
                self.jump()
        self.div_blocks_per_level(ta, tb, L)
        b("CBAD:")
        b(f"mov.u32 %{self.o_st}, 1;")
        b("bra.uni EXIT;")
        b("DONE:")
        b(f"mov.u32 %{self.o_st}, 0;")
        b("EXIT:")
        b(f"mov.u32 %{self.o_adr}, adr;")
        b("}")
        return b

    def rpn_ext(self):
        """Extended RPN interpreter: the basic RPN bodies (pushes, +, -, *, /
        on levels l and l+1), comparisons and logic, the unary functions on
        level l (leaving the block as in sform_ext), IF on levels l .. l+2 in
        the order its permutation index gives.  Same operands as sform_ext."""
        K, H, b = self.K, self.H, self.b
        b("{")
        b(f".reg .{self.ty} ta<{H}>, tb<{H}>, cA;")
        if self.xmode == "reg":
            b(f".reg .{self.ty} x<{H}>;")
        b(".reg .b32 code, pa, pb, pc, adr, dl, xa, xbase;")
        b(".reg .f32 e<8>;")
        b(".reg .pred p, q;")
        for ln in pdiv_regs(K, H).split("\n"):
            b(ln)
        if K > 1:
            b("mov.b64 one2, 0x3F8000003F800000;")
            b("mov.b64 mone2, 0xBF800000BF800000;")
        L = lambda l: [self.lev(l, i) for i in range(H)]
        ta = [f"ta{i}" for i in range(H)]
        tb = [f"tb{i}" for i in range(H)]
        T = self.t()
        table, bodies = {}, []
        for f, name in enumerate(RF_FORMS):
            for l in range(R):
                for op in range(4):
                    if name in ("PUSHX", "PUSHC") and op != 0:
                        continue
                    if name in ("OP", "OPR") and l + 1 >= R:
                        continue
                    code = rpn_code(f, l, op)
                    table[code] = f"C{code}"
                    bodies.append((code, "basic", name, l, op))
        for opr in range(2):
            for l in range(R - 1):
                for op in range(len(XB_OPS)):
                    code = RPX_BIN_BASE + (opr * R + l) * len(XB_OPS) + op
                    table[code] = f"C{code}"
                    bodies.append((code, "cmp", opr, l, op))
        for l in range(R):
            for fn in range(4):
                code = RPX_UN_BASE + l * 4 + fn
                table[code] = f"C{code}"
                bodies.append((code, "un", None, l, fn))
        for perm in range(6):
            for l in range(R - 2):
                code = RPX_IF_BASE + perm * R + l
                table[code] = f"C{code}"
                bodies.append((code, "if", perm, l, None))
        self.table(RPX_NCODES, table, slow_levels=range(R) if self.fold_div else ())
        b("RSTBL: .branchtargets " + ", ".join(f"RS{l}" for l in range(R)) + ";")
        b(f"mov.u32 adr, %{self.o_adr};")
        self.setup_inputs()
        b(f"setp.lt.u32 p, %{self.o_st}, {XEXIT};")
        b("@p bra.uni START;")
        b(f"and.b32 dl, %{self.o_st}, 7;")
        b("brx.idx.uni dl, RSTBL;")
        for l in range(R):
            b(f"RS{l}:")
            self.copy(L(l), T)
            b("bra.uni START;")
        b("START:")
        self.fetch()
        b("LOOP:")
        b("brx.idx.uni code, TBL;")
        for code, kind, name, l, op in bodies:
            b(f"C{code}:")
            if kind == "un":
                self.copy(T, L(l))
                b(f"mov.u32 %{self.o_st}, {XEXIT + op * 8 + l};")
                b("bra.uni EXIT;")
                continue
            if kind == "if":
                lc, la, lb = RPX_PERMS[name]
                self.fetch()
                self.elementwise(L(l), [L(l + lc), L(l + la), L(l + lb)], self.if_emit())
                self.jump()
                continue
            if kind == "cmp":
                a, c = (L(l), L(l + 1)) if name == 0 else (L(l + 1), L(l))
                self.fetch()
                self.elementwise(L(l), [a, c], self.cmp_emit(XB_OPS[op]))
                self.jump()
                continue
            if name == "PUSHX":
                if self.xmode == "reg":
                    self.fetch()
                    self.copy(L(l), [self.xreg(i) for i in range(H)])
                else:
                    self.load_x(L(l), "pa")
                    self.fetch()
                self.jump()
                continue
            if name == "PUSHC":
                src = self.const("cA", "pa")
                self.fetch()
                self.copy(L(l), src)
                self.jump()
                continue
            a, c = (L(l), L(l + 1)) if name == "OP" else (L(l + 1), L(l))
            self.fetch()
            if op == 3:
                self.copy(ta, a)
                self.copy(tb, c)
                b(f"bra.uni DIV{l};")
            else:
                self.vop(op, L(l), a, c)
                self.jump()
        self.div_blocks_per_level(ta, tb, L)
        b("CBAD:")
        b(f"mov.u32 %{self.o_st}, 1;")
        b("bra.uni EXIT;")
        b("DONE:")
        b(f"mov.u32 %{self.o_st}, 0;")
        b("EXIT:")
        b(f"mov.u32 %{self.o_adr}, adr;")
        b("}")
        return b

    def operand_macros(self):
        """C++ operand lists of the asm statement (outputs and inputs)."""
        K, H = self.K, self.H
        c = "f" if K == 1 else "l"
        outs = [f'"+{c}"(s[{i}])' for i in range(self.RH)] + [f'"+{c}"(t[{i}])' for i in range(H)]
        outs += ['"+r"(adr)', '"+r"(st)']
        if self.xmode == "reg":
            ins = [f'"f"(x[{j}])' for j in range(K)]
        else:
            ins = ['"r"(tile)']
        return ", ".join(outs), ", ".join(ins)


# ---------------------------------------------------------------------------
# Boolean interpreter (K words per thread, 32 cases per word)
# ---------------------------------------------------------------------------
class BoolGen:
    """Same dispatch as FloatGen, over K-word registers."""

    def __init__(self, K):
        self.K = K
        self.b = Block()
        self.stride = 128 * K

    def lev(self, l):
        return [f"s{l * self.K + j}" for j in range(self.K)]

    def load_x(self, dst, payload):
        K, b = self.K, self.b
        b(f"mad.lo.u32 xa, {payload}, {self.stride}, xbase;")
        if K == 1:
            b(f"ld.shared.b32 {dst[0]}, [xa];")
        elif K == 2:
            b(f"ld.shared.v2.b32 {{{dst[0]}, {dst[1]}}}, [xa];")
        else:
            for q in range(K // 4):
                d = dst[4 * q: 4 * q + 4]
                off = f"+{16 * q}" if q else ""
                b(f"ld.shared.v4.b32 {{{', '.join(d)}}}, [xa{off}];")
        return dst

    def fetch(self):
        self.b("ld.shared.v4.u32 {code, pa, pb, pc}, [adr];")
        self.b("add.u32 adr, adr, 16;")

    def jump(self):
        self.b("bra.uni LOOP;")

    def gen(self):
        K, b = self.K, self.b
        xA = [f"xA{j}" for j in range(K)]
        xB = [f"xB{j}" for j in range(K)]
        xC = [f"xC{j}" for j in range(K)]
        b("{")
        b(f".reg .b32 s<{R * K}>, xA<{K}>, xB<{K}>, xC<{K}>;")
        b(".reg .b32 code, pa, pb, pc, adr, xa, xbase;")
        for r in range(R * K):  # defined before the first jump (see FloatGen.header)
            b(f"mov.b32 s{r}, 0;")
        n_codes = BOOL_MOVX + 1
        table, bodies = {}, []
        for f, name in enumerate(BF_FORMS):
            for l in range(R):
                for op in range(4):
                    if name in ("SS", "SSR") and l + 1 >= R:
                        continue
                    code = (f * R + l) * 4 + op
                    table[code] = f"C{code}"
                    bodies.append((code, "bin", name, l, op))
        for fi, d in enumerate(if_descs()):
            m = sum(1 for v in d if v > 0)
            for l in range(R):
                if l + max(m - 1, 0) >= R:
                    continue
                code = BOOL_IF_BASE + fi * R + l
                table[code] = f"C{code}"
                bodies.append((code, "if", d, l, None))
        table[BOOL_MOVX] = "CMOV"
        labels = [table.get(c, "CBAD") for c in range(n_codes)] + ["DONE"]
        b("TBL: .branchtargets " + ", ".join(labels) + ";")
        b(f"mov.u32 adr, %{K + 1};")
        b(f"mov.u32 %{K}, 0;")
        b(f"mov.u32 xbase, %{K + 3};")
        self.fetch()
        b("LOOP:")
        b("brx.idx.uni code, TBL;")
        for code, kind, name, l, op in bodies:
            b(f"C{code}:")
            S = self.lev(l)
            if kind == "bin":
                if name == "SS":
                    a, c = S, self.lev(l + 1)
                elif name == "SSR":
                    a, c = self.lev(l + 1), S
                else:
                    a = S if name[0] == "S" else self.load_x(xA, "pa")
                    c = S if name[1] == "S" else self.load_x(xB, "pb")
                self.fetch()
                for j in range(K):
                    b(f"lop3.b32 {S[j]}, {a[j]}, {c[j]}, {c[j]}, 0x{LUT[op]:02X};")
            else:
                dc, da, db = name
                ops = []
                for dsc, pay, tmp in ((dc, "pa", xA), (da, "pb", xB), (db, "pc", xC)):
                    ops.append(self.load_x(tmp, pay) if dsc == 0 else self.lev(l + dsc - 1))
                self.fetch()
                cc, aa, bb = ops
                for j in range(K):
                    b(f"lop3.b32 {S[j]}, {cc[j]}, {aa[j]}, {bb[j]}, 0x{LUT_IF:02X};")
            self.jump()
        b("CMOV:")
        src = self.load_x(xA, "pa")
        self.fetch()
        S0 = self.lev(0)
        for j in range(K):
            b(f"mov.b32 {S0[j]}, {src[j]};")
        self.jump()
        b("CBAD:")
        b(f"mov.u32 %{K}, 1;")
        b("DONE:")
        for j in range(K):
            b(f"mov.b32 %{j}, s{j};")
        b("}")
        return b


def pdiv_macro(K, fold=True):
    """Standalone protected division of K values (exactly the interpreters'
    sequence), for the division checker: K == 1 operands %0 = q, %1 = a,
    %2 = b (f32); K == 4 operands %0, %1 = q pairs, %2, %3 = a pairs,
    %4, %5 = b pairs (b64).  fold: the slow path decided once per warp (the
    basic interpreters), else by a per-lane branch (the extended ones)."""
    b = Block()
    H = 1 if K == 1 else K // 2
    b("{")
    for ln in pdiv_regs(K, H).split("\n"):
        b(ln)
    ty = "f32" if K == 1 else "b64"
    b(f".reg .{ty} qa<{H}>, qb<{H}>, qq<{H}>;")
    if K > 1:
        b("mov.b64 one2, 0x3F8000003F800000;")
        b("mov.b64 mone2, 0xBF800000BF800000;")
    for i in range(H):
        b(f"mov.{ty} qa{i}, %{H + i};")
        b(f"mov.{ty} qb{i}, %{2 * H + i};")
    qa = [f"qa{i}" for i in range(H)]
    qb = [f"qb{i}" for i in range(H)]
    qq = [f"qq{i}" for i in range(H)]
    if fold:
        # one decision per warp, the slow body recomputing every element
        emit_pdiv(b, K, qa, qb, qq, "P", fold=lambda: b("@!dall bra.uni PSLOW;"))
        b("PRET:")
        for i in range(H):
            b(f"mov.{ty} %{i}, qq{i};")
        b("bra.uni PEND;")
        emit_pdiv_slow_body(b, K, qa, qb, qq, "P")
        b("bra.uni PRET;")
    else:
        # the quotient overwrites the numerator registers, as in the interpreters
        emit_pdiv(b, K, qa, qb, qa, "P")
        for i in range(H):
            b(f"mov.{ty} %{i}, qa{i};")
        b("bra.uni PEND;")
        emit_pdiv_slow(b, K, qa, qb, "P")
    b("PEND:")
    b("}")
    return b


def pdivi_macro(K, test=True):
    """Standalone division by a constant with its reciprocal (exactly the
    interpreters' SF_XI / SF_SI sequence, or with test=False the SF_CI one),
    for the division checker: K == 1 operands %0 = q, %1 = a, %2 = b,
    %3 = RN(1/b) (f32); K == 4 operands %0, %1 = q pairs, %2, %3 = a pairs
    (b64), %4 = b, %5 = RN(1/b) (f32).  With the test the slow path is
    decided once per warp, as in the interpreters."""
    b = Block()
    H = 1 if K == 1 else K // 2
    b("{")
    for ln in pdiv_regs(K, H).split("\n"):
        b(ln)
    ty = "f32" if K == 1 else "b64"
    b(f".reg .{ty} qa<{H}>, qq<{H}>;")
    if K > 1:
        b("mov.b64 one2, 0x3F8000003F800000;")
        b("mov.b64 mone2, 0xBF800000BF800000;")
    for i in range(H):
        b(f"mov.{ty} qa{i}, %{H + i};")
    if K == 1:
        b("mov.f32 cN, %2;")
        b("mov.f32 cY, %3;")
    else:
        b(f"mov.b64 cN, {{%{2 * H}, %{2 * H}}};")
        b(f"mov.b64 cY, {{%{2 * H + 1}, %{2 * H + 1}}};")
    qa = [f"qa{i}" for i in range(H)]
    qq = [f"qq{i}" for i in range(H)]
    if test:
        emit_pdivi(b, K, qa, "cN", "cY", qq, fold=lambda: b("@!dall bra.uni PSLOW;"))
    else:
        emit_pdivi(b, K, qa, "cN", "cY", qq)
    b("PRET:")
    for i in range(H):
        b(f"mov.{ty} %{i}, qq{i};")
    b("bra.uni PEND;")
    emit_pdivi_slow_body(b, K, qa, "cN", qq, "P")
    b("bra.uni PRET;")
    b("PEND:")
    b("}")
    return b


def generate() -> str:
    parts = ["// gen_interp.h -- generated by paper_1601_00221_gb300/gen_interp.py; do not edit.\n",
             "#pragma once\n"]
    parts.append(pdiv_macro(1).macro("GP_PTX_PDIV_K1", "protected division, one value, warp decision"))
    parts.append(pdiv_macro(4).macro("GP_PTX_PDIV_K4", "protected division, two packed pairs, warp decision"))
    parts.append(pdiv_macro(1, False).macro("GP_PTX_PDIV_LANE_K1", "protected division, one value, lane branch"))
    parts.append(pdiv_macro(4, False).macro("GP_PTX_PDIV_LANE_K4",
                                            "protected division, two packed pairs, lane branch"))
    parts.append(pdivi_macro(1).macro("GP_PTX_PDIVI_K1", "division by a constant with its reciprocal, one value"))
    parts.append(pdivi_macro(4).macro("GP_PTX_PDIVI_K4",
                                      "division by a constant with its reciprocal, two packed pairs"))
    parts.append(pdivi_macro(1, False).macro("GP_PTX_PDIVI_NT_K1",
                                             "division of a constant by a constant with its reciprocal, one value"))
    parts.append(pdivi_macro(4, False).macro("GP_PTX_PDIVI_NT_K4",
                                             "division of a constant by a constant with its reciprocal, two pairs"))
    for K in (1, 2, 4, 8):
        for xm in ("reg", "smem"):
            X = xm.upper()
            parts.append(FloatGen(K, xm).sform().macro(
                f"GP_PTX_SFORM_K{K}_{X}", f"S-form interpreter, K={K}, inputs in {xm}"))
            parts.append(FloatGen(K, xm).rpn().macro(
                f"GP_PTX_RPN_K{K}_{X}", f"RPN interpreter, K={K}, inputs in {xm}"))
        parts.append(FloatGen(K, "smem").linear().macro(
            f"GP_PTX_LINEAR_K{K}", f"register linear-GP interpreter, K={K}"))
        if K >= 2:
            parts.append(f"// the stack operands of the interpreters above (the caller's array s)\n"
                         f"#define GP_STACK_K{K} " + ", ".join(f'"+l"(s[{i}])' for i in range(R * K // 2)) + "\n")
        if K == 8:  # the pass loop inside the interpreter (sum of absolute errors)
            parts.append(FloatGenLoop().sform().macro(
                "GP_PTX_SFORM_K8_REG_PASSES",
                "S-form interpreter, K=8, input in registers, the passes and their error sums inside"))
        if K == 8:  # levels 4..7 in shared memory (the stack-register study)
            for xm in ("reg", "smem"):
                X = xm.upper()
                parts.append(FloatGen(K, xm, rl=4).sform().macro(
                    f"GP_PTX_SFORM_K{K}_{X}_RL4",
                    f"S-form interpreter, K={K}, inputs in {xm}, levels 4..7 in shared memory"))
        for xm in ("reg", "smem"):
            X = xm.upper()
            g = FloatGenX(K, xm)
            parts.append(g.sform_ext().macro(
                f"GP_PTX_SFORMX_K{K}_{X}", f"extended S-form interpreter, K={K}, inputs in {xm}"))
            parts.append(FloatGenX(K, xm).rpn_ext().macro(
                f"GP_PTX_RPNX_K{K}_{X}", f"extended RPN interpreter, K={K}, inputs in {xm}"))
            outs, ins = g.operand_macros()
            parts.append(f"#define GP_SFX_OUT_K{K}_{X} {outs}\n#define GP_SFX_IN_K{K}_{X} {ins}\n")
        parts.append(LinearRFGen(K).gen().macro(
            f"GP_PTX_LINEAR_RF_K{K}", f"register linear-GP interpreter, registers in shared memory, K={K}"))
        parts.append(BoolGen(K).gen().macro(f"GP_PTX_BOOL_K{K}", f"Boolean interpreter, K={K} words"))
    return "".join(parts)


def write(path: str) -> str:
    text = generate()
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            fh.write(text)
    return path


if __name__ == "__main__":
    import sys
    print(write(sys.argv[1] if len(sys.argv) > 1 else "gen_interp.h"))
