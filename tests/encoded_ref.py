"""Test-side reader of the encoded instruction streams (host, numpy binary32).

It restates the documented layout of the encoded programs (header of four
words, then four words per instruction: code, payloads) and runs them case by
case with numpy float32 arithmetic, so that the host encoder can be checked
against the CPU oracle without a GPU.  It is test code only.
"""
import numpy as np

R = 8
F_NAMES = "+-*/"
SF_FORMS = ["XX", "XC", "CX", "CC", "SX", "XS", "SC", "CS", "SS", "SSR", "MOVX", "MOVC", "XI", "SI", "CI"]
# division by a constant b (payload b) with RN(1/b) in payload c; numerator X, S or C
SF_RECIP = ("XI", "SI", "CI")
DIV_LO, DIV_HI = 0x26800000, 0x58800000  # 2^-50, 2^50 as binary32 bit patterns
RF_FORMS = ["PUSHX", "PUSHC", "OP", "OPR"]
BF_FORMS = ["XX", "XS", "SX", "SS", "SSR"]
BOOL_IF_BASE = 5 * R * 4
BOOL_MOVX = BOOL_IF_BASE + 16 * R


def if_descs():
    out = []
    for t in range(64):
        dc, da, db = t // 16, (t // 4) % 4, t % 4
        m = (dc > 0) + (da > 0) + (db > 0)
        used = []
        ok = True
        for d in (dc, da, db):
            if d > 0:
                if d - 1 >= m or (d - 1) in used:
                    ok = False
                used.append(d - 1)
        if ok:
            out.append((dc, da, db))
    assert len(out) == 16
    return out


IF_DESCS = if_descs()

# extended S-form codes (kind 5): comparisons/logic, unary functions, IF
SFX_BIN_BASE = len(SF_FORMS) * R * 4
XB_NAMES = ["GT", "LT", "EQ", "AND", "OR"]
SFX_UN_BASE = SFX_BIN_BASE + 10 * R * 5
UF_FORMS = ["X", "C", "S"]
SFX_IF_BASE = SFX_UN_BASE + 3 * R * 4


def xif_descs():
    out = []
    for t in range(125):
        d = (t // 25, (t // 5) % 5, t % 5)
        m = sum(1 for v in d if v >= 2)
        js = [v - 2 for v in d if v >= 2]
        if sorted(js) == list(range(m)):
            out.append(d)
    assert len(out) == 38
    return out


XIF_DESCS = xif_descs()

# extended RPN codes (kind 6)
RPX_BIN_BASE = len(RF_FORMS) * R * 4
RPX_UN_BASE = RPX_BIN_BASE + 2 * R * 5
RPX_IF_BASE = RPX_UN_BASE + R * 4
RPX_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _unary_ref(fn, a):
    """A valid binary32 implementation: the value nearest the binary64 result."""
    a64 = a.astype(np.float64)
    with np.errstate(all="ignore"):
        if fn == 3:
            return np.where(a == 0, np.float32(0), np.log(np.abs(a64)).astype(np.float32))
        return [np.sin, np.cos, np.exp][fn](a64).astype(np.float32)


def _xbin(op, a, b):
    with np.errstate(all="ignore"):
        v = [a > b, a < b, a == b, (a != 0) & (b != 0), (a != 0) | (b != 0)][op]
    return v.astype(np.float32)


def header(words):
    w = np.asarray(words, np.uint32)
    return {"kind": int(w[0]) & 0xFF, "order": (int(w[0]) >> 8) & 0xFF, "version": int(w[0]) >> 16,
            "n_instr": int(w[1]), "n_nodes": int(w[2]), "max_depth": int(w[3]) & 0xFFFF,
            "n_inputs_used": int(w[3]) >> 16}


def instrs(words):
    w = np.asarray(words, np.uint32)
    n = int(w[1])
    return [tuple(int(v) for v in w[4 + 4 * i: 8 + 4 * i]) for i in range(n)]


def _f(bits):
    return np.uint32(bits).view(np.float32)


def _apply(op, a, b):
    with np.errstate(all="ignore"):
        if op == 0:
            return (a + b).astype(np.float32)
        if op == 1:
            return (a - b).astype(np.float32)
        if op == 2:
            return (a * b).astype(np.float32)
        safe = np.where(b == 0, np.float32(1), b)
        return np.where(b == 0, np.float32(1), a / safe).astype(np.float32)


def run_float(words, x, register_file=False):
    """Per-case outputs of an encoded float program (S-form, extended S-form,
    RPN or register).  register_file: run a register program the way the
    shared-memory register-file interpreter does -- two values held beside
    the register file, A (the previous result) and B (what the load rules
    last put there); payload b says where each operand is (bits 0-1 for a,
    2-3 for b: 0 the file, 1 A, 2 B), an operand from the file is loaded into
    A or B by the rules (a into A, or into B when b is A; b into B, or into A
    when a is B), and a result flagged dead (bit 4) is not written to the
    register file -- so that wrong flags show as wrong outputs."""
    x = np.asarray(x, np.float32)
    n_cases = x.shape[1]
    h = header(words)
    full = lambda v: np.full(n_cases, v, np.float32)
    if h["kind"] == 3:
        r = [x[i].copy() if i < x.shape[0] else full(0.0) for i in range(8)]
        A, B = full(np.nan), full(np.nan)
        for code, d, flags, _ in instrs(words):
            op, a, b = code // 64, (code // 8) % 8, code % 8
            if not register_file:
                r[d] = _apply(op, r[a], r[b])
                continue
            assert flags < 32
            sa, sb = flags & 3, (flags >> 2) & 3
            assert sa < 3 and sb < 3
            va = r[a] if sa == 0 else (A if sa == 1 else B)
            vb = r[b] if sb == 0 else (A if sb == 1 else B)
            if sa == 0 and sb == 0:
                B = vb
            elif sa == 0 and sb == 1:
                B = va
            elif sa == 1 and sb == 0:
                B = vb
            A = _apply(op, va, vb)
            if not flags & 16:
                r[d] = A
        return r[0]
    S = [None] * R
    for code, pa, pb, pc in instrs(words):
        op, lvl, form = code & 3, (code >> 2) % R, (code >> 2) // R
        if h["kind"] == 5 and code >= SFX_BIN_BASE:
            X = lambda v: x[v]
            C = lambda bits: full(_f(bits))
            if code >= SFX_IF_BASE:
                f, lvl = (code - SFX_IF_BASE) // R, (code - SFX_IF_BASE) % R
                vals = [x[p_] if d == 0 else C(p_) if d == 1 else S[lvl + d - 2]
                        for d, p_ in zip(XIF_DESCS[f], (pa, pb, pc))]
                c, a, b = vals
                S[lvl] = np.where(c != 0, a, b).astype(np.float32)
            elif code >= SFX_UN_BASE:
                c = code - SFX_UN_BASE
                fn, lvl, uf = c % 4, (c // 4) % R, (c // 4) // R
                a = {"X": lambda: X(pa), "C": lambda: C(pa), "S": lambda: S[lvl]}[UF_FORMS[uf]]()
                S[lvl] = _unary_ref(fn, a)
            else:
                c = code - SFX_BIN_BASE
                xop, lvl, form = c % 5, (c // 5) % R, (c // 5) // R
                name = SF_FORMS[form]
                if name in ("SS", "SSR"):
                    a, b = (S[lvl], S[lvl + 1]) if name == "SS" else (S[lvl + 1], S[lvl])
                else:
                    a = S[lvl] if name[0] == "S" else (X(pa) if name[0] == "X" else C(pa))
                    b = S[lvl] if name[1] == "S" else (X(pb) if name[1] == "X" else C(pb))
                S[lvl] = _xbin(xop, a, b)
            continue
        if h["kind"] == 6 and code >= RPX_BIN_BASE:
            if code >= RPX_IF_BASE:
                perm, lvl = (code - RPX_IF_BASE) // R, (code - RPX_IF_BASE) % R
                lc, la, lb = RPX_PERMS[perm]
                S[lvl] = np.where(S[lvl + lc] != 0, S[lvl + la], S[lvl + lb]).astype(np.float32)
            elif code >= RPX_UN_BASE:
                lvl, fn = (code - RPX_UN_BASE) // 4, (code - RPX_UN_BASE) % 4
                S[lvl] = _unary_ref(fn, S[lvl])
            else:
                c = code - RPX_BIN_BASE
                xop, lvl, opr = c % 5, (c // 5) % R, (c // 5) // R
                a, b = (S[lvl], S[lvl + 1]) if opr == 0 else (S[lvl + 1], S[lvl])
                S[lvl] = _xbin(xop, a, b)
            continue
        if h["kind"] in (1, 5):
            name = SF_FORMS[form]
            X = lambda v: x[v]
            C = lambda bits: full(_f(bits))
            if name == "MOVX":
                S[0] = x[pa].copy(); continue
            if name == "MOVC":
                S[0] = C(pa); continue
            if name in SF_RECIP:
                # the layout's promise: a divisor in [2^-50, 2^50] and its
                # reciprocal rounded to nearest (numpy's IEEE binary32 division)
                assert op == 3 and DIV_LO <= (pb & 0x7FFFFFFF) <= DIV_HI, (code, pb)
                assert pc == int(np.array(np.float32(1) / _f(pb), np.float32).view(np.uint32)), (pb, pc)
                a = S[lvl] if name[0] == "S" else (X(pa) if name[0] == "X" else C(pa))
                S[lvl] = _apply(3, a, C(pb))
                continue
            if name in ("SS", "SSR"):
                a, b = (S[lvl], S[lvl + 1]) if name == "SS" else (S[lvl + 1], S[lvl])
            else:
                ka, kb = name[0], name[1]
                a = S[lvl] if ka == "S" else (X(pa) if ka == "X" else C(pa))
                b = S[lvl] if kb == "S" else (X(pb) if kb == "X" else C(pb))
            S[lvl] = _apply(op, a, b)
        else:
            name = RF_FORMS[form]
            if name == "PUSHX":
                S[lvl] = x[pa].copy()
            elif name == "PUSHC":
                S[lvl] = full(_f(pa))
            elif name == "OP":
                S[lvl] = _apply(op, S[lvl], S[lvl + 1])
            else:
                S[lvl] = _apply(op, S[lvl + 1], S[lvl])
    return S[0]


def run_bool(words, bits):
    bits = np.asarray(bits, np.uint32)
    S = [None] * R
    for code, pa, pb, pc in instrs(words):
        if code == BOOL_MOVX:
            S[0] = bits[pa].copy(); continue
        if code >= BOOL_IF_BASE:
            f, lvl = (code - BOOL_IF_BASE) // R, (code - BOOL_IF_BASE) % R
            ds = IF_DESCS[f]
            vals = [bits[p] if d == 0 else S[lvl + d - 1] for d, p in zip(ds, (pa, pb, pc))]
            c, a, b = vals
            S[lvl] = ((c & a) | (~c & b)).astype(np.uint32)
            continue
        op, lvl, form = code & 3, (code >> 2) % R, (code >> 2) // R
        name = BF_FORMS[form]
        if name == "SS":
            a, b = S[lvl], S[lvl + 1]
        elif name == "SSR":
            a, b = S[lvl + 1], S[lvl]
        else:
            a = S[lvl] if name[0] == "S" else bits[pa]
            b = S[lvl] if name[1] == "S" else bits[pb]
        v = [a & b, a | b, ~(a & b), ~(a | b)][op]
        S[lvl] = np.asarray(v, np.uint32)
    return S[0]


def render_sform(words):
    """Text of an encoded S-form program in the paper's notation, e.g. '+(XX) *(XS)'."""
    out = []
    for code, _, _, _ in instrs(words):
        op, form = code & 3, (code >> 2) // R
        name = SF_FORMS[form]
        ops = {"SSR": "SS", "XI": "XC", "SI": "SC", "CI": "CC"}.get(name, name)
        out.append(f"{F_NAMES[op]}({ops})")
    return " ".join(out)
