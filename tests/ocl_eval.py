"""Parser and evaluator for the OpenCL C subset the decompiler emits.

Test infrastructure.  It runs decompiled kernels work-item by work-item on the
same buffers as ``gcn_interp`` so the two results can be compared bit for bit.
It is also the structural well-formedness check: a text that does not parse,
uses an undeclared variable, or mixes operand types without an explicit cast
is rejected.  Semantics are C's with the following readings: integers wrap
(two's complement), >> of a signed value is arithmetic, the work-item
functions return uint (the decompiler treats them as 32-bit values), mad24 and
mul24 use the low 24 bits of their operands, mul_hi is the high half of the
full product, fma rounds once.
"""
from __future__ import annotations

import re

import numpy as np

from fp_exact import fma32, fma64

T = {"int": np.int32, "uint": np.uint32, "float": np.float32, "long": np.int64, "ulong": np.uint64,
     "double": np.float64}
INTS = ("int", "uint", "long", "ulong")
WIDTH = {"int": 32, "uint": 32, "float": 32, "long": 64, "ulong": 64, "double": 64}
UINT_OF = {32: np.uint32, 64: np.uint64}

_tok = re.compile(r"""
    (?P<ws>\s+)|
    (?P<num>(?:0x[0-9a-fA-F]+|\d+\.\d+(?:[eE][-+]?\d+)?f?|\d+)(?:UL|L|u)?)|
    (?P<id>[A-Za-z_][A-Za-z_0-9]*)|
    (?P<str>"(?:[^"\\]|\\.)*")|
    (?P<op><<|>>|<=|>=|==|!=|&&|\|\||[-+*/%&|^!<>=(){}\[\];,?:])
""", re.X)


class ParseError(Exception):
    pass


def lex(src: str):
    out, i = [], 0
    while i < len(src):
        m = _tok.match(src, i)
        if not m:
            raise ParseError(f"bad character at {i}: {src[i:i+20]!r}")
        i = m.end()
        if m.lastgroup == "ws":
            continue
        out.append((m.lastgroup, m.group()))
    return out


class Kernel:
    def __init__(self, name, params, decls, body):
        self.name = name
        self.params = params      # list of (kind 'ptr'/'val', type, name)
        self.decls = decls        # var name -> type
        self.body = body          # statements


class Parser:
    def __init__(self, toks):
        self.t = toks
        self.i = 0
        self.loops = 0  # do-while bodies being parsed (a break needs one)

    def peek(self, k=0):
        return self.t[self.i + k][1] if self.i + k < len(self.t) else None

    def eat(self, want=None):
        if self.i >= len(self.t):
            raise ParseError("unexpected end")
        v = self.t[self.i][1]
        if want is not None and v != want:
            raise ParseError(f"expected {want!r}, got {v!r} at token {self.i}")
        self.i += 1
        return v

    def kernels(self):
        ks = []
        while self.i < len(self.t):
            ks.append(self.kernel())
        return ks

    def kernel(self):
        self.eat("__kernel")
        self.eat("void")
        name = self.eat()
        self.eat("(")
        params = []
        if self.peek() == "void":
            self.eat()
        else:
            while True:
                if self.peek() in ("__global", "__constant", "__local"):
                    space = self.eat()
                    if self.peek() == "const":
                        self.eat()
                    ty = self.eat()
                    self.eat("*")
                    params.append(("ptr", ty, self.eat(), space))
                else:
                    ty = self.eat()
                    params.append(("val", ty, self.eat()))
                if self.peek() == ",":
                    self.eat()
                    continue
                break
        self.eat(")")
        self.eat("{")
        decls = {}
        while self.peek() in T and self.peek(2) == ";":
            ty = self.eat()
            nm = self.eat()
            self.eat(";")
            if nm in decls:
                raise ParseError(f"{nm} declared twice")
            decls[nm] = ty
        self.scope = {p[2]: p for p in params}
        self.decls = decls
        body = self.block_items()
        self.eat("}")
        return Kernel(name, params, decls, body)

    def block_items(self):
        items = []
        while self.peek() not in ("}", None):
            items.append(self.stmt())
        return items

    def stmt(self):
        p = self.peek()
        if p == "if":
            self.eat()
            self.eat("(")
            c = self.expr()
            self.eat(")")
            self.eat("{")
            th = self.block_items()
            self.eat("}")
            el = []
            if self.peek() == "else":
                self.eat()
                self.eat("{")
                el = self.block_items()
                self.eat("}")
            return ("if", c, th, el)
        if p == "do":
            self.eat()
            self.eat("{")
            self.loops += 1
            b = self.block_items()
            self.loops -= 1
            self.eat("}")
            self.eat("while")
            self.eat("(")
            c = self.expr()
            self.eat(")")
            self.eat(";")
            return ("do", b, c)
        if p == "barrier":  # barrier(CLK_LOCAL_MEM_FENCE);
            self.eat()
            self.eat("(")
            if self.eat() != "CLK_LOCAL_MEM_FENCE":
                raise ParseError("barrier flags")
            self.eat(")")
            self.eat(";")
            return ("barrier",)
        if p == "break":
            if not self.loops:
                raise ParseError("break outside a loop")
            self.eat()
            self.eat(";")
            return ("break",)
        if p == "__asm__":
            raise ParseError("inline asm")
        lhs = self.unary()
        self.eat("=")
        rhs = self.expr()
        self.eat(";")
        if lhs[0] not in ("var", "index", "deref"):
            raise ParseError("bad assignment target")
        return ("assign", lhs, rhs)

    # expression grammar with C precedence
    PREC = [("|",), ("^",), ("&",), ("==", "!="), ("<", ">", "<=", ">="), ("<<", ">>"), ("+", "-"), ("*",)]

    def expr(self, level=0):
        if level == 0:  # conditional: c ? a : b (right associative, lowest precedence)
            c = self.binary(0)
            if self.peek() != "?":
                return c
            self.eat("?")
            a = self.expr()
            self.eat(":")
            return ("cond", c, a, self.expr())
        return self.binary(level)

    def binary(self, level):
        if level == len(self.PREC):
            return self.unary()
        left = self.binary(level + 1)
        while self.peek() in self.PREC[level]:
            op = self.eat()
            right = self.binary(level + 1)
            left = ("bin", op, left, right)
        return left

    def unary(self):
        p = self.peek()
        if p == "!":
            self.eat()
            return ("not", self.unary())
        if p == "-" and self.t[self.i + 1][0] == "num":
            self.eat()
            return self.number(negate=True)
        if p == "*":
            self.eat()
            self.eat("(")
            self.eat("(")
            if self.peek() == "__global":
                self.eat()
            ty = self.eat()
            self.eat("*")
            self.eat(")")
            e = self.unary()
            self.eat(")")
            return ("deref", ty, e)
        if p == "(" and self.peek(1) in T and self.peek(2) == ")":
            self.eat()
            ty = self.eat()
            self.eat(")")
            return ("cast", ty, self.unary())
        return self.postfix()

    def number(self, negate=False):
        s = self.eat()
        suf = ""
        for k in ("UL", "L", "u", "f"):
            if s.endswith(k) and not s.startswith("0x"):
                suf = k
                s = s[: -len(k)]
                break
        if "." in s or suf == "f":
            v = float(s)
            if negate:
                v = -v
            return ("lit", "float" if suf == "f" else "double", v)
        v = int(s, 0)
        if negate:
            v = -v
        ty = {"": "int", "u": "uint", "L": "long", "UL": "ulong"}[suf]
        return ("lit", ty, v)

    def postfix(self):
        p = self.peek()
        kind = self.t[self.i][0]
        if p == "(":
            self.eat()
            e = self.expr()
            self.eat(")")
            return e
        if kind == "num":
            return self.number()
        if kind == "id":
            nm = self.eat()
            if self.peek() == "(":
                self.eat()
                args = []
                if self.peek() != ")":
                    args.append(self.expr())
                    while self.peek() == ",":
                        self.eat()
                        args.append(self.expr())
                self.eat(")")
                return ("call", nm, args)
            if self.peek() == "[":
                self.eat()
                idx = self.expr()
                self.eat("]")
                if nm not in self.scope or self.scope[nm][0] != "ptr":
                    raise ParseError(f"{nm} is not a pointer argument")
                return ("index", nm, idx)
            if nm in self.decls:
                return ("var", nm)
            if nm in self.scope and self.scope[nm][0] == "val":
                return ("arg", nm)
            raise ParseError(f"undeclared identifier {nm}")
        raise ParseError(f"unexpected token {p!r}")


def parse(text: str):
    return Parser(lex(text)).kernels()


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------
class EvalError(Exception):
    pass


def _wrap(v, ty):
    """Python int / float -> numpy scalar of type ty with C wrap-around."""
    if ty in INTS:
        bits = WIDTH[ty]
        v = int(v) & ((1 << bits) - 1)
        return np.array([v], dtype=UINT_OF[bits]).view(T[ty])[0]
    return T[ty](v)


class Env:
    def __init__(self, k: Kernel, buffers, scalars, ids):
        self.k = k
        self.buf = buffers
        self.sc = scalars
        self.ids = ids       # dict: gid, lid, grp, gofs -> tuple of 3
        self.vars = {}
        self.ptypes = {p[2]: p[1] for p in k.params}


def ev(e, env: Env):
    """Evaluate -> (type, numpy scalar)."""
    k = e[0]
    if k == "lit":
        ty, v = e[1], e[2]
        if ty in INTS:
            lo, hi = {"int": (-2**31, 2**31), "uint": (0, 2**32), "long": (-2**63, 2**63), "ulong": (0, 2**64)}[ty]
            if not (lo <= v < hi):
                raise EvalError(f"literal {v} out of range for {ty}")
        return ty, _wrap(v, ty) if ty in INTS else T[ty](v)
    if k == "var":
        if e[1] not in env.vars:
            raise EvalError(f"read of unassigned {e[1]}")
        return env.k.decls[e[1]], env.vars[e[1]]
    if k == "arg":
        ty = env.ptypes[e[1]]
        return ty, T[ty](env.sc[e[1]])
    if k == "index":
        ty = env.ptypes[e[1]]
        ity, iv = ev(e[2], env)
        if ity not in INTS:
            raise EvalError("non-integer index")
        arr = env.buf[e[1]]
        return ty, arr[int(iv)]
    if k == "cast":
        ty = e[1]
        sty, v = ev(e[2], env)
        return ty, convert(v, sty, ty)
    if k == "not":
        ty, v = ev(e[1], env)
        return "int", np.int32(0 if v != 0 else 1)
    if k == "call":
        return call(e[1], [ev(a, env) for a in e[2]], env)
    if k == "bin":
        op = e[1]
        lt, lv = ev(e[2], env)
        rt, rv = ev(e[3], env)
        if op in ("<<", ">>"):
            if lt not in INTS or rt not in INTS:
                raise EvalError("shift of non-integer")
            n = int(rv)
            if not (0 <= n < WIDTH[lt]):
                raise EvalError("shift count out of range")
            if op == "<<":
                return lt, _wrap(int(lv) << n, lt)
            return lt, _wrap(int(lv) >> n, lt)  # python >> on signed = arithmetic
        if lt != rt:
            raise EvalError(f"operand types differ: {lt} {op} {rt}")
        with np.errstate(all="ignore"):
            if op in ("==", "!=", "<", ">", "<=", ">="):
                r = {"==": lv == rv, "!=": lv != rv, "<": lv < rv, ">": lv > rv, "<=": lv <= rv, ">=": lv >= rv}[op]
                return "int", np.int32(1 if r else 0)
            if lt in INTS:
                a, b = int(lv), int(rv)
                r = {"+": a + b, "-": a - b, "*": a * b, "&": a & b, "|": a | b, "^": a ^ b}[op]
                return lt, _wrap(r, lt)
            if op in ("&", "|", "^"):
                raise EvalError("bitwise op on float")
            r = {"+": lv + rv, "-": lv - rv, "*": lv * rv}[op]
            return lt, T[lt](r)
    if k == "cond":  # both arms are evaluated (they have no side effects) and must agree in type
        ct, cv = ev(e[1], env)
        if ct not in INTS:
            raise EvalError("non-integer condition")
        at, av = ev(e[2], env)
        bt, bv = ev(e[3], env)
        if at != bt:
            raise EvalError(f"arms of ?: differ: {at} {bt}")
        return at, av if int(cv) != 0 else bv
    if k == "deref":
        raise EvalError("raw pointer dereference")
    raise EvalError(f"cannot evaluate {k}")


def convert(v, sty, ty):
    if sty == ty:
        return v
    with np.errstate(all="ignore"):
        if sty in INTS and ty in INTS:
            return _wrap(int(v), ty)
        if sty in INTS and ty in ("float", "double"):
            return T[ty](int(v))  # numpy rounds to nearest
        if sty in ("float", "double") and ty in ("float", "double"):
            return T[ty](v)
    raise EvalError(f"unsupported conversion {sty} -> {ty}")


def call(nm, args, env: Env):
    def want(n):
        if len(args) != n:
            raise EvalError(f"{nm} expects {n} args")

    if nm in ("get_global_id", "get_local_id", "get_group_id", "get_global_offset"):
        want(1)
        d = int(args[0][1])
        key = {"get_global_id": "gid", "get_local_id": "lid", "get_group_id": "grp", "get_global_offset": "gofs"}[nm]
        return "uint", np.uint32(env.ids[key][d])
    if nm in ("get_global_size", "get_num_groups"):
        want(1)
        d = int(args[0][1])
        return "uint", np.uint32(env.ids["gsize" if nm == "get_global_size" else "ngrp"][d])
    if nm == "get_work_dim":
        want(0)
        return "uint", np.uint32(env.ids["wdim"])
    if nm == "fma":
        want(3)
        tys = {a[0] for a in args}
        if len(tys) != 1 or tys.pop() not in ("float", "double"):
            raise EvalError("fma operand types")
        ty = args[0][0]
        f = fma32 if ty == "float" else fma64
        return ty, f(args[0][1], args[1][1], args[2][1])
    if nm in ("mad24", "mul24"):
        n = 3 if nm == "mad24" else 2
        want(n)
        if any(a[0] != "uint" for a in args):
            raise EvalError(f"{nm} operand types")
        r = (int(args[0][1]) & 0xFFFFFF) * (int(args[1][1]) & 0xFFFFFF)
        if nm == "mad24":
            r += int(args[2][1])
        return "uint", _wrap(r, "uint")
    if nm == "mul_hi":  # high half of the full product of two 32-bit integers of one type
        want(2)
        if args[0][0] != args[1][0] or args[0][0] not in ("int", "uint"):
            raise EvalError("mul_hi operand types")
        ty = args[0][0]
        x, y = int(args[0][1]), int(args[1][1])
        return ty, _wrap((x * y) >> 32, ty)
    if nm == "upsample":
        want(2)
        if args[0][0] != "uint" or args[1][0] != "uint":
            raise EvalError("upsample operand types")
        return "ulong", np.uint64((int(args[0][1]) << 32) | int(args[1][1]))
    if nm.startswith("as_"):
        want(1)
        ty = nm[3:]
        sty, v = args[0]
        if WIDTH[sty] != WIDTH[ty]:
            raise EvalError("as_ width mismatch")
        return ty, np.array([v], dtype=T[sty]).view(T[ty])[0]
    raise EvalError(f"unknown function {nm}")


class _Break(Exception):
    """`break;`: leaves the innermost do-while."""


def run_block(items, env):
    """Runs the statements of one work-item; a generator that yields at every barrier."""
    for s in items:
        if s[0] == "barrier":
            yield
            continue
        if s[0] == "break":
            raise _Break()
        if s[0] == "assign":
            lhs, rhs = s[1], s[2]
            rty, rv = ev(rhs, env)
            if lhs[0] == "var":
                ty = env.k.decls[lhs[1]]
                if ty != rty:
                    raise EvalError(f"assignment {lhs[1]}:{ty} = {rty}")
                env.vars[lhs[1]] = rv
            elif lhs[0] == "index":
                ty = env.ptypes[lhs[1]]
                if ty != rty:
                    raise EvalError(f"store {lhs[1]}:{ty} = {rty}")
                ity, iv = ev(lhs[2], env)
                if ity not in INTS:
                    raise EvalError("non-integer index")
                env.buf[lhs[1]][int(iv)] = rv
            else:
                raise EvalError("raw pointer store")
        elif s[0] == "if":
            _, c = ev(s[1], env)
            yield from run_block(s[2] if c != 0 else s[3], env)
        elif s[0] == "do":
            n = 0
            while True:
                try:
                    yield from run_block(s[1], env)
                except _Break:
                    break
                n += 1
                if n > 100000:
                    raise EvalError("loop limit")
                _, c = ev(s[2], env)
                if c == 0:
                    break


LOCAL_ELEMS = 4096  # elements of each __local buffer, per work-group


def run_ndrange(k: Kernel, buffers, scalars, cws, dims, groups=(2, 1), gofs=(0, 0, 0)):
    """Every work-group of the NDRange; inside a group the work-items run in turn up to the next
    barrier, and every work-item must reach the same barrier (or the end) before any goes on.
    Each group has fresh __local buffers."""
    c0, c1 = cws[0], (cws[1] if dims > 1 else 1)
    g1n = groups[1] if dims > 1 else 1
    local = [p for p in k.params if p[0] == "ptr" and len(p) > 3 and p[3] == "__local"]
    for g1 in range(g1n):
        for g0 in range(groups[0]):
            bufs = dict(buffers)
            for p in local:
                bufs[p[2]] = np.zeros(LOCAL_ELEMS, dtype=T[p[1]])
            items = []
            for l1 in range(c1):
                for l0 in range(c0):
                    ids = {"lid": (l0, l1, 0), "grp": (g0, g1, 0), "gofs": gofs,
                           "gid": ((g0 * c0 + l0 + gofs[0]) & 0xFFFFFFFF, (g1 * c1 + l1 + gofs[1]) & 0xFFFFFFFF, 0),
                           "gsize": (groups[0] * c0, g1n * c1, 1), "ngrp": (groups[0], g1n, 1), "wdim": dims}
                    items.append(run_block(k.body, Env(k, bufs, scalars, ids)))
            with np.errstate(all="ignore"):
                while items:
                    at_barrier = []
                    for g in items:
                        try:
                            next(g)
                            at_barrier.append(g)
                        except StopIteration:
                            pass
                    if at_barrier and len(at_barrier) != len(items):
                        raise EvalError("work-items of a group disagree on a barrier")
                    items = at_barrier
