"""A small wave64 interpreter for the GCN dialect the decompiler reads.

Test infrastructure: it runs the assembly itself over a tiny NDRange so that
the decompiled OpenCL (run by ``ocl_eval``) can be compared with the program's
real behaviour on random buffers.  It shares no code with the oracle or the
CUDA path.  Semantics follow the GCN machine model the paper describes
("The AMD GCN architecture"): 64 work-items per wavefront execute each
instruction together, vector writes are masked by the 64-bit exec mask, scalar
registers are shared by the wavefront, v0..v2 hold the local id, s6..s8 the
group id (with .useargs), s[4:5] points at the kernel settings (global
offsets at 0x0/0x8/0x10, arguments from 0x30 in 8-byte slots) and s[0:1] at the
dispatch packet (header and setup in the dword at 0x0, the dimension count in
setup bits 0..1; work-group size as 16-bit fields at 0x4/0x6/0x8; global size
as dwords at 0xc/0x10/0x14).
"""
from __future__ import annotations

import re
import struct

import numpy as np

from fp_exact import fma32, fma64

W = 64
KARG_BASE = 0x1_0000_0000
DISP_BASE = 0x2_0000_0000
# packet header: kernel dispatch type with fences; the reserved setup bits above the
# dimension count are not zero here, so that a wrong field width shows
DISP_HEADER = 0x1402
DISP_SETUP_RESERVED = 0x0054
SCRATCH = object()
INLINE_F = {"0.5": 0x3F000000, "-0.5": 0xBF000000, "1.0": 0x3F800000, "-1.0": 0xBF800000,
            "2.0": 0x40000000, "-2.0": 0xC0000000, "4.0": 0x40800000, "-4.0": 0xC0800000}
ELEM = {"int": np.int32, "uint": np.uint32, "float": np.float32, "double": np.float64,
        "long": np.int64, "ulong": np.uint64}


class KernelText:
    def __init__(self, text: str):
        self.name = None
        self.dims = 1
        self.cws = [1, 1, 1]
        self.args = []        # (name, hidden, pointer, elem)
        self.local_args = set()  # pointer arguments in the local address space (LDS)
        self.useargs = False
        self.instrs = []      # (mnemonic, [operand strings], modifiers dict)
        self.labels = {}
        state = None
        for raw in text.split("\n"):
            row = raw.strip()
            if not row:
                continue
            w = row.split()
            if w[0] == ".kernel":
                self.name = w[1]
                state = "k"
                continue
            if w[0] == ".config":
                state = "c"
                continue
            if w[0] == ".text":
                state = "t"
                continue
            if state == "c":
                if w[0] in (".dims", "dims"):
                    self.dims = len(w[1])
                elif w[0] == ".cws":
                    self.cws = [int(x) for x in row[4:].split(",")]
                elif w[0] == ".useargs":
                    self.useargs = True
                elif w[0] == ".arg":
                    f = [x.strip() for x in row[4:].split(",")]
                    ty = f[2]
                    ptr = ty.endswith("*")
                    self.args.append((f[0], f[0].startswith("_."), ptr, ty[:-1] if ptr else ty))
                    if ptr and len(f) > 3 and f[3] == "local":
                        self.local_args.add(f[0])
            elif state == "t":
                if len(w) == 1 and row.endswith(":"):
                    self.labels[row[:-1]] = len(self.instrs)
                    continue
                m = w[0]
                rest = row[len(m):].strip()
                ops, mods = [], {}
                if m != "s_waitcnt" and rest:
                    for fld in rest.split(","):
                        sub = fld.split()
                        ops.append(sub[0])
                        for s in sub[1:]:
                            if s.startswith("offset:"):
                                mods["offset"] = int(s[7:], 0)
                self.instrs.append((m, ops, mods))


_rng = re.compile(r"^([vs])\[(\d+):(\d+)\]$")
_one = re.compile(r"^([vs])(\d+)$")


class Wave:
    def __init__(self, prog: KernelText, mem, kargs: bytes, lid, grp, active, disp: bytes = b"", lds=None):
        self.p = prog
        self.mem = mem                    # dict base -> numpy array (buffers)
        self.lds = lds                    # the work-group's LDS bytes (uint8 array)
        self.karg = kargs
        self.disp = disp
        self.v = np.zeros((256, W), dtype=np.uint32)
        self.s = np.zeros(112, dtype=np.uint32)
        self.vcc = np.zeros(W, dtype=bool)
        self.exec = active.copy()
        self.scc = False
        self.scratch = {}
        for d in range(prog.dims):
            self.v[d] = lid[d]
            if prog.useargs:
                self.s[6 + d] = grp[d]
        self.s[4] = KARG_BASE & 0xFFFFFFFF
        self.s[5] = KARG_BASE >> 32
        self.s[0] = DISP_BASE & 0xFFFFFFFF
        self.s[1] = DISP_BASE >> 32

    # ---- operand access ------------------------------------------------------
    def regs(self, t):
        m = _rng.match(t)
        if m:
            return m.group(1), list(range(int(m.group(2)), int(m.group(3)) + 1))
        m = _one.match(t)
        if m:
            return m.group(1), [int(m.group(2))]
        raise ValueError(t)

    def const(self, t):
        if t in INLINE_F:
            return INLINE_F[t]
        return int(t, 0) & 0xFFFFFFFF

    def rd32(self, t) -> np.ndarray:
        if t == "vcc":
            raise ValueError("vcc as 32-bit")
        if t[0] in "vs" and (t[1:].isdigit()):
            k, r = self.regs(t)
            if k == "v":
                return self.v[r[0]].copy()
            return np.full(W, self.s[r[0]], dtype=np.uint32)
        return np.full(W, self.const(t), dtype=np.uint32)

    def rd64(self, t) -> np.ndarray:
        k, r = self.regs(t)
        if k == "v":
            return self.v[r[0]].astype(np.uint64) | (self.v[r[1]].astype(np.uint64) << np.uint64(32))
        return np.full(W, int(self.s[r[0]]) | (int(self.s[r[1]]) << 32), dtype=np.uint64)

    def wr32(self, t, val):
        k, r = self.regs(t)
        val = np.asarray(val).astype(np.uint32)
        if k == "v":
            self.v[r[0]] = np.where(self.exec, val, self.v[r[0]])
        else:
            self.s[r[0]] = val if val.ndim == 0 else val[0]

    def wr64(self, t, val):
        k, r = self.regs(t)
        val = np.asarray(val).astype(np.uint64)
        lo = (val & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        hi = (val >> np.uint64(32)).astype(np.uint32)
        if k == "v":
            self.v[r[0]] = np.where(self.exec, lo, self.v[r[0]])
            self.v[r[1]] = np.where(self.exec, hi, self.v[r[1]])
        else:
            self.s[r[0]], self.s[r[1]] = int(lo), int(hi)

    def mask64(self, t) -> int:
        if t == "exec":
            return _bits(self.exec)
        if t == "vcc":
            return _bits(self.vcc)
        k, r = self.regs(t)
        return int(self.s[r[0]]) | (int(self.s[r[1]]) << 32)

    def set_mask64(self, t, m: int):
        b = _unbits(m)
        if t == "exec":
            self.exec = b
        elif t == "vcc":
            self.vcc = b
        else:
            k, r = self.regs(t)
            self.s[r[0]] = m & 0xFFFFFFFF
            self.s[r[1]] = m >> 32

    # ---- memory ---------------------------------------------------------------
    def gaddr(self, addr: int):
        for base, arr in self.mem.items():
            off = addr - base
            if 0 <= off < arr.nbytes:
                return arr, off
        raise IndexError(f"address {addr:#x} outside every buffer")

    def karg_load(self, addr, nd):
        if DISP_BASE <= addr < DISP_BASE + len(self.disp):
            return struct.unpack_from(f"<{nd}I", self.disp, addr - DISP_BASE)
        off = addr - KARG_BASE
        if not 0 <= off <= len(self.karg) - 4 * nd:
            raise IndexError(f"scalar load at {addr:#x} outside the settings and the dispatch packet")
        return struct.unpack_from(f"<{nd}I", self.karg, off)

    # ---- execution --------------------------------------------------------------
    def run(self, max_steps=2_000_000):
        pc = 0
        steps = 0
        ins = self.p.instrs
        while pc < len(ins):
            steps += 1
            if steps > max_steps:
                raise RuntimeError("interpreter step limit")
            m, o, mods = ins[pc]
            pc += 1
            nxt = self.step(m, o, mods)
            if nxt == "end":
                return
            if nxt is not None:
                pc = nxt

    def step(self, m, o, mods):
        ex = self.exec
        u = np.uint32
        if m == "s_waitcnt":
            return None
        if m.startswith("s_load_dword"):
            nd = {"s_load_dword": 1, "s_load_dwordx2": 2, "s_load_dwordx4": 4}[m]
            base = self.mask64(o[1])
            vals = self.karg_load(base + self.const(o[2]), nd)
            k, r = self.regs(o[0])
            for i in range(nd):
                self.s[r[i]] = vals[i]
            return None
        if m == "s_mov_b32":
            self.wr32(o[0], self.rd32(o[1])[0])
            return None
        if m in ("s_mul_i32", "s_lshl_b32", "s_add_u32"):
            a, b = int(self.rd32(o[1])[0]), int(self.rd32(o[2])[0])
            if m == "s_mul_i32":
                r = (a * b) & 0xFFFFFFFF
            elif m == "s_lshl_b32":
                r = (a << (b & 31)) & 0xFFFFFFFF
                self.scc = r != 0
            else:
                r = (a + b) & 0xFFFFFFFF
                self.scc = a + b > 0xFFFFFFFF
            self.wr32(o[0], np.uint32(r))
            return None
        if m in ("s_lshr_b32", "s_bfe_u32"):
            a, b = int(self.rd32(o[1])[0]), int(self.rd32(o[2])[0])
            if m == "s_lshr_b32":
                r = a >> (b & 31)
            else:  # field: offset bits [4:0], width bits [22:16]
                w = (b >> 16) & 0x7F
                if w >= 32:
                    raise ValueError("s_bfe_u32 width >= 32")
                r = (a >> (b & 31)) & ((1 << w) - 1)
            self.scc = r != 0
            self.wr32(o[0], np.uint32(r))
            return None
        if m.startswith("s_cmp_"):
            _, _, cc, ty = m.split("_")
            a, b = int(self.rd32(o[0])[0]), int(self.rd32(o[1])[0])
            if ty == "i32":
                a, b = _s32(a), _s32(b)
            self.scc = _cmp(cc, a, b)
            return None
        if m == "s_and_saveexec_b64":
            old = self.mask64("exec")
            self.set_mask64(o[0], old)
            new = self.mask64(o[1]) & old
            self.set_mask64("exec", new)
            self.scc = new != 0
            return None
        if m == "s_or_saveexec_b64":
            old = self.mask64("exec")
            srcv = self.mask64(o[1])
            self.set_mask64(o[0], old)
            self.set_mask64("exec", srcv | old)
            return None
        if m in ("s_xor_b64", "s_or_b64"):
            a, b = self.mask64(o[1]), self.mask64(o[2])
            r = a ^ b if m == "s_xor_b64" else a | b
            self.set_mask64(o[0], r)
            self.scc = r != 0
            return None
        if m == "s_branch":
            return self.p.labels[o[0]]
        if m == "s_cbranch_scc0":
            return self.p.labels[o[0]] if not self.scc else None
        if m == "s_cbranch_scc1":
            return self.p.labels[o[0]] if self.scc else None
        if m == "s_cbranch_execz":
            return self.p.labels[o[0]] if not ex.any() else None
        if m == "s_endpgm":
            return "end"
        # ---- vector ----
        if m == "v_mov_b32":
            self.wr32(o[0], self.rd32(o[1]))
            return None
        if m in _VOP2_INT:
            a, b = self.rd32(o[1]).astype(np.uint64), self.rd32(o[2]).astype(np.uint64)
            self.wr32(o[0], _VOP2_INT[m](a, b) & np.uint64(0xFFFFFFFF))
            return None
        if m == "v_mad_u32_u24":
            a, b, c = (self.rd32(x).astype(np.uint64) for x in o[1:4])
            r = (a & np.uint64(0xFFFFFF)) * (b & np.uint64(0xFFFFFF)) + c
            self.wr32(o[0], r & np.uint64(0xFFFFFFFF))
            return None
        if m in ("v_add_f32", "v_sub_f32", "v_mul_f32"):
            a, b = self.rd32(o[1]).view(np.float32), self.rd32(o[2]).view(np.float32)
            with np.errstate(all="ignore"):
                r = a + b if m == "v_add_f32" else (a - b if m == "v_sub_f32" else a * b)
            self.wr32(o[0], r.astype(np.float32).view(np.uint32))
            return None
        if m == "v_fma_f32":
            a, b, c = (self.rd32(x).view(np.float32) for x in o[1:4])
            r = np.array([fma32(a[i], b[i], c[i]) if ex[i] else np.float32(0) for i in range(W)], dtype=np.float32)
            self.wr32(o[0], r.view(np.uint32))
            return None
        if m == "v_cvt_f32_i32":
            self.wr32(o[0], self.rd32(o[1]).view(np.int32).astype(np.float32).view(np.uint32))
            return None
        if m == "v_cvt_f32_u32":
            self.wr32(o[0], self.rd32(o[1]).astype(np.float32).view(np.uint32))
            return None
        if m == "v_cvt_f64_f32":
            self.wr64(o[0], self.rd32(o[1]).view(np.float32).astype(np.float64).view(np.uint64))
            return None
        if m == "v_cvt_f64_i32":
            self.wr64(o[0], self.rd32(o[1]).view(np.int32).astype(np.float64).view(np.uint64))
            return None
        if m == "v_cvt_f32_f64":
            with np.errstate(all="ignore"):
                self.wr32(o[0], self.rd64(o[1]).view(np.float64).astype(np.float32).view(np.uint32))
            return None
        if m.startswith("v_cmp_"):
            _, _, cc, ty = m.split("_")
            a, b = self.rd32(o[1]), self.rd32(o[2])
            if ty == "i32":
                a, b = a.view(np.int32), b.view(np.int32)
            elif ty == "f32":
                a, b = a.view(np.float32), b.view(np.float32)
            with np.errstate(all="ignore"):
                self.vcc = _cmpv(cc, a, b) & ex
            return None
        if m == "v_cndmask_b32":  # vD = vcc ? src1 : src0
            if o[3] != "vcc":
                raise ValueError("v_cndmask_b32 selects on vcc only")
            self.wr32(o[0], np.where(self.vcc, self.rd32(o[2]), self.rd32(o[1])))
            return None
        if m in ("v_add_co_u32", "v_sub_co_u32"):
            a, b = self.rd32(o[2]).astype(np.int64), self.rd32(o[3]).astype(np.int64)
            r = a + b if m == "v_add_co_u32" else a - b
            carry = (r > 0xFFFFFFFF) if m == "v_add_co_u32" else (r < 0)
            self.wr32(o[0], (r & 0xFFFFFFFF).astype(np.uint64))
            self.vcc = carry & ex
            return None
        if m in ("v_addc_co_u32", "v_subb_co_u32"):
            a, b = self.rd32(o[2]).astype(np.int64), self.rd32(o[3]).astype(np.int64)
            c = self.vcc.astype(np.int64)
            r = a + b + c if m == "v_addc_co_u32" else a - b - c
            carry = (r > 0xFFFFFFFF) if m == "v_addc_co_u32" else (r < 0)
            self.wr32(o[0], (r & 0xFFFFFFFF).astype(np.uint64))
            self.vcc = carry & ex
            return None
        if m == "v_lshlrev_b64":
            sh = self.rd32(o[1]).astype(np.uint64) & np.uint64(63)
            self.wr64(o[0], self.rd64(o[2]) << sh)
            return None
        if m in ("v_add_f64", "v_mul_f64"):
            a, b = self.rd64(o[1]).view(np.float64), self.rd64(o[2]).view(np.float64)
            with np.errstate(all="ignore"):
                r = a + b if m == "v_add_f64" else a * b
            self.wr64(o[0], r.view(np.uint64))
            return None
        if m == "v_fma_f64":
            a, b, c = (self.rd64(x).view(np.float64) for x in o[1:4])
            r = np.array([fma64(a[i], b[i], c[i]) if ex[i] else 0.0 for i in range(W)], dtype=np.float64)
            self.wr64(o[0], r.view(np.uint64))
            return None
        if m in ("global_load_dword", "global_load_dwordx2", "flat_load_dword", "flat_load_dwordx2"):
            # a FLAT access here always reaches global memory (the generator forms its address
            # from a buffer argument), so it behaves as the GLOBAL one
            addr = self.rd64(o[1])
            nb = 4 if m in ("global_load_dword", "flat_load_dword") else 8
            val = np.zeros(W, dtype=np.uint64)
            for i in range(W):
                if ex[i]:
                    arr, off = self.gaddr(int(addr[i]))
                    val[i] = int.from_bytes(arr.view(np.uint8)[off:off + nb].tobytes(), "little")
            if nb == 4:
                self.wr32(o[0], val)
            else:
                self.wr64(o[0], val)
            return None
        if m in ("global_store_dword", "global_store_dwordx2", "flat_store_dword", "flat_store_dwordx2"):
            addr = self.rd64(o[0])
            nb = 4 if m in ("global_store_dword", "flat_store_dword") else 8
            val = self.rd32(o[1]).astype(np.uint64) if nb == 4 else self.rd64(o[1])
            for i in range(W):
                if ex[i]:
                    arr, off = self.gaddr(int(addr[i]))
                    arr.view(np.uint8)[off:off + nb] = np.frombuffer(int(val[i]).to_bytes(nb, "little"), np.uint8)
            return None
        if m in ("ds_read_b32", "ds_read_b64"):
            addr = self.rd32(o[1]).astype(np.int64) + mods.get("offset", 0)
            nb = 4 if m == "ds_read_b32" else 8
            val = np.zeros(W, dtype=np.uint64)
            for i in range(W):
                if ex[i]:
                    a = int(addr[i])
                    val[i] = int.from_bytes(self.lds[a:a + nb].tobytes(), "little")
            if nb == 4:
                self.wr32(o[0], val)
            else:
                self.wr64(o[0], val)
            return None
        if m in ("ds_write_b32", "ds_write_b64"):
            addr = self.rd32(o[0]).astype(np.int64) + mods.get("offset", 0)
            nb = 4 if m == "ds_write_b32" else 8
            val = self.rd32(o[1]).astype(np.uint64) if nb == 4 else self.rd64(o[1])
            for i in range(W):
                if ex[i]:
                    a = int(addr[i])
                    self.lds[a:a + nb] = np.frombuffer(int(val[i]).to_bytes(nb, "little"), np.uint8)
            return None
        if m == "s_barrier":  # the group is one wave (run_ndrange checks): its lanes are in step
            return None
        if m == "buffer_store_dword":
            slot = mods.get("offset", 0)
            cur = self.scratch.get(slot, np.zeros(W, dtype=np.uint32))
            self.scratch[slot] = np.where(ex, self.rd32(o[0]), cur)
            return None
        if m == "buffer_load_dword":
            slot = mods.get("offset", 0)
            self.wr32(o[0], self.scratch.get(slot, np.zeros(W, dtype=np.uint32)))
            return None
        raise NotImplementedError(m)


def _bits(b) -> int:
    return int(sum(1 << i for i in range(W) if b[i]))


def _unbits(m: int):
    return np.array([(m >> i) & 1 == 1 for i in range(W)], dtype=bool)


def _sext24(x):
    x &= 0xFFFFFF
    return x - (1 << 24) if x & 0x800000 else x


def _s32(x):
    return x - (1 << 32) if x & 0x80000000 else x


def _cmp(cc, a, b):
    return {"eq": a == b, "lg": a != b, "ne": a != b, "neq": a != b, "gt": a > b, "lt": a < b,
            "ge": a >= b, "le": a <= b}[cc]


def _cmpv(cc, a, b):
    if cc in ("ne", "neq", "lg"):
        return a != b
    return {"eq": a == b, "gt": a > b, "lt": a < b, "ge": a >= b, "le": a <= b}[cc]


_M32 = np.uint64(0xFFFFFFFF)
_VOP2_INT = {
    "v_add_u32": lambda a, b: a + b,
    "v_sub_u32": lambda a, b: (a - b) & _M32,
    "v_mul_lo_u32": lambda a, b: (a * b) & _M32,
    "v_mul_u32_u24": lambda a, b: (a & np.uint64(0xFFFFFF)) * (b & np.uint64(0xFFFFFF)),
    # high 32 bits of the 48-bit product of the low 24 bits (zero- / sign-extended)
    "v_mul_hi_u32_u24": lambda a, b: ((a & np.uint64(0xFFFFFF)) * (b & np.uint64(0xFFFFFF))) >> np.uint64(32),
    "v_mul_hi_i32_i24": lambda a, b: np.array(
        [((_sext24(int(x)) * _sext24(int(y))) >> 32) & 0xFFFFFFFF for x, y in zip(a, b)], dtype=np.uint64),
    "v_and_b32": lambda a, b: a & b,
    "v_or_b32": lambda a, b: a | b,
    "v_xor_b32": lambda a, b: a ^ b,
    "v_lshlrev_b32": lambda a, b: (b << (a & np.uint64(31))) & _M32,
    "v_lshrrev_b32": lambda a, b: b >> (a & np.uint64(31)),
    "v_ashrrev_i32": lambda a, b: (b.astype(np.uint32).view(np.int32) >> (a & np.uint64(31)).astype(np.int32))
    .view(np.uint32).astype(np.uint64),
}


LDS_BYTES = 65536
LDS_SLICE = 16384  # LDS bytes given to each __local argument


def make_kargs(prog: KernelText, buf_base: dict, scalars: dict, gofs) -> bytes:
    b = bytearray(8 * len(prog.args) + 64)
    nloc = 0
    for i, (name, hidden, ptr, elem) in enumerate(prog.args):
        off = 8 * i
        if hidden:
            if name.startswith("_.global_offset_"):
                struct.pack_into("<Q", b, off, gofs[int(name[-1])])
            continue
        if name in prog.local_args:  # the low dword holds the buffer's LDS address
            struct.pack_into("<Q", b, off, LDS_SLICE * nloc)
            nloc += 1
            continue
        if ptr:
            struct.pack_into("<Q", b, off, buf_base[name])
        else:
            v = np.array([scalars[name]], dtype=ELEM[elem]).view(np.uint8).tobytes()
            b[off:off + len(v)] = v
    return bytes(b)


def make_dispatch(dims: int, wg, grid) -> bytes:
    """The 64-byte dispatch packet s[0:1] points at."""
    b = bytearray(64)
    struct.pack_into("<HH", b, 0, DISP_HEADER, dims | DISP_SETUP_RESERVED)
    struct.pack_into("<HHH", b, 4, *wg)
    struct.pack_into("<III", b, 0xc, *grid)
    return bytes(b)


def run_ndrange(text: str, buffers: dict, scalars: dict, groups=(2, 1), gofs=(0, 0, 0)):
    """Run every work-group of an NDRange of ``groups`` work-groups (per dim).

    ``buffers`` maps argument name -> numpy array (modified in place)."""
    prog = KernelText(text)
    base = {}
    mem = {}
    addr = 0x10_0000_0000
    for name, hidden, ptr, elem in prog.args:
        if ptr and not hidden and name not in prog.local_args:
            base[name] = addr
            mem[addr] = buffers[name]
            addr += 0x1_0000_0000
    kargs = make_kargs(prog, base, scalars, gofs)
    c0, c1 = prog.cws[0], prog.cws[1] if prog.dims > 1 else 1
    g1n = groups[1] if prog.dims > 1 else 1
    disp = make_dispatch(prog.dims, (c0, c1, 1), (groups[0] * c0, g1n * c1, 1))
    has_barrier = any(m == "s_barrier" for m, _, _ in prog.instrs)
    if has_barrier and c0 * c1 > W:
        raise NotImplementedError("barriers in a work-group of more than one wave")
    for g1 in range(g1n):
        for g0 in range(groups[0]):
            n = c0 * c1
            lds = np.zeros(LDS_BYTES, dtype=np.uint8)  # a fresh LDS per work-group
            for w0 in range(0, n, W):
                lanes = np.arange(w0, w0 + W)
                active = lanes < n
                lid0 = np.where(active, lanes % c0, 0).astype(np.uint32)
                lid1 = np.where(active, lanes // c0, 0).astype(np.uint32)
                wave = Wave(prog, mem, kargs, (lid0, lid1, np.zeros(W, np.uint32)), (g0, g1, 0), active, disp,
                            lds)
                wave.run()
    return prog
