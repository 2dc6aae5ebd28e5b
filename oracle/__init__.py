"""CPU oracle of the GCN -> OpenCL decompiler.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (``paper_2107_07809_gb300``)
never calls it and shares no code with it.

``oracle.cpp`` is a plain single-threaded decompiler written step by step from
the paper (body extraction, ABI register initialisation, instruction
processing, region graph, OpenCL generation).  This wrapper builds it with g++
and exposes it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

IR_INSTR, IR_PBLOCK_OF, IR_PBLOCKS, IR_LBLOCK_OF, IR_LBLOCKS, IR_HEADER, IR_STATS = range(7)
TYPES = ["none", "int", "uint", "float", "long", "ulong", "double", "top32", "top64"]
STATUS = {0: "OK", 1: "PARTIAL", 2: "PARSE_ERROR", 3: "FIXPOINT_CAP"}


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp, src])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
            L.oracle_decompile.restype = vp
            L.oracle_decompile.argtypes = [ctypes.c_char_p, u64]
            L.oracle_text_len.restype = u64
            L.oracle_text_len.argtypes = [vp]
            L.oracle_text.argtypes = [vp, ctypes.c_char_p]
            L.oracle_nkernels.argtypes = [vp]
            L.oracle_kernel_status.argtypes = [vp, i32]
            L.oracle_ir_len.restype = u64
            L.oracle_ir_len.argtypes = [vp, i32, i32]
            L.oracle_ir.argtypes = [vp, i32, i32, vp]
            L.oracle_free.argtypes = [vp]
            L.oracle_batch.restype = vp
            L.oracle_batch.argtypes = [vp, vp, u64, i32]
            L.oracle_batch_len.restype = u64
            L.oracle_batch_len.argtypes = [vp]
            L.oracle_batch_copy.argtypes = [vp, vp, vp, vp]
            L.oracle_batch_free.argtypes = [vp]
            L.oracle_reduce_graph.argtypes = [i32, vp, vp, vp, i32]
            L.oracle_type_join.argtypes = [i32, i32]
            L.oracle_set_type_sweep_limit.argtypes = [ctypes.c_uint32]
            L.oracle_set_class_depth.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


class Result:
    def __init__(self, text: str, status: list[int], ir: list[dict]):
        self.text = text
        self.status = status      # per kernel
        self.ir = ir              # per kernel: {which: bytes}

    @property
    def worst(self) -> int:
        return max(self.status) if self.status else 0


def decompile(text: bytes | str, with_ir: bool = False) -> Result:
    """Decompile one disassembly file (all of its kernels)."""
    if isinstance(text, str):
        text = text.encode()
    L = lib()
    h = L.oracle_decompile(text, len(text))
    try:
        n = L.oracle_text_len(h)
        buf = ctypes.create_string_buffer(n + 1)
        L.oracle_text(h, buf)
        nk = L.oracle_nkernels(h)
        st = [L.oracle_kernel_status(h, k) for k in range(nk)]
        ir = []
        if with_ir:
            for k in range(nk):
                d = {}
                for w in range(7):
                    m = L.oracle_ir_len(h, k, w)
                    b = ctypes.create_string_buffer(max(m, 1))
                    L.oracle_ir(h, k, w, b)
                    d[w] = b.raw[:m]
                ir.append(d)
        return Result(buf.raw[:n].decode(), st, ir)
    finally:
        L.oracle_free(h)


def set_type_sweep_limit(n: int = 0) -> None:
    """Sweep limit of the type fixed point for later calls (0 = the default, never reached).  A
    kernel whose types still change in the last allowed sweep is not decompiled: status 3 and the
    text `/* not decompiled: fixed-point limit */` (a test hook for the capped path)."""
    lib().oracle_set_type_sweep_limit(n)


def set_class_depth(d: int = -1) -> None:
    """Depth below which a node gets no class in later calls (negative = the default, 4).  A test
    hook: a class comes from operands at most three levels down, so any larger depth gives the
    same output."""
    lib().oracle_set_class_depth(d)


def decompile_batch(text: np.ndarray, offsets: np.ndarray, threads: int = 1):
    """Decompile files [offsets[i], offsets[i+1]) of ``text`` (uint8).

    Returns (out uint8 array, out_offsets uint64[n+1], worst status int32[n])."""
    L = lib()
    text = np.ascontiguousarray(text, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = len(offsets) - 1
    h = L.oracle_batch(text.ctypes.data, offsets.ctypes.data, n, threads)
    try:
        m = L.oracle_batch_len(h)
        out = np.empty(max(m, 1), dtype=np.uint8)
        oo = np.empty(n + 1, dtype=np.uint64)
        st = np.empty(n, dtype=np.int32)
        L.oracle_batch_copy(h, out.ctypes.data, oo.ctypes.data, st.ctypes.data)
        return out[:m], oo, st
    finally:
        L.oracle_batch_free(h)


def reduce_graph(succ0: list[int], succ1: list[int]):
    """Structural analysis alone on an abstract CFG; returns the merge log
    [(new_id, [members...]), ...] or None when it does not reduce."""
    n = len(succ0)
    a = np.asarray(succ0, dtype=np.int32)
    b = np.asarray(succ1, dtype=np.int32)
    out = np.zeros(4096, dtype=np.int32)
    w = lib().oracle_reduce_graph(n, a.ctypes.data, b.ctypes.data, out.ctypes.data, len(out))
    if w < 0:
        return None
    log, i = [], 0
    while i < w:
        nid, cnt = int(out[i]), int(out[i + 1])
        log.append((nid, [int(x) for x in out[i + 2:i + 2 + cnt]]))
        i += 2 + cnt
    return log


def type_join(a: int, b: int) -> int:
    return lib().oracle_type_join(a, b)
