"""Seeded synthetic GCN kernel generator (shared input module).

Both the CPU oracle and the CUDA path read what this module writes; it holds
none of the decompiler's arithmetic.  The C++ source (``gcngen.cpp``) lowers a
random typed program to CLRX-style GCN text; this file builds it (g++) and wraps
it with ctypes.

Workload presets (``preset(i)``) follow the five synthetic workloads:
  0  one kernel, ~200 instrs, (__global int *a, __global float *b, uint n),
     2D NDRange with work-group (16,16,1), one divergent if/else (first form)
  1  kernels of 50..2000 instrs (log-uniform), int/uint/float/double/long,
     if / if-else / counted loop mixed 50/30/20, nesting <= 3, 1..8 buffers
  2  same distribution as 1 (used for large batches)
  3  200,000-instr kernels, int32/int64, loops nested to depth 6, spills
  4  100..50,000-instr kernels with the mix of 1 (serving requests)
  5  the mix of 1 with selects (v_cndmask_b32, the ternary) in 15% of 32-bit operations
  6  the mix of 1 with system values read through the dispatch packet (get_global_size,
     get_num_groups, get_work_dim) and scalar bit fields / shifts in 10% of integer leaves
  7  the mix of 1 with FLAT loads and stores (30% of memory accesses) and double-suffix high
     multiplies v_mul_hi_u32_u24 / v_mul_hi_i32_i24 (10% of 32-bit integer operations)
  8  mixed uniform and divergent nesting (divergent if / if-else in all three forms, uniform
     if / if-else, loops; depth <= 4), 35% of loops with an early exit (break or continue)
  9  the mix of 1 (1-D) with a __local buffer argument and exchanges through it (write the
     work-item's element, barrier, read a neighbour's) in 15% of top-level statements
Seeds: ``SEED_BASE + workload index``; kernel k of a stream uses mix(seed, k).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

SEED_BASE = 2107078090
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgcngen.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("min_len", "max_len", "type_mask")] + [
        (n, ctypes.c_int32)
        for n in (
            "w_if", "w_ifelse", "w_loop", "w_uif", "p_ctrl", "max_depth", "min_bufs", "max_bufs",
            "vgpr_budget", "sgpr_budget", "spills", "max_locals", "expr_depth", "trip_max", "dims",
            "cws0", "cws1", "fixed_args", "one_ifelse", "form_mask", "p_select", "p_sysval", "p_flat", "p_mulhi", "p_break", "p_lds",
        )
    ]


def build(force: bool = False) -> str:
    """Compile libgcngen.so in-tree (g++, no architecture-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "gcngen.cpp")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
             "-o", tmp, src])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.gcngen_preset.argtypes = [ctypes.c_int, ctypes.POINTER(Params)]
            L.gcngen_generate.restype = ctypes.c_void_p
            L.gcngen_generate.argtypes = [ctypes.POINTER(Params), ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int]
            L.gcngen_size.restype = ctypes.c_uint64
            L.gcngen_size.argtypes = [ctypes.c_void_p]
            L.gcngen_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                      ctypes.c_void_p, ctypes.c_void_p]
            L.gcngen_free.argtypes = [ctypes.c_void_p]
            L.gcngen_truth.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            _lib = L
    return _lib


def preset(cfg: int, **over) -> Params:
    p = Params()
    if lib().gcngen_preset(cfg, ctypes.byref(p)) != 0:
        raise ValueError(f"unknown workload {cfg}")
    for k, v in over.items():
        setattr(p, k, v)
    return p


class Batch:
    """Concatenated kernel text plus per-kernel byte offsets and instruction counts."""

    def __init__(self, text: np.ndarray, offsets: np.ndarray, ninstr: np.ndarray, truth: np.ndarray | None = None):
        self.text = text          # uint8[N]
        self.offsets = offsets    # uint64[n+1]
        self.ninstr = ninstr      # uint64[n]
        # uint32[n, 4]: dims (bits 0-1) and bit 2 + d set when get_global_id(d) adds the global offset;
        # the numbers of ifs, else parts and counted loops the generator emitted
        self.truth = truth

    def __len__(self):
        return len(self.ninstr)

    def kernel(self, i: int) -> bytes:
        return self.text[self.offsets[i]:self.offsets[i + 1]].tobytes()

    @property
    def total_instr(self) -> int:
        return int(self.ninstr.sum())


def generate(params: Params | int, n: int, seed: int | None = None, first: int = 0,
             threads: int | None = None, out: np.ndarray | None = None) -> Batch:
    """Generate kernels [first, first+n) of the stream (params, seed).

    ``out`` may be a preallocated uint8 buffer (e.g. pinned host memory viewed
    as numpy) large enough for the text; otherwise one is allocated."""
    cfg = params if isinstance(params, int) else None
    if cfg is not None:
        params = preset(cfg)
        if seed is None:
            seed = SEED_BASE + cfg
    if seed is None:
        seed = SEED_BASE
    if threads is None:
        threads = max(1, min(os.cpu_count() or 1, 32, n))
    L = lib()
    h = L.gcngen_generate(ctypes.byref(params), seed, first, n, threads)
    if not h:
        raise RuntimeError("gcngen_generate failed")
    try:
        size = L.gcngen_size(h)
        if out is None:
            out = np.empty(size, dtype=np.uint8)
        elif out.nbytes < size:
            raise ValueError(f"output buffer too small: {out.nbytes} < {size}")
        offs = np.empty(n + 1, dtype=np.uint64)
        ni = np.empty(n, dtype=np.uint64)
        rc = L.gcngen_copy(h, out.ctypes.data, out.nbytes, offs.ctypes.data, ni.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"gcngen_copy failed: {rc}")
        truth = np.empty((n, 4), dtype=np.uint32)
        if L.gcngen_truth(h, truth.ctypes.data) != 0:
            raise RuntimeError("gcngen_truth failed")
    finally:
        L.gcngen_free(h)
    return Batch(out[:size], offs, ni, truth)
