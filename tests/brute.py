"""Brute-force semantic check: the GCN program and its decompiled OpenCL must
write identical output buffers for every work-item of a small NDRange.

The assembly runs in ``gcn_interp`` (wave64 with exec masks), the decompiled
text in ``ocl_eval`` (one work-item at a time), both on copies of the same
seeded random buffers, with non-zero global offsets so that get_global_id and
get_global_id - get_global_offset are told apart.
"""
from __future__ import annotations

import numpy as np

import gcn_interp
import ocl_eval

BUF_LEN = 4096
GOFS = (3, 5, 0)


def random_buffers(prog: gcn_interp.KernelText, seed: int, wide: bool = False):
    """Seeded buffers for the kernel's pointer arguments and values for its scalars.  With
    `wide`, 32-bit integer buffers take values over their whole range (so that the high half of
    a 24-bit product is not always zero); floats stay small and exact."""
    rng = np.random.default_rng(seed)
    bufs, scal = {}, {}
    for name, hidden, ptr, elem in prog.args:
        if hidden or name in prog.local_args:  # a __local buffer lives in each work-group's LDS
            continue
        if not ptr:
            scal[name] = int(rng.integers(0, 40))
            continue
        if elem == "int":
            a = (rng.integers(-2**31, 2**31, BUF_LEN) if wide else rng.integers(-1000, 1000, BUF_LEN)).astype(np.int32)
        elif elem == "uint":
            a = (rng.integers(0, 2**32, BUF_LEN) if wide else rng.integers(0, 2000, BUF_LEN)).astype(np.uint32)
        elif elem == "long":
            a = rng.integers(-10**6, 10**6, BUF_LEN).astype(np.int64)
        elif elem == "float":
            a = (rng.integers(-64, 64, BUF_LEN) / 8.0).astype(np.float32)
        elif elem == "double":
            a = (rng.integers(-64, 64, BUF_LEN) / 8.0).astype(np.float64)
        else:
            raise ValueError(elem)
        bufs[name] = a
    return bufs, scal


def check(asm_text: str, ocl_text: str, seed: int = 0, groups=(2, 1), wide: bool = False, scalars=None):
    """Returns None when both executions agree, else a description.  `scalars` overrides
    the seeded values of scalar arguments."""
    prog = gcn_interp.KernelText(asm_text)
    bufs, scal = random_buffers(prog, seed, wide)
    scal.update(scalars or {})
    b_asm = {k: v.copy() for k, v in bufs.items()}
    b_ocl = {k: v.copy() for k, v in bufs.items()}
    gcn_interp.run_ndrange(asm_text, b_asm, scal, groups=groups, gofs=GOFS)
    try:
        ks = ocl_eval.parse(ocl_text)
        assert len(ks) == 1
        ocl_eval.run_ndrange(ks[0], b_ocl, scal, prog.cws, prog.dims, groups=groups, gofs=GOFS)
    except (ocl_eval.ParseError, ocl_eval.EvalError, IndexError) as e:
        return f"decompiled text failed: {type(e).__name__}: {e}"
    for k in bufs:
        a, b = b_asm[k].view(np.uint8), b_ocl[k].view(np.uint8)
        if not np.array_equal(a, b):
            bad = np.nonzero(np.any((b_asm[k].view(np.uint8).reshape(BUF_LEN, -1) !=
                                     b_ocl[k].view(np.uint8).reshape(BUF_LEN, -1)), axis=1))[0]
            i = int(bad[0])
            return f"buffer {k} differs at {len(bad)} elements, first [{i}]: asm {b_asm[k][i]!r} ocl {b_ocl[k][i]!r}"
        del a, b
    changed = any(not np.array_equal(b_asm[k].view(np.uint8), bufs[k].view(np.uint8)) for k in bufs)
    if not changed:
        return "no buffer was written (check is vacuous)"
    return None
