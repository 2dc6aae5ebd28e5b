"""The C ABI library loads and exports every entry point of include/gcn_decomp.h
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

import paper_2107_07809_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gcn_decomp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcn_decomp_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gcn_decomp_create", "gcn_decomp_submit_batch", "gcn_decomp_fetch_opencl", "gcn_decomp_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    pkg.build()
    lib = pkg.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.GcnDecompError) as e:
        pkg.Decompiler(0)
    assert e.value.rc == pkg.GCN_EINVAL


def test_noalloc_rejects_on_the_host():
    """Argument and size checks of gcn_decomp_line_starts_noalloc happen before
    any CUDA call, so they answer the same without a GPU."""
    pkg.build()
    L = pkg.lib()
    fake = 1 << 20  # never dereferenced: both calls are rejected first
    assert L.gcn_decomp_line_starts_noalloc(fake, (1 << 30) + 1, fake, 16, fake, None) == pkg.GCN_ENOMEM
    assert L.gcn_decomp_line_starts_noalloc(fake, 100, fake, 0, fake, None) == pkg.GCN_EINVAL
    assert L.gcn_decomp_line_starts_noalloc(None, 100, fake, 16, fake, None) == pkg.GCN_EINVAL
    assert L.gcn_decomp_line_starts_noalloc(fake, 100, None, 16, fake, None) == pkg.GCN_EINVAL


def test_header_comments_are_intact():
    """No line of the header starts with a stray quote (a '\\n' that became a
    real line break inside a comment)."""
    lines = open(os.path.join(ROOT, "include", "gcn_decomp.h")).read().split("\n")
    assert not [i for i, l in enumerate(lines, 1) if l.startswith("'")]
