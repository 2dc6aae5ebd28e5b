"""gcn_decomp_line_starts_noalloc (static scratch, no allocation) against the
batch pipeline's own newline scan, through the C ABI.

The batch entry point (gcn_decomp_run_device) reports the number of rows it
tokenised in gcn_decomp_run_stats; the no-allocation call must report the same
count, and its line starts must be the offsets just past every '\\n'.  Two calls
in a row must both agree (the static scratch is cleared by each call)."""
import ctypes

import numpy as np
import pytest

import gcngen
import paper_2107_07809_gb300 as pkg

pytestmark = pytest.mark.gpu


def _text(n):
    p = gcngen.preset(1)
    b = gcngen.generate(p, n, seed=gcngen.SEED_BASE + 1)
    return b.text, b.offsets


def _expected_starts(host: np.ndarray) -> np.ndarray:
    nl = np.flatnonzero(host == 0x0A).astype(np.uint64) + 1
    return np.concatenate([np.zeros(1, np.uint64), nl]).astype(np.uint32)


def _call(torch, d_text_ptr, n, cap, sentinel=0xDEADBEEF):
    starts = torch.from_numpy(np.full(cap, sentinel, np.uint32).view(np.int32)).cuda()
    res = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pkg.line_starts_noalloc(d_text_ptr, n, starts.data_ptr(), cap, res.data_ptr(), stream)
    torch.cuda.synchronize()
    return starts.cpu().numpy().view(np.uint32), res.cpu().numpy().view(np.uint32)


def test_noalloc_matches_batch_entry_point_twice():
    torch = pytest.importorskip("torch")
    pkg.build()
    text, offs = _text(60)
    host = np.frombuffer(text, dtype=np.uint8)
    d_text = torch.from_numpy(host.copy()).cuda()
    d_off = torch.from_numpy(np.asarray(offs, dtype=np.uint64).view(np.int64)).cuda()
    with pkg.Decompiler(0) as dec:
        dec.run_device(d_text.data_ptr(), host.size, d_off.data_ptr(), len(offs) - 1,
                       torch.cuda.current_stream().cuda_stream)
        dec.result_device()
        lines = dec.run_stats()["lines"]
    want = _expected_starts(host)
    assert lines == want.size - 1
    for _ in range(2):
        starts, res = _call(torch, d_text.data_ptr(), host.size, want.size + 5)
        assert res[1] == 0, f"error bits {res[1]}"
        assert res[0] == lines
        assert np.array_equal(starts[: want.size], want)
        assert np.all(starts[want.size:] == 0xDEADBEEF)


def test_noalloc_unaligned_text_and_ragged_tail():
    torch = pytest.importorskip("torch")
    pkg.build()
    text, _ = _text(7)
    host = np.frombuffer(text, dtype=np.uint8)
    buf = torch.from_numpy(np.concatenate([np.zeros(3, np.uint8), host])).cuda()
    n = host.size - 11  # ends in the middle of a line
    want = _expected_starts(host[:n])
    for _ in range(2):
        starts, res = _call(torch, buf.data_ptr() + 3, n, want.size)
        assert res[1] == 0 and res[0] == want.size - 1
        assert np.array_equal(starts, want)


def test_noalloc_capacity_and_limits():
    torch = pytest.importorskip("torch")
    pkg.build()
    text, _ = _text(5)
    host = np.frombuffer(text, dtype=np.uint8)
    d_text = torch.from_numpy(host.copy()).cuda()
    want = _expected_starts(host)
    cap = want.size // 2
    starts, res = _call(torch, d_text.data_ptr(), host.size, cap)
    assert res[0] == want.size - 1
    assert res[1] == 4  # capacity too small: reported, nothing written past cap
    assert np.array_equal(starts, want[:cap])
    # empty text: one line start, no newline
    starts, res = _call(torch, d_text.data_ptr(), 0, 1)
    assert res[0] == 0 and res[1] == 0 and starts[0] == 0
    # rejected on the host before any work is queued
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.GcnDecompError) as e:
        pkg.line_starts_noalloc(d_text.data_ptr(), (1 << 30) + 1, dummy.data_ptr(), 4, dummy.data_ptr())
    assert e.value.rc == pkg.GCN_ENOMEM
    with pytest.raises(pkg.GcnDecompError) as e:
        pkg.line_starts_noalloc(d_text.data_ptr(), host.size, dummy.data_ptr(), 0, dummy.data_ptr())
    assert e.value.rc == pkg.GCN_EINVAL
