"""GPU parity at full size, through the C ABI, against the oracle run in parallel on the
host cores: every one of the 64 large-CFG kernels (200,000 instructions each; text and
IR arrays), every request of the serving pool (1,000 requests of 100..50,000
instructions, through the job service), and a sample spread over the whole
1,000,000-kernel stream (100 runs of 100 consecutive kernels, one every 10,000).
Integer, byte and index work: every byte must be identical."""
import os

import numpy as np
import pytest

import gcngen
import oracle
import paper_2107_07809_gb300 as pkg

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


def _oracle_texts(batch):
    out, oo, st = oracle.decompile_batch(batch.text, batch.offsets, THREADS)
    raw = out.tobytes()
    return [raw[oo[i]:oo[i + 1]] for i in range(len(oo) - 1)], [int(x) for x in st]


def _device_texts(batch):
    import torch

    d_text = torch.from_numpy(batch.text).cuda()
    d_off = torch.from_numpy(batch.offsets.view(np.int64)).cuda()
    with pkg.Decompiler(0) as dec:
        dec.run_device(d_text.data_ptr(), int(batch.text.nbytes), d_off.data_ptr(), len(batch), 0)
        dec.result_device()
        texts, st = dec.result_copy(0, len(batch))
    return [t.encode() for t in texts], st


class _Joined:
    """Several generated batches as one batch (text and file offsets)."""

    def __init__(self, batches):
        self.text = np.concatenate([b.text for b in batches])
        offs = [0]
        for b in batches:
            base = offs[-1]
            offs += [base + int(x) for x in b.offsets[1:]]
        self.offsets = np.asarray(offs, dtype=np.uint64)

    def __len__(self):
        return len(self.offsets) - 1


def _mismatches(a, b):
    return [i for i, (x, y) in enumerate(zip(a, b)) if x != y]


def test_large_cfg_all_64_kernels_text_and_ir():
    pkg.build()
    b = gcngen.generate(gcngen.preset(3), 64, seed=gcngen.SEED_BASE + 3, threads=THREADS)
    want, wst = _oracle_texts(b)
    got, gst = _device_texts(b)
    assert _mismatches(got, want) == [] and gst == wst
    files = [b.kernel(i) for i in range(len(b))]
    with pkg.Decompiler(0) as dec:
        ids = dec.submit_batch(files)
        for f, j in list(zip(files, ids))[:16]:
            ir = oracle.decompile(f, with_ir=True).ir
            for which in range(6):
                assert dec.fetch_ir(j, which) == b"".join(k[which] for k in ir), f"IR array {which}"
        dec.fetch_batch(ids)


def test_serving_pool_all_1000_requests_through_the_job_service():
    pkg.build()
    b = gcngen.generate(gcngen.preset(4), 1000, seed=gcngen.SEED_BASE + 4, threads=THREADS)
    want, wst = _oracle_texts(b)
    with pkg.Decompiler(0, mem_budget_bytes=20 << 30) as dec:
        files = [b.kernel(i) for i in range(len(b))]
        got, gst = [], []
        pos = 0
        while pos < len(files):  # the budget may admit a prefix at a time
            ids = dec.submit_batch(files[pos:])
            texts, st = dec.fetch_batch(ids)
            got += [t.encode() for t in texts]
            gst += st
            pos += len(ids)
    assert _mismatches(got, want) == [] and gst == wst


def test_million_kernel_stream_spread_sample():
    pkg.build()
    p = gcngen.preset(2)
    runs = [gcngen.generate(p, 100, seed=gcngen.SEED_BASE + 2, first=10_000 * c, threads=THREADS) for c in range(100)]
    v = _Joined(runs)
    want, wst = _oracle_texts(v)
    got, gst = _device_texts(v)
    assert len(got) == 10_000
    assert _mismatches(got, want) == [] and gst == wst


def test_million_kernel_stream_every_kernel():
    """Every one of the 1,000,000 kernels of the large-batch stream (5.46e8 instructions), in ten
    chunks of 100,000 through the job service (packed submit, raw fetch), against the oracle in
    parallel on the host cores: each chunk's whole output, its offsets and its statuses must be
    identical."""
    pkg.build()
    p = gcngen.preset(2)
    chunk = 100_000
    with pkg.Decompiler(0, max_slots=chunk + 1024) as dec:  # a chunk's jobs all admitted at once
        for c0 in range(0, 1_000_000, chunk):
            b = gcngen.generate(p, chunk, seed=gcngen.SEED_BASE + 2, first=c0, threads=THREADS)
            ids = dec.submit_packed(b.text, b.offsets)
            assert len(ids) == chunk
            want, woff, wst = oracle.decompile_batch(b.text, b.offsets, THREADS)  # while the GPU runs
            raw, off, st = dec.fetch_batch_raw(ids)
            assert len(off) == chunk + 1, f"chunk at {c0}"
            assert np.array_equal(np.asarray(st, dtype=np.int64), np.asarray(wst, dtype=np.int64)), f"statuses, chunk at {c0}"
            assert np.array_equal(np.asarray(off, dtype=np.uint64), np.asarray(woff, dtype=np.uint64)), f"offsets, chunk at {c0}"
            assert np.array_equal(raw[: int(off[-1])], want[: int(woff[-1])]), f"text, chunk at {c0}"
