"""The job service (continuous batching) through the C ABI.

Requests that arrive while others run are batched with whatever else is queued
when a worker lane frees up; a request's result must be the same alone and in
any mix (byte-identical: the work is integer, byte and index work), and equal
to the oracle's."""
import threading
import time

import pytest

import gcngen
import oracle
import paper_2107_07809_gb300 as pkg

pytestmark = pytest.mark.gpu


def _requests(cfg, n, seed_off=0, **over):
    p = gcngen.preset(cfg, **over)
    b = gcngen.generate(p, n, seed=gcngen.SEED_BASE + cfg + seed_off)
    return [b.kernel(i) for i in range(n)]


@pytest.fixture(scope="module")
def reqs():
    # serving-style requests (lengths log-uniform, capped for test time) and batch-style ones
    return _requests(4, 24, max_len=6000) + _requests(1, 40)


def test_alone_equals_mix_equals_oracle(reqs):
    pkg.build()
    with pkg.Decompiler(0) as dec:
        alone = []
        for r in reqs:
            (ident,) = dec.submit_batch([r])
            alone.append(dec.fetch_opencl(ident))
        mixed = dec.decompile(reqs)
    assert mixed == alone
    for r, (text, st) in zip(reqs[::7], alone[::7]):
        want = oracle.decompile(r)
        assert text == want.text and st == want.worst


def test_concurrent_clients_and_staggered_arrivals(reqs):
    """Two client threads submit requests one by one with gaps, so batches form
    from whatever arrived; every result must equal the request alone."""
    pkg.build()
    with pkg.Decompiler(0) as dec:
        ref = dec.decompile(reqs)
        got = [None] * len(reqs)

        def client(idx):
            ids = []
            for i in idx:
                ids += [(i, j) for j in dec.submit_batch([reqs[i]])]
                time.sleep(0.002)
            for i, j in ids:
                got[i] = dec.fetch_opencl(j)

        th = [threading.Thread(target=client, args=(range(k, len(reqs), 2),)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    assert got == ref


def test_poll_job_info_and_resident_ir(reqs):
    pkg.build()
    with pkg.Decompiler(0) as dec:
        ids = dec.submit_batch(reqs[:10])
        seen = []
        deadline = time.time() + 60
        while len(seen) < len(ids) and time.time() < deadline:
            seen += dec.poll(timeout_ms=100)
        assert sorted(seen) == sorted(ids)
        for j in ids:
            info = dec.job_info(j)
            assert info["state"] == 2
            assert 0 < info["t_submit"] <= info["t_start"] <= info["t_done"]
        # the IR of the last batch is still on the device until its jobs are fetched
        want = oracle.decompile(reqs[9], with_ir=True)
        assert dec.fetch_ir(ids[9], pkg.IR_INSTR) == b"".join(k[pkg.IR_INSTR] for k in want.ir)
        texts, _ = dec.fetch_batch(ids)
        assert texts[3] == oracle.decompile(reqs[3]).text
        with pytest.raises(pkg.GcnDecompError) as e:
            dec.fetch_opencl(ids[0])
        assert e.value.rc == pkg.GCN_ENOJOB


def test_admission_under_memory_budget(reqs):
    """A small budget admits a prefix of the jobs; fetching frees budget for the rest."""
    pkg.build()
    sizes = [len(r) for r in reqs]
    budget = 48 * sum(sizes[:5]) + 5 * (1 << 20) + 4096
    with pkg.Decompiler(0, mem_budget_bytes=1 << 40) as ref_dec:
        ref = ref_dec.decompile(reqs[:12])
    with pkg.Decompiler(0, mem_budget_bytes=budget) as dec:
        ids = dec.submit_batch(reqs[:12])
        assert 1 <= len(ids) < 12
        out = dec.fetch_batch(ids)
        rest = dec.submit_batch(reqs[len(ids):12])
        assert len(rest) >= 1
        out2 = dec.fetch_batch(rest)
    got = list(zip(out[0], out[1])) + list(zip(out2[0], out2[1]))
    assert got == ref[: len(got)]


def test_tuning_file(reqs, tmp_path):
    """Runtime parameters from a tuning file: one lane taking 1 MiB batches splits the
    requests into many batches; the results do not change.  A malformed file is refused."""
    pkg.build()
    good = tmp_path / "t.tune"
    good.write_text("# test\nlanes=1\nbatch_mib=1\nbig_kernel=1024\n")
    bad = tmp_path / "bad.tune"
    bad.write_text("lanes=99\n")
    with pkg.Decompiler(0) as dec:
        ref = dec.decompile(reqs)
    with pkg.Decompiler(0, tuning_file=str(good)) as dec:
        assert dec.decompile(reqs) == ref
    with pytest.raises(pkg.GcnDecompError) as e:
        pkg.Decompiler(0, tuning_file=str(bad))
    assert e.value.rc == pkg.GCN_EINVAL


def test_packed_submit_and_raw_fetch(reqs):
    """Files submitted back to back from one buffer, and fetched as one buffer with numpy
    offsets, give the same texts and statuses as the per-file calls."""
    import numpy as np

    pkg.build()
    offs = np.zeros(len(reqs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reqs])
    packed = np.frombuffer(b"".join(reqs), dtype=np.uint8)
    with pkg.Decompiler(0) as dec:
        want = dec.decompile(reqs)
        ids = dec.submit_packed(packed, offs)
        raw, o, st = dec.fetch_batch_raw(ids)
    got = [(raw[o[i]:o[i + 1]].tobytes().decode(), int(st[i])) for i in range(len(reqs))]
    assert got == want
