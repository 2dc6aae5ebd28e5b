"""Failure paths of the job service, made to happen on the host or by a bound on the device:
no test faults, traps or hangs the GPU.

* A fixed-point sweep limit (the tuning file's fixpoint_sweeps test hook, with the same limit in
  the oracle) caps the kernels that still change in their last sweep: those, and only those,
  get status 3 and the oracle's not-decompiled text; the others of the same batch are
  byte-identical to the oracle.
* A forced allocation failure (the fail_alloc_jobs test hook: every workspace request of a batch
  of more jobs than the limit fails as cudaMalloc would) drives a lane through freeing idle
  memory, retrying and splitting its batch; every job still comes back equal to the oracle.
* Three lanes under a tight memory budget never hold more workspace than the budget.
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(__file__))

import gcngen  # noqa: E402
import oracle  # noqa: E402
import paper_2107_07809_gb300 as pkg  # noqa: E402
from test_oracle import NO_OPERAND_TYPED, gold  # noqa: E402

pytestmark = pytest.mark.gpu


def _oracle_at(limit, texts):
    oracle.set_type_sweep_limit(limit)
    try:
        return [oracle.decompile(t) for t in texts]
    finally:
        oracle.set_type_sweep_limit(0)


def test_sweep_limit_caps_only_the_kernels_that_still_change(tmp_path):
    pkg.build()
    b = gcngen.generate(1, 24, seed=gcngen.SEED_BASE + 77)
    loops = gcngen.generate(gcngen.preset(1, w_if=0, w_ifelse=0, w_loop=1), 8, seed=gcngen.SEED_BASE + 78)
    texts = [b.kernel(i) for i in range(24)] + [loops.kernel(i) for i in range(8)]
    texts += [NO_OPERAND_TYPED.encode(), gold("listing3_copy.s").encode()]
    texts += [NO_OPERAND_TYPED.encode() + b.kernel(0)]  # a file with a capped and an uncapped kernel
    tune = tmp_path / "cap.tune"
    tune.write_text("fixpoint_sweeps=1\n")
    want = _oracle_at(1, texts)
    with pkg.Decompiler(0, tuning_file=str(tune)) as dec:
        got = dec.decompile(texts)
    statuses = [s for _, s in got]
    assert 3 in statuses and 0 in statuses
    for (text, st), w in zip(got, want):
        assert text == w.text and st == w.worst
    # without the hook nothing is capped, and the uncapped kernels print as before
    with pkg.Decompiler(0) as dec:
        free = dec.decompile(texts)
    assert all(s != 3 for _, s in free)
    for (text, st), (ct, cs) in zip(free, got):
        if cs != 3:
            assert (text, st) == (ct, cs)


def test_forced_allocation_failure_splits_the_batch(tmp_path):
    pkg.build()
    b = gcngen.generate(gcngen.preset(1, max_len=400), 48, seed=gcngen.SEED_BASE + 79)
    texts = [b.kernel(i) for i in range(48)]
    tune = tmp_path / "fail.tune"
    tune.write_text("lanes=1\nfail_alloc_jobs=5\n")
    with pkg.Decompiler(0, tuning_file=str(tune)) as dec:
        got = dec.decompile(texts)  # one submit: the lane takes all 48 jobs as one batch
        splits = dec.run_stats()["splits"]
    assert splits >= 1
    for (text, st), t in zip(got, texts):
        w = oracle.decompile(t)
        assert text == w.text and st == w.worst


def test_three_lanes_stay_within_a_tight_budget(tmp_path):
    pkg.build()
    b = gcngen.generate(gcngen.preset(4, max_len=8000), 120, seed=gcngen.SEED_BASE + 80)
    texts = [b.kernel(i) for i in range(120)]
    budget = 192 << 20
    tune = tmp_path / "lanes.tune"
    tune.write_text("lanes=3\nbatch_mib=1\n")
    with pkg.Decompiler(0, tuning_file=str(tune)) as dec:
        ref = dec.decompile(texts)
    with pkg.Decompiler(0, mem_budget_bytes=budget, tuning_file=str(tune)) as dec:
        got, pending, i = [], [], 0
        while i < len(texts) or pending:
            if i < len(texts):
                try:
                    ids = dec.submit_batch(texts[i:i + 16])
                except pkg.GcnDecompError as e:  # nothing admitted: fetch first
                    if e.rc != pkg.GCN_EAGAIN:
                        raise
                    ids = []
                pending += ids
                i += len(ids)
            if pending:
                take, pending = pending[:8], pending[8:]
                got += list(zip(*dec.fetch_batch(take)))
        peak = dec.run_stats()["peak_device_bytes"]
    assert got == ref
    assert 0 < peak <= budget
