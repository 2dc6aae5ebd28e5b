"""GPU parity on damaged input, through the C ABI, against the CPU oracle: generated files with
lines missing, repeated or swapped, misspelled mnemonics and operands, registers out of range,
undefined and doubled labels, bad configuration values, constant offsets, CRLF endings, comments
and truncation (tests/mutate.py).  Every byte of text, every status and every IR array must be
identical."""
import pytest

import gcngen
import mutate
import oracle
import paper_2107_07809_gb300 as pkg

pytestmark = pytest.mark.gpu


def _damaged(n, seed):
    texts = []
    for cfg in (0, 1, 2, 5, 6, 7, 8, 9):
        b = gcngen.generate(gcngen.preset(cfg, max_len=600), 40, seed=gcngen.SEED_BASE + 800 + cfg)
        texts += [b.kernel(i) for i in range(len(b))]
    return mutate.mutants(texts, n, seed)


def test_damaged_files_text_and_status():
    pkg.build()
    files = _damaged(1500, 21070)
    want = [oracle.decompile(f) for f in files]
    assert min(sum(1 for w in want if w.worst == s) for s in (0, 1, 2)) > 100
    with pkg.Decompiler(0) as dec:
        got = dec.decompile(files)
    for n, ((text, st), w) in enumerate(zip(got, want)):
        assert text == w.text, f"file {n}: OpenCL text differs"
        assert st == w.worst, f"file {n}: status {st} vs {w.worst}"


def test_damaged_files_ir_arrays():
    pkg.build()
    files = _damaged(300, 21071)
    with pkg.Decompiler(0) as dec:
        ids = dec.submit_batch(files)
        for n, (f, j) in enumerate(zip(files, ids)):
            want = oracle.decompile(f, with_ir=True)
            for which in range(6):
                exp = b"".join(k[which] for k in want.ir)
                assert dec.fetch_ir(j, which) == exp, f"file {n}: IR array {which} differs"
        dec.fetch_batch(ids)
