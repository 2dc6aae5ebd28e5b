"""GPU parity: the CUDA decompiler, called through the C ABI, against the CPU oracle.

Integer, byte and index work: every compared array and every byte of text must
be identical."""
import numpy as np
import pytest

import gcngen
import oracle
import paper_2107_07809_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dec():
    pkg.build()
    d = pkg.Decompiler(0)
    yield d
    d.close()


def _files(cfg, n, **over):
    p = gcngen.preset(cfg, **over)
    b = gcngen.generate(p, n, seed=gcngen.SEED_BASE + cfg)
    return [b.kernel(i) for i in range(n)]


def _check_ir(dec, files):
    ids = dec.submit_batch(files)
    assert len(ids) == len(files)
    for f, j in zip(files, ids):
        want = oracle.decompile(f, with_ir=True)
        for which in range(6):
            got = dec.fetch_ir(j, which)
            exp = b"".join(k[which] for k in want.ir)
            assert got == exp, f"IR array {which} differs"
        dec.fetch_opencl(j)


def test_ir_parity_small(dec):
    _check_ir(dec, _files(0, 1))


def test_ir_parity_config1_sample(dec):
    _check_ir(dec, _files(1, 300))


def test_ir_parity_multi_kernel_files(dec):
    ks = _files(1, 12, max_len=400)
    files = [b"".join(ks[0:4]), b"leading junk\n" + b"".join(ks[4:9]), ks[9], b"", b"".join(ks[10:12])]
    _check_ir(dec, files)


def test_ir_parity_golden_fixtures(dec):
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    files = [open(os.path.join(g, f), "rb").read() for f in sorted(os.listdir(g)) if f.endswith(".s")]
    _check_ir(dec, files)
