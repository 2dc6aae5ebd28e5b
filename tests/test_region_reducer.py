"""The CUDA path's region reducer (incremental restart search, S12), compiled
for the host, against the oracle's structural analysis on seeded random graphs:
structured programs (nested sequences, ifs, if-elses, do-while loops) and
arbitrary graphs (irreducible ones included).  The merge sequences, and so the
region trees, must be identical."""
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _reduce_oracle(s0, s1):
    n = len(s0)
    a = np.asarray(s0, dtype=np.int32)
    b = np.asarray(s1, dtype=np.int32)
    out = np.zeros(64 * n + 64, dtype=np.int32)
    w = oracle.lib().oracle_reduce_graph(n, a.ctypes.data, b.ctypes.data, out.ctypes.data, len(out))
    assert w != -2
    if w < 0:
        return None
    log, i = [], 0
    while i < w:
        nid, cnt = int(out[i]), int(out[i + 1])
        log.append((nid, [int(x) for x in out[i + 2:i + 2 + cnt]]))
        i += 2 + cnt
    return log


def _structured(rng, depth, budget):
    blocks = []

    def new():
        blocks.append([-1, -1])
        return len(blocks) - 1

    def link(x, tgt):
        if isinstance(x, tuple):
            blocks[x[1]][1] = tgt
        elif blocks[x][0] == -1:
            blocks[x][0] = tgt
        elif blocks[x][1] == -1:
            blocks[x][1] = tgt

    def stmt(d):
        r = rng.random()
        if d <= 0 or len(blocks) > budget or r < 0.3:
            b = new()
            return b, [b]
        if r < 0.5:  # sequence
            e1, x1 = stmt(d - 1)
            e2, x2 = stmt(d - 1)
            for x in x1:
                link(x, e2)
            return e1, x2
        if r < 0.7:  # if: header falls into the then part, branches to the join
            h = new()
            et, xt = stmt(d - 1)
            blocks[h][0] = et
            return h, xt + [("taken", h)]
        if r < 0.85:  # if-else, the then part jumps over the else part
            h = new()
            et, xt = stmt(d - 1)
            j = new()
            ee, xe = stmt(d - 1)
            blocks[h][0], blocks[h][1] = et, ee
            for x in xt:
                link(x, j)
            return h, xe + [j]
        eb, xb = stmt(d - 1)  # do-while: the latch branches back to the body
        latch = new()
        for x in xb:
            link(x, latch)
        blocks[latch][1] = eb
        return eb, [latch]

    e, xs = stmt(depth)
    end = new()
    for x in xs:
        link(x, end)
    n = len(blocks)
    perm = list(range(n))
    perm[0], perm[e] = perm[e], perm[0]
    inv = {perm[i]: i for i in range(n)}
    s0, s1 = [0] * n, [0] * n
    for old in range(n):
        a, b = blocks[old]
        s0[inv[old]] = inv[a] if a >= 0 else -1
        s1[inv[old]] = inv[b] if b >= 0 else -1
    return s0, s1


def _arbitrary(rng, n):
    s0, s1 = [], []
    for _ in range(n):
        r = rng.random()
        if r < 0.15:
            s0.append(-1)
            s1.append(-1)
        elif r < 0.6:
            s0.append(rng.randrange(n))
            s1.append(-1)
        else:
            s0.append(rng.randrange(n))
            s1.append(rng.randrange(n))
    return s0, s1


@pytest.fixture(scope="module")
def reducer(tmp_path_factory):
    if not shutil.which("nvcc"):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("red") / "region_host")
    subprocess.check_call(["nvcc", "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu",
                           os.path.join(HERE, "region_host.cu"), "-o", exe])
    return exe


def test_incremental_reducer_equals_restarting_search(reducer):
    rng = random.Random(2107078090)
    graphs = []
    for _ in range(1500):
        k = rng.random()
        if k < 0.6:
            graphs.append(_structured(rng, rng.randrange(1, 8), rng.randrange(5, 400)))
        elif k < 0.8:
            graphs.append(_arbitrary(rng, rng.randrange(1, 12)))
        else:
            graphs.append(_arbitrary(rng, rng.randrange(12, 80)))
    lines = [str(len(graphs))]
    for s0, s1 in graphs:
        lines.append(str(len(s0)))
        lines += [f"{a} {b}" for a, b in zip(s0, s1)]
    out = subprocess.run([reducer], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.splitlines()
    assert len(out) == len(graphs)
    reducible = 0
    for g, (s0, s1) in enumerate(graphs):
        parts = out[g].split("|")
        root = int(parts[0].split()[2])
        assert root != -2, f"graph {g}: work arrays overflowed"
        got = []
        for p in parts[1:]:
            xs = [int(x) for x in p.split()]
            got.append((xs[0], xs[1:]))
        want = _reduce_oracle(s0, s1)
        if want is None:
            assert root == -1, f"graph {g}: the oracle does not reduce it"
        else:
            reducible += 1
            assert root >= 0 and got == want, f"graph {g}: merge sequences differ"
    assert reducible > 500
