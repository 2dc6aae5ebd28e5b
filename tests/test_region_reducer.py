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


# ---- early exits: the linear-time finder against the rule written out ----------------------
def _breaks_definition(s0, s1, live):
    """The rule as stated: a two-way block b that is not a latch breaks out of the loop that holds
    it (the first latch l after b whose header is at or before b) when one successor is that
    loop's exit and the other stays in [header, l]; a latch with such a block is marked."""
    n = len(s0)
    cond = [s0[i] >= 0 and s1[i] >= 0 for i in range(n)]

    def header(l):
        if not cond[l] or (s0[l] <= l) == (s1[l] <= l):
            return None
        return s0[l] if s0[l] <= l else s1[l]

    brk = [-1] * n
    for b in range(n):
        if not live[b] or not cond[b] or header(b) is not None:
            continue
        for l in range(b + 1, n):
            h = header(l)
            if h is None or h > b:
                continue
            e = s1[l] if s0[l] == h else s0[l]
            if (s0[b] == e) != (s1[b] == e):
                x = s1[b] if s0[b] == e else s0[b]
                if h <= x <= l:
                    brk[b] = l
            break
    for b in range(n):
        if brk[b] >= 0:
            brk[brk[b]] = -2
    return brk


def test_find_breaks_equals_the_forward_search(tmp_path):
    if not shutil.which("nvcc"):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "breaks_host")
    subprocess.check_call(["nvcc", "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu",
                           os.path.join(HERE, "breaks_host.cu"), "-o", exe])
    rng = random.Random(2107)
    graphs = []
    for g in range(400):
        n = rng.randint(1, 70)
        s0, s1, live = [], [], []
        for b in range(n):
            def target():
                r = rng.random()
                if r < 0.35:
                    return b + 1 if b + 1 < n else -1
                if r < 0.6:
                    return rng.randint(0, b)  # at or before: a back edge
                return rng.randint(b, n - 1) if b < n - 1 else -1
            a, c = target(), (target() if rng.random() < 0.7 else -1)
            if a == c:
                c = -1
            s0.append(a)
            s1.append(c)
            live.append(1 if rng.random() < 0.9 else 0)
        graphs.append((s0, s1, live))
    text = [str(len(graphs))]
    for s0, s1, live in graphs:
        text.append(str(len(s0)))
        text += [f"{a} {c} {l}" for a, c, l in zip(s0, s1, live)]
    out = subprocess.run([exe], input="\n".join(text) + "\n", capture_output=True, text=True, check=True).stdout
    lines = out.strip().split("\n")
    assert len(lines) == len(graphs)
    breaks = 0
    for (s0, s1, live), line in zip(graphs, lines):
        got = [int(x) for x in line.split()]
        want = _breaks_definition(s0, s1, live)
        assert got == want
        breaks += sum(1 for x in want if x >= 0)
    assert breaks > 50  # the graphs do exercise the rule
