"""Autotuner for the runtime parameters of a decompiler handle on this GPU.

Measures, on seeded synthetic batches:
  * lanes x batch_mib: end-to-end time of a stream of 200,000 kernels of the large batch (lengths
    50..2000) through the job service, the way a client streams work: pieces of 8,192 kernels
    submitted while at most six pieces are unfetched, a second thread fetching each piece (a
    shorter stream ranks the configurations by its start-up and tail);
  * lanes x batch_mib for serving: end-to-end time of one burst of 10,000 kernels (lengths
    50..2000) submitted at once and fetched (a service under a device-memory budget that answers
    requests as they come wants fewer lanes and smaller batches than a sustained stream: with
    eight lanes of 256 MiB batches, the 20 GB serving budget runs out, and admissions wait);
  * big_kernel: device time of a 10,000-kernel batch plus a batch of serving-size kernels (lengths
    100..50,000), the size from which reachability and type inference give a kernel a whole
    thread block;
and writes the best values as two tuning files (`key=value` lines, the measurements as
comments) that `Decompiler(tuning_file=...)` / `gcn_decomp_config.tuning_file` read: one for
throughput, one for serving.

    python -m paper_2107_07809_gb300.autotune --out paper_2107_07809_gb300/tuning/gb300.tune \
        --out-serve paper_2107_07809_gb300/tuning/gb300_serve.tune
"""
from __future__ import annotations

import argparse
import datetime
import os
import queue
import statistics
import sys
import tempfile
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(_HERE))

import gcngen  # noqa: E402
import paper_2107_07809_gb300 as pkg  # noqa: E402


def _write(path, lanes, batch_mib, big_kernel, notes=()):
    with open(path, "w") as f:
        for line in notes:
            f.write(f"# {line}\n")
        f.write(f"lanes={lanes}\nbatch_mib={batch_mib}\nbig_kernel={big_kernel}\n")


def _stream_once(dec, batch, piece=8192, window=6):
    q = queue.Queue(maxsize=window)
    err = []

    def fetcher():
        try:
            while (ids := q.get()) is not None:
                dec.fetch_batch_raw(ids)
        except Exception as e:  # noqa: BLE001 - reported below
            err.append(e)

    th = threading.Thread(target=fetcher)
    t0 = time.perf_counter()
    th.start()
    n = len(batch)
    for p0 in range(0, n, piece):
        p1 = min(p0 + piece, n)
        ids = []
        while len(ids) < p1 - p0:
            got = dec.submit_packed(batch.text, batch.offsets[p0 + len(ids):p1 + 1])
            if not got:
                time.sleep(0.0005)
            ids += got
        q.put(ids)
    q.put(None)
    th.join()
    if err:
        raise err[0]
    return (time.perf_counter() - t0) * 1e3


def _e2e_ms(batch, tune, reps):
    with pkg.Decompiler(0, tuning_file=tune) as dec:
        _stream_once(dec, batch)  # warm-up: workspaces and pinned buffers grow once
        return statistics.median(_stream_once(dec, batch) for _ in range(reps))


def _burst_ms(files, tune, reps):
    with pkg.Decompiler(0, mem_budget_bytes=20 << 30, tuning_file=tune) as dec:
        ids = dec.submit_batch(files)  # warm-up: workspaces and pinned buffers grow once
        dec.fetch_batch_raw(ids)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            ids = dec.submit_batch(files)
            dec.fetch_batch_raw(ids)
            ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts)


def _device_ms(batch, tune, reps):
    import torch

    d_text = torch.from_numpy(batch.text).cuda()
    d_off = torch.from_numpy(batch.offsets.view(np.int64)).cuda()
    with pkg.Decompiler(0, tuning_file=tune) as dec:
        ts = []
        for it in range(reps + 1):
            dec.run_device(d_text.data_ptr(), int(batch.text.nbytes), d_off.data_ptr(), len(batch), 0)
            dec.result_device()
            if it:
                ts.append(sum(v for k, v in dec.stage_times().items() if k.startswith("S")))
    return statistics.median(ts)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(_HERE, "tuning", "gb300.tune"))
    ap.add_argument("--out-serve", default=os.path.join(_HERE, "tuning", "gb300_serve.tune"))
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    pkg.build()
    tmp = tempfile.mkdtemp()
    tune = os.path.join(tmp, "t.tune")

    b1 = gcngen.generate(gcngen.preset(1), 10_000, seed=gcngen.SEED_BASE + 1)
    b2 = gcngen.generate(gcngen.preset(2), 200_000, seed=gcngen.SEED_BASE + 2)
    table = []
    for lanes in (3, 4, 6, 8):
        for mib in (64, 128, 256):
            _write(tune, lanes, mib, 4096)
            ms = _e2e_ms(b2, tune, args.reps)
            table.append((ms, lanes, mib))
            print(f"lanes={lanes} batch_mib={mib}: {ms:.1f} ms", flush=True)
    best_ms, lanes, mib = min(table)

    files = [b1.kernel(i) for i in range(len(b1))]
    serve_table = []
    for s_lanes in (1, 2, 3, 4):
        for s_mib in (32, 64, 128, 256):
            _write(tune, s_lanes, s_mib, 4096)
            ms = _burst_ms(files, tune, args.reps)
            serve_table.append((ms, s_lanes, s_mib))
            print(f"serving: lanes={s_lanes} batch_mib={s_mib}: {ms:.1f} ms", flush=True)
    serve_ms, s_lanes, s_mib = min(serve_table)

    # the threshold serves both workloads: the objective is the sum of the device
    # times of the 10,000-kernel batch and of 100 serving-size kernels
    b4 = gcngen.generate(gcngen.preset(4), 100, seed=gcngen.SEED_BASE + 4)
    big_table = []
    for big in (1024, 2048, 4096, 8192, 16384):
        _write(tune, lanes, mib, big)
        m1 = _device_ms(b1, tune, args.reps)
        m4 = _device_ms(b4, tune, args.reps)
        big_table.append((m1 + m4, big, m1, m4))
        print(f"big_kernel={big}: batch {m1:.2f} ms + serving {m4:.2f} ms", flush=True)
    big_ms, big, _, _ = min(big_table)

    import torch

    notes = [f"written by paper_2107_07809_gb300/autotune.py on {torch.cuda.get_device_name(0)}, "
             f"{datetime.date.today().isoformat()}",
             f"e2e of a stream of 200,000 kernels ({int(b2.total_instr)} instrs), median of {args.reps} (ms):"]
    notes += [f"  lanes={l} batch_mib={m}: {t:.1f}" for t, l, m in sorted(table, key=lambda x: (x[1], x[2]))]
    notes += [f"device time (ms) of the 10,000-kernel batch + 100 serving-size kernels "
              f"({int(b4.total_instr)} instrs), medians:"]
    notes += [f"  big_kernel={g}: {a:.2f} + {c:.2f} = {t:.2f}" for t, g, a, c in sorted(big_table, key=lambda x: x[1])]
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    _write(args.out, lanes, mib, big, notes)
    s_notes = [notes[0], f"serving: e2e of a burst of 10,000 kernels ({int(b1.total_instr)} instrs) under a 20 GB "
                         f"budget, median of {args.reps} (ms):"]
    s_notes += [f"  lanes={l} batch_mib={m}: {t:.1f}" for t, l, m in sorted(serve_table, key=lambda x: (x[1], x[2]))]
    s_notes += ["big_kernel as for throughput (device time, see gb300.tune)"]
    _write(args.out_serve, s_lanes, s_mib, big, s_notes)
    print(f"best: lanes={lanes} batch_mib={mib} ({best_ms:.1f} ms), big_kernel={big} ({big_ms:.2f} ms) -> {args.out}; "
          f"serving lanes={s_lanes} batch_mib={s_mib} ({serve_ms:.1f} ms) -> {args.out_serve}")


if __name__ == "__main__":
    main()
