#!/usr/bin/env python3
"""Throughput benchmark: GCN instructions decompiled per second on GB300.

Default workload: the large batch, 1,000,000 seeded synthetic kernels with
log-uniform lengths 50..2000 (about 5.46e8 instructions and 20 GB of text),
decompiled in chunks of 100,000 kernels, one pipeline pass (every stage
S1..S13 of the method) per chunk.  One step is one pass over all chunks.

* ``value``: instructions per second with every chunk's text already in HBM
  when the timed region starts (gcn_decomp_run_device), timed with CUDA events;
  the chunks are spread over several handles, each with its own stream and
  host thread, so that the passes of different chunks overlap on the device.
* ``e2e``: the same stream through the job service's host-buffer entry points
  (gcn_decomp_submit_batch with the packed texts of each piece, then
  gcn_decomp_fetch_batch), host->device and device->host copies inside the
  timed region; the service's worker lanes overlap the copies of one batch
  with the passes of others.
* ``roofline``: the longest kernel of a pass, timed alone (one pass over all
  chunks on one stream) by the library's CUDA events around that kernel.
* extras: the 10,000-kernel batch in one pass (``batch``), the plain form, one
  pipeline run per kernel (``per_kernel``), the large-CFG workload
  (``large_cfg``), and the job service under open-loop Poisson arrivals at 1k,
  10k and 100k requests/s (``serve``, p50/p99 latency).

--impl reference times the CPU oracle (single-threaded) on bounded samples of
the same workload, the comparison arm.  Multi-GPU (torchrun): every rank
decompiles its own slice of the stream (weak scaling); there is no collective.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# runtime parameters picked by paper_2107_07809_gb300/autotune.py on a GB300 (if present)
TUNING = os.path.join(ROOT, "paper_2107_07809_gb300", "tuning", "gb300.tune")
# the job service under a memory budget and latency targets takes its own tuning (fewer lanes,
# smaller batches): the autotuner writes both files
TUNING_SERVE = os.path.join(ROOT, "paper_2107_07809_gb300", "tuning", "gb300_serve.tune")

import gcngen  # noqa: E402

WORKLOADS = {
    # name: (preset, kernels)
    "config1": (1, 10_000),
    "config2": (2, 1_000_000),  # streamed in chunks
    "config3": (3, 64),
    "select": (5, 10_000),  # the batch mix with ternaries (v_cndmask_b32)
    "sysval": (6, 10_000),  # the batch mix with dispatch-packet system values and scalar bit fields
    "flatmulhi": (7, 10_000),  # the batch mix with FLAT accesses and double-suffix high multiplies
    "mixed": (8, 10_000),  # mixed uniform/divergent nesting, loops with early exits
    "lds": (9, 10_000),  # 1-D kernels exchanging values through a __local buffer around a barrier
    "serving": (4, 1_000),  # the serving length mix (100..50,000 instructions) as one batch
}
METRIC = "GCN instrs decompiled/sec"
# the library's event timing of single kernels (gcn_decomp_stage_times names)
# DRAM bytes (read + write) per instruction of one k_items launch: ncu on the first 4,000 kernels of
# the batch distribution (the k_items capture under profiles/: 814.1 MB over 2,201,608 instructions);
# it holds for the code captured there, and is scaled by the instructions of a launch
K_ITEMS_DRAM_PER_INSTR = (573.546240e6 + 240.553216e6) / 2_201_608
KERNEL_TIMINGS = ("k_line_scan (S1)", "k_decode (S4)", "k_nodes (S7)", "k_node_fwd (S9-S10)",
                  "k_node_cache (S9-S10)", "k_items (S13 print)")


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_first(rank, per_rank):
    """First kernel of a rank's slice of the seeded stream: every rank decompiles its own
    `per_rank` consecutive kernels (weak scaling), so the slices are disjoint and together are
    the first world * per_rank kernels of the stream."""
    return rank * per_rank


def max_over_ranks(torch, value, device):
    """The largest of every rank's value (the job's time is its slowest rank's); the value
    itself with one rank.  The only collective of the benchmark: there is no data exchange."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def tuning_file(serve=False):
    t = TUNING_SERVE if serve else TUNING
    return t if os.path.exists(t) else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name, rank, kernels=None):
    cfg, n = WORKLOADS[name]
    if kernels:
        n = kernels
    params = gcngen.preset(cfg)
    batch = gcngen.generate(params, n, seed=gcngen.SEED_BASE + cfg, first=rank_first(rank, n),
                            threads=os.cpu_count() or 4)
    return cfg, batch


def oracle_rate(batch, budget_s, start=0):
    """Single-threaded oracle over consecutive kernels until `budget_s` elapses."""
    import oracle

    done_instr, t0, k = 0, time.perf_counter(), start
    n = len(batch)
    while time.perf_counter() - t0 < budget_s and k < start + n:
        hi = min(k + 50, start + n)
        lo_, hi_ = k % n, (hi - 1) % n + 1
        oracle.decompile_batch(batch.text, batch.offsets[lo_:hi_ + 1] if hi_ > lo_ else batch.offsets[lo_:lo_ + 2], 1)
        done_instr += int(batch.ninstr[lo_:hi_].sum())
        k = hi
    dt = time.perf_counter() - t0
    return done_instr / dt, done_instr, k - start, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # a prefix of the same seeded stream: the oracle never gets past it within the bounded sample
    name = args.workload
    cfg, total = WORKLOADS[name]
    cfg, batch = make_workload(name, 0, min(args.kernels or total, 20_000))
    per_step = 6.0
    for _ in range(args.warmup):
        oracle_rate(batch, 1.0)
    rates, instrs, kern = [], 0, 0
    pos = 0
    for _ in range(args.steps):
        r, ni, nk, dt = oracle_rate(batch, per_step, start=pos)
        pos = (pos + nk) % len(batch)
        rates.append(r)
        instrs += ni
        kern += nk
    value = float(statistics.mean(rates))
    sample = (f"{kern} kernels ({instrs} instrs) of the first {len(batch)} kernels of the stream, over "
              f"{args.steps} steps of ~{per_step:.0f} s, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "instr/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{name}: {total} seeded synthetic kernels (preset {cfg})"},
        "cpu_baseline": {"value": value, "unit": "instr/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "instr/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def per_kernel_form(pkg, torch, batch, local, n_sample):
    """The plain form: one pipeline run (one launch sequence) per kernel, its
    text already in HBM; each kernel's text starts 256-byte aligned."""
    n = min(n_sample, len(batch))
    offs = batch.offsets.astype(np.int64)
    sizes = offs[1:n + 1] - offs[:n]
    starts = np.zeros(n + 1, np.int64)
    starts[1:] = np.cumsum((sizes + 255) // 256 * 256)
    host = np.zeros(int(starts[-1]) + 256, np.uint8)
    for i in range(n):
        host[starts[i]:starts[i] + sizes[i]] = batch.text[offs[i]:offs[i + 1]]
    d_text = torch.from_numpy(host).to(f"cuda:{local}")
    pairs = np.zeros((n, 2), np.int64)
    pairs[:, 1] = sizes
    d_pairs = torch.from_numpy(pairs).to(f"cuda:{local}")
    dec = pkg.Decompiler(local)
    stream = torch.cuda.current_stream()
    base, pbase = d_text.data_ptr(), d_pairs.data_ptr()

    def one(i):
        dec.run_device(base + int(starts[i]), int(sizes[i]), pbase + 16 * i, 1, stream.cuda_stream)

    for i in range(min(n, 8)):
        one(i)
    torch.cuda.synchronize()
    launches = dec.launches()
    t0 = time.perf_counter()
    for i in range(n):
        one(i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dec.close()
    ni = int(batch.ninstr[:n].sum())
    return {"value": ni / dt, "unit": "instr/s", "kernels": n, "instrs": ni, "ms_per_kernel": dt * 1e3 / n,
            "launches_per_kernel": launches, "form": "one pipeline run per kernel, text in HBM",
            "kernels_from": "the first kernels of the 10,000-kernel batch"}


def serve(pkg, local, rates, n_pool=1000, min_requests=100_000, min_seconds=10.0, budget=20 << 30):
    """Open-loop Poisson arrivals of single-kernel requests (lengths 100..50,000,
    the batch mix) through submit_batch / poll / fetch_batch; latency is from
    the scheduled arrival to the job's finish time.  Each rate runs for
    min_seconds of arrivals or min_requests requests, whichever is fewer
    requests: 10 s at 1k/s and 10k/s, 100,000 requests (1 s) at 100k/s.  Every result's length, and
    the whole text of every 16th request, is compared with the pool decompiled in one batch (the
    full comparison of every result is tests/test_gpu_serving.py's)."""
    params = gcngen.preset(4)
    pool = gcngen.generate(params, n_pool, seed=gcngen.SEED_BASE + 4, threads=os.cpu_count() or 4)
    texts = [pool.kernel(i) for i in range(n_pool)]
    ninstr = pool.ninstr.astype(np.int64)
    out = {"budget_bytes": budget, "pool": f"{n_pool} seeded requests (lengths 100..50000), cycled",
           "latency": "scheduled arrival -> job finished (CLOCK_MONOTONIC)", "rates": []}
    with pkg.Decompiler(local, mem_budget_bytes=budget, tuning_file=tuning_file(serve=True)) as dec:
        ids = dec.submit_batch(texts)
        raw, offs, _ = dec.fetch_batch_raw(ids)
        ref = [raw[offs[i]:offs[i + 1]].tobytes() for i in range(n_pool)]
        ref_len = np.array([len(r) for r in ref], dtype=np.int64)
        for rate in rates:
            rng = np.random.default_rng(2107078090 + rate)
            n = int(min(min_requests, rate * min_seconds))
            arr = np.cumsum(rng.exponential(1.0 / rate, n))
            which = rng.integers(0, n_pool, n)
            id_to_req = {}
            lock = threading.Lock()
            lat = np.zeros(n)
            done_ns = np.zeros(n, np.int64)
            mism = [0]
            full = [0]
            t0 = time.monotonic_ns() + 20_000_000
            arr_ns = (t0 + arr * 1e9).astype(np.int64)

            def submitter():
                i = 0
                while i < n:
                    now = time.monotonic_ns()
                    j = int(np.searchsorted(arr_ns, now, side="right"))
                    if j <= i:
                        time.sleep(max(0.0, min(0.001, (arr_ns[i] - now) / 1e9)))
                        continue
                    try:
                        got = dec.submit_batch([texts[w] for w in which[i:j]])
                    except pkg.GcnDecompError as e:
                        if e.rc != pkg.GCN_EAGAIN:
                            raise
                        got = []
                    with lock:
                        for q, jid in enumerate(got):
                            id_to_req[jid] = i + q
                    i += len(got)
                    if i < j:
                        time.sleep(0.0005)  # slots or memory budget full: retry soon

            def fetcher():
                seen = 0
                waiting = []
                while seen < n:
                    got = dec.poll(cap=8192, timeout_ms=20)
                    waiting += got
                    if not waiting:
                        continue
                    with lock:
                        ready = [j for j in waiting if j in id_to_req]
                    if not ready:
                        continue
                    rs = set(ready)
                    waiting = [j for j in waiting if j not in rs]
                    t_done = dec.job_info_batch(ready)[:, 3].astype(np.int64)
                    raw, offs, _ = dec.fetch_batch_raw(ready)
                    rq = np.fromiter((id_to_req[j] for j in ready), np.int64, len(ready))
                    done_ns[rq] = t_done
                    lat[rq] = (t_done - arr_ns[rq]) / 1e6
                    # every result's length; the whole text of every 16th request (copying and
                    # comparing all of them in this thread would bound the rate measured)
                    lens = np.diff(offs)
                    mism[0] += int(np.count_nonzero(lens != ref_len[which[rq]]))
                    for q in np.nonzero(rq % 16 == 0)[0]:
                        full[0] += 1
                        if raw[offs[q]:offs[q + 1]].tobytes() != ref[which[rq[q]]]:
                            mism[0] += 1
                    seen += len(ready)

            th = [threading.Thread(target=submitter), threading.Thread(target=fetcher)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            served = int(ninstr[which].sum())
            span = (done_ns.max() - arr_ns[0]) / 1e9
            out["rates"].append({
                "rate_rps": rate, "requests": n, "arrival_window_s": float(arr[-1]),
                "offered_instr_s": float(rate * ninstr[which].mean()),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "throughput_instr_s": served / span, "mismatches": mism[0],
                "compared": f"the length of every result, the whole text of {full[0]} (every 16th request)"})
    return out


def algorithmic_bytes(st):
    """Contract bytes of one pass: text in + OpenCL out + the IR arrays the
    parity tests compare (instruction records, block ids, block tables, headers)."""
    return {
        "text_in": st["text_bytes"],
        "text_out": st["out_bytes"],
        "ir": 32 * st["instrs"] + 4 * st["instrs"] + 4 * st["instrs"] + 16 * st["pblocks"] + 16 * st["lblocks"]
        + 32 * st["kernels"],
    }


def check_parity(dec, batch, files):
    """Byte-exact comparison of files of the handle's last device-resident run with the oracle."""
    import oracle

    bad = 0
    for f in files:
        texts, sts = dec.result_copy(f, f + 1)
        want = oracle.decompile(batch.kernel(f))
        bad += int(texts[0] != want.text or sts[0] != want.worst)
    return len(files), bad


def device_batch(torch, batch, local):
    d_text = torch.from_numpy(batch.text).to(f"cuda:{local}")
    d_off = torch.from_numpy(batch.offsets.view(np.int64)).to(f"cuda:{local}")
    return d_text, d_off


def single_batch_value(pkg, torch, dec, batch, local, steps, warmup, check=50):
    """One pipeline pass over a whole batch per step, text in HBM: instr/s, ms per pass, parity."""
    d_text, d_off = device_batch(torch, batch, local)
    stream = torch.cuda.current_stream()

    def step():
        dec.run_device(d_text.data_ptr(), int(batch.text.nbytes), d_off.data_ptr(), len(batch), stream.cuda_stream)

    for _ in range(max(warmup, 1)):
        step()
    dec.result_device()
    n = len(batch)
    checked, bad = check_parity(dec, batch, sorted(set(int(x) for x in np.linspace(0, n - 1, min(check, n)))))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": batch.total_instr / (ms / 1e3), "unit": "instr/s", "ms_per_pass": ms,
            "kernels": n, "instrs": batch.total_instr, "text_bytes": int(batch.text.nbytes),
            "parity": {"checked": checked, "mismatches": bad}}


def e2e_stream(pkg, dec, chunks, piece, window):
    """The stream through the job service: a submitting thread hands the packed
    texts of `piece` kernels at a time to gcn_decomp_submit_batch while at most
    `window` pieces are unfetched; a fetching thread takes each piece's results
    with gcn_decomp_fetch_batch (waiting for them).  Returns wall seconds and
    bytes copied each way."""
    import queue

    q = queue.Queue(maxsize=window)
    d2h = [0]
    err = []

    def fetcher():
        try:
            while True:
                ids = q.get()
                if ids is None:
                    break
                raw, offs, st = dec.fetch_batch_raw(ids)
                d2h[0] += len(raw) + 12 * len(ids)
        except Exception as e:  # noqa: BLE001 - reported by the caller
            err.append(e)

    th = threading.Thread(target=fetcher)
    t0 = time.perf_counter()
    th.start()
    h2d = 0
    for b in chunks:
        n = len(b)
        for p0 in range(0, n, piece):
            p1 = min(p0 + piece, n)
            ids = []
            while len(ids) < p1 - p0:
                got = dec.submit_packed(b.text, b.offsets[p0 + len(ids):p1 + 1])
                if not got:
                    time.sleep(0.0005)
                ids += got
            h2d += int(b.offsets[p1] - b.offsets[p0]) + 8 * (p1 - p0 + 1)
            q.put(ids)
            if err:
                break
    q.put(None)
    th.join()
    if err:
        raise err[0]
    return time.perf_counter() - t0, h2d, d2h[0]


def stream_main(args, pkg, torch, rank, world, local):
    """The default measurement: the 1,000,000-kernel stream in chunks."""
    cfg, total = WORKLOADS["config2"]
    total = args.kernels or total
    chunk = min(args.chunk, total)
    params = gcngen.preset(cfg)
    first0 = rank_first(rank, total)
    threads = os.cpu_count() or 4
    t_gen = time.perf_counter()
    chunks = [gcngen.generate(params, min(chunk, total - c0), seed=gcngen.SEED_BASE + cfg, first=first0 + c0,
                              threads=threads) for c0 in range(0, total, chunk)]
    t_gen = time.perf_counter() - t_gen
    instr_total = sum(b.total_instr for b in chunks)
    bytes_total = sum(int(b.text.nbytes) for b in chunks)
    dev = [device_batch(torch, b, local) for b in chunks]
    S = max(1, args.streams)
    decs = [pkg.Decompiler(local, tuning_file=tuning_file()) for _ in range(S)]
    streams = [torch.cuda.current_stream()] + [torch.cuda.Stream(device=local) for _ in range(S - 1)]

    def run_chunk(h, c):
        d_text, d_off = dev[c]
        decs[h].run_device(d_text.data_ptr(), int(chunks[c].text.nbytes), d_off.data_ptr(), len(chunks[c]),
                           streams[h].cuda_stream)

    def steps_over_handles(nsteps):
        """nsteps passes over every chunk; chunk c goes to handle c % S, each handle driven by its own
        host thread (the library releases the interpreter lock while it runs)."""
        errs = []

        def drive(h):
            try:
                with torch.cuda.stream(streams[h]):
                    for _ in range(nsteps):
                        for c in range(h, len(chunks), S):
                            run_chunk(h, c)
            except Exception as e:  # noqa: BLE001
                errs.append(e)

        ths = [threading.Thread(target=drive, args=(h,)) for h in range(S)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        if errs:
            raise errs[0]

    # warm-up: grows every handle's workspace to the largest chunk
    steps_over_handles(max(args.warmup, 3))
    torch.cuda.synchronize()

    # parity on every chunk (outside the timed region) and the pass statistics
    stats_sum = {k: 0 for k in ("text_bytes", "out_bytes", "instrs", "pblocks", "lblocks", "kernels")}
    parity = {"checked": 0, "mismatches": 0}
    launches_per_step = 0
    for c, b in enumerate(chunks):
        run_chunk(0, c)
        decs[0].result_device()
        st = decs[0].run_stats()
        st["text_bytes"] = int(b.text.nbytes)
        for k in stats_sum:
            stats_sum[k] += st[k]
        launches_per_step += decs[0].launches()
        if rank == 0:
            n = len(b)
            files = sorted(set(int(x) for x in np.linspace(0, n - 1, min(args.check, n))))
            k_, bad = check_parity(decs[0], b, files)
            parity["checked"] += k_
            parity["mismatches"] += bad
    torch.cuda.synchronize()
    for d in decs:
        d.stage_totals(reset=True)

    # the timed region: K passes over every chunk, text in HBM
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    main = streams[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(main)
        for s in streams[1:]:
            s.wait_event(e0)
        steps_over_handles(args.steps)
        for s in streams[1:]:
            ev = torch.cuda.Event()
            ev.record(s)
            main.wait_event(ev)
        e1.record(main)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(torch, ms, f"cuda:{local}")
    value = instr_total * world / (ms / 1e3)
    # stage and kernel times summed over the timed passes of every handle (overlapping on the device)
    timed_stage_ms = {}
    timed_runs = 0
    for d in decs:
        tot, runs = d.stage_totals(reset=True)
        timed_runs += runs
        for k, v in tot.items():
            timed_stage_ms[k] = timed_stage_ms.get(k, 0.0) + v / args.steps

    # the longest kernels timed alone: one pass over every chunk on one stream
    for c in range(len(chunks)):
        run_chunk(0, c)
    alone, _ = decs[0].stage_totals(reset=True)
    for d in decs[1:]:
        d.close()
    decs = decs[:1]
    torch.cuda.synchronize()

    # end to end through the job service (host buffers)
    e2e = None
    if args.e2e_steps > 0:
        with pkg.Decompiler(local, tuning_file=tuning_file()) as jd:
            e2e_stream(pkg, jd, chunks[:1], args.piece, args.window)  # warm-up: pinned slabs, engines
            runs = [e2e_stream(pkg, jd, chunks, args.piece, args.window) for _ in range(args.e2e_steps)]
        secs = statistics.median(r[0] for r in runs)
        secs = max_over_ranks(torch, secs, f"cuda:{local}")
        e2e = {"value": instr_total * world / secs, "unit": "instr/s", "h2d_bytes_per_step": runs[-1][1],
               "d2h_bytes_per_step": runs[-1][2], "ms_per_step": secs * 1e3,
               "path": "gcn_decomp_submit_batch (packed host texts, pieces of "
                       f"{args.piece} kernels, at most {args.window} pieces unfetched) + gcn_decomp_fetch_batch",
               "copies_declared": True}

    peaks, src = measured_peaks()
    ab = algorithmic_bytes(stats_sum)
    bytes_per_step = ab["text_in"] + ab["text_out"] + ab["ir"]
    stage_alone = {k: v for k, v in alone.items() if k not in KERNEL_TIMINGS}
    kern_alone = {k: alone.get(k, 0.0) for k in KERNEL_TIMINGS}
    dom = max(kern_alone, key=kern_alone.get)
    dom_ms = kern_alone[dom]
    achieved = bytes_per_step / (dom_ms / 1e3) / 1e9
    roofline = {
        "bound": "hbm", "kernel": f"{dom}: the longest kernel of a pass",
        "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
        "peak_source": src, "bytes_per_instr": bytes_per_step / instr_total,
        "kernel_ms_per_step": dom_ms,
        "timing": "CUDA events around each launch inside the library, summed over one pass of every chunk on "
                  "one stream (kernel timed alone)",
        "traffic": (K_ITEMS_DRAM_PER_INSTR * instr_total / len(chunks)) if dom.startswith("k_items") else None,
        "traffic_note": "DRAM bytes per launch (one chunk): the ncu capture of k_items on 4,000 kernels of the "
                        "same distribution (under profiles/), 370 B per instruction, times "
                        "the instructions of a launch; not re-taken in this run",
        "path_frac": bytes_per_step / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
        "path_note": "the whole pass: algorithmic bytes / ms_per_step against the same peak",
        "kernels_ms_per_step_alone": kern_alone,
    }

    extras = {}
    cpu = None
    if rank == 0 and not args.no_extras:
        c1cfg, c1 = make_workload("config1", 0)
        extras["batch"] = dict(single_batch_value(pkg, torch, decs[0], c1, local, 10, 3),
                               workload=f"config1: 10,000 seeded synthetic kernels (preset {c1cfg}) in one pass")
        if args.per_kernel > 0:
            extras["per_kernel"] = per_kernel_form(pkg, torch, c1, local, args.per_kernel)
        c3cfg, c3 = make_workload("config3", 0)
        extras["large_cfg"] = dict(single_batch_value(pkg, torch, decs[0], c3, local, 3, 1, check=2),
                                   workload=f"config3: 64 seeded synthetic kernels of 200,000 instrs (preset {c3cfg})")
        del c3
        if not args.no_serve:
            decs[0].close()
            decs = []
            extras["serve"] = serve(pkg, local, [1000, 10000, 100000])
    if rank == 0 and not args.no_cpu_baseline:
        r, ni, nk, dt = oracle_rate(chunks[0], 12.0)
        cpu = {"value": r, "unit": "instr/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {nk} kernels of the stream ({ni} instrs, {dt:.1f} s), single thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "instr/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"config2: {total} seeded synthetic kernels (preset {cfg}) per GPU in chunks of "
                                   f"{chunk}, {instr_total} instrs, {bytes_total} text bytes",
                       "kernels": total, "chunk": chunk, "instrs": instr_total, "text_bytes": bytes_total,
                       "handles": S,
                       "l2": "inputs larger than L2 (every chunk's text > 129 MB); no flush between steps",
                       "form": f"batched: one pipeline pass per chunk, chunks spread over {S} handles "
                               f"(streams and host threads), text in HBM"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "launches_per_pass": launches_per_step / len(chunks),
            "clocks": clk.summary(), "parity": parity,
            "stage_ms_per_step_alone": stage_alone, "stage_ms_per_step_timed": timed_stage_ms,
            "run_stats_per_step": stats_sum, "generate_s": t_gen,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    for d in decs:
        d.close()


def batch_main(args, pkg, torch, rank, world, local):
    """A single-batch workload (--workload config1/config3/select/sysval): one pass per step."""
    cfg, batch = make_workload(args.workload, rank, args.kernels)
    dec = pkg.Decompiler(local, tuning_file=tuning_file())
    d_text, d_off = device_batch(torch, batch, local)
    stream = torch.cuda.current_stream()
    n_files = len(batch)

    def step():
        dec.run_device(d_text.data_ptr(), int(batch.text.nbytes), d_off.data_ptr(), n_files, stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    dec.result_device()
    parity = {"checked": 0, "mismatches": 0}
    if rank == 0:
        files = sorted(set(int(x) for x in np.linspace(0, n_files - 1, min(args.check, n_files))))
        parity["checked"], parity["mismatches"] = check_parity(dec, batch, files)
    stats = dec.run_stats()
    stats["text_bytes"] = int(batch.text.nbytes)
    launches = dec.launches()
    dec.stage_totals(reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tot, runs = dec.stage_totals(reset=True)
    per = {k: v / max(runs, 1) for k, v in tot.items()}
    ms = max_over_ranks(torch, ms, f"cuda:{local}")
    value = batch.total_instr * world / (ms / 1e3)

    e2e = None
    if args.e2e_steps > 0:
        e2e_ms, d2h = [], 0
        for _ in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ids = dec.submit_packed(batch.text, batch.offsets)
            raw, offs, sts = dec.fetch_batch_raw(ids)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            d2h = len(raw) + 12 * n_files
        e2e_ms = e2e_ms[1:]
        e2e = {"value": batch.total_instr * world / (statistics.median(e2e_ms) / 1e3), "unit": "instr/s",
               "h2d_bytes_per_step": int(batch.text.nbytes) + 8 * (n_files + 1), "d2h_bytes_per_step": d2h,
               "ms_per_step": statistics.median(e2e_ms), "copies_declared": True}

    peaks, src = measured_peaks()
    ab = algorithmic_bytes(stats)
    bytes_per_pass = ab["text_in"] + ab["text_out"] + ab["ir"]
    kern = {k: per.get(k, 0.0) for k in KERNEL_TIMINGS}
    dom = max(kern, key=kern.get)
    achieved = bytes_per_pass / (kern[dom] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": f"{dom}: the longest kernel of a pass", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": src,
                "bytes_per_instr": bytes_per_pass / batch.total_instr, "kernel_ms": kern[dom], "traffic": None,
                "path_frac": bytes_per_pass / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], "kernels_ms": kern}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, ni, nk, dt = oracle_rate(batch, 12.0)
        cpu = {"value": r, "unit": "instr/s", "cores": 1, "kind": "oracle",
               "sample": f"first {nk} kernels of the workload ({ni} instrs, {dt:.1f} s), single thread"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "instr/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {n_files} seeded synthetic kernels (preset {cfg}), "
                                   f"{batch.total_instr} instrs, {stats['text_bytes']} text bytes per GPU",
                       "kernels": n_files, "instrs": batch.total_instr, "text_bytes": stats["text_bytes"],
                       "l2": ("inputs larger than L2 (text > 129 MB); no flush between steps"
                              if stats["text_bytes"] > 129e6 else
                              "text smaller than L2 but the IR arrays of a pass exceed it; no flush"),
                       "form": "batched: one pipeline pass over all kernels per step"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches * args.steps, "clocks": clk.summary(),
            "stage_ms": {k: v for k, v in per.items() if k not in KERNEL_TIMINGS},
            "parity": parity, "run_stats": stats,
        }
        if args.per_kernel > 0:
            line["per_kernel"] = per_kernel_form(pkg, torch, batch, local, args.per_kernel)
        print(json.dumps(line), flush=True)
    dec.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config2", choices=sorted(WORKLOADS))
    ap.add_argument("--kernels", type=int, default=None, help="kernels per GPU (default: the workload's)")
    ap.add_argument("--chunk", type=int, default=100_000, help="kernels per pass of the config2 stream")
    ap.add_argument("--streams", type=int, default=1, help="handles (streams, host threads) the chunks spread over")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--piece", type=int, default=8192, help="kernels per submit_batch call of the e2e stream")
    ap.add_argument("--window", type=int, default=6, help="pieces submitted and not yet fetched in the e2e stream")
    ap.add_argument("--check", type=int, default=20, help="files per chunk compared with the oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-kernel", type=int, default=2000, help="kernels timed in the one-run-per-kernel form")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch, plain-form, large-CFG and serving lines")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2107_07809_gb300 as pkg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.build()
    if args.workload == "config2":
        stream_main(args, pkg, torch, rank, world, local)
    else:
        batch_main(args, pkg, torch, rank, world, local)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
