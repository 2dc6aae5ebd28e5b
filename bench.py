#!/usr/bin/env python3
"""Throughput benchmark: GCN instructions decompiled per second on GB300.

One step decompiles the whole workload batch (every stage S1..S13 of the
method) through the C ABI.  Default workload: 10,000 seeded synthetic kernels
with log-uniform lengths 50..2000 (the plain-method-at-scale configuration),
one kernel per file, text resident in HBM when the timed region starts
(`value`).  `e2e` measures the same through the job service's host-buffer
entry points (submit_batch, given the whole batch as one buffer and its
offsets, and fetch_batch), host<->device copies inside the timed region.
`per_kernel` times the plain form (one pipeline run per kernel) on a sample of
the same kernels; `serve` drives the job service with open-loop Poisson
arrivals at 1k, 10k and 100k requests/s and reports p50/p99 latency.

--impl reference times the CPU oracle (single-threaded) on bounded samples of
the same workload, the comparison arm.  Multi-GPU (torchrun): every rank
decompiles its own kernels (weak scaling); there is no collective.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# runtime parameters picked by paper_2107_07809_gb300/autotune.py on a GB300 (if present)
TUNING = os.path.join(ROOT, "paper_2107_07809_gb300", "tuning", "gb300.tune")

import gcngen  # noqa: E402

WORKLOADS = {
    # name: (preset, kernels)
    "config1": (1, 10_000),
    "config2": (2, 1_000_000),  # streamed in chunks (large_batch)
    "config3": (3, 64),
    "select": (5, 10_000),  # the batch mix with ternaries (v_cndmask_b32)
    "sysval": (6, 10_000),  # the batch mix with dispatch-packet system values and scalar bit fields
}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


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
    batch = gcngen.generate(params, n, seed=gcngen.SEED_BASE + cfg, first=rank * n)
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
    cfg, batch = make_workload(args.workload, 0, args.kernels)
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
    sample = f"{kern} kernels ({instrs} instrs) over {args.steps} steps of ~{per_step:.0f} s, single thread"
    line = {
        "impl": "reference", "metric": "GCN instrs decompiled/sec", "value": value, "unit": "instr/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {len(batch)} seeded synthetic kernels (preset {cfg})"},
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
    t0 = time.perf_counter()
    for i in range(n):
        one(i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dec.close()
    ni = int(batch.ninstr[:n].sum())
    return {"value": ni / dt, "unit": "instr/s", "kernels": n, "instrs": ni, "ms_per_kernel": dt * 1e3 / n,
            "form": "one pipeline run per kernel, text in HBM"}


def serve(pkg, local, rates, n_pool=1000, max_requests=20000, max_seconds=5.0, budget=20 << 30):
    """Open-loop Poisson arrivals of single-kernel requests (lengths 100..50,000,
    the batch mix) through submit_batch / poll / fetch_batch; latency is from
    the scheduled arrival to the job's finish time."""
    import threading

    params = gcngen.preset(4)
    pool = gcngen.generate(params, n_pool, seed=gcngen.SEED_BASE + 4, threads=os.cpu_count() or 4)
    texts = [pool.kernel(i) for i in range(n_pool)]
    ninstr = pool.ninstr.astype(np.int64)
    out = {"budget_bytes": budget, "pool": f"{n_pool} seeded requests (lengths 100..50000), cycled",
           "latency": "scheduled arrival -> job finished (CLOCK_MONOTONIC)", "rates": []}
    with pkg.Decompiler(local, mem_budget_bytes=budget,
                        tuning_file=TUNING if os.path.exists(TUNING) else None) as dec:
        ids = dec.submit_batch(texts)
        raw, offs, _ = dec.fetch_batch_raw(ids)
        ref = [raw[offs[i]:offs[i + 1]].tobytes() for i in range(n_pool)]
        for rate in rates:
            rng = np.random.default_rng(2107078090 + rate)
            n = int(min(max_requests, rate * max_seconds))
            arr = np.cumsum(rng.exponential(1.0 / rate, n))
            which = rng.integers(0, n_pool, n)
            id_to_req = {}
            lock = threading.Lock()
            lat = np.zeros(n)
            done_ns = np.zeros(n, np.int64)
            mism = [0]
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
                    infos = [dec.job_info(j)["t_done"] for j in ready]
                    raw, offs, _ = dec.fetch_batch_raw(ready)
                    for q, j in enumerate(ready):
                        r = id_to_req[j]
                        done_ns[r] = infos[q]
                        lat[r] = (infos[q] - arr_ns[r]) / 1e6
                        if raw[offs[q]:offs[q + 1]].tobytes() != ref[which[r]]:
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
                "rate_rps": rate, "requests": n, "offered_instr_s": float(rate * ninstr[which].mean()),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "throughput_instr_s": served / span, "mismatches": mism[0]})
    return out


# the library's event timing of the statement-printing kernel alone (not a stage)
KERNEL_TIMING = "k_items (S13 print)"
# ncu counters of one k_items launch (4,000 kernels of the batch distribution)
K_ITEMS_TRAFFIC = {"instrs": 2201608, "bytes": 0.579754240e9 + 0.252110336e9}


def large_batch(args, pkg, torch, rank, world, local):
    """The 1,000,000-kernel stream (the batch distribution), decompiled in chunks of
    --chunk kernels: each chunk is generated and copied to HBM outside the timed
    region, then one pipeline pass decompiles it; value = all instructions / the
    summed CUDA-event time of the passes.  A sample of every chunk is checked
    against the oracle."""
    import oracle

    cfg, total = WORKLOADS["config2"]
    total = args.kernels or total
    chunk = min(args.chunk, total)
    params = gcngen.preset(cfg)
    dec = pkg.Decompiler(local, tuning_file=TUNING if os.path.exists(TUNING) else None)
    stream = torch.cuda.current_stream()
    ms_total, instr_total, bytes_total, kern_ms, parity = 0.0, 0, 0, 0.0, {"checked": 0, "mismatches": 0}
    first0 = rank * total
    warm = False
    with Clocks(local) as clk:
        for c0 in range(0, total, chunk):
            n = min(chunk, total - c0)
            b = gcngen.generate(params, n, seed=gcngen.SEED_BASE + cfg, first=first0 + c0,
                                threads=os.cpu_count() or 4)
            d_text = torch.from_numpy(b.text).to(f"cuda:{local}")
            d_off = torch.from_numpy(b.offsets.view(np.int64)).to(f"cuda:{local}")
            if not warm:  # grow the workspace once
                for _ in range(max(args.warmup, 3)):
                    dec.run_device(d_text.data_ptr(), int(b.text.nbytes), d_off.data_ptr(), n, stream.cuda_stream)
                warm = True
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dec.run_device(d_text.data_ptr(), int(b.text.nbytes), d_off.data_ptr(), n, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            dec.result_device()
            ms_total += e0.elapsed_time(e1)
            kern_ms += dec.stage_times().get(KERNEL_TIMING, 0.0)
            instr_total += int(b.total_instr)
            bytes_total += int(b.text.nbytes)
            if rank == 0:
                k = min(20, n)
                texts, sts = dec.result_copy(0, k)
                for f in range(k):
                    want = oracle.decompile(b.kernel(f))
                    parity["checked"] += 1
                    parity["mismatches"] += int(texts[f] != want.text or sts[f] != want.worst)
            del d_text, d_off, b
    if world > 1:
        t = torch.tensor([ms_total], device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    value = instr_total * world / (ms_total / 1e3)
    if rank == 0:
        line = {
            "metric": "GCN instrs decompiled/sec", "value": value, "unit": "instr/s", "n_gpus": world,
            "steps": (total + chunk - 1) // chunk, "warmup": max(args.warmup, 3),
            "ms_per_step": ms_total / ((total + chunk - 1) // chunk), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"config2: {total} seeded synthetic kernels (preset {cfg}) in chunks of {chunk}, "
                                   f"{instr_total} instrs, {bytes_total} text bytes per GPU",
                       "kernels": total, "chunk": chunk, "instrs": instr_total, "text_bytes": bytes_total,
                       "l2": "every chunk's text exceeds L2; no flush",
                       "form": "batched: one pipeline pass per chunk, text in HBM"},
            "kernel_ms_total": kern_ms, "e2e": None, "clocks": clk.summary(), "parity": parity,
        }
        print(json.dumps(line), flush=True)
    dec.close()


def algorithmic_bytes(st):
    """Contract bytes of one pass: text in + OpenCL out + the IR arrays the
    parity tests compare (instruction records, block ids, block tables, headers)."""
    return {
        "text_in": st["text_bytes"],
        "text_out": st["out_bytes"],
        "ir": 32 * st["instrs"] + 4 * st["instrs"] + 4 * st["instrs"] + 16 * st["pblocks"] + 16 * st["lblocks"]
        + 32 * st["kernels"],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config1", choices=sorted(WORKLOADS))
    ap.add_argument("--kernels", type=int, default=None)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-kernel", type=int, default=300, help="kernels timed in the one-run-per-kernel form")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--chunk", type=int, default=100_000, help="kernels per pass of the config2 stream")
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
        return large_batch(args, pkg, torch, rank, world, local)
    cfg, batch = make_workload(args.workload, rank, args.kernels)
    n_files = len(batch)
    total_instr = batch.total_instr
    d_text = torch.from_numpy(batch.text).to(f"cuda:{local}")
    d_off = torch.from_numpy(batch.offsets.view(np.int64)).to(f"cuda:{local}")
    dec = pkg.Decompiler(local, tuning_file=TUNING if os.path.exists(TUNING) else None)
    stream = torch.cuda.current_stream()

    def step():
        dec.run_device(d_text.data_ptr(), int(batch.text.nbytes), d_off.data_ptr(), n_files, stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    out_ptr, off_ptr, st_ptr, out_bytes = dec.result_device()

    # byte-exact parity on a sample of the benchmarked batch (outside the timed region)
    parity = {"checked": 0, "mismatches": 0}
    if rank == 0:
        import oracle

        n_check = min(200, n_files)
        texts, statuses = dec.result_copy(0, n_check)
        for f in range(n_check):
            want = oracle.decompile(batch.kernel(f))
            parity["checked"] += 1
            parity["mismatches"] += int(texts[f] != want.text or statuses[f] != want.worst)

    stats = dec.run_stats()
    stats["text_bytes"] = int(batch.text.nbytes)
    launches = dec.launches()

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
    stage_ms = dec.stage_times()
    if world > 1:
        t = torch.tensor([ms], device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = total_instr * world / (ms / 1e3)

    # end to end through the host-buffer API
    h2d = int(batch.text.nbytes) + 8 * (n_files + 1)
    e2e_ms = []
    d2h = 0
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = dec.submit_packed(batch.text, batch.offsets)
        raw, offs, sts = dec.fetch_batch_raw(ids)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        d2h = len(raw) + 12 * n_files
    e2e_val = total_instr * world / (statistics.median(e2e_ms) / 1e3) if e2e_ms else None

    plain = per_kernel_form(pkg, torch, batch, local, args.per_kernel) if args.per_kernel > 0 else None
    served = None
    if rank == 0 and not args.no_serve:
        served = serve(pkg, local, [1000, 10000, 100000])

    peaks, src = measured_peaks()
    ab = algorithmic_bytes(stats)
    bytes_per_pass = ab["text_in"] + ab["text_out"] + ab["ir"]
    kern_ms = stage_ms.pop(KERNEL_TIMING, None)
    dom = max(stage_ms, key=stage_ms.get)
    roofline = {"bound": "hbm", "kernel": "k_items (S13 statement printing, the longest kernel of a pass)",
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "peak_source": src,
                "bytes_per_instr": bytes_per_pass / total_instr,
                "traffic_source": f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_items launch on "
                                  f"{K_ITEMS_TRAFFIC['instrs']} instructions, scaled by instructions "
                                  f"(profiles/k_items_config1_4000.md)",
                "dominant_stage": {"name": dom, "ms": stage_ms[dom],
                                   "achieved": bytes_per_pass / (stage_ms[dom] / 1e3) / 1e9},
                "path_frac": bytes_per_pass / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    if kern_ms:
        achieved = bytes_per_pass / (kern_ms / 1e3) / 1e9
        roofline.update({"achieved": achieved, "frac": achieved / peaks["hbm_gbs"], "kernel_ms": kern_ms,
                         "traffic": K_ITEMS_TRAFFIC["bytes"] / K_ITEMS_TRAFFIC["instrs"] * total_instr})

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, ni, nk, dt = oracle_rate(batch, 12.0)
        cpu = {"value": r, "unit": "instr/s", "cores": 1, "kind": "oracle",
               "sample": f"first {nk} kernels of the workload ({ni} instrs, {dt:.1f} s), single thread"}

    if rank == 0:
        line = {
            "metric": "GCN instrs decompiled/sec", "value": value, "unit": "instr/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {n_files} seeded synthetic kernels (preset {cfg}), "
                                   f"{total_instr} instrs, {stats['text_bytes']} text bytes per GPU",
                       "kernels": n_files, "instrs": total_instr, "text_bytes": stats["text_bytes"],
                       "l2": ("inputs larger than L2 (text > 129 MB); no flush between steps"
                              if stats["text_bytes"] > 129e6 else
                              "text smaller than L2 but the IR arrays of a pass exceed it; no flush"),
                       "form": "batched: one pipeline pass over all kernels per step"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "instr/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.median(e2e_ms) if e2e_ms else None},
            "per_kernel": plain, "serve": served,
            "gpu_launches": launches * args.steps, "clocks": clk.summary(), "stage_ms": stage_ms,
            "parity": parity, "run_stats": stats,
        }
        print(json.dumps(line), flush=True)
    dec.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
