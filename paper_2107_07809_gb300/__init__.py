"""GB300 (sm_103a) GCN -> OpenCL decompiler: thin ctypes binding of libgcndecomp.so.

Every stage of the decompiler runs in the CUDA kernels of ``csrc/``; this module
only marshals arguments to the C ABI declared in ``include/gcn_decomp.h``.  When
the shared library is missing, or no GPU is present, calls raise — there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libgcndecomp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]

GCN_OK, GCN_EINVAL, GCN_ENOMEM, GCN_EAGAIN, GCN_ENOJOB, GCN_ECUDA = 0, -1, -2, -3, -4, -5
ST_OK, ST_PARTIAL, ST_PARSE_ERROR, ST_FIXPOINT_CAP = 0, 1, 2, 3
IR_INSTR, IR_PBLOCK_OF, IR_PBLOCKS, IR_LBLOCK_OF, IR_LBLOCKS, IR_HEADER = range(6)

_lock = threading.Lock()
_lib = None


def _sources():
    return sorted(os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(_ROOT, "include", "gcn_decomp.h")]


def build(force: bool = False, jobs: int | None = None) -> str:
    """Compile every .cu for sm_103a (in parallel) and link libgcndecomp.so in-tree."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()
    newest_hdr = max(os.path.getmtime(h) for h in _headers())
    objs = []
    todo = []
    for src in srcs:
        obj = os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_hdr):
            todo.append((src, obj))

    def compile_one(so):
        src, obj = so
        tmp = obj + f".{os.getpid()}.tmp.o"
        cmd = ["nvcc", *ARCH, *NVCC_FLAGS, "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, obj)

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(8, len(todo))) as ex:
            list(ex.map(compile_one, todo))
    if force or todo or not os.path.exists(LIB_PATH):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_uint32),
                ("tuning_file", ctypes.c_char_p), ("flags", ctypes.c_uint32)]


def lib():
    """Load libgcndecomp.so (it must have been built; there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2107_07809_gb300.build() first")
            L = ctypes.CDLL(LIB_PATH)
            vp, u64, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
            L.gcn_decomp_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
            L.gcn_decomp_destroy.argtypes = [vp]
            L.gcn_decomp_destroy.restype = None
            L.gcn_decomp_submit_batch.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(sz), sz,
                                                  ctypes.POINTER(u64), ctypes.POINTER(sz)]
            L.gcn_decomp_fetch_opencl.argtypes = [vp, u64, vp, sz, ctypes.POINTER(sz), ctypes.POINTER(i32),
                                                  ctypes.c_uint32]
            L.gcn_decomp_fetch_ir.argtypes = [vp, u64, i32, vp, sz, ctypes.POINTER(sz)]
            L.gcn_decomp_run_device.argtypes = [vp, vp, u64, vp, u64, vp]
            L.gcn_decomp_result_device.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                   ctypes.POINTER(u64)]
            L.gcn_decomp_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float),
                                                 ctypes.POINTER(ctypes.c_char_p), i32]
            L.gcn_decomp_last_error.restype = ctypes.c_char_p
            L.gcn_decomp_result_copy.argtypes = [vp, u64, u64, vp, sz, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_int32)]
            L.gcn_decomp_run_stats.argtypes = [vp, ctypes.POINTER(u64), i32]
            L.gcn_decomp_stage_totals.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_char_p), i32, ctypes.POINTER(u64), i32]
            L.gcn_decomp_launches.argtypes = [vp]
            L.gcn_decomp_launches.restype = u64
            L.gcn_decomp_line_starts_noalloc.argtypes = [vp, u64, vp, u64, vp, vp]
            L.gcn_decomp_fetch_batch.argtypes = [vp, ctypes.POINTER(u64), sz, vp, sz, ctypes.POINTER(u64),
                                                 ctypes.POINTER(ctypes.c_int32), ctypes.c_uint32]
            L.gcn_decomp_poll.argtypes = [vp, ctypes.POINTER(u64), sz, ctypes.POINTER(sz), i32]
            L.gcn_decomp_job_info.argtypes = [vp, u64, ctypes.POINTER(u64), i32]
            L.gcn_decomp_job_info_batch.argtypes = [vp, ctypes.POINTER(u64), sz, ctypes.POINTER(u64), i32]
            _lib = L
    return _lib


class GcnDecompError(RuntimeError):
    def __init__(self, rc: int, what: str):
        msg = lib().gcn_decomp_last_error().decode(errors="replace")
        super().__init__(f"{what} failed ({rc}): {msg}")
        self.rc = rc


def _ck(rc: int, what: str):
    if rc != GCN_OK:
        raise GcnDecompError(rc, what)


class Decompiler:
    """One handle on ``device``: device memory, CUDA streams and the worker lanes of the job service."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_slots: int = 0,
                 tuning_file: str | None = None):
        self._h = ctypes.c_void_p()
        cfg = Config(device, mem_budget_bytes, max_slots, tuning_file.encode() if tuning_file else None, 0)
        _ck(lib().gcn_decomp_create(ctypes.byref(cfg), ctypes.byref(self._h)), "gcn_decomp_create")

    def close(self):
        if self._h:
            lib().gcn_decomp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host-buffer API -----------------------------------------------------
    def submit_batch(self, texts: list[bytes]) -> list[int]:
        n = len(texts)
        arr = (ctypes.c_char_p * n)(*texts)
        lens = (ctypes.c_size_t * n)(*[len(t) for t in texts])
        ids = (ctypes.c_uint64 * n)()
        got = ctypes.c_size_t()
        _ck(lib().gcn_decomp_submit_batch(self._h, arr, lens, n, ids, ctypes.byref(got)), "gcn_decomp_submit_batch")
        return list(ids[: got.value])

    def submit_packed(self, text, offsets) -> list[int]:
        """submit_batch for files held back to back in one buffer: file i is
        text[offsets[i]:offsets[i+1]] (``text`` a contiguous uint8 numpy array,
        ``offsets`` n+1 integers).  The pointer and length arrays are built with
        numpy instead of one Python object per file."""
        import numpy as np

        text = np.ascontiguousarray(text, dtype=np.uint8)
        offs = np.asarray(offsets, dtype=np.uint64)
        n = len(offs) - 1
        if n <= 0:
            return []
        ptrs = (np.uint64(text.ctypes.data) + offs[:-1]).astype(np.uint64)
        lens = (offs[1:] - offs[:-1]).astype(np.uint64)
        ids = np.zeros(n, dtype=np.uint64)
        got = ctypes.c_size_t()
        _ck(lib().gcn_decomp_submit_batch(self._h, ptrs.ctypes.data_as(ctypes.POINTER(ctypes.c_char_p)),
                                          lens.ctypes.data_as(ctypes.POINTER(ctypes.c_size_t)), n,
                                          ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(got)),
            "gcn_decomp_submit_batch")
        return ids[: got.value].tolist()

    def fetch_opencl(self, job: int, wait: bool = True) -> tuple[str, int]:
        n = ctypes.c_size_t()
        st = ctypes.c_int()
        _ck(lib().gcn_decomp_fetch_opencl(self._h, job, None, 0, ctypes.byref(n), ctypes.byref(st), 1 if wait else 0),
            "gcn_decomp_fetch_opencl")
        buf = ctypes.create_string_buffer(max(n.value, 1))
        _ck(lib().gcn_decomp_fetch_opencl(self._h, job, buf, n.value, ctypes.byref(n), ctypes.byref(st), 1 if wait else 0),
            "gcn_decomp_fetch_opencl")
        return buf.raw[: n.value].decode(), st.value

    def fetch_ir(self, job: int, which: int) -> bytes:
        n = ctypes.c_size_t()
        _ck(lib().gcn_decomp_fetch_ir(self._h, job, which, None, 0, ctypes.byref(n)), "gcn_decomp_fetch_ir")
        buf = ctypes.create_string_buffer(max(n.value, 1))
        _ck(lib().gcn_decomp_fetch_ir(self._h, job, which, buf, n.value, ctypes.byref(n)), "gcn_decomp_fetch_ir")
        return buf.raw[: n.value]

    def fetch_batch(self, ids: list[int], wait: bool = True) -> tuple[list[str], list[int]]:
        """Texts and statuses of jobs `ids` (one call; the jobs are released)."""
        n = len(ids)
        arr = (ctypes.c_uint64 * max(n, 1))(*ids)
        offs = (ctypes.c_uint64 * (n + 1))()
        st = (ctypes.c_int32 * max(n, 1))()
        fl = 1 if wait else 0
        _ck(lib().gcn_decomp_fetch_batch(self._h, arr, n, None, 0, offs, st, fl), "gcn_decomp_fetch_batch")
        buf = ctypes.create_string_buffer(max(int(offs[n]), 1))
        _ck(lib().gcn_decomp_fetch_batch(self._h, arr, n, buf, int(offs[n]), offs, st, fl), "gcn_decomp_fetch_batch")
        raw = buf.raw
        return [raw[offs[i]:offs[i + 1]].decode() for i in range(n)], [int(st[i]) for i in range(n)]

    def fetch_batch_raw(self, ids: list[int]):
        """Like fetch_batch, without splitting or decoding: (texts back to back as a numpy uint8
        array, offsets and statuses as numpy arrays)."""
        import numpy as np

        n = len(ids)
        arr = np.asarray(ids if n else [0], dtype=np.uint64)
        offs = np.zeros(n + 1, dtype=np.uint64)
        st = np.zeros(max(n, 1), dtype=np.int32)
        pa = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        po = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        ps = st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        _ck(lib().gcn_decomp_fetch_batch(self._h, pa, n, None, 0, po, ps, 1), "gcn_decomp_fetch_batch")
        buf = np.empty(max(int(offs[n]), 1), dtype=np.uint8)
        _ck(lib().gcn_decomp_fetch_batch(self._h, pa, n, buf.ctypes.data, int(offs[n]), po, ps, 1),
            "gcn_decomp_fetch_batch")
        return buf[: int(offs[n])], offs.astype(np.int64), st[:n]

    def poll(self, cap: int = 4096, timeout_ms: int = 0) -> list[int]:
        """Finished jobs not reported before (waits up to timeout_ms for one)."""
        ids = (ctypes.c_uint64 * cap)()
        got = ctypes.c_size_t()
        _ck(lib().gcn_decomp_poll(self._h, ids, cap, ctypes.byref(got), timeout_ms), "gcn_decomp_poll")
        return list(ids[: got.value])

    def job_info(self, job: int) -> dict[str, int]:
        """State (0 queued, 1 running, 2 done), CLOCK_MONOTONIC ns timestamps, IR residency."""
        v = (ctypes.c_uint64 * 5)()
        n = lib().gcn_decomp_job_info(self._h, job, v, 5)
        if n < 0:
            raise GcnDecompError(n, "gcn_decomp_job_info")
        keys = ["state", "t_submit", "t_start", "t_done", "ir_resident"]
        return {keys[i]: int(v[i]) for i in range(n)}

    def job_info_batch(self, jobs: list[int]):
        """job_info for many jobs in one call: an (n, 5) uint64 numpy array (columns as job_info;
        all zero for an unknown job)."""
        import numpy as np

        n = len(jobs)
        ids = (ctypes.c_uint64 * max(n, 1))(*jobs)
        out = np.zeros((n, 5), np.uint64)
        _ck(lib().gcn_decomp_job_info_batch(self._h, ids, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), 5),
            "gcn_decomp_job_info_batch")
        return out

    def decompile(self, texts: list[bytes]) -> list[tuple[str, int]]:
        ids = self.submit_batch(texts)
        outs, st = self.fetch_batch(ids)
        return list(zip(outs, st))

    # ---- device-buffer API -----------------------------------------------------
    def run_device(self, text_ptr: int, text_len: int, off_ptr: int, n_files: int, stream: int = 0):
        _ck(lib().gcn_decomp_run_device(self._h, text_ptr, text_len, off_ptr, n_files, stream or None),
            "gcn_decomp_run_device")

    def result_device(self):
        o, oo, st = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        nb = ctypes.c_uint64()
        _ck(lib().gcn_decomp_result_device(self._h, ctypes.byref(o), ctypes.byref(oo), ctypes.byref(st),
                                           ctypes.byref(nb)), "gcn_decomp_result_device")
        return o.value, oo.value, st.value, nb.value

    def run_stats(self) -> dict[str, int]:
        """Sizes of the last run (lines, kernels, instructions, labels, blocks, state words, output and
        device bytes), the handle's peak workspace bytes and its batches split after allocation failures."""
        v = (ctypes.c_uint64 * 11)()
        n = lib().gcn_decomp_run_stats(self._h, v, 11)
        keys = ["lines", "kernels", "instrs", "labels", "pblocks", "lblocks", "state_words", "out_bytes",
                "device_bytes", "peak_device_bytes", "splits"]
        return {keys[i]: int(v[i]) for i in range(max(n, 0))}

    def launches(self) -> int:
        """CUDA kernels launched by the last pipeline run."""
        return int(lib().gcn_decomp_launches(self._h))

    def result_copy(self, f0: int, f1: int) -> tuple[list[str], list[int]]:
        """Texts and statuses of files [f0, f1) of the last device-resident run."""
        n = f1 - f0
        offs = (ctypes.c_uint64 * (n + 1))()
        st = (ctypes.c_int32 * max(n, 1))()
        _ck(lib().gcn_decomp_result_copy(self._h, f0, f1, None, 0, offs, st), "gcn_decomp_result_copy")
        buf = ctypes.create_string_buffer(max(int(offs[n]), 1))
        _ck(lib().gcn_decomp_result_copy(self._h, f0, f1, buf, int(offs[n]), offs, st), "gcn_decomp_result_copy")
        raw = buf.raw
        return [raw[offs[i]:offs[i + 1]].decode() for i in range(n)], [int(st[i]) for i in range(n)]

    def stage_totals(self, reset: bool = False) -> tuple[dict[str, float], int]:
        """Stage and kernel times summed over the device-resident runs since the last reset, and the
        number of runs."""
        ms = (ctypes.c_double * 32)()
        nm = (ctypes.c_char_p * 32)()
        runs = ctypes.c_uint64()
        n = lib().gcn_decomp_stage_totals(self._h, ms, nm, 32, ctypes.byref(runs), 1 if reset else 0)
        if n < 0:
            raise GcnDecompError(n, "gcn_decomp_stage_totals")
        return {nm[i].decode(): float(ms[i]) for i in range(n)}, int(runs.value)

    def stage_times(self) -> dict[str, float]:
        ms = (ctypes.c_float * 32)()
        nm = (ctypes.c_char_p * 32)()
        n = lib().gcn_decomp_stage_times(self._h, ms, nm, 32)
        return {nm[i].decode(): float(ms[i]) for i in range(max(n, 0))}


def line_starts_noalloc(d_text: int, text_len: int, d_line_start: int, line_cap: int, d_result: int,
                        stream: int = 0) -> None:
    """gcn_decomp_line_starts_noalloc: newline scan into caller device buffers, no allocation.

    ``d_result`` (2 x u32 on the device) receives the newline count and error bits
    once the stream has run the work."""
    _ck(lib().gcn_decomp_line_starts_noalloc(d_text, text_len, d_line_start, line_cap, d_result, stream or None),
        "gcn_decomp_line_starts_noalloc")
