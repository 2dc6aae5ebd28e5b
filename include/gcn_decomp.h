/* gcn_decomp.h — C ABI of the GB300 (sm_103a) GCN -> OpenCL decompiler.
 *
 * The operation is the one the paper states as its problem ("A method for
 * decompilation of AMD GCN kernels to OpenCL", "Statement of the problem"):
 * a disassembled GCN file goes in, the equivalent OpenCL text comes out.  A
 * file may hold several kernels (the body-extraction algorithm of Listing 2
 * splits them at `.kernel`); unsupported instructions are kept as inline
 * assembly ("Practical implementation").  Every stage of the method runs as a
 * CUDA kernel on one GPU; nothing here falls back to the CPU.
 *
 * Conventions for every call:
 *  - Return value: 0 on success, a negative GCN_E* code on failure.  No call
 *    throws or aborts; a failed CUDA call returns GCN_ECUDA and leaves the
 *    handle usable for gcn_decomp_destroy.
 *  - Host pointers are plain process memory; "device" pointers are CUDA
 *    global-memory addresses on the handle's device.  The caller keeps
 *    ownership of every buffer it passes; the library copies what it needs
 *    before returning (host inputs) or reads it on the given stream (device
 *    inputs) and never frees caller memory.
 *  - Text is bytes, not NUL-terminated; lines end with '\n'.
 *  - One handle owns its device memory, its CUDA streams and its worker
 *    threads.  Every call is thread-safe; different handles are independent.
 *
 * Jobs (submit_batch / fetch_*) are served by continuous batching: admitted
 * jobs queue on the host; each of the handle's worker lanes (a host thread
 * with its own CUDA stream) takes everything queued when it becomes free, up
 * to 64 MiB of text (tuning: batch_mib), and runs it as one batch, so jobs that arrive while
 * others are on the GPU start as soon as a lane frees up, and the batches of
 * different lanes overlap on the device.  A job's result does not depend on
 * which jobs share its batch.
 *
 * Which calls follow a passage of the paper: submit_batch, fetch_opencl,
 * fetch_batch and run_device/result_* carry the operation the paper states
 * (disassembly in, OpenCL out; Listing 2's split of a file into kernels;
 * inline assembly for unsupported instructions).  create, destroy, poll,
 * job_info, fetch_ir, stage_times, stage_totals, run_stats, launches,
 * line_starts_noalloc and last_error are infrastructure of this library
 * (handles, serving, parity access, measurement) with no counterpart in the
 * paper.
 */
#ifndef GCN_DECOMP_H
#define GCN_DECOMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define GCN_OK 0
#define GCN_EINVAL (-1)  /* bad argument (NULL where not allowed, bad size, unknown id) */
#define GCN_ENOMEM (-2)  /* device or host allocation failed, or a size exceeds a limit */
#define GCN_EAGAIN (-3)  /* nothing admitted (memory budget), or the job is not finished */
#define GCN_ENOJOB (-4)  /* unknown or already fetched job id */
#define GCN_ECUDA (-5)   /* a CUDA call failed; the message is in gcn_decomp_last_error */

/* per-kernel status, worst over a file's kernels for a job (numeric max) */
#define GCN_ST_OK 0            /* fully decompiled */
#define GCN_ST_PARTIAL 1       /* inline asm, unstructured control flow or pseudo-code present */
#define GCN_ST_PARSE_ERROR 2   /* malformed configuration, operand, label or exec-mask form */
#define GCN_ST_FIXPOINT_CAP 3  /* a device-side iteration limit was reached */

/* flags */
#define GCN_WAIT 1u            /* gcn_decomp_fetch_opencl: block until the job is done */

typedef struct gcn_decomp gcn_decomp_t; /* opaque */

typedef struct {
  int device;                 /* CUDA device ordinal */
  uint64_t mem_budget_bytes;  /* device memory the handle may hold (0 = no limit) */
  uint32_t max_slots;         /* jobs resident at once (0 = 65536) */
  const char *tuning_file;    /* NULL, or a file of "key=value" lines written by the autotuner:
                                 lanes (worker lanes, 1..8; default 2), batch_mib (text one lane
                                 takes at once; default 64), big_kernel (instructions from which
                                 a kernel is analysed by a thread block instead of a warp;
                                 default 4096); a malformed file makes create fail (GCN_EINVAL).
                                 Test hooks: fail_alloc_jobs=M makes every workspace allocation
                                 of a job batch of more than M jobs fail as if cudaMalloc had
                                 (GCN_ENOMEM inside a lane, which then frees idle memory, retries
                                 and splits the batch); fixpoint_sweeps=S caps the type fixed
                                 point at S sweeps (a kernel still changing in sweep S gets
                                 GCN_ST_FIXPOINT_CAP) */
  uint32_t flags;             /* reserved (0) */
} gcn_decomp_config;

/* Create a handle on cfg->device.  *out receives the handle.  Errors:
 * GCN_EINVAL (NULL cfg/out, bad device), GCN_ECUDA. */
int gcn_decomp_create(const gcn_decomp_config *cfg, gcn_decomp_t **out);

/* Submit n jobs; job i is one disassembly file text[i][0..len[i]).  The
 * library copies the texts before returning (a '\n' is appended when the last
 * line lacks one) and queues them; the call does not wait for the GPU.
 * job_ids[i] receives the id of job i; *n_admitted the number of jobs taken:
 * jobs are admitted in order while a job slot is free (max_slots) and the
 * estimated device memory of admitted, unfetched jobs (48 bytes per input
 * byte + 1 MiB each) stays within mem_budget_bytes; the first job is always
 * admitted when nothing else is.  A job's slot and budget share are given
 * back when it is fetched.
 * Errors: GCN_EINVAL, GCN_EAGAIN (none admitted: no slot or budget). */
int gcn_decomp_submit_batch(gcn_decomp_t *h, const char *const *text, const size_t *len, size_t n,
                            uint64_t *job_ids, size_t *n_admitted);

/* Copy the OpenCL text of a job (its kernels joined by a blank line) into
 * buf[0..cap).  buf == NULL only reports the size.  *len_out = bytes of the
 * text; *status_out = worst GCN_ST_* of the job's kernels (either may be
 * NULL).  With GCN_WAIT the call blocks until the job is done.  On success
 * with buf != NULL the job's slot is released and its id becomes unknown.
 * Errors: GCN_ENOJOB, GCN_EINVAL (cap too small: nothing is copied and the
 * job stays), GCN_EAGAIN (not finished and no GCN_WAIT), or the error of the
 * batch that ran the job (GCN_ENOMEM, GCN_ECUDA; the job is released). */
int gcn_decomp_fetch_opencl(gcn_decomp_t *h, uint64_t job_id, char *buf, size_t cap, size_t *len_out,
                            int *status_out, uint32_t flags);

/* Results of n jobs at once: off_out[0..n] (u64) receives the boundaries
 * of their texts placed back to back in job_ids order, status_out[0..n) (i32,
 * may be NULL) their worst status.  buf == NULL only fills off_out and
 * status_out; otherwise buf[0..cap) receives the texts and all n jobs are
 * released.  With GCN_WAIT the call blocks until every job is done.
 * Errors: as gcn_decomp_fetch_opencl for the first job that has one (nothing
 * is copied or released then). */
int gcn_decomp_fetch_batch(gcn_decomp_t *h, const uint64_t *job_ids, size_t n, char *buf, size_t cap,
                           uint64_t *off_out, int32_t *status_out, uint32_t flags);

/* Ids of finished jobs not yet reported by an earlier poll (and not yet
 * fetched), in completion order: up to cap of them into job_ids, their
 * number into *n_out.  When none is ready the call waits up to timeout_ms
 * (0 = do not wait, negative = no limit).  Errors: GCN_EINVAL. */
int gcn_decomp_poll(gcn_decomp_t *h, uint64_t *job_ids, size_t cap, size_t *n_out, int timeout_ms);

/* State and timestamps of a job not yet fetched: info[0..4] = state (0
 * queued, 1 running, 2 done), submit time, batch start time, finish time
 * (CLOCK_MONOTONIC nanoseconds, 0 = not yet), and 1 when its IR is still
 * resident on the device.  Returns the number of values written (<= cap).
 * Errors: GCN_ENOJOB, GCN_EINVAL. */
int gcn_decomp_job_info(gcn_decomp_t *h, uint64_t job_id, uint64_t *info, int cap);

/* gcn_decomp_job_info for n jobs under one lock (infrastructure: a client
 * that fetches thousands of jobs a second reads their times in one call):
 * info[i * per .. i * per + per) receives the first per (1..5) values for
 * job_ids[i], all zero for a job that is not known (never submitted, or
 * already fetched).  Errors: GCN_EINVAL (h or a pointer NULL with n > 0, per
 * outside 1..5); nothing is written then. */
int gcn_decomp_job_info_batch(gcn_decomp_t *h, const uint64_t *job_ids, size_t n, uint64_t *info, int per);

/* Intermediate arrays of a job, for parity checks: `which` selects
 *   0 instruction records (32 bytes each: u16 op, u8 nops, u8 flags, u32 imm,
 *     u32 target, u32 operand[5]),
 *   1 physical block of each instruction (u32),  2 physical blocks (u32 first,end,succ0,succ1),
 *   3 logical block of each instruction (u32, 0xFFFFFFFF = exec bookkeeping),
 *   4 logical blocks (as 2),  5 per-kernel configuration header (8 x u32:
 *     dims, cws x/y/z, sgprs, vgprs, useargs, user args)
 * concatenated over the job's kernels in file order.  Sizes as for fetch.
 * Waits for the job; does not release it.  The IR stays on the device until
 * the job is fetched, unless the memory budget runs out or more than 32
 * batches are finished and unfetched (then the oldest batches' IR is dropped
 * and this returns GCN_ENOJOB).  Errors: GCN_ENOJOB, GCN_EINVAL. */
int gcn_decomp_fetch_ir(gcn_decomp_t *h, uint64_t job_id, int which, void *buf, size_t cap, size_t *len_out);

/* Stop the worker lanes (a batch already on the GPU finishes; queued jobs are
 * dropped), wait for in-flight work and free every resource of the handle
 * (NULL is a no-op). */
void gcn_decomp_destroy(gcn_decomp_t *h);

/* Device-resident batch: decompile n_files files already in device memory,
 * file f = d_text[d_file_off[f] .. d_file_off[f+1]), each ending with '\n',
 * total at most 4 GiB.  Work is queued on `stream` (a cudaStream_t, NULL =
 * the handle's stream) and the call returns without synchronising; results
 * stay in the handle's device memory until the next run_device call.
 * Errors: GCN_EINVAL, GCN_ENOMEM, GCN_ECUDA. */
int gcn_decomp_run_device(gcn_decomp_t *h, const uint8_t *d_text, uint64_t text_len, const uint64_t *d_file_off,
                          uint64_t n_files, void *stream);

/* Results of the last run_device call, as device pointers owned by the
 * handle: d_out = concatenated OpenCL text, d_out_off = u64[n_files+1] byte
 * offsets per file, d_status = i32[n_files] worst status per file; *out_bytes
 * = total text size (synchronises the stream).  Errors: GCN_EINVAL (no run). */
int gcn_decomp_result_device(gcn_decomp_t *h, const uint8_t **d_out, const uint64_t **d_out_off,
                             const int32_t **d_status, uint64_t *out_bytes);

/* Copy files [f0, f1) of the last run_device result to host memory:
 * buf[0..cap) receives their OpenCL text back to back, off_out[0..f1-f0]
 * (u64, relative to buf) their boundaries, status_out[0..f1-f0) (i32) their
 * worst status; either array may be NULL.  buf == NULL only fills off_out.
 * Synchronises the handle's stream.  Errors: GCN_EINVAL (no run, bad range,
 * cap too small), GCN_ECUDA. */
int gcn_decomp_result_copy(gcn_decomp_t *h, uint64_t f0, uint64_t f1, void *buf, size_t cap, uint64_t *off_out,
                           int32_t *status_out);

/* Per-stage device times of the last finished run of either form
 * (milliseconds, CUDA events on the run's stream), stage names in *names
 * (static strings): the ten stages S1..S13, then six kernels alone (the S1
 * newline scan, S4 decoding, S7 node building, the two S9-S10 node-cache
 * passes, S13 statement printing; 0 when a run did not launch one).  A
 * device-resident run counts as finished once result_device was called or
 * the next run_device passed its first synchronisation.  Returns the number
 * of stages (<= cap) or a negative code. */
int gcn_decomp_stage_times(gcn_decomp_t *h, float *ms, const char **names, int cap);

/* The times of gcn_decomp_stage_times summed over every device-resident run
 * (run_device) since the handle was created or the sums were last reset;
 * *runs (may be NULL) receives the number of runs summed.  The call waits for
 * the runs still in flight on the device.  reset != 0 clears the sums after
 * they are read.  Returns the number of stages (<= cap) or a negative code. */
int gcn_decomp_stage_totals(gcn_decomp_t *h, double *ms, const char **names, int cap, uint64_t *runs, int reset);

/* Sizes of the last pipeline run (either form): out[0..8] = lines, kernels,
 * instructions, labels, physical blocks, logical blocks, register-state
 * words, output bytes, device bytes held by the engine that ran it; then two
 * values of the handle: out[9] = the most device bytes its workspaces have
 * held at once (never above mem_budget_bytes when that is set), out[10] = job
 * batches split after an allocation failure.  Returns the number of values
 * written (<= cap) or a negative code. */
int gcn_decomp_run_stats(gcn_decomp_t *h, uint64_t *out, int cap);

/* Number of CUDA kernels the library launched for the last pipeline run
 * (either form); 0 before the first run. */
uint64_t gcn_decomp_launches(gcn_decomp_t *h);

/* Line tokenisation without any allocation (the paper has no counterpart:
 * this is a service for callers, not a step of the method).
 *
 * For callers that cannot let a library allocate device memory (code running
 * while their own CUDA graph is being captured, where cudaMalloc is not
 * allowed; a process whose memory pool owns all device memory; a real-time
 * path that must not block on the allocator).  It runs the S1 newline scan of
 * the batch pipeline on a text already in device memory, with its scratch in
 * a fixed 256 KiB array compiled into the library instead of handle memory.
 * No handle is needed; nothing is allocated by the CUDA runtime or any
 * library.
 *
 *  d_text[0..text_len)   device bytes of the current device (any alignment;
 *                        16-byte aligned is faster), at most 1 GiB.
 *  d_line_start[0..line_cap)  device u32, receives the byte offset of every
 *                        line start: [0] = 0, [k] = 1 + offset of the k-th
 *                        '\n' (so a text ending with '\n' yields lines+1
 *                        entries).  Needs line_cap >= 1 + number of '\n'.
 *  d_result[0..2)        device u32: [0] = number of '\n' bytes, [1] = error
 *                        bits (0 = ok; 4 = line_cap too small, the offsets
 *                        past it were not written; 1 or 2 = a bounded
 *                        device-side wait gave up, the output is invalid).
 *  stream                cudaStream_t (NULL = legacy default stream).
 *
 * Work is queued on `stream` and the call returns without synchronising;
 * read d_result after the stream has finished.  Runs on the calling thread's
 * current device.  The first call on a device looks the scratch address up
 * once (that may load the module): make it before any stream capture starts.
 * The scratch is shared by all calls on a device, so calls whose device work
 * could overlap (other streams, other threads) must be serialised by the
 * caller; overlapping calls race and give wrong results.  The cached address
 * belongs to the device's primary context: do not call this across a
 * cudaDeviceReset of the device (the cache would point into the old context).
 * Errors: GCN_EINVAL (NULL pointer, line_cap 0), GCN_ENOMEM (text longer
 * than 1 GiB: rejected before anything is queued), GCN_ECUDA. */
int gcn_decomp_line_starts_noalloc(const uint8_t *d_text, uint64_t text_len, uint32_t *d_line_start,
                                   uint64_t line_cap, uint32_t *d_result, void *stream);

/* Last error message of this thread (static storage; never NULL). */
const char *gcn_decomp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GCN_DECOMP_H */
