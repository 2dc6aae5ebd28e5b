// capi.cu — host runtime of the CUDA stages and the C ABI of gcn_decomp.h.
//
// An Engine is one execution context of the pipeline: a grow-only workspace of
// device arrays, stage events and pinned counters.  One pipeline run takes a
// batch of files resident in device memory and executes the stages in order:
// S1 newline scan, S2 row segmentation, S3 configuration, S4 decoding, S5
// physical CFG, S6 logical CFG, S7/S8 dataflow, S9-S11 analysis, S12 regions,
// S13 emission.  The host reads back a few counters between stages (lines,
// kernels/instructions, blocks, output bytes) to size the next arrays;
// everything else stays on the device.
//
// A handle runs two kinds of work:
//  - the device-resident form (run_device): one engine on the handle's
//    stream, input and output in device memory;
//  - jobs (submit_batch / fetch_*): a continuous-batching service.  Jobs are
//    admitted under the slot limit and the device-memory budget and queued;
//    each worker lane (a host thread with its own CUDA stream and pinned
//    staging buffers) takes everything queued when it becomes free (up to a
//    batch limit), stages it, runs the pipeline on an engine of a pool and
//    publishes the results, so batches of different lanes overlap on the
//    device.  A finished batch keeps its engine (and so its IR) until all its
//    jobs are fetched; only when the pool is at its limit or the memory
//    budget runs out is the IR of the oldest finished batches dropped (their
//    texts stay fetchable).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gcn_decomp.h"
#include "gd_kernels.h"

using namespace gd;

namespace {

thread_local std::string g_err = "no error";
void set_err(const std::string& s) { g_err = s; }

#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      set_err(std::string(#x) + ": " + cudaGetErrorString(e_));                 \
      throw GCN_ECUDA;                                                          \
    }                                                                           \
  } while (0)

struct Workspace {
  struct Buf {
    void* p = nullptr;
    size_t cap = 0;
  };
  std::map<std::string, Buf> bufs;
  size_t total = 0;
  uint64_t budget = 0;                         // device bytes all workspaces of a handle may hold (0 = no limit)
  std::atomic<uint64_t>* pool = nullptr;       // bytes held by all workspaces of the handle
  std::atomic<uint64_t>* peak = nullptr;       // the most *pool has ever been
  uint32_t fail_jobs = 0;   // test hook: with more jobs than this in the batch, allocations fail (0 = off)
  uint32_t cur_jobs = 0;    // jobs of the batch being run (0: a device-resident run)
  template <class T>
  T* get(const char* name, size_t n) {
    size_t bytes = std::max<size_t>(n * sizeof(T), 256);
    Buf& b = bufs[name];
    if (b.cap < bytes) {
      if (b.p) {
        cudaFree(b.p);
        total -= b.cap;
        if (pool) *pool -= b.cap;
        b.p = nullptr;
        b.cap = 0;
      }
      const uint64_t want = bytes + bytes / 8;
      // reserve the bytes against the budget before allocating: the lanes of a
      // handle allocate concurrently, and a separate check and add would let
      // two of them pass the check together and overshoot the budget
      if (pool) {
        uint64_t cur = pool->load();
        do {
          if (budget && cur + want > budget) {
            set_err(std::string("memory budget exceeded allocating ") + name);
            throw GCN_ENOMEM;
          }
        } while (!pool->compare_exchange_weak(cur, cur + want));
        if (peak) {
          uint64_t pk = peak->load();
          while (cur + want > pk && !peak->compare_exchange_weak(pk, cur + want)) {
          }
        }
      }
      const bool fake_fail = fail_jobs && cur_jobs > fail_jobs;
      if (fake_fail || cudaMalloc(&b.p, want) != cudaSuccess) {
        if (!fake_fail) cudaGetLastError();
        if (pool) *pool -= want;
        b.p = nullptr;
        set_err(std::string(fake_fail ? "allocation refused by the fail_alloc_jobs test hook for "
                                      : "cudaMalloc failed for ") + name);
        throw GCN_ENOMEM;
      }
      b.cap = want;
      total += want;
    }
    return (T*)b.p;
  }
  void release() {
    for (auto& kv : bufs)
      if (kv.second.p) cudaFree(kv.second.p);
    bufs.clear();
    if (pool) *pool -= total;
    total = 0;
  }
};

const char* kStageNames[] = {"S1 tokenise", "S2 segment", "S3 config", "S4 decode", "S5 cfg", "S6 logical cfg",
                             "S7-S8 dataflow", "S9-S11 analysis", "S12 regions", "S13 emit",
                             // the longest kernels alone (KTimed order)
                             "k_line_scan (S1)", "k_decode (S4)", "k_nodes (S7)", "k_node_fwd (S9-S10)",
                             "k_node_cache (S9-S10)", "k_items (S13 print)"};
constexpr int kStages = 10;
constexpr int kTimings = kStages + KT_COUNT;  // the stages, then the timed kernels
static_assert(sizeof(kStageNames) / sizeof(kStageNames[0]) == kTimings, "one name per timing");

// The events of one pass: stage boundaries, the region reduction's own stream,
// the timed kernels.  An engine alternates between two sets, so that the times
// of a pass are read (at the first synchronisation of the next pass) without
// stalling the device between passes.
struct PassEvents {
  cudaEvent_t st[kStages + 1] = {};
  cudaEvent_t rs[2] = {};
  KernelTimer kt{};
  bool pending = false;  // recorded by a finished pass whose times are not yet read
};

// The type lattice is finite and every sweep of the fixed point that changes
// something raises a type, so this limit is never reached by a real kernel; a
// smaller one (the tuning file's fixpoint_sweeps, a test hook) caps kernels.
constexpr uint32_t kTypeSweeps = 100000;

struct Run {
  bool valid = false;
  Batch b{};
  std::vector<KHdr> kh;           // host copy (after the run)
  std::vector<uint32_t> file_k0;  // first kernel of each file (F + 1)
  uint64_t out_bytes = 0;
};

// one execution context of the pipeline
struct Engine {
  Workspace ws;
  Run run;
  PassEvents pe[2];
  int cur = 0;                 // the set of the latest pass
  float stage_ms[kTimings] = {0};  // the latest pass whose events were read
  double sum_ms[kTimings] = {0};   // summed over the passes read since the last reset
  uint64_t sum_runs = 0;
  uint64_t launches = 0;
  uint32_t* h_tot = nullptr;  // pinned counters
  uint32_t big_kernel = 4096;  // size-bucket threshold
  uint32_t type_sweeps = kTypeSweeps;  // sweep limit of the type fixed point
  SideStream fk{};             // second stream for launches that overlap the main one
  SideStream rs{};             // stream of the region reduction (S12), beside S7-S11
  // job service: the batch whose IR the workspace holds and its unfetched jobs
  uint64_t batch = 0;
  uint32_t live = 0;
  bool busy = false;
};

enum JobState : int { JOB_PENDING = 0, JOB_RUNNING = 1, JOB_DONE = 2 };

struct JobRec {
  const uint8_t* in = nullptr;  // input file text in a pinned slab (ends with '\n'); until run
  size_t in_len = 0;
  int slab = -1;                // the slab holding it
  std::string text;  // OpenCL output
  int status = 0;
  int rc = GCN_OK;   // a batch failure reported at fetch
  int state = JOB_PENDING;
  uint64_t est = 0;  // device bytes charged to the budget at admission
  uint64_t t_submit = 0, t_start = 0, t_done = 0;
  Engine* eng = nullptr;  // engine holding the job's IR (null = not resident)
  uint64_t batch = 0;
  uint32_t run_file = 0;
};

// a worker: host thread, CUDA stream, pinned staging buffers
struct Lane {
  std::thread th;
  cudaStream_t stream = nullptr;
  uint8_t* h_in = nullptr;
  size_t h_in_cap = 0;
  uint8_t* h_out = nullptr;
  size_t h_out_cap = 0;
  uint64_t* h_off = nullptr;  // file offsets in, then file output offsets out
  size_t h_off_cap = 0;
  int32_t* h_st = nullptr;
  size_t h_st_cap = 0;
};

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Runtime parameters of a handle (defaults, or a tuning file written by the
// project's autotuner: `lanes=`, `batch_mib=`, `big_kernel=` lines).
struct Tuning {
  int lanes = 2;                     // worker lanes of the job service
  uint64_t batch_bytes = 64ull << 20;  // text bytes one lane takes at once
  uint32_t big_kernel = 4096;        // kernels of this many instructions or more get a thread block
  uint32_t fail_alloc_jobs = 0;      // test hook: batches of more jobs fail every workspace allocation
  uint32_t type_sweeps = kTypeSweeps;  // test hook (fixpoint_sweeps): sweep limit of the type fixed point
};
constexpr int kMaxLanes = 8;
// Job texts are copied once, at submit, into pinned host slabs; a batch whose
// texts are contiguous in one slab goes to the device with one copy.  A slab is
// reused when none of its jobs is left to run.
struct Slab {
  uint8_t* p = nullptr;
  size_t cap = 0, used = 0;
  uint32_t refs = 0;  // jobs whose text is in the slab and not yet run
};
constexpr size_t kSlabBytes = 256ull << 20;
// engines of the job service: a finished batch keeps its engine (its IR) until
// its jobs are fetched; the pool grows up to this many, and beyond it (or when
// the memory budget runs out) the IR of the oldest finished batches is dropped
constexpr int kMaxEngines = 32;
constexpr uint64_t kEstPerTextByte = 48;  // device bytes per input byte (admission estimate)
constexpr uint64_t kEstPerJob = 1ull << 20;

bool read_tuning(const char* path, Tuning* t) {
  FILE* f = fopen(path, "r");
  if (!f) {
    set_err(std::string("cannot open tuning file ") + path);
    return false;
  }
  char line[256];
  bool ok = true;
  while (ok && fgets(line, sizeof line, f)) {
    char* p = line;
    while (*p == ' ' || *p == '\t') ++p;
    if (*p == '#' || *p == '\n' || *p == '\r' || !*p) continue;
    char key[64];
    unsigned long long v = 0;
    if (sscanf(p, "%63[a-z_] = %llu", key, &v) != 2) {
      ok = false;
      break;
    }
    const std::string k = key;
    if (k == "lanes" && v >= 1 && v <= (unsigned long long)kMaxLanes) t->lanes = (int)v;
    else if (k == "batch_mib" && v >= 1 && v <= 4095) t->batch_bytes = v << 20;
    else if (k == "big_kernel" && v >= 32 && v <= (1ull << 26)) t->big_kernel = (uint32_t)v;
    else if (k == "fail_alloc_jobs" && v <= (1ull << 31)) t->fail_alloc_jobs = (uint32_t)v;
    else if (k == "fixpoint_sweeps" && v >= 1 && v <= kTypeSweeps) t->type_sweeps = (uint32_t)v;
    else ok = false;
  }
  fclose(f);
  if (!ok) set_err(std::string("malformed tuning file ") + path);
  return ok;
}

}  // namespace

struct gcn_decomp {
  int device = 0;
  cudaStream_t stream = nullptr;
  // device-resident form
  std::mutex dmu;
  Engine direct;
  cudaStream_t direct_stream = nullptr;  // stream of the last run_device call
  uint64_t run_id = 0;
  // job service
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<uint64_t, JobRec> jobs;
  std::deque<uint64_t> pending;
  std::deque<uint64_t> done_q;  // finished jobs not yet reported by poll
  std::vector<std::unique_ptr<Engine>> engines;
  std::vector<std::unique_ptr<Lane>> lanes;
  bool stop = false;
  uint64_t next_job = 1, next_batch = 1;
  uint32_t max_slots = 65536;
  uint64_t budget = 0;
  Tuning tune;
  uint64_t admitted = 0;  // estimated device bytes of admitted, unfetched jobs
  std::vector<Slab> slabs;
  std::atomic<uint64_t> pool{0};
  std::atomic<uint64_t> pool_peak{0};
  std::atomic<uint64_t> splits{0};  // batches split after an allocation failure
  // most recent completed pipeline run (either form)
  std::mutex smu;
  float last_ms[kTimings] = {0};
  uint64_t last_stats[9] = {0};
  uint64_t last_launches = 0;
};

namespace {

// Read the times of the pass recorded in event set `set` (waiting for it) and
// add them to the engine's sums; a set is read once.
void fold_times(Engine* E, int set) {
  PassEvents& p = E->pe[set];
  if (!p.pending) return;
  p.pending = false;
  CK(cudaEventSynchronize(p.st[kStages]));
  float ms[kTimings] = {0};
  for (int i = 0; i < kStages; ++i) cudaEventElapsedTime(&ms[i], p.st[i], p.st[i + 1]);
  cudaEventElapsedTime(&ms[8], p.rs[0], p.rs[1]);  // S12 ran on its own stream
  for (int w = 0; w < KT_COUNT; ++w)
    if (cudaEventElapsedTime(&ms[kStages + w], p.kt.ev[2 * w], p.kt.ev[2 * w + 1]) != cudaSuccess) ms[kStages + w] = 0;
  cudaGetLastError();
  for (int i = 0; i < kTimings; ++i) {
    E->stage_ms[i] = ms[i];
    E->sum_ms[i] += ms[i];
  }
  ++E->sum_runs;
}

// points the launchers' kernel timer at a pass's events for the scope of the pass
struct TimerScope {
  explicit TimerScope(KernelTimer* t) { kernel_timer() = t; }
  ~TimerScope() { kernel_timer() = nullptr; }
};

// the whole pipeline on a device-resident batch
void run_pipeline(Engine* h, const uint8_t* text, uint64_t n, const uint64_t* file_off, uint32_t F,
                  cudaStream_t s) {
  Workspace& W = h->ws;
  Run& R = h->run;
  R.valid = false;
  const uint64_t launches0 = launch_counter();
  // this pass records into the other event set; the set's previous pass (two
  // passes ago) is read first, and the last pass's after the first read-back
  h->cur ^= 1;
  fold_times(h, h->cur);
  PassEvents& pe = h->pe[h->cur];
  cudaEvent_t* ev = pe.st;
  TimerScope timer_scope(&pe.kt);
  for (int w = 0; w < KT_COUNT; ++w) {  // a kernel a pass does not launch reads 0 ms
    CK(cudaEventRecord(pe.kt.ev[2 * w], s));
    CK(cudaEventRecord(pe.kt.ev[2 * w + 1], s));
  }
  Batch& b = R.b;
  b = Batch{};
  b.text = text;
  b.text_len = n;
  b.file_off = file_off;
  b.F = F;
  b.big_kernel = h->big_kernel;
  b.type_sweeps = h->type_sweeps;
  uint32_t* tot = W.get<uint32_t>("totals", 16);
  uint32_t* err = W.get<uint32_t>("err", 4);
  b.err = err;
  CK(cudaMemsetAsync(err, 0, 16, s));
  CK(cudaMemsetAsync(tot, 0, 64, s));
  auto sync_totals = [&]() {
    CK(cudaMemcpyAsync(h->h_tot, tot, 64, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  };
  CK(cudaEventRecord(ev[0], s));
  // S1
  uint32_t* line_start = W.get<uint32_t>("line_start", n + 2);
  uint64_t* tstat = W.get<uint64_t>("tile_status", std::max<uint64_t>(line_scan_tiles(n), scan_tiles((uint32_t)n + 1)) + 64);
  uint32_t* counters = W.get<uint32_t>("counters", 4);
  LineScan2 two{};
  if (const uint32_t lt = line_scan_tiles(n) - 1; lt > kLsOnePass) {
    two.masks = W.get<uint16_t>("ls_masks", (size_t)lt * (kLsTileBytes / 16));
    two.counts = W.get<uint32_t>("ls_counts", lt);
    two.prefix = W.get<uint32_t>("ls_prefix", lt);
  }
  launch_line_scan(text, n, line_start, tstat, counters, err, two, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[1], s));
  uint32_t L = 0;
  CK(cudaMemcpyAsync(&h->h_tot[8], counters + 1, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  L = h->h_tot[8];
  b.L = L;
  fold_times(h, h->cur ^ 1);  // the previous pass (complete: read-backs wait for the stream)
  b.line_start = line_start;
  ScanScratch sc{tstat, W.get<uint32_t>("scan_counter", 4)};
  // S2
  RowArrays ra;
  ra.file_start = W.get<uint8_t>("file_start", L + 1);
  ra.kind = W.get<uint8_t>("kind", L + 1);
  ra.rowtype = W.get<uint8_t>("rowtype", L + 1);
  ra.t0 = W.get<uint32_t>("t0", L + 1);
  ra.t1 = W.get<uint32_t>("t1", L + 1);
  ra.t2 = W.get<uint32_t>("t2", L + 1);
  ra.mkmax = W.get<uint32_t>("mkmax", L + 1);
  ra.fsmax = W.get<uint32_t>("fsmax", L + 1);
  ra.kcnt = W.get<uint32_t>("kcnt", L + 1);
  ra.instr_excl = W.get<uint32_t>("instr_excl", L + 1);
  ra.label_excl = W.get<uint32_t>("label_excl", L + 1);
  ra.cfg_excl = W.get<uint32_t>("cfg_excl", L + 1);
  uint64_t* status3 = W.get<uint64_t>("tile_status3", scan3_status_words(L) + 8);
  if (L) launch_rows(text, line_start, L, file_off, F, ra, sc, status3, tot, err, s);
  CK(cudaGetLastError());
  sync_totals();
  b.K = h->h_tot[0];
  b.I = h->h_tot[1];
  if (b.K <= kBlockPerKernelBatch) b.big_kernel = 0;  // every kernel its own thread block
  b.NL = h->h_tot[2];
  b.NC = h->h_tot[14];
  b.rowtype = ra.rowtype;
  b.file_start = ra.file_start;
  b.kind = ra.kind;
  b.kcnt = ra.kcnt;
  b.kh = W.get<KHdr>("kh", b.K + 1);
  b.args = W.get<ArgRec>("args", (size_t)b.K * kMaxArgs + 1);
  b.instr_line = W.get<uint32_t>("instr_line", b.I + 1);
  b.label_line = W.get<uint32_t>("label_line", b.NL + 1);
  b.label_instr = W.get<uint32_t>("label_instr", b.NL + 1);
  b.label_hash = W.get<uint32_t>("label_hash", b.NL + 1);
  b.label_tab_mask = 1;
  while (b.label_tab_mask + 1 < 2ull * b.NL) b.label_tab_mask = 2 * b.label_tab_mask + 1;
  b.label_tab = W.get<uint32_t>("label_tab", (size_t)b.label_tab_mask + 1);
  b.cfg_line = W.get<uint32_t>("cfg_line", b.NC + 1);
  if (L) launch_scatter_rows(L, ra, b.instr_line, b.label_line, b.label_instr, b.cfg_line, b.kh, s);
  CK(cudaEventRecord(ev[2], s));
  // S3
  launch_config(b, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[3], s));
  // S4 + S5
  b.ikern = W.get<uint32_t>("ikern", b.I + 1);
  b.blen = W.get<uint32_t>("blen", b.I + 1);
  b.ins = W.get<InstrRec>("ins", b.I + 1);
  b.branch_hash = W.get<uint32_t>("branch_hash", b.I + 1);
  b.branch_pos = W.get<uint32_t>("branch_pos", b.I + 1);
  b.pleader = W.get<uint32_t>("pleader", b.I + 1);
  b.lleader = W.get<uint32_t>("lleader", b.I + 1);
  b.pblock_of = W.get<uint32_t>("pblock_of", b.I + 1);
  launch_decode(b, sc, tot, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[4], s));
  sync_totals();
  b.NPB = h->h_tot[3];
  b.pblocks = W.get<BlockRec>("pblocks", b.NPB + 1);
  uint32_t* blk_kern = W.get<uint32_t>("blk_kern", std::max(b.NPB, b.I) + 1);
  launch_pblocks(b, blk_kern, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[5], s));
  // S6
  b.ctl = W.get<uint8_t>("ctl", b.I + 1);
  b.sense = W.get<uint8_t>("sense", b.I + 1);
  b.ltarget = W.get<uint32_t>("ltarget", b.I + 1);
  b.lblock_of = W.get<uint32_t>("lblock_of", b.I + 1);
  b.exec_list = W.get<uint32_t>("exec_list", b.I + 1);
  launch_logical(b, sc, tot, s);
  CK(cudaGetLastError());
  sync_totals();
  b.NLB = h->h_tot[4];
  b.lblocks = W.get<BlockRec>("lblocks", b.NLB + 1);
  b.lterm = W.get<uint32_t>("lterm", b.NLB + 1);
  launch_lblocks(b, blk_kern, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[6], s));
  // S7 + S8
  DfScratch d{};
  d.kstate = W.get<uint32_t>("kstate", b.K + 1);
  d.kstate_off = W.get<uint32_t>("kstate_off", b.K + 1);
  d.kbits = W.get<uint32_t>("kbits", b.K + 1);
  d.bits_off = W.get<uint32_t>("bits_off", b.K + 1);
  d.pcount = W.get<uint32_t>("pcount", b.NLB + 2);
  d.blk_kern = blk_kern;
  b.fused = W.get<uint8_t>("fused", b.I + 1);
  b.co_idx = W.get<uint32_t>("co_idx", b.I + 1);
  b.pred_off = W.get<uint32_t>("pred_off", b.NLB + 2);
  b.pred_fill = W.get<uint32_t>("pred_fill", b.NLB + 1);
  launch_df_counts(b, d, sc, tot, s);
  CK(cudaGetLastError());
  sync_totals();
  // S12 needs the logical CFG and the parse flags only, final once the sizes above are taken:
  // it runs on its own stream beside S7-S11
  b.rg = W.get<uint32_t>("regions", 12ull * kRegionsPerBlock * b.NLB + 24);
  b.brk = W.get<uint32_t>("break_of", b.NLB + 1);
  // region reduction work: 64 words per block + 128 per kernel (red_work_words)
  uint32_t* rwork = W.get<uint32_t>("rg_work", 64ull * b.NLB + 128ull * b.K + 64);
  uint32_t* rstk = W.get<uint32_t>("rg_stack", (size_t)kStackPerBlock * b.NLB + 4);
  uint8_t* alive = W.get<uint8_t>("rg_alive", (size_t)kRegionsPerBlock * b.NLB + 2);
  uint8_t* cond = W.get<uint8_t>("rg_cond", b.NLB + 1);
  CK(cudaEventRecord(h->rs.fork, s));
  CK(cudaStreamWaitEvent(h->rs.side, h->rs.fork, 0));
  CK(cudaEventRecord(pe.rs[0], h->rs.side));
  launch_regions(b, rwork, rstk, alive, cond, h->rs.side);
  CK(cudaGetLastError());
  CK(cudaEventRecord(pe.rs[1], h->rs.side));
  CK(cudaEventRecord(h->rs.join, h->rs.side));
  b.NS = h->h_tot[5];
  d.NW = h->h_tot[6];
  uint32_t NE = h->h_tot[7];
  b.preds = W.get<uint32_t>("preds", NE + 1);
  b.idom = W.get<uint32_t>("idom", b.NLB + 1);
  b.rpo = W.get<uint32_t>("rpo", b.NLB + 1);
  b.scratch32 = W.get<uint32_t>("scratch32", b.NLB + 1);
  d.rpo_index = W.get<uint32_t>("rpo_index", b.NLB + 1);
  d.stack = W.get<uint32_t>("dfs_stack", b.NLB + 1);
  d.child = W.get<uint8_t>("dfs_child", b.NLB + 1);
  b.st_in = W.get<uint32_t>("st_in", b.NS + 1);
  b.st_out = W.get<uint32_t>("st_out", b.NS + 1);
  b.has_phi = W.get<uint8_t>("has_phi", b.NS + 1);
  d.defbits = W.get<uint32_t>("defbits", d.NW + 1);
  d.phibits = W.get<uint32_t>("phibits", d.NW + 1);
  d.rows = W.get<uint32_t>("rows", b.NS + 1);
  b.nodes = W.get<Node>("nodes", 4ull * b.I + 4);
  launch_df_main(b, d, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[7], s));
  // S9 - S11
  b.ncls = W.get<uint8_t>("ncls", 4ull * b.I + 4);
  b.nclsk = W.get<uint8_t>("nclsk", 4ull * b.I + 4);
  b.nsrcf = W.get<uint32_t>("nsrcf", 12ull * b.I + 12);
  b.mem_arg = W.get<uint32_t>("mem_arg", b.I + 1);
  b.mem_idx = W.get<uint32_t>("mem_idx", b.I + 1);
  launch_node_cache(b, W.get<uint8_t>("kviews", 2 * (size_t)b.K * kview_bytes() + 16), s);
  b.uses = W.get<uint32_t>("uses", 4ull * b.I + 4);
  b.nflag = W.get<uint8_t>("nflag", 4ull * b.I + 4);
  b.ntype = W.get<uint8_t>("ntype", 4ull * b.I + 4);
  b.var_of = W.get<int32_t>("var_of", 4ull * b.I + 4);
  b.phi_used = W.get<uint8_t>("phi_used", b.NS + 1);
  b.plist = d.rows;  // the dataflow rows are dead once the nodes exist
  b.phi_type = W.get<uint8_t>("phi_type", b.NS + 1);
  b.phi_var = W.get<int32_t>("phi_var", b.NS + 1);
  b.var_type = W.get<uint8_t>("var_type", 4ull * b.I + b.NS + 4);
  b.dyn_count = W.get<uint32_t>("dyn_count", b.K + 1);
  uint32_t* wlsz = W.get<uint32_t>("wl_size", b.K + 1);
  uint32_t* wloff = W.get<uint32_t>("wl_off", b.K + 1);
  launch_wl_size(b, wlsz, wloff, sc, &tot[9], s);
  sync_totals();
  uint32_t* wl = W.get<uint32_t>("wl", (size_t)h->h_tot[9] + 8);
  uint64_t nbw = 3 * ((4ull * b.I + 63) / 32) + (b.NS + 63) / 32 + 4;
  uint32_t* bits = W.get<uint32_t>("reach_bits", nbw);
  const uint64_t nvc = (uint64_t)b.NS + 4ull * b.I + 1;  // variable candidates (+ end)
  uint32_t* vflag = W.get<uint32_t>("var_flag", nvc);
  uint32_t* vpos = W.get<uint32_t>("var_pos", nvc);
  ScanScratch scv = sc;
  if (scan_tiles((uint32_t)nvc) + 64 > std::max<uint64_t>(line_scan_tiles(n), scan_tiles((uint32_t)n + 1)) + 64)
    scv.status = W.get<uint64_t>("tile_status_var", scan_tiles((uint32_t)nvc) + 64);
  // the kernels longest first, for the work queues of the per-kernel stages
  KernelOrder ko{W.get<uint32_t>("kernel_order", (size_t)b.K + 1), W.get<uint32_t>("kernel_order_info", 4),
                 W.get<uint32_t>("work_queue_heads", 8)};
  launch_kernel_order(b, ko, s);
  launch_analysis(b, wl, bits, nbw, blk_kern, vflag, vpos, scv, h->fk, ko, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[8], s));
  // S12, launched beside S7-S11, joined here
  CK(cudaStreamWaitEvent(s, h->rs.join, 0));
  CK(cudaEventRecord(ev[9], s));
  // S13: layout (count, scan, write), item sizes, scan, item text
  b.kout_off = W.get<uint32_t>("kout_off", b.K + 1);
  uint32_t* icnt = W.get<uint32_t>("item_cnt", b.K + 1);
  uint32_t* ibase = W.get<uint32_t>("item_base", b.K + 1);
  const uint32_t* pbits = bits + 3 * ((4ull * b.I + 63) / 32);  // used join versions (reachability)
  // copies on every CFG edge into a join block
  b.cs_off = W.get<uint32_t>("cs_off", 2ull * b.NLB + 1);
  b.cs_cnt = W.get<uint32_t>("cs_cnt", 2ull * b.NLB + 1);
  b.cs_cyc = W.get<uint8_t>("cs_cyc", 2ull * b.NLB + 1);
  launch_copy_sets(b, blk_kern, pbits, b.cs_cnt, 0, s);  // bounds, then their scan
  if (b.NLB) launch_scan(b.cs_cnt, b.cs_off, 2 * b.NLB + 1, 0, false, sc, &tot[10], b.err, s);
  // layout slices: bounds and their scan (the total has a host-side bound)
  uint32_t* loff = W.get<uint32_t>("layout_off", b.K + 1);
  launch_layout(b, nullptr, loff, nullptr, nullptr, 0, s);
  if (b.K) launch_scan(loff, loff, b.K, 0, false, sc, &tot[14], b.err, s);
  CK(cudaGetLastError());
  sync_totals();
  const uint32_t NCS = b.NLB ? h->h_tot[10] : 0;
  const uint32_t LUB = b.K ? h->h_tot[14] : 0;
  b.cs_reg = W.get<uint32_t>("cs_reg", (size_t)NCS + 1);
  uint32_t* cs_src = W.get<uint32_t>("cs_src", (size_t)NCS + 1);
  launch_copy_sets(b, blk_kern, pbits, cs_src, 1, s);
  Item* lstage = W.get<Item>("layout_stage", (size_t)LUB + 1);
  launch_layout(b, lstage, loff, icnt, rstk, 1, s);
  if (b.K) launch_scan(icnt, ibase, b.K, 0, false, sc, &tot[10], b.err, s);
  CK(cudaGetLastError());
  sync_totals();
  uint32_t NI = b.K ? h->h_tot[10] : 0;
  Item* items = W.get<Item>("items", (size_t)NI + 1);
  launch_items_place(lstage, loff, b.K, LUB, icnt, ibase, items, s);
  uint32_t* iw = W.get<uint32_t>("item_weight", (size_t)NI + 1);
  uint32_t* sub0 = W.get<uint32_t>("item_sub0", (size_t)NI + 1);
  uint32_t* pflag = W.get<uint32_t>("print_flag", (size_t)b.I + 1);
  uint32_t* prank = W.get<uint32_t>("print_rank", (size_t)b.I + 1);
  uint32_t* plist = W.get<uint32_t>("print_instr", (size_t)b.I + 1);
  launch_print_list(b, pflag, nullptr, nullptr, 0, s);
  launch_scan(pflag, prank, b.I + 1, 0, false, sc, nullptr, b.err, s);
  launch_print_list(b, pflag, prank, plist, 1, s);
  launch_subitems(b, items, NI, prank, iw, nullptr, nullptr, 0, 0, s);
  if (NI) launch_scan(iw, sub0, NI, 0, false, sc, &tot[12], b.err, s);
  CK(cudaGetLastError());
  sync_totals();
  const uint32_t NS2 = NI ? h->h_tot[12] : 0;
  CK(cudaMemcpyAsync(sub0 + NI, &tot[12], 4, cudaMemcpyDeviceToDevice, s));
  ScanScratch sc2 = sc;
  if (scan_tiles(NS2 + 1) + 64 > std::max<uint64_t>(line_scan_tiles(n), scan_tiles((uint32_t)n + 1)) + 64)
    sc2.status = W.get<uint64_t>("tile_status_sub", scan_tiles(NS2 + 1) + 64);
  uint32_t* sitem = W.get<uint32_t>("sub_item", (size_t)NS2 + 1);
  uint32_t* ilen = W.get<uint32_t>("sub_len", (size_t)NS2 + 1);
  uint32_t* ioff = W.get<uint32_t>("sub_off", (size_t)NS2 + 1);
  launch_subitems(b, items, NI, prank, nullptr, sub0, sitem, NS2, 1, s);
  if (NS2) launch_scan(sitem, sitem, NS2, 1, true, sc2, nullptr, b.err, s);
  uint8_t* stage = W.get<uint8_t>("emit_stage", (size_t)NS2 * kEmitSlot + 16);
  uint32_t* ovl = W.get<uint32_t>("emit_overflow", (size_t)NS2 + 1);
  CK(cudaMemsetAsync(&tot[13], 0, 4, s));
  // one thread per statement while staging (measured faster than a warp per
  // statement on large batches; a small batch takes a warp per statement, for
  // latency); one warp per statement for the few long ones redone in place
  uint32_t* skey = W.get<uint32_t>("sub_key", (size_t)NS2 + 1);
  uint32_t* sorder = W.get<uint32_t>("sub_order", (size_t)NS2 + 1);
  uint32_t* shist = W.get<uint32_t>("sub_hist", shape_buckets() + 1);
  launch_sub_order(b, items, sitem, sub0, prank, plist, NS2, skey, shist, sorder, sc2, s);
  b.prec = reinterpret_cast<PRec*>(W.get<uint4>("print_rec", 4ull * b.I + 4));
  static_assert(sizeof(uint4) == kPRecBytes, "one uint4 per print record");
  launch_print_records(b, s);
  ktime(KT_ITEMS, 0, s);
  launch_items(b, items, sitem, sub0, prank, plist, NS2, sorder, ilen, ioff, stage, ovl, &tot[13],
               NS2 <= kSmallBatchStmts ? 5u : 0u, s);
  ktime(KT_ITEMS, 1, s);
  if (NS2) launch_scan(ilen, ioff, NS2, 0, false, sc2, &tot[11], b.err, s);
  CK(cudaGetLastError());
  sync_totals();
  uint32_t total = NS2 ? h->h_tot[11] : 0;
  const uint32_t novf = NS2 ? h->h_tot[13] : 0;
  b.out = W.get<uint8_t>("out", (size_t)total + 16);
  b.file_out_off = W.get<uint64_t>("file_out_off", b.F + 2);
  b.file_status = W.get<int32_t>("file_status", b.F + 1);
  launch_compact(stage, ilen, ioff, NS2, b.out, s);
  launch_items(b, items, sitem, sub0, prank, plist, novf, ovl, ilen, ioff, nullptr, nullptr, nullptr, 5, s);
  launch_finish(b, ibase, sub0, ioff, total, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev[10], s));
  R.out_bytes = total;
  R.valid = true;
  pe.pending = true;
  h->launches = launch_counter() - launches0;
}

void finish_run(Engine* h, cudaStream_t s) {
  Run& R = h->run;
  Batch& b = R.b;
  CK(cudaMemcpyAsync(&h->h_tot[15], b.err, 4, cudaMemcpyDeviceToHost, s));
  R.kh.resize(b.K);
  if (b.K) CK(cudaMemcpyAsync(R.kh.data(), b.kh, sizeof(KHdr) * b.K, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  fold_times(h, h->cur);
  if (uint32_t e = h->h_tot[15]) {
    set_err("device error flags " + std::to_string(e));
    throw GCN_ECUDA;
  }
  R.file_k0.assign(b.F + 1, 0);
  // kernels are in file order: first kernel of each file
  uint32_t k = 0;
  for (uint32_t f = 0; f <= b.F; ++f) {
    while (k < b.K && R.kh[k].file < f) ++k;
    R.file_k0[f] = k;
  }
}

void engine_init(gcn_decomp* h, Engine* E) {
  E->big_kernel = h->tune.big_kernel;
  E->type_sweeps = h->tune.type_sweeps;
  E->ws.budget = h->budget;
  E->ws.pool = &h->pool;
  E->ws.peak = &h->pool_peak;
  E->ws.fail_jobs = h->tune.fail_alloc_jobs;
  for (PassEvents& p : E->pe) {
    for (auto& e : p.st) CK(cudaEventCreate(&e));
    for (auto& e : p.rs) CK(cudaEventCreate(&e));
    for (auto& e : p.kt.ev) CK(cudaEventCreate(&e));
  }
  for (SideStream* q : {&E->fk, &E->rs}) {
    CK(cudaStreamCreateWithFlags(&q->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&q->fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&q->join, cudaEventDisableTiming));
  }
  CK(cudaMallocHost(&E->h_tot, 64));
}

void engine_free(Engine* E) {
  E->ws.release();
  for (PassEvents& p : E->pe) {
    for (auto& e : p.st)
      if (e) cudaEventDestroy(e);
    for (auto& e : p.rs)
      if (e) cudaEventDestroy(e);
    for (auto& e : p.kt.ev)
      if (e) cudaEventDestroy(e);
    p = PassEvents{};
  }
  for (SideStream* q : {&E->fk, &E->rs}) {
    if (q->side) cudaStreamDestroy(q->side);
    if (q->fork) cudaEventDestroy(q->fork);
    if (q->join) cudaEventDestroy(q->join);
    *q = SideStream{};
  }
  if (E->h_tot) cudaFreeHost(E->h_tot);
  E->h_tot = nullptr;
}

void note_run(gcn_decomp* h, const Engine* E) {
  std::lock_guard<std::mutex> g(h->smu);
  const Batch& b = E->run.b;
  const uint64_t v[9] = {b.L, b.K, b.I, b.NL, b.NPB, b.NLB, b.NS, E->run.out_bytes, E->ws.total};
  for (int i = 0; i < 9; ++i) h->last_stats[i] = v[i];
  for (int i = 0; i < kTimings; ++i) h->last_ms[i] = E->stage_ms[i];
  h->last_launches = E->launches;
}

template <class T>
void grow_pinned(T*& p, size_t& cap, size_t n) {
  if (cap >= n) return;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  size_t want = n + n / 4 + 64;
  CK(cudaMallocHost((void**)&p, want * sizeof(T)));
  cap = want;
}

// drop the IR of every job whose batch lives on engine E (their texts stay)
void drop_ir(gcn_decomp* h, Engine* E) {
  if (!E->live) return;
  for (auto& kv : h->jobs)
    if (kv.second.eng == E) kv.second.eng = nullptr;
  E->live = 0;
}

// an engine for a new batch (called with h->mu held)
Engine* acquire_engine(gcn_decomp* h) {
  Engine* pick = nullptr;
  for (auto& e : h->engines)
    if (!e->busy && !e->live && (!pick || e->ws.total > pick->ws.total)) pick = e.get();
  if (!pick && (int)h->engines.size() < kMaxEngines) {
    h->engines.emplace_back(new Engine);
    pick = h->engines.back().get();
    engine_init(h, pick);
  }
  if (!pick) {  // the finished batch that is oldest gives its engine back
    for (auto& e : h->engines)
      if (!e->busy && (!pick || e->batch < pick->batch)) pick = e.get();
    drop_ir(h, pick);
  }
  pick->busy = true;
  return pick;
}

// free the workspaces of idle engines (called with h->mu held)
void shrink_pool(gcn_decomp* h) {
  for (auto& e : h->engines)
    if (!e->busy) {
      drop_ir(h, e.get());
      e->ws.release();
    }
}

// one batch of jobs on engine E through lane L; fills the jobs' results
void run_jobs(gcn_decomp* h, Lane* L, Engine* E, const std::vector<JobRec*>& js) {
  cudaStream_t s = L->stream;
  const size_t n = js.size();
  grow_pinned(L->h_off, L->h_off_cap, n + 1);
  grow_pinned(L->h_st, L->h_st_cap, n + 1);
  uint64_t N = 0;
  for (size_t i = 0; i < n; ++i) {
    L->h_off[i] = N;
    N += js[i]->in_len;
  }
  L->h_off[n] = N;
  if (N >= (1ull << 32)) {
    set_err("batch text exceeds 4 GiB");
    throw GCN_ENOMEM;
  }
  // the texts of consecutively submitted jobs lie back to back in their slab
  bool contiguous = true;
  for (size_t i = 1; i < n && contiguous; ++i)
    contiguous = js[i]->slab == js[0]->slab && js[i]->in == js[i - 1]->in + js[i - 1]->in_len;
  const uint8_t* src = n ? js[0]->in : nullptr;
  if (!contiguous) {
    grow_pinned(L->h_in, L->h_in_cap, N + 1);
    for (size_t i = 0; i < n; ++i) memcpy(L->h_in + L->h_off[i], js[i]->in, js[i]->in_len);
    src = L->h_in;
  }
  E->ws.cur_jobs = (uint32_t)n;
  uint8_t* d_text = E->ws.get<uint8_t>("in_text", N + 16);
  uint64_t* d_off = E->ws.get<uint64_t>("in_off", n + 1);
  if (N) CK(cudaMemcpyAsync(d_text, src, N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_off, L->h_off, sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  run_pipeline(E, d_text, N, d_off, (uint32_t)n, s);
  const Batch& b = E->run.b;
  const uint64_t T = E->run.out_bytes;
  grow_pinned(L->h_out, L->h_out_cap, T + 1);
  if (b.file_out_off) {
    CK(cudaMemcpyAsync(L->h_off, b.file_out_off, sizeof(uint64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(L->h_st, b.file_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    if (T) CK(cudaMemcpyAsync(L->h_out, b.out, T, cudaMemcpyDeviceToHost, s));
  }
  finish_run(E, s);
  for (size_t i = 0; i < n; ++i) {
    JobRec& j = *js[i];
    j.text.assign((const char*)L->h_out + L->h_off[i], L->h_off[i + 1] - L->h_off[i]);
    j.status = L->h_st[i];
    j.run_file = (uint32_t)i;
  }
}

void finish_jobs(gcn_decomp* h, const std::vector<uint64_t>& ids, Engine* E, uint64_t batch, int rc) {
  const uint64_t t = now_ns();
  for (uint64_t id : ids) {
    JobRec& j = h->jobs[id];
    j.state = JOB_DONE;
    j.rc = rc;
    j.t_done = t;
    if (j.slab >= 0) {
      Slab& sl = h->slabs[j.slab];
      if (--sl.refs == 0) sl.used = 0;
    }
    j.slab = -1;
    j.in = nullptr;
    j.in_len = 0;
    j.eng = rc == GCN_OK ? E : nullptr;
    j.batch = batch;
    h->done_q.push_back(id);
  }
  while (h->done_q.size() > 2ull * h->max_slots + 1024) h->done_q.pop_front();  // never polled
  if (rc == GCN_OK) {
    E->batch = batch;
    E->live = (uint32_t)ids.size();
  }
  E->busy = false;
}

void lane_main(gcn_decomp* h, Lane* L) {
  cudaSetDevice(h->device);
  std::unique_lock<std::mutex> lk(h->mu);
  while (true) {
    h->cv_work.wait(lk, [&] { return h->stop || !h->pending.empty(); });
    if (h->stop) break;
    // continuous batching: everything queued now, up to the batch limit
    std::vector<uint64_t> ids;
    std::vector<JobRec*> js;
    uint64_t bytes = 0;
    const uint64_t t = now_ns();
    while (!h->pending.empty()) {
      JobRec& j = h->jobs[h->pending.front()];
      if (!ids.empty() && bytes + j.in_len > h->tune.batch_bytes) break;
      ids.push_back(h->pending.front());
      js.push_back(&j);
      h->pending.pop_front();
      bytes += j.in_len;
      j.state = JOB_RUNNING;
      j.t_start = t;
    }
    if (!h->pending.empty()) h->cv_work.notify_one();
    Engine* E = acquire_engine(h);
    const uint64_t batch = h->next_batch++;
    lk.unlock();
    int rc = GCN_OK;
    bool shrunk = false;
    while (true) {
      try {
        run_jobs(h, L, E, js);
        rc = GCN_OK;
      } catch (int e) {
        rc = e;
      }
      if (rc != GCN_ENOMEM || (shrunk && js.size() == 1)) break;
      // out of the memory budget: first give back the memory of idle engines
      // (and start this engine afresh), then run half of the batch and queue
      // the other half again
      lk.lock();
      shrink_pool(h);
      E->ws.release();
      if (shrunk) {
        h->splits.fetch_add(1);
        const size_t keep = js.size() / 2;
        for (size_t q = js.size(); q-- > keep;) {
          js[q]->state = JOB_PENDING;
          h->pending.push_front(ids[q]);
        }
        ids.resize(keep);
        js.resize(keep);
        h->cv_work.notify_one();
      }
      shrunk = true;
      lk.unlock();
    }
    lk.lock();
    if (rc == GCN_OK) note_run(h, E);
    finish_jobs(h, ids, E, batch, rc);
    h->cv_done.notify_all();
  }
}

void start_lanes(gcn_decomp* h) {
  for (int i = 0; i < h->tune.lanes; ++i) {
    h->lanes.emplace_back(new Lane);
    Lane* L = h->lanes.back().get();
    CK(cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking));
  }
  for (auto& L : h->lanes) L->th = std::thread(lane_main, h, L.get());
}

void stop_lanes(gcn_decomp* h) {
  {
    std::lock_guard<std::mutex> g(h->mu);
    h->stop = true;
  }
  h->cv_work.notify_all();
  h->cv_done.notify_all();
  for (auto& L : h->lanes) {
    if (L->th.joinable()) L->th.join();
    if (L->stream) {
      cudaStreamSynchronize(L->stream);
      cudaStreamDestroy(L->stream);
    }
    if (L->h_in) cudaFreeHost(L->h_in);
    if (L->h_out) cudaFreeHost(L->h_out);
    if (L->h_off) cudaFreeHost(L->h_off);
    if (L->h_st) cudaFreeHost(L->h_st);
  }
  h->lanes.clear();
}

// release a fetched job (called with h->mu held)
void release_job(gcn_decomp* h, std::map<uint64_t, JobRec>::iterator it) {
  JobRec& j = it->second;
  h->admitted -= std::min(h->admitted, j.est);
  if (j.eng && j.eng->batch == j.batch && j.eng->live) --j.eng->live;
  h->jobs.erase(it);
}

// wait until job `id` is done (or report why not); called with the lock held
int wait_job(gcn_decomp* h, std::unique_lock<std::mutex>& lk, uint64_t id, bool wait,
             std::map<uint64_t, JobRec>::iterator* out) {
  auto it = h->jobs.find(id);
  if (it == h->jobs.end()) {
    set_err("unknown job");
    return GCN_ENOJOB;
  }
  if (it->second.state != JOB_DONE) {
    if (!wait) {
      set_err("job not finished");
      return GCN_EAGAIN;
    }
    h->cv_done.wait(lk, [&] {
      auto q = h->jobs.find(id);
      return h->stop || q == h->jobs.end() || q->second.state == JOB_DONE;
    });
    it = h->jobs.find(id);
    if (it == h->jobs.end() || it->second.state != JOB_DONE) {
      set_err("job no longer known");
      return GCN_ENOJOB;
    }
  }
  *out = it;
  return GCN_OK;
}

}  // namespace

// error text for entry points defined in other translation units
void gd::set_api_error(const char* msg) { set_err(msg); }

extern "C" {

const char* gcn_decomp_last_error(void) { return g_err.c_str(); }

int gcn_decomp_create(const gcn_decomp_config* cfg, gcn_decomp_t** out) {
  if (!cfg || !out) {
    set_err("NULL argument");
    return GCN_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    set_err("no such CUDA device");
    return GCN_EINVAL;
  }
  gcn_decomp* h = new gcn_decomp;
  try {
    h->device = cfg->device;
    h->budget = cfg->mem_budget_bytes;
    if (cfg->max_slots) h->max_slots = cfg->max_slots;
    if (cfg->tuning_file && !read_tuning(cfg->tuning_file, &h->tune)) throw GCN_EINVAL;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaDeviceSetLimit(cudaLimitStackSize, 16384));
    engine_init(h, &h->direct);
    init_decode_tables();
    CK(cudaGetLastError());
    start_lanes(h);
  } catch (int rc) {
    gcn_decomp_destroy(h);
    return rc;
  }
  *out = h;
  return GCN_OK;
}

void gcn_decomp_destroy(gcn_decomp_t* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  stop_lanes(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& e : h->engines) engine_free(e.get());
  h->engines.clear();
  engine_free(&h->direct);
  for (auto& sl : h->slabs)
    if (sl.p) cudaFreeHost(sl.p);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int gcn_decomp_run_device(gcn_decomp_t* h, const uint8_t* d_text, uint64_t text_len, const uint64_t* d_file_off,
                          uint64_t n_files, void* stream) {
  if (!h || (!d_text && text_len) || !d_file_off || text_len >= (1ull << 32) || n_files >= (1ull << 31)) {
    set_err("bad argument");
    return GCN_EINVAL;
  }
  std::lock_guard<std::mutex> lk(h->dmu);
  try {
    CK(cudaSetDevice(h->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    h->direct_stream = s;
    h->direct.ws.cur_jobs = 0;
    run_pipeline(&h->direct, d_text, text_len, d_file_off, (uint32_t)n_files, s);
    ++h->run_id;
    note_run(h, &h->direct);
  } catch (int rc) {
    h->direct.run.valid = false;
    return rc;
  }
  return GCN_OK;
}

int gcn_decomp_result_device(gcn_decomp_t* h, const uint8_t** d_out, const uint64_t** d_out_off,
                             const int32_t** d_status, uint64_t* out_bytes) {
  if (!h) return GCN_EINVAL;
  std::lock_guard<std::mutex> lk(h->dmu);
  if (!h->direct.run.valid) {
    set_err("no completed run");
    return GCN_EINVAL;
  }
  try {
    CK(cudaSetDevice(h->device));
    finish_run(&h->direct, h->direct_stream);
  } catch (int rc) {
    return rc;
  }
  note_run(h, &h->direct);
  const Run& R = h->direct.run;
  if (d_out) *d_out = R.b.out;
  if (d_out_off) *d_out_off = R.b.file_out_off;
  if (d_status) *d_status = R.b.file_status;
  if (out_bytes) *out_bytes = R.out_bytes;
  return GCN_OK;
}

int gcn_decomp_result_copy(gcn_decomp_t* h, uint64_t f0, uint64_t f1, void* buf, size_t cap, uint64_t* off_out,
                           int32_t* status_out) {
  if (!h) return GCN_EINVAL;
  std::lock_guard<std::mutex> lk(h->dmu);
  if (!h->direct.run.valid || f0 > f1 || f1 > h->direct.run.b.F) {
    set_err("no run or bad file range");
    return GCN_EINVAL;
  }
  try {
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->direct_stream));
    const Batch& b = h->direct.run.b;
    std::vector<uint64_t> o(f1 - f0 + 1);
    CK(cudaMemcpy(o.data(), b.file_out_off + f0, 8 * o.size(), cudaMemcpyDeviceToHost));
    uint64_t bytes = o.back() - o.front();
    if (off_out)
      for (size_t i = 0; i < o.size(); ++i) off_out[i] = o[i] - o[0];
    if (status_out && f1 > f0) CK(cudaMemcpy(status_out, b.file_status + f0, 4 * (f1 - f0), cudaMemcpyDeviceToHost));
    if (buf) {
      if (cap < bytes) {
        set_err("buffer too small");
        return GCN_EINVAL;
      }
      if (bytes) CK(cudaMemcpy(buf, b.out + o[0], bytes, cudaMemcpyDeviceToHost));
    }
  } catch (int rc) {
    return rc;
  }
  return GCN_OK;
}

int gcn_decomp_submit_batch(gcn_decomp_t* h, const char* const* text, const size_t* len, size_t n,
                            uint64_t* job_ids, size_t* n_admitted) {
  if (!h || (n && (!text || !len || !job_ids))) {
    set_err("bad argument");
    return GCN_EINVAL;
  }
  if (n_admitted) *n_admitted = 0;
  std::unique_lock<std::mutex> lk(h->mu);
  // admission: slots and the memory budget
  size_t take = 0;
  uint64_t total = 0, est_sum = 0, pinned = 0;
  for (; take < n; ++take) {
    if (h->jobs.size() + take >= h->max_slots) break;
    const size_t l = len[take];
    if (l && !text[take]) break;
    const uint64_t est = kEstPerTextByte * (uint64_t)l + kEstPerJob;
    if (h->budget && (h->admitted + est_sum) && h->admitted + est_sum + est > h->budget) break;
    est_sum += est;
    total += l;
    pinned += l + ((l && text[take][l - 1] != '\n') ? 1 : 0);
  }
  // one contiguous region of a pinned slab for all of their texts
  int si = -1;
  for (size_t q = 0; q < h->slabs.size() && si < 0; ++q) {
    Slab& sl = h->slabs[q];
    if (!sl.refs) sl.used = 0;
    if (sl.cap - sl.used >= pinned) si = (int)q;
  }
  if (si < 0 && take) {
    Slab sl;
    sl.cap = std::max<size_t>(kSlabBytes, pinned);
    if (cudaMallocHost(&sl.p, sl.cap) != cudaSuccess) {
      cudaGetLastError();
      set_err("cannot allocate pinned host memory for the job texts");
      return GCN_ENOMEM;
    }
    h->slabs.push_back(sl);
    si = (int)h->slabs.size() - 1;
  }
  uint8_t* region = take ? h->slabs[si].p + h->slabs[si].used : nullptr;
  if (take) {
    h->slabs[si].used += pinned;
    h->slabs[si].refs += (uint32_t)take;
  }
  const uint64_t t = now_ns();
  std::vector<JobRec*> recs;
  recs.reserve(take);
  size_t off = 0;
  for (size_t i = 0; i < take; ++i) {
    const size_t l = len[i];
    const uint64_t id = h->next_job++;
    JobRec& j = h->jobs[id];
    const bool nl = l && text[i][l - 1] == '\n';
    j.in = region + off;
    j.in_len = l + ((l && !nl) ? 1 : 0);
    j.slab = si;
    if (j.in_len > l) region[off + l] = '\n';
    off += j.in_len;
    j.est = kEstPerTextByte * (uint64_t)l + kEstPerJob;
    j.t_submit = t;
    h->admitted += j.est;
    recs.push_back(&j);
    job_ids[i] = id;
  }
  lk.unlock();
  // copy the texts (outside the lock; the jobs are not queued yet)
  auto copy_range = [&](size_t a, size_t z) {
    for (size_t i = a; i < z; ++i)
      if (len[i]) memcpy((uint8_t*)recs[i]->in, text[i], len[i]);
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nth = total >= (16ull << 20) ? std::min<size_t>({(size_t)8, (size_t)hw, take}) : 1;
  if (nth > 1) {
    std::vector<std::thread> th;
    for (size_t q = 1; q < nth; ++q) th.emplace_back(copy_range, take * q / nth, take * (q + 1) / nth);
    copy_range(0, take / nth);
    for (auto& x : th) x.join();
  } else {
    copy_range(0, take);
  }
  lk.lock();
  for (size_t i = 0; i < take; ++i) h->pending.push_back(job_ids[i]);
  if (n_admitted) *n_admitted = take;
  lk.unlock();
  if (take) h->cv_work.notify_all();
  if (n && !take) {
    set_err("nothing admitted: no free job slot or memory budget");
    return GCN_EAGAIN;
  }
  return GCN_OK;
}

int gcn_decomp_fetch_opencl(gcn_decomp_t* h, uint64_t job_id, char* buf, size_t cap, size_t* len_out,
                            int* status_out, uint32_t flags) {
  if (!h) return GCN_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu);
  std::map<uint64_t, JobRec>::iterator it;
  int rc = wait_job(h, lk, job_id, (flags & GCN_WAIT) != 0, &it);
  if (rc != GCN_OK) return rc;
  JobRec& j = it->second;
  if (j.rc != GCN_OK) {
    rc = j.rc;
    set_err("the batch of this job failed");
    release_job(h, it);
    return rc;
  }
  if (len_out) *len_out = j.text.size();
  if (status_out) *status_out = j.status;
  if (!buf) return GCN_OK;
  if (cap < j.text.size()) {
    set_err("buffer too small");
    return GCN_EINVAL;
  }
  memcpy(buf, j.text.data(), j.text.size());
  release_job(h, it);
  return GCN_OK;
}

int gcn_decomp_fetch_batch(gcn_decomp_t* h, const uint64_t* job_ids, size_t n, char* buf, size_t cap,
                           uint64_t* off_out, int32_t* status_out, uint32_t flags) {
  if (!h || (n && (!job_ids || !off_out))) {
    set_err("bad argument");
    return GCN_EINVAL;
  }
  std::unique_lock<std::mutex> lk(h->mu);
  std::vector<std::map<uint64_t, JobRec>::iterator> its(n);
  for (size_t i = 0; i < n; ++i) {
    int rc = wait_job(h, lk, job_ids[i], (flags & GCN_WAIT) != 0, &its[i]);
    if (rc != GCN_OK) return rc;
  }
  for (size_t i = 0; i < n; ++i) {
    its[i] = h->jobs.find(job_ids[i]);  // re-find: waiting released the lock
    if (its[i] == h->jobs.end()) {
      set_err("job no longer known");
      return GCN_ENOJOB;
    }
    if (its[i]->second.rc != GCN_OK) {
      set_err("the batch of a job failed");
      return its[i]->second.rc;
    }
  }
  uint64_t o = 0;
  for (size_t i = 0; i < n; ++i) {
    off_out[i] = o;
    o += its[i]->second.text.size();
    if (status_out) status_out[i] = its[i]->second.status;
  }
  off_out[n] = o;
  if (!buf) return GCN_OK;
  if (cap < o) {
    set_err("buffer too small");
    return GCN_EINVAL;
  }
  auto copy_range = [&](size_t a, size_t z) {
    for (size_t i = a; i < z; ++i) {
      const std::string& t = its[i]->second.text;
      if (!t.empty()) memcpy(buf + off_out[i], t.data(), t.size());
    }
  };
  // large fetches are copied by several threads (the jobs are done: nothing else writes them)
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nth = o >= (16ull << 20) ? std::min<size_t>({(size_t)8, (size_t)hw, n}) : 1;
  if (nth > 1) {
    std::vector<std::thread> th;
    for (size_t q = 1; q < nth; ++q) th.emplace_back(copy_range, n * q / nth, n * (q + 1) / nth);
    copy_range(0, n / nth);
    for (auto& x : th) x.join();
  } else {
    copy_range(0, n);
  }
  for (size_t i = 0; i < n; ++i) release_job(h, its[i]);
  return GCN_OK;
}

int gcn_decomp_poll(gcn_decomp_t* h, uint64_t* job_ids, size_t cap, size_t* n_out, int timeout_ms) {
  if (!h || !n_out || (cap && !job_ids)) {
    set_err("bad argument");
    return GCN_EINVAL;
  }
  std::unique_lock<std::mutex> lk(h->mu);
  if (h->done_q.empty() && timeout_ms != 0) {
    auto ready = [&] { return h->stop || !h->done_q.empty(); };
    if (timeout_ms < 0) h->cv_done.wait(lk, ready);
    else h->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  size_t k = 0;
  while (k < cap && !h->done_q.empty()) {
    const uint64_t id = h->done_q.front();
    h->done_q.pop_front();
    if (h->jobs.count(id)) job_ids[k++] = id;
  }
  *n_out = k;
  return GCN_OK;
}

int gcn_decomp_job_info(gcn_decomp_t* h, uint64_t job_id, uint64_t* info, int cap) {
  if (!h || !info || cap < 0) return GCN_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->jobs.find(job_id);
  if (it == h->jobs.end()) {
    set_err("unknown job");
    return GCN_ENOJOB;
  }
  const JobRec& j = it->second;
  const uint64_t v[5] = {(uint64_t)j.state, j.t_submit, j.t_start, j.t_done, j.eng != nullptr};
  int n = cap < 5 ? cap : 5;
  for (int i = 0; i < n; ++i) info[i] = v[i];
  return n;
}

int gcn_decomp_job_info_batch(gcn_decomp_t* h, const uint64_t* job_ids, size_t n, uint64_t* info, int per) {
  if (!h || per < 1 || per > 5 || (n && (!job_ids || !info))) {
    set_err("bad argument");
    return GCN_EINVAL;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  for (size_t i = 0; i < n; ++i) {
    uint64_t* o = info + i * (size_t)per;
    auto it = h->jobs.find(job_ids[i]);
    if (it == h->jobs.end()) {
      for (int q = 0; q < per; ++q) o[q] = 0;
      continue;
    }
    const JobRec& j = it->second;
    const uint64_t v[5] = {(uint64_t)j.state, j.t_submit, j.t_start, j.t_done, j.eng != nullptr};
    for (int q = 0; q < per; ++q) o[q] = v[q];
  }
  return GCN_OK;
}

int gcn_decomp_fetch_ir(gcn_decomp_t* h, uint64_t job_id, int which, void* buf, size_t cap, size_t* len_out) {
  if (!h || which < 0 || which > 5) return GCN_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu);
  std::map<uint64_t, JobRec>::iterator it;
  int rc = wait_job(h, lk, job_id, true, &it);
  if (rc != GCN_OK) return rc;
  const JobRec& j = it->second;
  if (j.rc != GCN_OK || !j.eng || j.eng->batch != j.batch || !j.eng->run.valid) {
    set_err("job IR no longer resident");
    return GCN_ENOJOB;
  }
  const Run& R = j.eng->run;
  const Batch& b = R.b;
  uint32_t f = j.run_file;
  std::vector<uint8_t> v;
  try {
    CK(cudaSetDevice(h->device));
    for (uint32_t k = R.file_k0[f]; k < R.file_k0[f + 1]; ++k) {
      const KHdr& K = R.kh[k];
      auto grab = [&](const void* dev, size_t bytes) {
        size_t o = v.size();
        v.resize(o + bytes);
        if (bytes) CK(cudaMemcpy(v.data() + o, dev, bytes, cudaMemcpyDeviceToHost));
      };
      bool lbad = (K.bad & ~3u) != 0 || (K.bad & 3u) != 0;
      switch (which) {
        case 0: if (!(K.bad & 1u)) grab(b.ins + K.first_instr, sizeof(InstrRec) * K.n_instr); break;
        case 1: if (!(K.bad & 1u)) grab(b.pblock_of + K.first_instr, 4ull * K.n_instr); break;
        case 2: if (!(K.bad & 1u)) grab(b.pblocks + K.first_pblock, sizeof(BlockRec) * K.n_pblock); break;
        case 3: if (!lbad) grab(b.lblock_of + K.first_instr, 4ull * K.n_instr); break;
        case 4: if (!lbad) grab(b.lblocks + K.first_lblock, sizeof(BlockRec) * K.n_lblock); break;
        case 5: {
          uint32_t hd[8] = {K.dims, K.cws[0], K.cws[1], K.cws[2], K.sgprs, K.vgprs, K.useargs, K.nuser};
          size_t o = v.size();
          v.resize(o + sizeof hd);
          memcpy(v.data() + o, hd, sizeof hd);
          break;
        }
      }
    }
  } catch (int e) {
    return e;
  }
  if (len_out) *len_out = v.size();
  if (!buf) return GCN_OK;
  if (cap < v.size()) return GCN_EINVAL;
  memcpy(buf, v.data(), v.size());
  return GCN_OK;
}

uint64_t gcn_decomp_launches(gcn_decomp_t* h) {
  if (!h) return 0;
  std::lock_guard<std::mutex> g(h->smu);
  return h->last_launches;
}

int gcn_decomp_run_stats(gcn_decomp_t* h, uint64_t* out, int cap) {
  if (!h || !out || cap < 0) return GCN_EINVAL;
  std::lock_guard<std::mutex> g(h->smu);
  const uint64_t v[11] = {h->last_stats[0], h->last_stats[1], h->last_stats[2], h->last_stats[3],
                          h->last_stats[4], h->last_stats[5], h->last_stats[6], h->last_stats[7],
                          h->last_stats[8], h->pool_peak.load(), h->splits.load()};
  int n = cap < 11 ? cap : 11;
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

int gcn_decomp_stage_totals(gcn_decomp_t* h, double* ms, const char** names, int cap, uint64_t* runs, int reset) {
  if (!h || cap < 0) return GCN_EINVAL;
  std::lock_guard<std::mutex> lk(h->dmu);
  Engine& E = h->direct;
  try {
    CK(cudaSetDevice(h->device));
    fold_times(&E, E.cur ^ 1);  // the older pass first: sums in pass order
    fold_times(&E, E.cur);
  } catch (int rc) {
    return rc;
  }
  int n = std::min(cap, kTimings);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = E.sum_ms[i];
    if (names) names[i] = kStageNames[i];
  }
  if (runs) *runs = E.sum_runs;
  if (reset) {
    for (double& x : E.sum_ms) x = 0;
    E.sum_runs = 0;
  }
  return n;
}

int gcn_decomp_stage_times(gcn_decomp_t* h, float* ms, const char** names, int cap) {
  if (!h || cap < 0) return GCN_EINVAL;
  std::lock_guard<std::mutex> g(h->smu);
  int n = std::min(cap, kTimings);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = h->last_ms[i];
    if (names) names[i] = kStageNames[i];
  }
  return n;
}

}  // extern "C"
