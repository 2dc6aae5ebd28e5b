// gd_kernels.h — host-side launchers of the CUDA stages (one translation unit each).
#pragma once
#include "gd_common.cuh"

namespace gd {

// sets the text gcn_decomp_last_error returns on this thread
void set_api_error(const char* msg);

// kernels launched by the calling host thread (one instance across units)
inline uint64_t& launch_counter() {
  thread_local uint64_t c = 0;
  return c;
}

// Device-time events around the pipeline's longest kernels, for the per-kernel
// figures of gcn_decomp_stage_times: the engine running a pass points
// kernel_timer() at its events (per host thread, like the launch counter).
enum KTimed : int { KT_LINE_SCAN = 0, KT_DECODE, KT_NODES, KT_NODE_FWD, KT_NODE_CACHE, KT_ITEMS, KT_COUNT };
struct KernelTimer {
  cudaEvent_t ev[2 * KT_COUNT];
};
inline KernelTimer*& kernel_timer() {
  thread_local KernelTimer* t = nullptr;
  return t;
}
// edge 0 before the launch, 1 after it
inline void ktime(int which, int edge, cudaStream_t s) {
  if (KernelTimer* t = kernel_timer()) cudaEventRecord(t->ev[2 * which + edge], s);
}

// line kinds and row types
enum : uint8_t { LK_BLANK = 0, LK_KERNEL = 1, LK_CONFIG = 2, LK_TEXT = 3, LK_LABEL = 4, LK_ROW = 5 };
enum : uint8_t { RT_NONE = 0, RT_CFG = 1, RT_LABEL = 2, RT_INSTR = 3, RT_KERNEL = 4 };

struct ScanScratch {
  uint64_t* status;   // >= scan_tiles(n) words
  uint32_t* counter;  // 1 word
};

struct RowArrays {    // per line
  uint8_t* file_start;
  uint8_t* kind;
  uint8_t* rowtype;
  uint32_t *t0, *t1, *t2;
  uint32_t *mkmax, *fsmax, *kcnt, *instr_excl, *label_excl, *cfg_excl;
};

// everything the per-kernel stages read and write (device pointers)
struct KView;  // a kernel's view of the batch arrays (k_analysis.cuh)

struct Batch {
  const uint8_t* text;
  uint64_t text_len;
  const uint64_t* file_off;
  uint32_t F, L, K, I, NL, NC;   // files, lines, kernels, instructions, labels, configuration rows
  uint32_t big_kernel;           // size buckets: kernels this long or longer get a thread block
  uint32_t type_sweeps;          // sweep limit of the type fixed point (a kernel that reaches it is capped)
  uint32_t NPB, NLB;             // physical / logical blocks
  uint64_t NS;                   // block x register state words
  const uint32_t* line_start;
  const uint8_t* rowtype;
  const uint8_t* file_start;
  const uint8_t* kind;
  KHdr* kh;
  ArgRec* args;                  // K * kMaxArgs
  uint32_t* instr_line;          // I
  uint32_t* ikern;               // I: kernel of each instruction
  uint32_t* blen;                // I: length of a branch's label operand
  const uint32_t* kcnt;          // L: running count of .kernel rows
  uint32_t* cfg_line;            // NC: line of each configuration row
  uint32_t* label_line;          // NL
  uint32_t* label_instr;         // NL (global instruction index)
  uint32_t* label_hash;          // NL
  uint32_t* dyn_count;           // K: nodes of each kernel whose type comes from their operands
  struct PRec* prec;             // 4I: the printer's record of every node slot (S13)
  uint32_t* label_tab;           // open-addressing table of label indices (kNone = empty), label_tab_mask + 1 slots
  uint32_t label_tab_mask;
  InstrRec* ins;                 // I
  uint32_t* branch_hash;         // I (label name hash of a branch)
  uint32_t* branch_pos;          // I (byte offset | len<<24 of the label operand)
  // physical CFG
  uint32_t* pleader;             // I (scratch flag / scan)
  uint32_t* pblock_of;           // I (kernel-relative)
  BlockRec* pblocks;             // NPB
  // logical CFG
  uint8_t* ctl;                  // I
  uint8_t* sense;                // I
  uint32_t* ltarget;             // I (kernel-relative)
  uint32_t* lleader;             // I
  uint32_t* exec_list;           // I: the exec-mask form instructions, in order (S6 scratch)
  uint32_t* lblock_of;           // I (kernel-relative, kNone = dropped)
  BlockRec* lblocks;             // NLB (kernel-relative indices)
  uint32_t* lterm;               // NLB (kernel-relative instruction)
  // dataflow
  uint8_t* fused;                // I
  uint32_t* co_idx;              // I (kernel-relative)
  uint32_t* pred_off;            // NLB + 1 (global)
  uint32_t* preds;               // (kernel-relative block ids)
  uint32_t* pred_fill;           // NLB
  uint32_t* idom;                // NLB (kernel-relative)
  uint32_t* rpo;                 // NLB (kernel-relative, per-kernel order)
  uint32_t* df_off;              // NLB + 1
  uint32_t* df;                  // dominance frontier lists
  uint32_t* scratch32;           // NLB (dfs stacks etc.)
  uint32_t* st_in;               // NS
  uint32_t* st_out;              // NS
  uint8_t* has_phi;              // NS
  Node* nodes;                   // 4 * I
  // analysis
  uint8_t* ncls;                 // 4 * I: class of each node (null until cached)
  uint8_t* nclsk;                // 4 * I
  uint32_t* nsrcf;               // 12 * I: forwarded sources of each node
  uint32_t* mem_arg;             // I: matched argument (kNone = raw address)
  uint32_t* mem_idx;             // I: index value reference (kTop = constant 0)
  uint32_t* uses;                // 4 * I
  uint8_t* nflag;                // 4 * I: 1 reach, 2 cross-block, 4 join input
  uint8_t* ntype;                // 4 * I
  int32_t* var_of;               // 4 * I
  uint8_t* phi_used;             // NS
  uint32_t* plist;               // NS: used join versions of each kernel (block << 10 | reg)
  uint8_t* phi_type;             // NS
  int32_t* phi_var;              // NS
  uint8_t* var_type;             // per kernel: at most 4*I + NS ... (indexed by var_base + v)
  uint32_t* var_base;            // K
  uint64_t* wl;                  // reachability work lists
  // regions
  uint32_t* rg;                  // region records, 12 words per region
  uint32_t* brk;                 // NLB: per block, the latch an early exit leaves by, kBrkLatch or kNone
  // per kernel, its view built once (k_make_views): with the forwarded sources only (for the class
  // pass), and with every cache; threads take references into them instead of each building its
  // own view in local memory
  const KView* kview_sf;
  const KView* kview;
  // emission
  uint32_t* kout_len;            // K (text length of each kernel incl. separator)
  uint32_t* kout_off;            // K (exclusive scan)
  uint32_t* cs_off;              // 2 NLB + 1: copies on each CFG edge (2 per logical block)
  uint32_t* cs_cnt;              // 2 NLB
  uint8_t* cs_cyc;               // 2 NLB: the copies form a cycle
  uint32_t* cs_reg;              // registers of the copies, in printing order
  uint8_t* out;                  // output text
  uint64_t* file_out_off;        // F + 1
  int32_t* file_status;          // F
  uint32_t* err;
};

// Per-kernel serial walks run one warp per kernel, its lane 0 working: 32
// kernels packed into one warp would run their diverging walks one after the
// other, while a warp each lets the SMs interleave them (and a batch of a few
// large kernels spreads over several SMs instead of sharing one).
// A batch of few kernels (at most a few per SM) gives each its own thread block, so that each
// walk has an SM's L1 cache to itself; larger batches pack four kernels per block.
__device__ __forceinline__ uint32_t walk_kernel() {
  return (threadIdx.x & 31u) ? 0xFFFFFFFFu : blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
}
inline uint32_t walk_warps(uint32_t K) { return K <= 1024 ? 1u : 4u; }
inline uint32_t walk_blocks(uint32_t K) { return (K + walk_warps(K) - 1) / walk_warps(K); }
inline uint32_t walk_threads(uint32_t K) { return 32 * walk_warps(K); }

// Size buckets: a kernel of fewer than b.big_kernel instructions (a tuning
// parameter) is handled by one warp (Team<true>), a longer one by a whole
// thread block (Team<false>); both launches cover every kernel and a team
// leaves the kernels of the other bucket alone.
constexpr int kBigTeam = 512;
// A batch of at most this many kernels (one per SM) puts every kernel in the block bucket: the
// teams then occupy no more than the GPU's SMs, and a block finishes a kernel's walks sooner.
constexpr uint32_t kBlockPerKernelBatch = 152;

template <bool WARP>
struct Team {
  static __device__ __forceinline__ uint32_t kid() {
    return WARP ? blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32 : blockIdx.x;
  }
  static __device__ __forceinline__ uint32_t tid() { return WARP ? (threadIdx.x & 31u) : threadIdx.x; }
  static __device__ __forceinline__ uint32_t size() { return WARP ? 32u : blockDim.x; }
  static __device__ __forceinline__ uint32_t slot() { return WARP ? threadIdx.x / 32 : 0u; }
  static __device__ __forceinline__ void sync() {
    if (WARP) __syncwarp();
    else __syncthreads();
  }
  static __device__ __forceinline__ bool any(bool p) {
    if (WARP) return __any_sync(0xFFFFFFFFu, p);
    return __syncthreads_or(p) != 0;
  }
  static __device__ __forceinline__ bool mine(const KHdr& K, uint32_t big) { return (K.n_instr >= big) != WARP; }
  // the next kernel of a device work queue: entry *head (then advanced) of list[0..n), kNone when
  // the list is exhausted; every thread of the team gets the same answer
  static __device__ __forceinline__ uint32_t next(uint32_t* head, const uint32_t* list, uint32_t n) {
    if (WARP) {
      uint32_t i = 0;
      if ((threadIdx.x & 31u) == 0) i = atomicAdd(head, 1u);
      i = __shfl_sync(0xFFFFFFFFu, i, 0);
      return i < n ? list[i] : kNone;
    }
    __shared__ uint32_t s_i;
    if (threadIdx.x == 0) s_i = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t i = s_i;
    __syncthreads();  // read by every thread before thread 0 takes the next one
    return i < n ? list[i] : kNone;
  }
};

// The kernels of a batch in the order the per-kernel work queues hand them out: those of the block
// bucket (big_kernel instructions or more) first, then the rest, each by decreasing size (a
// counting sort by the size's binary logarithm), so that the longest start first.  order[K],
// info[0] = the number in the block bucket.
struct KernelOrder {
  uint32_t* order;
  uint32_t* info;
  uint32_t* heads;  // work-queue heads, zeroed before the launches that use them
};
void launch_kernel_order(const Batch& b, const KernelOrder& ko, cudaStream_t s);

// k_text.cu
uint32_t line_scan_tiles(uint64_t n);
uint32_t scan_tiles(uint32_t n);
// scratch of the two-pass S1 (texts of more than kLsOnePass 32 KiB tiles): per tile its newline
// count, the exclusive scan of the counts, and 2048 16-bit newline masks
constexpr uint32_t kLsOnePass = 256;
constexpr uint32_t kLsTileBytes = 32768;  // the S1 tile (LS_TILE)
struct LineScan2 {
  uint16_t* masks;   // tiles * 2048
  uint32_t* counts;  // tiles
  uint32_t* prefix;  // tiles
};
void launch_line_scan(const uint8_t* text, uint64_t n, uint32_t* line_start, uint64_t* tile_status,
                      uint32_t* counters, uint32_t* err, const LineScan2& two, cudaStream_t s);
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t n, int op, bool inclusive, ScanScratch sc,
                 uint32_t* total_out, uint32_t* err, cudaStream_t s);
// status3: scan3_status_words(L) look-back words for the three-channel row scans
void launch_rows(const uint8_t* text, const uint32_t* line_start, uint32_t L, const uint64_t* file_off, uint32_t F,
                 RowArrays& ra, ScanScratch sc, uint64_t* status3, uint32_t* totals, uint32_t* err, cudaStream_t s);
uint32_t scan3_status_words(uint32_t n);
void launch_scatter_rows(uint32_t L, RowArrays& ra, uint32_t* instr_line, uint32_t* label_line, uint32_t* label_instr,
                         uint32_t* cfg_line, KHdr* kh, cudaStream_t s);

// k_decode.cu
void init_decode_tables();
void launch_config(Batch& b, cudaStream_t s);
void launch_decode(Batch& b, ScanScratch sc, uint32_t* totals, cudaStream_t s);
void launch_pblocks(Batch& b, uint32_t* blk_kern, cudaStream_t s);
void launch_logical(Batch& b, ScanScratch sc, uint32_t* totals, cudaStream_t s);
void launch_lblocks(Batch& b, uint32_t* blk_kern, cudaStream_t s);

// k_dataflow.cu
struct DfScratch {
  uint32_t *kstate, *kstate_off, *kbits, *bits_off;  // K
  uint32_t *pcount, *blk_kern;                       // NLB + 1
  uint32_t *rpo_index, *stack;                       // NLB
  uint8_t* child;                                    // NLB
  uint32_t *defbits, *phibits;                       // NW
  uint32_t* rows;                                    // NS: working register rows
  uint32_t NW;
};
void launch_df_counts(Batch& b, DfScratch& d, ScanScratch sc, uint32_t* totals, cudaStream_t s);
void launch_df_main(Batch& b, DfScratch& d, cudaStream_t s);

// k_analysis.cu
void launch_wl_size(Batch& b, uint32_t* sz, uint32_t* off, ScanScratch sc, uint32_t* total, cudaStream_t s);
size_t kview_bytes();
void launch_node_cache(Batch& b, void* views, cudaStream_t s);  // views: 2 * K * kview_bytes() bytes
// a second stream for launches that may overlap those of the main stream, with
// the events that fork work onto it and join it back
struct SideStream {
  cudaStream_t side;
  cudaEvent_t fork, join;
};
void launch_analysis(Batch& b, uint32_t* wl, uint32_t* bits, uint64_t nbits_words, const uint32_t* blk_kern,
                     uint32_t* vflag, uint32_t* vpos, ScanScratch sc, SideStream fk, const KernelOrder& ko, cudaStream_t s);

// k_region.cu
void launch_regions(Batch& b, uint32_t* work, uint32_t* stk, uint8_t* alive, uint8_t* cond, cudaStream_t s);

// k_emit.cu
struct Item {
  uint32_t kl;  // kind | level << 8
  uint32_t k;   // kernel
  uint32_t a, b;
};
void launch_copy_sets(Batch& b, const uint32_t* blk_kern, const uint32_t* pbits, uint32_t* bound_or_tmp, int phase,
                      cudaStream_t s);
void launch_layout(Batch& b, Item* stage, uint32_t* stage_off, uint32_t* item_cnt, uint32_t* stk, int phase,
                   cudaStream_t s);
void launch_items_place(const Item* stage, const uint32_t* stage_off, uint32_t K, uint32_t total,
                        const uint32_t* item_cnt, const uint32_t* item_base, Item* items, cudaStream_t s);
constexpr uint32_t kPRecBytes = 16;  // size of a print record (k_emit.cu)
constexpr uint32_t kEmitSlot = 1024;  // staging bytes per emission sub-item
// A batch of at most this many statements prints one statement per warp (lane 0
// works) instead of one per thread: the warps then fit on the GPU at once, and a
// warp no longer runs the printing paths of 32 different statements one after
// another, which sets the latency of a small batch.
constexpr uint32_t kSmallBatchStmts = 4096;
void launch_print_list(Batch& b, uint32_t* flag, const uint32_t* rank, uint32_t* list, int phase, cudaStream_t s);
void launch_subitems(Batch& b, const Item* items, uint32_t NI, const uint32_t* prank, uint32_t* weight,
                     const uint32_t* sub0, uint32_t* sub_item, uint32_t NS2, int phase, cudaStream_t s);
void launch_sub_order(Batch& b, const Item* items, const uint32_t* sub_item, const uint32_t* sub0,
                      const uint32_t* prank, const uint32_t* pinstr, uint32_t N, uint32_t* key, uint32_t* hist,
                      uint32_t* order, ScanScratch sc, cudaStream_t s);
uint32_t shape_buckets();
void launch_print_records(Batch& b, cudaStream_t s);
void launch_items(Batch& b, const Item* items, const uint32_t* sub_item, const uint32_t* sub0, const uint32_t* prank,
                  const uint32_t* pinstr, uint32_t N, const uint32_t* list, uint32_t* item_len,
                  const uint32_t* item_off, uint8_t* stage, uint32_t* ovf_list, uint32_t* ovf_count,
                  uint32_t lane_shift, cudaStream_t s);
void launch_compact(const uint8_t* stage, const uint32_t* item_len, const uint32_t* item_off, uint32_t N,
                    uint8_t* out, cudaStream_t s);
void launch_finish(Batch& b, const uint32_t* item_base, const uint32_t* sub0, const uint32_t* item_off,
                   uint32_t total, cudaStream_t s);

}  // namespace gd
