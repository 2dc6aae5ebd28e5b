// k_text.cu — tokenisation and body extraction on the GPU.
//
// S1 (line tokenisation): every byte of the batch text is read once, a 16 KiB
// tile per block moved into shared memory by one bulk copy (k_linescan.cuh);
// a block scan plus a single-pass decoupled look-back (the whole block looking
// back 256 tiles at a time) gives each newline its global rank, and the line
// starts are written.
// S2 (body extraction, Listing 2 of the paper): the row state machine
// (.kernel / .config / .text) becomes three scans over the rows — the last
// state marker, the last file start and the running count of .kernel rows —
// after which every row knows its kernel and its section independently.
#include "gd_kernels.h"
#include "k_linescan.cuh"

namespace gd {

// ---------------------------------------------------------------------------
// S1: newline scan
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(LS_THREADS) k_line_scan(const __grid_constant__ LineScanArgs a) {
  __shared__ LineScanSmem sm;
  line_scan_tile(sm, a);
}

void launch_line_scan(const uint8_t* text, uint64_t n, uint32_t* line_start, uint64_t* tile_status,
                      uint32_t* counters, uint32_t* err, cudaStream_t s) {
  uint32_t tiles = (uint32_t)((n + LS_TILE - 1) / LS_TILE);
  if (!tiles) tiles = 1;
  cudaMemsetAsync(tile_status, 0, sizeof(uint64_t) * tiles, s);
  cudaMemsetAsync(counters, 0, 2 * sizeof(uint32_t), s);
  LineScanArgs a;
  a.text = text;
  a.n = n;
  a.use_bulk = (reinterpret_cast<uintptr_t>(text) & 15u) == 0;
  a.line_start = line_start;
  a.cap = n + 2;  // the array holds n + 2 entries: never more newlines than bytes
  a.status = tile_status;
  a.counter = &counters[0];
  a.ntiles = tiles;
  a.lines_out = &counters[1];
  a.err = err;
  ktime(KT_LINE_SCAN, 0, s);
  k_line_scan<<<tiles, LS_THREADS, 0, s>>>(a);
  ktime(KT_LINE_SCAN, 1, s);
  ++launch_counter();
}
uint32_t line_scan_tiles(uint64_t n) { return (uint32_t)((n + LS_TILE - 1) / LS_TILE) + 1; }

// ---------------------------------------------------------------------------
// generic single-pass scan of u32 arrays
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 256, SC_ITEMS = 8, SC_TILE = SC_THREADS * SC_ITEMS;

template <class Op, bool Incl>
__global__ void __launch_bounds__(SC_THREADS) k_scan(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     uint32_t n, uint64_t* status, uint32_t* counter,
                                                     uint32_t* total_out, uint32_t* err) {
  __shared__ uint32_t sm[SC_TILE];
  __shared__ uint32_t s_tile, s_prefix, s_warp[32];
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * SC_TILE;
  for (int k = 0; k < SC_ITEMS; ++k) {
    uint64_t i = base + (uint64_t)k * SC_THREADS + threadIdx.x;
    sm[k * SC_THREADS + threadIdx.x] = i < n ? in[i] : Op::id;
  }
  __syncthreads();
  uint32_t v[SC_ITEMS];
  uint32_t acc = Op::id;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    acc = Op::op(acc, sm[threadIdx.x * SC_ITEMS + k]);
    v[k] = acc;
  }
  uint32_t total;
  uint32_t incl = block_incl_scan<Op>(acc, s_warp, &total);
  // exclusive prefix of this thread inside the tile: inclusive minus own (for sum),
  // or the previous thread's inclusive value (general)
  uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t texcl = lane ? prev : (warp ? s_warp[warp - 1] : Op::id);
  if (threadIdx.x < 32) {
    uint32_t p = lookback<Op>(status, tile, total, err);
    if (threadIdx.x == 0) {
      s_prefix = p;
      if (tile == gridDim.x - 1 && total_out) *total_out = Op::op(p, total);
    }
  }
  __syncthreads();
  const uint32_t pre = Op::op(s_prefix, texcl);
  uint32_t run = pre;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    uint32_t r = Op::op(pre, v[k]);
    sm[threadIdx.x * SC_ITEMS + k] = Incl ? r : run;
    run = r;
  }
  __syncthreads();
  for (int k = 0; k < SC_ITEMS; ++k) {
    uint64_t i = base + (uint64_t)k * SC_THREADS + threadIdx.x;
    if (i < n) out[i] = sm[k * SC_THREADS + threadIdx.x];
  }
}

void launch_scan(const uint32_t* in, uint32_t* out, uint32_t n, int op, bool inclusive, ScanScratch sc,
                 uint32_t* total_out, uint32_t* err, cudaStream_t s) {
  uint32_t tiles = (n + SC_TILE - 1) / SC_TILE;
  if (!tiles) tiles = 1;
  cudaMemsetAsync(sc.status, 0, sizeof(uint64_t) * tiles, s);
  cudaMemsetAsync(sc.counter, 0, sizeof(uint32_t), s);
  if (op == 0 && inclusive) {
    k_scan<ScanSum, true><<<tiles, SC_THREADS, 0, s>>>(in, out, n, sc.status, sc.counter, total_out, err);
    ++launch_counter();
  }
  if (op == 0 && !inclusive) {
    k_scan<ScanSum, false><<<tiles, SC_THREADS, 0, s>>>(in, out, n, sc.status, sc.counter, total_out, err);
    ++launch_counter();
  }
  if (op == 1 && inclusive) {
    k_scan<ScanMax, true><<<tiles, SC_THREADS, 0, s>>>(in, out, n, sc.status, sc.counter, total_out, err);
    ++launch_counter();
  }
  if (op == 1 && !inclusive) {
    k_scan<ScanMax, false><<<tiles, SC_THREADS, 0, s>>>(in, out, n, sc.status, sc.counter, total_out, err);
    ++launch_counter();
  }
}
uint32_t scan_tiles(uint32_t n) { return (n + SC_TILE - 1) / SC_TILE + 1; }

// ---------------------------------------------------------------------------
// S2: rows, files, kernels
// ---------------------------------------------------------------------------
// first line of every non-empty file (files end with '\n', so a file start is a line start)
__global__ void k_file_starts(const uint32_t* __restrict__ line_start, uint32_t L, const uint64_t* __restrict__ file_off,
                              uint32_t F, uint8_t* __restrict__ file_start) {
  uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  uint64_t a = file_off[f], b = file_off[f + 1];
  if (a >= b) return;
  uint32_t lo = 0, hi = L;  // first line with start >= a
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (line_start[mid] < a) lo = mid + 1;
    else hi = mid;
  }
  if (lo < L) file_start[lo] = 1;
}

__global__ void k_classify(const uint8_t* __restrict__ text, const uint32_t* __restrict__ line_start, uint32_t L,
                           const uint8_t* __restrict__ file_start, uint8_t* __restrict__ kind, uint32_t* __restrict__ mk,
                           uint32_t* __restrict__ fs, uint32_t* __restrict__ kf) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const uint8_t* p = text + line_start[i];
  const uint8_t* e = text + line_start[i + 1] - 1;  // the '\n'
  while (p < e && is_space(*p)) ++p;
  while (e > p && is_space(e[-1])) --e;
  uint8_t k = LK_BLANK;
  if (p < e && !(*p == '#' || *p == ';' || (e - p >= 2 && p[0] == '/' && p[1] == '/'))) {
    const uint8_t* t = p;
    while (t < e && !is_space(*t)) ++t;
    if (tok_eq(p, t, ".kernel")) k = LK_KERNEL;
    else if (tok_eq(p, t, ".config")) k = LK_CONFIG;
    else if (tok_eq(p, t, ".text")) k = LK_TEXT;
    else if (t == e && e - p >= 2 && e[-1] == ':') k = LK_LABEL;
    else k = LK_ROW;
  }
  kind[i] = k;
  mk[i] = (k == LK_KERNEL || k == LK_CONFIG || k == LK_TEXT) ? i + 1 : 0;
  fs[i] = file_start[i] ? i + 1 : 0;
  kf[i] = k == LK_KERNEL ? 1 : 0;
}

// row type of every line: state from the last marker, kernel from the .kernel count
__global__ void k_assign(const uint8_t* __restrict__ kind, const uint32_t* __restrict__ mkmax,
                         const uint32_t* __restrict__ fsmax, const uint32_t* __restrict__ kcnt, uint32_t L,
                         uint8_t* __restrict__ rowtype, uint32_t* __restrict__ is_instr, uint32_t* __restrict__ is_label,
                         uint32_t* __restrict__ is_cfg) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  uint8_t rt = RT_NONE;
  uint32_t f0 = fsmax[i] - 1;  // a file start precedes every line
  uint32_t before = kcnt[f0] - (kind[f0] == LK_KERNEL ? 1u : 0u);
  if (kcnt[i] > before) {  // a .kernel row of this file has been seen
    uint8_t k = kind[i];
    uint8_t st = kind[mkmax[i] - 1];
    if (k == LK_KERNEL) rt = RT_KERNEL;
    else if (k == LK_LABEL || k == LK_ROW) {
      if (st == LK_CONFIG) rt = RT_CFG;
      else if (st == LK_TEXT) rt = k == LK_LABEL ? RT_LABEL : RT_INSTR;
    }
  }
  rowtype[i] = rt;
  is_instr[i] = rt == RT_INSTR;
  is_label[i] = rt == RT_LABEL;
  is_cfg[i] = rt == RT_CFG;
}

__global__ void k_scatter_rows(const uint8_t* __restrict__ rowtype, const uint32_t* __restrict__ instr_excl,
                               const uint32_t* __restrict__ label_excl, const uint32_t* __restrict__ cfg_excl,
                               const uint32_t* __restrict__ kcnt, uint32_t L, uint32_t* __restrict__ instr_line,
                               uint32_t* __restrict__ label_line, uint32_t* __restrict__ label_instr,
                               uint32_t* __restrict__ cfg_line, KHdr* __restrict__ kh) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  uint8_t rt = rowtype[i];
  if (rt == RT_INSTR) instr_line[instr_excl[i]] = i;
  else if (rt == RT_LABEL) {
    label_line[label_excl[i]] = i;
    label_instr[label_excl[i]] = instr_excl[i];
  } else if (rt == RT_CFG) {
    cfg_line[cfg_excl[i]] = i;
  } else if (rt == RT_KERNEL) {
    KHdr& k = kh[kcnt[i] - 1];
    k.line = i;
    k.first_instr = instr_excl[i];
    k.first_label = label_excl[i];
    k.first_cfg = cfg_excl[i];
  }
}

void launch_rows(const uint8_t* text, const uint32_t* line_start, uint32_t L, const uint64_t* file_off, uint32_t F,
                 RowArrays& ra, ScanScratch sc, uint32_t* totals, uint32_t* err, cudaStream_t s) {
  const int T = 256;
  cudaMemsetAsync(ra.file_start, 0, L, s);
  if (F) {
    k_file_starts<<<(F + T - 1) / T, T, 0, s>>>(line_start, L, file_off, F, ra.file_start);
    ++launch_counter();
  }
  k_classify<<<(L + T - 1) / T, T, 0, s>>>(text, line_start, L, ra.file_start, ra.kind, ra.t0, ra.t1, ra.t2);
  ++launch_counter();
  launch_scan(ra.t0, ra.mkmax, L, 1, true, sc, nullptr, err, s);
  launch_scan(ra.t1, ra.fsmax, L, 1, true, sc, nullptr, err, s);
  launch_scan(ra.t2, ra.kcnt, L, 0, true, sc, &totals[0], err, s);  // totals[0] = kernels
  k_assign<<<(L + T - 1) / T, T, 0, s>>>(ra.kind, ra.mkmax, ra.fsmax, ra.kcnt, L, ra.rowtype, ra.t0, ra.t1, ra.t2);
  ++launch_counter();
  launch_scan(ra.t0, ra.instr_excl, L, 0, false, sc, &totals[1], err, s);  // totals[1] = instructions
  launch_scan(ra.t1, ra.label_excl, L, 0, false, sc, &totals[2], err, s);  // totals[2] = labels
  launch_scan(ra.t2, ra.cfg_excl, L, 0, false, sc, &totals[14], err, s);   // totals[14] = configuration rows
}

void launch_scatter_rows(uint32_t L, RowArrays& ra, uint32_t* instr_line, uint32_t* label_line, uint32_t* label_instr,
                         uint32_t* cfg_line, KHdr* kh, cudaStream_t s) {
  const int T = 256;
  k_scatter_rows<<<(L + T - 1) / T, T, 0, s>>>(ra.rowtype, ra.instr_excl, ra.label_excl, ra.cfg_excl, ra.kcnt, L,
                                               instr_line, label_line, label_instr, cfg_line, kh);
  ++launch_counter();
}

}  // namespace gd
