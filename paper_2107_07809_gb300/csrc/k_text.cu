// k_text.cu — tokenisation and body extraction on the GPU.
//
// S1 (line tokenisation): the line start after every newline, by rank.  A
// text of more than kLsOnePass tiles takes two passes and a scan: the count
// pass reads the text once (32 KiB tiles, coalesced 16-byte loads) and writes
// each tile's newline count and a newline bit mask (one bit per text byte, an
// eighth of the text); the tile counts are scanned; the write pass reads the
// masks, ranks the newlines of its tile with a block scan, stages the line
// starts in shared memory in rank order and stores them contiguously.  This
// moves the text once and about a quarter of its size more, with no waiting
// between blocks: measured twice as fast as the single-pass scan with
// decoupled look-back on 200 MB and 2 GB texts, whose look-back holds every
// block until its predecessors publish.  A small text (one launch matters
// more than bandwidth there) keeps the single pass (k_linescan.cuh), which the
// allocation-free entry point also uses.
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

// the newline bits of 16 text bytes (bit j: byte j is '\n')
__device__ __forceinline__ uint32_t nl_mask16(uint4 w) {
  uint32_t m = 0;
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t x = ls_newlines(ws[q]);  // 0xFF in every '\n' byte
    m |= (((x >> 7) & 1u) | ((x >> 14) & 2u) | ((x >> 21) & 4u) | ((x >> 28) & 8u)) << (4 * q);
  }
  return m;
}

// count pass: tile t, thread t', row k covers text bytes (k * LS_THREADS + t') * 16 ..+16 of the
// tile; its mask is masks[t * LS_CHUNK_MASKS + k * LS_THREADS + t'] (chunk order = text order)
constexpr uint32_t LS_CHUNK_MASKS = LS_TILE / 16;
static_assert(LS_TILE == kLsTileBytes, "the scratch the pass sizes is per LS_TILE");
__global__ void __launch_bounds__(LS_THREADS) k_ls_count(const uint8_t* __restrict__ text, uint64_t n, int vec,
                                                         uint32_t* __restrict__ counts, uint16_t* __restrict__ masks) {
  __shared__ uint32_t s_warp[LS_WARPS];
  const uint32_t tile = blockIdx.x, tid = threadIdx.x;
  const uint64_t base = (uint64_t)tile * LS_TILE;
  uint4 w[LS_CHUNKS];
#pragma unroll
  for (int k = 0; k < LS_CHUNKS; ++k) {
    const uint64_t at = base + ((uint64_t)k * LS_THREADS + tid) * 16;
    if (vec && at + 16 <= n) {
      w[k] = __ldcs(reinterpret_cast<const uint4*>(text + at));
    } else {  // the tail, or a text that does not start 16-byte aligned
      uint32_t t[4] = {0, 0, 0, 0};
      for (int q = 0; q < 16; ++q)
        if (at + q < n) t[q / 4] |= (uint32_t)text[at + q] << (8 * (q % 4));
      w[k] = make_uint4(t[0], t[1], t[2], t[3]);
    }
  }
  uint32_t c = 0;
  uint16_t* mk = masks + (uint64_t)tile * LS_CHUNK_MASKS;
#pragma unroll
  for (int k = 0; k < LS_CHUNKS; ++k) {
    const uint32_t m = nl_mask16(w[k]);
    mk[k * LS_THREADS + tid] = (uint16_t)m;
    c += __popc(m);
  }
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((tid & 31) == 0) s_warp[tid >> 5] = c;
  __syncthreads();
  if (tid < 32) {
    uint32_t v = tid < LS_WARPS ? s_warp[tid] : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (tid == 0) counts[tile] = v;
  }
}

// write pass: the tile's masks, its newlines ranked by a block scan of the packed row counts
// (ls_block_scan), the line starts staged in rank order and stored contiguously (a tile of more
// newlines than the stage holds stores them in place)
__global__ void __launch_bounds__(LS_THREADS) k_ls_write(const uint16_t* __restrict__ masks, const uint32_t* __restrict__ prefix,
                                                         uint32_t* __restrict__ line_start, uint64_t cap, uint32_t* err) {
  __shared__ LineScanSmem sm;
  const uint32_t tile = blockIdx.x, tid = threadIdx.x;
  const uint64_t base = (uint64_t)tile * LS_TILE;
  const uint16_t* mk = masks + (uint64_t)tile * LS_CHUNK_MASKS;
  uint32_t m[LS_CHUNKS];
  uint64_t packed = 0;
#pragma unroll
  for (int k = 0; k < LS_CHUNKS; ++k) {
    m[k] = __ldcs(mk + k * LS_THREADS + tid);
    packed |= (uint64_t)__popc(m[k]) << (16 * k);
  }
  uint64_t tot;
  const uint64_t incl = ls_block_scan(packed, sm, &tot);
  const uint64_t excl = incl - packed;
  const uint32_t t0 = (uint32_t)(tot & 0xFFFF), t1 = (uint32_t)((tot >> 16) & 0xFFFF),
                 t2 = (uint32_t)((tot >> 32) & 0xFFFF), t3 = (uint32_t)(tot >> 48);
  const uint32_t count = t0 + t1 + t2 + t3;
  const uint64_t first = 1 + (uint64_t)prefix[tile];  // slot of the tile's first line start
  if (tile == 0 && tid == 0) line_start[0] = 0;
  if (first + count > cap) {  // cannot happen (a line start per byte at most): flag, write nothing
    if (tid == 0) atomicOr(err, ERR_CAPACITY);
    return;
  }
  const uint32_t row_base[LS_CHUNKS] = {0, t0, t0 + t1, t0 + t1 + t2};
  uint32_t* st = reinterpret_cast<uint32_t*>(sm.buf);
  constexpr uint32_t kStage = LS_TILE / 4;  // line starts the tile buffer holds
  const bool staged = count <= kStage;
#pragma unroll
  for (int k = 0; k < LS_CHUNKS; ++k) {
    uint32_t rank = row_base[k] + (uint32_t)((excl >> (16 * k)) & 0xFFFF);
    const uint32_t at = (uint32_t)(base + ((uint64_t)k * LS_THREADS + tid) * 16) + 1;
    uint32_t x = m[k];
    while (x) {
      const uint32_t v = at + (uint32_t)(__ffs(x) - 1);
      if (staged) st[rank] = v;
      else line_start[first + rank] = v;
      ++rank;
      x &= x - 1;
    }
  }
  if (!staged) return;
  __syncthreads();
  uint32_t* dst = line_start + first;
  for (uint32_t j = tid; j < count; j += LS_THREADS) dst[j] = st[j];
}

void launch_line_scan(const uint8_t* text, uint64_t n, uint32_t* line_start, uint64_t* tile_status,
                      uint32_t* counters, uint32_t* err, const LineScan2& two, cudaStream_t s) {
  uint32_t tiles = (uint32_t)((n + LS_TILE - 1) / LS_TILE);
  if (!tiles) tiles = 1;
  if (tiles > kLsOnePass) {
    ktime(KT_LINE_SCAN, 0, s);
    k_ls_count<<<tiles, LS_THREADS, 0, s>>>(text, n, (reinterpret_cast<uintptr_t>(text) & 15u) == 0, two.counts,
                                            two.masks);
    ++launch_counter();
    launch_scan(two.counts, two.prefix, tiles, 0, false, ScanScratch{tile_status, &counters[0]}, &counters[1], err, s);
    k_ls_write<<<tiles, LS_THREADS, 0, s>>>(two.masks, two.prefix, line_start, n + 2, err);
    ++launch_counter();
    ktime(KT_LINE_SCAN, 1, s);
    return;
  }
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
// A tile of 4096 elements per 256-thread block.  The tile moves between global and shared memory
// in 16-byte pieces (four consecutive elements per thread and row, when both arrays are 16-byte
// aligned) and sits in shared memory with a pad word after every 32, so that a thread's run of 16
// consecutive elements (the sequential part of the scan) and the rows of 16-byte pieces both read
// and write without bank conflicts.
constexpr int SC_THREADS = 256, SC_ITEMS = 16, SC_TILE = SC_THREADS * SC_ITEMS;
constexpr int SC_ROWS = SC_ITEMS / 4;  // rows of 4 * SC_THREADS elements
__device__ __forceinline__ uint32_t sc_at(uint32_t e) { return e + (e >> 5); }

template <class Op, bool Incl>
__global__ void __launch_bounds__(SC_THREADS) k_scan(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     uint32_t n, uint64_t* status, uint32_t* counter,
                                                     uint32_t* total_out, uint32_t* err) {
  __shared__ uint32_t sm[SC_TILE + SC_TILE / 32];
  __shared__ uint32_t s_tile, s_prefix, s_warp[32];
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * SC_TILE;
  const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
#pragma unroll
  for (int r = 0; r < SC_ROWS; ++r) {
    const uint32_t e = 4 * (threadIdx.x + r * SC_THREADS);  // the first of four consecutive elements
    const uint64_t i = base + e;
    uint32_t x[4];
    if (vec && i + 3 < n) {
      const uint4 q = *reinterpret_cast<const uint4*>(in + i);
      x[0] = q.x, x[1] = q.y, x[2] = q.z, x[3] = q.w;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = i + c < n ? in[i + c] : Op::id;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sm[sc_at(e + c)] = x[c];
  }
  __syncthreads();
  uint32_t v[SC_ITEMS];
  uint32_t acc = Op::id;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    acc = Op::op(acc, sm[sc_at(threadIdx.x * SC_ITEMS + k)]);
    v[k] = acc;
  }
  uint32_t total;
  uint32_t incl = block_incl_scan<Op>(acc, s_warp, &total);
  // exclusive prefix of this thread inside the tile: the previous thread's inclusive value
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
    sm[sc_at(threadIdx.x * SC_ITEMS + k)] = Incl ? r : run;
    run = r;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SC_ROWS; ++r) {
    const uint32_t e = 4 * (threadIdx.x + r * SC_THREADS);
    const uint64_t i = base + e;
    uint32_t x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = sm[sc_at(e + c)];
    if (vec && i + 3 < n) {
      *reinterpret_cast<uint4*>(out + i) = make_uint4(x[0], x[1], x[2], x[3]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (i + c < n) out[i + c] = x[c];
    }
  }
}

// Three scans of the same length in one pass (S2's row scans): each block stages a 2048-element
// tile of every channel, scans the three locally, and warps 0, 1 and 2 run the three look-backs
// side by side (channel c's status words at status + c * tiles).
constexpr int S3_ITEMS = 8, S3_TILE = SC_THREADS * S3_ITEMS;

template <class Op>
__device__ __forceinline__ void s3_stage(const uint32_t* __restrict__ in, uint32_t* sm, uint64_t base, uint32_t n,
                                         bool vec) {
#pragma unroll
  for (int r = 0; r < S3_ITEMS / 4; ++r) {
    const uint32_t e = 4 * (threadIdx.x + r * SC_THREADS);
    const uint64_t i = base + e;
    uint32_t x[4];
    if (vec && i + 3 < n) {
      const uint4 q = *reinterpret_cast<const uint4*>(in + i);
      x[0] = q.x, x[1] = q.y, x[2] = q.z, x[3] = q.w;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = i + c < n ? in[i + c] : Op::id;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sm[sc_at(e + c)] = x[c];
  }
}

// the thread's inclusive run over its S3_ITEMS elements (v), and the exclusive prefix of the run
// inside the tile; *total = the tile's aggregate
template <class Op>
__device__ __forceinline__ uint32_t s3_local(const uint32_t* sm, uint32_t* v, uint32_t* s_warp, uint32_t* total) {
  uint32_t acc = Op::id;
#pragma unroll
  for (int k = 0; k < S3_ITEMS; ++k) {
    acc = Op::op(acc, sm[sc_at(threadIdx.x * S3_ITEMS + k)]);
    v[k] = acc;
  }
  const uint32_t incl = block_incl_scan<Op>(acc, s_warp, total);
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  return lane ? prev : (warp ? s_warp[warp - 1] : Op::id);
}

template <class Op, bool Incl>
__device__ __forceinline__ void s3_write(uint32_t* sm, const uint32_t* v, uint32_t pre) {
  uint32_t run = pre;
#pragma unroll
  for (int k = 0; k < S3_ITEMS; ++k) {
    const uint32_t r = Op::op(pre, v[k]);
    sm[sc_at(threadIdx.x * S3_ITEMS + k)] = Incl ? r : run;
    run = r;
  }
}

__device__ __forceinline__ void s3_store(const uint32_t* sm, uint32_t* __restrict__ out, uint64_t base, uint32_t n,
                                         bool vec) {
#pragma unroll
  for (int r = 0; r < S3_ITEMS / 4; ++r) {
    const uint32_t e = 4 * (threadIdx.x + r * SC_THREADS);
    const uint64_t i = base + e;
    uint32_t x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = sm[sc_at(e + c)];
    if (vec && i + 3 < n) {
      *reinterpret_cast<uint4*>(out + i) = make_uint4(x[0], x[1], x[2], x[3]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (i + c < n) out[i + c] = x[c];
    }
  }
}

struct Scan3 {
  const uint32_t* in[3];
  uint32_t* out[3];
  uint32_t n;
  uint64_t* status;  // 3 * tiles words, zeroed before the launch
  uint32_t* counter;
  uint32_t* total_out[3];  // null: not wanted
  uint32_t* err;
};

template <class O0, class O1, class O2, bool Incl>
__global__ void __launch_bounds__(SC_THREADS) k_scan3(const __grid_constant__ Scan3 a) {
  __shared__ uint32_t sm[3][S3_TILE + S3_TILE / 32];
  __shared__ uint32_t s_tile, s_prefix[3], s_warp[3][32];
  if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * S3_TILE;
  bool vec = true;
  for (int c = 0; c < 3; ++c)
    vec = vec && ((reinterpret_cast<uintptr_t>(a.in[c]) | reinterpret_cast<uintptr_t>(a.out[c])) & 15u) == 0;
  s3_stage<O0>(a.in[0], sm[0], base, a.n, vec);
  s3_stage<O1>(a.in[1], sm[1], base, a.n, vec);
  s3_stage<O2>(a.in[2], sm[2], base, a.n, vec);
  __syncthreads();
  uint32_t v0[S3_ITEMS], v1[S3_ITEMS], v2[S3_ITEMS], t0, t1, t2;
  const uint32_t x0 = s3_local<O0>(sm[0], v0, s_warp[0], &t0);
  const uint32_t x1 = s3_local<O1>(sm[1], v1, s_warp[1], &t1);
  const uint32_t x2 = s3_local<O2>(sm[2], v2, s_warp[2], &t2);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const bool last = tile == gridDim.x - 1;
  if (warp == 0) {
    const uint32_t p = lookback<O0>(a.status, tile, t0, a.err);
    if (lane == 0) {
      s_prefix[0] = p;
      if (last && a.total_out[0]) *a.total_out[0] = O0::op(p, t0);
    }
  } else if (warp == 1) {
    const uint32_t p = lookback<O1>(a.status + gridDim.x, tile, t1, a.err);
    if (lane == 0) {
      s_prefix[1] = p;
      if (last && a.total_out[1]) *a.total_out[1] = O1::op(p, t1);
    }
  } else if (warp == 2) {
    const uint32_t p = lookback<O2>(a.status + 2ull * gridDim.x, tile, t2, a.err);
    if (lane == 0) {
      s_prefix[2] = p;
      if (last && a.total_out[2]) *a.total_out[2] = O2::op(p, t2);
    }
  }
  __syncthreads();
  s3_write<O0, Incl>(sm[0], v0, O0::op(s_prefix[0], x0));
  s3_write<O1, Incl>(sm[1], v1, O1::op(s_prefix[1], x1));
  s3_write<O2, Incl>(sm[2], v2, O2::op(s_prefix[2], x2));
  __syncthreads();
  s3_store(sm[0], a.out[0], base, a.n, vec);
  s3_store(sm[1], a.out[1], base, a.n, vec);
  s3_store(sm[2], a.out[2], base, a.n, vec);
}

template <class O0, class O1, class O2, bool Incl>
static void launch_scan3(Scan3 a, cudaStream_t s) {
  uint32_t tiles = (a.n + S3_TILE - 1) / S3_TILE;
  if (!tiles) tiles = 1;
  cudaMemsetAsync(a.status, 0, sizeof(uint64_t) * 3 * tiles, s);
  cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), s);
  k_scan3<O0, O1, O2, Incl><<<tiles, SC_THREADS, 0, s>>>(a);
  ++launch_counter();
}
uint32_t scan3_status_words(uint32_t n) { return 3 * ((n + S3_TILE - 1) / S3_TILE + 1); }

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
                 RowArrays& ra, ScanScratch sc, uint64_t* status3, uint32_t* totals, uint32_t* err, cudaStream_t s) {
  const int T = 256;
  cudaMemsetAsync(ra.file_start, 0, L, s);
  if (F) {
    k_file_starts<<<(F + T - 1) / T, T, 0, s>>>(line_start, L, file_off, F, ra.file_start);
    ++launch_counter();
  }
  k_classify<<<(L + T - 1) / T, T, 0, s>>>(text, line_start, L, ra.file_start, ra.kind, ra.t0, ra.t1, ra.t2);
  ++launch_counter();
  // the last state marker, the last file start (inclusive maxima) and the running .kernel count
  launch_scan3<ScanMax, ScanMax, ScanSum, true>(
      Scan3{{ra.t0, ra.t1, ra.t2}, {ra.mkmax, ra.fsmax, ra.kcnt}, L, status3, sc.counter,
            {nullptr, nullptr, &totals[0]}, err},  // totals[0] = kernels
      s);
  k_assign<<<(L + T - 1) / T, T, 0, s>>>(ra.kind, ra.mkmax, ra.fsmax, ra.kcnt, L, ra.rowtype, ra.t0, ra.t1, ra.t2);
  ++launch_counter();
  // ranks of the instruction, label and configuration rows; totals[1] = instructions, totals[2] =
  // labels, totals[14] = configuration rows
  launch_scan3<ScanSum, ScanSum, ScanSum, false>(
      Scan3{{ra.t0, ra.t1, ra.t2}, {ra.instr_excl, ra.label_excl, ra.cfg_excl}, L, status3, sc.counter,
            {&totals[1], &totals[2], &totals[14]}, err},
      s);
}

void launch_scatter_rows(uint32_t L, RowArrays& ra, uint32_t* instr_line, uint32_t* label_line, uint32_t* label_instr,
                         uint32_t* cfg_line, KHdr* kh, cudaStream_t s) {
  const int T = 256;
  k_scatter_rows<<<(L + T - 1) / T, T, 0, s>>>(ra.rowtype, ra.instr_excl, ra.label_excl, ra.cfg_excl, ra.kcnt, L,
                                               instr_line, label_line, label_instr, cfg_line, kh);
  ++launch_counter();
}

}  // namespace gd
