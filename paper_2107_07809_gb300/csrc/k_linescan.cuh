// k_linescan.cuh — the single-pass S1 newline scan (line tokenisation of
// Listing 2's `for current_row in file`): used by the batch pipeline for small
// texts (k_text.cu, which takes a two-pass count/scan/write form for large
// ones) and by the allocation-free entry point (k_noalloc.cu).
//
// One 512-thread block per 32 KiB tile, four blocks resident per SM: the tile
// comes into shared memory with one bulk copy (cp.async.bulk + mbarrier).
// Tile ids come from an atomic counter in block start order, so the
// single-pass decoupled look-back (warp 0) that gives each tile the number of
// newlines before it only waits for tiles whose blocks already run.
//
// The look-back bounds this form: every block waits until its predecessors
// publish, so on large texts it reaches about a fifth of the copy bandwidth.
// Widening the look-back window (256 predecessors per round trip) measured
// slower, not faster; the two-pass form avoids the wait altogether.
//
// Within a tile each thread reads four 16-byte chunks at stride 8 KiB (thread
// t, chunk k: bytes (k*512 + t)*16 ..+16), so the reads of a warp from shared
// memory are conflict-free and the line starts it writes for one chunk row are
// consecutive.  The four chunk counts of a thread are packed into one 64-bit
// value (16 bits each: at most 8192 newlines per chunk row), so one block scan
// ranks every newline of the tile.
#pragma once
#include "gd_common.cuh"

namespace gd {

constexpr int LS_THREADS = 512;
constexpr int LS_CHUNKS = 4;                              // 16-byte chunks per thread and tile
constexpr uint32_t LS_TILE = LS_THREADS * 16 * LS_CHUNKS;  // 32 KiB
constexpr int LS_WARPS = LS_THREADS / 32;

struct LineScanSmem {
  __align__(128) uint8_t buf[LS_TILE];
  __align__(8) uint64_t mbar;
  uint64_t warp[LS_WARPS];
  uint32_t tile;
  uint32_t prefix;
};

struct LineScanArgs {
  const uint8_t* text;
  uint64_t n;
  int use_bulk;          // text is 16-byte aligned: the tile moves by bulk copy
  uint32_t* line_start;  // [0] = 0, [1 + r] = 1 + offset of the r-th '\n'
  uint64_t cap;          // entries line_start may receive
  uint64_t* status;      // look-back word per tile, zeroed before the launch
  uint32_t* counter;     // tile counter, zeroed before the launch
  uint32_t ntiles;
  uint32_t* lines_out;   // receives the number of '\n' bytes
  uint32_t* err;
};

__device__ __forceinline__ uint32_t ls_newlines(uint32_t w) { return __vcmpeq4(w, 0x0A0A0A0Au); }

__device__ __forceinline__ uint64_t ls_block_scan(uint64_t v, LineScanSmem& sm, uint64_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if ((int)lane >= o) v += t;
  }
  if (lane == 31) sm.warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < LS_WARPS ? sm.warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < LS_WARPS; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if ((int)lane >= o) w += t;
    }
    if (lane < LS_WARPS) sm.warp[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += sm.warp[warp - 1];
  *total = sm.warp[LS_WARPS - 1];
  return v;
}

// one tile: every block of the grid runs this once
__device__ __forceinline__ void line_scan_tile(LineScanSmem& sm, const LineScanArgs& a) {
  const uint32_t tid = threadIdx.x;
  if (tid == 0) sm.tile = atomicAdd(a.counter, 1u);
  __syncthreads();
  const uint32_t tile = sm.tile;
  const uint64_t base = (uint64_t)tile * LS_TILE;
  const uint64_t rem = a.n > base ? a.n - base : 0;
  const uint32_t nbytes = rem < LS_TILE ? (uint32_t)rem : LS_TILE;
  // bulk-copy part: a 16-byte multiple from a 16-byte aligned source (a text that
  // does not start 16-byte aligned is read with plain loads)
  const uint32_t bulk = a.use_bulk ? (nbytes & ~15u) : 0u;
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&sm.mbar);
  if (tid == 0 && bulk) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(sm.buf);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bulk) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(a.text + base), "r"(bulk), "r"(mb)
        : "memory");
  }
  for (uint32_t j = bulk + tid; j < LS_TILE; j += LS_THREADS) sm.buf[j] = j < nbytes ? a.text[base + j] : 0;
  __syncthreads();  // the barrier is initialised before anyone waits on it
  if (bulk) {
    uint32_t done = 0, spins = 0;
    while (!done) {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
          : "=r"(done)
          : "r"(mb)
          : "memory");
      if (!done && ++spins > (1u << 22)) {  // the copy never landed: flag it (the output is invalid)
        atomicOr(a.err, ERR_MBAR);
        break;
      }
    }
  }
  uint4 w[LS_CHUNKS];
  uint64_t packed = 0;
#pragma unroll
  for (int k = 0; k < LS_CHUNKS; ++k) {
    w[k] = *reinterpret_cast<const uint4*>(sm.buf + ((uint32_t)k * LS_THREADS + tid) * 16);
    const uint32_t c = (__popc(ls_newlines(w[k].x)) + __popc(ls_newlines(w[k].y)) + __popc(ls_newlines(w[k].z)) +
                        __popc(ls_newlines(w[k].w))) >> 3;
    packed |= (uint64_t)c << (16 * k);
  }
  uint64_t tot;
  const uint64_t incl = ls_block_scan(packed, sm, &tot);
  const uint64_t excl = incl - packed;
  const uint32_t t0 = (uint32_t)(tot & 0xFFFF), t1 = (uint32_t)((tot >> 16) & 0xFFFF),
                 t2 = (uint32_t)((tot >> 32) & 0xFFFF), t3 = (uint32_t)(tot >> 48);
  const uint32_t count = t0 + t1 + t2 + t3;
  if (tid < 32) {  // warp 0: decoupled look-back
    const uint32_t p = lookback<ScanSum>(a.status, tile, count, a.err);
    if (tid == 0) {
      sm.prefix = p;
      if (tile == a.ntiles - 1) *a.lines_out = p + count;
    }
  }
  __syncthreads();
  const uint32_t prefix = sm.prefix;
  if (tile == 0 && tid == 0) a.line_start[0] = 0;
  const uint32_t row_base[LS_CHUNKS] = {0, t0, t0 + t1, t0 + t1 + t2};
  bool over = false;
#pragma unroll
  for (int k = 0; k < LS_CHUNKS; ++k) {
    uint64_t rank = (uint64_t)prefix + row_base[k] + (uint32_t)((excl >> (16 * k)) & 0xFFFF);
    const uint64_t at = base + ((uint64_t)k * LS_THREADS + tid) * 16;
    const uint32_t ws[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t m = ls_newlines(ws[q]);
      while (m) {
        const uint32_t byte = (uint32_t)(__ffs(m) - 1) >> 3;  // lowest byte first = text order
        const uint64_t slot = 1 + rank++;
        if (slot < a.cap) a.line_start[slot] = (uint32_t)(at + q * 4 + byte + 1);
        else over = true;
        m &= ~(0xFFu << (byte * 8));
      }
    }
  }
  if (over) atomicOr(a.err, ERR_CAPACITY);
}

}  // namespace gd
