// k_noalloc.cu — line tokenisation (the S1 newline scan) for callers that must
// not allocate device memory.
//
// The batch pipeline keeps its scan scratch (per-tile look-back status and the
// dynamic tile counter) in memory the handle allocates.  Some callers cannot
// let a library allocate: code that runs while a CUDA graph of theirs is being
// captured (cudaMalloc is not a capturable operation), code inside a
// memory-pool discipline that forbids foreign allocations, or a process that
// has already reserved all device memory it will use.  For them this file
// offers the same scan with its scratch in a fixed-size file-scope __device__
// array: the call allocates nothing, neither through the CUDA runtime nor
// through any library.
//
// Scratch: kNaMaxTiles look-back words (8 bytes each) plus one tile counter,
// 512 KiB in all, enough for texts up to kNaMaxTiles * 16 KiB = 1 GiB.  Longer
// texts are rejected on the host before anything is queued.  The look-back
// words of the tiles a call uses and the tile counter must start at zero; the
// call clears them on its stream before the scan kernel.
//
// The scratch is one array per device and per process, shared by every call
// on that device: two calls whose work overlaps on the device (different
// streams, or different host threads) race on it and give wrong results.
// Callers serialise such calls (one stream, or events between streams).
//
// Set-up: the first call on a device, with that device current, looks up the
// scratch array's device address once (cudaGetSymbolAddress) and caches it.
// That first lookup may load the module and is not a stream operation, so the
// first call on each device should happen before any stream capture begins.
#include <cstdint>
#include <mutex>

#include "../../include/gcn_decomp.h"
#include "gd_kernels.h"

namespace gd {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 64;
constexpr int NA_TILE = NA_THREADS * NA_PER_THREAD;  // 16 KiB of text per block
constexpr uint32_t kNaMaxTiles = 65536;               // 1 GiB of text
constexpr int kNaMaxDevices = 64;

// [0, kNaMaxTiles): look-back status per tile; [kNaMaxTiles]: tile counter
static __device__ __align__(256) uint64_t g_na_scratch[kNaMaxTiles + 1];

std::mutex g_na_mu;
uint64_t* g_na_ptr[kNaMaxDevices];  // scratch address per device, set once

// The S1 scan with three differences from the batch kernel: the tile counter
// and look-back words come from the static scratch, a text pointer that is not
// 16-byte aligned is read with plain loads instead of the bulk copy, and the
// line-start writes are bounded by the caller's capacity (ERR_CAPACITY when the
// text has more lines than fit).
__global__ void __launch_bounds__(NA_THREADS)
    k_line_scan_static(const uint8_t* __restrict__ text, uint64_t n, int use_bulk, uint32_t* __restrict__ line_start,
                       uint64_t cap, uint64_t* __restrict__ status, uint32_t* result) {
  __shared__ __align__(128) uint8_t buf[NA_TILE];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tile, s_prefix, s_warp[32];
  uint32_t* err = result + 1;
  uint32_t* counter = reinterpret_cast<uint32_t*>(status + kNaMaxTiles);
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * NA_TILE;
  const uint64_t rem = n > base ? n - base : 0;
  const uint32_t nbytes = rem < (uint64_t)NA_TILE ? (uint32_t)rem : (uint32_t)NA_TILE;
  const uint32_t bulk = use_bulk ? (nbytes & ~15u) : 0u;
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf);
  if (threadIdx.x == 0 && bulk) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bulk) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(text + base), "r"(bulk), "r"(mb)
        : "memory");
  }
  for (uint32_t j = bulk + threadIdx.x; j < (uint32_t)NA_TILE; j += blockDim.x) buf[j] = j < nbytes ? text[base + j] : 0;
  __syncthreads();
  if (bulk) {
    uint32_t done = 0, spins = 0;
    while (!done) {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
          : "=r"(done)
          : "r"(mb)
          : "memory");
      if (!done && ++spins > (1u << 22)) {
        atomicOr(err, ERR_MBAR);
        break;
      }
    }
  }
  const uint4* mine = reinterpret_cast<const uint4*>(buf + threadIdx.x * NA_PER_THREAD);
  uint4 w[4];
  uint32_t cnt = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[k] = mine[k];
    cnt += __popc(__vcmpeq4(w[k].x, 0x0A0A0A0Au)) + __popc(__vcmpeq4(w[k].y, 0x0A0A0A0Au)) +
           __popc(__vcmpeq4(w[k].z, 0x0A0A0A0Au)) + __popc(__vcmpeq4(w[k].w, 0x0A0A0A0Au));
  }
  cnt >>= 3;
  uint32_t total;
  uint32_t incl = block_incl_scan<ScanSum>(cnt, s_warp, &total);
  if (threadIdx.x < 32) {
    uint32_t p = lookback<ScanSum>(status, tile, total, err);
    if (threadIdx.x == 0) {
      s_prefix = p;
      if (tile == gridDim.x - 1) result[0] = p + total;  // number of lines
    }
  }
  __syncthreads();
  uint64_t rank = (uint64_t)s_prefix + incl - cnt;
  if (tile == 0 && threadIdx.x == 0) line_start[0] = 0;
  const uint64_t my0 = base + (uint64_t)threadIdx.x * NA_PER_THREAD;
  bool over = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint32_t ws[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t m = __vcmpeq4(ws[q], 0x0A0A0A0Au);
      while (m) {
        int bit = __ffs(m) - 1;
        uint32_t byte = (uint32_t)bit >> 3;
        uint64_t slot = 1 + rank++;
        if (slot < cap)
          line_start[slot] = (uint32_t)(my0 + k * 16 + q * 4 + byte + 1);
        else
          over = true;
        m &= ~(0xFFu << (byte * 8));
      }
    }
  }
  if (over) atomicOr(err, ERR_CAPACITY);
}

uint64_t* scratch_for_current_device(int* dev_out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_api_error(cudaGetErrorString(e));
    return nullptr;
  }
  if (dev < 0 || dev >= kNaMaxDevices) {
    set_api_error("device ordinal beyond the static scratch table");
    return nullptr;
  }
  *dev_out = dev;
  std::lock_guard<std::mutex> g(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      set_api_error(e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned NULL");
      return nullptr;
    }
    g_na_ptr[dev] = static_cast<uint64_t*>(p);
  }
  return g_na_ptr[dev];
}

}  // namespace
}  // namespace gd

extern "C" int gcn_decomp_line_starts_noalloc(const uint8_t* d_text, uint64_t text_len, uint32_t* d_line_start,
                                              uint64_t line_cap, uint32_t* d_result, void* stream) {
  using namespace gd;
  if ((!d_text && text_len) || !d_line_start || line_cap == 0 || !d_result) {
    set_api_error("bad argument");
    return GCN_EINVAL;
  }
  const uint64_t tiles64 = text_len ? (text_len + NA_TILE - 1) / NA_TILE : 1;
  if (tiles64 > kNaMaxTiles) {
    set_api_error("text longer than the static scratch allows (1 GiB)");
    return GCN_ENOMEM;
  }
  const uint32_t tiles = (uint32_t)tiles64;
  int dev = -1;
  uint64_t* scratch = scratch_for_current_device(&dev);
  if (!scratch) return GCN_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint64_t) * tiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kNaMaxTiles, 0, sizeof(uint64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_result, 0, 2 * sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    const int use_bulk = (reinterpret_cast<uintptr_t>(d_text) & 15u) == 0;
    k_line_scan_static<<<tiles, NA_THREADS, 0, s>>>(d_text, text_len, use_bulk, d_line_start, line_cap, scratch,
                                                     d_result);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_api_error(cudaGetErrorString(e));
    return GCN_ECUDA;
  }
  return GCN_OK;
}
