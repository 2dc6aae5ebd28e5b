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
// 256 KiB in all, enough for texts up to kNaMaxTiles * 32 KiB = 1 GiB.  Longer
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
#include "k_linescan.cuh"

namespace gd {
namespace {

constexpr uint32_t kNaMaxTiles = 32768;  // look-back words: 1 GiB of text in 32 KiB tiles
constexpr int kNaMaxDevices = 64;
static_assert((uint64_t)kNaMaxTiles * LS_TILE == (1ull << 30), "the scratch covers 1 GiB of text");

// [0, kNaMaxTiles): look-back status per tile; [kNaMaxTiles]: tile counter
static __device__ __align__(256) uint64_t g_na_scratch[kNaMaxTiles + 1];

std::mutex g_na_mu;
uint64_t* g_na_ptr[kNaMaxDevices];  // scratch address per device, set once

// The S1 scan of the batch pipeline (the same tile routine), with the tile
// counter and look-back words in the static scratch and the line-start writes
// bounded by the caller's capacity (ERR_CAPACITY when the text has more lines
// than fit).
__global__ void __launch_bounds__(LS_THREADS) k_line_scan_static(const __grid_constant__ LineScanArgs a) {
  __shared__ LineScanSmem sm;
  line_scan_tile(sm, a);
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
  const uint64_t tiles64 = text_len ? (text_len + LS_TILE - 1) / LS_TILE : 1;
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
    LineScanArgs a;
    a.text = d_text;
    a.n = text_len;
    a.use_bulk = (reinterpret_cast<uintptr_t>(d_text) & 15u) == 0;
    a.line_start = d_line_start;
    a.cap = line_cap;
    a.status = scratch;
    a.counter = reinterpret_cast<uint32_t*>(scratch + kNaMaxTiles);
    a.ntiles = tiles;
    a.lines_out = d_result;
    a.err = d_result + 1;
    k_line_scan_static<<<tiles, LS_THREADS, 0, s>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_api_error(cudaGetErrorString(e));
    return GCN_ECUDA;
  }
  return GCN_OK;
}
