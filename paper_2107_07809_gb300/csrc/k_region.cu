// k_region.cu — S12: region graph and structural analysis ("Search for
// control structures", Fig. 3).  One thread per kernel marks the blocks
// reached from the entry, finds the early exits of loops (a project
// extension), and runs the reduction of region_red.cuh (the restarting
// pre-order search, resumed incrementally after each merge).
#include "gd_kernels.h"
#include "region_red.cuh"

namespace gd {

__global__ void k_regions(const __grid_constant__ Batch b, uint32_t* __restrict__ work_all,
                          uint32_t* __restrict__ stk_all, uint8_t* __restrict__ alive_all,
                          uint8_t* __restrict__ cond_all) {
  uint32_t k = walk_kernel();
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  K.root = kNone;
  if (K.bad || !K.n_lblock) return;
  const uint32_t n = K.n_lblock, base = K.first_lblock;
  RedInc rd;
  rd.rg = b.rg + (size_t)kRegionsPerBlock * base * RGW;
  rd.alive = alive_all + kRegionsPerBlock * (size_t)base;
  rd.B = b.lblocks + base;
  uint8_t* cnd = cond_all + base;
  rd.cond = cnd;
  rd.n = n;
  for (uint32_t x = 0; x < n; ++x)
    cnd[x] = b.ctl[K.first_instr + b.lterm[base + x]] == C_CBR && rd.B[x].succ1 != kNone;
  // blocks reached from the entry
  for (uint32_t x = 0; x < kRegionsPerBlock * n; ++x) rd.alive[x] = 0;
  uint32_t* stk = stk_all + kStackPerBlock * (size_t)base;
  uint32_t sp = 0;
  stk[sp++] = 0;
  rd.alive[0] = 1;
  while (sp) {
    uint32_t x = stk[--sp];
    for (int q = 0; q < 2; ++q) {
      uint32_t s = q == 0 ? rd.B[x].succ0 : rd.B[x].succ1;
      if (s != kNone && !rd.alive[s]) {
        rd.alive[s] = 1;
        stk[sp++] = s;
      }
    }
  }
  // early exits from loops: find them on the blocks as they are, then take the break blocks'
  // exit edges out of the graph (they print as `break`)
  uint32_t* brk = b.brk + base;
  find_breaks(rd.B, cnd, rd.alive, n, brk, stk);  // the search stack is free again: its scratch
  for (uint32_t x = 0; x < n; ++x)
    if (brk[x] != kNone && brk[x] != kBrkLatch) cnd[x] = 0;
  rd.brk = brk;
  rd.init(work_all + 128 * (size_t)k + 64 * (size_t)base);  // red_work_words of the kernels before
  bool capacity = false;
  uint32_t root = rd.run(&capacity);
  if (capacity) atomicOr(b.err, ERR_CAPACITY);
  if (root != kNone && !rd.breaks_in_place()) root = kNone;  // a break that would leave another loop
  K.root = root;
}

void launch_regions(Batch& b, uint32_t* work, uint32_t* stk, uint8_t* alive, uint8_t* cond, cudaStream_t s) {
  if (!b.K) return;
  k_regions<<<walk_blocks(b.K), walk_threads(b.K), 0, s>>>(b, work, stk, alive, cond);
  ++launch_counter();
}

}  // namespace gd
