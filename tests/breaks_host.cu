// Host build of the CUDA path's early-exit finder (find_breaks, region_red.cuh) for tests:
// reads graphs from stdin (count, then per graph n and n lines "succ0 succ1 live", -1 = none)
// and prints per graph one line of brk values (-1 = none, -2 = a latch with a break).
#include <cstdio>
#include <vector>
#include "../paper_2107_07809_gb300/csrc/region_red.cuh"
using namespace gd;
int main() {
  int ng;
  if (scanf("%d", &ng) != 1) return 1;
  for (int g = 0; g < ng; ++g) {
    int n;
    if (scanf("%d", &n) != 1) return 1;
    std::vector<BlockRec> B(n);
    std::vector<uint8_t> cond(n), live(n);
    for (int i = 0; i < n; ++i) {
      int a, b, l;
      if (scanf("%d %d %d", &a, &b, &l) != 3) return 1;
      B[i] = BlockRec{0, 0, a < 0 ? kNone : (uint32_t)a, b < 0 ? kNone : (uint32_t)b};
      cond[i] = a >= 0 && b >= 0;
      live[i] = (uint8_t)l;
    }
    std::vector<uint32_t> brk(n), stk(n + 1);
    find_breaks(B.data(), cond.data(), live.data(), (uint32_t)n, brk.data(), stk.data());
    for (int i = 0; i < n; ++i)
      printf("%d ", brk[i] == kNone ? -1 : brk[i] == kBrkLatch ? -2 : (int)brk[i]);
    printf("\n");
  }
  return 0;
}
