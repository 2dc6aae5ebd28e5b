// Host build of the CUDA path's region reducer (S12) for tests: reads abstract
// graphs from stdin (count, then per graph n and n lines "succ0 succ1", -1 =
// none; entry 0; every block takes part, as in the oracle's abstract-graph
// entry point) and prints per graph "G <index> <root|-1 unstructured|-2 full>"
// followed by the merges "|<new id> <members...>".
#include <cstdio>
#include <vector>
#include "../paper_2107_07809_gb300/csrc/region_red.cuh"
using namespace gd;
int main() {
  int ng;
  if (scanf("%d", &ng) != 1) return 1;
  for (int g = 0; g < ng; ++g) {
    int n;
    scanf("%d", &n);
    std::vector<BlockRec> B(n);
    std::vector<uint8_t> cond(n);
    for (int i = 0; i < n; ++i) {
      int a, b;
      scanf("%d %d", &a, &b);
      uint32_t s0 = a < 0 ? kNone : (uint32_t)a, s1 = b < 0 ? kNone : (uint32_t)b;
      if (s1 == s0) s1 = kNone;
      if (s0 == kNone) { s0 = s1; s1 = kNone; }
      B[i] = BlockRec{0, 0, s0, s1};
      cond[i] = s0 != kNone && s1 != kNone;
    }
    std::vector<uint32_t> rg(12 * 3 * n + 24);
    std::vector<uint8_t> alive(3 * n + 2, 0);
    std::vector<uint32_t> work(red_work_words(n));
    // every block takes part, as in the oracle's abstract-graph entry point
    for (int i = 0; i < n; ++i) alive[i] = 1;
    RedInc rd;
    rd.rg = rg.data(); rd.alive = alive.data(); rd.B = B.data(); rd.cond = cond.data(); rd.n = n;
    rd.init(work.data());
    bool capf = false;
    uint32_t root = rd.run(&capf);
    printf("G %d %d", g, capf ? -2 : (root == kNone ? -1 : (int)root));
    for (uint32_t r = n; r < rd.nreg; ++r) {
      uint32_t* X = rd.R(r);
      printf(" |%u", r);
      for (uint32_t q = 0; q < X[RG_NCH]; ++q) printf(" %u", X[RG_CH + q]);
    }
    printf("\n");
  }
  return 0;
}
