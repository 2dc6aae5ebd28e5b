// k_region.cu — S12: region graph and structural analysis ("Search for
// control structures", Fig. 3).
//
// One thread per kernel runs the reduction: depth-first pre-order from the
// entry region (successors in fall-through, taken order), templates tried in
// the order self-loop, header+latch loop, if-else, if, linear; the first match
// is merged into a new region and the search restarts, until one region is
// left.  Template readings (the figures are missing from the paper):
//   linear(a,b):   succ(a)={b}, pred(b)={a}, |succ(b)|<=1
//   if(h,t,j):     succ(h)={t,j}, pred(t)={h}, succ(t)={j}; j joins when pred(j)={h,t}
//   if-else:       succ(h)={t,e}, pred(t)=pred(e)={h}, succ(t)=succ(e), |.|<=1;
//                  j joins when pred(j)={t,e}
//   loop:          a conditional exit of the region branches back to its head.
// Regions keep their successor lists and the number of distinct predecessors;
// "pred(x) = {a}" is "npred(x) = 1 and x is a successor of a".
#include "gd_kernels.h"

namespace gd {

enum : uint32_t { R_BLOCK = 0, R_SEQ = 1, R_IF = 2, R_IFELSE = 3, R_LOOP = 4 };
// region record (12 words): kind, nch, ch[4], block, s0, s1, npred, head, tail
enum { RG_KIND = 0, RG_NCH = 1, RG_CH = 2, RG_BLOCK = 6, RG_S0 = 7, RG_S1 = 8, RG_NPRED = 9, RG_HEAD = 10, RG_TAIL = 11 };
constexpr int RGW = 12;

struct Red {
  uint32_t* rg;        // 3n regions of this kernel
  uint32_t* seen;      // epoch per region
  uint32_t* stk;
  uint8_t* alive;
  const BlockRec* B;   // logical blocks of the kernel
  const uint8_t* cond; // block ends with a two-way branch
  uint32_t n, nreg, entry, epoch;
  __device__ uint32_t* R(uint32_t r) { return rg + (size_t)r * RGW; }
  __device__ uint32_t ns(uint32_t r) { return (R(r)[RG_S0] != kNone) + (R(r)[RG_S1] != kNone); }
  __device__ bool has_succ(uint32_t r, uint32_t x) { return R(r)[RG_S0] == x || R(r)[RG_S1] == x; }
  __device__ bool pred1(uint32_t x, uint32_t a) { return R(x)[RG_NPRED] == 1 && has_succ(a, x); }
  __device__ bool pred2(uint32_t x, uint32_t a, uint32_t c) {
    return R(x)[RG_NPRED] == 2 && has_succ(a, x) && has_succ(c, x);
  }
  // tail block has a two-way branch back to the head block of region h
  __device__ bool latch_of(uint32_t body, uint32_t h) {
    uint32_t t = R(body)[RG_TAIL];
    if (t == kNone || !cond[t]) return false;
    uint32_t hb = R(h)[RG_HEAD];
    return B[t].succ0 == hb || B[t].succ1 == hb;
  }
  __device__ bool cond_tail(uint32_t r) {
    uint32_t t = R(r)[RG_TAIL];
    return t != kNone && cond[t];
  }

  __device__ void merge(uint32_t kind, const uint32_t* ch, int nch, uint32_t ns0, uint32_t ns1) {
    uint32_t id = nreg++;
    uint32_t* X = R(id);
    X[RG_KIND] = kind;
    X[RG_NCH] = (uint32_t)nch;
    for (int q = 0; q < 4; ++q) X[RG_CH + q] = q < nch ? ch[q] : kNone;
    X[RG_BLOCK] = kNone;
    X[RG_HEAD] = R(ch[0])[RG_HEAD];
    switch (kind) {
      case R_SEQ: X[RG_TAIL] = R(ch[1])[RG_TAIL]; break;
      case R_IF: X[RG_TAIL] = nch == 3 ? R(ch[2])[RG_TAIL] : kNone; break;
      case R_IFELSE: X[RG_TAIL] = nch == 4 ? R(ch[3])[RG_TAIL] : kNone; break;
      default: X[RG_TAIL] = R(ch[nch - 1])[RG_TAIL]; break;
    }
    auto inS = [&](uint32_t x) {
      for (int q = 0; q < nch; ++q)
        if (ch[q] == x) return true;
      return false;
    };
    // successors of the new region, members mapped to it, deduplicated in order
    uint32_t s[2] = {kNone, kNone};
    int c = 0;
    for (uint32_t y : {ns0, ns1}) {
      if (y == kNone) continue;
      uint32_t z = inS(y) ? id : y;
      if (c == 1 && s[0] == z) continue;
      s[c++] = z;
    }
    X[RG_S0] = s[0];
    X[RG_S1] = s[1];
    // new predecessor counts of its successors (before members die)
    for (int q = 0; q < c; ++q) {
      uint32_t y = s[q];
      if (y == id) continue;
      uint32_t from_members = 0;
      for (int m = 0; m < nch; ++m) from_members += has_succ(ch[m], y);
      R(y)[RG_NPRED] = R(y)[RG_NPRED] - from_members + 1;
    }
    for (int q = 0; q < nch; ++q) alive[ch[q]] = 0;
    alive[id] = 1;
    // regions outside that pointed into the members now point to the new region
    uint32_t np = 0;
    for (uint32_t x = 0; x < id; ++x) {
      if (!alive[x]) continue;
      uint32_t* P = R(x);
      bool hit = (P[RG_S0] != kNone && inS(P[RG_S0])) || (P[RG_S1] != kNone && inS(P[RG_S1]));
      if (!hit) continue;
      ++np;
      uint32_t a = P[RG_S0] != kNone && inS(P[RG_S0]) ? id : P[RG_S0];
      uint32_t bb = P[RG_S1] != kNone && inS(P[RG_S1]) ? id : P[RG_S1];
      if (bb == a) bb = kNone;
      if (a == kNone) { a = bb; bb = kNone; }
      P[RG_S0] = a;
      P[RG_S1] = bb;
    }
    X[RG_NPRED] = np + ((s[0] == id || s[1] == id) ? 1u : 0u);
    if (inS(entry)) entry = id;
  }

  __device__ bool try_at(uint32_t h) {
    uint32_t* H = R(h);
    uint32_t nsh = ns(h), s0 = H[RG_S0], s1 = H[RG_S1];
    // loop: self loop
    if (nsh == 2 && (s0 == h || s1 == h) && latch_of(h, h)) {
      uint32_t x = s0 == h ? s1 : s0;
      uint32_t ch[1] = {h};
      merge(R_LOOP, ch, 1, x, kNone);
      return true;
    }
    // loop: header + latch
    if (nsh == 1 && s0 != h) {
      uint32_t bb = s0;
      uint32_t* Bb = R(bb);
      if (pred1(bb, h) && ns(bb) == 2 && (Bb[RG_S0] == h || Bb[RG_S1] == h) && latch_of(bb, h)) {
        uint32_t x = Bb[RG_S0] == h ? Bb[RG_S1] : Bb[RG_S0];
        uint32_t ch[2] = {h, bb};
        merge(R_LOOP, ch, 2, x, kNone);
        return true;
      }
    }
    if (nsh == 2 && cond_tail(h)) {
      uint32_t t = s0, e = s1;
      if (t != h && e != h && t != e && pred1(t, h) && pred1(e, h)) {
        uint32_t nt = ns(t), ne = ns(e);
        bool same = nt == ne && nt <= 1 && (nt == 0 || R(t)[RG_S0] == R(e)[RG_S0]);
        if (same) {
          if (nt == 1) {
            uint32_t j = R(t)[RG_S0];
            if (j != h && j != t && j != e) {
              if (pred2(j, t, e)) {
                uint32_t ch[4] = {h, t, e, j};
                uint32_t* J = R(j);
                merge(R_IFELSE, ch, 4, J[RG_S0], J[RG_S1]);
              } else {
                uint32_t ch[3] = {h, t, e};
                merge(R_IFELSE, ch, 3, j, kNone);
              }
              return true;
            }
          } else {
            uint32_t ch[3] = {h, t, e};
            merge(R_IFELSE, ch, 3, kNone, kNone);
            return true;
          }
        }
      }
      for (int q = 0; q < 2; ++q) {
        uint32_t tt = q == 0 ? s0 : s1, j = q == 0 ? s1 : s0;
        if (tt == h || j == h) continue;
        if (!pred1(tt, h)) continue;
        if (ns(tt) != 1 || R(tt)[RG_S0] != j) continue;
        if (pred2(j, h, tt)) {
          uint32_t ch[3] = {h, tt, j};
          uint32_t* J = R(j);
          merge(R_IF, ch, 3, J[RG_S0], J[RG_S1]);
        } else {
          uint32_t ch[2] = {h, tt};
          merge(R_IF, ch, 2, j, kNone);
        }
        return true;
      }
    }
    // linear
    if (nsh == 1 && s0 != h) {
      uint32_t bb = s0;
      if (pred1(bb, h) && ns(bb) <= 1) {
        uint32_t ch[2] = {h, bb};
        uint32_t* Bb = R(bb);
        merge(R_SEQ, ch, 2, Bb[RG_S0], Bb[RG_S1]);
        return true;
      }
    }
    return false;
  }
};

__global__ void k_regions(const __grid_constant__ Batch b, uint32_t* __restrict__ seen_all, uint32_t* __restrict__ stk_all,
                          uint8_t* __restrict__ alive_all, uint8_t* __restrict__ cond_all) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  K.root = kNone;
  if (K.bad || !K.n_lblock) return;
  uint32_t n = K.n_lblock, base = K.first_lblock;
  Red rd;
  rd.rg = b.rg + (size_t)kRegionsPerBlock * base * RGW;
  rd.seen = seen_all + kRegionsPerBlock * (size_t)base;
  rd.stk = stk_all + kStackPerBlock * (size_t)base;
  rd.alive = alive_all + kRegionsPerBlock * (size_t)base;
  rd.B = b.lblocks + base;
  rd.cond = cond_all + base;
  rd.n = n;
  rd.nreg = n;
  rd.entry = 0;
  rd.epoch = 0;
  uint8_t* cnd = cond_all + base;
  // reachable blocks from the entry (the stack doubles as the DFS stack)
  for (uint32_t x = 0; x < kRegionsPerBlock * n; ++x) {
    rd.alive[x] = 0;
    rd.seen[x] = 0;
  }
  uint32_t sp = 0;
  rd.stk[sp++] = 0;
  rd.alive[0] = 1;
  while (sp) {
    uint32_t x = rd.stk[--sp];
    for (uint32_t s : {rd.B[x].succ0, rd.B[x].succ1})
      if (s != kNone && !rd.alive[s]) {
        rd.alive[s] = 1;
        rd.stk[sp++] = s;
      }
  }
  for (uint32_t x = 0; x < n; ++x) {
    uint32_t* X = rd.R(x);
    X[RG_KIND] = R_BLOCK;
    X[RG_NCH] = 0;
    X[RG_BLOCK] = x;
    X[RG_HEAD] = x;
    X[RG_TAIL] = x;
    X[RG_NPRED] = 0;
    X[RG_S0] = X[RG_S1] = kNone;
    uint32_t term = b.lterm[base + x];
    cnd[x] = b.ctl[K.first_instr + term] == C_CBR && rd.B[x].succ1 != kNone;
    if (!rd.alive[x]) continue;
    X[RG_S0] = rd.B[x].succ0;
    X[RG_S1] = rd.B[x].succ1;
    if (X[RG_S0] == kNone) { X[RG_S0] = X[RG_S1]; X[RG_S1] = kNone; }
  }
  for (uint32_t x = 0; x < n; ++x) {
    if (!rd.alive[x]) continue;
    uint32_t* X = rd.R(x);
    if (X[RG_S0] != kNone) rd.R(X[RG_S0])[RG_NPRED]++;
    if (X[RG_S1] != kNone) rd.R(X[RG_S1])[RG_NPRED]++;
  }
  uint32_t nalive = 0;
  for (uint32_t x = 0; x < n; ++x) nalive += rd.alive[x];
  while (nalive > 1) {
    if (rd.nreg >= kRegionsPerBlock * n) { atomicOr(b.err, ERR_CAPACITY); return; }  // cannot happen: < 3n
    ++rd.epoch;
    sp = 0;
    rd.stk[sp++] = rd.entry;
    bool merged = false;
    while (sp && !merged) {
      uint32_t x = rd.stk[--sp];
      if (rd.seen[x] == rd.epoch) continue;
      rd.seen[x] = rd.epoch;
      uint32_t before = rd.nreg;
      if (rd.try_at(x)) {
        merged = true;
        nalive = nalive + 1 - rd.R(before)[RG_NCH];
        break;
      }
      uint32_t* X = rd.R(x);
      if (X[RG_S1] != kNone && rd.seen[X[RG_S1]] != rd.epoch) {
        if (sp >= kStackPerBlock * n) { atomicOr(b.err, ERR_CAPACITY); return; }
        rd.stk[sp++] = X[RG_S1];
      }
      if (X[RG_S0] != kNone && rd.seen[X[RG_S0]] != rd.epoch) {
        if (sp >= kStackPerBlock * n) { atomicOr(b.err, ERR_CAPACITY); return; }
        rd.stk[sp++] = X[RG_S0];
      }
    }
    if (!merged) return;  // does not reduce: unstructured
  }
  K.root = rd.entry;
}

void launch_regions(Batch& b, uint32_t* seen, uint32_t* stk, uint8_t* alive, uint8_t* cond, cudaStream_t s) {
  if (!b.K) return;
  k_regions<<<(b.K + 63) / 64, 64, 0, s>>>(b, seen, stk, alive, cond);
  ++launch_counter();
}

}  // namespace gd
