// region_red.cuh — S12 structural analysis of one kernel ("Search for control
// structures", Fig. 3), usable from device code and from host code.
//
// The method: depth-first pre-order search from the entry region (successors
// in fall-through, taken order); at each region the templates are tried in
// the order self-loop, header+latch loop, if-else, if, linear; the first match
// is merged into a new region and the search starts again from the entry,
// until one region is left.  Template readings (the figures are missing):
//   linear(a,b):   succ(a)={b}, pred(b)={a}, |succ(b)|<=1
//   if(h,t,j):     succ(h)={t,j}, pred(t)={h}, succ(t)={j}; j joins when pred(j)={h,t}
//   if-else:       succ(h)={t,e}, pred(t)=pred(e)={h}, succ(t)=succ(e), |.|<=1;
//                  j joins when pred(j)={t,e}
//   loop:          a conditional exit of the region branches back to its head.
//
// Restarting the search from the entry after every merge costs O(n) per merge.
// The search is deterministic, so after a merge the new search repeats the
// previous one step for step until it pops a region whose template outcome or
// successor list may differ: a merged member, a predecessor of a member (its
// successors were redirected), a predecessor of those (it looks at its
// successors' successors), or a region within two predecessor steps of an
// external successor of the members (whose predecessor count changed).  The
// search is therefore resumed at the earliest such pop of the previous
// search: the stack is persistent (a log of pushes with links), every pop
// records the stack it started from, and the visits from that pop on are
// undone.  The merges, and so the region tree, are exactly those of the
// restarting search.
#pragma once
#include "gd_common.cuh"

#ifndef GD_HD
#define GD_HD __host__ __device__
#endif

namespace gd {

enum : uint32_t { R_BLOCK = 0, R_SEQ = 1, R_IF = 2, R_IFELSE = 3, R_LOOP = 4 };
// region record (12 words): kind, nch, ch[4], block, s0, s1, npred, head, tail
enum { RG_KIND = 0, RG_NCH = 1, RG_CH = 2, RG_BLOCK = 6, RG_S0 = 7, RG_S1 = 8, RG_NPRED = 9, RG_HEAD = 10, RG_TAIL = 11 };
constexpr int RGW = 12;

// work words the reducer needs for a kernel of n blocks
GD_HD inline size_t red_work_words(uint32_t n) { return 64ull * n + 128; }

// Early exits from counted loops (a project extension: the paper restores no loops).  A latch
// is a two-way block with exactly one successor at or before it (the header, the back edge) and
// the other after it (the exit).  A two-way block b that is not a latch breaks out of the loop
// that holds it -- the first latch l after b whose header is at or before b (for nested loops in
// program order, the innermost) -- when one of its successors is that loop's exit and the other
// stays in [header, l].  brk[b] = l for such a block; brk[l] = kBrkLatch for a latch with at least
// one; kNone otherwise.  The reduction leaves the edge b -> exit out.
constexpr uint32_t kBrkLatch = 0xFFFFFFFEu;
GD_HD inline uint32_t latch_header(const BlockRec* B, const uint8_t* cond, uint32_t l) {
  if (!cond[l]) return kNone;
  const uint32_t s0 = B[l].succ0, s1 = B[l].succ1;
  if ((s0 <= l) == (s1 <= l)) return kNone;
  return s0 <= l ? s0 : s1;
}
GD_HD inline uint32_t latch_exit(const BlockRec* B, uint32_t l, uint32_t h) {
  return B[l].succ0 == h ? B[l].succ1 : B[l].succ0;
}
// live[x]: block x is reached from the entry (an unreached block breaks out of nothing).
// The loop that holds b is found for every b in one backward sweep (linear time; a forward search
// from each block was quadratic on large CFGs): stk (n words of scratch) holds the latches after
// b that can still be the first one whose header is at or before b.  Entering b, latch b + 1
// joins and removes every latch whose header is at or after its own (b + 1 qualifies whenever
// they do, and comes first); then the latches whose header lies after b leave for good (no
// earlier block is inside them).  The top is the answer: the stack holds latches in increasing
// order from the top and headers in decreasing order.
GD_HD inline void find_breaks(const BlockRec* B, const uint8_t* cond, const uint8_t* live, uint32_t n, uint32_t* brk,
                              uint32_t* stk) {
  for (uint32_t x = 0; x < n; ++x) brk[x] = kNone;
  uint32_t sp = 0;
  for (uint32_t b = n; b-- > 0;) {
    if (b + 1 < n) {
      const uint32_t h = latch_header(B, cond, b + 1);
      if (h != kNone) {
        while (sp && latch_header(B, cond, stk[sp - 1]) >= h) --sp;
        stk[sp++] = b + 1;
      }
    }
    while (sp && latch_header(B, cond, stk[sp - 1]) > b) --sp;
    if (!sp || !live[b] || !cond[b] || latch_header(B, cond, b) != kNone) continue;
    const uint32_t l = stk[sp - 1], h = latch_header(B, cond, l);  // only the loop that holds b
    const uint32_t E = latch_exit(B, l, h), s0 = B[b].succ0, s1 = B[b].succ1;
    if ((s0 == E) != (s1 == E)) {
      const uint32_t x = s0 == E ? s1 : s0;
      if (x >= h && x <= l) brk[b] = l;
    }
  }
  for (uint32_t b = 0; b < n; ++b)
    if (brk[b] != kNone && brk[b] != kBrkLatch) brk[brk[b]] = kBrkLatch;
}

struct RedInc {
  // inputs
  uint32_t* rg;         // 3n region records (RGW words each)
  uint8_t* alive;       // 3n
  const BlockRec* B;    // the kernel's logical blocks (succ0/succ1 kernel-relative, kNone = none)
  const uint8_t* cond;  // block ends with a two-way branch (not counting a cut edge)
  const uint32_t* brk = nullptr;  // find_breaks() of the blocks (null: no early exits)
  uint32_t n;
  // state
  uint32_t nreg, entry, nalive;
  bool overflow;
  // search: persistent stack (push log), pop records, visit pop of each region
  uint32_t *vpop, *logv, *logb, *recT, *recL, *recV;
  uint32_t T, L, Q, cap_log;
  // predecessor lists: cells (src, next), head / tail per region, marks
  uint32_t *csrc, *cnext, *head, *tail, *mark;
  uint32_t ncell, cap_cell, epoch;
  // first pop of the previous search that a merge may have changed
  uint32_t qmin;

  GD_HD uint32_t* R(uint32_t r) { return rg + (size_t)r * RGW; }
  GD_HD uint32_t ns(uint32_t r) { return (R(r)[RG_S0] != kNone) + (R(r)[RG_S1] != kNone); }
  GD_HD bool has_succ(uint32_t r, uint32_t x) { return R(r)[RG_S0] == x || R(r)[RG_S1] == x; }
  GD_HD bool pred1(uint32_t x, uint32_t a) { return R(x)[RG_NPRED] == 1 && has_succ(a, x); }
  GD_HD bool pred2(uint32_t x, uint32_t a, uint32_t c) {
    return R(x)[RG_NPRED] == 2 && has_succ(a, x) && has_succ(c, x);
  }
  GD_HD bool latch_of(uint32_t body, uint32_t h) {
    uint32_t t = R(body)[RG_TAIL];
    if (t == kNone || !cond[t]) return false;
    uint32_t hb = R(h)[RG_HEAD];
    return B[t].succ0 == hb || B[t].succ1 == hb;
  }
  GD_HD bool cond_tail(uint32_t r) {
    uint32_t t = R(r)[RG_TAIL];
    return t != kNone && cond[t];
  }

  // ---- predecessor lists -----------------------------------------------------------
  GD_HD void add_cell(uint32_t r, uint32_t src) {
    if (ncell >= cap_cell) {
      overflow = true;
      return;
    }
    uint32_t c = ncell++;
    csrc[c] = src;
    cnext[c] = kNone;
    if (head[r] == kNone) head[r] = c;
    else cnext[tail[r]] = c;
    tail[r] = c;
  }
  GD_HD void lower(uint32_t r) {
    if (vpop[r] != kNone && vpop[r] < qmin) qmin = vpop[r];
  }
  // predecessors of r (stale cells are dropped on the way); f(src)
  template <class F>
  GD_HD void for_preds(uint32_t r, F f) {
    uint32_t prev = kNone, c = head[r];
    while (c != kNone) {
      uint32_t nx = cnext[c], s = csrc[c];
      if (alive[s] && has_succ(s, r)) {
        f(s);
        prev = c;
      } else {  // unlink
        if (prev == kNone) head[r] = nx;
        else cnext[prev] = nx;
        if (tail[r] == c) tail[r] = prev;
      }
      c = nx;
    }
  }

  // ---- merge ------------------------------------------------------------------------
  GD_HD void merge(uint32_t kind, const uint32_t* ch, int nch, uint32_t ns0, uint32_t ns1) {
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
    for (int q = 0; q < 2; ++q) {
      uint32_t y = q == 0 ? ns0 : ns1;
      if (y == kNone) continue;
      uint32_t z = inS(y) ? id : y;
      if (c == 1 && s[0] == z) continue;
      s[c++] = z;
    }
    X[RG_S0] = s[0];
    X[RG_S1] = s[1];
    head[id] = tail[id] = kNone;
    vpop[id] = kNone;
    for (int q = 0; q < nch; ++q) lower(ch[q]);
    // external predecessors: redirect their edges into the members to the new
    // region, count them once, note them and their predecessors for the resume
    ++epoch;
    uint32_t np = 0;
    for (int q = 0; q < nch; ++q) {
      for_preds(ch[q], [&](uint32_t p) {
        if (inS(p) || mark[p] == epoch) return;
        mark[p] = epoch;
        ++np;
        lower(p);
        uint32_t* P = R(p);
        uint32_t a = P[RG_S0] != kNone && inS(P[RG_S0]) ? id : P[RG_S0];
        uint32_t bb = P[RG_S1] != kNone && inS(P[RG_S1]) ? id : P[RG_S1];
        if (bb == a) bb = kNone;
        if (a == kNone) { a = bb; bb = kNone; }
        P[RG_S0] = a;
        P[RG_S1] = bb;
        for_preds(p, [&](uint32_t u) { lower(u); });
      });
    }
    // the members' lists become the new region's list (stale cells drop later)
    for (int q = 0; q < nch; ++q) {
      uint32_t m = ch[q];
      if (head[m] == kNone) continue;
      if (head[id] == kNone) head[id] = head[m];
      else cnext[tail[id]] = head[m];
      tail[id] = tail[m];
      head[m] = tail[m] = kNone;
    }
    const bool self = s[0] == id || s[1] == id;
    if (self) add_cell(id, id);
    // new predecessor counts of the external successors (before members die)
    for (int q = 0; q < c; ++q) {
      uint32_t y = s[q];
      if (y == id) continue;
      uint32_t from_members = 0;
      for (int m = 0; m < nch; ++m) from_members += has_succ(ch[m], y);
      R(y)[RG_NPRED] = R(y)[RG_NPRED] - from_members + 1;
      add_cell(y, id);
    }
    for (int q = 0; q < nch; ++q) alive[ch[q]] = 0;
    alive[id] = 1;
    X[RG_NPRED] = np + (self ? 1u : 0u);
    nalive = nalive + 1 - (uint32_t)nch;
    // regions within two predecessor steps of the external successors
    for (int q = 0; q < c; ++q) {
      if (s[q] == id) continue;
      for_preds(s[q], [&](uint32_t u) {
        lower(u);
        for_preds(u, [&](uint32_t w) { lower(w); });
      });
    }
    if (inS(entry)) {
      entry = id;
      qmin = 0;
    }
  }

  GD_HD bool try_at(uint32_t h) {
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

  // ---- search -------------------------------------------------------------------
  GD_HD void push(uint32_t v) {
    if (L >= cap_log) {
      overflow = true;
      return;
    }
    logv[L] = v;
    logb[L] = T;
    T = L++;
  }

  // Set up the region graph from the blocks (alive[] marks the blocks reached
  // from the entry) and carve the work area (red_work_words(n) words).
  GD_HD void init(uint32_t* work) {
    const uint32_t nr = 3 * n;
    cap_log = 6 * n + 8;
    uint32_t* w = work;
    vpop = w; w += nr;
    logv = w; w += cap_log;
    logb = w; w += cap_log;
    recT = w; w += cap_log;
    recL = w; w += cap_log;
    recV = w; w += cap_log;
    cap_cell = 8 * n + 8;
    csrc = w; w += cap_cell;
    cnext = w; w += cap_cell;
    head = w; w += nr;
    tail = w; w += nr;
    mark = w; w += nr;  // total 17n + 6 (6n + 8) + ... <= 64n + 128
    ncell = 0;
    epoch = 0;
    overflow = false;
    nreg = n;
    entry = 0;
    nalive = 0;
    for (uint32_t x = 0; x < nr; ++x) {
      vpop[x] = kNone;
      head[x] = tail[x] = kNone;
      mark[x] = 0;
    }
    for (uint32_t x = 0; x < n; ++x) {
      uint32_t* X = R(x);
      X[RG_KIND] = R_BLOCK;
      X[RG_NCH] = 0;
      X[RG_BLOCK] = x;
      X[RG_HEAD] = x;
      X[RG_TAIL] = x;
      X[RG_NPRED] = 0;
      X[RG_S0] = X[RG_S1] = kNone;
      if (!alive[x]) continue;
      ++nalive;
      X[RG_S0] = B[x].succ0;
      X[RG_S1] = B[x].succ1;
      if (brk && brk[x] != kNone && brk[x] != kBrkLatch) {  // leave the exit edge out
        const uint32_t l = brk[x], E = latch_exit(B, l, latch_header(B, cond, l));
        if (X[RG_S0] == E) X[RG_S0] = kNone;
        else if (X[RG_S1] == E) X[RG_S1] = kNone;
      }
      if (X[RG_S0] == kNone) {
        X[RG_S0] = X[RG_S1];
        X[RG_S1] = kNone;
      }
    }
    for (uint32_t x = 0; x < n; ++x) {
      if (!alive[x]) continue;
      uint32_t* X = R(x);
      for (int q = 0; q < 2; ++q) {
        uint32_t y = X[RG_S0 + q];
        if (y == kNone) continue;
        R(y)[RG_NPRED]++;
        add_cell(y, x);
      }
    }
    T = kNone;
    L = 0;
    Q = 0;
    push(entry);
  }

  // Every break block (brk[b] a latch) must sit inside the do-while of its own loop: the
  // nearest loop region above it in the tree has that latch as its tail.  Uses mark[] (free
  // once the reduction is over) for the parents.
  GD_HD bool breaks_in_place() {
    uint32_t* parent = mark;
    for (uint32_t r = 0; r < nreg; ++r) parent[r] = kNone;
    for (uint32_t r = n; r < nreg; ++r) {
      const uint32_t* X = R(r);
      for (uint32_t q = 0; q < X[RG_NCH]; ++q) parent[X[RG_CH + q]] = r;
    }
    for (uint32_t b = 0; brk && b < n; ++b) {
      if (brk[b] == kNone || brk[b] == kBrkLatch) continue;
      uint32_t r = parent[b];
      while (r != kNone && R(r)[RG_KIND] != R_LOOP) r = parent[r];
      if (r == kNone) return false;
      const uint32_t* X = R(r);
      if (R(X[RG_CH + X[RG_NCH] - 1])[RG_TAIL] != brk[b]) return false;
    }
    return true;
  }

  // Reduce until one region is left.  Returns the root region, or kNone when
  // the graph does not reduce (or a work array overflowed: *capacity set).
  GD_HD uint32_t run(bool* capacity) {
    *capacity = false;
    while (nalive > 1) {
      bool merged = false;
      while (T != kNone && !merged) {
        const uint32_t q = Q;
        if (q >= cap_log) {
          overflow = true;
          break;
        }
        const uint32_t v = logv[T];
        recT[q] = T;
        recL[q] = L;
        recV[q] = v;
        T = logb[T];
        Q = q + 1;
        if (vpop[v] != kNone) continue;
        vpop[v] = q;
        if (nreg >= 3 * n) {
          overflow = true;
          break;
        }
        qmin = q;
        if (try_at(v)) {
          merged = true;
          break;
        }
        uint32_t* X = R(v);
        if (X[RG_S1] != kNone && vpop[X[RG_S1]] == kNone) push(X[RG_S1]);
        if (X[RG_S0] != kNone && vpop[X[RG_S0]] == kNone) push(X[RG_S0]);
      }
      if (overflow) {
        *capacity = true;
        return kNone;
      }
      if (!merged) return kNone;  // does not reduce: unstructured
      if (nalive <= 1) break;
      // resume at pop qmin: undo the visits from there, restore its stack
      for (uint32_t q = qmin; q < Q; ++q)
        if (vpop[recV[q]] == q) vpop[recV[q]] = kNone;
      if (qmin == 0) {
        T = kNone;
        L = 0;
        Q = 0;
        push(entry);
      } else {
        T = recT[qmin];
        L = recL[qmin];
        Q = qmin;
      }
    }
    return entry;
  }
};

}  // namespace gd
