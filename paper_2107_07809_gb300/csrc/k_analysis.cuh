// k_analysis.cuh — device functions shared by the analysis (S9-S11) and
// emission (S13) kernels of the CUDA path: value forwarding, system-value and
// argument classification, memory-access matching, node types.
#pragma once
#include "gd_kernels.h"

namespace gd {

// kernel view: node / argument arrays of one kernel
// Inlining of the recursive pattern matchers: left to the compiler by
// default; a translation unit that calls them from many places (the printer)
// defines GD_MATCH_INLINE as __noinline__ before including this header.
#ifndef GD_MATCH_INLINE
#define GD_MATCH_INLINE
#endif

struct KView {
  const KHdr* K;
  const Node* N;      // b.nodes + 4 * first_instr
  const ArgRec* A;    // b.args + k * kMaxArgs
  uint32_t k;
  // caches filled by k_node_cache (null while it runs): class of each node,
  // forwarded sources of each node, memory match of each load/store
  const uint8_t* cc;
  const uint8_t* ck;
  const uint32_t* sf;
  const uint32_t* marg;
  const uint32_t* midx;
  __device__ const Node& node(uint32_t id) const { return N[id]; }
};

// a kernel view with the caches of the batch
__device__ __forceinline__ KView make_view(const Batch& b, const KHdr& K, uint32_t k) {
  const size_t nb = 4 * (size_t)K.first_instr;
  KView v{&K, b.nodes + nb, b.args + (size_t)k * kMaxArgs, k, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (b.ncls) {
    v.cc = b.ncls + nb;
    v.ck = b.nclsk + nb;
    v.sf = b.nsrcf + 3 * nb;
    v.marg = b.mem_arg + K.first_instr;
    v.midx = b.mem_idx + K.first_instr;
  }
  return v;
}

__device__ __forceinline__ bool is_copy_node(const Node& n) {
  return n.kind == N_OP && (n.op == O_V_MOV_B32 || n.op == O_S_MOV_B32 || n.op == O_BUFFER_STORE_DWORD ||
                            n.op == O_BUFFER_LOAD_DWORD);
}

// a copy is the value it copies; the halves of a split pair are its sources;
// a pair of the low and high part of one 64-bit value is that value
// (a function of the kernel's node array alone, so that a caller's view need not be kept in local
// memory for the call)
static __device__ GD_MATCH_INLINE uint32_t fwd_n(const Node* N, uint32_t r, int depth) {
  for (int step = 0; step < 512 && depth < 64; ++step) {
    if (r == kTop) return kUndef;
    if (!r_node(r)) return r;
    const Node& n = N[rid(r)];
    uint32_t part = rpart(r);
    if (is_copy_node(n) && part == PART_ENTIRE) {
      r = n.src[0];
      continue;
    }
    if (n.kind == N_PAIR) {
      if (part == PART_LO) { r = n.src[0]; continue; }
      if (part == PART_HI) { r = n.src[1]; continue; }
      uint32_t lo = fwd_n(N, n.src[0], depth + 1), hi = fwd_n(N, n.src[1], depth + 1);
      if ((r_node(lo) || r_leaf(lo)) && rpart(lo) == PART_LO && hi == ((lo & ~3u) | PART_HI)) return lo & ~3u;
      return r;
    }
    return r;
  }
  return r;
}
__device__ __forceinline__ uint32_t fwd_d(const KView& v, uint32_t r, int depth) { return fwd_n(v.N, r, depth); }
__device__ __forceinline__ uint32_t fwd(const KView& v, uint32_t r) { return fwd_d(v, r, 0); }
// forwarded source q of node n (n must live in v.N)
__device__ __forceinline__ uint32_t nsrc(const KView& v, const Node& n, int q) {
  return v.sf ? v.sf[3 * (size_t)(&n - v.N) + q] : fwd_d(v, n.src[q], 0);
}

// classes of values
enum : uint8_t { K_NONE = 0, K_LID, K_GRP, K_KARG, K_UNDEF, K_GOFS64, K_GOFSLO, K_MULGRP, K_GIDNO, K_GID, K_ARGPTR,
                 K_ARG32, K_ARG64, K_CONST32, K_CONST64,
                 K_DISP,    // the dispatch packet pointer s[0:1]
                 K_DISP0,   // the packet's first dword (header, setup): an intermediate like K_MULGRP
                 K_GSIZE,   // get_global_size(d): the dword at 0xc + 4d
                 K_NGRP,    // get_num_groups(d): global size >> log2(work-group size)
                 K_WDIM,    // get_work_dim(): field 0x20010 (offset 16, width 2) of the first dword
                 K_LPTR };  // the LDS address of a __local pointer argument (the low dword of its slot)
struct Cls {
  uint8_t c, k;
};
__device__ __forceinline__ bool leaf_like(uint8_t c) { return c != K_NONE && c != K_MULGRP && c != K_DISP0; }
__device__ __forceinline__ bool ty64(uint8_t t) { return t == TY_LONG || t == TY_ULONG || t == TY_DOUBLE || t == TY_TOP64; }
__device__ __forceinline__ int ilog2_exact(uint32_t x) {
  return (x && !(x & (x - 1)) && x < (1u << 31)) ? (31 - __clz(x)) : -1;
}

// A class other than none is derived from operands at most three levels down
// (get_global_id <- group id * size + local id <- group id * size <- group id;
// a settings load <- the settings pointer; get_num_groups / get_work_dim <- a
// dispatch packet load <- the packet pointer), and an operand without a class
// can only keep a pattern from matching.  So the recursion stops below
// kClassDepth levels without changing any class, which bounds the work on
// long chains of additions.
constexpr int kClassDepth = 4;
static __device__ Cls classify_d(const KView& v, uint32_t r, int d);

// the operations whose class depends on their operands (every other operation has none)
__device__ __forceinline__ bool class_op(uint16_t op) {
  switch (op) {
    case O_S_LOAD_DWORD: case O_S_LOAD_DWORDX2: case O_S_LOAD_DWORDX4: case O_S_MUL_I32: case O_S_LSHL_B32:
    case O_S_LSHR_B32: case O_S_BFE_U32: case O_V_ADD_U32: case O_V_MAD_U32_U24: return true;
  }
  return false;
}
__device__ __forceinline__ Cls leaf_class(uint32_t r) {
  const uint32_t id = rid(r) & 0x0FFFFFFFu;
  const uint32_t kind = id >> 8, k = id & 0xFF;
  if (rpart(r) != PART_ENTIRE) return Cls{K_NONE, 0};
  if (kind == LEAF_LID) return Cls{K_LID, (uint8_t)k};
  if (kind == LEAF_GRP) return Cls{K_GRP, (uint8_t)k};
  if (kind == LEAF_KARG) return Cls{K_KARG, 0};
  if (kind == LEAF_DISP) return Cls{K_DISP, 0};
  return Cls{K_NONE, 0};
}
// classify_d(v, r, d), answered in line wherever no operand needs a look (undefined values,
// cached classes, leaves, constants, operations without a class): only a node whose class
// depends on its operands costs a call.  Used at the top of a classification; the recursion
// itself stays in classify_d (screening its operands in line there made the class pass slower).
__device__ __forceinline__ Cls classify_q(const KView& v, uint32_t r, int d) {
  if (r == kUndef || r == kTop) return Cls{K_UNDEF, 0};
  if (v.cc && r_node(r) && rpart(r) == PART_ENTIRE) return Cls{v.cc[rid(r)], v.ck[rid(r)]};
  if (d > kClassDepth && r_node(r)) return Cls{K_NONE, 0};
  if (r_leaf(r)) return leaf_class(r);
  if (!r_node(r)) return Cls{K_NONE, 0};
  const Node& n = v.node(rid(r));
  if (n.kind == N_CONST) return Cls{K_CONST32, 0};
  if (n.kind == N_OP ? !class_op(n.op) : (n.kind != N_PAIR && n.kind != N_SLOAD64B)) return Cls{K_NONE, 0};
  return classify_d(v, r, d);
}

static __device__ GD_MATCH_INLINE Cls settings_load(const KView& v, const Node& n, uint32_t part, bool wide, int d) {
  Cls none{K_NONE, 0};
  Cls base = classify_d(v, nsrc(v, n, 0), d + 1);
  if (base.c == K_DISP) {  // dispatch packet: header/setup dword at 0x0, global sizes at 0xc/0x10/0x14
    if (wide || part != PART_ENTIRE) return none;
    if (n.cval == 0) return Cls{K_DISP0, 0};
    if (n.cval == 0xc || n.cval == 0x10 || n.cval == 0x14) return Cls{K_GSIZE, (uint8_t)((n.cval - 0xc) / 4)};
    return none;
  }
  if (base.c != K_KARG || (n.cval & 7u)) return none;
  uint32_t slot = n.cval / 8;
  if (slot >= v.K->nargs) return none;
  const ArgRec& a = v.A[slot];
  if (wide) {
    if (a.hidden && a.gofs) {
      if (part == PART_ENTIRE) return Cls{K_GOFS64, (uint8_t)(a.gofs - 1)};
      if (part == PART_LO) return Cls{K_GOFSLO, (uint8_t)(a.gofs - 1)};
      return none;
    }
    if (a.hidden || part != PART_ENTIRE) return none;
    if (a.pointer) return Cls{K_ARGPTR, (uint8_t)slot};
    if (ty64(a.elem)) return Cls{K_ARG64, (uint8_t)slot};
    return none;
  }
  // a __local pointer argument: the low dword of its slot is the buffer's LDS address
  if (!a.hidden && a.pointer && a.space == 2 && part == PART_ENTIRE) return Cls{K_LPTR, (uint8_t)slot};
  if (a.hidden || a.pointer || ty64(a.elem) || part != PART_ENTIRE) return none;
  return Cls{K_ARG32, (uint8_t)slot};
}

__device__ __forceinline__ int64_t const_of_f(const KView& v, uint32_t s) {
  if (!r_node(s) || rpart(s) != PART_ENTIRE) return -1;
  const Node& n = v.node(rid(s));
  return n.kind == N_CONST ? (int64_t)n.cval : -1;
}
// constant value of forwarded source q of node n, -1 if not a constant
__device__ __forceinline__ int64_t const_src(const KView& v, const Node& n, int q) {
  return const_of_f(v, nsrc(v, n, q));
}

// a scalar load (the only source of settings and dispatch packet values)
__device__ __forceinline__ bool may_sload(const KView& v, uint32_t r) {
  if (!r_node(r)) return false;
  const Node& n = v.node(rid(r));
  return n.kind == N_SLOAD64B ||
         (n.kind == N_OP && (n.op == O_S_LOAD_DWORD || n.op == O_S_LOAD_DWORDX2 || n.op == O_S_LOAD_DWORDX4));
}
// a value that may be a part of the global id chain: the local id (a leaf),
// group id * size, the offset-free id, or the low half of a global offset
__device__ __forceinline__ bool may_gid_part(const KView& v, uint32_t r) {
  if (r_leaf(r)) return true;
  if (!r_node(r)) return false;
  const Node& n = v.node(rid(r));
  if (n.kind == N_SLOAD64B) return true;
  if (n.kind != N_OP) return false;
  switch (n.op) {
    case O_S_LOAD_DWORD: case O_S_LOAD_DWORDX2: case O_S_LOAD_DWORDX4: case O_S_MUL_I32: case O_S_LSHL_B32:
    case O_V_ADD_U32: case O_V_MAD_U32_U24: return true;
  }
  return false;
}

static __device__ GD_MATCH_INLINE Cls classify_d(const KView& v, uint32_t r, int d) {
  Cls none{K_NONE, 0};
  if (r == kUndef || r == kTop) return Cls{K_UNDEF, 0};
  if (v.cc && r_node(r) && rpart(r) == PART_ENTIRE) return Cls{v.cc[rid(r)], v.ck[rid(r)]};
  if (d > kClassDepth && r_node(r)) return none;
  if (r_leaf(r)) return leaf_class(r);
  if (!r_node(r)) return none;
  const Node& n = v.node(rid(r));
  uint32_t part = rpart(r);
  if (n.kind == N_CONST) return Cls{K_CONST32, 0};
  if (n.kind == N_PAIR && part == PART_ENTIRE) {
    Cls a = classify_d(v, nsrc(v, n, 0), d + 1), b = classify_d(v, nsrc(v, n, 1), d + 1);
    return (a.c == K_CONST32 && b.c == K_CONST32) ? Cls{K_CONST64, 0} : none;
  }
  if (n.kind == N_SLOAD64B) return settings_load(v, n, part, true, d);
  if (n.kind != N_OP) return none;
  if (n.op == O_S_LOAD_DWORDX2 || n.op == O_S_LOAD_DWORDX4) return settings_load(v, n, part, true, d);
  if (n.op == O_S_LOAD_DWORD) return settings_load(v, n, part, false, d);
  if (part != PART_ENTIRE) return none;
  // Operand screens: each pattern below needs its operands to be of particular
  // kinds (a leaf for the group or local id, a scalar load for a settings or
  // packet value, one of the chain's operations), so an operand of any other
  // kind gives no class and the recursion into it is skipped.  This only
  // avoids work: the class returned is the same.
  switch (n.op) {
    case O_S_MUL_I32:
      if (!r_leaf(nsrc(v, n, 0)) && !r_leaf(nsrc(v, n, 1))) return none;
      break;
    case O_S_LSHL_B32:
      if (!r_leaf(nsrc(v, n, 0))) return none;
      break;
    case O_S_LSHR_B32: case O_S_BFE_U32:
      if (!may_sload(v, nsrc(v, n, 0))) return none;
      break;
    case O_V_ADD_U32:
      if (!may_gid_part(v, nsrc(v, n, 0)) || !may_gid_part(v, nsrc(v, n, 1))) return none;
      break;
    case O_V_MAD_U32_U24:
      if (!r_leaf(nsrc(v, n, 2)) || (!r_leaf(nsrc(v, n, 0)) && !r_leaf(nsrc(v, n, 1)))) return none;
      break;
  }
  const uint32_t* cws = v.K->cws;
  auto cw = [&](int d) -> int64_t { return d < 3 ? (int64_t)cws[d] : -1; };
  switch (n.op) {
    case O_S_MUL_I32: {
      Cls a = classify_d(v, nsrc(v, n, 0), d + 1), b = classify_d(v, nsrc(v, n, 1), d + 1);
      if (a.c == K_GRP && const_src(v, n, 1) == cw(a.k)) return Cls{K_MULGRP, a.k};
      if (b.c == K_GRP && const_src(v, n, 0) == cw(b.k)) return Cls{K_MULGRP, b.k};
      return none;
    }
    case O_S_LSHL_B32: {
      Cls a = classify_d(v, nsrc(v, n, 0), d + 1);
      if (a.c == K_GRP) {
        int l = ilog2_exact((uint32_t)cw(a.k));
        if (l >= 0 && const_src(v, n, 1) == l) return Cls{K_MULGRP, a.k};
      }
      return none;
    }
    case O_S_LSHR_B32: {  // global size / work-group size, the size a power of two
      Cls a = classify_d(v, nsrc(v, n, 0), d + 1);
      if (a.c == K_GSIZE) {
        int l = ilog2_exact((uint32_t)cw(a.k));
        if (l >= 0 && const_src(v, n, 1) == l) return Cls{K_NGRP, a.k};
      }
      return none;
    }
    case O_S_BFE_U32: {
      Cls a = classify_d(v, nsrc(v, n, 0), d + 1);
      return (a.c == K_DISP0 && const_src(v, n, 1) == 0x20010) ? Cls{K_WDIM, 0} : none;
    }
    case O_V_ADD_U32: {
      Cls a = classify_d(v, nsrc(v, n, 0), d + 1), b = classify_d(v, nsrc(v, n, 1), d + 1);
      if (a.c == K_MULGRP && b.c == K_LID && a.k == b.k) return Cls{K_GIDNO, a.k};
      if (b.c == K_MULGRP && a.c == K_LID && a.k == b.k) return Cls{K_GIDNO, a.k};
      if (a.c == K_GIDNO && b.c == K_GOFSLO && a.k == b.k) return Cls{K_GID, a.k};
      if (b.c == K_GIDNO && a.c == K_GOFSLO && a.k == b.k) return Cls{K_GID, a.k};
      return none;
    }
    case O_V_MAD_U32_U24: {
      Cls a = classify_d(v, nsrc(v, n, 0), d + 1), b = classify_d(v, nsrc(v, n, 1), d + 1), c = classify_d(v, nsrc(v, n, 2), d + 1);
      if (c.c != K_LID) return none;
      if (a.c == K_GRP && a.k == c.k && const_src(v, n, 1) == cw(a.k)) return Cls{K_GIDNO, a.k};
      if (b.c == K_GRP && b.k == c.k && const_src(v, n, 0) == cw(b.k)) return Cls{K_GIDNO, b.k};
      return none;
    }
  }
  return none;
}

// the class of value r
__device__ __forceinline__ Cls classify(const KView& v, uint32_t r) { return classify_q(v, r, 0); }

// memory access: argument pointer + (32-bit index, extended) << log2(element size)
struct Mem {
  bool ok;
  uint32_t arg;
  uint32_t idx;  // kTop = constant 0
};

static __device__ GD_MATCH_INLINE Mem match_addr(const KView& v, uint32_t addr, uint32_t width) {
  Mem m{false, kNone, kTop};
  Cls c = classify(v, addr);
  if (c.c == K_ARGPTR) {
    if ((ty64(v.A[c.k].elem) ? 8u : 4u) != width) return m;
    m.ok = true;
    m.arg = c.k;
    return m;
  }
  if (!r_node(addr) || rpart(addr) != PART_ENTIRE) return m;
  const Node& n = v.node(rid(addr));
  if (n.kind != N_OP || n.op != O_V_ADDC_CO_U32 || !n.fused) return m;
  for (int o = 0; o < 2; ++o) {
    uint32_t X = nsrc(v, n, o), Y = nsrc(v, n, 1 - o);
    Cls cx = classify(v, X);
    if (cx.c != K_ARGPTR) continue;
    uint32_t es = ty64(v.A[cx.k].elem) ? 8u : 4u;
    if (es != width) continue;
    if (!r_node(Y) || rpart(Y) != PART_ENTIRE) continue;
    const Node& sh = v.node(rid(Y));
    if (sh.kind != N_OP || sh.op != O_V_LSHLREV_B64) continue;
    if (const_src(v, sh, 0) != ilog2_exact(es)) continue;
    uint32_t V = nsrc(v, sh, 1);
    if (!r_node(V) || rpart(V) != PART_ENTIRE || v.node(rid(V)).kind != N_PAIR) continue;
    const Node& p = v.node(rid(V));
    uint32_t lo = nsrc(v, p, 0), hi = nsrc(v, p, 1);
    bool ext = false;
    if (r_node(hi) && rpart(hi) == PART_ENTIRE && v.node(rid(hi)).kind == N_CONST && v.node(rid(hi)).cval == 0)
      ext = true;
    if (r_node(hi) && rpart(hi) == PART_ENTIRE) {
      const Node& a = v.node(rid(hi));
      if (a.kind == N_OP && a.op == O_V_ASHRREV_I32 && const_src(v, a, 0) == 31 && nsrc(v, a, 1) == lo)
        ext = true;
    }
    if (!ext) continue;
    m.ok = true;
    m.arg = cx.k;
    m.idx = lo;
    return m;
  }
  return m;
}

// LDS access: the __local buffer's 32-bit LDS address plus the index shifted by log2 of the
// element size (v_lshlrev_b32 then v_add_u32, either operand order), or the address alone
static __device__ GD_MATCH_INLINE Mem match_lds(const KView& v, uint32_t addr, uint32_t width) {
  Mem m{false, kNone, kTop};
  Cls c = classify(v, addr);
  if (c.c == K_LPTR) {
    if ((ty64(v.A[c.k].elem) ? 8u : 4u) != width) return m;
    m.ok = true;
    m.arg = c.k;
    return m;
  }
  if (!r_node(addr) || rpart(addr) != PART_ENTIRE) return m;
  const Node& n = v.node(rid(addr));
  if (n.kind != N_OP || n.op != O_V_ADD_U32) return m;
  for (int o = 0; o < 2; ++o) {
    uint32_t X = nsrc(v, n, o), Y = nsrc(v, n, 1 - o);
    Cls cx = classify(v, X);
    if (cx.c != K_LPTR) continue;
    uint32_t es = ty64(v.A[cx.k].elem) ? 8u : 4u;
    if (es != width) continue;
    if (!r_node(Y) || rpart(Y) != PART_ENTIRE) continue;
    const Node& sh = v.node(rid(Y));
    if (sh.kind != N_OP || sh.op != O_V_LSHLREV_B32) continue;
    if (const_src(v, sh, 0) != ilog2_exact(es)) continue;
    m.ok = true;
    m.arg = cx.k;
    m.idx = nsrc(v, sh, 1);
    return m;
  }
  return m;
}
// the match of load / store node n's address, by its kind of access
__device__ __forceinline__ Mem match_mem(const KView& v, const Node& n) {
  return op_lds(n.op) ? match_lds(v, nsrc(v, n, 0), op_mem_width(n.op)) : match_addr(v, nsrc(v, n, 0), op_mem_width(n.op));
}

__device__ __forceinline__ bool op_vcmp(uint16_t op) { return op >= O_V_CMP0 && op < O_V_CMP0 + 18; }
__device__ __forceinline__ bool op_scmp(uint16_t op) { return op >= O_S_CMP0 && op < O_S_CMP0 + 12; }
__device__ __forceinline__ bool op_wide(uint16_t op) {
  return op == O_S_LOAD_DWORDX2 || op == O_V_CVT_F64_F32 || op == O_V_CVT_F64_I32 || op == O_V_LSHLREV_B64 ||
         op == O_V_ADD_F64 || op == O_V_MUL_F64 || op == O_V_FMA_F64 || op == O_GLOBAL_LOAD_DWORDX2 ||
         op == O_FLAT_LOAD_DWORDX2 || op == O_DS_READ_B64;
}

__device__ __forceinline__ int node_width(const KView& v, uint32_t id) {
  const Node& n = v.node(id);
  if (n.kind == N_PAIR || n.kind == N_SLOAD64B) return 64;
  if (n.kind == N_OP) {
    if (op_wide(n.op) || n.op == O_S_LOAD_DWORDX4) return 64;
    if ((n.op == O_V_ADDC_CO_U32 || n.op == O_V_SUBB_CO_U32) && n.fused) return 64;
  }
  return 32;
}

__device__ __forceinline__ uint8_t tjoin(uint8_t a, uint8_t b) {
  if (a == TY_NONE) return b;
  if (b == TY_NONE) return a;
  if (a == b) return a;
  return (ty64(a) || ty64(b)) ? TY_TOP64 : TY_TOP32;
}
__device__ __forceinline__ uint8_t tresolve(uint8_t t, int width) {
  if (t == TY_NONE) return width == 64 ? TY_ULONG : TY_UINT;
  if (t == TY_TOP32) return TY_UINT;
  if (t == TY_TOP64) return TY_ULONG;
  return t;
}

// children printed with a node (after forwarding); returns the count (<= 3)
// memory match of load/store node `id` (slot 0 of its instruction)
__device__ __forceinline__ Mem mem_of(const KView& v, uint32_t id) {
  if (v.marg) return Mem{v.marg[id / 4] != kNone, v.marg[id / 4], v.midx[id / 4]};
  return match_mem(v, v.node(id));
}

static __device__ int node_children(const KView& v, uint32_t id, uint32_t* ch) {
  const Node& n = v.node(id);
  if (leaf_like(classify(v, mkref(id, PART_ENTIRE)).c)) return 0;
  int c = 0;
  if (n.kind == N_PAIR) {
    ch[c++] = nsrc(v, n, 0);
    ch[c++] = nsrc(v, n, 1);
    return c;
  }
  if (n.kind != N_OP) return 0;
  if (op_gload(n.op) || op_store(n.op)) {
    Mem m = mem_of(v, id);
    if (m.ok) {
      if (m.idx != kTop) ch[c++] = m.idx;
    } else {
      ch[c++] = nsrc(v, n, 0);
    }
    if (op_store(n.op)) ch[c++] = nsrc(v, n, 1);
    return c;
  }
  if (n.op == O_UNKNOWN || n.op == O_S_LOAD_DWORD || n.op == O_S_LOAD_DWORDX2 || n.op == O_S_LOAD_DWORDX4) return 0;
  for (int q = 0; q < n.nsrc && q < 3; ++q) ch[c++] = nsrc(v, n, q);
  return c;
}

}  // namespace gd
