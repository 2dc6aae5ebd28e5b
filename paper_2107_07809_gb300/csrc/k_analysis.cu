// k_analysis.cu — S9-S11 kernels: what is printed, how often, and its type.
//
// Roots (stores, loads, unsupported instructions, branch conditions) are
// followed through printed operands and through the versions created at
// joins; a node becomes a variable when it is a load, is used twice, is used
// in another block, or feeds a join version.  Types ("Data type recovery"):
// arguments fix the types of loads and scalars, instruction suffixes fix the
// rest, bitwise operations and join versions take the join of their inputs in
// the lattice none < {int, uint, float} < top32 (64-bit likewise), iterated to
// the least fixed point.  A warp (short kernels) or a thread block (long
// kernels) walks a kernel's nodes.
#include "k_analysis.cuh"
#include <algorithm>

namespace gd {

__device__ __forceinline__ uint32_t out_val(const Batch& b, const KHdr& K, uint32_t p, uint32_t reg) {
  uint32_t v = b.st_out[K.state_off + (size_t)p * K.R + reg];
  return v == kTop ? kUndef : v;
}
__device__ __forceinline__ uint32_t phi_blk(uint32_t r) { return (rid(r) >> 10) & 0x3FFFF; }
__device__ __forceinline__ uint32_t phi_reg(uint32_t r) { return rid(r) & 0x3FF; }

// Reachability and use counts, one team per kernel.  Its threads pop up to
// one entry each of the kernel's stack at a time; the first visit of a node or join
// version is claimed with an atomic bit, use counts are atomic adds, so the
// result does not depend on the order the lanes happen to take.
__device__ __forceinline__ bool claim(uint32_t* bits, uint64_t g) {
  uint32_t m = 1u << (g & 31);
  return !(atomicOr(&bits[g >> 5], m) & m);
}

template <bool WARP>
__device__ __forceinline__ void reach_one(const Batch& b, uint32_t k, uint32_t* __restrict__ wl_all, uint32_t* __restrict__ rbits,
                                          uint32_t* __restrict__ cbits, uint32_t* __restrict__ ibits, uint32_t* __restrict__ pbits) {
  using T = Team<WARP>;
  __shared__ uint32_t s_top[4], s_npl[4];
  const uint32_t wid = T::slot(), lane = T::tid(), TS = T::size();
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad || !T::mine(K, b.big_kernel)) return;
  const KView& v = b.kview[k];
  const size_t nb = 4 * (size_t)K.first_instr;
  uint32_t* uses = b.uses + nb;
  uint8_t* pu = b.phi_used + K.state_off;
  uint32_t* wl = wl_all + K.wl_off;
  uint32_t* pl = b.plist + K.state_off;
  const uint32_t nn = 4 * K.n_instr;
  const uint32_t cap = nn + K.n_lblock * K.R + 8;
  // uses and phi_used start zeroed for the whole batch (a memset before the launch)
  if (lane == 0) {
    s_top[wid] = 0;
    s_npl[wid] = 0;
  }
  T::sync();
  auto push = [&](uint32_t r) {
    uint32_t at = atomicAdd(&s_top[wid], 1u);
    if (at < cap) wl[at] = r;
    else atomicOr(b.err, ERR_CAPACITY);
  };
  auto use = [&](uint32_t r, uint32_t blk) {
    if (r_phi(r)) {
      uint32_t B = (rid(r) >> 10) & 0x3FFFF, reg = rid(r) & 0x3FF;
      size_t slot = (size_t)B * K.R + reg;
      if (claim(pbits, K.state_off + slot)) {
        pu[slot] = 1;
        pl[atomicAdd(&s_npl[wid], 1u)] = (B << 10) | reg;
        push(r);
      }
      return;
    }
    if (!r_node(r)) return;
    uint32_t id = rid(r);
    atomicAdd(&uses[id], 1u);
    if (b.lblock_of[K.first_instr + id / 4] != blk) claim(cbits, nb + id);
    if (claim(rbits, nb + id)) push(r & ~3u);
  };
  // roots: stores, loads, unsupported instructions (expanded), branch conditions (used)
  for (uint32_t i = lane; i < K.n_instr; i += TS) {
    uint32_t gi = K.first_instr + i;
    uint32_t bl = b.lblock_of[gi];
    if (bl == kNone) continue;
    const Node& n = v.node(4 * i);
    if (n.kind != N_OP) continue;
    if (b.ctl[gi] == C_CBR) {
      if (b.lblocks[K.first_lblock + bl].succ1 != kNone) use(nsrc(v, n, 0), bl);
      continue;
    }
    if ((op_store(n.op) || op_gload(n.op) || n.op == O_UNKNOWN) && claim(rbits, nb + 4 * i)) push(mkref(4 * i, 0));
  }
  T::sync();
  for (;;) {
    uint32_t top = s_top[wid];
    if (top > cap) top = cap;
    uint32_t take = top < TS ? top : TS;
    if (!take) break;
    uint32_t r = lane < take ? wl[top - 1 - lane] : kTop;
    T::sync();
    if (lane == 0) s_top[wid] = top - take;
    T::sync();
    if (r != kTop) {
      if (r_phi(r)) {
        uint32_t B = (rid(r) >> 10) & 0x3FFFF, reg = rid(r) & 0x3FF;
        for (uint32_t pi = b.pred_off[K.first_lblock + B]; pi < b.pred_off[K.first_lblock + B + 1]; ++pi) {
          uint32_t p = b.preds[pi];
          uint32_t x = fwd(v, out_val(b, K, p, reg));
          if (r_node(x)) claim(ibits, nb + rid(x));
          use(x, p);
        }
      } else {
        uint32_t id = rid(r);
        uint32_t blk = b.lblock_of[K.first_instr + id / 4];
        uint32_t ch[3];
        int c = node_children(v, id, ch);
        for (int q = 0; q < c; ++q) use(ch[q], blk);
      }
    }
    T::sync();
  }
  T::sync();
  if (lane == 0) K.n_phis = s_npl[wid];
}

// a persistent team (a warp, or a block for the block bucket) per slot of the GPU, taking kernels
// from the work queue of its bucket, longest first
template <bool WARP>
__global__ void __launch_bounds__(WARP ? 128 : kBigTeam, WARP ? 8 : 1)
    k_reach(const __grid_constant__ Batch b, uint32_t* __restrict__ wl_all, uint32_t* __restrict__ rbits,
            uint32_t* __restrict__ cbits, uint32_t* __restrict__ ibits, uint32_t* __restrict__ pbits,
            const __grid_constant__ KernelOrder ko) {
  const uint32_t nbig = ko.info[0];
  const uint32_t* list = WARP ? ko.order + nbig : ko.order;
  const uint32_t n = WARP ? b.K - nbig : nbig;
  for (uint32_t k; (k = Team<WARP>::next(&ko.heads[WARP ? 1 : 0], list, n)) != kNone;)
    reach_one<WARP>(b, k, wl_all, rbits, cbits, ibits, pbits);
}

// node flags from the reachability bitmaps (reached, used in another block,
// feeds a join version): one thread per instruction, its four slots' bytes at once
__global__ void k_reach_flags(const __grid_constant__ Batch b, const uint32_t* __restrict__ rbits,
                              const uint32_t* __restrict__ cbits, const uint32_t* __restrict__ ibits) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  const uint64_t g = 4ull * gi;  // four bits of one word
  const uint32_t sh = (uint32_t)(g & 31), w = (uint32_t)(g >> 5);
  const uint32_t r = (rbits[w] >> sh) & 0xFu, c = (cbits[w] >> sh) & 0xFu, x = (ibits[w] >> sh) & 0xFu;
  uint32_t f = 0;
  for (int q = 0; q < 4; ++q) f |= (((r >> q) & 1u) | (((c >> q) & 1u) << 1) | (((x >> q) & 1u) << 2)) << (8 * q);
  reinterpret_cast<uint32_t*>(b.nflag)[gi] = f;
}

// ---------------------------------------------------------------------------
// types
// ---------------------------------------------------------------------------
__device__ uint8_t ref_type(const KView& v, const uint8_t* nt, const uint8_t* pt, uint32_t r) {
  if (r_phi(r)) return pt[(size_t)phi_blk(r) * v.K->R + phi_reg(r)];
  if (r_leaf(r)) {
    Cls c = classify(v, r);
    return (c.c == K_LID || c.c == K_GRP) ? TY_UINT : TY_NONE;
  }
  if (!r_node(r)) return TY_NONE;
  if (rpart(r) != PART_ENTIRE) return TY_UINT;
  return nt[rid(r)];
}

__device__ uint8_t node_type(const KView& v, const uint8_t* nt, const uint8_t* pt, uint32_t id) {
  const Node& n = v.node(id);
  Cls c = classify(v, mkref(id, PART_ENTIRE));
  switch (c.c) {
    case K_GID: case K_GIDNO: case K_LID: case K_GRP: case K_GOFSLO: case K_GSIZE: case K_NGRP: case K_WDIM:
    case K_LPTR:
      return TY_UINT;
    case K_GOFS64: case K_ARGPTR: case K_KARG: return TY_ULONG;
    case K_ARG32: case K_ARG64: return v.A[c.k].elem;
    case K_CONST32: case K_CONST64: case K_UNDEF: return TY_NONE;
  }
  auto st = [&](int q) { return ref_type(v, nt, pt, nsrc(v, n, q)); };
  if (n.kind == N_PAIR || n.kind == N_SLOAD64B) return TY_ULONG;
  if (n.kind == N_CARRY) return TY_UINT;
  if (n.kind != N_OP) return TY_NONE;
  switch (n.op) {
    case O_S_MUL_I32: return TY_INT;
    case O_S_ADD_U32: return TY_UINT;
    case O_S_LSHL_B32: return st(0);
    case O_S_LSHR_B32: case O_S_BFE_U32: return TY_UINT;
    case O_V_ADD_U32: case O_V_SUB_U32: case O_V_MUL_LO_U32: case O_V_MAD_U32_U24: case O_V_MUL_U32_U24: return TY_UINT;
    case O_V_AND_B32: case O_V_OR_B32: case O_V_XOR_B32: case O_V_CNDMASK_B32: return tjoin(st(0), st(1));
    case O_V_LSHLREV_B32: return st(1);
    case O_V_LSHRREV_B32: return TY_UINT;
    case O_V_ASHRREV_I32: return TY_INT;
    case O_V_ADD_F32: case O_V_SUB_F32: case O_V_MUL_F32: case O_V_FMA_F32: case O_V_CVT_F32_I32:
    case O_V_CVT_F32_U32: case O_V_CVT_F32_F64: return TY_FLOAT;
    case O_V_CVT_F64_F32: case O_V_CVT_F64_I32: case O_V_ADD_F64: case O_V_MUL_F64: case O_V_FMA_F64: return TY_DOUBLE;
    case O_V_ADD_CO_U32: case O_V_SUB_CO_U32: return TY_UINT;
    case O_V_ADDC_CO_U32: case O_V_SUBB_CO_U32: return n.fused ? tjoin(st(0), st(1)) : TY_UINT;
    case O_V_LSHLREV_B64: return st(1);
    case O_V_MUL_HI_U32_U24: return TY_UINT;
    case O_V_MUL_HI_I32_I24: return TY_INT;
    case O_GLOBAL_LOAD_DWORD: case O_GLOBAL_LOAD_DWORDX2: case O_FLAT_LOAD_DWORD: case O_FLAT_LOAD_DWORDX2:
    case O_DS_READ_B32: case O_DS_READ_B64: {
      Mem m = mem_of(v, id);
      if (m.ok) return v.A[m.arg].elem;
      return op_mem_width(n.op) == 8 ? TY_ULONG : TY_UINT;
    }
    case O_S_LOAD_DWORD: return TY_UINT;
    case O_S_LOAD_DWORDX2: case O_S_LOAD_DWORDX4: return TY_ULONG;
    case O_UNKNOWN: return node_width(v, id) == 64 ? TY_ULONG : TY_UINT;
  }
  if (op_scmp(n.op) || op_vcmp(n.op)) return TY_INT;
  return TY_NONE;
}

// least fixed point of the type equations: one team per kernel, its threads
// update nodes and used join versions concurrently until a vote finds no
// change (the equations are monotone, so every such iteration reaches the same
// solution)
// nodes whose type comes from the types of their operands (the others' types
// follow from their operation, class or argument alone)
__device__ __forceinline__ bool type_from_operands(const Node& n) {
  if (n.kind != N_OP) return false;
  switch (n.op) {
    case O_S_LSHL_B32: case O_V_AND_B32: case O_V_OR_B32: case O_V_XOR_B32: case O_V_LSHLREV_B32:
    case O_V_LSHLREV_B64: case O_V_CNDMASK_B32: return true;
    case O_V_ADDC_CO_U32: case O_V_SUBB_CO_U32: return n.fused != 0;
  }
  return false;
}

// A node typed by its operation alone is final after one evaluation (its
// equation has no unknowns): one thread per instruction types those of its four
// slots and lists the others, whose type comes from their operands, in its
// kernel's list for the iteration (the reachability work list, free again).
__global__ void __launch_bounds__(128, 12) k_types_static(const __grid_constant__ Batch b, uint32_t* __restrict__ wl_all) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  const uint32_t k = b.ikern[gi];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const KView& v = b.kview[k];
  const size_t nb = 4 * (size_t)K.first_instr;
  uint8_t* nt = b.ntype + nb;
  const uint8_t* pt = b.phi_type + K.state_off;
  const uint32_t id0 = 4 * (gi - K.first_instr);
  const uint32_t f4 = reinterpret_cast<const uint32_t*>(b.nflag)[gi];
  uint32_t t4 = 0;
  for (uint32_t s = 0; s < 4; ++s) {
    uint8_t t = TY_NONE;
    if ((f4 >> (8 * s)) & 1u) {
      if (type_from_operands(v.node(id0 + s))) wl_all[K.wl_off + atomicAdd(&b.dyn_count[k], 1u)] = id0 + s;
      else t = node_type(v, nt, pt, id0 + s);
    }
    t4 |= (uint32_t)t << (8 * s);
  }
  reinterpret_cast<uint32_t*>(b.ntype)[gi] = t4;
}

template <bool WARP>
__device__ __forceinline__ void types_one(const Batch& b, uint32_t k, uint32_t* __restrict__ wl_all) {
  using T = Team<WARP>;
  const uint32_t lane = T::tid(), TS = T::size();
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad || !T::mine(K, b.big_kernel)) return;
  const KView& v = b.kview[k];
  const size_t nb = 4 * (size_t)K.first_instr;
  uint8_t* nt = b.ntype + nb;
  uint8_t* pt = b.phi_type + K.state_off;
  const uint32_t* pl = b.plist + K.state_off;
  uint32_t* dyn = wl_all + K.wl_off;  // the reachability work list is free again
  for (uint32_t q = lane; q < K.n_phis; q += TS) {
    uint32_t e = pl[q];
    pt[(size_t)(e >> 10) * K.R + (e & 0x3FF)] = TY_NONE;
  }
  T::sync();
  const uint32_t nd = b.dyn_count[k];  // listed by k_types_static
  bool changed = true;
  uint32_t sweeps = 0;
  while (changed && sweeps++ < b.type_sweeps) {
    bool ch = false;
    for (uint32_t q = lane; q < nd; q += TS) {
      const uint32_t id = dyn[q];
      uint8_t t = tjoin(nt[id], node_type(v, nt, pt, id));
      if (t != nt[id]) {
        nt[id] = t;
        ch = true;
      }
    }
    T::sync();
    for (uint32_t q = lane; q < K.n_phis; q += TS) {
      uint32_t e = pl[q];
      uint32_t B = e >> 10, reg = e & 0x3FF;
      size_t slot = (size_t)B * K.R + reg;
      uint8_t t = pt[slot];
      for (uint32_t pi = b.pred_off[K.first_lblock + B]; pi < b.pred_off[K.first_lblock + B + 1]; ++pi)
        t = tjoin(t, ref_type(v, nt, pt, fwd(v, out_val(b, K, b.preds[pi], reg))));
      if (t != pt[slot]) {
        pt[slot] = t;
        ch = true;
      }
    }
    T::sync();
    changed = T::any(ch);
  }
  // still changing in the last allowed sweep: this kernel is not decompiled (FIXPOINT_CAP)
  if (lane == 0) K.capped = changed ? 1u : 0u;
}

template <bool WARP>
__global__ void __launch_bounds__(WARP ? 128 : kBigTeam, WARP ? 8 : 1)
    k_types(const __grid_constant__ Batch b, uint32_t* __restrict__ wl_all, const __grid_constant__ KernelOrder ko) {
  const uint32_t nbig = ko.info[0];
  const uint32_t* list = WARP ? ko.order + nbig : ko.order;
  const uint32_t n = WARP ? b.K - nbig : nbig;
  for (uint32_t k; (k = Team<WARP>::next(&ko.heads[WARP ? 3 : 2], list, n)) != kNone;) types_one<WARP>(b, k, wl_all);
}

__device__ __forceinline__ bool is_var_node(const KView& v, const uint32_t* uses, const uint8_t* fl, uint32_t id) {
  if (!(fl[id] & 1)) return false;
  const Node& n = v.node(id);
  if (leaf_like(classify(v, mkref(id, PART_ENTIRE)).c)) return false;
  if (n.kind == N_OP && op_store(n.op)) return false;
  if (n.kind == N_OP && (op_gload(n.op) || n.op == O_UNKNOWN)) return true;
  return uses[id] >= 2 || (fl[id] & 6);
}

// Variable numbers: per block its join versions (by register), then its
// nodes by (instruction, slot); this is the order of their program points.
// Every candidate gets a position in that order inside its kernel's range of
// a batch-wide array (join version r of block bl at bl*R + 4*first(bl) + r,
// node slot s of instruction i of block bl at (bl+1)*R + 4*i + s; the range of
// kernel k starts at state_off + 4*first_instr), a flag is set for each
// variable, and one exclusive scan numbers them all.
__device__ __forceinline__ size_t vbase(const KHdr& K) { return (size_t)K.state_off + 4 * (size_t)K.first_instr; }

// one thread per instruction over its four node slots
__global__ void __launch_bounds__(128, 12) k_var_flag_nodes(const __grid_constant__ Batch b, uint32_t* __restrict__ vflag) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  const uint32_t bl = b.lblock_of[gi];
  if (bl == kNone) return;
  const uint32_t f4 = reinterpret_cast<const uint32_t*>(b.nflag)[gi];
  if (!(f4 & 0x01010101u)) return;  // no slot is reached
  const uint32_t k = b.ikern[gi];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const KView& v = b.kview[k];
  const size_t nb = 4 * (size_t)K.first_instr;
  const uint32_t id0 = 4 * (gi - K.first_instr);
  uint32_t* f = vflag + vbase(K) + (size_t)(bl + 1) * K.R;
  for (uint32_t s = 0; s < 4; ++s)
    if (((f4 >> (8 * s)) & 1) && is_var_node(v, b.uses + nb, b.nflag + nb, id0 + s)) f[id0 + s] = 1;
}

__global__ void k_var_flag_joins(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern,
                                 uint32_t* __restrict__ vflag) {
  const uint32_t gb = blockIdx.x * blockDim.x + threadIdx.x;
  if (gb >= b.NLB) return;
  const uint32_t k = blk_kern[gb];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const uint32_t bl = gb - K.first_lblock;
  const uint8_t* pu = b.phi_used + K.state_off + (size_t)bl * K.R;
  uint32_t* f = vflag + vbase(K) + (size_t)bl * K.R + 4 * (size_t)b.lblocks[gb].first;
  for (uint32_t r = 0; r < K.R; ++r)
    if (pu[r]) f[r] = 1;
}

__global__ void k_var_nodes(const __grid_constant__ Batch b, const uint32_t* __restrict__ vflag,
                            const uint32_t* __restrict__ vpos) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  const uint32_t k = b.ikern[gi];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const size_t nb = 4 * (size_t)K.first_instr;
  const uint32_t id0 = 4 * (gi - K.first_instr);
  const uint32_t bl = b.lblock_of[gi];
  int4 x4 = make_int4(-1, -1, -1, -1);
  if (bl != kNone) {
    const size_t at = vbase(K) + (size_t)(bl + 1) * K.R + id0;
    const uint32_t base = vpos[vbase(K)];
    int* x = &x4.x;
    for (uint32_t s = 0; s < 4; ++s) {
      if (vflag[at + s]) {
        x[s] = (int32_t)(vpos[at + s] - base);
        const KView v = make_view(b, K, k);
        b.var_type[nb + K.state_off + x[s]] = tresolve(b.ntype[nb + id0 + s], node_width(v, id0 + s));
      }
    }
  }
  reinterpret_cast<int4*>(b.var_of)[gi] = x4;
}

__global__ void k_var_joins(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern,
                            const uint32_t* __restrict__ vflag, const uint32_t* __restrict__ vpos) {
  const uint32_t gb = blockIdx.x * blockDim.x + threadIdx.x;
  if (gb >= b.NLB) return;
  const uint32_t k = blk_kern[gb];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const uint32_t bl = gb - K.first_lblock;
  const size_t q0 = (size_t)bl * K.R;
  const size_t at0 = vbase(K) + q0 + 4 * (size_t)b.lblocks[gb].first;
  const uint32_t p0 = vpos[vbase(K)];
  const size_t nb = 4 * (size_t)K.first_instr;
  for (uint32_t r = 0; r < K.R; ++r) {
    int32_t x = -1;
    if (vflag[at0 + r]) {
      x = (int32_t)(vpos[at0 + r] - p0);
      b.var_type[nb + K.state_off + x] = tresolve(b.phi_type[K.state_off + q0 + r], 32);
    }
    b.phi_var[K.state_off + q0 + r] = x;
  }
}

__global__ void k_var_count(const __grid_constant__ Batch b, const uint32_t* __restrict__ vpos) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  const size_t end = k + 1 < b.K ? vbase(b.kh[k + 1]) : (size_t)b.NS + 4 * (size_t)b.I;
  K.n_vars = K.bad ? 0u : vpos[end] - vpos[vbase(K)];
}

__global__ void k_wl_size(const __grid_constant__ Batch b, uint32_t* __restrict__ sz) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  const KHdr& K = b.kh[k];
  sz[k] = K.bad ? 0u : 4 * K.n_instr + K.n_lblock * K.R + 3 * K.R + 8;
}
__global__ void k_wl_off(const __grid_constant__ Batch b, const uint32_t* __restrict__ off) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  b.kh[k].wl_off = off[k];
}

void launch_wl_size(Batch& b, uint32_t* sz, uint32_t* off, ScanScratch sc, uint32_t* total, cudaStream_t s) {
  if (!b.K) return;
  k_wl_size<<<(b.K + 127) / 128, 128, 0, s>>>(b, sz);
  ++launch_counter();
  launch_scan(sz, off, b.K, 0, false, sc, total, b.err, s);
  k_wl_off<<<(b.K + 127) / 128, 128, 0, s>>>(b, off);
  ++launch_counter();
}

// one thread per node: its class, its forwarded sources and, for a load or
// store, its memory match; later stages read these instead of recomputing
// Node caches, in two passes of one thread per instruction over its four node
// slots (most instructions define one value, so a thread per slot left three
// lanes in four idle).  First the forwarded sources of every node, then the
// classes and memory matches, whose pattern walks read those sources.
// fwd_n(v.N, r, 0) with its loop in line: only a whole pair (its two halves
// forwarded separately) makes a recursive call
__device__ __forceinline__ uint32_t fwd_inline(const KView& v, uint32_t r) {
  for (int step = 0; step < 512; ++step) {
    if (r == kTop) return kUndef;
    if (!r_node(r)) return r;
    const Node& n = v.node(rid(r));
    const uint32_t part = rpart(r);
    if (is_copy_node(n) && part == PART_ENTIRE) {
      r = n.src[0];
      continue;
    }
    if (n.kind == N_PAIR) {
      if (part == PART_LO) { r = n.src[0]; continue; }
      if (part == PART_HI) { r = n.src[1]; continue; }
      return fwd_n(v.N, r, 0);
    }
    return r;
  }
  return r;
}

// classify(v, r) for a node without a class cache, with the nodes that
// classify_d turns down before looking at any operand answered in line
__device__ __forceinline__ Cls classify_node(const KView& v, uint32_t id) {
  const Node& n = v.node(id);
  if (n.kind == N_CONST) return Cls{K_CONST32, 0};
  if (n.kind == N_OP ? !class_op(n.op) : (n.kind != N_PAIR && n.kind != N_SLOAD64B)) return Cls{K_NONE, 0};
  return classify_d(v, mkref(id, PART_ENTIRE), 0);
}

__global__ void __launch_bounds__(128, 12)
    k_node_fwd(const __grid_constant__ Batch b, uint32_t* __restrict__ sf) {
  // a block's results (12 words per instruction, consecutive for consecutive instructions) are
  // gathered in shared memory and stored as whole 16-byte pieces
  __shared__ __align__(16) uint32_t s_sf[128 * 12];
  const uint32_t g0 = blockIdx.x * blockDim.x, gi = g0 + threadIdx.x;
  if (gi < b.I) {
    const uint32_t k = b.ikern[gi];
    const KHdr& K = b.kh[k];
    const KView v = make_view(b, K, k);  // b carries no caches here
    const bool bad = K.bad;
    const uint32_t id0 = 4 * (gi - K.first_instr);
    for (int s = 0; s < 4; ++s) {
      const Node& n = v.node(id0 + s);
      for (int q = 0; q < 3; ++q)
        s_sf[12 * threadIdx.x + 3 * s + q] = (!bad && q < n.nsrc) ? fwd_inline(v, n.src[q]) : kTop;
    }
  }
  __syncthreads();
  const uint32_t nw = 12 * min(blockDim.x, b.I - g0);  // a multiple of 4
  uint32_t* dst = sf + 12ull * g0;
  if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
    for (uint32_t q = threadIdx.x; q < nw / 4; q += blockDim.x)
      reinterpret_cast<uint4*>(dst)[q] = reinterpret_cast<const uint4*>(s_sf)[q];
  } else {
    for (uint32_t q = threadIdx.x; q < nw; q += blockDim.x) dst[q] = s_sf[q];
  }
}

// the views of every kernel, once: with the forwarded sources only, and with every cache
__global__ void k_make_views(const __grid_constant__ Batch b, KView* __restrict__ vsf, KView* __restrict__ vall) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KView v = make_view(b, b.kh[k], k);  // b carries the caches' arrays here
  vall[k] = v;
  v.cc = nullptr;
  v.ck = nullptr;
  v.marg = nullptr;
  v.midx = nullptr;
  vsf[k] = v;
}

__global__ void __launch_bounds__(128, 12)
    k_node_cache(const __grid_constant__ Batch b, uint8_t* __restrict__ cc, uint8_t* __restrict__ ck,
                 const uint32_t* __restrict__ sf, uint32_t* __restrict__ marg, uint32_t* __restrict__ midx) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  const uint32_t k = b.ikern[gi];
  const KHdr& K = b.kh[k];
  const KView& v = b.kview_sf[k];  // the forwarded sources, no class caches yet
  const bool bad = K.bad;
  const uint32_t id0 = 4 * (gi - K.first_instr);
  uint32_t cls = 0, clk = 0;
  for (int s = 0; s < 4; ++s) {
    const Node& n = v.node(id0 + s);
    Cls c{K_NONE, 0};
    if (!bad && n.kind != N_NONE) c = classify_node(v, id0 + s);
    cls |= (uint32_t)c.c << (8 * s);
    clk |= (uint32_t)c.k << (8 * s);
  }
  reinterpret_cast<uint32_t*>(cc)[gi] = cls;
  reinterpret_cast<uint32_t*>(ck)[gi] = clk;
  uint32_t a = kNone, x = kTop;
  const Node& n = v.node(id0);
  if (!bad && n.kind == N_OP && (op_gload(n.op) || op_store(n.op))) {
    Mem m = match_mem(v, n);
    if (m.ok) {
      a = m.arg;
      x = m.idx;
    }
  }
  marg[gi] = a;
  midx[gi] = x;
}

size_t kview_bytes() { return sizeof(KView); }

void launch_node_cache(Batch& b, void* views, cudaStream_t s) {
  if (!b.I) return;
  KView* vsf = static_cast<KView*>(views);
  b.kview_sf = vsf;
  b.kview = vsf + b.K;
  k_make_views<<<(b.K + 127) / 128, 128, 0, s>>>(b, vsf, vsf + b.K);
  ++launch_counter();
  Batch raw = b;
  raw.ncls = nullptr;
  ktime(KT_NODE_FWD, 0, s);
  k_node_fwd<<<(b.I + 127) / 128, 128, 0, s>>>(raw, b.nsrcf);
  ktime(KT_NODE_FWD, 1, s);
  ktime(KT_NODE_CACHE, 0, s);
  k_node_cache<<<(b.I + 127) / 128, 128, 0, s>>>(raw, b.ncls, b.nclsk, b.nsrcf, b.mem_arg, b.mem_idx);
  ktime(KT_NODE_CACHE, 1, s);
  ++launch_counter();
  ++launch_counter();
}

// One block: a histogram of the kernels by (bucket, size class) in shared memory, its exclusive
// scan (the class of the largest kernels first), then every kernel placed at its class's cursor.
constexpr int kOrderClasses = 64;  // 32 size classes (binary logarithm) per bucket
__global__ void __launch_bounds__(1024) k_kernel_order(const __grid_constant__ Batch b, const __grid_constant__ KernelOrder ko) {
  __shared__ uint32_t cnt[kOrderClasses];
  const uint32_t t = threadIdx.x;
  if (t < kOrderClasses) cnt[t] = 0;
  __syncthreads();
  auto cls = [&](uint32_t k) {
    const uint32_t n = b.kh[k].n_instr;
    const uint32_t lg = 31u - (uint32_t)__clz(n | 1u);
    return (n >= b.big_kernel ? 0u : 32u) + (31u - lg);
  };
  for (uint32_t k = t; k < b.K; k += blockDim.x) atomicAdd(&cnt[cls(k)], 1u);
  __syncthreads();
  if (t == 0) {
    uint32_t run = 0, big = 0;
    for (int c = 0; c < kOrderClasses; ++c) {
      const uint32_t x = cnt[c];
      cnt[c] = run;
      run += x;
      if (c == 31) big = run;
    }
    ko.info[0] = big;
  }
  __syncthreads();
  for (uint32_t k = t; k < b.K; k += blockDim.x) ko.order[atomicAdd(&cnt[cls(k)], 1u)] = k;
}

void launch_kernel_order(const Batch& b, const KernelOrder& ko, cudaStream_t s) {
  if (!b.K) return;
  k_kernel_order<<<1, 1024, 0, s>>>(b, ko);
  ++launch_counter();
}

// blocks of a team kernel resident on the whole GPU at once (the persistent grid), per device
template <class F>
static uint32_t resident_blocks(F kernel, int threads, int* cache) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = per_sm > 0 && sms > 0 ? per_sm * sms : 1;
  }
  return (uint32_t)cache[dev];
}

void launch_analysis(Batch& b, uint32_t* wl, uint32_t* bits, uint64_t nbits_words, const uint32_t* blk_kern,
                     uint32_t* vflag, uint32_t* vpos, ScanScratch sc, SideStream fk, const KernelOrder& ko,
                     cudaStream_t s) {
  if (!b.K) return;
  // four bitmaps: reached nodes, cross-block uses, join inputs (4I bits each), used joins (NS bits)
  uint64_t wn = (4ull * b.I + 63) / 32;
  uint32_t *rb = bits, *cb = bits + wn, *ib = bits + 2 * wn, *pb = bits + 3 * wn;
  cudaMemsetAsync(bits, 0, sizeof(uint32_t) * nbits_words, s);
  // the two size buckets touch disjoint kernels (shared bitmap words only through atomics):
  // the block-per-kernel bucket runs on the side stream, beside the warp-per-kernel one
  cudaMemsetAsync(b.uses, 0, sizeof(uint32_t) * 4ull * b.I, s);
  if (b.NS) cudaMemsetAsync(b.phi_used, 0, b.NS, s);
  cudaMemsetAsync(b.dyn_count, 0, sizeof(uint32_t) * b.K, s);
  static int res_reach[2][64], res_types[2][64];
  const uint32_t gw = std::min<uint32_t>((b.K + 3) / 4, resident_blocks(k_reach<true>, 128, res_reach[1]));
  const uint32_t gb = std::min<uint32_t>(b.K, resident_blocks(k_reach<false>, kBigTeam, res_reach[0]));
  cudaMemsetAsync(ko.heads, 0, 4 * sizeof(uint32_t), s);
  cudaEventRecord(fk.fork, s);
  cudaStreamWaitEvent(fk.side, fk.fork, 0);
  k_reach<false><<<gb, kBigTeam, 0, fk.side>>>(b, wl, rb, cb, ib, pb, ko);
  k_reach<true><<<gw, 128, 0, s>>>(b, wl, rb, cb, ib, pb, ko);
  cudaEventRecord(fk.join, fk.side);
  cudaStreamWaitEvent(s, fk.join, 0);
  if (b.I) {
    k_reach_flags<<<(b.I + 255) / 256, 256, 0, s>>>(b, rb, cb, ib);
    k_types_static<<<(b.I + 127) / 128, 128, 0, s>>>(b, wl);
    launch_counter() += 2;
  }
  cudaEventRecord(fk.fork, s);
  cudaStreamWaitEvent(fk.side, fk.fork, 0);
  const uint32_t tw = std::min<uint32_t>((b.K + 3) / 4, resident_blocks(k_types<true>, 128, res_types[1]));
  const uint32_t tb = std::min<uint32_t>(b.K, resident_blocks(k_types<false>, kBigTeam, res_types[0]));
  k_types<false><<<tb, kBigTeam, 0, fk.side>>>(b, wl, ko);
  k_types<true><<<tw, 128, 0, s>>>(b, wl, ko);
  cudaEventRecord(fk.join, fk.side);
  cudaStreamWaitEvent(s, fk.join, 0);
  launch_counter() += 4;
  // variable numbers over the candidate array of NS + 4I positions
  const uint64_t nc = (uint64_t)b.NS + 4ull * b.I;
  cudaMemsetAsync(vflag, 0, sizeof(uint32_t) * (nc + 1), s);
  if (b.I) {
    k_var_flag_nodes<<<(b.I + 127) / 128, 128, 0, s>>>(b, vflag);
    ++launch_counter();
  }
  if (b.NLB) {
    k_var_flag_joins<<<(b.NLB + 127) / 128, 128, 0, s>>>(b, blk_kern, vflag);
    ++launch_counter();
  }
  launch_scan(vflag, vpos, (uint32_t)(nc + 1), 0, false, sc, nullptr, b.err, s);
  if (b.I) {
    k_var_nodes<<<(b.I + 127) / 128, 128, 0, s>>>(b, vflag, vpos);
    ++launch_counter();
  }
  if (b.NLB) {
    k_var_joins<<<(b.NLB + 127) / 128, 128, 0, s>>>(b, blk_kern, vflag, vpos);
    ++launch_counter();
  }
  k_var_count<<<(b.K + 127) / 128, 128, 0, s>>>(b, vpos);
  ++launch_counter();
}

}  // namespace gd
