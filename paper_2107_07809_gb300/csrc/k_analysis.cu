// k_analysis.cu — S9-S11 kernels: what is printed, how often, and its type.
//
// Roots (stores, loads, unsupported instructions, branch conditions) are
// followed through printed operands and through the versions created at
// joins; a node becomes a variable when it is a load, is used twice, is used
// in another block, or feeds a join version.  Types ("Data type recovery"):
// arguments fix the types of loads and scalars, instruction suffixes fix the
// rest, bitwise operations and join versions take the join of their inputs in
// the lattice none < {int, uint, float} < top32 (64-bit likewise), iterated to
// the least fixed point.  One thread per kernel walks its nodes.
#include "k_analysis.cuh"

namespace gd {

__device__ __forceinline__ uint32_t out_val(const Batch& b, const KHdr& K, uint32_t p, uint32_t reg) {
  uint32_t v = b.st_out[K.state_off + (size_t)p * K.R + reg];
  return v == kTop ? kUndef : v;
}
__device__ __forceinline__ uint32_t phi_blk(uint32_t r) { return (rid(r) >> 10) & 0x3FFFF; }
__device__ __forceinline__ uint32_t phi_reg(uint32_t r) { return rid(r) & 0x3FF; }

__global__ void k_reach(Batch b, uint32_t* __restrict__ wl_all) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad) return;
  KView v = make_view(b, K, k);
  const size_t nb = 4 * (size_t)K.first_instr;
  uint32_t* uses = b.uses + nb;
  uint8_t* fl = b.nflag + nb;
  uint8_t* pu = b.phi_used + K.state_off;
  uint32_t* wl = wl_all + K.wl_off;
  uint32_t cap = 4 * K.n_instr + K.n_lblock * K.R + 8, sp = 0;
  uint32_t nn = 4 * K.n_instr;
  for (uint32_t q = 0; q < nn; ++q) {
    uses[q] = 0;
    fl[q] = 0;
  }
  for (size_t q = 0; q < (size_t)K.n_lblock * K.R; ++q) pu[q] = 0;
  // a reference from block `blk`: count it; queue first visits for expansion
  auto use = [&](uint32_t r, uint32_t blk) {
    if (r_phi(r)) {
      uint32_t B = phi_blk(r), reg = phi_reg(r);
      uint8_t& u = pu[(size_t)B * K.R + reg];
      if (!u) {
        u = 1;
        if (sp < cap) wl[sp++] = r;
        else atomicOr(b.err, ERR_CAPACITY);
      }
      return;
    }
    if (!r_node(r)) return;
    uint32_t id = rid(r);
    uses[id]++;
    if (b.lblock_of[K.first_instr + id / 4] != blk) fl[id] |= 2;
    if (!(fl[id] & 1)) {
      fl[id] |= 1;
      if (sp < cap) wl[sp++] = r & ~3u;
      else atomicOr(b.err, ERR_CAPACITY);
    }
  };
  for (uint32_t bl = 0; bl < K.n_lblock; ++bl) {
    const BlockRec& B = b.lblocks[K.first_lblock + bl];
    for (uint32_t i = B.first; i < B.end; ++i) {
      uint32_t gi = K.first_instr + i;
      if (b.lblock_of[gi] != bl) continue;
      const Node& n = v.node(4 * i);
      if (n.kind != N_OP) continue;
      if (b.ctl[gi] == C_CBR) {
        if (B.succ1 != kNone) use(nsrc(v, n, 0), bl);
        continue;
      }
      if (op_store(n.op) || op_gload(n.op) || n.op == O_UNKNOWN) {
        if (!(fl[4 * i] & 1)) {
          fl[4 * i] |= 1;
          uint32_t ch[3];
          int c = node_children(v, 4 * i, ch);
          for (int q = 0; q < c; ++q) use(ch[q], bl);
        }
      }
    }
  }
  while (sp) {
    uint32_t r = wl[--sp];
    if (r_phi(r)) {
      uint32_t B = phi_blk(r), reg = phi_reg(r);
      for (uint32_t pi = b.pred_off[K.first_lblock + B]; pi < b.pred_off[K.first_lblock + B + 1]; ++pi) {
        uint32_t p = b.preds[pi];
        uint32_t x = fwd(v, out_val(b, K, p, reg));
        if (r_node(x)) fl[rid(x)] |= 4;
        use(x, p);
      }
      continue;
    }
    uint32_t id = rid(r);
    uint32_t blk = b.lblock_of[K.first_instr + id / 4];
    uint32_t ch[3];
    int c = node_children(v, id, ch);
    for (int q = 0; q < c; ++q) use(ch[q], blk);
  }
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
    case K_GID: case K_GIDNO: case K_LID: case K_GRP: case K_GOFSLO: return TY_UINT;
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
    case O_V_ADD_U32: case O_V_SUB_U32: case O_V_MUL_LO_U32: case O_V_MAD_U32_U24: case O_V_MUL_U32_U24: return TY_UINT;
    case O_V_AND_B32: case O_V_OR_B32: case O_V_XOR_B32: return tjoin(st(0), st(1));
    case O_V_LSHLREV_B32: return st(1);
    case O_V_LSHRREV_B32: return TY_UINT;
    case O_V_ASHRREV_I32: return TY_INT;
    case O_V_ADD_F32: case O_V_SUB_F32: case O_V_MUL_F32: case O_V_FMA_F32: case O_V_CVT_F32_I32:
    case O_V_CVT_F32_U32: case O_V_CVT_F32_F64: return TY_FLOAT;
    case O_V_CVT_F64_F32: case O_V_CVT_F64_I32: case O_V_ADD_F64: case O_V_MUL_F64: case O_V_FMA_F64: return TY_DOUBLE;
    case O_V_ADD_CO_U32: case O_V_SUB_CO_U32: return TY_UINT;
    case O_V_ADDC_CO_U32: case O_V_SUBB_CO_U32: return n.fused ? tjoin(st(0), st(1)) : TY_UINT;
    case O_V_LSHLREV_B64: return st(1);
    case O_GLOBAL_LOAD_DWORD: case O_GLOBAL_LOAD_DWORDX2: {
      Mem m = mem_of(v, id);
      if (m.ok) return v.A[m.arg].elem;
      return n.op == O_GLOBAL_LOAD_DWORDX2 ? TY_ULONG : TY_UINT;
    }
    case O_S_LOAD_DWORD: return TY_UINT;
    case O_S_LOAD_DWORDX2: case O_S_LOAD_DWORDX4: return TY_ULONG;
    case O_UNKNOWN: return node_width(v, id) == 64 ? TY_ULONG : TY_UINT;
  }
  if (op_scmp(n.op) || op_vcmp(n.op)) return TY_INT;
  return TY_NONE;
}

__global__ void k_types(Batch b) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad) return;
  KView v = make_view(b, K, k);
  const size_t nb = 4 * (size_t)K.first_instr;
  uint8_t* nt = b.ntype + nb;
  const uint8_t* fl = b.nflag + nb;
  uint8_t* pt = b.phi_type + K.state_off;
  const uint8_t* pu = b.phi_used + K.state_off;
  uint32_t nn = 4 * K.n_instr;
  size_t np = (size_t)K.n_lblock * K.R;
  for (uint32_t q = 0; q < nn; ++q) nt[q] = TY_NONE;
  for (size_t q = 0; q < np; ++q) pt[q] = TY_NONE;
  bool changed = true;
  int guard = 0;
  while (changed && guard++ < 100000) {
    changed = false;
    for (uint32_t id = 0; id < nn; ++id) {
      if (!(fl[id] & 1)) continue;
      uint8_t t = tjoin(nt[id], node_type(v, nt, pt, id));
      if (t != nt[id]) { nt[id] = t; changed = true; }
    }
    for (size_t q = 0; q < np; ++q) {
      if (!pu[q]) continue;
      uint32_t B = (uint32_t)(q / K.R), reg = (uint32_t)(q % K.R);
      uint8_t t = pt[q];
      for (uint32_t pi = b.pred_off[K.first_lblock + B]; pi < b.pred_off[K.first_lblock + B + 1]; ++pi)
        t = tjoin(t, ref_type(v, nt, pt, fwd(v, out_val(b, K, b.preds[pi], reg))));
      if (t != pt[q]) { pt[q] = t; changed = true; }
    }
  }
  if (changed) atomicOr(b.err, ERR_CAPACITY);
}

__device__ __forceinline__ bool is_var_node(const KView& v, const uint32_t* uses, const uint8_t* fl, uint32_t id) {
  if (!(fl[id] & 1)) return false;
  const Node& n = v.node(id);
  if (leaf_like(classify(v, mkref(id, PART_ENTIRE)).c)) return false;
  if (n.kind == N_OP && op_store(n.op)) return false;
  if (n.kind == N_OP && (op_gload(n.op) || n.op == O_UNKNOWN)) return true;
  return uses[id] >= 2 || (fl[id] & 6);
}

// variable numbers: per block its join versions (by register), then its nodes
// by (instruction, slot); this is the order of their program points
__global__ void k_vars(Batch b) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad) return;
  KView v = make_view(b, K, k);
  const size_t nb = 4 * (size_t)K.first_instr;
  int32_t* vo = b.var_of + nb;
  const uint32_t* uses = b.uses + nb;
  const uint8_t* fl = b.nflag + nb;
  const uint8_t* nt = b.ntype + nb;
  int32_t* pv = b.phi_var + K.state_off;
  const uint8_t* pu = b.phi_used + K.state_off;
  const uint8_t* pt = b.phi_type + K.state_off;
  uint8_t* vt = b.var_type + nb + K.state_off;
  for (uint32_t q = 0; q < 4 * K.n_instr; ++q) vo[q] = -1;
  int32_t n = 0;
  for (uint32_t bl = 0; bl < K.n_lblock; ++bl) {
    for (uint32_t r = 0; r < K.R; ++r) {
      size_t q = (size_t)bl * K.R + r;
      if (pu[q]) {
        pv[q] = n;
        vt[n++] = tresolve(pt[q], 32);
      } else {
        pv[q] = -1;
      }
    }
    const BlockRec& B = b.lblocks[K.first_lblock + bl];
    for (uint32_t i = B.first; i < B.end; ++i) {
      if (b.lblock_of[K.first_instr + i] != bl) continue;
      for (uint32_t s = 0; s < 4; ++s) {
        uint32_t id = 4 * i + s;
        if (is_var_node(v, uses, fl, id)) {
          vo[id] = n;
          vt[n++] = tresolve(nt[id], node_width(v, id));
        }
      }
    }
  }
  K.n_vars = (uint32_t)n;
}

__global__ void k_wl_size(Batch b, uint32_t* __restrict__ sz) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  const KHdr& K = b.kh[k];
  sz[k] = K.bad ? 0u : 4 * K.n_instr + K.n_lblock * K.R + 3 * K.R + 8;
}
__global__ void k_wl_off(Batch b, const uint32_t* __restrict__ off) {
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
__global__ void k_node_cache(Batch b, uint8_t* __restrict__ cc, uint8_t* __restrict__ ck, uint32_t* __restrict__ sf,
                             uint32_t* __restrict__ marg, uint32_t* __restrict__ midx) {
  uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 4ull * b.I) return;
  uint32_t gi = (uint32_t)(g / 4);
  uint32_t k = b.ikern[gi];
  const KHdr& K = b.kh[k];
  KView v = make_view(b, K, k);  // b carries no caches here
  uint32_t id = (uint32_t)(g - 4ull * K.first_instr);
  const Node& n = v.node(id);
  Cls c{K_NONE, 0};
  if (!K.bad && n.kind != N_NONE) c = classify(v, mkref(id, PART_ENTIRE));
  cc[g] = c.c;
  ck[g] = c.k;
  for (int q = 0; q < 3; ++q) sf[3 * g + q] = (!K.bad && q < n.nsrc) ? fwd(v, n.src[q]) : kTop;
  if ((g & 3) == 0) {
    uint32_t a = kNone, x = kTop;
    if (!K.bad && n.kind == N_OP && (op_gload(n.op) || op_store(n.op))) {
      uint32_t w = (n.op == O_GLOBAL_LOAD_DWORDX2 || n.op == O_GLOBAL_STORE_DWORDX2) ? 8 : 4;
      Mem m = match_addr(v, fwd(v, n.src[0]), w);
      if (m.ok) {
        a = m.arg;
        x = m.idx;
      }
    }
    marg[gi] = a;
    midx[gi] = x;
  }
}

void launch_node_cache(Batch& b, cudaStream_t s) {
  if (!b.I) return;
  Batch raw = b;
  raw.ncls = nullptr;
  uint64_t n = 4ull * b.I;
  k_node_cache<<<(uint32_t)((n + 255) / 256), 256, 0, s>>>(raw, b.ncls, b.nclsk, b.nsrcf, b.mem_arg, b.mem_idx);
  ++launch_counter();
}

void launch_analysis(Batch& b, uint32_t* wl, cudaStream_t s) {
  if (!b.K) return;
  const int T = 64;
  k_reach<<<(b.K + T - 1) / T, T, 0, s>>>(b, wl);
  ++launch_counter();
  k_types<<<(b.K + T - 1) / T, T, 0, s>>>(b);
  ++launch_counter();
  k_vars<<<(b.K + T - 1) / T, T, 0, s>>>(b);
  ++launch_counter();
}

}  // namespace gd
