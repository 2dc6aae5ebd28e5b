// k_dataflow.cu — S7/S8: register versions and expression nodes.
//
// The paper assigns versions to registers and creates variables where a
// block with several predecessors sees different versions ("Search for
// control structures", last paragraphs).  The placement computed here is the
// minimal one: register r gets a new version at block B exactly when B is in
// the iterated dominance frontier of r's defining blocks (the entry defines
// every register with its ABI value).  GPU mapping:
//   - 64-bit carry pairs: one thread per instruction; a block's definitions:
//     one warp per block, 32 instructions at a time (k_local_defs);
//   - dominators (reverse postorder + iterative intersection): one warp per
//     kernel, lane 0 walking;
//   - the frontier closure for all registers at once: a warp per kernel, or a
//     thread block for a long kernel; its threads take join blocks and walk the
//     dominator-tree paths from their predecessors, the bitsets of all
//     registers at once, in sweeps until nothing changes;
//   - values: the same team walks blocks in reverse postorder, threads over registers;
//   - nodes: one warp per block, 32 instructions at a time (k_nodes).
#include "gd_kernels.h"

namespace gd {

struct RegMap {
  uint32_t vg, sg;
  __device__ __forceinline__ uint32_t v(uint32_t i) const { return i; }
  __device__ __forceinline__ uint32_t s(uint32_t i) const { return vg + i; }
  __device__ __forceinline__ uint32_t vcc() const { return vg + sg; }
  __device__ __forceinline__ uint32_t scc() const { return vg + sg + 1; }
  __device__ __forceinline__ uint32_t spill(uint32_t k) const { return vg + sg + 2 + k; }
};

struct Def {
  uint32_t reg, val;
};

__device__ __forceinline__ bool vcmp(uint16_t op) { return op >= O_V_CMP0 && op < O_V_CMP0 + 18; }
__device__ __forceinline__ bool scmp(uint16_t op) { return op >= O_S_CMP0 && op < O_S_CMP0 + 12; }
__device__ __forceinline__ bool wide_result(uint16_t op) {
  return op == O_S_LOAD_DWORDX2 || op == O_V_CVT_F64_F32 || op == O_V_CVT_F64_I32 || op == O_V_LSHLREV_B64 ||
         op == O_V_ADD_F64 || op == O_V_MUL_F64 || op == O_V_FMA_F64 || op == O_GLOBAL_LOAD_DWORDX2 ||
         op == O_FLAT_LOAD_DWORDX2 || op == O_DS_READ_B64;
}

// register index of the first register of an operand word (v/s/vcc)
__device__ __forceinline__ uint32_t reg_of(const RegMap& M, uint32_t o, uint32_t k) {
  uint32_t tg = otag(o);
  if (tg == TG_VGPR) return M.v(opay(o) + k);
  if (tg == TG_SGPR) return M.s(opay(o) + k);
  return M.vcc();
}

// definitions of kernel-relative instruction i (at most 4)
__device__ __forceinline__ int idefs(const Batch& b, const KHdr& K, const RegMap& M, uint32_t i, Def* d) {
  uint32_t gi = K.first_instr + i;
  if (b.ctl[gi] != C_NORMAL) return 0;
  const InstrRec& r = b.ins[gi];
  uint32_t base = 4 * i;
  int n = 0;
  switch (r.op) {
    case O_S_WAITCNT: case O_GLOBAL_STORE_DWORD: case O_GLOBAL_STORE_DWORDX2: case O_FLAT_STORE_DWORD:
    case O_FLAT_STORE_DWORDX2: case O_DS_WRITE_B32: case O_DS_WRITE_B64: case O_S_BARRIER: return 0;
    case O_S_LOAD_DWORD: d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_ENTIRE)}; return n;
    case O_S_LOAD_DWORDX4:
      d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_LO)};
      d[n++] = {reg_of(M, r.opnd[0], 1), mkref(base, PART_HI)};
      d[n++] = {reg_of(M, r.opnd[0], 2), mkref(base + 1, PART_LO)};
      d[n++] = {reg_of(M, r.opnd[0], 3), mkref(base + 1, PART_HI)};
      return n;
    case O_S_ADD_U32: case O_S_MUL_I32: case O_S_LSHL_B32: case O_S_LSHR_B32: case O_S_BFE_U32:
      d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_ENTIRE)};
      d[n++] = {M.scc(), kUndef};
      return n;
    case O_V_ADD_CO_U32: case O_V_SUB_CO_U32:
      d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_ENTIRE)};
      d[n++] = {M.vcc(), mkref(base + 3, PART_ENTIRE)};
      return n;
    case O_V_ADDC_CO_U32: case O_V_SUBB_CO_U32:
      if (b.fused[gi]) {
        const InstrRec& lo = b.ins[K.first_instr + b.co_idx[gi]];
        d[n++] = {reg_of(M, lo.opnd[0], 0), mkref(base, PART_LO)};
        d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_HI)};
      } else {
        d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_ENTIRE)};
      }
      d[n++] = {M.vcc(), kUndef};
      return n;
    case O_BUFFER_STORE_DWORD: d[n++] = {M.spill(r.imm / 4), mkref(base, PART_ENTIRE)}; return n;
    case O_UNKNOWN: {
      if (!r.nops) return 0;
      uint32_t o = r.opnd[0], tg = otag(o);
      if (tg != TG_VGPR && tg != TG_SGPR && tg != TG_VCC) return 0;
      uint32_t c = tg == TG_VCC ? 1 : ocnt(o);
      if (c == 2) {
        d[n++] = {reg_of(M, o, 0), mkref(base, PART_LO)};
        d[n++] = {reg_of(M, o, 1), mkref(base, PART_HI)};
      } else {
        for (uint32_t q = 0; q < c && n < 4; ++q) d[n++] = {reg_of(M, o, q), mkref(base, PART_ENTIRE)};
      }
      return n;
    }
    default:
      if (scmp(r.op)) { d[n++] = {M.scc(), mkref(base, PART_ENTIRE)}; return n; }
      if (vcmp(r.op)) { d[n++] = {M.vcc(), mkref(base, PART_ENTIRE)}; return n; }
      if (wide_result(r.op)) {
        d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_LO)};
        d[n++] = {reg_of(M, r.opnd[0], 1), mkref(base, PART_HI)};
      } else {
        d[n++] = {reg_of(M, r.opnd[0], 0), mkref(base, PART_ENTIRE)};
      }
      return n;
  }
}

__device__ __forceinline__ bool defines_vcc(const InstrRec& r) {
  return r.op == O_V_ADD_CO_U32 || r.op == O_V_SUB_CO_U32 || r.op == O_V_ADDC_CO_U32 || r.op == O_V_SUBB_CO_U32 ||
         vcmp(r.op) || (r.op == O_UNKNOWN && r.nops && otag(r.opnd[0]) == TG_VCC);
}

// ---------------------------------------------------------------------------
// sizes: spill slots, register count, limits
// ---------------------------------------------------------------------------
// spill slots: the largest scratch offset of a buffer load/store (thread per instruction)
__global__ void k_df_spill(const __grid_constant__ Batch b) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  const InstrRec& r = b.ins[gi];
  if (r.op == O_BUFFER_LOAD_DWORD || r.op == O_BUFFER_STORE_DWORD) atomicMax(&b.kh[b.ikern[gi]].nspill, r.imm / 4 + 1);
}

// the entry block may not be the target of a branch (thread per logical block)
__global__ void k_df_entry(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.NLB) return;
  const BlockRec& B = b.lblocks[g];
  if (B.succ0 == 0 || B.succ1 == 0) atomicOr(&b.kh[blk_kern[g]].entry_target, 1u);
}

__global__ void k_df_sizes(const __grid_constant__ Batch b, uint32_t* __restrict__ kstate) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  K.R = K.vgprs + K.sgprs + 2 + K.nspill;
  if (!K.bad && (K.R > kMaxRegs || K.n_lblock >= kMaxBlocks || K.n_instr >= (1u << 26))) K.bad |= 16u;
  if (!K.bad && K.n_lblock && K.entry_target) K.bad |= 32u;
  kstate[k] = K.bad ? 0u : K.n_lblock * K.R;
}

__global__ void k_state_off(const __grid_constant__ Batch b, const uint32_t* __restrict__ off) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  b.kh[k].state_off = off[k];
}

// ---------------------------------------------------------------------------
// 64-bit carry pairs: v_addc_co_u32 / v_subb_co_u32 completing the low half of
// the last carry-out of the same block (whose register still holds it)
// ---------------------------------------------------------------------------
__global__ void k_fusion(const __grid_constant__ Batch b) {
  uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  b.fused[gi] = 0;
  b.co_idx[gi] = kNone;
  const InstrRec& r = b.ins[gi];
  if (r.op != O_V_ADDC_CO_U32 && r.op != O_V_SUBB_CO_U32) return;
  const KHdr& K = b.kh[b.ikern[gi]];
  if (K.bad || b.ctl[gi] != C_NORMAL) return;
  uint32_t i = gi - K.first_instr;
  uint32_t blk = b.lblock_of[gi];
  if (blk == kNone) return;
  uint32_t first = b.lblocks[K.first_lblock + blk].first;
  int j = -1;
  for (int q = (int)i - 1; q >= (int)first; --q) {
    uint32_t gq = K.first_instr + q;
    if (b.lblock_of[gq] != blk || b.ctl[gq] != C_NORMAL) continue;
    if (defines_vcc(b.ins[gq])) { j = q; break; }
  }
  uint16_t want = r.op == O_V_ADDC_CO_U32 ? O_V_ADD_CO_U32 : O_V_SUB_CO_U32;
  if (j < 0 || b.ins[K.first_instr + j].op != want) return;
  // the operand pairs take slots 1 and 2 and a constant high source slot 3: at most one constant
  uint32_t t2 = otag(r.opnd[2]), t3 = otag(r.opnd[3]);
  if (!(t2 == TG_VGPR || t2 == TG_SGPR || t2 == TG_VCC) && !(t3 == TG_VGPR || t3 == TG_SGPR || t3 == TG_VCC)) return;
  RegMap M{K.vgprs, K.sgprs};
  uint32_t lo = M.v(opay(b.ins[K.first_instr + j].opnd[0]));
  uint32_t hi = M.v(opay(r.opnd[0]));
  if (lo == hi) return;
  for (uint32_t q = (uint32_t)j + 1; q < i; ++q) {
    if (b.lblock_of[K.first_instr + q] != blk) continue;
    Def d[4];
    int n = idefs(b, K, M, q, d);  // no carry instruction sits between j and i
    for (int t = 0; t < n; ++t)
      if (d[t].reg == lo) return;
  }
  b.fused[gi] = 1;
  b.co_idx[gi] = (uint32_t)j;
}

// ---------------------------------------------------------------------------
// predecessors (CSR, sorted)
// ---------------------------------------------------------------------------
__global__ void k_pred_count(const __grid_constant__ Batch b, uint32_t* __restrict__ cnt, const uint32_t* __restrict__ blk_kern) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.NLB) return;
  const KHdr& K = b.kh[blk_kern[g]];
  const BlockRec& B = b.lblocks[g];
  if (B.succ0 != kNone) atomicAdd(&cnt[K.first_lblock + B.succ0], 1u);
  if (B.succ1 != kNone) atomicAdd(&cnt[K.first_lblock + B.succ1], 1u);
}

__global__ void k_pred_fill(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.NLB) return;
  const KHdr& K = b.kh[blk_kern[g]];
  const BlockRec& B = b.lblocks[g];
  uint32_t rel = g - K.first_lblock;
  if (B.succ0 != kNone) {
    uint32_t s = K.first_lblock + B.succ0;
    b.preds[b.pred_off[s] + atomicAdd(&b.pred_fill[s], 1u)] = rel;
  }
  if (B.succ1 != kNone) {
    uint32_t s = K.first_lblock + B.succ1;
    b.preds[b.pred_off[s] + atomicAdd(&b.pred_fill[s], 1u)] = rel;
  }
}

__global__ void k_pred_sort(const __grid_constant__ Batch b) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.NLB) return;
  uint32_t a = b.pred_off[g], e = b.pred_off[g + 1];
  for (uint32_t x = a + 1; x < e; ++x) {  // insertion sort: lists are short
    uint32_t v = b.preds[x];
    uint32_t y = x;
    while (y > a && b.preds[y - 1] > v) {
      b.preds[y] = b.preds[y - 1];
      --y;
    }
    b.preds[y] = v;
  }
}

// ---------------------------------------------------------------------------
// dominators: depth-first reverse postorder, then iterative intersection
// ---------------------------------------------------------------------------
__global__ void k_dominators(const __grid_constant__ Batch b, uint32_t* __restrict__ rpo_index, uint32_t* __restrict__ stk,
                             uint8_t* __restrict__ child) {
  uint32_t k = walk_kernel();
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  uint32_t nb = K.n_lblock, base = K.first_lblock;
  if (K.bad || !nb) return;
  const BlockRec* B = b.lblocks + base;
  uint32_t* order = b.rpo + base;
  uint32_t* ri = rpo_index + base;
  uint32_t* idom = b.idom + base;
  uint32_t* st = stk + base;
  uint8_t* ch = child + base;
  for (uint32_t x = 0; x < nb; ++x) {
    ri[x] = kNone;
    idom[x] = kNone;
    ch[x] = 0;
  }
  // iterative DFS; postorder written backwards gives the reverse postorder
  uint32_t sp = 0, npost = 0;
  st[sp++] = 0;
  ri[0] = 0;  // "seen"
  uint32_t* post = b.scratch32 + base;
  while (sp) {
    uint32_t x = st[sp - 1];
    uint32_t s = kNone;
    while (ch[x] < 2 && s == kNone) {
      uint32_t c = ch[x] == 0 ? B[x].succ0 : B[x].succ1;
      ++ch[x];
      if (c != kNone && ri[c] == kNone) s = c;
    }
    if (s != kNone) {
      ri[s] = 0;
      st[sp++] = s;
    } else {
      post[npost++] = x;
      --sp;
    }
  }
  for (uint32_t q = 0; q < nb; ++q) ri[q] = kNone;
  for (uint32_t q = 0; q < npost; ++q) {
    order[q] = post[npost - 1 - q];
    ri[order[q]] = q;
  }
  for (uint32_t q = npost; q < nb; ++q) order[q] = kNone;
  idom[0] = 0;
  bool changed = true;
  while (changed) {
    changed = false;
    for (uint32_t q = 1; q < npost; ++q) {
      uint32_t x = order[q], nd = kNone;
      for (uint32_t pi = b.pred_off[base + x]; pi < b.pred_off[base + x + 1]; ++pi) {
        uint32_t p = b.preds[pi];
        if (ri[p] == kNone || idom[p] == kNone) continue;
        if (nd == kNone) nd = p;
        else {
          uint32_t a1 = p, a2 = nd;
          while (a1 != a2) {
            while (ri[a1] > ri[a2]) a1 = idom[a1];
            while (ri[a2] > ri[a1]) a2 = idom[a2];
          }
          nd = a1;
        }
      }
      if (nd != idom[x]) {
        idom[x] = nd;
        changed = true;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// per-block definitions: last definition of every register (into st_out) and
// the block's definition bitset
// ---------------------------------------------------------------------------
// Registers are hashed into buckets; a bucket's mask holds the lanes of the
// chunk that define a register of that bucket, so a lookup checks only those.
constexpr uint32_t kDefBuckets = 64;

// the latest lane below `below` (a lane mask) that defines reg, or -1; its definition slot in *slot
__device__ __forceinline__ int last_def(const uint32_t (*dreg)[4], const uint32_t* dmask, uint32_t reg,
                                        uint32_t below, int* slot) {
  uint32_t cand = dmask[reg % kDefBuckets] & below;
  while (cand) {
    const int m = 31 - __clz(cand);
    for (int t = 3; t >= 0; --t)
      if (dreg[m][t] == reg) {
        *slot = t;
        return m;
      }
    cand &= ~(1u << m);
  }
  return -1;
}

// One warp per block, 32 instructions at a time: the lanes list their
// instructions' definitions in shared memory, set the definition bits, and the
// chunk's last definition of each register is written (later chunks overwrite
// earlier ones, so the row ends as the block's last definitions).
constexpr int kDefWarps = 4;
__global__ void __launch_bounds__(32 * kDefWarps, 16)
    k_local_defs(const __grid_constant__ Batch b, uint32_t* __restrict__ defbits, const uint32_t* __restrict__ bits_off,
                 const uint32_t* __restrict__ blk_kern) {
  __shared__ uint32_t s_reg[kDefWarps][32][4], s_mask[kDefWarps][kDefBuckets];
  const uint32_t wp = threadIdx.x / 32, lane = threadIdx.x & 31u;
  const uint32_t g = blockIdx.x * kDefWarps + wp;
  if (g >= b.NLB) return;
  const uint32_t k = blk_kern[g];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const uint32_t bl = g - K.first_lblock;
  const BlockRec& B = b.lblocks[g];
  const RegMap M{K.vgprs, K.sgprs};
  const uint32_t words = (K.R + 31) / 32;
  uint32_t* db = defbits + bits_off[k] + (size_t)bl * words;
  uint32_t* out = b.st_out + K.state_off + (size_t)bl * K.R;
  for (uint32_t first = B.first; first < B.end; first += 32) {
    const uint32_t i = first + lane;
    Def d[4];
    const int n = (i < B.end && b.lblock_of[K.first_instr + i] == bl) ? idefs(b, K, M, i, d) : 0;
    for (int t = 0; t < 4; ++t) s_reg[wp][lane][t] = t < n ? d[t].reg : kNone;
    for (uint32_t q = lane; q < kDefBuckets; q += 32) s_mask[wp][q] = 0;
    __syncwarp();
    // (loops of constant trip count over d, so that it stays in registers)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < n) atomicOr(&s_mask[wp][d[t].reg % kDefBuckets], 1u << lane);
    __syncwarp();
    const uint32_t above = ~((2u << lane) - 1u);  // lanes after this one
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= n) continue;
      const uint32_t reg = d[t].reg;
      atomicOr(&db[reg >> 5], 1u << (reg & 31));
      bool last = true;
#pragma unroll
      for (int u = t + 1; u < 4; ++u) last = last && (u >= n || d[u].reg != reg);
      int u;
      if (last && last_def(s_reg[wp], s_mask[wp], reg, above, &u) < 0) out[reg] = d[t].val;
    }
    __syncwarp();
  }
}

__device__ __forceinline__ uint32_t entry_value(const KHdr& K, uint32_t r) {
  if (r < K.vgprs) {
    if (r < K.dims && r < 3) return leafref(LEAF_LID, r, PART_ENTIRE);
    return kUndef;
  }
  if (r < K.vgprs + K.sgprs) {
    uint32_t s = r - K.vgprs;
    if (K.useargs && s >= 6 && s < 6 + K.dims && s < 9) return leafref(LEAF_GRP, s - 6, PART_ENTIRE);
    if (K.sgprs > 5 && s == 4) return leafref(LEAF_KARG, 0, PART_LO);
    if (K.sgprs > 5 && s == 5) return leafref(LEAF_KARG, 0, PART_HI);
    if (K.sgprs > 1 && s == 0) return leafref(LEAF_DISP, 0, PART_LO);  // the dispatch packet pointer
    if (K.sgprs > 1 && s == 1) return leafref(LEAF_DISP, 0, PART_HI);
  }
  return kUndef;
}

// ---------------------------------------------------------------------------
// versions: frontier closure (a team per kernel, threads over join blocks),
// then values in reverse postorder (threads over registers)
// ---------------------------------------------------------------------------
// a word another thread of the team may be writing (read afresh every time)
__device__ __forceinline__ uint32_t volatile_ld(const uint32_t* p) { return *(const volatile uint32_t*)p; }

template <bool WARP>
__global__ void __launch_bounds__(WARP ? 128 : kBigTeam)
    k_versions(const __grid_constant__ Batch b, uint32_t* __restrict__ defbits, uint32_t* __restrict__ phibits,
               const uint32_t* __restrict__ bits_off, uint32_t* __restrict__ err) {
  using T = Team<WARP>;
  const uint32_t k = T::kid(), tid = T::tid(), TS = T::size();
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad || !K.n_lblock || !T::mine(K, b.big_kernel)) return;
  uint32_t nb = K.n_lblock, base = K.first_lblock, R = K.R, words = (R + 31) / 32;
  uint32_t* db = defbits + bits_off[k];
  uint32_t* pb = phibits + bits_off[k];
  const uint32_t* idom = b.idom + base;
  // the entry defines every register
  for (uint32_t w = tid; w < words; w += TS) db[w] = 0xFFFFFFFFu;
  T::sync();
  // Join versions: the iterated dominance frontier of the defining blocks.  Each
  // thread takes join blocks x and adds, along the dominator-tree path from each
  // predecessor up to idom(x), the definitions and versions found there; sweeps
  // repeat until nothing changes (a monotone closure: the order does not matter).
  bool changed = true;
  uint32_t sweeps = 0;
  while (changed) {
    changed = false;
    if (++sweeps > 4 * nb + 8) {  // cannot happen for a closure; bounded all the same
      if (tid == 0) atomicOr(err, ERR_CAPACITY);
      break;
    }
    for (uint32_t x = tid; x < nb; x += TS) {
      uint32_t np = b.pred_off[base + x + 1] - b.pred_off[base + x];
      if (np < 2 || idom[x] == kNone) continue;
      for (uint32_t pi = b.pred_off[base + x]; pi < b.pred_off[base + x + 1]; ++pi) {
        uint32_t r = b.preds[pi];
        if (idom[r] == kNone) continue;  // unreachable predecessor
        while (r != idom[x]) {
          for (uint32_t w = 0; w < words; ++w) {
            const uint32_t add =
                (db[(size_t)r * words + w] | volatile_ld(&pb[(size_t)r * words + w])) & ~pb[(size_t)x * words + w];
            if (add) {
              pb[(size_t)x * words + w] |= add;
              changed = true;
            }
          }
          r = idom[r];
        }
      }
    }
    T::sync();
    changed = T::any(changed);
  }
  T::sync();
  // values, block by block in reverse postorder, threads over registers
  uint32_t* in = b.st_in + K.state_off;
  uint32_t* out = b.st_out + K.state_off;
  uint8_t* hp = b.has_phi + K.state_off;
  for (uint32_t q = 0; q < nb; ++q) {
    uint32_t x = b.rpo[base + q];
    if (x == kNone) break;
    for (uint32_t r = tid; r < R; r += TS) {
      bool phi = (pb[(size_t)x * words + (r >> 5)] >> (r & 31)) & 1u;
      hp[(size_t)x * R + r] = phi;
      uint32_t v = phi ? phiref(x, r) : (x == 0 ? entry_value(K, r) : out[(size_t)idom[x] * R + r]);
      in[(size_t)x * R + r] = v;
      uint32_t o = out[(size_t)x * R + r];
      if (o == kTop) out[(size_t)x * R + r] = v;
    }
    T::sync();
  }
}

// ---------------------------------------------------------------------------
// nodes: one warp per block
// ---------------------------------------------------------------------------
struct NodeCtx {
  const Batch* b;
  const KHdr* K;
  RegMap M;
  uint32_t i;
  const uint32_t* row;  // register values at the start of the current chunk of the block
  // definitions of the chunk's instructions (lane m: instruction first + m), kNone when absent
  const uint32_t (*dreg)[4];
  const uint32_t (*dval)[4];
  const uint32_t* dmask;  // per register bucket (reg % kDefBuckets): the lanes defining such a register
  uint32_t lane;  // this instruction's place in the chunk
};

// value of register reg just before instruction c.i: the last definition of
// an earlier instruction of the chunk, else the value at the chunk's start
__device__ __forceinline__ uint32_t reg_now(const NodeCtx& c, uint32_t reg) {
  int t;
  const int m = last_def(c.dreg, c.dmask, reg, (1u << c.lane) - 1u, &t);
  const uint32_t v = m >= 0 ? c.dval[m][t] : c.row[reg];
  return v == kTop ? kUndef : v;
}

__device__ __forceinline__ uint32_t src32(const NodeCtx& c, Node* nodes, const InstrRec& r, uint32_t o,
                                          uint32_t slot) {
  uint32_t tg = otag(o);
  if (tg == TG_VGPR) return reg_now(c, c.M.v(opay(o)));
  if (tg == TG_SGPR) return reg_now(c, c.M.s(opay(o)));
  if (tg == TG_VCC) return reg_now(c, c.M.vcc());
  Node& n = nodes[slot];
  n.kind = N_CONST;
  if (tg == TG_ICONST) {
    uint32_t p = opay(o);
    n.cval = (p & 0x800000u) ? (p | 0xFF000000u) : p;
  } else if (tg == TG_FCONST) {
    const uint32_t fb[8] = {0x3f000000u, 0xbf000000u, 0x3f800000u, 0xbf800000u,
                            0x40000000u, 0xc0000000u, 0x40800000u, 0xc0800000u};
    n.cval = fb[opay(o) & 7];
  } else {
    n.cval = r.imm;
  }
  return mkref(4 * c.i + slot, PART_ENTIRE);
}

__device__ __forceinline__ uint32_t make_pair(const NodeCtx& c, Node* nodes, uint32_t lo, uint32_t hi,
                                              uint32_t slot) {
  if ((r_node(lo) || r_leaf(lo)) && rpart(lo) == PART_LO && hi == ((lo & ~3u) | PART_HI)) return lo & ~3u;
  Node& p = nodes[slot];
  p.kind = N_PAIR;
  p.nsrc = 2;
  p.src[0] = lo;
  p.src[1] = hi;
  return mkref(4 * c.i + slot, PART_ENTIRE);
}

__device__ __forceinline__ uint32_t src64(const NodeCtx& c, Node* nodes, uint32_t o, uint32_t slot) {
  uint32_t a = reg_now(c, reg_of(c.M, o, 0)), h = reg_now(c, reg_of(c.M, o, 1));
  return make_pair(c, nodes, a, h, slot);
}

// nodes of instruction c.i (kernel-relative); `knodes` = the kernel's nodes
__device__ __forceinline__ void build_instr_nodes(const Batch& b, const KHdr& K, NodeCtx& c, Node* knodes) {
  uint32_t gi = K.first_instr + c.i;
  Node* nodes = knodes + 4 * (size_t)c.i;
  const InstrRec& r = b.ins[gi];
  uint8_t ctl = b.ctl[gi];
  Node& nd = nodes[0];
  if (ctl != C_NORMAL && ctl != C_CBR) return;
  nd.kind = N_OP;
  nd.op = r.op;
  if (ctl == C_CBR) {
    nd.nsrc = 1;
    nd.src[0] = reg_now(c, r.op == O_S_AND_SAVEEXEC ? c.M.vcc() : c.M.scc());
    return;
  }
  uint32_t s[3];
  int ns = 0;
  switch (r.op) {
    case O_S_WAITCNT: break;
    case O_S_LOAD_DWORD: case O_S_LOAD_DWORDX2: case O_S_LOAD_DWORDX4:
      s[ns++] = src64(c, nodes, r.opnd[1], 2);
      nd.cval = r.imm;
      break;
    case O_BUFFER_STORE_DWORD: s[ns++] = src32(c, nodes, r, r.opnd[0], 1); break;
    case O_BUFFER_LOAD_DWORD: s[ns++] = reg_now(c, c.M.spill(r.imm / 4)); break;
    case O_V_ADDC_CO_U32: case O_V_SUBB_CO_U32: {
      const bool f = b.fused[gi] != 0;  // fused: a constant high source sits in slot 3
      uint32_t a = src32(c, nodes, r, r.opnd[2], f ? 3 : 1), bb = src32(c, nodes, r, r.opnd[3], f ? 3 : 2);
      if (f) {
        // the low half's sources, as its node (built earlier in this walk) holds them
        const Node& lo = knodes[4 * (size_t)b.co_idx[gi]];
        s[ns++] = make_pair(c, nodes, lo.src[0], a, 1);
        s[ns++] = make_pair(c, nodes, lo.src[1], bb, 2);
        nd.fused = 1;
      } else {
        s[ns++] = a;
        s[ns++] = bb;
        s[ns++] = reg_now(c, c.M.vcc());
      }
      break;
    }
    case O_UNKNOWN:
      for (int q = 1; q < r.nops && ns < 3; ++q) {
        uint32_t o = r.opnd[q], tg = otag(o);
        if (tg == TG_VGPR || tg == TG_SGPR || tg == TG_VCC) {
          uint32_t cnt = tg == TG_VCC ? 1 : ocnt(o);
          if (cnt == 2) s[ns] = src64(c, nodes, o, 1 + ns);
          else s[ns] = reg_now(c, reg_of(c.M, o, 0));
          ++ns;
        }
      }
      break;
    default: {
      const char* sig = c_sig[r.op];
      int nop = sig_count(r.op);
      for (int q = 0; q < nop && ns < 3; ++q) {
        char sc = sig[2 * q];
        bool dst = (q == 0 && (sc == 'V' || sc == 'W' || sc == 's' || sc == 'p' || sc == 'q' || sc == 'c')) ||
                   (q == 1 && sc == 'c' && (r.op == O_V_ADD_CO_U32 || r.op == O_V_SUB_CO_U32));
        if (op_store(r.op) || scmp(r.op)) dst = false;
        if (dst || sc == 'o') continue;
        uint32_t slot = 1 + ns;
        if (sc == 'W' || sc == 'p') s[ns] = src64(c, nodes, r.opnd[q], slot);
        else s[ns] = src32(c, nodes, r, r.opnd[q], slot);
        ++ns;
      }
    }
  }
  nd.nsrc = (uint8_t)ns;
  for (int q = 0; q < ns; ++q) nd.src[q] = s[q];
  if (r.op == O_S_LOAD_DWORDX4) {
    Node& h2 = nodes[1];
    h2.kind = N_SLOAD64B;
    h2.nsrc = 1;
    h2.src[0] = nd.src[0];
    h2.cval = r.imm + 8;
  }
  if (r.op == O_V_ADD_CO_U32 || r.op == O_V_SUB_CO_U32) nodes[3].kind = N_CARRY;
}

// every node slot to "no node" (instruction i's four 24-byte slots as six 16-byte stores)
__global__ void k_clear_nodes(const __grid_constant__ Batch b) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;  // 16-byte word
  if (g >= 6ull * b.I) return;
  // a cleared Node: kind, nsrc, fused, pad, op, pad2 = 0; src[3] = kTop; cval = 0
  const uint32_t w = (uint32_t)(g % 6);  // word w of an instruction's 96 bytes: bytes 16w..16w+15
  uint32_t q[4];
  for (int e = 0; e < 4; ++e) {
    const uint32_t byte = 16 * w + 4 * e, off = byte % 24;  // offset inside its Node
    q[e] = (off >= 8 && off < 20) ? kTop : 0u;
  }
  reinterpret_cast<uint4*>(b.nodes)[g] = make_uint4(q[0], q[1], q[2], q[3]);
}

// One warp per logical block.  The warp copies the block's in-state into a
// working row, then takes the block's instructions 32 at a time: every lane
// lists its instruction's definitions in shared memory, builds its nodes
// (a source register takes the last definition of an earlier lane, else the
// row), and the chunk's last definition of each register goes into the row.
// Carry halves fused with a low half of the same chunk are built after the
// other nodes, as they read the low half's node.
constexpr int kNodeWarps = 4;
__global__ void __launch_bounds__(32 * kNodeWarps, 16)
    k_nodes(const __grid_constant__ Batch b, uint32_t* __restrict__ rows, const uint32_t* __restrict__ blk_kern) {
  __shared__ uint32_t s_reg[kNodeWarps][32][4], s_val[kNodeWarps][32][4], s_mask[kNodeWarps][kDefBuckets];
  const uint32_t wp = threadIdx.x / 32, lane = threadIdx.x & 31u;
  const uint32_t g = blockIdx.x * kNodeWarps + wp;
  if (g >= b.NLB) return;
  const uint32_t k = blk_kern[g];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const uint32_t bl = g - K.first_lblock;
  const BlockRec& B = b.lblocks[g];
  uint32_t* row = rows + K.state_off + (size_t)bl * K.R;
  const uint32_t* in = b.st_in + K.state_off + (size_t)bl * K.R;
  for (uint32_t r = lane; r < K.R; r += 32) row[r] = in[r];
  __syncwarp();
  NodeCtx c;
  c.b = &b;
  c.K = &K;
  c.M = RegMap{K.vgprs, K.sgprs};
  c.row = row;
  c.dreg = s_reg[wp];
  c.dval = s_val[wp];
  c.dmask = s_mask[wp];
  c.lane = lane;
  Node* knodes = b.nodes + 4 * (size_t)K.first_instr;
  for (uint32_t first = B.first; first < B.end; first += 32) {
    const uint32_t i = first + lane;
    const bool mine = i < B.end && b.lblock_of[K.first_instr + i] == bl;
    Def d[4];
    const int n = mine ? idefs(b, K, c.M, i, d) : 0;
    for (int t = 0; t < 4; ++t) {
      s_reg[wp][lane][t] = t < n ? d[t].reg : kNone;
      s_val[wp][lane][t] = t < n ? d[t].val : kNone;
    }
    for (uint32_t q = lane; q < kDefBuckets; q += 32) s_mask[wp][q] = 0;
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < n) atomicOr(&s_mask[wp][d[t].reg % kDefBuckets], 1u << lane);
    __syncwarp();
    c.i = i;
    const uint32_t gi = K.first_instr + i;
    const bool late = mine && b.fused[gi];  // fused carry half
    // two trips, one call site (in line: the context stays in registers): the other nodes, then the
    // fused carry halves, which read their low half's node
    for (int trip = 0; trip < 2; ++trip) {
      if (mine && late == (trip == 1)) build_instr_nodes(b, K, c, knodes);
      if (trip == 0) __syncwarp();
    }
    // the row after the chunk: a register takes the chunk's last definition of it
    const uint32_t above = ~((2u << lane) - 1u);  // lanes after this one
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= n) continue;
      const uint32_t reg = d[t].reg;
      bool last = true;
#pragma unroll
      for (int u = t + 1; u < 4; ++u) last = last && (u >= n || d[u].reg != reg);
      int u;
      if (last && last_def(s_reg[wp], s_mask[wp], reg, above, &u) < 0) row[reg] = d[t].val;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
__global__ void k_bits_size(const __grid_constant__ Batch b, uint32_t* __restrict__ kbits) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  const KHdr& K = b.kh[k];
  kbits[k] = K.bad ? 0u : K.n_lblock * ((K.R + 31) / 32);
}

void launch_df_counts(Batch& b, DfScratch& d, ScanScratch sc, uint32_t* totals, cudaStream_t s) {
  const int T = 256;
  if (!b.K) return;
  if (b.I) {
    k_df_spill<<<(b.I + T - 1) / T, T, 0, s>>>(b);
    ++launch_counter();
  }
  if (b.NLB) {
    k_df_entry<<<(b.NLB + T - 1) / T, T, 0, s>>>(b, d.blk_kern);
    ++launch_counter();
  }
  k_df_sizes<<<(b.K + 127) / 128, 128, 0, s>>>(b, d.kstate);
  ++launch_counter();
  k_bits_size<<<(b.K + 127) / 128, 128, 0, s>>>(b, d.kbits);
  ++launch_counter();
  launch_scan(d.kstate, d.kstate_off, b.K, 0, false, sc, &totals[5], b.err, s);  // totals[5] = state words
  launch_scan(d.kbits, d.bits_off, b.K, 0, false, sc, &totals[6], b.err, s);     // totals[6] = bitset words
  if (b.I) {
    k_fusion<<<(b.I + T - 1) / T, T, 0, s>>>(b);
    ++launch_counter();
  }
  if (b.NLB) {
    cudaMemsetAsync(d.pcount, 0, sizeof(uint32_t) * (b.NLB + 1), s);
    k_pred_count<<<(b.NLB + T - 1) / T, T, 0, s>>>(b, d.pcount, d.blk_kern);
    ++launch_counter();
    launch_scan(d.pcount, b.pred_off, b.NLB + 1, 0, false, sc, &totals[7], b.err, s);  // totals[7] = edges
  }
}

void launch_df_main(Batch& b, DfScratch& d, cudaStream_t s) {
  const int T = 256;
  if (!b.K) return;
  k_state_off<<<(b.K + 127) / 128, 128, 0, s>>>(b, d.kstate_off);
  ++launch_counter();
  if (b.NLB) {
    cudaMemsetAsync(b.pred_fill, 0, sizeof(uint32_t) * b.NLB, s);
    k_pred_fill<<<(b.NLB + T - 1) / T, T, 0, s>>>(b, d.blk_kern);
    ++launch_counter();
    k_pred_sort<<<(b.NLB + T - 1) / T, T, 0, s>>>(b);
    ++launch_counter();
    k_dominators<<<walk_blocks(b.K), walk_threads(b.K), 0, s>>>(b, d.rpo_index, d.stack, d.child);
    ++launch_counter();
  }
  if (b.NS) cudaMemsetAsync(b.st_out, 0xFF, sizeof(uint32_t) * b.NS, s);
  if (d.NW) {
    cudaMemsetAsync(d.defbits, 0, sizeof(uint32_t) * d.NW, s);
    cudaMemsetAsync(d.phibits, 0, sizeof(uint32_t) * d.NW, s);
  }
  if (b.NLB) {
    k_local_defs<<<(b.NLB + kDefWarps - 1) / kDefWarps, 32 * kDefWarps, 0, s>>>(b, d.defbits, d.bits_off, d.blk_kern);
    ++launch_counter();
  }
  k_versions<true><<<(b.K + 3) / 4, 128, 0, s>>>(b, d.defbits, d.phibits, d.bits_off, b.err);
  k_versions<false><<<b.K, kBigTeam, 0, s>>>(b, d.defbits, d.phibits, d.bits_off, b.err);
  launch_counter() += 2;
  if (b.I) {
    const uint64_t nw = 6ull * b.I;
    k_clear_nodes<<<(uint32_t)((nw + T - 1) / T), T, 0, s>>>(b);
    ++launch_counter();
  }
  if (b.NLB) {
    ktime(KT_NODES, 0, s);
    k_nodes<<<(b.NLB + kNodeWarps - 1) / kNodeWarps, 32 * kNodeWarps, 0, s>>>(b, d.rows, d.blk_kern);
    ktime(KT_NODES, 1, s);
    ++launch_counter();
  }
}

}  // namespace gd
