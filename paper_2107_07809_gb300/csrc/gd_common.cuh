// gd_common.cuh — records, constants and device helpers of the CUDA decompiler.
//
// Layouts here are the frozen contract of the intermediate arrays (instruction
// records, block tables, configuration header) that parity tests compare
// byte for byte with the CPU oracle; the oracle defines the same layouts in
// its own code.  Everything else is private to the CUDA path.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gd {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kMaxArgs = 32;        // .arg rows per kernel
constexpr int kMaxExecDepth = 64;   // nested exec-mask forms per kernel
constexpr uint32_t kMaxRegs = 1024; // tracked registers per kernel (join ids use 10 bits)
constexpr uint32_t kMaxBlocks = 1u << 18;
// regions per logical block: every merge makes one region; merges that do not
// shrink the graph are the self-loop ones (at most one per block), so a kernel
// of n blocks ends with fewer than 3n regions
constexpr uint32_t kRegionsPerBlock = 3;
// stack words per logical block: the reduction's search (< 2 pushes per live
// region) and the printer's frames (2 words, at most 2 per level of a tree of
// fewer than 3n regions)
constexpr uint32_t kStackPerBlock = 12;

// ---- error bits (kernel-wide `err` word) ----------------------------------------
enum : uint32_t { ERR_LOOKBACK = 1, ERR_MBAR = 2, ERR_CAPACITY = 4, ERR_STACK = 8 };

// ---- per-kernel status -------------------------------------------------------------
enum : uint32_t { ST_OK = 0, ST_PARTIAL = 1, ST_PARSE_ERROR = 2, ST_FIXPOINT_CAP = 3 };

// ---- value types ---------------------------------------------------------------------
enum : uint8_t { TY_NONE = 0, TY_INT = 1, TY_UINT = 2, TY_FLOAT = 3, TY_LONG = 4, TY_ULONG = 5, TY_DOUBLE = 6,
                 TY_TOP32 = 7, TY_TOP64 = 8 };

// ---- opcodes (numbering of the dialect table) ------------------------------------
enum : uint16_t {
  O_UNKNOWN = 0, O_S_LOAD_DWORD = 1, O_S_LOAD_DWORDX2 = 2, O_S_LOAD_DWORDX4 = 3, O_S_WAITCNT = 4,
  O_S_MOV_B32 = 5, O_S_MUL_I32 = 6, O_S_LSHL_B32 = 7, O_S_ADD_U32 = 8, O_S_CMP0 = 9,
  O_S_AND_SAVEEXEC = 21, O_S_XOR_B64 = 22, O_S_OR_B64 = 23, O_S_OR_SAVEEXEC = 24, O_S_BRANCH = 25,
  O_S_CBRANCH_SCC0 = 26, O_S_CBRANCH_SCC1 = 27, O_S_CBRANCH_EXECZ = 28, O_S_ENDPGM = 29,
  O_V_MOV_B32 = 30, O_V_ADD_U32 = 31, O_V_SUB_U32 = 32, O_V_MUL_LO_U32 = 33, O_V_MAD_U32_U24 = 34,
  O_V_MUL_U32_U24 = 35, O_V_AND_B32 = 36, O_V_OR_B32 = 37, O_V_XOR_B32 = 38, O_V_LSHLREV_B32 = 39,
  O_V_LSHRREV_B32 = 40, O_V_ASHRREV_I32 = 41, O_V_ADD_F32 = 42, O_V_SUB_F32 = 43, O_V_MUL_F32 = 44,
  O_V_FMA_F32 = 45, O_V_CVT_F32_I32 = 46, O_V_CVT_F32_U32 = 47, O_V_CVT_F64_F32 = 48, O_V_CVT_F64_I32 = 49,
  O_V_CVT_F32_F64 = 50, O_V_CMP0 = 51, O_V_ADD_CO_U32 = 69, O_V_ADDC_CO_U32 = 70, O_V_SUB_CO_U32 = 71,
  O_V_SUBB_CO_U32 = 72, O_V_LSHLREV_B64 = 73, O_V_ADD_F64 = 74, O_V_MUL_F64 = 75, O_V_FMA_F64 = 76,
  O_GLOBAL_LOAD_DWORD = 77, O_GLOBAL_LOAD_DWORDX2 = 78, O_GLOBAL_STORE_DWORD = 79, O_GLOBAL_STORE_DWORDX2 = 80,
  O_BUFFER_LOAD_DWORD = 81, O_BUFFER_STORE_DWORD = 82,
  O_V_CNDMASK_B32 = 83,  // the ternary ("Search for control structures"): vD = vcc ? src1 : src0
  O_S_LSHR_B32 = 84, O_S_BFE_U32 = 85,  // scalar shift right, bit-field extract (get_num_groups, get_work_dim)
  // FLAT memory instructions ("The body extraction": prefix flat, a VGPR pair holds the address)
  // and the double-suffix high multiplies (result type, then operand type)
  O_FLAT_LOAD_DWORD = 86, O_FLAT_LOAD_DWORDX2 = 87, O_FLAT_STORE_DWORD = 88, O_FLAT_STORE_DWORDX2 = 89,
  O_V_MUL_HI_U32_U24 = 90, O_V_MUL_HI_I32_I24 = 91,
  // data share operations on the LDS (OpenCL local memory; prefix ds) and the work-group barrier
  O_DS_READ_B32 = 92, O_DS_READ_B64 = 93, O_DS_WRITE_B32 = 94, O_DS_WRITE_B64 = 95, O_S_BARRIER = 96,
  O_COUNT = 97
};

// ---- operand word: tag<<28 | count<<24 | payload -----------------------------------
enum : uint32_t { TG_NONE = 0, TG_VGPR = 1, TG_SGPR = 2, TG_VCC = 3, TG_EXEC = 4, TG_ICONST = 5, TG_FCONST = 6,
                  TG_LIT = 7, TG_LABEL = 8, TG_OFF = 9 };
__host__ __device__ __forceinline__ uint32_t opw(uint32_t tag, uint32_t cnt, uint32_t pay) {
  return (tag << 28) | ((cnt & 15u) << 24) | (pay & 0xFFFFFFu);
}
__host__ __device__ __forceinline__ uint32_t otag(uint32_t o) { return o >> 28; }
__host__ __device__ __forceinline__ uint32_t ocnt(uint32_t o) { return (o >> 24) & 15u; }
__host__ __device__ __forceinline__ uint32_t opay(uint32_t o) { return o & 0xFFFFFFu; }

enum : uint8_t { FL_UNSUPPORTED = 1, FL_BAD = 2, FL_REGRANGE = 4, FL_NOLABEL = 8 };

// operand signature of every opcode: V vgpr, W vgpr pair, s sgpr, p sgpr pair,
// q sgpr quad, S 32-bit source, M 64-bit mask, c vcc, o off, K constant, L label, * free
// (global memory, not the constant bank: lanes read the signatures of different opcodes)
static __device__ char c_sig[O_COUNT][12] = {
    "?", "s,p,K", "p,p,K", "q,p,K", "*", "s,S", "s,S,S", "s,S,S", "s,S,S",
    "S,S", "S,S", "S,S", "S,S", "S,S", "S,S", "S,S", "S,S", "S,S", "S,S", "S,S", "S,S",
    "M,M", "M,M,M", "M,M,M", "M,M", "L", "L", "L", "L", "",
    "V,S", "V,S,S", "V,S,S", "V,S,S", "V,S,S,S", "V,S,S", "V,S,S", "V,S,S", "V,S,S", "V,S,S", "V,S,S",
    "V,S,S", "V,S,S", "V,S,S", "V,S,S", "V,S,S,S", "V,S", "V,S", "W,S", "W,S", "V,W",
    "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S",
    "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S", "c,S,S",
    "V,c,S,S", "V,c,S,S,c", "V,c,S,S", "V,c,S,S,c", "W,S,W", "W,W,W", "W,W,W", "W,W,W,W",
    "V,W,o", "W,W,o", "W,V,o", "W,W,o", "V,o,q,s", "V,o,q,s", "V,S,S,c", "s,S,S", "s,S,S",
    "V,W", "W,W", "W,V", "W,W", "V,S,S", "V,S,S", "V,V", "W,V", "V,V", "V,W", ""};
__device__ __forceinline__ int sig_count(uint16_t op) {
  const char* s = c_sig[op];
  int n = 0;
  while (s[n]) ++n;
  return n ? (n + 1) / 2 : 0;
}

struct __align__(4) InstrRec {
  uint16_t op;
  uint8_t nops;
  uint8_t flags;
  uint32_t imm;
  uint32_t target;
  uint32_t opnd[5];
};
static_assert(sizeof(InstrRec) == 32, "InstrRec is 32 bytes");

// Memory accesses: global and FLAT accesses are the same access in this dialect (a FLAT address
// is always formed from a __global buffer argument); the LDS accesses (ds_) are loads and stores
// of a __local buffer, with their own address match.
__host__ __device__ __forceinline__ bool op_lds(uint16_t op) { return op >= O_DS_READ_B32 && op <= O_DS_WRITE_B64; }
__host__ __device__ __forceinline__ bool op_store(uint16_t op) {
  return op == O_GLOBAL_STORE_DWORD || op == O_GLOBAL_STORE_DWORDX2 || op == O_FLAT_STORE_DWORD ||
         op == O_FLAT_STORE_DWORDX2 || op == O_DS_WRITE_B32 || op == O_DS_WRITE_B64;
}
__host__ __device__ __forceinline__ bool op_gload(uint16_t op) {
  return op == O_GLOBAL_LOAD_DWORD || op == O_GLOBAL_LOAD_DWORDX2 || op == O_FLAT_LOAD_DWORD ||
         op == O_FLAT_LOAD_DWORDX2 || op == O_DS_READ_B32 || op == O_DS_READ_B64;
}
// bytes one load or store moves
__host__ __device__ __forceinline__ uint32_t op_mem_width(uint16_t op) {
  return (op == O_GLOBAL_LOAD_DWORDX2 || op == O_GLOBAL_STORE_DWORDX2 || op == O_FLAT_LOAD_DWORDX2 ||
          op == O_FLAT_STORE_DWORDX2 || op == O_DS_READ_B64 || op == O_DS_WRITE_B64)
             ? 8u
             : 4u;
}

struct BlockRec {
  uint32_t first, end, succ0, succ1;
};

struct ArgRec {
  uint32_t name_off;  // byte offset in the batch text
  uint16_t name_len;
  uint8_t hidden, pointer, is_const, elem, space, gofs;  // gofs = 1 + d for _.global_offset_d
};

// per-kernel record
struct KHdr {
  uint32_t line;                  // the .kernel line
  uint32_t file;
  uint32_t name_off, name_len;
  uint32_t first_cfg, n_cfg;       // the kernel's configuration rows (into cfg_line)
  uint32_t first_instr, n_instr;
  uint32_t first_label, n_label;
  uint32_t first_pblock, n_pblock;
  uint32_t first_lblock, n_lblock;
  uint32_t dims, cws[3], sgprs, vgprs, useargs, nargs, nuser;
  uint32_t R, nspill;
  uint32_t entry_target;          // some block branches to the entry block
  uint32_t state_off;             // into block x register arrays
  uint32_t region_off;            // into region arrays (2 per block)
  uint32_t wl_off;                // into the reachability worklist
  uint32_t status;                // ST_*
  uint32_t bad;                   // parse/config failure
  uint32_t partial;
  uint32_t n_vars;
  uint32_t n_phis;                // used join versions (listed by the reachability walk)
  uint32_t out_len;
  uint32_t root;                  // root region (kernel-relative) or kNone
  uint32_t capped;                // the type fixed point hit its sweep limit (status FIXPOINT_CAP)
};

// ---- control kinds of the logical CFG ------------------------------------------------
enum : uint8_t { C_NORMAL = 0, C_DROP = 1, C_CBR = 2, C_JMP = 3, C_END = 4 };

// ---- expression nodes --------------------------------------------------------------
enum : uint8_t { N_NONE = 0, N_OP = 1, N_CONST = 2, N_PAIR = 3, N_CARRY = 4, N_SLOAD64B = 5 };
struct Node {
  uint8_t kind;
  uint8_t nsrc;
  uint8_t fused;
  uint8_t pad;
  uint16_t op;
  uint16_t pad2;
  uint32_t src[3];
  uint32_t cval;
};
static_assert(sizeof(Node) == 24, "Node is 24 bytes");

// value references: id << 2 | part; ids: node = 4*instr+slot, join = 1<<28 | block<<10 | reg,
// ABI leaf = 2<<28 | kind<<8 | k
enum : uint32_t { PART_ENTIRE = 0, PART_LO = 1, PART_HI = 2 };
constexpr uint32_t kTop = 0xFFFFFFFFu;
constexpr uint32_t kIdPhi = 1u << 28, kIdLeaf = 2u << 28;
constexpr uint32_t LEAF_UNDEF = 0, LEAF_LID = 1, LEAF_GRP = 2, LEAF_KARG = 3, LEAF_DISP = 4;
constexpr uint32_t kUndef = kIdLeaf << 2;
__host__ __device__ __forceinline__ uint32_t mkref(uint32_t id, uint32_t part) { return (id << 2) | part; }
__host__ __device__ __forceinline__ uint32_t rid(uint32_t r) { return r >> 2; }
__host__ __device__ __forceinline__ uint32_t rpart(uint32_t r) { return r & 3u; }
__host__ __device__ __forceinline__ bool r_node(uint32_t r) { return r != kTop && (rid(r) >> 28) == 0; }
__host__ __device__ __forceinline__ bool r_phi(uint32_t r) { return r != kTop && (rid(r) >> 28) == 1; }
__host__ __device__ __forceinline__ bool r_leaf(uint32_t r) { return r != kTop && (rid(r) >> 28) == 2; }
__host__ __device__ __forceinline__ uint32_t phiref(uint32_t b, uint32_t reg) {
  return mkref(kIdPhi | (b << 10) | reg, PART_ENTIRE);
}
__host__ __device__ __forceinline__ uint32_t leafref(uint32_t kind, uint32_t k, uint32_t part) {
  return mkref(kIdLeaf | (kind << 8) | k, part);
}

// ---- small device helpers --------------------------------------------------------------
__device__ __forceinline__ bool is_space(uint8_t c) { return c == ' ' || c == '\t' || c == '\r'; }

// parse an integer token [p, e): decimal (optional '-') or 0x hex, value < 2^32
__device__ __forceinline__ bool dparse_int(const uint8_t* p, const uint8_t* e, int64_t* out, bool* hex) {
  *hex = false;
  if (p >= e) return false;
  bool neg = false;
  if (*p == '-') { neg = true; ++p; }
  if (p >= e) return false;
  uint64_t x = 0;
  if (e - p > 2 && p[0] == '0' && (p[1] == 'x' || p[1] == 'X')) {
    *hex = true;
    p += 2;
    for (; p < e; ++p) {
      uint8_t c = *p;
      uint32_t d;
      if (c >= '0' && c <= '9') d = c - '0';
      else if (c >= 'a' && c <= 'f') d = c - 'a' + 10;
      else if (c >= 'A' && c <= 'F') d = c - 'A' + 10;
      else return false;
      x = x * 16 + d;
      if (x > 0xFFFFFFFFull) return false;
    }
  } else {
    for (; p < e; ++p) {
      uint8_t c = *p;
      if (c < '0' || c > '9') return false;
      x = x * 10 + (c - '0');
      if (x > 0xFFFFFFFFull) return false;
    }
  }
  *out = neg ? -(int64_t)x : (int64_t)x;
  return true;
}

__device__ __forceinline__ bool tok_eq(const uint8_t* p, const uint8_t* e, const char* s) {
  while (p < e && *s) {
    if (*p != (uint8_t)*s) return false;
    ++p;
    ++s;
  }
  return p == e && *s == 0;
}

__host__ __device__ __forceinline__ uint32_t fnv1a(const uint8_t* p, uint32_t n) {
  uint32_t h = 2166136261u;
  for (uint32_t i = 0; i < n; ++i) h = (h ^ p[i]) * 16777619u;
  return h;
}

// ---- single-pass scan with decoupled look-back --------------------------------------
// status word per tile: flag (1 = aggregate, 2 = inclusive prefix) << 32 | value.
// Tiles take ids from an atomic counter, so a tile only waits for tiles that
// started earlier; every wait is bounded and reports ERR_LOOKBACK instead of
// hanging.
struct ScanSum {
  __device__ __forceinline__ static uint32_t op(uint32_t a, uint32_t b) { return a + b; }
  static constexpr uint32_t id = 0;
};
struct ScanMax {
  __device__ __forceinline__ static uint32_t op(uint32_t a, uint32_t b) { return a > b ? a : b; }
  static constexpr uint32_t id = 0;
};

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// exclusive prefix (under Op) of everything before tile `tile`, computed by warp 0.
// `agg` is this tile's aggregate; publishes it first, then the inclusive value.
template <class Op>
__device__ uint32_t lookback(uint64_t* status, uint32_t tile, uint32_t agg, uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31u;
  if (tile == 0) {
    if (lane == 0) st_release_u64(&status[0], (2ull << 32) | agg);
    return Op::id;
  }
  if (lane == 0) st_release_u64(&status[tile], (1ull << 32) | agg);
  uint32_t prefix = Op::id;
  int64_t base = (int64_t)tile - 1;
  while (true) {
    int64_t idx = base - (int64_t)lane;
    uint64_t s = (2ull << 32) | Op::id;  // beyond tile 0: identity, already inclusive
    if (idx >= 0) {
      uint32_t spins = 0;
      s = ld_volatile_u64(&status[idx]);
      while ((s >> 32) == 0) {
        if (++spins > (1u << 22)) {
          atomicOr(err, ERR_LOOKBACK);
          s = (2ull << 32) | Op::id;
          break;
        }
        __nanosleep(20);
        s = ld_volatile_u64(&status[idx]);
      }
    }
    uint32_t flag = (uint32_t)(s >> 32), val = (uint32_t)s;
    unsigned incl_mask = __ballot_sync(0xFFFFFFFFu, flag == 2);
    int stop = incl_mask ? __ffs(incl_mask) - 1 : 32;  // nearest inclusive predecessor
    // reduce lanes [0, stop] (lane order = nearest first; the op is commutative)
    uint32_t v = (int)lane <= stop ? val : Op::id;
    for (int o = 16; o; o >>= 1) v = Op::op(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    prefix = Op::op(prefix, v);
    if (incl_mask) break;
    base -= 32;
  }
  if (lane == 0) st_release_u64(&status[tile], (2ull << 32) | Op::op(prefix, agg));
  return prefix;
}

// block-wide inclusive scan of one value per thread (blockDim.x multiple of 32, <= 1024)
template <class Op>
__device__ uint32_t block_incl_scan(uint32_t v, uint32_t* smem32, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if ((int)lane >= o) v = Op::op(v, t);
  }
  if (lane == 31) smem32[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? smem32[lane] : Op::id;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if ((int)lane >= o) w = Op::op(w, t);
    }
    if (lane < nw) smem32[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v = Op::op(smem32[warp - 1], v);
  *total = smem32[nw - 1];
  __syncthreads();
  return v;
}

}  // namespace gd
