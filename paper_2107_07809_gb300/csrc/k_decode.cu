// k_decode.cu — configuration, instruction decoding and control-flow graphs.
//
// S3 (configuration, Listings 1 and 3): a warp per kernel reads its .config
//    rows, one row per lane: dims, .cws, register counts, .useargs and the .arg
//    table (8-byte settings slots in declaration order; "_."-names are hidden).
// S4 (decoding, prefix_root_suffix names of "The body extraction"): one thread
//    per instruction row produces a fixed 32-byte record; mnemonics are found
//    through an FNV-1a hash table in global memory.
// S5 (CFG, "Search for control structures"): leaders by flags, block ids by a
//    device-wide scan, block table by one thread per block.
// S6 (logical CFG, Fig. 4/5): the exec-mask if / if-else forms are matched by
//    one thread per kernel with a bounded stack and rewritten into per-work-item
//    branches; logical leaders and blocks follow as for S5.
#include <cstring>

#include "gd_kernels.h"

namespace gd {

// ---------------------------------------------------------------------------
// mnemonic table (the dialect) and operand signatures
// ---------------------------------------------------------------------------
struct OpName {
  const char* n;
  const char* sig;
};
// signature letters: V vgpr, W vgpr pair, s sgpr, p sgpr pair, q sgpr quad,
// S 32-bit source, M 64-bit mask, c vcc, o off, K constant, L label, * free
static const OpName kOps[O_COUNT] = {
    {"", "?"}, {"s_load_dword", "s,p,K"}, {"s_load_dwordx2", "p,p,K"}, {"s_load_dwordx4", "q,p,K"},
    {"s_waitcnt", "*"}, {"s_mov_b32", "s,S"}, {"s_mul_i32", "s,S,S"}, {"s_lshl_b32", "s,S,S"},
    {"s_add_u32", "s,S,S"},
    {"s_cmp_eq_u32", "S,S"}, {"s_cmp_lg_u32", "S,S"}, {"s_cmp_gt_u32", "S,S"}, {"s_cmp_lt_u32", "S,S"},
    {"s_cmp_ge_u32", "S,S"}, {"s_cmp_le_u32", "S,S"}, {"s_cmp_eq_i32", "S,S"}, {"s_cmp_lg_i32", "S,S"},
    {"s_cmp_gt_i32", "S,S"}, {"s_cmp_lt_i32", "S,S"}, {"s_cmp_ge_i32", "S,S"}, {"s_cmp_le_i32", "S,S"},
    {"s_and_saveexec_b64", "M,M"}, {"s_xor_b64", "M,M,M"}, {"s_or_b64", "M,M,M"}, {"s_or_saveexec_b64", "M,M"},
    {"s_branch", "L"}, {"s_cbranch_scc0", "L"}, {"s_cbranch_scc1", "L"}, {"s_cbranch_execz", "L"},
    {"s_endpgm", ""}, {"v_mov_b32", "V,S"}, {"v_add_u32", "V,S,S"}, {"v_sub_u32", "V,S,S"},
    {"v_mul_lo_u32", "V,S,S"}, {"v_mad_u32_u24", "V,S,S,S"}, {"v_mul_u32_u24", "V,S,S"}, {"v_and_b32", "V,S,S"},
    {"v_or_b32", "V,S,S"}, {"v_xor_b32", "V,S,S"}, {"v_lshlrev_b32", "V,S,S"}, {"v_lshrrev_b32", "V,S,S"},
    {"v_ashrrev_i32", "V,S,S"}, {"v_add_f32", "V,S,S"}, {"v_sub_f32", "V,S,S"}, {"v_mul_f32", "V,S,S"},
    {"v_fma_f32", "V,S,S,S"}, {"v_cvt_f32_i32", "V,S"}, {"v_cvt_f32_u32", "V,S"}, {"v_cvt_f64_f32", "W,S"},
    {"v_cvt_f64_i32", "W,S"}, {"v_cvt_f32_f64", "V,W"},
    {"v_cmp_eq_i32", "c,S,S"}, {"v_cmp_ne_i32", "c,S,S"}, {"v_cmp_gt_i32", "c,S,S"}, {"v_cmp_lt_i32", "c,S,S"},
    {"v_cmp_ge_i32", "c,S,S"}, {"v_cmp_le_i32", "c,S,S"}, {"v_cmp_eq_u32", "c,S,S"}, {"v_cmp_ne_u32", "c,S,S"},
    {"v_cmp_gt_u32", "c,S,S"}, {"v_cmp_lt_u32", "c,S,S"}, {"v_cmp_ge_u32", "c,S,S"}, {"v_cmp_le_u32", "c,S,S"},
    {"v_cmp_eq_f32", "c,S,S"}, {"v_cmp_neq_f32", "c,S,S"}, {"v_cmp_gt_f32", "c,S,S"}, {"v_cmp_lt_f32", "c,S,S"},
    {"v_cmp_ge_f32", "c,S,S"}, {"v_cmp_le_f32", "c,S,S"},
    {"v_add_co_u32", "V,c,S,S"}, {"v_addc_co_u32", "V,c,S,S,c"}, {"v_sub_co_u32", "V,c,S,S"},
    {"v_subb_co_u32", "V,c,S,S,c"}, {"v_lshlrev_b64", "W,S,W"}, {"v_add_f64", "W,W,W"}, {"v_mul_f64", "W,W,W"},
    {"v_fma_f64", "W,W,W,W"}, {"global_load_dword", "V,W,o"}, {"global_load_dwordx2", "W,W,o"},
    {"global_store_dword", "W,V,o"}, {"global_store_dwordx2", "W,W,o"}, {"buffer_load_dword", "V,o,q,s"},
    {"buffer_store_dword", "V,o,q,s"}, {"v_cndmask_b32", "V,S,S,c"}, {"s_lshr_b32", "s,S,S"},
    {"s_bfe_u32", "s,S,S"},
    {"flat_load_dword", "V,W"}, {"flat_load_dwordx2", "W,W"}, {"flat_store_dword", "W,V"},
    {"flat_store_dwordx2", "W,W"}, {"v_mul_hi_u32_u24", "V,S,S"}, {"v_mul_hi_i32_i24", "V,S,S"},
    {"ds_read_b32", "V,V"}, {"ds_read_b64", "W,V"}, {"ds_write_b32", "V,V"}, {"ds_write_b64", "V,W"},
    {"s_barrier", ""},
};

constexpr int kHash = 512;
constexpr uint32_t kNameWords = 6;  // a mnemonic of at most 23 bytes, packed little-endian
struct DecodeTables {
  uint32_t namew[O_COUNT][kNameWords];  // the name's bytes, zero beyond its length
  uint8_t name_len[O_COUNT];
  uint16_t ht[kHash];  // hash slot -> op + 1 (0 = empty)
};
// in global memory, not the constant bank: lanes look up different mnemonics,
// and the constant cache serves one address per access
__device__ DecodeTables c_tab;

static const uint32_t kInlineFloatBits[8] = {0x3f000000u, 0xbf000000u, 0x3f800000u, 0xbf800000u,
                                             0x40000000u, 0xc0000000u, 0x40800000u, 0xc0800000u};
__constant__ uint32_t c_fbits[8];

// hash of a packed mnemonic (the same on host and device)
__host__ __device__ __forceinline__ uint32_t name_hash(const uint32_t (&w)[kNameWords], uint32_t n) {
  uint32_t h = n * 0x9E3779B1u;
#pragma unroll
  for (uint32_t k = 0; k < kNameWords; ++k) h = (h ^ w[k]) * 0x85EBCA77u;
  return (h ^ (h >> 15)) & (kHash - 1);
}

void init_decode_tables() {
  static bool done = false;
  if (done) return;
  DecodeTables t;
  memset(&t, 0, sizeof t);
  for (int i = 1; i < O_COUNT; ++i) {
    const size_t n = strlen(kOps[i].n);
    uint32_t w[kNameWords] = {0, 0, 0, 0, 0, 0};
    for (size_t j = 0; j < n; ++j) w[j / 4] |= (uint32_t)(uint8_t)kOps[i].n[j] << (8 * (j % 4));
    memcpy(t.namew[i], w, sizeof w);
    t.name_len[i] = (uint8_t)n;
    uint32_t h = name_hash(w, (uint32_t)n);
    while (t.ht[h]) h = (h + 1) & (kHash - 1);
    t.ht[h] = (uint16_t)(i + 1);
  }
  cudaMemcpyToSymbol(c_tab, &t, sizeof t);
  cudaMemcpyToSymbol(c_fbits, kInlineFloatBits, sizeof kInlineFloatBits);
  done = true;
}

// the opcode whose mnemonic, packed into w (zero beyond its n bytes), is that of a table entry,
// or O_UNKNOWN
__device__ int find_op(const uint32_t (&w)[kNameWords], uint32_t n) {
  if (n == 0 || n >= 4 * kNameWords) return O_UNKNOWN;
  uint32_t h = name_hash(w, n);
  for (int probe = 0; probe < kHash; ++probe) {
    const uint16_t v = c_tab.ht[h];
    if (!v) return O_UNKNOWN;
    const int op = v - 1;
    if (c_tab.name_len[op] == n) {
      const uint32_t* q = c_tab.namew[op];
      bool eq = true;
#pragma unroll
      for (uint32_t k = 0; k < kNameWords; ++k) eq &= q[k] == w[k];
      if (eq) return op;
    }
    h = (h + 1) & (kHash - 1);
  }
  return O_UNKNOWN;
}

// ---------------------------------------------------------------------------
// S3: configuration
// ---------------------------------------------------------------------------
__device__ uint8_t type_code(const uint8_t* p, const uint8_t* e) {
  if (tok_eq(p, e, "int")) return TY_INT;
  if (tok_eq(p, e, "uint")) return TY_UINT;
  if (tok_eq(p, e, "float")) return TY_FLOAT;
  if (tok_eq(p, e, "long")) return TY_LONG;
  if (tok_eq(p, e, "ulong")) return TY_ULONG;
  if (tok_eq(p, e, "double")) return TY_DOUBLE;
  return TY_NONE;
}

__device__ __forceinline__ void trim(const uint8_t*& p, const uint8_t*& e) {
  while (p < e && is_space(*p)) ++p;
  while (e > p && is_space(e[-1])) --e;
}

// What one configuration row sets: flags of the fields it assigns, their
// values, and an argument record for an .arg row with at least three fields.
enum : uint32_t {
  CF_DIMS = 1, CF_CWS0 = 2, CF_SGPRS = 16, CF_VGPRS = 32, CF_USEARGS = 64, CF_ARG = 128, CF_BAD = 256
};
struct CfgRow {
  uint32_t set;  // CF_* bits (CF_CWS0 << d for .cws component d)
  uint32_t dims, cws[3], regs;
  ArgRec a;
};

__device__ void config_row(const Batch& b, uint32_t l, CfgRow& r) {
  const uint8_t* T = b.text;
  r.set = 0;
  const uint8_t* p = T + b.line_start[l];
  const uint8_t* e = T + b.line_start[l + 1] - 1;
  trim(p, e);
  const uint8_t* t = p;
  while (t < e && !is_space(*t)) ++t;
  const uint8_t* w1 = t;
  while (w1 < e && is_space(*w1)) ++w1;
  const uint8_t* w1e = w1;
  while (w1e < e && !is_space(*w1e)) ++w1e;
  if (tok_eq(p, t, ".dims") || tok_eq(p, t, "dims")) {
    if (w1 == w1e) { r.set = CF_BAD; return; }
    r.set = CF_DIMS;
    r.dims = (uint32_t)(w1e - w1);
    if (r.dims < 1 || r.dims > 3) r.set |= CF_BAD;
  } else if (tok_eq(p, t, ".cws")) {
    const uint8_t* q = p + 4;  // the row after ".cws"
    for (int idx = 0; idx < 3; ++idx) {
      const uint8_t* fe = q;
      while (fe < e && *fe != ',') ++fe;
      const uint8_t *a = q, *z = fe;
      trim(a, z);
      int64_t v;
      bool hx;
      if (!dparse_int(a, z, &v, &hx) || v < 1 || v > 1024) {
        r.set |= CF_BAD;
      } else {
        r.set |= CF_CWS0 << idx;
        r.cws[idx] = (uint32_t)v;
      }
      if (fe >= e) break;
      q = fe + 1;
    }
  } else if (tok_eq(p, t, ".sgprsnum") || tok_eq(p, t, ".vgprsnum")) {
    int64_t v;
    bool hx;
    if (w1 == w1e || !dparse_int(w1, w1e, &v, &hx) || v < 0 || v > 1024) { r.set = CF_BAD; return; }
    r.set = p[1] == 's' ? CF_SGPRS : CF_VGPRS;
    r.regs = (uint32_t)v;
  } else if (tok_eq(p, t, ".useargs")) {
    r.set = CF_USEARGS;
  } else if (tok_eq(p, t, ".arg")) {
    // fields of the row after ".arg", split at commas and trimmed
    const uint8_t* fs[6];
    const uint8_t* fe[6];
    int nf = 0;
    const uint8_t* q = p + 4;
    while (true) {
      const uint8_t* z = q;
      while (z < e && *z != ',') ++z;
      const uint8_t *a = q, *y = z;
      trim(a, y);
      if (nf < 6) { fs[nf] = a; fe[nf] = y; }
      ++nf;
      if (z >= e) break;
      q = z + 1;
    }
    if (nf < 3) { r.set = CF_BAD; return; }
    ArgRec& a = r.a;
    a.name_off = (uint32_t)(fs[0] - T);
    a.name_len = (uint16_t)(fe[0] - fs[0]);
    a.hidden = (fe[0] - fs[0]) >= 2 && fs[0][0] == '_' && fs[0][1] == '.';
    a.gofs = 0;
    if (a.hidden && fe[0] - fs[0] == 17) {
      const char* g = "_.global_offset_";
      bool m = true;
      for (int i = 0; i < 16 && m; ++i) m = fs[0][i] == (uint8_t)g[i];
      if (m && fs[0][16] >= '0' && fs[0][16] <= '2') a.gofs = (uint8_t)(1 + fs[0][16] - '0');
    }
    a.pointer = 0;
    a.is_const = 0;
    a.space = 0;
    if (fe[2] > fs[2] && fe[2][-1] == '*') {
      a.pointer = 1;
      a.elem = type_code(fs[2], fe[2] - 1);
      if (nf > 3) {
        if (tok_eq(fs[3], fe[3], "constant")) a.space = 1;
        else if (tok_eq(fs[3], fe[3], "local")) a.space = 2;
      }
      a.is_const = nf > 4 && tok_eq(fs[4], fe[4], "const");
    } else {
      a.elem = type_code(fs[2], fe[2]);
    }
    r.set = CF_ARG;
  }
}

// S3, a warp per kernel.  Lane 0 reads the .kernel row (the name), finds the
// file and the kernel's counts; the lanes then parse the configuration rows 32
// at a time, one row each, and the rows' effects are combined in row order: a
// field takes the value of the last row that sets it, an argument is appended
// at its rank among the .arg rows before it (rows beyond kMaxArgs arguments
// are errors), and any error marks the kernel bad.
__global__ void __launch_bounds__(128, 12) k_config(const __grid_constant__ Batch b) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  const uint8_t* T = b.text;
  if (lane == 0) {
    // name: second word of the .kernel row
    {
      const uint8_t* p = T + b.line_start[K.line];
      const uint8_t* e = T + b.line_start[K.line + 1] - 1;
      trim(p, e);
      while (p < e && !is_space(*p)) ++p;
      while (p < e && is_space(*p)) ++p;
      const uint8_t* q = p;
      while (q < e && !is_space(*q)) ++q;
      K.name_off = (uint32_t)(p - T);
      K.name_len = (uint32_t)(q - p);
    }
    // file: last f with file_off[f] <= pos; empty files share their start with
    // the next file, so this is the (non-empty) file that holds the row
    {
      uint64_t pos = b.line_start[K.line];
      uint32_t lo = 0, hi = b.F;
      while (lo + 1 < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (b.file_off[mid] <= pos) lo = mid;
        else hi = mid;
      }
      K.file = lo;
    }
    K.n_instr = (k + 1 < b.K ? b.kh[k + 1].first_instr : b.I) - K.first_instr;
    K.n_label = (k + 1 < b.K ? b.kh[k + 1].first_label : b.NL) - K.first_label;
    K.first_pblock = K.n_pblock = K.first_lblock = K.n_lblock = 0;
    K.partial = 0;
    K.capped = 0;
    K.nspill = 0;
    K.entry_target = 0;
    K.status = 0;
    K.n_cfg = (k + 1 < b.K ? b.kh[k + 1].first_cfg : b.NC) - K.first_cfg;
  }
  const uint32_t first_cfg = K.first_cfg;
  const uint32_t n_cfg = (k + 1 < b.K ? b.kh[k + 1].first_cfg : b.NC) - first_cfg;
  ArgRec* A = b.args + (size_t)k * kMaxArgs;
  uint32_t dims = 1, cws[3] = {1, 1, 1}, sgprs = 104, vgprs = 256, useargs = 0, nargs = 0, nuser = 0, bad = 0;
  for (uint32_t c0 = 0; c0 < n_cfg; c0 += 32) {
    CfgRow r;
    r.set = 0;
    if (c0 + lane < n_cfg) config_row(b, b.cfg_line[first_cfg + c0 + lane], r);
    // last row (highest lane) that sets each field
    const auto last = [&](uint32_t flag, uint32_t val, uint32_t& field) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, (r.set & flag) != 0);
      if (m) field = __shfl_sync(0xFFFFFFFFu, val, 31 - __clz(m));
    };
    last(CF_DIMS, r.dims, dims);
    last(CF_CWS0, r.cws[0], cws[0]);
    last(CF_CWS0 << 1, r.cws[1], cws[1]);
    last(CF_CWS0 << 2, r.cws[2], cws[2]);
    last(CF_SGPRS, r.regs, sgprs);
    last(CF_VGPRS, r.regs, vgprs);
    if (__any_sync(0xFFFFFFFFu, (r.set & CF_USEARGS) != 0)) useargs = 1;
    bool my_bad = (r.set & CF_BAD) != 0;
    const unsigned am = __ballot_sync(0xFFFFFFFFu, (r.set & CF_ARG) != 0);
    bool user = false;
    if (r.set & CF_ARG) {
      const uint32_t at = nargs + __popc(am & ((1u << lane) - 1u));
      if (at >= (uint32_t)kMaxArgs) {
        my_bad = true;
      } else {
        A[at] = r.a;
        if (!r.a.hidden) {
          user = true;
          if (r.a.elem == TY_NONE) my_bad = true;
        }
      }
    }
    nuser += __popc(__ballot_sync(0xFFFFFFFFu, user));
    nargs = min(nargs + (uint32_t)__popc(am), (uint32_t)kMaxArgs);
    if (__any_sync(0xFFFFFFFFu, my_bad)) bad = 1;
  }
  if (lane == 0) {
    K.dims = dims;
    K.cws[0] = cws[0];
    K.cws[1] = cws[1];
    K.cws[2] = cws[2];
    K.sgprs = sgprs;
    K.vgprs = vgprs;
    K.useargs = useargs;
    K.nargs = nargs;
    K.nuser = nuser;
    K.bad = bad;
  }
}

void launch_config(Batch& b, cudaStream_t s) {
  if (!b.K) return;
  k_config<<<(uint32_t)(((uint64_t)b.K * 32 + 127) / 128), 128, 0, s>>>(b);
  ++launch_counter();
}

// ---------------------------------------------------------------------------
// S4: instruction decoding
// ---------------------------------------------------------------------------
__device__ bool parse_operand(const uint8_t* p, const uint8_t* e, uint32_t* word, bool* is_lit, uint32_t* lit) {
  *is_lit = false;
  const uint32_t n = (uint32_t)(e - p);
  const uint8_t c0 = p[0];
  if (n == 3 && c0 == 'v' && p[1] == 'c' && p[2] == 'c') { *word = opw(TG_VCC, 2, 0); return true; }
  if (n == 4 && c0 == 'e' && p[1] == 'x' && p[2] == 'e' && p[3] == 'c') { *word = opw(TG_EXEC, 2, 0); return true; }
  if (n == 3 && c0 == 'o' && p[1] == 'f' && p[2] == 'f') { *word = opw(TG_OFF, 0, 0); return true; }
  if ((c0 == 'v' || c0 == 's') && n >= 2) {
    const uint32_t tag = c0 == 'v' ? TG_VGPR : TG_SGPR;
    if (p[1] == '[') {
      const uint8_t *colon = nullptr, *close = nullptr;
      for (const uint8_t* q = p; q < e; ++q) {
        if (!colon && *q == ':') colon = q;
        if (!close && *q == ']') close = q;
      }
      if (!colon || !close || close != e - 1 || colon > close) return false;
      int64_t a, bb;
      bool h1, h2;
      if (!dparse_int(p + 2, colon, &a, &h1) || !dparse_int(colon + 1, close, &bb, &h2)) return false;
      if ((colon - (p + 2) >= 2 && p[2] == '0' && p[3] == 'x') || a < 0 || bb < a || bb - a + 1 > 8 || bb > 1023)
        return false;
      *word = opw(tag, (uint32_t)(bb - a + 1), (uint32_t)a);
      return true;
    }
    // a register number: decimal digits only (a '-' or hex prefix is no register)
    uint32_t a = 0;
    for (const uint8_t* q = p + 1; q < e; ++q) {
      if (*q < '0' || *q > '9') return false;
      a = a * 10 + (*q - '0');
      if (a > 1023) return false;
    }
    *word = opw(tag, 1, a);
    return true;
  }
  // the inline float constants 0.5, 1.0, 2.0, 4.0 and their negations (table order: value, then
  // its negation)
  if ((n == 3 || n == 4) && p[n - 2] == '.') {
    const bool neg = c0 == '-';
    if (n == 3 + (uint32_t)neg) {
      const uint8_t d = p[neg], f = p[neg + 2];
      int k = -1;
      if (d == '0' && f == '5') k = 0;
      else if (f == '0') k = d == '1' ? 1 : d == '2' ? 2 : d == '4' ? 3 : -1;
      if (k >= 0) { *word = opw(TG_FCONST, 1, (uint32_t)(2 * k + neg)); return true; }
    }
  }
  int64_t v;
  bool hex;
  if (dparse_int(p, e, &v, &hex)) {
    // a parsed integer holds an 'x' only as its hex prefix
    if (!hex && v >= -16 && v <= 64) {
      *word = opw(TG_ICONST, 1, (uint32_t)v & 0xFFFFFFu);
      return true;
    }
    *word = opw(TG_LIT, 1, 0);
    *is_lit = true;
    *lit = (uint32_t)(uint64_t)v;
    return true;
  }
  return false;
}

__device__ bool sig_ok(char s, uint32_t o) {
  uint32_t tg = otag(o), n = ocnt(o);
  switch (s) {
    case 'V': return tg == TG_VGPR && n == 1;
    case 'W': return tg == TG_VGPR && n == 2;
    case 's': return tg == TG_SGPR && n == 1;
    case 'p': return tg == TG_SGPR && n == 2;
    case 'q': return tg == TG_SGPR && n == 4;
    case 'S': return ((tg == TG_VGPR || tg == TG_SGPR) && n == 1) || tg == TG_ICONST || tg == TG_FCONST || tg == TG_LIT;
    case 'M': return (tg == TG_SGPR && n == 2) || tg == TG_VCC || tg == TG_EXEC;
    case 'c': return tg == TG_VCC;
    case 'o': return tg == TG_OFF;
    case 'K': return tg == TG_ICONST || tg == TG_LIT;
  }
  return false;
}

// Scanners over the bytes of one line; positions are offsets from a base.
// BitScan serves a line staged in shared memory, through the warp's bitmaps of
// space (' ', '\t', '\r') and comma bytes: a scan to the next token boundary
// is a few word operations instead of a loop over bytes.  ByteScan is the same
// over plain bytes, for a line the stage does not hold.
constexpr uint32_t DEC_STAGE = 2048;  // staged text bytes per warp
constexpr uint32_t kStageWords = DEC_STAGE / 4;
struct BitScan {
  const uint32_t* sp;  // bit j: byte j is a space
  const uint32_t* cm;  // bit j: byte j is a comma
  // first j in [from, to) whose bit in B (inverted by inv) is set, else to
  __device__ __forceinline__ static uint32_t first(const uint32_t* B, uint32_t inv, uint32_t from, uint32_t to) {
    if (from >= to) return to;
    uint32_t w = from >> 5;
    uint32_t x = (B[w] ^ inv) & (0xFFFFFFFFu << (from & 31));
    while (!x) {
      if ((++w << 5) >= to) return to;
      x = B[w] ^ inv;
    }
    const uint32_t j = (w << 5) + (uint32_t)(__ffs(x) - 1);
    return j < to ? j : to;
  }
  __device__ __forceinline__ uint32_t space(uint32_t from, uint32_t to) const { return first(sp, 0u, from, to); }
  __device__ __forceinline__ uint32_t nonspace(uint32_t from, uint32_t to) const { return first(sp, ~0u, from, to); }
  __device__ __forceinline__ uint32_t comma(uint32_t from, uint32_t to) const { return first(cm, 0u, from, to); }
  // bytes [p, p + n) of the 16-byte aligned stage t, packed into words (n < 24): seven aligned
  // word loads and funnel shifts, the same for every lane (no loop over the bytes)
  __device__ __forceinline__ static void pack(const uint8_t* t, uint32_t p, uint32_t n, uint32_t (&w)[kNameWords]) {
    const uint32_t* t32 = reinterpret_cast<const uint32_t*>(t);
    const uint32_t w0 = p >> 2, sh = 8 * (p & 3);
    uint32_t x[kNameWords + 1];
#pragma unroll
    for (uint32_t k = 0; k <= kNameWords; ++k) x[k] = w0 + k < kStageWords ? t32[w0 + k] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kNameWords; ++k) {
      const uint32_t v = __funnelshift_r(x[k], x[k + 1], sh);
      const uint32_t lo = 4 * k;  // bytes lo..lo+3 of the name
      w[k] = n >= lo + 4 ? v : n <= lo ? 0u : v & (0xFFFFFFFFu >> (8 * (lo + 4 - n)));
    }
  }
  // one past the last non-space of [from, to), else from
  __device__ __forceinline__ uint32_t trim_end(uint32_t from, uint32_t to) const {
    if (from >= to) return from;
    uint32_t w = (to - 1) >> 5;
    uint32_t x = ~sp[w] & (0xFFFFFFFFu >> (31 - ((to - 1) & 31)));
    while (!x) {
      if ((w << 5) <= from) return from;
      x = ~sp[--w];
    }
    const uint32_t j = (w << 5) + 31 - (uint32_t)__clz(x);
    return j >= from ? j + 1 : from;
  }
};
struct ByteScan {
  const uint8_t* t;
  __device__ __forceinline__ uint32_t space(uint32_t from, uint32_t to) const {
    while (from < to && !is_space(t[from])) ++from;
    return from;
  }
  __device__ __forceinline__ uint32_t nonspace(uint32_t from, uint32_t to) const {
    while (from < to && is_space(t[from])) ++from;
    return from;
  }
  __device__ __forceinline__ uint32_t comma(uint32_t from, uint32_t to) const {
    while (from < to && t[from] != ',') ++from;
    return from;
  }
  __device__ __forceinline__ uint32_t trim_end(uint32_t from, uint32_t to) const {
    while (to > from && is_space(t[to - 1])) --to;
    return to;
  }
  __device__ __forceinline__ static void pack(const uint8_t* t, uint32_t p, uint32_t n, uint32_t (&w)[kNameWords]) {
#pragma unroll
    for (uint32_t k = 0; k < kNameWords; ++k) w[k] = 0;
    for (uint32_t j = 0; j < n; ++j) w[j >> 2] |= (uint32_t)t[p + j] << (8 * (j & 3));
  }
};

// The record of the instruction row [P0, E0) (positions of scanner S over the
// bytes at t; the row without its '\n'): the mnemonic (first word), then the
// operand fields split at commas, each trimmed; a field's first word is the
// operand, its further words modifiers, of which offset:K is read.  A branch's
// label operand is returned as its text position (ls = the text offset of P0)
// and length.
template <class S>
__device__ __forceinline__ InstrRec decode_row(const S& sc, const uint8_t* t, uint32_t P0, uint32_t E0, uint64_t ls,
                                               uint32_t* lbl_pos, uint32_t* lbl_len) {
  const uint32_t p = sc.nonspace(P0, E0);
  const uint32_t e = sc.trim_end(p, E0);
  const uint32_t me = sc.space(p, e);  // the mnemonic
  InstrRec r;
  {
    uint32_t w[kNameWords];
    const uint32_t n = me - p < 4 * kNameWords ? me - p : 0u;  // longer: no mnemonic, O_UNKNOWN
    S::pack(t, p, n, w);
    r.op = (uint16_t)find_op(w, n);
  }
  r.nops = 0;
  r.flags = r.op == O_UNKNOWN ? FL_UNSUPPORTED : 0;
  r.imm = 0;
  r.target = kNone;
  for (int q = 0; q < 5; ++q) r.opnd[q] = 0;
  *lbl_pos = 0;
  *lbl_len = 0;
  const char* sig = c_sig[r.op];
  const uint32_t rp = sc.nonspace(me, e);
  if (r.op != O_S_WAITCNT && rp < e) {
    int nlit = 0;
    uint32_t q = rp;
    while (true) {
      const uint32_t z = sc.comma(q, e);
      const uint32_t a = sc.nonspace(q, z);
      const uint32_t y = sc.trim_end(a, z);
      const uint32_t s0 = sc.space(a, y);  // the operand is [a, s0), modifiers follow
      if (a == y) {
        r.flags |= FL_BAD;
      } else {
        uint32_t m = s0;
        while (m < y) {
          m = sc.nonspace(m, y);
          const uint32_t me2 = sc.space(m, y);
          const uint8_t* w = t + m;
          if (me2 - m >= 7 && w[0] == 'o' && w[1] == 'f' && w[2] == 'f' && w[3] == 's' && w[4] == 'e' && w[5] == 't' &&
              w[6] == ':') {
            int64_t v;
            bool hx;
            if (!dparse_int(w + 7, t + me2, &v, &hx) || v < 0) r.flags |= FL_BAD;
            else r.imm = (uint32_t)v;
          }
          m = me2;
        }
        uint32_t word = 0, lit = 0;
        bool is_lit = false, ok = true;
        if (sig[0] == 'L') {
          *lbl_pos = (uint32_t)(ls + (a - P0));
          *lbl_len = s0 - a;
          word = opw(TG_LABEL, 0, 0);
        } else if (!parse_operand(t + a, t + s0, &word, &is_lit, &lit)) {
          r.flags |= FL_BAD;
          ok = false;
        }
        if (ok) {
          if (is_lit) {
            if (nlit++) r.flags |= FL_BAD;
            r.imm = lit;
          }
          if (r.nops < 5) r.opnd[r.nops++] = word;
          else r.flags |= FL_BAD;
        }
      }
      if (z >= e) break;
      q = z + 1;
    }
  }
  return r;
}

// A warp decodes `per` consecutive instructions, one per lane: 32, or 1 for a
// small batch, where the lanes of a warp would otherwise run the parsing paths
// of 32 different lines one after another on the critical path.  The lines
// lie close together in the text, so the warp first copies the span they cover
// into shared memory with coalesced 16-byte loads and marks its space and
// comma bytes in two bitmaps (a ballot per 32 bytes); each lane then parses
// its line from there.  A line beyond the staged span (a kernel's
// configuration block between two instructions can make the span long) is
// parsed straight from global memory.
constexpr int DEC_THREADS = 256;
constexpr uint32_t DEC_SMALL = 8192;     // at most this many instructions: one per warp

__global__ void __launch_bounds__(DEC_THREADS) k_decode(const __grid_constant__ Batch b, uint32_t per) {
  __shared__ __align__(16) uint8_t stage[DEC_THREADS / 32][DEC_STAGE];
  __shared__ uint32_t s_sp[DEC_THREADS / 32][DEC_STAGE / 32], s_cm[DEC_THREADS / 32][DEC_STAGE / 32];
  const uint32_t lane = threadIdx.x & 31u, wp = threadIdx.x >> 5;
  const uint32_t w0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * per;  // the warp's first instruction
  if (w0 >= b.I) return;  // the whole warp
  const uint32_t i = w0 + lane;
  const uint32_t wl = b.I - w0 < per ? b.I - w0 : per;
  const uint32_t line = lane < wl ? b.instr_line[i] : 0;
  const uint32_t l_first = __shfl_sync(0xFFFFFFFFu, line, 0), l_last = __shfl_sync(0xFFFFFFFFu, line, wl - 1);
  const uint64_t a0 = b.line_start[l_first] & ~15ull;
  const uint64_t s1 = b.line_start[l_last + 1];
  const uint32_t span = (uint32_t)(s1 - a0 < DEC_STAGE ? s1 - a0 : DEC_STAGE);  // within the text
  uint8_t* st = stage[wp];
  if ((reinterpret_cast<uintptr_t>(b.text) & 15u) == 0) {
    const uint32_t nv = span / 16;
    for (uint32_t q = lane; q < nv; q += 32)
      reinterpret_cast<uint4*>(st)[q] = reinterpret_cast<const uint4*>(b.text + a0)[q];
    for (uint32_t j = nv * 16 + lane; j < span; j += 32) st[j] = b.text[a0 + j];
  } else {
    for (uint32_t j = lane; j < span; j += 32) st[j] = b.text[a0 + j];
  }
  __syncwarp();
  for (uint32_t j0 = 0; j0 < span; j0 += 32) {
    const uint8_t c = j0 + lane < span ? st[j0 + lane] : (uint8_t)'\n';
    const unsigned sp = __ballot_sync(0xFFFFFFFFu, is_space(c)), cm = __ballot_sync(0xFFFFFFFFu, c == ',');
    if (lane == 0) {
      s_sp[wp][j0 >> 5] = sp;
      s_cm[wp][j0 >> 5] = cm;
    }
  }
  __syncwarp();
  if (lane >= wl) return;
  uint32_t k = b.kcnt[line] - 1;
  const KHdr& K = b.kh[k];
  const uint64_t ls = b.line_start[line], le = b.line_start[line + 1] - 1;  // the line without its '\n'
  const bool staged = le <= a0 + span;
  uint32_t lbl_pos, lbl_len;
  InstrRec r;
  if (staged)
    r = decode_row(BitScan{s_sp[wp], s_cm[wp]}, st, (uint32_t)(ls - a0), (uint32_t)(le - a0), ls, &lbl_pos, &lbl_len);
  else
    r = decode_row(ByteScan{b.text + ls}, b.text + ls, 0u, (uint32_t)(le - ls), ls, &lbl_pos, &lbl_len);
  const char* sig = c_sig[r.op];
  if (r.op && r.op != O_S_WAITCNT) {
    int want = sig_count(r.op);
    if (r.nops != want) r.flags |= FL_BAD;
    else
      for (int q = 0; q < want; ++q)
        if (sig[2 * q] != 'L' && !sig_ok(sig[2 * q], r.opnd[q])) r.flags |= FL_BAD;
    if ((r.op == O_S_LOAD_DWORD || r.op == O_S_LOAD_DWORDX2 || r.op == O_S_LOAD_DWORDX4) && r.nops == 3 &&
        otag(r.opnd[2]) == TG_ICONST) {
      uint32_t pay = opay(r.opnd[2]);
      r.imm = (pay & 0x800000u) ? (pay | 0xFF000000u) : pay;
    }
    if ((r.op == O_BUFFER_LOAD_DWORD || r.op == O_BUFFER_STORE_DWORD) && (r.imm & 3u)) r.flags |= FL_BAD;
    // a global, FLAT or LDS access with a constant byte offset: not folded into the address, so
    // the instruction stays inline assembly
    if ((op_gload(r.op) || op_store(r.op)) && r.imm) {
      r.op = O_UNKNOWN;
      r.flags |= FL_UNSUPPORTED;
    }
  }
  if (r.op == O_S_WAITCNT) r.nops = 0;
  for (int q = 0; q < r.nops; ++q) {
    uint32_t o = r.opnd[q], tg = otag(o);
    if (tg == TG_VGPR && opay(o) + ocnt(o) > K.vgprs) r.flags |= FL_REGRANGE;
    if (tg == TG_SGPR && opay(o) + ocnt(o) > K.sgprs) r.flags |= FL_REGRANGE;
  }
  b.ins[i] = r;
  b.branch_hash[i] = lbl_len ? fnv1a(b.text + lbl_pos, lbl_len) : 0;
  b.branch_pos[i] = lbl_len ? lbl_pos : kNone;
  b.blen[i] = lbl_len;
  b.ikern[i] = k;
}

// Labels are found through a batch-wide open-addressing table keyed by
// (kernel, FNV-1a of the name): a branch probes from its key's slot to the
// first empty one and takes the lowest label index whose name matches exactly
// (the first definition of a label wins).
__device__ __forceinline__ uint32_t label_slot(uint32_t k, uint32_t h, uint32_t mask) {
  uint32_t x = h ^ (k * 0x9E3779B1u);
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  return x & mask;
}

__global__ void k_label_hash(const __grid_constant__ Batch b) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.NL) return;
  uint32_t line = b.label_line[j];
  const uint8_t* p = b.text + b.line_start[line];
  const uint8_t* e = b.text + b.line_start[line + 1] - 1;
  trim(p, e);
  const uint32_t h = fnv1a(p, (uint32_t)(e - p - 1));
  b.label_hash[j] = h;
  uint32_t slot = label_slot(b.kcnt[line] - 1, h, b.label_tab_mask);
  for (uint32_t probe = 0; probe <= b.label_tab_mask; ++probe) {
    if (atomicCAS(&b.label_tab[slot], kNone, j) == kNone) return;
    slot = (slot + 1) & b.label_tab_mask;
  }
  atomicOr(b.err, ERR_CAPACITY);  // more labels than slots: cannot happen (twice as many slots)
}

// branch targets (first definition of the label wins), per-kernel parse flags, leaders
__global__ void k_resolve(const __grid_constant__ Batch b) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.I) return;
  uint32_t k = b.ikern[i];
  KHdr& K = b.kh[k];
  InstrRec& r = b.ins[i];
  if (b.branch_pos[i] != kNone) {
    uint32_t len = b.blen[i];
    const uint8_t* s = b.text + b.branch_pos[i];
    uint32_t h = b.branch_hash[i];
    uint32_t best = kNone;  // lowest matching label index
    uint32_t slot = label_slot(k, h, b.label_tab_mask);
    for (uint32_t probe = 0; probe <= b.label_tab_mask; ++probe) {
      const uint32_t j = b.label_tab[slot];
      if (j == kNone) break;
      slot = (slot + 1) & b.label_tab_mask;
      if (j >= best || b.label_hash[j] != h || j < K.first_label || j >= K.first_label + K.n_label) continue;
      const uint8_t* p = b.text + b.line_start[b.label_line[j]];
      while (is_space(*p)) ++p;
      bool eq = true;
      for (uint32_t q = 0; q < len && eq; ++q) eq = p[q] == s[q];
      if (eq && p[len] == ':') best = j;
    }
    if (best == kNone) r.flags |= FL_NOLABEL;
    else r.target = b.label_instr[best] - K.first_instr;
  }
  if (r.flags & (FL_BAD | FL_REGRANGE | FL_NOLABEL)) atomicOr(&K.bad, 2u);
}

__device__ __forceinline__ bool is_br(uint16_t op) {
  return op == O_S_BRANCH || op == O_S_CBRANCH_SCC0 || op == O_S_CBRANCH_SCC1 || op == O_S_CBRANCH_EXECZ;
}

__global__ void k_pleaders(const __grid_constant__ Batch b) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.I) return;
  const KHdr& K = b.kh[b.ikern[i]];
  uint32_t rel = i - K.first_instr, n = K.n_instr;
  const InstrRec& r = b.ins[i];
  if (rel == 0) b.pleader[i] = 1;
  if (is_br(r.op) && r.target < n) b.pleader[K.first_instr + r.target] = 1;
  if ((is_br(r.op) || r.op == O_S_ENDPGM) && rel + 1 < n) b.pleader[i + 1] = 1;
}

// after the inclusive scan of leaders: block ids and block starts
__global__ void k_pblocks(const __grid_constant__ Batch b, const uint32_t* __restrict__ incl, uint32_t* __restrict__ blk_kern) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.I) return;
  uint32_t k = b.ikern[i];
  KHdr& K = b.kh[k];
  uint32_t g = incl[i] - 1;
  uint32_t base = incl[K.first_instr] - 1;
  uint32_t rel = i - K.first_instr;
  b.pblock_of[i] = g - base;
  if (rel == 0) {
    K.first_pblock = base;
    K.n_pblock = (K.n_instr ? incl[K.first_instr + K.n_instr - 1] : base) - base;
  }
  if (b.pleader[i]) {
    b.pblocks[g].first = rel;
    blk_kern[g] = k;
  }
}

__global__ void k_pblock_edges(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.NPB) return;
  const KHdr& K = b.kh[blk_kern[g]];
  uint32_t n = K.n_instr;
  BlockRec& B = b.pblocks[g];
  B.end = (g + 1 < K.first_pblock + K.n_pblock) ? b.pblocks[g + 1].first : n;
  const InstrRec& last = b.ins[K.first_instr + B.end - 1];
  uint32_t ft = B.end < n ? b.pblock_of[K.first_instr + B.end] : kNone;
  uint32_t tg = last.target < n ? b.pblock_of[K.first_instr + last.target] : kNone;
  B.succ0 = kNone;
  B.succ1 = kNone;
  if (last.op == O_S_BRANCH) B.succ0 = tg;
  else if (is_br(last.op)) { B.succ0 = ft; B.succ1 = tg; }
  else if (last.op != O_S_ENDPGM) B.succ0 = ft;
}

void launch_decode(Batch& b, ScanScratch sc, uint32_t* totals, cudaStream_t s) {
  const int T = 256;
  if (!b.I) return;
  ktime(KT_DECODE, 0, s);
  const uint32_t per = b.I <= DEC_SMALL ? 1u : 32u;
  const uint64_t warps = (b.I + per - 1) / per;
  k_decode<<<(uint32_t)((warps * 32 + DEC_THREADS - 1) / DEC_THREADS), DEC_THREADS, 0, s>>>(b, per);
  ktime(KT_DECODE, 1, s);
  ++launch_counter();
  if (b.NL) {
    cudaMemsetAsync(b.label_tab, 0xFF, sizeof(uint32_t) * ((size_t)b.label_tab_mask + 1), s);
    k_label_hash<<<(b.NL + T - 1) / T, T, 0, s>>>(b);
    ++launch_counter();
  }
  k_resolve<<<(b.I + T - 1) / T, T, 0, s>>>(b);
  ++launch_counter();
  cudaMemsetAsync(b.pleader, 0, sizeof(uint32_t) * b.I, s);
  k_pleaders<<<(b.I + T - 1) / T, T, 0, s>>>(b);
  ++launch_counter();
  launch_scan(b.pleader, b.lleader, b.I, 0, true, sc, &totals[3], b.err, s);  // totals[3] = physical blocks
}

void launch_pblocks(Batch& b, uint32_t* blk_kern, cudaStream_t s) {
  const int T = 256;
  if (!b.I) return;
  k_pblocks<<<(b.I + T - 1) / T, T, 0, s>>>(b, b.lleader, blk_kern);
  ++launch_counter();
  if (b.NPB) {
    k_pblock_edges<<<(b.NPB + T - 1) / T, T, 0, s>>>(b, blk_kern);
    ++launch_counter();
  }
}

// ---------------------------------------------------------------------------
// S6: exec-mask forms -> standard form, logical blocks
// ---------------------------------------------------------------------------
struct Form {
  uint32_t save, xor1, ez1, els, xor2, ez2;
};

__device__ __forceinline__ bool same_pair(uint32_t a, uint32_t bb) { return otag(a) == TG_SGPR && a == bb; }

// every instruction: default control, branches and s_endpgm; flag the
// instructions that take part in exec-mask forms
__device__ __forceinline__ bool exec_form_op(uint16_t op) {
  return op == O_S_AND_SAVEEXEC || op == O_S_XOR_B64 || op == O_S_CBRANCH_EXECZ || op == O_S_OR_SAVEEXEC ||
         op == O_S_OR_B64;
}

__global__ void k_exec_init(const __grid_constant__ Batch b, uint32_t* __restrict__ flag) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi > b.I) return;
  if (gi == b.I) {
    flag[gi] = 0;
    return;
  }
  const InstrRec& r = b.ins[gi];
  uint8_t c = C_NORMAL, sn = 0;
  uint32_t t = kNone;
  if (r.op == O_S_BRANCH) {
    c = C_JMP;
    t = r.target;
  } else if (r.op == O_S_CBRANCH_SCC0 || r.op == O_S_CBRANCH_SCC1) {
    c = C_CBR;
    t = r.target;
    sn = r.op == O_S_CBRANCH_SCC1;
  } else if (r.op == O_S_ENDPGM) {
    c = C_END;
  }
  b.ctl[gi] = c;
  b.ltarget[gi] = t;
  b.sense[gi] = sn;
  flag[gi] = exec_form_op(r.op);
}

__global__ void k_exec_list(uint32_t I, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                            uint32_t* __restrict__ list) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi < I && flag[gi]) list[pos[gi]] = gi;
}

// per kernel: the exec-mask forms, matched over the kernel's exec-form
// instructions only (in program order) with a stack of open forms
// A warp per kernel: the lanes load the kernel's next 32 exec-mask instructions
// into shared memory together, then lane 0 runs the form matcher over them.
__global__ void k_exec_forms(const __grid_constant__ Batch b, const uint32_t* __restrict__ pos,
                             const uint32_t* __restrict__ list) {
  __shared__ InstrRec s_rec[4][32];
  __shared__ uint32_t s_idx[4][32];
  const uint32_t wp = threadIdx.x / 32, lane = threadIdx.x & 31u;
  const uint32_t k = blockIdx.x * (blockDim.x / 32) + wp;  // at most four warps per block (walk_threads)
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  const InstrRec* R = b.ins + K.first_instr;
  uint8_t* ctl = b.ctl + K.first_instr;
  uint32_t* lt = b.ltarget + K.first_instr;
  uint8_t* sense = b.sense + K.first_instr;
  const uint32_t c0 = pos[K.first_instr], c1 = pos[K.first_instr + K.n_instr];
  Form st[kMaxExecDepth];
  int sp = 0;
  bool bad = false;
  for (uint32_t base = c0; base < c1; base += 32) {
    if (base + lane < c1) {
      const uint32_t i = list[base + lane] - K.first_instr;
      s_idx[wp][lane] = i;
      s_rec[wp][lane] = R[i];
    }
    __syncwarp();
    const uint32_t m = min(32u, c1 - base);
    for (uint32_t q = 0; lane == 0 && q < m && !bad; ++q) {
    const uint32_t i = s_idx[wp][q];
    const InstrRec& r = s_rec[wp][q];
    switch (r.op) {
      case O_S_AND_SAVEEXEC:
        if (otag(r.opnd[0]) != TG_SGPR || otag(r.opnd[1]) != TG_VCC || sp == kMaxExecDepth) { bad = true; break; }
        st[sp++] = Form{i, kNone, kNone, kNone, kNone, kNone};
        break;
      case O_S_XOR_B64: {
        if (!sp) { bad = true; break; }
        Form& f = st[sp - 1];
        uint32_t S = R[f.save].opnd[0];
        if (f.els == kNone && f.xor1 == kNone && i == f.save + 1 && same_pair(r.opnd[0], S) &&
            otag(r.opnd[1]) == TG_EXEC && same_pair(r.opnd[2], S))
          f.xor1 = i;
        else if (f.els != kNone && f.xor2 == kNone && i == f.els + 1 && otag(r.opnd[0]) == TG_EXEC &&
                 otag(r.opnd[1]) == TG_EXEC && same_pair(r.opnd[2], S))
          f.xor2 = i;
        else
          bad = true;
        break;
      }
      case O_S_CBRANCH_EXECZ: {
        if (!sp) { bad = true; break; }
        Form& f = st[sp - 1];
        if (f.els == kNone && f.ez1 == kNone && i == (f.xor1 != kNone ? f.xor1 : f.save) + 1) f.ez1 = i;
        else if (f.xor2 != kNone && f.ez2 == kNone && i == f.xor2 + 1) f.ez2 = i;
        else bad = true;
        break;
      }
      case O_S_OR_SAVEEXEC: {
        if (!sp) { bad = true; break; }
        Form& f = st[sp - 1];
        uint32_t S = R[f.save].opnd[0];
        if (f.xor1 == kNone || f.els != kNone || !same_pair(r.opnd[0], S) || !same_pair(r.opnd[1], S)) {
          bad = true;
          break;
        }
        f.els = i;
        break;
      }
      case O_S_OR_B64: {
        if (!sp) { bad = true; break; }
        Form f = st[sp - 1];
        uint32_t S = R[f.save].opnd[0];
        if (otag(r.opnd[0]) != TG_EXEC || otag(r.opnd[1]) != TG_EXEC || !same_pair(r.opnd[2], S) ||
            (f.xor1 == kNone) != (f.els == kNone) || (f.els != kNone && f.xor2 == kNone)) {
          bad = true;
          break;
        }
        --sp;
        // standard form: branch on the compare, jump from the then part to the join
        ctl[f.save] = C_CBR;
        sense[f.save] = 0;
        if (f.xor1 != kNone) ctl[f.xor1] = C_DROP;
        if (f.ez1 != kNone) ctl[f.ez1] = C_DROP;
        if (f.els != kNone) {
          ctl[f.els] = C_JMP;
          ctl[f.xor2] = C_DROP;
          if (f.ez2 != kNone) ctl[f.ez2] = C_DROP;
          lt[f.save] = (f.ez2 != kNone ? f.ez2 : f.xor2) + 1;
          lt[f.els] = i + 1;
        } else {
          lt[f.save] = i + 1;
        }
        ctl[i] = C_DROP;
        break;
      }
      default:
        break;
    }
    }
    if (__shfl_sync(0xFFFFFFFFu, (int)bad, 0)) break;
    __syncwarp();
  }
  if (lane == 0) {
    if (sp) bad = true;
    if (bad) K.bad |= 4u;
  }
}

__device__ __forceinline__ uint32_t resolve_t(const uint8_t* ctl, uint32_t t, uint32_t n) {
  while (t < n && ctl[t] == C_DROP) ++t;
  return t;
}

__global__ void k_lleaders(const __grid_constant__ Batch b) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.I) return;
  const KHdr& K = b.kh[b.ikern[i]];
  if (K.bad) return;
  const uint8_t* ctl = b.ctl + K.first_instr;
  uint32_t n = K.n_instr, rel = i - K.first_instr;
  uint32_t& t = b.ltarget[i];
  if (t != kNone) t = resolve_t(ctl, t, n);
  if (rel == resolve_t(ctl, 0, n)) b.pleader[i] = 1;
  uint8_t c = ctl[rel];
  if ((c == C_CBR || c == C_JMP) && t < n) b.pleader[K.first_instr + t] = 1;
  if (c == C_CBR || c == C_JMP || c == C_END) {
    uint32_t nx = resolve_t(ctl, rel + 1, n);
    if (nx < n) b.pleader[K.first_instr + nx] = 1;
  }
}

__global__ void k_lblocks(const __grid_constant__ Batch b, const uint32_t* __restrict__ incl, uint32_t* __restrict__ blk_kern) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.I) return;
  uint32_t k = b.ikern[i];
  KHdr& K = b.kh[k];
  uint32_t rel = i - K.first_instr;
  uint32_t before = K.first_instr ? incl[K.first_instr - 1] : 0;  // blocks of earlier kernels
  if (rel == 0) {
    K.first_lblock = before;
    K.n_lblock = (K.n_instr ? incl[K.first_instr + K.n_instr - 1] : before) - before;
  }
  if (K.bad) { b.lblock_of[i] = kNone; return; }
  uint32_t g = incl[i];
  b.lblock_of[i] = (b.ctl[i] == C_DROP || g == before) ? kNone : g - 1 - before;
  if (b.pleader[i]) {
    b.lblocks[g - 1].first = rel;
    blk_kern[g - 1] = k;
  }
}

__global__ void k_lblock_edges(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.NLB) return;
  const KHdr& K = b.kh[blk_kern[g]];
  uint32_t n = K.n_instr;
  const uint8_t* ctl = b.ctl + K.first_instr;
  BlockRec& B = b.lblocks[g];
  B.end = (g + 1 < K.first_lblock + K.n_lblock) ? b.lblocks[g + 1].first : n;
  uint32_t t = B.end - 1;
  while (t > B.first && ctl[t] == C_DROP) --t;
  b.lterm[g] = t;
  uint32_t nx = resolve_t(ctl, t + 1, n);
  uint32_t ft = nx < n ? b.lblock_of[K.first_instr + nx] : kNone;
  uint32_t tt = b.ltarget[K.first_instr + t];
  uint32_t tg = tt < n ? b.lblock_of[K.first_instr + tt] : kNone;
  B.succ0 = kNone;
  B.succ1 = kNone;
  switch (ctl[t]) {
    case C_CBR: B.succ0 = ft; B.succ1 = tg == ft ? kNone : tg; break;
    case C_JMP: B.succ0 = tg; break;
    case C_END: break;
    default: B.succ0 = ft;
  }
}

void launch_logical(Batch& b, ScanScratch sc, uint32_t* totals, cudaStream_t s) {
  const int T = 256;
  if (!b.I) return;
  // pleader / lleader serve as flag and position arrays of the exec-form
  // instructions until the logical leaders are computed
  k_exec_init<<<(b.I + 1 + T - 1) / T, T, 0, s>>>(b, b.pleader);
  ++launch_counter();
  launch_scan(b.pleader, b.lleader, b.I + 1, 0, false, sc, nullptr, b.err, s);
  k_exec_list<<<(b.I + T - 1) / T, T, 0, s>>>(b.I, b.pleader, b.lleader, b.exec_list);
  ++launch_counter();
  k_exec_forms<<<walk_blocks(b.K), walk_threads(b.K), 0, s>>>(b, b.lleader, b.exec_list);
  ++launch_counter();
  cudaMemsetAsync(b.pleader, 0, sizeof(uint32_t) * b.I, s);
  k_lleaders<<<(b.I + T - 1) / T, T, 0, s>>>(b);
  ++launch_counter();
  launch_scan(b.pleader, b.lleader, b.I, 0, true, sc, &totals[4], b.err, s);  // totals[4] = logical blocks
}

void launch_lblocks(Batch& b, uint32_t* blk_kern, cudaStream_t s) {
  const int T = 256;
  if (!b.I) return;
  k_lblocks<<<(b.I + T - 1) / T, T, 0, s>>>(b, b.lleader, blk_kern);
  ++launch_counter();
  if (b.NLB) {
    k_lblock_edges<<<(b.NLB + T - 1) / T, T, 0, s>>>(b, blk_kern);
    ++launch_counter();
  }
}

}  // namespace gd
