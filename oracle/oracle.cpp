// CPU ORACLE for the GCN -> OpenCL decompiler.  TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded decompiler that follows the paper ("A method
// for decompilation of AMD GCN kernels to OpenCL") step by step, as its
// "Statement of the problem" lists them:
//   1. separation of body, configuration and kernel name  (Listing 2, Listing 1/3)
//   2. initialisation of registers and parameters from the ABI ("Search for memory accesses")
//   3. instruction processing: CFG, memory accesses, system values, arithmetic, types
//   4. control-flow graph -> region graph ("Search for control structures", Fig. 3)
//   5. OpenCL generation
// Where the paper is silent (missing figures, loops, exact output format) the
// readings written down beside each step are used; the CUDA path reproduces
// the same results with its own code.  Nothing here is shared with the CUDA
// path, and only tests, the smoke check and the benchmark's CPU baseline may
// call it.  Loops are an extension: the paper does not restore them.

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <thread>
#include <vector>

namespace {

// ============================================================================
// Text helpers
// ============================================================================
bool is_ws(char c) { return c == ' ' || c == '\t' || c == '\r'; }

std::string trim(const std::string& s) {
  size_t a = 0, b = s.size();
  while (a < b && is_ws(s[a])) ++a;
  while (b > a && is_ws(s[b - 1])) --b;
  return s.substr(a, b - a);
}

std::vector<std::string> split_ws(const std::string& s) {
  std::vector<std::string> out;
  size_t i = 0;
  while (i < s.size()) {
    while (i < s.size() && is_ws(s[i])) ++i;
    size_t j = i;
    while (j < s.size() && !is_ws(s[j])) ++j;
    if (j > i) out.push_back(s.substr(i, j - i));
    i = j;
  }
  return out;
}

std::vector<std::string> split_commas(const std::string& s) {
  std::vector<std::string> out;
  std::string cur;
  for (char c : s) {
    if (c == ',') {
      out.push_back(trim(cur));
      cur.clear();
    } else {
      cur += c;
    }
  }
  out.push_back(trim(cur));
  return out;
}

// parse a decimal (optionally negative) or 0x-hex integer; the whole token must be used
bool parse_int(const std::string& t, int64_t* v) {
  if (t.empty()) return false;
  size_t i = 0;
  bool neg = false;
  if (t[0] == '-') {
    neg = true;
    i = 1;
  }
  if (i >= t.size()) return false;
  uint64_t x = 0;
  if (t.size() > i + 2 && t[i] == '0' && (t[i + 1] == 'x' || t[i + 1] == 'X')) {
    i += 2;
    for (; i < t.size(); ++i) {
      char c = t[i];
      int d;
      if (c >= '0' && c <= '9') d = c - '0';
      else if (c >= 'a' && c <= 'f') d = c - 'a' + 10;
      else if (c >= 'A' && c <= 'F') d = c - 'A' + 10;
      else return false;
      x = x * 16 + (uint64_t)d;
      if (x > 0xFFFFFFFFull) return false;
    }
  } else {
    for (; i < t.size(); ++i) {
      char c = t[i];
      if (c < '0' || c > '9') return false;
      x = x * 10 + (uint64_t)(c - '0');
      if (x > 0xFFFFFFFFull) return false;
    }
  }
  *v = neg ? -(int64_t)x : (int64_t)x;
  return true;
}

// ============================================================================
// Step 1: body extraction (Listing 2).  Readings: rows are trimmed and the
// first word is compared; dispatch is on the parse state; rows before the first
// `.kernel` are ignored; a `.kernel` flushes the previous kernel whatever the
// state; blank rows and comment rows ('#', ';', "//") are skipped.
// ============================================================================
struct RawKernel {
  std::string name;
  std::vector<std::string> config;  // trimmed config rows
  std::vector<std::string> text;    // trimmed .text rows (labels and instructions)
};

bool is_comment(const std::string& r) {
  return r.empty() || r[0] == '#' || r[0] == ';' || (r.size() >= 2 && r[0] == '/' && r[1] == '/');
}

std::vector<RawKernel> extract_bodies(const char* text, size_t len) {
  std::vector<RawKernel> out;
  enum { START, KERNEL, CONFIG, INSTR } state = START;
  RawKernel cur;
  size_t pos = 0;
  while (pos < len) {
    size_t e = pos;
    while (e < len && text[e] != '\n') ++e;
    std::string row = trim(std::string(text + pos, e - pos));
    pos = e + 1;
    if (is_comment(row)) continue;
    std::vector<std::string> w = split_ws(row);
    if (w[0] == ".kernel") {
      if (state != START) out.push_back(cur);
      cur = RawKernel();
      cur.name = w.size() > 1 ? w[1] : std::string();
      state = KERNEL;
      continue;
    }
    if (state == START) continue;
    if (w[0] == ".config") state = CONFIG;
    else if (w[0] == ".text") state = INSTR;
    else if (state == CONFIG) cur.config.push_back(row);
    else if (state == INSTR) cur.text.push_back(row);
  }
  if (state != START) out.push_back(cur);
  return out;
}

// ============================================================================
// Step 1b: configuration (Listing 1, Listing 3).  `dims xyz` and `.dims x` are
// both accepted (dims = number of letters).  Every `.arg` takes an 8-byte slot
// of the kernel settings in declaration order; names beginning with "_." are
// the hidden arguments and are not printed.
// ============================================================================
enum Type : int { T_NONE = 0, T_INT = 1, T_UINT = 2, T_FLOAT = 3, T_LONG = 4, T_ULONG = 5, T_DOUBLE = 6, T_TOP32 = 7, T_TOP64 = 8 };

struct Arg {
  std::string name;
  bool hidden = false;
  bool pointer = false;
  bool is_const = false;
  int elem = T_NONE;  // pointee type for pointers, value type for scalars
  int space = 0;      // 0 global, 1 constant, 2 local
  int user_index = -1;
};

struct Config {
  int dims = 1;
  int cws[3] = {1, 1, 1};
  int sgprs = 104, vgprs = 256;
  bool useargs = false;
  std::vector<Arg> args;  // all .arg rows in order
  bool bad = false;
};

int type_from_name(const std::string& s) {
  if (s == "int") return T_INT;
  if (s == "uint") return T_UINT;
  if (s == "float") return T_FLOAT;
  if (s == "long") return T_LONG;
  if (s == "ulong") return T_ULONG;
  if (s == "double") return T_DOUBLE;
  return T_NONE;
}

Config parse_config(const std::vector<std::string>& rows) {
  Config c;
  int user = 0;
  for (const std::string& r : rows) {
    std::vector<std::string> w = split_ws(r);
    const std::string& k = w[0];
    if (k == ".dims" || k == "dims") {
      if (w.size() < 2) { c.bad = true; continue; }
      c.dims = (int)w[1].size();
      if (c.dims < 1 || c.dims > 3) c.bad = true;
    } else if (k == ".cws") {
      std::string rest = trim(r.substr(4));
      std::vector<std::string> f = split_commas(rest);
      for (size_t i = 0; i < f.size() && i < 3; ++i) {
        int64_t v;
        if (!parse_int(f[i], &v) || v < 1 || v > 1024) c.bad = true;
        else c.cws[i] = (int)v;
      }
    } else if (k == ".sgprsnum" || k == ".vgprsnum") {
      int64_t v;
      if (w.size() < 2 || !parse_int(w[1], &v) || v < 0 || v > 1024) { c.bad = true; continue; }
      if (k == ".sgprsnum") c.sgprs = (int)v;
      else c.vgprs = (int)v;
    } else if (k == ".useargs") {
      c.useargs = true;
    } else if (k == ".arg") {
      std::string rest = trim(r.substr(4));
      std::vector<std::string> f = split_commas(rest);
      Arg a;
      if (f.size() < 3) { c.bad = true; continue; }
      a.name = f[0];
      a.hidden = a.name.size() >= 2 && a.name[0] == '_' && a.name[1] == '.';
      std::string ty = f[2];
      if (!ty.empty() && ty.back() == '*') {
        a.pointer = true;
        a.elem = type_from_name(ty.substr(0, ty.size() - 1));
        std::string sp = f.size() > 3 ? f[3] : std::string("global");
        a.space = sp == "constant" ? 1 : (sp == "local" ? 2 : 0);
        a.is_const = f.size() > 4 && f[4] == "const";
      } else {
        a.elem = type_from_name(ty);
      }
      if (!a.hidden) {
        if (a.elem == T_NONE) c.bad = true;
        a.user_index = user++;
      }
      c.args.push_back(a);
    }
  }
  return c;
}

// ============================================================================
// Step 3a: instruction decoding ("The body extraction": prefix_root_suffix).
// The mnemonic table is the dialect; an unknown mnemonic is kept for inline asm.
// ============================================================================
enum Op : uint16_t {
  OP_UNKNOWN = 0,
  S_LOAD_DWORD = 1, S_LOAD_DWORDX2 = 2, S_LOAD_DWORDX4 = 3, S_WAITCNT = 4, S_MOV_B32 = 5,
  S_MUL_I32 = 6, S_LSHL_B32 = 7, S_ADD_U32 = 8,
  S_CMP_FIRST = 9,  // 9..20: s_cmp_{eq,lg,gt,lt,ge,le}_{u32,i32}
  S_AND_SAVEEXEC_B64 = 21, S_XOR_B64 = 22, S_OR_B64 = 23, S_OR_SAVEEXEC_B64 = 24,
  S_BRANCH = 25, S_CBRANCH_SCC0 = 26, S_CBRANCH_SCC1 = 27, S_CBRANCH_EXECZ = 28, S_ENDPGM = 29,
  V_MOV_B32 = 30, V_ADD_U32 = 31, V_SUB_U32 = 32, V_MUL_LO_U32 = 33, V_MAD_U32_U24 = 34,
  V_MUL_U32_U24 = 35, V_AND_B32 = 36, V_OR_B32 = 37, V_XOR_B32 = 38, V_LSHLREV_B32 = 39,
  V_LSHRREV_B32 = 40, V_ASHRREV_I32 = 41, V_ADD_F32 = 42, V_SUB_F32 = 43, V_MUL_F32 = 44,
  V_FMA_F32 = 45, V_CVT_F32_I32 = 46, V_CVT_F32_U32 = 47, V_CVT_F64_F32 = 48, V_CVT_F64_I32 = 49,
  V_CVT_F32_F64 = 50,
  V_CMP_FIRST = 51,  // 51..68: v_cmp_{eq,ne,gt,lt,ge,le}_{i32,u32,f32}
  V_ADD_CO_U32 = 69, V_ADDC_CO_U32 = 70, V_SUB_CO_U32 = 71, V_SUBB_CO_U32 = 72,
  V_LSHLREV_B64 = 73, V_ADD_F64 = 74, V_MUL_F64 = 75, V_FMA_F64 = 76,
  GLOBAL_LOAD_DWORD = 77, GLOBAL_LOAD_DWORDX2 = 78, GLOBAL_STORE_DWORD = 79, GLOBAL_STORE_DWORDX2 = 80,
  BUFFER_LOAD_DWORD = 81, BUFFER_STORE_DWORD = 82,
  V_CNDMASK_B32 = 83,  // the ternary: vD = vcc ? src1 : src0
  S_LSHR_B32 = 84, S_BFE_U32 = 85,  // scalar shift right and bit-field extract (get_num_groups, get_work_dim)
  // "The body extraction": FLAT instructions (prefix "flat", a VGPR pair holds the 64-bit
  // address) and the double-suffix V_MUL_HI family (result type, then operand type)
  FLAT_LOAD_DWORD = 86, FLAT_LOAD_DWORDX2 = 87, FLAT_STORE_DWORD = 88, FLAT_STORE_DWORDX2 = 89,
  V_MUL_HI_U32_U24 = 90, V_MUL_HI_I32_I24 = 91,
  // "The body extraction": data share operations (prefix "ds") on the LDS, the equivalent of
  // OpenCL local memory ("The AMD GCN architecture"), and the work-group barrier
  DS_READ_B32 = 92, DS_READ_B64 = 93, DS_WRITE_B32 = 94, DS_WRITE_B64 = 95, S_BARRIER = 96,
  OP_COUNT = 97
};

// comparison codes shared by s_cmp and v_cmp: eq, ne(lg/neq), gt, lt, ge, le
const char* kCmpSym[6] = {"==", "!=", ">", "<", ">=", "<="};

// operand signature letters:
//  V vgpr  W vgpr pair  s sgpr  p sgpr pair  q sgpr quad  S 32-bit source (v/s/const)
//  M 64-bit mask (sgpr pair, vcc or exec)  c vcc  o off  K constant  L label  * anything
struct OpInfo {
  const char* name;
  const char* sig;
};

std::vector<OpInfo> build_table() {
  std::vector<OpInfo> t(OP_COUNT, OpInfo{nullptr, nullptr});
  auto set = [&](int op, const char* n, const char* s) { t[op] = OpInfo{n, s}; };
  set(S_LOAD_DWORD, "s_load_dword", "s,p,K");
  set(S_LOAD_DWORDX2, "s_load_dwordx2", "p,p,K");
  set(S_LOAD_DWORDX4, "s_load_dwordx4", "q,p,K");
  set(S_WAITCNT, "s_waitcnt", "*");
  set(S_MOV_B32, "s_mov_b32", "s,S");
  set(S_MUL_I32, "s_mul_i32", "s,S,S");
  set(S_LSHL_B32, "s_lshl_b32", "s,S,S");
  set(S_ADD_U32, "s_add_u32", "s,S,S");
  set(S_LSHR_B32, "s_lshr_b32", "s,S,S");
  set(S_BFE_U32, "s_bfe_u32", "s,S,S");
  static const char* scc[6] = {"eq", "lg", "gt", "lt", "ge", "le"};
  static const char* sty[2] = {"u32", "i32"};
  static std::vector<std::string> names;
  names.reserve(64);
  for (int ty = 0; ty < 2; ++ty)
    for (int c = 0; c < 6; ++c) {
      names.push_back(std::string("s_cmp_") + scc[c] + "_" + sty[ty]);
      set(S_CMP_FIRST + 6 * ty + c, names.back().c_str(), "S,S");
    }
  set(S_AND_SAVEEXEC_B64, "s_and_saveexec_b64", "M,M");
  set(S_XOR_B64, "s_xor_b64", "M,M,M");
  set(S_OR_B64, "s_or_b64", "M,M,M");
  set(S_OR_SAVEEXEC_B64, "s_or_saveexec_b64", "M,M");
  set(S_BRANCH, "s_branch", "L");
  set(S_CBRANCH_SCC0, "s_cbranch_scc0", "L");
  set(S_CBRANCH_SCC1, "s_cbranch_scc1", "L");
  set(S_CBRANCH_EXECZ, "s_cbranch_execz", "L");
  set(S_ENDPGM, "s_endpgm", "");
  set(V_MOV_B32, "v_mov_b32", "V,S");
  set(V_ADD_U32, "v_add_u32", "V,S,S");
  set(V_SUB_U32, "v_sub_u32", "V,S,S");
  set(V_MUL_LO_U32, "v_mul_lo_u32", "V,S,S");
  set(V_MAD_U32_U24, "v_mad_u32_u24", "V,S,S,S");
  set(V_MUL_U32_U24, "v_mul_u32_u24", "V,S,S");
  set(V_AND_B32, "v_and_b32", "V,S,S");
  set(V_OR_B32, "v_or_b32", "V,S,S");
  set(V_XOR_B32, "v_xor_b32", "V,S,S");
  set(V_LSHLREV_B32, "v_lshlrev_b32", "V,S,S");
  set(V_LSHRREV_B32, "v_lshrrev_b32", "V,S,S");
  set(V_ASHRREV_I32, "v_ashrrev_i32", "V,S,S");
  set(V_ADD_F32, "v_add_f32", "V,S,S");
  set(V_SUB_F32, "v_sub_f32", "V,S,S");
  set(V_MUL_F32, "v_mul_f32", "V,S,S");
  set(V_FMA_F32, "v_fma_f32", "V,S,S,S");
  set(V_CVT_F32_I32, "v_cvt_f32_i32", "V,S");
  set(V_CVT_F32_U32, "v_cvt_f32_u32", "V,S");
  set(V_CVT_F64_F32, "v_cvt_f64_f32", "W,S");
  set(V_CVT_F64_I32, "v_cvt_f64_i32", "W,S");
  set(V_CVT_F32_F64, "v_cvt_f32_f64", "V,W");
  static const char* vcc[6] = {"eq", "ne", "gt", "lt", "ge", "le"};
  static const char* vty[3] = {"i32", "u32", "f32"};
  for (int ty = 0; ty < 3; ++ty)
    for (int c = 0; c < 6; ++c) {
      std::string cc = vcc[c];
      if (ty == 2 && c == 1) cc = "neq";
      names.push_back(std::string("v_cmp_") + cc + "_" + vty[ty]);
      set(V_CMP_FIRST + 6 * ty + c, names.back().c_str(), "c,S,S");
    }
  set(V_ADD_CO_U32, "v_add_co_u32", "V,c,S,S");
  set(V_ADDC_CO_U32, "v_addc_co_u32", "V,c,S,S,c");
  set(V_SUB_CO_U32, "v_sub_co_u32", "V,c,S,S");
  set(V_SUBB_CO_U32, "v_subb_co_u32", "V,c,S,S,c");
  set(V_LSHLREV_B64, "v_lshlrev_b64", "W,S,W");
  set(V_ADD_F64, "v_add_f64", "W,W,W");
  set(V_MUL_F64, "v_mul_f64", "W,W,W");
  set(V_FMA_F64, "v_fma_f64", "W,W,W,W");
  set(V_CNDMASK_B32, "v_cndmask_b32", "V,S,S,c");
  set(GLOBAL_LOAD_DWORD, "global_load_dword", "V,W,o");
  set(GLOBAL_LOAD_DWORDX2, "global_load_dwordx2", "W,W,o");
  set(GLOBAL_STORE_DWORD, "global_store_dword", "W,V,o");
  set(GLOBAL_STORE_DWORDX2, "global_store_dwordx2", "W,W,o");
  set(BUFFER_LOAD_DWORD, "buffer_load_dword", "V,o,q,s");
  set(BUFFER_STORE_DWORD, "buffer_store_dword", "V,o,q,s");
  set(FLAT_LOAD_DWORD, "flat_load_dword", "V,W");
  set(FLAT_LOAD_DWORDX2, "flat_load_dwordx2", "W,W");
  set(FLAT_STORE_DWORD, "flat_store_dword", "W,V");
  set(FLAT_STORE_DWORDX2, "flat_store_dwordx2", "W,W");
  set(V_MUL_HI_U32_U24, "v_mul_hi_u32_u24", "V,S,S");
  set(V_MUL_HI_I32_I24, "v_mul_hi_i32_i24", "V,S,S");
  set(DS_READ_B32, "ds_read_b32", "V,V");
  set(DS_READ_B64, "ds_read_b64", "W,V");
  set(DS_WRITE_B32, "ds_write_b32", "V,V");
  set(DS_WRITE_B64, "ds_write_b64", "V,W");
  set(S_BARRIER, "s_barrier", "");
  return t;
}

const std::vector<OpInfo>& table() {
  static std::vector<OpInfo> t = build_table();
  return t;
}

int lookup_op(const std::string& m) {
  const auto& t = table();
  for (int i = 1; i < OP_COUNT; ++i)
    if (t[i].name && m == t[i].name) return i;
  return OP_UNKNOWN;
}

// operand tags (InstrRec operand word: tag<<28 | count<<24 | payload)
enum Tag : uint32_t { TG_NONE = 0, TG_VGPR = 1, TG_SGPR = 2, TG_VCC = 3, TG_EXEC = 4, TG_ICONST = 5,
                      TG_FCONST = 6, TG_LIT = 7, TG_LABEL = 8, TG_OFF = 9 };
const uint32_t kInlineFloat[8] = {0x3f000000u, 0xbf000000u, 0x3f800000u, 0xbf800000u,
                                  0x40000000u, 0xc0000000u, 0x40800000u, 0xc0800000u};
const char* kInlineFloatText[8] = {"0.5", "-0.5", "1.0", "-1.0", "2.0", "-2.0", "4.0", "-4.0"};

enum Flag : uint8_t { F_UNSUPPORTED = 1, F_BAD = 2, F_REGRANGE = 4, F_NOLABEL = 8 };

#pragma pack(push, 1)
struct InstrRec {
  uint16_t op;
  uint8_t nops;
  uint8_t flags;
  uint32_t imm;
  uint32_t target;
  uint32_t opnd[5];
};
#pragma pack(pop)
static_assert(sizeof(InstrRec) == 32, "InstrRec is 32 bytes");

uint32_t enc(uint32_t tag, uint32_t count, uint32_t payload) {
  return (tag << 28) | ((count & 15u) << 24) | (payload & 0xFFFFFFu);
}
uint32_t tag_of(uint32_t o) { return o >> 28; }
uint32_t cnt_of(uint32_t o) { return (o >> 24) & 15u; }
uint32_t pay_of(uint32_t o) { return o & 0xFFFFFFu; }

// one operand word; returns false when the text is not an operand
bool parse_operand(const std::string& t, uint32_t* word, bool* is_lit, uint32_t* lit) {
  *is_lit = false;
  if (t == "vcc") { *word = enc(TG_VCC, 2, 0); return true; }
  if (t == "exec") { *word = enc(TG_EXEC, 2, 0); return true; }
  if (t == "off") { *word = enc(TG_OFF, 0, 0); return true; }
  if ((t[0] == 'v' || t[0] == 's') && t.size() >= 2) {
    uint32_t tag = t[0] == 'v' ? TG_VGPR : TG_SGPR;
    if (t[1] == '[') {
      size_t colon = t.find(':'), close = t.find(']');
      if (colon == std::string::npos || close != t.size() - 1 || colon > close) return false;
      int64_t a, b;
      if (!parse_int(t.substr(2, colon - 2), &a) || !parse_int(t.substr(colon + 1, close - colon - 1), &b))
        return false;
      if (t.substr(2, 2) == "0x" || a < 0 || b < a || b - a + 1 > 8 || b > 1023) return false;
      *word = enc(tag, (uint32_t)(b - a + 1), (uint32_t)a);
      return true;
    }
    bool digits = true;
    for (size_t i = 1; i < t.size(); ++i)
      if (t[i] < '0' || t[i] > '9') digits = false;
    if (digits) {
      int64_t a;
      if (!parse_int(t.substr(1), &a) || a > 1023) return false;
      *word = enc(tag, 1, (uint32_t)a);
      return true;
    }
    return false;
  }
  for (int i = 0; i < 8; ++i)
    if (t == kInlineFloatText[i]) { *word = enc(TG_FCONST, 1, (uint32_t)i); return true; }
  int64_t v;
  if (parse_int(t, &v)) {
    bool hex = t.find('x') != std::string::npos || t.find('X') != std::string::npos;
    if (!hex && v >= -16 && v <= 64) {
      *word = enc(TG_ICONST, 1, (uint32_t)v & 0xFFFFFFu);
      return true;
    }
    *word = enc(TG_LIT, 1, 0);
    *is_lit = true;
    *lit = (uint32_t)(uint64_t)v;
    return true;
  }
  return false;
}

int32_t iconst_value(uint32_t o) {
  uint32_t p = pay_of(o);
  return (p & 0x800000u) ? (int32_t)(p | 0xFF000000u) : (int32_t)p;
}

bool sig_ok(char s, uint32_t o) {
  uint32_t tg = tag_of(o), n = cnt_of(o);
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

struct Decoded {
  std::vector<InstrRec> ins;
  std::vector<std::string> text;  // instruction rows (for inline asm)
  bool bad = false;
};

Decoded decode(const std::vector<std::string>& rows, const Config& cfg) {
  Decoded d;
  std::map<std::string, uint32_t> labels;  // first definition wins
  std::vector<std::string> branch_label;
  for (const std::string& r : rows) {
    std::vector<std::string> w = split_ws(r);
    if (w.size() == 1 && w[0].size() >= 2 && w[0].back() == ':') {
      std::string nm = w[0].substr(0, w[0].size() - 1);
      if (!labels.count(nm)) labels[nm] = (uint32_t)d.ins.size();
      continue;
    }
    InstrRec rec;
    memset(&rec, 0, sizeof rec);
    rec.target = 0xFFFFFFFFu;
    const std::string& m = w[0];
    rec.op = (uint16_t)lookup_op(m);
    if (rec.op == OP_UNKNOWN) rec.flags |= F_UNSUPPORTED;
    std::string lbl;
    std::string rest = trim(r.substr(r.find(m) + m.size()));
    const char* sig = rec.op ? table()[rec.op].sig : "?";
    if (rec.op != S_WAITCNT && !rest.empty()) {
      std::vector<std::string> fields = split_commas(rest);
      int nlit = 0;
      for (size_t k = 0; k < fields.size(); ++k) {
        std::vector<std::string> sub = split_ws(fields[k]);
        if (sub.empty()) { rec.flags |= F_BAD; continue; }
        for (size_t q = 1; q < sub.size(); ++q) {  // modifiers: offset:K
          if (sub[q].compare(0, 7, "offset:") == 0) {
            int64_t v;
            if (!parse_int(sub[q].substr(7), &v) || v < 0) rec.flags |= F_BAD;
            else rec.imm = (uint32_t)v;
          }
        }
        uint32_t word = 0, lit = 0;
        bool is_lit = false;
        bool want_label = sig[0] == 'L';
        if (want_label) {
          lbl = sub[0];
          word = enc(TG_LABEL, 0, 0);
        } else if (!parse_operand(sub[0], &word, &is_lit, &lit)) {
          rec.flags |= F_BAD;
          continue;
        }
        if (is_lit) {
          if (nlit++) rec.flags |= F_BAD;
          rec.imm = lit;
        }
        if (rec.nops < 5) rec.opnd[rec.nops++] = word;
        else rec.flags |= F_BAD;
      }
    }
    // signature check
    if (rec.op && rec.op != S_WAITCNT) {
      int want = sig[0] ? (int)(strlen(sig) + 1) / 2 : 0;
      if (rec.nops != want) rec.flags |= F_BAD;
      else
        for (int k = 0; k < want; ++k)
          if (sig[2 * k] != 'L' && !sig_ok(sig[2 * k], rec.opnd[k])) rec.flags |= F_BAD;
      // the constant offset of a scalar load is its imm
      if ((rec.op == S_LOAD_DWORD || rec.op == S_LOAD_DWORDX2 || rec.op == S_LOAD_DWORDX4) && rec.nops == 3 &&
          tag_of(rec.opnd[2]) == TG_ICONST)
        rec.imm = (uint32_t)iconst_value(rec.opnd[2]);
      if ((rec.op == BUFFER_LOAD_DWORD || rec.op == BUFFER_STORE_DWORD) && (rec.imm & 3u)) rec.flags |= F_BAD;
      // a global or FLAT access with a constant byte offset reaches another element than its
      // address operand names; offsets are not folded into the address, so the instruction
      // stays inline assembly
      if (rec.op >= GLOBAL_LOAD_DWORD && rec.op <= GLOBAL_STORE_DWORDX2 && rec.imm) rec.op = OP_UNKNOWN;
      if (rec.op >= FLAT_LOAD_DWORD && rec.op <= FLAT_STORE_DWORDX2 && rec.imm) rec.op = OP_UNKNOWN;
      if (rec.op >= DS_READ_B32 && rec.op <= DS_WRITE_B64 && rec.imm) rec.op = OP_UNKNOWN;
      if (rec.op == OP_UNKNOWN) rec.flags |= F_UNSUPPORTED;
    }
    if (rec.op == S_WAITCNT) rec.nops = 0;
    // register ranges against the configuration
    for (int k = 0; k < rec.nops; ++k) {
      uint32_t o = rec.opnd[k], tg = tag_of(o);
      if (tg == TG_VGPR && pay_of(o) + cnt_of(o) > (uint32_t)cfg.vgprs) rec.flags |= F_REGRANGE;
      if (tg == TG_SGPR && pay_of(o) + cnt_of(o) > (uint32_t)cfg.sgprs) rec.flags |= F_REGRANGE;
    }
    d.ins.push_back(rec);
    d.text.push_back(r);
    branch_label.push_back(lbl);
  }
  for (size_t i = 0; i < d.ins.size(); ++i) {
    if (branch_label[i].empty()) continue;
    auto it = labels.find(branch_label[i]);
    if (it == labels.end()) d.ins[i].flags |= F_NOLABEL;
    else d.ins[i].target = it->second;
  }
  for (auto& r : d.ins)
    if (r.flags & (F_BAD | F_REGRANGE | F_NOLABEL)) d.bad = true;
  return d;
}

bool is_branch(int op) {
  return op == S_BRANCH || op == S_CBRANCH_SCC0 || op == S_CBRANCH_SCC1 || op == S_CBRANCH_EXECZ;
}

// ============================================================================
// Step 3b: the control-flow graph (first step of "Search for control
// structures").  Leaders: the first instruction, branch targets, and the
// instruction after a branch or s_endpgm.
// ============================================================================
const uint32_t NONE = 0xFFFFFFFFu;

#pragma pack(push, 1)
struct BlockRec {
  uint32_t first, end, succ0, succ1;
};
#pragma pack(pop)

struct PhysCfg {
  std::vector<uint32_t> block_of;
  std::vector<BlockRec> blocks;
};

PhysCfg physical_cfg(const Decoded& d) {
  PhysCfg g;
  uint32_t n = (uint32_t)d.ins.size();
  std::vector<char> leader(n + 1, 0);
  if (n) leader[0] = 1;
  for (uint32_t i = 0; i < n; ++i) {
    int op = d.ins[i].op;
    if (is_branch(op) && d.ins[i].target < n) leader[d.ins[i].target] = 1;
    if ((is_branch(op) || op == S_ENDPGM) && i + 1 < n) leader[i + 1] = 1;
  }
  g.block_of.assign(n, NONE);
  for (uint32_t i = 0; i < n; ++i) {
    if (leader[i]) g.blocks.push_back(BlockRec{i, i, NONE, NONE});
    g.block_of[i] = (uint32_t)g.blocks.size() - 1;
    g.blocks.back().end = i + 1;
  }
  for (auto& b : g.blocks) {
    const InstrRec& last = d.ins[b.end - 1];
    uint32_t ft = b.end < n ? g.block_of[b.end] : NONE;
    uint32_t tg = last.target < n ? g.block_of[last.target] : NONE;
    if (last.op == S_BRANCH) b.succ0 = tg;
    else if (is_branch(last.op)) { b.succ0 = ft; b.succ1 = tg; }
    else if (last.op != S_ENDPGM) b.succ0 = ft;
  }
  return g;
}

// ============================================================================
// Step 3c: exec-mask if / if-else forms -> standard form (Fig. 4, Fig. 5).
// Reading of the missing figures: a divergent if is
//   v_cmp; s_and_saveexec_b64 S, vcc; [s_cbranch_execz L]; <then>; L: s_or_b64 exec, exec, S
// and an if-else is
//   v_cmp; s_and_saveexec_b64 S, vcc; s_xor_b64 S, exec, S; [s_cbranch_execz La]; <then>;
//   [La:] s_or_saveexec_b64 S, S; s_xor_b64 exec, exec, S; [s_cbranch_execz Lb]; <else>;
//   [Lb:] s_or_b64 exec, exec, S
// with both branches present (first form), only the first (second form: label in
// the if part) or only the second (third form: label in the else part).  Forms
// two and three are first turned into the first form by inserting the missing
// (fake) label and conditional jump, then the first form is reduced to the
// standard form: a per-work-item branch on the compare result to the then part
// or the else part, and a jump from the end of the then part to the join.
// ============================================================================
enum Ctl : uint8_t { C_NORMAL = 0, C_DROP = 1, C_CBR = 2, C_JMP = 3, C_END = 4 };

struct ExecForm {
  uint32_t save, xor1, ez1, els, xor2, ez2, restore;
  bool fake_ez1 = false, fake_ez2 = false;  // inserted by the normalisation
};

struct LogicalCfg {
  std::vector<uint8_t> ctl;        // per instruction
  std::vector<uint32_t> ltarget;   // CBR taken target / JMP target (instruction index)
  std::vector<uint8_t> sense;      // CBR: taken when the condition equals sense
  std::vector<uint32_t> block_of;  // logical block per instruction (NONE for dropped)
  std::vector<BlockRec> blocks;
  std::vector<uint32_t> term;      // index of the last non-dropped instruction per block
  bool bad = false;
};

bool same_pair(uint32_t a, uint32_t b) { return tag_of(a) == TG_SGPR && a == b; }

LogicalCfg logical_cfg(const Decoded& d) {
  LogicalCfg L;
  uint32_t n = (uint32_t)d.ins.size();
  L.ctl.assign(n, C_NORMAL);
  L.ltarget.assign(n, NONE);
  L.sense.assign(n, 0);
  // match the forms with a stack
  std::vector<ExecForm> stack, forms;
  for (uint32_t i = 0; i < n; ++i) {
    const InstrRec& r = d.ins[i];
    switch (r.op) {
      case S_AND_SAVEEXEC_B64: {
        if (tag_of(r.opnd[0]) != TG_SGPR || tag_of(r.opnd[1]) != TG_VCC) { L.bad = true; break; }
        ExecForm f{i, NONE, NONE, NONE, NONE, NONE, NONE};
        stack.push_back(f);
        break;
      }
      case S_XOR_B64: {
        if (stack.empty()) { L.bad = true; break; }
        ExecForm& f = stack.back();
        uint32_t S = d.ins[f.save].opnd[0];
        if (f.els == NONE && f.xor1 == NONE && i == f.save + 1 && same_pair(r.opnd[0], S) &&
            tag_of(r.opnd[1]) == TG_EXEC && same_pair(r.opnd[2], S))
          f.xor1 = i;
        else if (f.els != NONE && f.xor2 == NONE && i == f.els + 1 && tag_of(r.opnd[0]) == TG_EXEC &&
                 tag_of(r.opnd[1]) == TG_EXEC && same_pair(r.opnd[2], S))
          f.xor2 = i;
        else
          L.bad = true;
        break;
      }
      case S_CBRANCH_EXECZ: {
        if (stack.empty()) { L.bad = true; break; }
        ExecForm& f = stack.back();
        if (f.els == NONE && f.ez1 == NONE && i == (f.xor1 != NONE ? f.xor1 : f.save) + 1) f.ez1 = i;
        else if (f.xor2 != NONE && f.ez2 == NONE && i == f.xor2 + 1) f.ez2 = i;
        else L.bad = true;
        break;
      }
      case S_OR_SAVEEXEC_B64: {
        if (stack.empty()) { L.bad = true; break; }
        ExecForm& f = stack.back();
        uint32_t S = d.ins[f.save].opnd[0];
        if (f.xor1 == NONE || f.els != NONE || !same_pair(r.opnd[0], S) || !same_pair(r.opnd[1], S)) {
          L.bad = true;
          break;
        }
        f.els = i;
        break;
      }
      case S_OR_B64: {
        if (stack.empty()) { L.bad = true; break; }
        ExecForm f = stack.back();
        uint32_t S = d.ins[f.save].opnd[0];
        if (tag_of(r.opnd[0]) != TG_EXEC || tag_of(r.opnd[1]) != TG_EXEC || !same_pair(r.opnd[2], S)) {
          L.bad = true;
          break;
        }
        if ((f.xor1 == NONE) != (f.els == NONE) || (f.els != NONE && f.xor2 == NONE)) { L.bad = true; break; }
        f.restore = i;
        stack.pop_back();
        forms.push_back(f);
        break;
      }
      default:
        break;
    }
  }
  if (!stack.empty()) L.bad = true;
  if (L.bad) return L;
  // normalisation to the first form: the second form (no branch over the else
  // part) and the third form (no branch over the then part) receive a fake
  // conditional jump and a fake label; the jump sits where the first form has
  // its s_cbranch_execz, the label before the exec restore that follows.
  for (ExecForm& f : forms) {
    if (f.els == NONE) continue;  // plain if: no else part, nothing to insert
    if (f.ez1 == NONE) { f.ez1 = f.xor1; f.fake_ez1 = true; }  // jump over the then part
    if (f.ez2 == NONE) { f.ez2 = f.xor2; f.fake_ez2 = true; }  // jump over the else part
  }
  // reduction of the first form to the standard form
  for (const ExecForm& f : forms) {
    L.ctl[f.save] = C_CBR;  // branch on the compare: work-items where it is false skip the then part
    L.sense[f.save] = 0;
    if (f.xor1 != NONE) L.ctl[f.xor1] = C_DROP;
    if (f.ez1 != NONE && !f.fake_ez1) L.ctl[f.ez1] = C_DROP;
    if (f.els != NONE) {
      L.ctl[f.els] = C_JMP;  // end of the then part: jump to the join
      L.ctl[f.xor2] = C_DROP;
      if (!f.fake_ez2) L.ctl[f.ez2] = C_DROP;
      uint32_t else_entry = (f.fake_ez2 ? f.xor2 : f.ez2) + 1;
      L.ltarget[f.save] = else_entry;
      L.ltarget[f.els] = f.restore + 1;
    } else {
      L.ltarget[f.save] = f.restore + 1;
    }
    L.ctl[f.restore] = C_DROP;
  }
  // plain branches and the end
  for (uint32_t i = 0; i < n; ++i) {
    int op = d.ins[i].op;
    if (op == S_BRANCH) { L.ctl[i] = C_JMP; L.ltarget[i] = d.ins[i].target; }
    if (op == S_CBRANCH_SCC0 || op == S_CBRANCH_SCC1) {
      L.ctl[i] = C_CBR;
      L.ltarget[i] = d.ins[i].target;
      L.sense[i] = op == S_CBRANCH_SCC1 ? 1 : 0;
    }
    if (op == S_ENDPGM) L.ctl[i] = C_END;
  }
  // targets resolve to the first instruction that is not dropped
  auto resolve = [&](uint32_t t) {
    while (t < n && L.ctl[t] == C_DROP) ++t;
    return t;
  };
  for (uint32_t i = 0; i < n; ++i)
    if (L.ltarget[i] != NONE) L.ltarget[i] = resolve(L.ltarget[i]);
  // logical leaders and blocks
  std::vector<char> leader(n + 1, 0);
  uint32_t first = resolve(0);
  if (first < n) leader[first] = 1;
  for (uint32_t i = 0; i < n; ++i) {
    if (L.ctl[i] == C_CBR || L.ctl[i] == C_JMP) {
      if (L.ltarget[i] < n) leader[L.ltarget[i]] = 1;
    }
    if (L.ctl[i] == C_CBR || L.ctl[i] == C_JMP || L.ctl[i] == C_END) {
      uint32_t nx = resolve(i + 1);
      if (nx < n) leader[nx] = 1;
    }
  }
  L.block_of.assign(n, NONE);
  for (uint32_t i = 0; i < n; ++i) {
    if (leader[i]) {
      L.blocks.push_back(BlockRec{i, i + 1, NONE, NONE});
      L.term.push_back(i);
    }
    if (L.blocks.empty()) continue;
    if (L.ctl[i] != C_DROP) {
      L.block_of[i] = (uint32_t)L.blocks.size() - 1;
      L.term.back() = i;
    }
  }
  for (size_t b = 0; b < L.blocks.size(); ++b)
    L.blocks[b].end = b + 1 < L.blocks.size() ? L.blocks[b + 1].first : n;
  for (size_t b = 0; b < L.blocks.size(); ++b) {
    BlockRec& B = L.blocks[b];
    uint32_t t = L.term[b];
    uint32_t nx = resolve(t + 1);
    uint32_t ft = nx < n ? L.block_of[nx] : NONE;
    uint32_t tg = L.ltarget[t] < n ? L.block_of[L.ltarget[t]] : NONE;
    switch (L.ctl[t]) {
      case C_CBR: B.succ0 = ft; B.succ1 = tg == ft ? NONE : tg; break;
      case C_JMP: B.succ0 = tg; break;
      case C_END: break;
      default: B.succ0 = ft; break;
    }
  }
  return L;
}

// ============================================================================
// Steps 2 and 3d: registers, versions and joins.
// The Register record of the paper (version, type, integrity) becomes a value
// reference: which definition (a node id, or a join version) the register holds
// and which part of it (entire / low_part / high_part of a 64-bit value).
// Registers are initialised from the ABI: v0..v2 = get_local_id(0..2),
// s6..s8 = get_group_id(0..2) with .useargs, s[4:5] = settings pointer,
// s[0:1] = dispatch packet pointer.
// At a block with several predecessors a register whose definitions differ
// receives a new version (a join); versions that are used become variables.
// ============================================================================
enum Part : uint32_t { P_ENTIRE = 0, P_LO = 1, P_HI = 2 };
const uint32_t ID_PHI = 1u << 28, ID_LEAF = 2u << 28;
const uint32_t LEAF_UNDEF = 0, LEAF_LID = 1, LEAF_GRP = 2, LEAF_KARG = 3, LEAF_DISP = 4;
const uint32_t TOP = 0xFFFFFFFFu;  // unvisited

uint32_t ref(uint32_t id, uint32_t part) { return (id << 2) | part; }
uint32_t rid(uint32_t r) { return r >> 2; }
uint32_t rpart(uint32_t r) { return r & 3u; }
uint32_t node_ref(uint32_t instr, uint32_t slot, uint32_t part) { return ref(4 * instr + slot, part); }
uint32_t leaf_ref(uint32_t kind, uint32_t k, uint32_t part) { return ref(ID_LEAF | (kind << 8) | k, part); }
uint32_t phi_ref(uint32_t block, uint32_t reg) { return ref(ID_PHI | (block << 10) | reg, P_ENTIRE); }
const uint32_t UNDEF = (ID_LEAF << 2);  // leaf_ref(LEAF_UNDEF, 0, 0)
bool is_node(uint32_t r) { return r != TOP && (rid(r) >> 28) == 0; }
bool is_phi(uint32_t r) { return r != TOP && (rid(r) >> 28) == 1; }
bool is_leaf(uint32_t r) { return r != TOP && (rid(r) >> 28) == 2; }

struct Regs {
  uint32_t vgprs, sgprs, nspill, R;
  uint32_t v(uint32_t i) const { return i; }
  uint32_t s(uint32_t i) const { return vgprs + i; }
  uint32_t vcc() const { return vgprs + sgprs; }
  uint32_t scc() const { return vgprs + sgprs + 1; }
  uint32_t spill(uint32_t k) const { return vgprs + sgprs + 2 + k; }
};

// register index list of an operand word
std::vector<uint32_t> regs_of(const Regs& R, uint32_t o) {
  std::vector<uint32_t> v;
  uint32_t tg = tag_of(o), n = cnt_of(o), p = pay_of(o);
  if (tg == TG_VGPR) for (uint32_t k = 0; k < n; ++k) v.push_back(R.v(p + k));
  if (tg == TG_SGPR) for (uint32_t k = 0; k < n; ++k) v.push_back(R.s(p + k));
  if (tg == TG_VCC) v.push_back(R.vcc());
  return v;
}

bool is64_result(int op) {
  return op == S_LOAD_DWORDX2 || op == V_CVT_F64_F32 || op == V_CVT_F64_I32 || op == V_LSHLREV_B64 ||
         op == V_ADD_F64 || op == V_MUL_F64 || op == V_FMA_F64 || op == GLOBAL_LOAD_DWORDX2 ||
         op == FLAT_LOAD_DWORDX2 || op == DS_READ_B64;
}
bool is_scmp(int op) { return op >= S_CMP_FIRST && op < S_CMP_FIRST + 12; }
bool is_vcmp(int op) { return op >= V_CMP_FIRST && op < V_CMP_FIRST + 18; }

struct Def {
  uint32_t reg, val;
};

// definitions of instruction i (the paper's register update); `fused` says
// whether an add-with-carry / subtract-with-borrow completes a 64-bit add/sub
std::vector<Def> defs_of(const Decoded& d, const LogicalCfg& L, const Regs& R, uint32_t i, bool fused,
                         uint32_t co_dst) {
  std::vector<Def> out;
  if (L.ctl[i] != C_NORMAL) return out;  // bookkeeping, branches, end
  const InstrRec& r = d.ins[i];
  int op = r.op;
  auto dst = [&](int k) { return regs_of(R, r.opnd[k]); };
  switch (op) {
    case S_WAITCNT: break;
    case S_LOAD_DWORD: out.push_back({dst(0)[0], node_ref(i, 0, P_ENTIRE)}); break;
    case S_LOAD_DWORDX4: {
      auto g = dst(0);
      out.push_back({g[0], node_ref(i, 0, P_LO)});
      out.push_back({g[1], node_ref(i, 0, P_HI)});
      out.push_back({g[2], node_ref(i, 1, P_LO)});
      out.push_back({g[3], node_ref(i, 1, P_HI)});
      break;
    }
    case S_ADD_U32: case S_MUL_I32: case S_LSHL_B32: case S_LSHR_B32: case S_BFE_U32:
      out.push_back({dst(0)[0], node_ref(i, 0, P_ENTIRE)});
      out.push_back({R.scc(), UNDEF});
      break;
    case V_ADD_CO_U32: case V_SUB_CO_U32:
      out.push_back({dst(0)[0], node_ref(i, 0, P_ENTIRE)});
      out.push_back({R.vcc(), node_ref(i, 3, P_ENTIRE)});
      break;
    case V_ADDC_CO_U32: case V_SUBB_CO_U32:
      if (fused) {
        out.push_back({co_dst, node_ref(i, 0, P_LO)});
        out.push_back({dst(0)[0], node_ref(i, 0, P_HI)});
      } else {
        out.push_back({dst(0)[0], node_ref(i, 0, P_ENTIRE)});
      }
      out.push_back({R.vcc(), UNDEF});
      break;
    case GLOBAL_STORE_DWORD: case GLOBAL_STORE_DWORDX2: case FLAT_STORE_DWORD: case FLAT_STORE_DWORDX2:
    case DS_WRITE_B32: case DS_WRITE_B64: case S_BARRIER: break;
    case BUFFER_STORE_DWORD: out.push_back({R.spill(r.imm / 4), node_ref(i, 0, P_ENTIRE)}); break;
    case OP_UNKNOWN: {
      if (r.nops == 0) break;
      auto g = dst(0);
      if (g.size() == 2) {
        out.push_back({g[0], node_ref(i, 0, P_LO)});
        out.push_back({g[1], node_ref(i, 0, P_HI)});
      } else {
        for (uint32_t x : g) out.push_back({x, node_ref(i, 0, P_ENTIRE)});
      }
      break;
    }
    default:
      if (is_scmp(op)) { out.push_back({R.scc(), node_ref(i, 0, P_ENTIRE)}); break; }
      if (is_vcmp(op)) { out.push_back({R.vcc(), node_ref(i, 0, P_ENTIRE)}); break; }
      if (is64_result(op)) {
        auto g = dst(0);
        out.push_back({g[0], node_ref(i, 0, P_LO)});
        out.push_back({g[1], node_ref(i, 0, P_HI)});
      } else {
        out.push_back({dst(0)[0], node_ref(i, 0, P_ENTIRE)});
      }
  }
  return out;
}

// ============================================================================
// Expression nodes (Step 3: memory accesses, system values, arithmetic).
// Node id = 4 * instruction + slot: slot 0 is the instruction's result, slots
// 1..3 hold the pair or constant built for its source operands 0..2 (slot 3 is
// also the carry of an add/sub with carry-out; slot 1 the second half of a
// 4-dword scalar load).
// ============================================================================
enum NodeKind : uint8_t { N_NONE = 0, N_OP = 1, N_CONST = 2, N_PAIR = 3, N_CARRY = 4, N_SLOAD64B = 5 };

struct Node {
  uint8_t kind = N_NONE;
  uint16_t op = 0;
  uint8_t nsrc = 0;
  uint32_t src[3] = {TOP, TOP, TOP};  // value references
  uint32_t cval = 0;                  // constant bits / scalar load offset
  bool fused = false;                 // 64-bit add/sub formed from a carry pair
};

// ============================================================================
// Per-kernel decompiler state
// ============================================================================
struct Kernel {
  std::string name;
  Config cfg;
  Decoded dec;
  PhysCfg pcfg;
  LogicalCfg lcfg;
  Regs R{};
  std::vector<std::vector<uint32_t>> in;   // in-state per block
  std::vector<std::vector<uint32_t>> out;  // out-state per block
  std::vector<std::vector<uint32_t>> preds;
  std::vector<Node> nodes;                 // 4 per instruction
  std::vector<char> fusedv;                // per instruction: 64-bit carry pair completed
  std::vector<uint32_t> co_dst;            // per instruction: register of the low half
  std::vector<uint32_t> co_idx;            // per instruction: the add/sub with carry-out
  int status = 0;
  std::string out_text;
  uint32_t sweeps = 0, undef_reads = 0, n_vars = 0, n_phis = 0, trivial_phis = 0;
  bool capped = false;
};

enum Status { ST_OK = 0, ST_PARTIAL = 1, ST_PARSE_ERROR = 2, ST_FIXPOINT_CAP = 3 };

void find_fusions(Kernel& K) {
  const auto& d = K.dec;
  uint32_t n = (uint32_t)d.ins.size();
  K.fusedv.assign(n, 0);
  K.co_dst.assign(n, NONE);
  K.co_idx.assign(n, NONE);
  for (uint32_t i = 0; i < n; ++i) {
    int op = d.ins[i].op;
    if (op != V_ADDC_CO_U32 && op != V_SUBB_CO_U32) continue;
    if (K.lcfg.ctl[i] != C_NORMAL) continue;
    uint32_t b = K.lcfg.block_of[i];
    if (b == NONE) continue;
    // last instruction before i in the same block that defines vcc
    int j = -1;
    for (int k = (int)i - 1; k >= (int)K.lcfg.blocks[b].first; --k) {
      if (K.lcfg.block_of[k] != b || K.lcfg.ctl[k] != C_NORMAL) continue;
      bool defs_vcc = false;
      int ok = d.ins[k].op;
      if (ok == V_ADD_CO_U32 || ok == V_SUB_CO_U32 || ok == V_ADDC_CO_U32 || ok == V_SUBB_CO_U32 || is_vcmp(ok))
        defs_vcc = true;
      if (ok == OP_UNKNOWN && d.ins[k].nops && tag_of(d.ins[k].opnd[0]) == TG_VCC) defs_vcc = true;
      if (defs_vcc) { j = k; break; }
    }
    int want = op == V_ADDC_CO_U32 ? V_ADD_CO_U32 : V_SUB_CO_U32;
    if (j < 0 || d.ins[j].op != want) continue;
    // the two 64-bit operands take the instruction's slots 1 and 2, which leaves one
    // slot (3) for a constant high source: two constants are left unfused
    auto is_reg = [&](uint32_t o) {
      uint32_t tg = tag_of(o);
      return tg == TG_VGPR || tg == TG_SGPR || tg == TG_VCC;
    };
    if (!is_reg(d.ins[i].opnd[2]) && !is_reg(d.ins[i].opnd[3])) continue;
    uint32_t lo = K.R.v(pay_of(d.ins[j].opnd[0]));
    uint32_t hi = K.R.v(pay_of(d.ins[i].opnd[0]));
    if (lo == hi) continue;
    // the low half must still be in its register
    bool clobbered = false;
    for (uint32_t k = (uint32_t)j + 1; k < i && !clobbered; ++k) {
      if (K.lcfg.block_of[k] != b) continue;
      for (const Def& df : defs_of(d, K.lcfg, K.R, k, K.fusedv[k], K.co_dst[k]))
        if (df.reg == lo) clobbered = true;
    }
    if (clobbered) continue;
    K.fusedv[i] = 1;
    K.co_dst[i] = lo;
    K.co_idx[i] = (uint32_t)j;
  }
}

std::vector<uint32_t> entry_state(const Kernel& K) {
  std::vector<uint32_t> s(K.R.R, UNDEF);
  for (int dd = 0; dd < K.cfg.dims && dd < 3; ++dd) {
    if ((uint32_t)dd < K.R.vgprs) s[K.R.v(dd)] = leaf_ref(LEAF_LID, dd, P_ENTIRE);
    if (K.cfg.useargs && (uint32_t)(6 + dd) < K.R.sgprs) s[K.R.s(6 + dd)] = leaf_ref(LEAF_GRP, dd, P_ENTIRE);
  }
  if (K.R.sgprs > 5) {
    s[K.R.s(4)] = leaf_ref(LEAF_KARG, 0, P_LO);
    s[K.R.s(5)] = leaf_ref(LEAF_KARG, 0, P_HI);
  }
  if (K.R.sgprs > 1) {  // the dispatch packet pointer (global size, dimension count)
    s[K.R.s(0)] = leaf_ref(LEAF_DISP, 0, P_LO);
    s[K.R.s(1)] = leaf_ref(LEAF_DISP, 0, P_HI);
  }
  return s;
}

// Versions at joins (minimal SSA, Cytron et al.): register r receives a new
// version at block B exactly when B lies in the iterated dominance frontier
// of the blocks that define r (the entry block defines every register with
// its ABI value).  A block without a new version inherits the value at the
// end of its immediate dominator.  This placement is unique, whatever order
// an implementation visits the blocks in.
void dominators(const LogicalCfg& L, const std::vector<std::vector<uint32_t>>& preds, std::vector<uint32_t>* rpo_out,
                std::vector<uint32_t>* idom_out) {
  uint32_t nb = (uint32_t)L.blocks.size();
  std::vector<uint32_t> rpo_index(nb, NONE), order;
  // iterative depth-first search: successors in (fall-through, taken) order
  std::vector<char> seen(nb, 0);
  std::vector<std::pair<uint32_t, int>> st;
  if (nb) { st.push_back({0, 0}); seen[0] = 1; }
  while (!st.empty()) {
    auto& [b, k] = st.back();
    uint32_t s = NONE;
    while (k < 2 && s == NONE) {
      uint32_t c = k == 0 ? L.blocks[b].succ0 : L.blocks[b].succ1;
      ++k;
      if (c != NONE && !seen[c]) s = c;
    }
    if (s != NONE) { seen[s] = 1; st.push_back({s, 0}); }
    else { order.push_back(b); st.pop_back(); }
  }
  std::reverse(order.begin(), order.end());
  for (uint32_t i = 0; i < order.size(); ++i) rpo_index[order[i]] = i;
  std::vector<uint32_t> idom(nb, NONE);
  if (nb) idom[0] = 0;
  auto intersect = [&](uint32_t a, uint32_t b) {
    while (a != b) {
      while (rpo_index[a] > rpo_index[b]) a = idom[a];
      while (rpo_index[b] > rpo_index[a]) b = idom[b];
    }
    return a;
  };
  bool changed = true;
  while (changed) {
    changed = false;
    for (uint32_t i = 1; i < order.size(); ++i) {
      uint32_t b = order[i], nd = NONE;
      for (uint32_t p : preds[b]) {
        if (rpo_index[p] == NONE || idom[p] == NONE) continue;
        nd = nd == NONE ? p : intersect(p, nd);
      }
      if (nd != idom[b]) { idom[b] = nd; changed = true; }
    }
  }
  *rpo_out = order;
  *idom_out = idom;
}

void dataflow(Kernel& K) {
  const auto& L = K.lcfg;
  uint32_t nb = (uint32_t)L.blocks.size();
  K.preds.assign(nb, {});
  for (uint32_t b = 0; b < nb; ++b) {
    if (L.blocks[b].succ0 != NONE) K.preds[L.blocks[b].succ0].push_back(b);
    if (L.blocks[b].succ1 != NONE) K.preds[L.blocks[b].succ1].push_back(b);
  }
  K.in.assign(nb, std::vector<uint32_t>(K.R.R, TOP));
  K.out.assign(nb, std::vector<uint32_t>(K.R.R, TOP));
  if (!nb) return;
  if (!K.preds[0].empty()) { K.capped = true; return; }  // the entry may not be a loop header
  std::vector<uint32_t> rpo, idom;
  dominators(L, K.preds, &rpo, &idom);
  // dominance frontiers
  std::vector<std::vector<uint32_t>> df(nb);
  for (uint32_t b = 0; b < nb; ++b) {
    if (idom[b] == NONE || K.preds[b].size() < 2) continue;
    for (uint32_t p : K.preds[b]) {
      if (idom[p] == NONE) continue;  // unreachable predecessor
      uint32_t x = p;
      while (x != idom[b]) {
        if (std::find(df[x].begin(), df[x].end(), b) == df[x].end()) df[x].push_back(b);
        x = idom[x];
      }
    }
  }
  // last definition of each register in each block
  std::vector<std::map<uint32_t, uint32_t>> local(nb);
  std::vector<std::vector<uint32_t>> defblocks(K.R.R);
  for (uint32_t b = 0; b < nb; ++b) {
    for (uint32_t i = L.blocks[b].first; i < L.blocks[b].end; ++i) {
      if (L.block_of[i] != b) continue;
      for (const Def& df_ : defs_of(K.dec, L, K.R, i, K.fusedv[i], K.co_dst[i])) local[b][df_.reg] = df_.val;
    }
    for (auto& kv : local[b]) defblocks[kv.first].push_back(b);
  }
  // iterated dominance frontier per register
  std::vector<std::vector<char>> has_phi(nb, std::vector<char>(K.R.R, 0));
  for (uint32_t r = 0; r < K.R.R; ++r) {
    std::vector<char> isdef(nb, 0);
    std::vector<uint32_t> work = defblocks[r];
    work.push_back(0);
    for (uint32_t x : work) isdef[x] = 1;
    while (!work.empty()) {
      uint32_t x = work.back();
      work.pop_back();
      for (uint32_t y : df[x]) {
        if (has_phi[y][r]) continue;
        has_phi[y][r] = 1;
        if (!isdef[y]) { isdef[y] = 1; work.push_back(y); }
      }
    }
  }
  // values in reverse postorder (every immediate dominator comes first)
  std::vector<uint32_t> entry = entry_state(K);
  for (uint32_t b : rpo) {
    for (uint32_t r = 0; r < K.R.R; ++r) {
      if (has_phi[b][r]) K.in[b][r] = phi_ref(b, r);
      else K.in[b][r] = b == 0 ? entry[r] : K.out[idom[b]][r];
    }
    K.out[b] = K.in[b];
    for (auto& kv : local[b]) K.out[b][kv.first] = kv.second;
  }
  K.sweeps = 1;
}

// node creation: walk each block from its in-state and record every node
void build_nodes(Kernel& K) {
  const auto& d = K.dec;
  const auto& L = K.lcfg;
  uint32_t n = (uint32_t)d.ins.size();
  K.nodes.assign(4 * (size_t)n, Node());
  for (size_t b = 0; b < L.blocks.size(); ++b) {
    std::vector<uint32_t> st = K.in[b];
    for (uint32_t& x : st)
      if (x == TOP) x = UNDEF;
    for (uint32_t i = L.blocks[b].first; i < L.blocks[b].end; ++i) {
      if (L.block_of[i] != b) continue;
      const InstrRec& r = d.ins[i];
      int op = r.op;
      // source operands (by signature position)
      std::vector<uint32_t> srcs;
      auto read32 = [&](uint32_t o, uint32_t slot) -> uint32_t {
        uint32_t tg = tag_of(o);
        if (tg == TG_VGPR) return st[K.R.v(pay_of(o))];
        if (tg == TG_SGPR) return st[K.R.s(pay_of(o))];
        if (tg == TG_VCC) return st[K.R.vcc()];
        Node& c = K.nodes[4 * i + slot];
        c.kind = N_CONST;
        c.cval = tg == TG_ICONST ? (uint32_t)iconst_value(o) : (tg == TG_FCONST ? kInlineFloat[pay_of(o)] : r.imm);
        return node_ref(i, slot, P_ENTIRE);
      };
      auto pair_of = [&](uint32_t lo, uint32_t hi, uint32_t slot) -> uint32_t {
        if (is_node(lo) || is_leaf(lo) || is_phi(lo))
          if (rpart(lo) == P_LO && hi == ((lo & ~3u) | P_HI)) return lo & ~3u;
        Node& p = K.nodes[4 * i + slot];
        p.kind = N_PAIR;
        p.nsrc = 2;
        p.src[0] = lo;
        p.src[1] = hi;
        return node_ref(i, slot, P_ENTIRE);
      };
      auto read64 = [&](uint32_t o, uint32_t slot) -> uint32_t {
        auto g = regs_of(K.R, o);
        return pair_of(st[g[0]], st[g[1]], slot);
      };
      Node& nd = K.nodes[4 * i];
      if (L.ctl[i] == C_NORMAL || L.ctl[i] == C_CBR) {
        nd.kind = N_OP;
        nd.op = (uint16_t)op;
      }
      if (L.ctl[i] == C_CBR) {  // the branch condition (vcc for the exec forms, scc otherwise)
        nd.nsrc = 1;
        nd.src[0] = op == S_AND_SAVEEXEC_B64 ? st[K.R.vcc()] : st[K.R.scc()];
      } else if (L.ctl[i] == C_NORMAL) {
        const char* sig = op ? table()[op].sig : "";
        int sidx = 0;
        switch (op) {
          case S_WAITCNT: break;
          case S_LOAD_DWORD: case S_LOAD_DWORDX2: case S_LOAD_DWORDX4:
            // slot 2 holds a split base pair; slot 1 is the second 8 bytes of x4
            srcs.push_back(read64(r.opnd[1], 2));
            nd.cval = r.imm;
            break;
          case BUFFER_STORE_DWORD: srcs.push_back(read32(r.opnd[0], 1)); break;
          case BUFFER_LOAD_DWORD: srcs.push_back(st[K.R.spill(r.imm / 4)]); break;
          case V_ADDC_CO_U32: case V_SUBB_CO_U32: {
            // fused: slots 1 and 2 hold the operand pairs, so the (at most one) constant
            // high source sits in slot 3
            bool f = K.fusedv[i] != 0;
            uint32_t a = read32(r.opnd[2], f ? 3 : 1), bsrc = read32(r.opnd[3], f ? 3 : 2);
            if (f) {
              const Node& lo = K.nodes[4 * (size_t)K.co_idx[i]];
              srcs.push_back(pair_of(lo.src[0], a, 1));
              srcs.push_back(pair_of(lo.src[1], bsrc, 2));
              nd.fused = true;
            } else {
              srcs.push_back(a);
              srcs.push_back(bsrc);
              srcs.push_back(st[K.R.vcc()]);
            }
            break;
          }
          case OP_UNKNOWN:
            for (int k = 1; k < r.nops && sidx < 3; ++k) {
              uint32_t tg = tag_of(r.opnd[k]);
              if (tg == TG_VGPR || tg == TG_SGPR || tg == TG_VCC) {
                auto g = regs_of(K.R, r.opnd[k]);
                srcs.push_back(g.size() == 2 ? pair_of(st[g[0]], st[g[1]], 1 + sidx) : st[g[0]]);
                ++sidx;
              }
            }
            break;
          default: {
            // generic: every operand after the destination(s) that is a source
            int nop = (int)(strlen(sig) + 1) / 2;
            for (int k = 0; k < nop; ++k) {
              char s = sig[2 * k];
              bool is_dst = (k == 0 && (s == 'V' || s == 'W' || s == 's' || s == 'p' || s == 'q' || s == 'c')) ||
                            (k == 1 && s == 'c' && (op == V_ADD_CO_U32 || op == V_SUB_CO_U32));
              if (op == GLOBAL_STORE_DWORD || op == GLOBAL_STORE_DWORDX2 || op == FLAT_STORE_DWORD ||
                  op == FLAT_STORE_DWORDX2 || op == DS_WRITE_B32 || op == DS_WRITE_B64)
                is_dst = false;
              if (is_scmp(op)) is_dst = false;
              if (is_dst || s == 'o') continue;
              uint32_t slot = 1 + (uint32_t)srcs.size();
              if (s == 'W' || s == 'p') srcs.push_back(read64(r.opnd[k], slot));
              else srcs.push_back(read32(r.opnd[k], slot));
            }
          }
        }
        nd.nsrc = (uint8_t)srcs.size();
        for (size_t k = 0; k < srcs.size() && k < 3; ++k) nd.src[k] = srcs[k];
        if (op == S_LOAD_DWORDX4) {
          Node& h = K.nodes[4 * i + 1];
          h.kind = N_SLOAD64B;
          h.nsrc = 1;
          h.src[0] = nd.src[0];
          h.cval = r.imm + 8;
        }
        if (op == V_ADD_CO_U32 || op == V_SUB_CO_U32) {
          Node& c = K.nodes[4 * i + 3];
          c.kind = N_CARRY;
        }
      }
      for (const Def& df : defs_of(d, L, K.R, i, K.fusedv[i], K.co_dst[i])) st[df.reg] = df.val;
    }
  }
}

}  // namespace

namespace {

// ============================================================================
// Value forwarding: a register copy (v_mov/s_mov, spill store/load) is the
// value it copies; a 64-bit pair whose halves are the low and high part of the
// same 64-bit value is that value (the integrity field of the paper's Register).
// ============================================================================
bool is_copy(const Node& n) {
  return n.kind == N_OP && (n.op == V_MOV_B32 || n.op == S_MOV_B32 || n.op == BUFFER_STORE_DWORD ||
                            n.op == BUFFER_LOAD_DWORD);
}

uint32_t fwd(const Kernel& K, uint32_t r, int depth = 0) {
  for (int step = 0; step < 512 && depth < 64; ++step) {
    if (r == TOP) return UNDEF;
    if (!is_node(r)) return r;
    const Node& n = K.nodes[rid(r)];
    uint32_t part = rpart(r);
    if (is_copy(n) && part == P_ENTIRE) { r = n.src[0]; continue; }
    if (n.kind == N_PAIR) {
      if (part == P_LO) { r = n.src[0]; continue; }
      if (part == P_HI) { r = n.src[1]; continue; }
      uint32_t lo = fwd(K, n.src[0], depth + 1), hi = fwd(K, n.src[1], depth + 1);
      if ((is_node(lo) || is_leaf(lo)) && rpart(lo) == P_LO && hi == ((lo & ~3u) | P_HI)) return lo & ~3u;
      return r;
    }
    return r;
  }
  return r;
}

// ============================================================================
// System values ("Search for memory accesses", steps one to five) and kernel
// arguments.  s_load from the settings pointer s[4:5]: offsets 0x0/0x8/0x10 are
// get_global_offset(0..2) (64-bit, used through their low part), later 8-byte
// slots are the kernel arguments in declaration order.  The work-group size is
// the .cws constant; the chains
//   group_id(d) * cws(d) + local_id(d)            -> get_global_id(d) - get_global_offset(d)
//   (that) + low part of get_global_offset(d)     -> get_global_id(d)
// are recognised with the multiplication as s_mul_i32, s_lshl_b32 by log2(cws)
// or folded into v_mad_u32_u24, in either operand order.
// The global size, the number of groups and the dimension count come from a
// second pointer, s[0:1], to the dispatch packet (the settings block cannot hold
// both the offsets and the sizes at 0x10):
//   s_load_dword from s[0:1] + 0xc/0x10/0x14     -> get_global_size(0/1/2)
//   (that) >> log2(cws(d)), cws(d) a power of two  -> get_num_groups(d)
//     (global size / work-group size; the paper gives no instruction for the division)
//   s_bfe_u32 of the dword at s[0:1] + 0x0 with field 0x20010 (offset 16, width 2)
//                                                  -> get_work_dim()
// ============================================================================
enum Cls { K_NONE, K_LID, K_GRP, K_KARG, K_UNDEF, K_GOFS64, K_GOFSLO, K_MULGRP, K_GIDNO, K_GID, K_ARGPTR,
           K_ARG32, K_ARG64, K_CONST32, K_CONST64,
           K_DISP,    // the dispatch packet pointer s[0:1]
           K_DISP0,   // its first dword (header and setup; an intermediate, like K_MULGRP)
           K_GSIZE,   // get_global_size(d)
           K_NGRP,    // get_num_groups(d)
           K_WDIM,    // get_work_dim()
           K_LPTR };  // the LDS address of a __local pointer argument (the low dword of its slot)
struct ClsV {
  int c = K_NONE;
  int k = 0;
};

int log2_exact(int v) {
  for (int i = 0; i < 31; ++i)
    if ((1 << i) == v) return i;
  return -1;
}

bool is_64type(int t) { return t == T_LONG || t == T_ULONG || t == T_DOUBLE || t == T_TOP64; }

// A class other than none comes from operands at most three levels below the value (the deepest
// is get_global_id: group id * size + local id, the product, the group id), and an operand without
// a class only keeps a pattern from matching; so a node reached more than g_class_depth levels
// down has no class, which changes no class and bounds the recursion on long chains (a damaged
// file can hold thousands of nested 64-bit pairs).  Leaves are classified at any depth.  The
// bound is a test hook (oracle_set_class_depth) so that a test can show it changes nothing.
int g_class_depth = 4;

ClsV classify(const Kernel& K, uint32_t r, int d = 0);

ClsV settings_load(const Kernel& K, const Node& n, uint32_t part, bool wide, int d) {
  ClsV v;
  ClsV base = classify(K, fwd(K, n.src[0]), d + 1);
  if (base.c == K_DISP) {
    // the dispatch packet: the dword at 0x0 holds the dimension count in its setup
    // field, the dwords at 0xc/0x10/0x14 the global size of dimension 0/1/2
    if (wide || part != P_ENTIRE) return v;
    if (n.cval == 0) return ClsV{K_DISP0, 0};
    if (n.cval == 0xc || n.cval == 0x10 || n.cval == 0x14) return ClsV{K_GSIZE, (int)(n.cval - 0xc) / 4};
    return v;
  }
  if (base.c != K_KARG || (n.cval & 7u)) return v;
  uint32_t slot = n.cval / 8;
  if (slot >= K.cfg.args.size()) return v;
  const Arg& a = K.cfg.args[slot];
  if (wide) {
    if (a.hidden && a.name.size() == 17 && a.name.compare(0, 16, "_.global_offset_") == 0 &&
        a.name[16] >= '0' && a.name[16] <= '2') {
      int d = a.name[16] - '0';
      if (part == P_ENTIRE) return ClsV{K_GOFS64, d};
      if (part == P_LO) return ClsV{K_GOFSLO, d};
      return v;
    }
    if (a.hidden || part != P_ENTIRE) return v;
    if (a.pointer) return ClsV{K_ARGPTR, (int)slot};
    if (is_64type(a.elem)) return ClsV{K_ARG64, (int)slot};
    return v;
  }
  // a __local pointer argument: the low dword of its slot is the buffer's LDS address
  if (!a.hidden && a.pointer && a.space == 2 && part == P_ENTIRE) return ClsV{K_LPTR, (int)slot};
  if (a.hidden || a.pointer || is_64type(a.elem) || part != P_ENTIRE) return v;
  return ClsV{K_ARG32, (int)slot};
}

ClsV classify(const Kernel& K, uint32_t r, int d) {
  ClsV v;
  if (r == UNDEF || r == TOP) return ClsV{K_UNDEF, 0};
  if (d > g_class_depth && is_node(r)) return v;
  if (is_leaf(r)) {
    uint32_t id = rid(r) & 0x0FFFFFFFu;
    uint32_t kind = id >> 8, k = id & 0xFF;
    if (kind == LEAF_LID && rpart(r) == P_ENTIRE) return ClsV{K_LID, (int)k};
    if (kind == LEAF_GRP && rpart(r) == P_ENTIRE) return ClsV{K_GRP, (int)k};
    if (kind == LEAF_KARG && rpart(r) == P_ENTIRE) return ClsV{K_KARG, 0};
    if (kind == LEAF_DISP && rpart(r) == P_ENTIRE) return ClsV{K_DISP, 0};
    return v;
  }
  if (!is_node(r)) return v;
  const Node& n = K.nodes[rid(r)];
  uint32_t part = rpart(r);
  if (n.kind == N_CONST) return ClsV{K_CONST32, 0};
  if (n.kind == N_PAIR && part == P_ENTIRE) {
    ClsV a = classify(K, fwd(K, n.src[0]), d + 1), b = classify(K, fwd(K, n.src[1]), d + 1);
    if (a.c == K_CONST32 && b.c == K_CONST32) return ClsV{K_CONST64, 0};
    return v;
  }
  if (n.kind == N_SLOAD64B) return settings_load(K, n, part, true, d);
  if (n.kind != N_OP) return v;
  switch (n.op) {
    case S_LOAD_DWORDX2: case S_LOAD_DWORDX4: return settings_load(K, n, part, true, d);
    case S_LOAD_DWORD: return settings_load(K, n, part, false, d);
    default: break;
  }
  if (part != P_ENTIRE) return v;
  auto cl = [&](int k) { return classify(K, fwd(K, n.src[k]), d + 1); };
  auto cval = [&](int k) -> int64_t {
    uint32_t s = fwd(K, n.src[k]);
    if (!is_node(s) || K.nodes[rid(s)].kind != N_CONST || rpart(s) != P_ENTIRE) return -1;
    return K.nodes[rid(s)].cval;
  };
  auto cws = [&](int d) { return d >= 0 && d < 3 ? K.cfg.cws[d] : -1; };
  switch (n.op) {
    case S_MUL_I32: {
      ClsV a = cl(0), b = cl(1);
      if (a.c == K_GRP && cval(1) == cws(a.k)) return ClsV{K_MULGRP, a.k};
      if (b.c == K_GRP && cval(0) == cws(b.k)) return ClsV{K_MULGRP, b.k};
      return v;
    }
    case S_LSHL_B32: {
      ClsV a = cl(0);
      if (a.c == K_GRP && log2_exact(cws(a.k)) >= 0 && cval(1) == log2_exact(cws(a.k))) return ClsV{K_MULGRP, a.k};
      return v;
    }
    case S_LSHR_B32: {  // global size / work-group size, the size a power of two
      ClsV a = cl(0);
      if (a.c == K_GSIZE && log2_exact(cws(a.k)) >= 0 && cval(1) == log2_exact(cws(a.k))) return ClsV{K_NGRP, a.k};
      return v;
    }
    case S_BFE_U32: {  // 0x20010: offset 16, width 2 = the dimension count
      if (cl(0).c == K_DISP0 && cval(1) == 0x20010) return ClsV{K_WDIM, 0};
      return v;
    }
    case V_ADD_U32: {
      ClsV a = cl(0), b = cl(1);
      if (a.c == K_MULGRP && b.c == K_LID && a.k == b.k) return ClsV{K_GIDNO, a.k};
      if (b.c == K_MULGRP && a.c == K_LID && a.k == b.k) return ClsV{K_GIDNO, a.k};
      if (a.c == K_GIDNO && b.c == K_GOFSLO && a.k == b.k) return ClsV{K_GID, a.k};
      if (b.c == K_GIDNO && a.c == K_GOFSLO && a.k == b.k) return ClsV{K_GID, a.k};
      return v;
    }
    case V_MAD_U32_U24: {
      ClsV a = cl(0), b = cl(1), c = cl(2);
      if (c.c != K_LID) return v;
      if (a.c == K_GRP && a.k == c.k && cval(1) == cws(a.k)) return ClsV{K_GIDNO, a.k};
      if (b.c == K_GRP && b.k == c.k && cval(0) == cws(b.k)) return ClsV{K_GIDNO, b.k};
      return v;
    }
  }
  return v;
}

bool leaf_like(int c) { return c != K_NONE && c != K_MULGRP && c != K_DISP0; }

// ============================================================================
// Memory accesses: base pointer (an argument's 8-byte slot, as a lo/hi pair)
// plus a 32-bit index zero- or sign-extended and shifted left by
// log2(sizeof(element)) becomes arg[index].
// ============================================================================
struct MemRef {
  bool ok = false;
  int arg = -1;         // index into cfg.args
  uint32_t idx = TOP;   // index value reference, TOP = constant 0
};

int elem_size(int t) { return is_64type(t) ? 8 : 4; }

MemRef match_addr(const Kernel& K, uint32_t addr, int width) {
  MemRef m;
  ClsV c = classify(K, addr);
  if (c.c == K_ARGPTR) {
    if (elem_size(K.cfg.args[c.k].elem) != width) return m;
    m.ok = true;
    m.arg = c.k;
    return m;
  }
  if (!is_node(addr) || rpart(addr) != P_ENTIRE) return m;
  const Node& n = K.nodes[rid(addr)];
  if (n.kind != N_OP || n.op != V_ADDC_CO_U32 || !n.fused) return m;
  for (int o = 0; o < 2; ++o) {
    uint32_t X = fwd(K, n.src[o]), Y = fwd(K, n.src[1 - o]);
    ClsV cx = classify(K, X);
    if (cx.c != K_ARGPTR) continue;
    int es = elem_size(K.cfg.args[cx.k].elem);
    if (es != width) continue;
    if (!is_node(Y) || rpart(Y) != P_ENTIRE) continue;
    const Node& sh = K.nodes[rid(Y)];
    if (sh.kind != N_OP || sh.op != V_LSHLREV_B64) continue;
    uint32_t s0 = fwd(K, sh.src[0]);
    if (!is_node(s0) || K.nodes[rid(s0)].kind != N_CONST || K.nodes[rid(s0)].cval != (uint32_t)log2_exact(es))
      continue;
    uint32_t V = fwd(K, sh.src[1]);
    if (!is_node(V) || rpart(V) != P_ENTIRE || K.nodes[rid(V)].kind != N_PAIR) continue;
    const Node& p = K.nodes[rid(V)];
    uint32_t lo = fwd(K, p.src[0]), hi = fwd(K, p.src[1]);
    bool ext = false;
    if (is_node(hi) && rpart(hi) == P_ENTIRE && K.nodes[rid(hi)].kind == N_CONST && K.nodes[rid(hi)].cval == 0)
      ext = true;
    if (is_node(hi) && rpart(hi) == P_ENTIRE) {
      const Node& a = K.nodes[rid(hi)];
      if (a.kind == N_OP && a.op == V_ASHRREV_I32) {
        uint32_t c31 = fwd(K, a.src[0]);
        if (is_node(c31) && K.nodes[rid(c31)].kind == N_CONST && K.nodes[rid(c31)].cval == 31 &&
            fwd(K, a.src[1]) == lo)
          ext = true;
      }
    }
    if (!ext) continue;
    m.ok = true;
    m.arg = cx.k;
    m.idx = lo;
    return m;
  }
  return m;
}

// An LDS access (ds_read / ds_write): the address is 32 bits, the __local buffer's LDS address
// plus the index shifted by log2 of the element size (v_lshlrev_b32 then v_add_u32, either
// operand order), or the buffer's address alone (element 0).
MemRef match_lds(const Kernel& K, uint32_t addr, int width) {
  MemRef m;
  ClsV c = classify(K, addr);
  if (c.c == K_LPTR) {
    if (elem_size(K.cfg.args[c.k].elem) != width) return m;
    m.ok = true;
    m.arg = c.k;
    return m;
  }
  if (!is_node(addr) || rpart(addr) != P_ENTIRE) return m;
  const Node& n = K.nodes[rid(addr)];
  if (n.kind != N_OP || n.op != V_ADD_U32) return m;
  for (int o = 0; o < 2; ++o) {
    uint32_t X = fwd(K, n.src[o]), Y = fwd(K, n.src[1 - o]);
    ClsV cx = classify(K, X);
    if (cx.c != K_LPTR) continue;
    int es = elem_size(K.cfg.args[cx.k].elem);
    if (es != width) continue;
    if (!is_node(Y) || rpart(Y) != P_ENTIRE) continue;
    const Node& sh = K.nodes[rid(Y)];
    if (sh.kind != N_OP || sh.op != V_LSHLREV_B32) continue;
    uint32_t s0 = fwd(K, sh.src[0]);
    if (!is_node(s0) || K.nodes[rid(s0)].kind != N_CONST || K.nodes[rid(s0)].cval != (uint32_t)log2_exact(es))
      continue;
    m.ok = true;
    m.arg = cx.k;
    m.idx = fwd(K, sh.src[1]);
    return m;
  }
  return m;
}

// ============================================================================
// Emission state: reachability, variables, types ("Data type recovery")
// ============================================================================
const char* type_name(int t) {
  switch (t) {
    case T_INT: return "int";
    case T_UINT: return "uint";
    case T_FLOAT: return "float";
    case T_LONG: return "long";
    case T_ULONG: return "ulong";
    case T_DOUBLE: return "double";
  }
  return "uint";
}
int width_of_type(int t) { return is_64type(t) ? 64 : 32; }
int tjoin(int a, int b) {
  if (a == T_NONE) return b;
  if (b == T_NONE) return a;
  if (a == b) return a;
  return (width_of_type(a) == 64 || width_of_type(b) == 64) ? T_TOP64 : T_TOP32;
}
int resolve_type(int t, int width) {
  if (t == T_NONE) return width == 64 ? T_ULONG : T_UINT;
  if (t == T_TOP32) return T_UINT;
  if (t == T_TOP64) return T_ULONG;
  return t;
}

// Memory accesses.  FLAT instructions may address global memory, LDS or scratch
// ("The body extraction"); in this dialect their address is always formed from
// a __global buffer argument, exactly as for the GLOBAL instructions, so both
// are the same access: the same dataflow, address match and output.  The LDS
// accesses are loads and stores of a __local buffer, with their own address
// match (match_lds).
bool is_lds(int op) { return op >= DS_READ_B32 && op <= DS_WRITE_B64; }
bool is_store(int op) {
  return op == GLOBAL_STORE_DWORD || op == GLOBAL_STORE_DWORDX2 || op == FLAT_STORE_DWORD || op == FLAT_STORE_DWORDX2 ||
         op == DS_WRITE_B32 || op == DS_WRITE_B64;
}
bool is_gload(int op) {
  return op == GLOBAL_LOAD_DWORD || op == GLOBAL_LOAD_DWORDX2 || op == FLAT_LOAD_DWORD || op == FLAT_LOAD_DWORDX2 ||
         op == DS_READ_B32 || op == DS_READ_B64;
}
// bytes one access moves
int mem_width(int op) {
  return op == GLOBAL_LOAD_DWORDX2 || op == GLOBAL_STORE_DWORDX2 || op == FLAT_LOAD_DWORDX2 ||
                 op == FLAT_STORE_DWORDX2 || op == DS_READ_B64 || op == DS_WRITE_B64
             ? 8
             : 4;
}
MemRef match_mem(const Kernel& K, int op, uint32_t addr) {
  return is_lds(op) ? match_lds(K, addr, mem_width(op)) : match_addr(K, addr, mem_width(op));
}

// Sweep limit of the type fixed point.  The lattice is finite and a sweep that
// changes something raises at least one type, so the default is never reached;
// a smaller limit (oracle_set_type_sweep_limit, a test hook) caps kernels, which
// are then not decompiled (FIXPOINT_CAP).
constexpr uint32_t kTypeSweepDefault = 100000;
static uint32_t g_type_sweep_limit = kTypeSweepDefault;

struct Emitter {
  Kernel& K;
  uint32_t nb;
  std::vector<uint32_t> uses;            // per node: reference count
  std::vector<char> reach, cross, phi_in;
  std::set<uint32_t> used_phis;          // phi refs
  std::vector<int> ntype;                // per node: type lattice value
  std::map<uint32_t, int> ptype;         // per phi ref
  std::vector<int> var_of;               // per node: variable number or -1
  std::map<uint32_t, int> phi_var;       // per phi ref
  std::vector<int> var_type;
  bool partial = false;

  explicit Emitter(Kernel& k) : K(k), nb((uint32_t)k.lcfg.blocks.size()) {}

  uint32_t block_of_node(uint32_t id) const { return K.lcfg.block_of[id / 4]; }
  uint32_t phi_block(uint32_t r) const { return (rid(r) >> 10) & 0x3FFFF; }
  uint32_t phi_reg(uint32_t r) const { return rid(r) & 0x3FF; }

  ClsV cls(uint32_t r) const { return classify(K, r); }

  // the width of a node's value
  int node_width(uint32_t id) const {
    const Node& n = K.nodes[id];
    if (n.kind == N_PAIR || n.kind == N_SLOAD64B) return 64;
    if (n.kind == N_OP) {
      if (is64_result(n.op) || n.op == S_LOAD_DWORDX4) return 64;
      if ((n.op == V_ADDC_CO_U32 || n.op == V_SUBB_CO_U32) && n.fused) return 64;
    }
    return 32;
  }

  // children of a node that are printed with it
  std::vector<uint32_t> children(uint32_t id) const {
    std::vector<uint32_t> ch;
    const Node& n = K.nodes[id];
    uint32_t r = ref(id, P_ENTIRE);
    if (leaf_like(cls(r).c)) return ch;
    if (n.kind == N_PAIR) {
      ch.push_back(fwd(K, n.src[0]));
      ch.push_back(fwd(K, n.src[1]));
      return ch;
    }
    if (n.kind != N_OP) return ch;
    if (is_gload(n.op) || is_store(n.op)) {
      MemRef m = match_mem(K, n.op, fwd(K, n.src[0]));
      if (m.ok) {
        if (m.idx != TOP) ch.push_back(m.idx);
      } else {
        ch.push_back(fwd(K, n.src[0]));
      }
      if (is_store(n.op)) ch.push_back(fwd(K, n.src[1]));
      return ch;
    }
    if (n.op == OP_UNKNOWN) return ch;
    if (n.op == S_LOAD_DWORD || n.op == S_LOAD_DWORDX2 || n.op == S_LOAD_DWORDX4) return ch;
    for (int k = 0; k < n.nsrc; ++k) ch.push_back(fwd(K, n.src[k]));
    return ch;
  }

  // out-value of register `reg` at the end of block p
  uint32_t out_val(uint32_t p, uint32_t reg) const {
    uint32_t v = K.out[p][reg];
    return v == TOP ? UNDEF : v;
  }

  void mark_reach() {
    size_t nn = K.nodes.size();
    uses.assign(nn, 0);
    reach.assign(nn, 0);
    cross.assign(nn, 0);
    phi_in.assign(nn, 0);
    std::vector<std::pair<uint32_t, uint32_t>> work;  // (ref, using block)
    auto use = [&](uint32_t r, uint32_t blk) { work.push_back({r, blk}); };
    // roots in program order
    for (uint32_t b = 0; b < nb; ++b) {
      for (uint32_t i = K.lcfg.blocks[b].first; i < K.lcfg.blocks[b].end; ++i) {
        if (K.lcfg.block_of[i] != b) continue;
        const Node& n = K.nodes[4 * i];
        if (n.kind != N_OP) continue;
        if (K.lcfg.ctl[i] == C_CBR) {
          if (K.lcfg.blocks[b].succ1 != NONE) use(fwd(K, n.src[0]), b);
          continue;
        }
        if (is_store(n.op) || is_gload(n.op) || n.op == OP_UNKNOWN) {
          uint32_t id = 4 * i;
          if (!reach[id]) {
            reach[id] = 1;
            for (uint32_t c : children(id)) use(c, b);
          }
        }
      }
    }
    while (!work.empty()) {
      auto [r, blk] = work.back();
      work.pop_back();
      if (is_phi(r)) {
        if (used_phis.insert(r).second) {
          uint32_t B = phi_block(r), reg = phi_reg(r);
          for (uint32_t p : K.preds[B]) {
            uint32_t v = fwd(K, out_val(p, reg));
            if (is_node(v)) phi_in[rid(v)] = 1;
            use(v, p);
          }
        }
        continue;
      }
      if (!is_node(r)) continue;
      uint32_t id = rid(r);
      uses[id]++;
      if (block_of_node(id) != blk) cross[id] = 1;
      if (!reach[id]) {
        reach[id] = 1;
        uint32_t b = block_of_node(id);
        for (uint32_t c : children(id)) use(c, b);
      }
    }
  }

  bool is_var_node(uint32_t id) const {
    if (!reach[id]) return false;
    const Node& n = K.nodes[id];
    if (leaf_like(cls(ref(id, P_ENTIRE)).c)) return false;
    if (n.kind == N_OP && is_store(n.op)) return false;
    if (n.kind == N_OP && (is_gload(n.op) || n.op == OP_UNKNOWN)) return true;
    return uses[id] >= 2 || cross[id] || phi_in[id];
  }

  // type lattice fixpoint over reachable nodes and used joins
  int ref_type(uint32_t r) const {
    if (is_phi(r)) {
      auto it = ptype.find(r);
      return it == ptype.end() ? T_NONE : it->second;
    }
    if (is_leaf(r)) {
      ClsV c = cls(r);
      if (c.c == K_LID || c.c == K_GRP) return T_UINT;
      return T_NONE;
    }
    if (!is_node(r)) return T_NONE;
    if (rpart(r) != P_ENTIRE) {
      ClsV c = cls(r);
      return c.c == K_GOFSLO ? T_UINT : T_UINT;
    }
    return ntype[rid(r)];
  }

  int node_type(uint32_t id) const {
    const Node& n = K.nodes[id];
    uint32_t r = ref(id, P_ENTIRE);
    ClsV c = cls(r);
    switch (c.c) {
      case K_GID: case K_GIDNO: case K_LID: case K_GRP: case K_GOFSLO: case K_GSIZE: case K_NGRP: case K_WDIM:
      case K_LPTR:
        return T_UINT;
      case K_GOFS64: case K_ARGPTR: case K_KARG: return T_ULONG;
      case K_ARG32: case K_ARG64: return K.cfg.args[c.k].elem;
      case K_CONST32: case K_CONST64: case K_UNDEF: return T_NONE;
    }
    auto st = [&](int k) { return ref_type(fwd(K, n.src[k])); };
    if (n.kind == N_PAIR) return T_ULONG;
    if (n.kind == N_SLOAD64B) return T_ULONG;
    if (n.kind == N_CARRY) return T_UINT;
    if (n.kind != N_OP) return T_NONE;
    switch (n.op) {
      case S_MUL_I32: return T_INT;
      case S_ADD_U32: return T_UINT;
      case S_LSHL_B32: return st(0);
      case S_LSHR_B32: case S_BFE_U32: return T_UINT;
      case V_ADD_U32: case V_SUB_U32: case V_MUL_LO_U32: case V_MAD_U32_U24: case V_MUL_U32_U24: return T_UINT;
      case V_AND_B32: case V_OR_B32: case V_XOR_B32: case V_CNDMASK_B32: return tjoin(st(0), st(1));
      case V_LSHLREV_B32: return st(1);
      case V_LSHRREV_B32: return T_UINT;
      case V_ASHRREV_I32: return T_INT;
      case V_ADD_F32: case V_SUB_F32: case V_MUL_F32: case V_FMA_F32: case V_CVT_F32_I32: case V_CVT_F32_U32:
      case V_CVT_F32_F64: return T_FLOAT;
      case V_CVT_F64_F32: case V_CVT_F64_I32: case V_ADD_F64: case V_MUL_F64: case V_FMA_F64: return T_DOUBLE;
      case V_ADD_CO_U32: case V_SUB_CO_U32: return T_UINT;
      case V_ADDC_CO_U32: case V_SUBB_CO_U32: return n.fused ? tjoin(st(0), st(1)) : T_UINT;
      case V_LSHLREV_B64: return st(1);
      case V_MUL_HI_U32_U24: return T_UINT;
      case V_MUL_HI_I32_I24: return T_INT;
      case GLOBAL_LOAD_DWORD: case GLOBAL_LOAD_DWORDX2: case FLAT_LOAD_DWORD: case FLAT_LOAD_DWORDX2:
      case DS_READ_B32: case DS_READ_B64: {
        int w = mem_width(n.op);
        MemRef m = match_mem(K, n.op, fwd(K, n.src[0]));
        if (m.ok) return K.cfg.args[m.arg].elem;
        return w == 8 ? T_ULONG : T_UINT;
      }
      case S_LOAD_DWORD: return T_UINT;
      case S_LOAD_DWORDX2: case S_LOAD_DWORDX4: return T_ULONG;
      case OP_UNKNOWN: return node_width(id) == 64 ? T_ULONG : T_UINT;
    }
    if (is_scmp(n.op) || is_vcmp(n.op)) return T_INT;
    return T_NONE;
  }

  // A node whose type is its operands' type ("Data type recovery": the b32/b64
  // suffixes carry no type, so bitwise operations, shifts that keep their
  // operand's type, selects and the high half of a fused 64-bit add take the
  // type of what flows into them).  Every other node has its type from its
  // operation, its suffix or the argument it reads, whatever its operands are.
  static bool typed_by_operands(const Node& n) {
    if (n.kind != N_OP) return false;
    switch (n.op) {
      case S_LSHL_B32: case V_AND_B32: case V_OR_B32: case V_XOR_B32: case V_LSHLREV_B32: case V_LSHLREV_B64:
      case V_CNDMASK_B32: return true;
      case V_ADDC_CO_U32: case V_SUBB_CO_U32: return n.fused != 0;
    }
    return false;
  }

  // The least fixed point of the type equations: nodes typed by their
  // operation are set once; the nodes typed by their operands and the used join
  // versions start at the bottom and are swept (in node order, then the joins)
  // until a sweep changes nothing.  A kernel still changing in sweep number
  // g_type_sweep_limit is capped (types_capped).
  bool types_capped = false;
  void infer_types() {
    ntype.assign(K.nodes.size(), T_NONE);
    std::vector<uint32_t> dyn;
    for (uint32_t id = 0; id < K.nodes.size(); ++id) {
      if (!reach[id]) continue;
      if (typed_by_operands(K.nodes[id])) dyn.push_back(id);
      else ntype[id] = node_type(id);
    }
    for (uint32_t r : used_phis) ptype[r] = T_NONE;
    bool changed = true;
    uint32_t sweeps = 0;
    while (changed && sweeps < g_type_sweep_limit) {
      ++sweeps;
      changed = false;
      for (uint32_t id : dyn) {
        int t = tjoin(ntype[id], node_type(id));
        if (t != ntype[id]) { ntype[id] = t; changed = true; }
      }
      for (uint32_t r : used_phis) {
        int t = ptype[r];
        uint32_t B = phi_block(r), reg = phi_reg(r);
        for (uint32_t p : K.preds[B]) t = tjoin(t, ref_type(fwd(K, out_val(p, reg))));
        if (ptype[r] != t) { ptype[r] = t; changed = true; }
      }
    }
    types_capped = changed;
  }

  void number_vars() {
    // order: joins at the start of their block (by register), then nodes by
    // (instruction, slot)
    std::vector<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>> keys;  // (instr, kind, sub, token)
    for (uint32_t r : used_phis)
      keys.push_back({K.lcfg.blocks[phi_block(r)].first, 0, phi_reg(r), r});
    for (uint32_t id = 0; id < K.nodes.size(); ++id)
      if (is_var_node(id)) keys.push_back({id / 4, 1, id % 4, id});
    std::sort(keys.begin(), keys.end());
    var_of.assign(K.nodes.size(), -1);
    for (size_t k = 0; k < keys.size(); ++k) {
      auto [i, kind, sub, tok] = keys[k];
      (void)i;
      (void)sub;
      if (kind == 0) {
        phi_var[tok] = (int)k;
        var_type.push_back(resolve_type(ptype[tok], 32));
      } else {
        var_of[tok] = (int)k;
        var_type.push_back(resolve_type(ntype[tok], node_width(tok)));
      }
    }
  }

  // -------------------------------------------------------------------------
  // printing
  // -------------------------------------------------------------------------
  static std::string u64s(uint64_t v) { return std::to_string(v); }

  // exact short decimal of a float/double when it has few binary fraction
  // digits; otherwise the bit pattern through as_float / as_double
  static std::string float_lit(uint64_t bits, bool dbl) {
    int mbits = dbl ? 52 : 23, ebits = dbl ? 11 : 8;
    int bias = dbl ? 1023 : 127;
    uint64_t sign = bits >> (mbits + ebits);
    uint64_t ex = (bits >> mbits) & ((1ull << ebits) - 1);
    uint64_t man = bits & ((1ull << mbits) - 1);
    std::string fb = dbl ? "as_double(" + u64s(bits) + "UL)" : "as_float(" + u64s(bits) + "u)";
    std::string suf = dbl ? "" : "f";
    if (bits == 0) return "0.0" + suf;
    if (ex == (1ull << ebits) - 1 || ex == 0) return fb;
    uint64_t m = man | (1ull << mbits);
    int e = (int)ex - bias - mbits;
    while ((m & 1) == 0 && e < 0) { m >>= 1; ++e; }
    std::string s = sign ? "-" : "";
    if (e >= 0) {
      if (e > 62 || (m >> (63 - e)) != 0) return fb;
      return s + u64s(m << e) + ".0" + suf;
    }
    int k = -e;
    if (k > 16) return fb;
    uint64_t p5 = 1;
    for (int i = 0; i < k; ++i) p5 *= 5;
    if (m > UINT64_MAX / p5) return fb;
    uint64_t N = m * p5;
    uint64_t p10 = 1;
    for (int i = 0; i < k; ++i) p10 *= 10;
    uint64_t ip = N / p10, fp = N % p10;
    std::string frac = u64s(fp);
    while ((int)frac.size() < k) frac = "0" + frac;
    while (frac.size() > 1 && frac.back() == '0') frac.pop_back();
    return s + u64s(ip) + "." + frac + suf;
  }

  static std::string lit32(uint32_t bits, int want) {
    switch (want) {
      case T_INT: {
        int32_t v = (int32_t)bits;
        if (v == INT32_MIN) return "(-2147483647 - 1)";
        return std::to_string(v);
      }
      case T_FLOAT: return float_lit(bits, false);
      default: return u64s(bits) + "u";
    }
  }
  static std::string lit64(uint64_t bits, int want) {
    switch (want) {
      case T_LONG: {
        int64_t v = (int64_t)bits;
        if (v == INT64_MIN) return "(-9223372036854775807L - 1L)";
        return std::to_string(v) + "L";
      }
      case T_DOUBLE: return float_lit(bits, true);
      default: return u64s(bits) + "UL";
    }
  }

  static bool is_int_type(int t) { return t == T_INT || t == T_UINT || t == T_LONG || t == T_ULONG; }

  std::string conv(const std::string& e, int from, int want) {
    if (want == T_NONE || from == want) return e;
    if (is_int_type(from) && is_int_type(want)) return std::string("(") + type_name(want) + ")" + e;
    if (width_of_type(from) == width_of_type(want)) return std::string("as_") + type_name(want) + "(" + e + ")";
    return std::string("(") + type_name(want) + ")" + e;
  }

  struct Ex {
    std::string s;
    int t;
  };

  std::string E(uint32_t r, int want) {
    Ex x = expr(r, want);
    return conv(x.s, x.t, want);
  }

  std::string shamt(uint32_t r, uint32_t mask) {
    uint32_t f = fwd(K, r);
    if (is_node(f) && K.nodes[rid(f)].kind == N_CONST && rpart(f) == P_ENTIRE)
      return std::to_string(K.nodes[rid(f)].cval & mask);
    return "(" + E(f, T_UINT) + " & " + std::to_string(mask) + "u)";
  }

  std::string memref(const Node& n, int width, int* elem) {
    MemRef m = match_mem(K, n.op, fwd(K, n.src[0]));
    if (m.ok) {
      *elem = K.cfg.args[m.arg].elem;
      std::string idx = m.idx == TOP ? std::string("0") : E(m.idx, T_NONE);
      return K.cfg.args[m.arg].name + "[" + idx + "]";
    }
    *elem = width == 8 ? T_ULONG : T_UINT;
    if (is_lds(n.op)) {  // an LDS address that is no buffer element: pseudo-code
      partial = true;
      return std::string("*((__local ") + type_name(*elem) + " *)(" + E(fwd(K, n.src[0]), T_UINT) + "))";
    }
    return std::string("*((__global ") + type_name(*elem) + " *)(" + E(fwd(K, n.src[0]), T_ULONG) + "))";
  }

  Ex binop(const Node& n, const char* sym, int ot) {
    return Ex{"(" + E(fwd(K, n.src[0]), ot) + " " + sym + " " + E(fwd(K, n.src[1]), ot) + ")", ot};
  }

  // expression of node `id` itself (ignoring its own variable)
  Ex node_expr(uint32_t id) {
    const Node& n = K.nodes[id];
    int NT = resolve_type(ntype[id], node_width(id));
    auto S = [&](int k, int t) { return E(fwd(K, n.src[k]), t); };
    if (n.kind == N_PAIR) return Ex{"upsample(" + S(1, T_UINT) + ", " + S(0, T_UINT) + ")", T_ULONG};
    if (n.kind == N_CARRY || n.kind == N_SLOAD64B) { partial = true; return Ex{"0u", T_UINT}; }
    if (n.kind != N_OP) { partial = true; return Ex{"0u", T_UINT}; }
    int op = n.op;
    if (is_scmp(op) || is_vcmp(op)) {
      int cc, ot;
      if (is_scmp(op)) { cc = (op - S_CMP_FIRST) % 6; ot = (op - S_CMP_FIRST) / 6 == 0 ? T_UINT : T_INT; }
      else { cc = (op - V_CMP_FIRST) % 6; int ty = (op - V_CMP_FIRST) / 6; ot = ty == 0 ? T_INT : (ty == 1 ? T_UINT : T_FLOAT); }
      return Ex{"(" + S(0, ot) + " " + kCmpSym[cc] + " " + S(1, ot) + ")", T_INT};
    }
    switch (op) {
      case S_ADD_U32: return binop(n, "+", T_UINT);
      case S_MUL_I32: return binop(n, "*", T_INT);
      case S_LSHL_B32: return Ex{"(" + S(0, NT) + " << " + shamt(n.src[1], 31) + ")", NT};
      case S_LSHR_B32: return Ex{"(" + S(0, T_UINT) + " >> " + shamt(n.src[1], 31) + ")", T_UINT};
      case S_BFE_U32: {
        // field operand: offset in bits [4:0], width in bits [22:16]; the result is
        // (src >> offset) masked to width bits.  A field that is not a constant, or a
        // width of 32 or more, is not written out.
        uint32_t f = fwd(K, n.src[1]);
        if (!is_node(f) || K.nodes[rid(f)].kind != N_CONST || rpart(f) != P_ENTIRE) { partial = true; return Ex{"0u", T_UINT}; }
        uint32_t c = (uint32_t)K.nodes[rid(f)].cval, off = c & 31u, w = (c >> 16) & 0x7Fu;
        if (w == 0) return Ex{"0u", T_UINT};
        if (w >= 32) { partial = true; return Ex{"0u", T_UINT}; }
        return Ex{"((" + S(0, T_UINT) + " >> " + std::to_string(off) + ") & " + lit32((1u << w) - 1u, T_UINT) + ")", T_UINT};
      }
      case V_ADD_U32: return binop(n, "+", T_UINT);
      case V_SUB_U32: return binop(n, "-", T_UINT);
      case V_MUL_LO_U32: return binop(n, "*", T_UINT);
      case V_MAD_U32_U24: return Ex{"mad24(" + S(0, T_UINT) + ", " + S(1, T_UINT) + ", " + S(2, T_UINT) + ")", T_UINT};
      case V_MUL_U32_U24: return Ex{"mul24(" + S(0, T_UINT) + ", " + S(1, T_UINT) + ")", T_UINT};
      // the double-suffix high multiplies: the high 32 bits of the 48-bit product of the low 24
      // bits of the operands, zero-extended (u24) or sign-extended (i24); OpenCL's mul_hi of the
      // operands reduced to 24 bits is exactly that
      case V_MUL_HI_U32_U24:
        return Ex{"mul_hi((" + S(0, T_UINT) + " & 16777215u), (" + S(1, T_UINT) + " & 16777215u))", T_UINT};
      case V_MUL_HI_I32_I24:
        return Ex{"mul_hi(((int)(" + S(0, T_UINT) + " << 8) >> 8), ((int)(" + S(1, T_UINT) + " << 8) >> 8))", T_INT};
      case V_AND_B32: return binop(n, "&", NT);
      case V_OR_B32: return binop(n, "|", NT);
      case V_XOR_B32: return binop(n, "^", NT);
      case V_LSHLREV_B32: return Ex{"(" + S(1, NT) + " << " + shamt(n.src[0], 31) + ")", NT};
      case V_LSHRREV_B32: return Ex{"(" + S(1, T_UINT) + " >> " + shamt(n.src[0], 31) + ")", T_UINT};
      case V_ASHRREV_I32: return Ex{"(" + S(1, T_INT) + " >> " + shamt(n.src[0], 31) + ")", T_INT};
      case V_ADD_F32: return binop(n, "+", T_FLOAT);
      case V_SUB_F32: return binop(n, "-", T_FLOAT);
      case V_MUL_F32: return binop(n, "*", T_FLOAT);
      case V_FMA_F32: return Ex{"fma(" + S(0, T_FLOAT) + ", " + S(1, T_FLOAT) + ", " + S(2, T_FLOAT) + ")", T_FLOAT};
      case V_CVT_F32_I32: return Ex{"(float)" + S(0, T_INT), T_FLOAT};
      case V_CVT_F32_U32: return Ex{"(float)" + S(0, T_UINT), T_FLOAT};
      case V_CVT_F64_F32: return Ex{"(double)" + S(0, T_FLOAT), T_DOUBLE};
      case V_CVT_F64_I32: return Ex{"(double)" + S(0, T_INT), T_DOUBLE};
      case V_CVT_F32_F64: return Ex{"(float)" + S(0, T_DOUBLE), T_FLOAT};
      case V_ADD_CO_U32: return binop(n, "+", T_UINT);
      case V_SUB_CO_U32: return binop(n, "-", T_UINT);
      case V_ADDC_CO_U32:
        if (n.fused) return binop(n, "+", NT);
        partial = true;
        return Ex{"(" + S(0, T_UINT) + " + " + S(1, T_UINT) + ")", T_UINT};
      case V_SUBB_CO_U32:
        if (n.fused) return binop(n, "-", NT);
        partial = true;
        return Ex{"(" + S(0, T_UINT) + " - " + S(1, T_UINT) + ")", T_UINT};
      case V_LSHLREV_B64: return Ex{"(" + S(1, NT) + " << " + shamt(n.src[0], 63) + ")", NT};
      case V_ADD_F64: return binop(n, "+", T_DOUBLE);
      case V_MUL_F64: return binop(n, "*", T_DOUBLE);
      case V_FMA_F64: return Ex{"fma(" + S(0, T_DOUBLE) + ", " + S(1, T_DOUBLE) + ", " + S(2, T_DOUBLE) + ")", T_DOUBLE};
      case V_CNDMASK_B32:  // "Search for control structures": the ternary operator, one instruction
        return Ex{"(" + S(2, T_NONE) + " ? " + S(1, NT) + " : " + S(0, NT) + ")", NT};
      case GLOBAL_LOAD_DWORD: case GLOBAL_LOAD_DWORDX2: case FLAT_LOAD_DWORD: case FLAT_LOAD_DWORDX2:
      case DS_READ_B32: case DS_READ_B64: {
        int elem;
        std::string m = memref(n, mem_width(op), &elem);
        return Ex{m, elem};
      }
    }
    partial = true;
    return Ex{NT == T_ULONG ? "0UL" : "0u", NT == T_ULONG ? T_ULONG : T_UINT};
  }

  Ex expr(uint32_t r, int want) {
    r = fwd(K, r);
    if (is_phi(r)) {
      int v = phi_var.count(r) ? phi_var[r] : -1;
      if (v < 0) { partial = true; return Ex{"0u", T_UINT}; }
      return Ex{"var" + std::to_string(v), var_type[v]};
    }
    ClsV c = cls(r);
    switch (c.c) {
      case K_UNDEF: partial = true; return Ex{"0u", T_UINT};
      case K_LID: return Ex{"get_local_id(" + std::to_string(c.k) + ")", T_UINT};
      case K_GRP: return Ex{"get_group_id(" + std::to_string(c.k) + ")", T_UINT};
      case K_GID: return Ex{"get_global_id(" + std::to_string(c.k) + ")", T_UINT};
      case K_GIDNO:
        return Ex{"(get_global_id(" + std::to_string(c.k) + ") - get_global_offset(" + std::to_string(c.k) + "))", T_UINT};
      case K_GOFSLO: return Ex{"get_global_offset(" + std::to_string(c.k) + ")", T_UINT};
      case K_GOFS64: return Ex{"get_global_offset(" + std::to_string(c.k) + ")", T_ULONG};
      case K_ARG32: case K_ARG64: return Ex{K.cfg.args[c.k].name, K.cfg.args[c.k].elem};
      case K_ARGPTR: return Ex{"(ulong)" + K.cfg.args[c.k].name, T_ULONG};
      case K_LPTR: partial = true; return Ex{"(uint)(ulong)" + K.cfg.args[c.k].name, T_UINT};
      case K_KARG: case K_DISP: partial = true; return Ex{"0UL", T_ULONG};
      case K_GSIZE: return Ex{"get_global_size(" + std::to_string(c.k) + ")", T_UINT};
      case K_NGRP: return Ex{"get_num_groups(" + std::to_string(c.k) + ")", T_UINT};
      case K_WDIM: return Ex{"get_work_dim()", T_UINT};
      case K_CONST32: {
        int w = want == T_NONE ? T_UINT : want;
        if (width_of_type(w) == 64) w = T_UINT;
        return Ex{lit32(K.nodes[rid(r)].cval, w), w};
      }
      case K_CONST64: {
        const Node& p = K.nodes[rid(r)];
        uint64_t lo = K.nodes[rid(fwd(K, p.src[0]))].cval, hi = K.nodes[rid(fwd(K, p.src[1]))].cval;
        int w = want == T_NONE ? T_ULONG : want;
        if (width_of_type(w) == 32) w = T_ULONG;
        return Ex{lit64(lo | (hi << 32), w), w};
      }
    }
    if (!is_node(r)) { partial = true; return Ex{"0u", T_UINT}; }
    uint32_t id = rid(r);
    if (rpart(r) != P_ENTIRE) {
      Ex b = expr(ref(id, P_ENTIRE), T_NONE);
      bool dbl = b.t == T_DOUBLE;
      if (rpart(r) == P_LO) return Ex{dbl ? "(uint)as_ulong(" + b.s + ")" : "(uint)" + b.s, T_UINT};
      return Ex{dbl ? "(uint)(as_ulong(" + b.s + ") >> 32)" : "(uint)(" + b.s + " >> 32)", T_UINT};
    }
    if (var_of[id] >= 0) return Ex{"var" + std::to_string(var_of[id]), var_type[var_of[id]]};
    return node_expr(id);
  }

  // -------------------------------------------------------------------------
  // statements
  // -------------------------------------------------------------------------
  std::string out;
  void line(int lvl, const std::string& s) {
    out.append(4 * (size_t)lvl, ' ');
    out += s;
    out += '\n';
  }

  static std::string escape(const std::string& s) {
    std::string o;
    for (char c : s) {
      if (c == '"' || c == '\\') o += '\\';
      o += c;
    }
    return o;
  }

  void block_stmts(uint32_t b, int lvl) {
    for (uint32_t i = K.lcfg.blocks[b].first; i < K.lcfg.blocks[b].end; ++i) {
      if (K.lcfg.block_of[i] != b) continue;
      static const int order[4] = {1, 2, 3, 0};
      for (int q = 0; q < 4; ++q) {
        uint32_t id = 4 * i + (uint32_t)order[q];
        const Node& n = K.nodes[id];
        if (n.kind == N_OP && order[q] == 0 && n.op == OP_UNKNOWN && reach[id]) {
          line(lvl, "__asm__(\"" + escape(K.dec.text[i]) + "\");");
          partial = true;
          continue;
        }
        if (n.kind == N_OP && order[q] == 0 && is_store(n.op) && reach[id]) {
          int elem;
          std::string m = memref(n, mem_width(n.op), &elem);
          line(lvl, m + " = " + E(fwd(K, n.src[1]), elem) + ";");
          continue;
        }
        if (n.kind == N_OP && order[q] == 0 && n.op == S_BARRIER) {  // at its program point
          line(lvl, "barrier(CLK_LOCAL_MEM_FENCE);");
          continue;
        }
        if (var_of[id] >= 0) {
          Ex x = node_expr(id);
          line(lvl, "var" + std::to_string(var_of[id]) + " = " + conv(x.s, x.t, var_type[var_of[id]]) + ";");
        }
      }
    }
  }

  // copies into the join versions of block s along the edge p -> s
  void copies(uint32_t p, uint32_t s, int lvl) {
    struct Cp {
      uint32_t reg, dst, src;
    };
    std::vector<Cp> pend;
    for (uint32_t r : used_phis) {
      if (phi_block(r) != s) continue;
      uint32_t src = fwd(K, out_val(p, phi_reg(r)));
      if (src == r || src == UNDEF) continue;
      pend.push_back({phi_reg(r), r, src});
    }
    std::sort(pend.begin(), pend.end(), [](const Cp& a, const Cp& b) { return a.reg < b.reg; });
    while (!pend.empty()) {
      size_t pick = pend.size();
      for (size_t k = 0; k < pend.size() && pick == pend.size(); ++k) {
        bool read = false;
        for (size_t q = 0; q < pend.size(); ++q)
          if (q != k && pend[q].src == pend[k].dst) read = true;
        if (!read) pick = k;
      }
      if (pick == pend.size()) {  // a cycle of copies: not supported
        partial = true;
        pick = 0;
      }
      const Cp c = pend[pick];
      int v = phi_var[c.dst];
      line(lvl, "var" + std::to_string(v) + " = " + E(c.src, var_type[v]) + ";");
      pend.erase(pend.begin() + (long)pick);
    }
  }
};

// ============================================================================
// Step 4: region graph and structural analysis ("Search for control
// structures", Fig. 3).  Pre-order depth-first search from the entry,
// successors in (fall-through, taken) order; at each region the templates are
// tried in the order loop (self loop), loop (header + latch), if-else, if,
// linear; the first match is merged into a new region and the search restarts,
// until one region remains.  Reading of the figure-less templates:
//   linear(a,b): succ(a)={b}, pred(b)={a}, |succ(b)|<=1
//   if(h,t,j):   succ(h)={t,j}, pred(t)={h}, succ(t)={j}; j is merged too when
//                pred(j)={h,t}, otherwise only {h,t}
//   if-else(h,t,e[,j]): succ(h)={t,e}, pred(t)=pred(e)={h}, succ(t)=succ(e), |.|<=1;
//                j merged when pred(j)={t,e}
//   loop: a region whose conditional exit branches back to its own head (a
//   do-while), or a header followed by such a latch.
// ============================================================================
enum RKind { R_BLOCK = 0, R_SEQ = 1, R_IF = 2, R_IFELSE = 3, R_LOOP = 4 };

struct Region {
  int kind;
  std::vector<int> ch;
  uint32_t block;
};

struct Reducer {
  std::vector<Region> reg;
  std::vector<std::vector<int>> succ;
  std::vector<std::set<int>> pred;
  std::vector<char> alive;
  int entry = 0;
  std::vector<std::vector<int>> log;  // merged member lists, in order
  // block-level info for the tail / conditional checks
  std::vector<char> cond_block;       // block ends with a two-way branch (not counting a cut break edge)
  std::vector<std::vector<int>> bsucc;
  std::vector<int> brk_latch;         // per block: the latch of the loop it breaks out of, or -1

  int head(int r) const { return reg[r].kind == R_BLOCK ? (int)reg[r].block : head(reg[r].ch[0]); }
  int tail(int r) const {
    const Region& R = reg[r];
    switch (R.kind) {
      case R_BLOCK: return (int)R.block;
      case R_SEQ: return tail(R.ch[1]);
      case R_IF: return R.ch.size() == 3 ? tail(R.ch[2]) : -1;
      case R_IFELSE: return R.ch.size() == 4 ? tail(R.ch[3]) : -1;
      case R_LOOP: return tail(R.ch.back());
    }
    return -1;
  }
  bool cond_tail(int r) const {
    int t = tail(r);
    return t >= 0 && cond_block[t];
  }
  bool latch_of(int body_tail_region, int head_region) const {
    int t = tail(body_tail_region);
    if (t < 0 || !cond_block[t]) return false;
    int h = head(head_region);
    for (int s : bsucc[t])
      if (s == h) return true;
    return false;
  }
  bool pred_is(int x, std::initializer_list<int> s) const {
    std::set<int> want(s);
    return pred[x] == want;
  }

  std::vector<int> mapped(const std::vector<int>& v, const std::set<int>& S, int id) const {
    std::vector<int> o;
    for (int x : v) {
      int y = S.count(x) ? id : x;
      if (std::find(o.begin(), o.end(), y) == o.end()) o.push_back(y);
    }
    return o;
  }

  void merge(int kind, std::vector<int> ch, const std::vector<int>& nsucc) {
    int id = (int)reg.size();
    reg.push_back(Region{kind, ch, 0});
    std::set<int> S(ch.begin(), ch.end());
    succ.push_back(mapped(nsucc, S, id));
    pred.push_back({});
    alive.push_back(1);
    for (int c : ch) alive[c] = 0;
    for (int c : ch)
      for (int x : pred[c])
        if (!S.count(x)) pred[id].insert(x);
    if (std::find(succ[id].begin(), succ[id].end(), id) != succ[id].end()) pred[id].insert(id);
    for (int x : pred[id])
      if (x != id) succ[x] = mapped(succ[x], S, id);
    for (int y : succ[id]) {
      if (y == id) continue;
      std::set<int> np;
      for (int x : pred[y])
        if (!S.count(x)) np.insert(x);
      np.insert(id);
      pred[y] = np;
    }
    if (S.count(entry)) entry = id;
    log.push_back(ch);
  }

  bool try_at(int h) {
    const std::vector<int>& sh = succ[h];
    // loop: self loop
    if (sh.size() == 2 && (sh[0] == h || sh[1] == h) && latch_of(h, h)) {
      int x = sh[0] == h ? sh[1] : sh[0];
      merge(R_LOOP, {h}, {x});
      return true;
    }
    // loop: header + latch
    if (sh.size() == 1 && sh[0] != h) {
      int b = sh[0];
      const std::vector<int>& sb = succ[b];
      if (pred_is(b, {h}) && sb.size() == 2 && (sb[0] == h || sb[1] == h) && latch_of(b, h)) {
        int x = sb[0] == h ? sb[1] : sb[0];
        merge(R_LOOP, {h, b}, {x});
        return true;
      }
    }
    if (sh.size() == 2 && cond_tail(h)) {
      int t = sh[0], e = sh[1];
      // if-else
      if (t != h && e != h && t != e && pred_is(t, {h}) && pred_is(e, {h})) {
        std::vector<int> st = succ[t], se = succ[e];
        std::sort(st.begin(), st.end());
        std::sort(se.begin(), se.end());
        if (st == se && st.size() <= 1) {
          if (st.size() == 1) {
            int j = st[0];
            if (j != h && j != t && j != e) {
              if (pred_is(j, {t, e})) merge(R_IFELSE, {h, t, e, j}, succ[j]);
              else merge(R_IFELSE, {h, t, e}, {j});
              return true;
            }
          } else {
            merge(R_IFELSE, {h, t, e}, {});
            return true;
          }
        }
      }
      // if (either successor may be the then part)
      for (int q = 0; q < 2; ++q) {
        int tt = sh[q], j = sh[1 - q];
        if (tt == h || j == h) continue;
        if (!pred_is(tt, {h})) continue;
        if (succ[tt].size() != 1 || succ[tt][0] != j) continue;
        if (pred_is(j, {h, tt})) merge(R_IF, {h, tt, j}, succ[j]);
        else merge(R_IF, {h, tt}, {j});
        return true;
      }
    }
    // linear
    if (sh.size() == 1 && sh[0] != h) {
      int b = sh[0];
      if (pred_is(b, {h}) && succ[b].size() <= 1) {
        merge(R_SEQ, {h, b}, succ[b]);
        return true;
      }
    }
    return false;
  }

  // Every break block must print inside the do-while of its own loop: the nearest loop region
  // above it in the region tree is the loop whose latch the break rule found.  Otherwise the
  // `break` would leave another loop, and the kernel counts as unstructured.
  bool breaks_in_place(int root) const {
    std::vector<int> parent(reg.size(), -1);
    for (size_t r = 0; r < reg.size(); ++r)
      for (int c : reg[r].ch) parent[c] = (int)r;
    for (size_t b = 0; b < brk_latch.size(); ++b) {
      if (brk_latch[b] < 0 || !is_in_tree(root, (int)b, parent)) continue;
      int r = parent[b];
      while (r >= 0 && reg[r].kind != R_LOOP) r = parent[r];
      if (r < 0 || tail(reg[r].ch.back()) != brk_latch[b]) return false;
    }
    return true;
  }
  static bool is_in_tree(int root, int x, const std::vector<int>& parent) {
    while (x >= 0 && x != root) x = parent[x];
    return x == root;
  }

  // returns the root region, or -1 when the graph does not reduce to one region
  int run() {
    for (;;) {
      int n_alive = 0;
      for (char a : alive) n_alive += a;
      if (n_alive <= 1) return n_alive == 1 && breaks_in_place(entry) ? entry : -1;
      std::vector<char> seen(reg.size(), 0);
      std::vector<int> stack{entry};
      bool merged = false;
      while (!stack.empty() && !merged) {
        int x = stack.back();
        stack.pop_back();
        if (seen[x]) continue;
        seen[x] = 1;
        if (try_at(x)) { merged = true; break; }
        for (int k = (int)succ[x].size() - 1; k >= 0; --k)
          if (!seen[succ[x][k]]) stack.push_back(succ[x][k]);
      }
      if (!merged) return -1;
    }
  }
};

// Early exits from counted loops (a project extension: the paper restores no loops).  A latch
// is a two-way block with exactly one successor at or before it (the header H, the back edge)
// and the other after it (the exit E).  A two-way block b that is not a latch breaks out of the
// loop whose body holds it when one of its successors is that loop's exit and the other stays
// in the loop; the loop that holds b is the first latch l after b whose header is at or before
// b (for nested loops laid out in program order, the innermost one).  The edge b -> E is left
// out of the graph the regions are reduced on, and b prints `if (c) { break; }` after its
// statements.  A jump to the latch (continue) needs no rule: it is an if.
std::vector<int> break_latches(const LogicalCfg& L, const std::vector<char>& cond) {
  const uint32_t n = (uint32_t)L.blocks.size();
  std::vector<int> hdr(n, -1), out(n, -1);
  for (uint32_t l = 0; l < n; ++l) {
    if (!cond[l]) continue;
    const uint32_t s0 = L.blocks[l].succ0, s1 = L.blocks[l].succ1;
    if ((s0 <= l) != (s1 <= l)) hdr[l] = (int)(s0 <= l ? s0 : s1);
  }
  for (uint32_t b = 0; b < n; ++b) {
    if (!cond[b] || hdr[b] >= 0) continue;
    for (uint32_t l = b + 1; l < n; ++l) {
      if (hdr[l] < 0 || hdr[l] > (int)b) continue;
      const uint32_t E = L.blocks[l].succ0 == (uint32_t)hdr[l] ? L.blocks[l].succ1 : L.blocks[l].succ0;
      const uint32_t s0 = L.blocks[b].succ0, s1 = L.blocks[b].succ1;
      if ((s0 == E) != (s1 == E)) {
        const uint32_t x = s0 == E ? s1 : s0;
        if ((int)x >= hdr[l] && x <= l) out[b] = (int)l;
      }
      break;  // only the loop that holds b
    }
  }
  return out;
}

Reducer make_reducer(const Kernel& K, std::vector<char>* reachable) {
  Reducer rd;
  const auto& L = K.lcfg;
  uint32_t nb = (uint32_t)L.blocks.size();
  std::vector<char> live(nb, 0);
  std::vector<uint32_t> st;
  if (nb) { st.push_back(0); live[0] = 1; }
  while (!st.empty()) {
    uint32_t b = st.back();
    st.pop_back();
    for (uint32_t s : {L.blocks[b].succ0, L.blocks[b].succ1})
      if (s != NONE && !live[s]) { live[s] = 1; st.push_back(s); }
  }
  rd.reg.resize(nb);
  rd.succ.resize(nb);
  rd.pred.resize(nb);
  rd.alive.assign(nb, 0);
  rd.cond_block.assign(nb, 0);
  rd.bsucc.resize(nb);
  for (uint32_t b = 0; b < nb; ++b) rd.cond_block[b] = L.ctl[L.term[b]] == C_CBR && L.blocks[b].succ1 != NONE;
  rd.brk_latch = break_latches(L, rd.cond_block);
  for (uint32_t b = 0; b < nb; ++b) {
    rd.reg[b] = Region{R_BLOCK, {}, b};
    if (!live[b]) { rd.brk_latch[b] = -1; continue; }
    rd.alive[b] = 1;
    int cut = -1;  // a break edge is not part of the reduced graph
    if (rd.brk_latch[b] >= 0) {
      const uint32_t l = (uint32_t)rd.brk_latch[b];
      const uint32_t h = L.blocks[l].succ0 <= l ? L.blocks[l].succ0 : L.blocks[l].succ1;
      cut = (int)(L.blocks[l].succ0 == h ? L.blocks[l].succ1 : L.blocks[l].succ0);
      rd.cond_block[b] = 0;
    }
    for (uint32_t s : {L.blocks[b].succ0, L.blocks[b].succ1})
      if (s != NONE) {
        if ((int)s != cut) rd.succ[b].push_back((int)s);
        rd.bsucc[b].push_back((int)s);
      }
  }
  for (uint32_t b = 0; b < nb; ++b)
    for (int s : rd.succ[b]) rd.pred[s].insert((int)b);
  *reachable = live;
  return rd;
}

// ============================================================================
// Step 5: OpenCL generation from the region tree
// ============================================================================
struct RegionPrinter {
  Emitter& em;
  Reducer& rd;
  const Kernel& K;

  // condition under which the terminator of block t goes to block dst
  std::string cond_to(uint32_t t, uint32_t dst) {
    uint32_t i = K.lcfg.term[t];
    uint32_t c = fwd(K, K.nodes[4 * i].src[0]);
    uint32_t ft = K.lcfg.blocks[t].succ0;
    bool sense = K.lcfg.sense[i] != 0;
    bool to_taken = dst != ft;
    bool positive = to_taken ? sense : !sense;  // goes to dst when cond == positive
    std::string s;
    if (is_node(c) && rpart(c) == P_ENTIRE && K.nodes[rid(c)].kind == N_OP &&
        (is_scmp(K.nodes[rid(c)].op) || is_vcmp(K.nodes[rid(c)].op)) && em.var_of[rid(c)] < 0) {
      std::string full = em.node_expr(rid(c)).s;  // "(a op b)"
      s = positive ? full.substr(1, full.size() - 2) : "!" + full;
    } else {
      std::string e = em.E(c, T_NONE);
      s = positive ? e : "!(" + e + ")";
    }
    return s;
  }

  void emit(int r, int lvl) {
    const Region& R = rd.reg[r];
    switch (R.kind) {
      case R_BLOCK: {
        uint32_t b = R.block;
        em.block_stmts(b, lvl);
        if (rd.brk_latch[b] >= 0) {  // an early exit: the join copies of each edge on its own path
          const uint32_t l = (uint32_t)rd.brk_latch[b];
          const uint32_t h = K.lcfg.blocks[l].succ0 <= l ? K.lcfg.blocks[l].succ0 : K.lcfg.blocks[l].succ1;
          const uint32_t E = K.lcfg.blocks[l].succ0 == h ? K.lcfg.blocks[l].succ1 : K.lcfg.blocks[l].succ0;
          const uint32_t x = K.lcfg.blocks[b].succ0 == E ? K.lcfg.blocks[b].succ1 : K.lcfg.blocks[b].succ0;
          em.line(lvl, "if (" + cond_to(b, E) + ") {");
          em.copies(b, E, lvl + 1);
          em.line(lvl + 1, "break;");
          em.line(lvl, "}");
          em.copies(b, x, lvl);
        } else if (!rd.cond_block[b] && K.lcfg.blocks[b].succ0 != NONE) {
          em.copies(b, K.lcfg.blocks[b].succ0, lvl);
        }
        break;
      }
      case R_SEQ:
        emit(R.ch[0], lvl);
        emit(R.ch[1], lvl);
        break;
      case R_IF: {
        emit(R.ch[0], lvl);
        uint32_t t = (uint32_t)rd.tail(R.ch[0]);
        uint32_t th = (uint32_t)rd.head(R.ch[1]);
        uint32_t other = K.lcfg.blocks[t].succ0 == th ? K.lcfg.blocks[t].succ1 : K.lcfg.blocks[t].succ0;
        em.line(lvl, "if (" + cond_to(t, th) + ") {");
        emit(R.ch[1], lvl + 1);
        size_t mark = em.out.size();
        em.line(lvl, "} else {");
        size_t mark2 = em.out.size();
        em.copies(t, other, lvl + 1);
        if (em.out.size() == mark2) em.out.resize(mark);
        em.line(lvl, "}");
        if (R.ch.size() == 3) emit(R.ch[2], lvl);
        break;
      }
      case R_IFELSE: {
        emit(R.ch[0], lvl);
        uint32_t t = (uint32_t)rd.tail(R.ch[0]);
        uint32_t th = (uint32_t)rd.head(R.ch[1]);
        em.line(lvl, "if (" + cond_to(t, th) + ") {");
        emit(R.ch[1], lvl + 1);
        em.line(lvl, "} else {");
        emit(R.ch[2], lvl + 1);
        em.line(lvl, "}");
        if (R.ch.size() == 4) emit(R.ch[3], lvl);
        break;
      }
      case R_LOOP: {
        uint32_t h = (uint32_t)rd.head(R.ch[0]);
        uint32_t t = (uint32_t)rd.tail(R.ch.back());
        uint32_t exitb = K.lcfg.blocks[t].succ0 == h ? K.lcfg.blocks[t].succ1 : K.lcfg.blocks[t].succ0;
        // With an early exit, the exit block's join versions are also assigned before the
        // `break`, so the latch's exit copies cannot follow the loop (they would overwrite
        // those): they go at the end of every iteration, before the loop-carried copies.  They
        // assign only versions of the exit block, which the loop does not read.
        bool has_break = false;
        for (int l : rd.brk_latch) has_break |= l == (int)t;
        em.line(lvl, "do {");
        for (int c : R.ch) emit(c, lvl + 1);
        if (has_break && exitb != NONE) em.copies(t, exitb, lvl + 1);
        em.copies(t, h, lvl + 1);
        em.line(lvl, "} while (" + cond_to(t, h) + ");");
        if (!has_break && exitb != NONE) em.copies(t, exitb, lvl);
        break;
      }
    }
  }
};

std::string arg_list(const Config& c) {
  std::string s;
  for (const Arg& a : c.args) {
    if (a.hidden) continue;
    if (!s.empty()) s += ", ";
    if (a.pointer) {
      s += a.space == 1 ? "__constant " : (a.space == 2 ? "__local " : "__global ");
      if (a.is_const) s += "const ";
      s += std::string(type_name(a.elem)) + " *" + a.name;
    } else {
      s += std::string(type_name(a.elem)) + " " + a.name;
    }
  }
  return s.empty() ? "void" : s;
}

void decompile_kernel(Kernel& K, const RawKernel& raw) {
  K.name = raw.name;
  K.cfg = parse_config(raw.config);
  auto fail = [&](int st, const char* why, bool args) {
    K.status = st;
    K.out_text = "__kernel void " + K.name + "(" + (args ? arg_list(K.cfg) : std::string()) + ")\n{\n    /* not decompiled: " +
                 why + " */\n}\n";
  };
  if (K.cfg.bad) return fail(ST_PARSE_ERROR, "parse error", false);
  K.dec = decode(raw.text, K.cfg);
  K.pcfg = physical_cfg(K.dec);
  if (K.dec.bad) return fail(ST_PARSE_ERROR, "parse error", false);
  K.lcfg = logical_cfg(K.dec);
  if (K.lcfg.bad) return fail(ST_PARSE_ERROR, "parse error", false);
  uint32_t nspill = 0;
  for (const auto& r : K.dec.ins)
    if (r.op == BUFFER_LOAD_DWORD || r.op == BUFFER_STORE_DWORD) nspill = std::max(nspill, r.imm / 4 + 1);
  K.R = Regs{(uint32_t)K.cfg.vgprs, (uint32_t)K.cfg.sgprs, nspill,
             (uint32_t)K.cfg.vgprs + (uint32_t)K.cfg.sgprs + 2 + nspill};
  if (K.R.R > 1024 || K.lcfg.blocks.size() >= (1u << 18) || K.dec.ins.size() >= (1u << 26))
    return fail(ST_PARSE_ERROR, "parse error", false);
  find_fusions(K);
  dataflow(K);
  if (K.capped) return fail(ST_PARSE_ERROR, "parse error", false);
  build_nodes(K);
  Emitter em(K);
  em.mark_reach();
  em.infer_types();
  if (em.types_capped) return fail(ST_FIXPOINT_CAP, "fixed-point limit", true);
  em.number_vars();
  for (uint32_t id = 0; id < K.nodes.size(); ++id) {
    if (!em.reach[id]) continue;
    for (uint32_t c : em.children(id))
      if (c == UNDEF) ++K.undef_reads;
  }
  for (uint32_t r : em.used_phis) {
    std::set<uint32_t> vals;
    for (uint32_t p : K.preds[em.phi_block(r)]) {
      uint32_t v = fwd(K, em.out_val(p, em.phi_reg(r)));
      if (v == UNDEF) ++K.undef_reads;
      if (v != r) vals.insert(v);
    }
    if (vals.size() < 2) ++K.trivial_phis;
  }
  K.n_vars = (uint32_t)em.var_type.size();
  K.n_phis = (uint32_t)em.used_phis.size();
  std::vector<char> live;
  Reducer rd = make_reducer(K, &live);
  int root = K.lcfg.blocks.empty() ? -2 : rd.run();
  if (root == -1) return fail(ST_PARTIAL, "unstructured control flow", true);
  std::string head = "__kernel void " + K.name + "(" + arg_list(K.cfg) + ")\n{\n";
  for (size_t v = 0; v < em.var_type.size(); ++v)
    head += std::string("    ") + type_name(em.var_type[v]) + " var" + std::to_string(v) + ";\n";
  if (root >= 0) {
    RegionPrinter rp{em, rd, K};
    rp.emit(root, 1);
  }
  K.out_text = head + em.out + "}\n";
  K.status = em.partial ? ST_PARTIAL : ST_OK;
}

struct FileResult {
  std::vector<Kernel> kernels;
  std::string text;
  int status = 0;
};

void run_file(FileResult& F, const char* text, size_t len) {
  std::vector<RawKernel> raws = extract_bodies(text, len);
  F.kernels.resize(raws.size());
  for (size_t k = 0; k < raws.size(); ++k) {
    decompile_kernel(F.kernels[k], raws[k]);
    if (k) F.text += "\n";
    F.text += F.kernels[k].out_text;
    F.status = std::max(F.status, F.kernels[k].status);
  }
}

}  // namespace

// ============================================================================
// C ABI of the oracle (used by tests and the benchmark's CPU baseline)
// ============================================================================
extern "C" {

// test hook: the depth below which classify gives no class (the default 4 changes no class)
void oracle_set_class_depth(int d) { g_class_depth = d < 0 ? 4 : d; }

void* oracle_decompile(const char* text, uint64_t len) {
  FileResult* F = new FileResult;
  run_file(*F, text, len);
  return F;
}
uint64_t oracle_text_len(void* h) { return ((FileResult*)h)->text.size(); }
void oracle_text(void* h, char* dst) {
  const std::string& s = ((FileResult*)h)->text;
  memcpy(dst, s.data(), s.size());
}
int oracle_nkernels(void* h) { return (int)((FileResult*)h)->kernels.size(); }
// sweep limit of the type fixed point for later calls (0 = the default); a test hook
void oracle_set_type_sweep_limit(uint32_t n) { g_type_sweep_limit = n ? n : kTypeSweepDefault; }
int oracle_kernel_status(void* h, int k) { return ((FileResult*)h)->kernels[k].status; }

// IR arrays: 0 InstrRec[n]; 1 physical block_of[n]; 2 physical blocks;
// 3 logical block_of[n]; 4 logical blocks; 5 used joins (block, reg, type, var);
// 6 variable types (u32 per variable)
static std::vector<uint8_t> ir_bytes(const Kernel& K, int which) {
  std::vector<uint8_t> v;
  auto put = [&](const void* p, size_t n) {
    const uint8_t* b = (const uint8_t*)p;
    v.insert(v.end(), b, b + n);
  };
  switch (which) {
    case 0: put(K.dec.ins.data(), K.dec.ins.size() * sizeof(InstrRec)); break;
    case 1: put(K.pcfg.block_of.data(), K.pcfg.block_of.size() * 4); break;
    case 2: put(K.pcfg.blocks.data(), K.pcfg.blocks.size() * sizeof(BlockRec)); break;
    case 3: put(K.lcfg.block_of.data(), K.lcfg.block_of.size() * 4); break;
    case 4: put(K.lcfg.blocks.data(), K.lcfg.blocks.size() * sizeof(BlockRec)); break;
    case 5: {  // configuration header
      uint32_t nuser = 0;
      for (const Arg& a : K.cfg.args) nuser += a.hidden ? 0 : 1;
      uint32_t h[8] = {(uint32_t)K.cfg.dims, (uint32_t)K.cfg.cws[0], (uint32_t)K.cfg.cws[1], (uint32_t)K.cfg.cws[2],
                       (uint32_t)K.cfg.sgprs, (uint32_t)K.cfg.vgprs, (uint32_t)K.cfg.useargs, nuser};
      put(h, sizeof h);
      break;
    }
    case 6: {  // statistics: dataflow sweeps, undefined reads, variables, used joins, trivial joins
      uint32_t h[5] = {K.sweeps, K.undef_reads, K.n_vars, K.n_phis, K.trivial_phis};
      put(h, sizeof h);
      break;
    }
  }
  return v;
}
uint64_t oracle_ir_len(void* h, int k, int which) { return ir_bytes(((FileResult*)h)->kernels[k], which).size(); }
void oracle_ir(void* h, int k, int which, void* dst) {
  std::vector<uint8_t> v = ir_bytes(((FileResult*)h)->kernels[k], which);
  memcpy(dst, v.data(), v.size());
}
void oracle_free(void* h) { delete (FileResult*)h; }

// test hook: the type-lattice join
int oracle_type_join(int a, int b) { return tjoin(a, b); }

// many files [off[i], off[i+1]) of `text`, `threads` host threads
struct Batch {
  std::vector<std::string> out;
  std::vector<int> status;
  std::vector<int> nkern;
};
void* oracle_batch(const char* text, const uint64_t* off, uint64_t nfiles, int threads) {
  Batch* B = new Batch;
  B->out.resize(nfiles);
  B->status.resize(nfiles);
  B->nkern.resize(nfiles);
  if (threads < 1) threads = 1;
  auto work = [&](int t) {
    for (uint64_t f = (uint64_t)t; f < nfiles; f += (uint64_t)threads) {
      FileResult F;
      run_file(F, text + off[f], off[f + 1] - off[f]);
      B->out[f] = std::move(F.text);
      B->status[f] = F.status;
      B->nkern[f] = (int)F.kernels.size();
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < threads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  return B;
}
uint64_t oracle_batch_len(void* h) {
  uint64_t n = 0;
  for (auto& s : ((Batch*)h)->out) n += s.size();
  return n;
}
void oracle_batch_copy(void* h, char* dst, uint64_t* out_off, int32_t* status) {
  Batch* B = (Batch*)h;
  uint64_t p = 0;
  for (size_t f = 0; f < B->out.size(); ++f) {
    out_off[f] = p;
    memcpy(dst + p, B->out[f].data(), B->out[f].size());
    p += B->out[f].size();
    status[f] = B->status[f];
  }
  out_off[B->out.size()] = p;
}
void oracle_batch_free(void* h) { delete (Batch*)h; }

// Structural analysis alone on an abstract graph (blocks 0..n-1, entry 0;
// succ1 = -1 for one successor, succ0 = -1 for none).  Every block with two
// successors counts as a conditional branch.  Writes the merges as
// [new id, member count, members...] and returns the number of ints written,
// or -1 when the graph does not reduce.
int oracle_reduce_graph(int n, const int* succ0, const int* succ1, int* out, int cap) {
  Reducer rd;
  rd.reg.resize(n);
  rd.succ.resize(n);
  rd.pred.resize(n);
  rd.alive.assign(n, 1);
  rd.cond_block.assign(n, 0);
  rd.bsucc.resize(n);
  for (int b = 0; b < n; ++b) {
    rd.reg[b] = Region{R_BLOCK, {}, (uint32_t)b};
    if (succ0[b] >= 0) rd.succ[b].push_back(succ0[b]);
    if (succ1[b] >= 0 && succ1[b] != succ0[b]) rd.succ[b].push_back(succ1[b]);
    rd.bsucc[b] = rd.succ[b];
    rd.cond_block[b] = rd.succ[b].size() == 2;
  }
  for (int b = 0; b < n; ++b)
    for (int s : rd.succ[b]) rd.pred[s].insert(b);
  int root = rd.run();
  int w = 0;
  for (size_t k = 0; k < rd.log.size(); ++k) {
    if (w + 2 + (int)rd.log[k].size() > cap) return -2;
    out[w++] = n + (int)k;
    out[w++] = (int)rd.log[k].size();
    for (int m : rd.log[k]) out[w++] = m;
  }
  return root < 0 ? -1 : w;
}

}  // extern "C"
