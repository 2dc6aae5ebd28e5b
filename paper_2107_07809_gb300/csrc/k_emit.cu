// k_emit.cu — S13: OpenCL generation.
//
// Output conventions (the paper fixes none; these are the project's): the
// signature lists the user arguments (`__global T *name`, scalars `T name`);
// variables `varN` are declared first, numbered in program order; every
// binary operation is parenthesised; an operand whose recovered type differs
// from the operation's type gets a cast (integers) or as_T (reinterpretation);
// a value at a join is assigned on the edges into the join; 4-space indent.
// Unsupported instructions stay as inline asm ("Practical implementation").
//
// Layout: a warp per kernel (lane 0) walks the region tree (explicit stack)
// and lays out items: the head, declaration chunks, the statements of a block,
// join copies and control lines.  Printing: the statements of blocks become
// one sub-item per printing instruction, every other item one sub-item.  The
// sub-items are ordered by shape (a counting sort on the item kind, the
// printing node's operation and the shapes of its first two operands), so
// that the lanes of a warp print alike statements; one thread per sub-item
// prints into a fixed staging slot (expressions recursively, one call frame
// per level, with a depth guard; operations, leaves and conversions through
// tables) and records the exact length, a scan places every sub-item, a
// warp-per-32 copy moves the staged bytes, and the few sub-items longer than
// a slot are printed again straight into place.  The printer calls the
// pattern matchers from many places; inlining them there made the emission
// kernel megabytes long (instruction-cache bound).
#define GD_MATCH_INLINE __noinline__
#include "k_analysis.cuh"
#include "region_red.cuh"

namespace gd {

// Byte writer.  Bytes go out through an inline-asm store the compiler does
// not treat as a memory access: a plain byte store may alias anything, which
// made every character reload and store the cursor of a stack-resident
// writer.  The output buffer is never read back through C++ accesses (only
// through ld_u8 below), so hiding the stores is safe.
__device__ __forceinline__ void st_u8(uint8_t* a, char ch) {
  asm volatile("st.u8 [%0], %1;" ::"l"(a), "h"((unsigned short)(uint8_t)ch));
}
__device__ __forceinline__ uint8_t ld_u8(const uint8_t* a) {
  unsigned short v;
  asm volatile("ld.u8 %0, [%1];" : "=h"(v) : "l"(a));
  return (uint8_t)v;
}

struct Wr {
  uint8_t* p;
  uint32_t n;    // bytes produced so far (also those beyond cap)
  uint32_t cap;  // bytes that may be stored at p
  bool ovf;      // some byte fell beyond cap
  __device__ __forceinline__ void c(char ch) {
    if (n < cap) st_u8(p + n, ch);
    else ovf = true;
    ++n;
  }
  __device__ __noinline__ void s(const char* z) {
    uint32_t m = n;
    for (; *z; ++z, ++m) {
      if (m < cap) st_u8(p + m, *z);
      else ovf = true;
    }
    n = m;
  }
  __device__ __noinline__ void mem(const uint8_t* a, uint32_t len) {
    uint32_t m = n;
    for (uint32_t i = 0; i < len; ++i, ++m) {
      if (m < cap) st_u8(p + m, (char)a[i]);
      else ovf = true;
    }
    n = m;
  }
  __device__ __noinline__ void u64(uint64_t v) {
    char t[20];
    int k = 0;
    do {
      t[k++] = (char)('0' + v % 10);
      v /= 10;
    } while (v);
    uint32_t m = n;
    while (k) {
      if (m < cap) st_u8(p + m, t[--k]);
      else {
        ovf = true;
        --k;
      }
      ++m;
    }
    n = m;
  }
  __device__ void i64(int64_t v) {
    if (v < 0) {
      c('-');
      u64(0 - (uint64_t)v);
    } else {
      u64((uint64_t)v);
    }
  }
  __device__ __noinline__ void indent(int lvl) {
    uint32_t m = n;
    for (int i = 0; i < 4 * lvl; ++i, ++m) {
      if (m < cap) st_u8(p + m, ' ');
      else ovf = true;
    }
    n = m;
  }
};

__device__ const char* tname(uint8_t t) {
  switch (t) {
    case TY_INT: return "int";
    case TY_UINT: return "uint";
    case TY_FLOAT: return "float";
    case TY_LONG: return "long";
    case TY_ULONG: return "ulong";
    case TY_DOUBLE: return "double";
  }
  return "uint";
}
__device__ __forceinline__ bool tint(uint8_t t) { return t == TY_INT || t == TY_UINT || t == TY_LONG || t == TY_ULONG; }
__device__ __forceinline__ int twidth(uint8_t t) { return ty64(t) ? 64 : 32; }

// exact short decimal when the value has few binary fraction digits, else as_float/as_double
__device__ __noinline__ void float_lit(Wr& w, uint64_t bits, bool dbl) {
  int mbits = dbl ? 52 : 23, ebits = dbl ? 11 : 8, bias = dbl ? 1023 : 127;
  uint64_t sign = bits >> (mbits + ebits);
  uint64_t ex = (bits >> mbits) & ((1ull << ebits) - 1);
  uint64_t man = bits & ((1ull << mbits) - 1);
  auto fallback = [&]() {
    w.s(dbl ? "as_double(" : "as_float(");
    w.u64(bits);
    w.s(dbl ? "UL)" : "u)");
  };
  if (bits == 0) {
    w.s(dbl ? "0.0" : "0.0f");
    return;
  }
  if (ex == (1ull << ebits) - 1 || ex == 0) return fallback();
  uint64_t m = man | (1ull << mbits);
  int e = (int)ex - bias - mbits;
  while ((m & 1) == 0 && e < 0) {
    m >>= 1;
    ++e;
  }
  if (e >= 0) {
    if (e > 62 || (m >> (63 - e)) != 0) return fallback();
    if (sign) w.c('-');
    w.u64(m << e);
    w.s(dbl ? ".0" : ".0f");
    return;
  }
  int k = -e;
  if (k > 16) return fallback();
  uint64_t p5 = 1;
  for (int i = 0; i < k; ++i) p5 *= 5;
  if (m > UINT64_MAX / p5) return fallback();
  uint64_t N = m * p5, p10 = 1;
  for (int i = 0; i < k; ++i) p10 *= 10;
  uint64_t ip = N / p10, fp = N % p10;
  char d[20];
  for (int i = k - 1; i >= 0; --i) {
    d[i] = (char)('0' + fp % 10);
    fp /= 10;
  }
  int len = k;
  while (len > 1 && d[len - 1] == '0') --len;
  if (sign) w.c('-');
  w.u64(ip);
  w.c('.');
  for (int i = 0; i < len; ++i) w.c(d[i]);
  if (!dbl) w.c('f');
}

__device__ __noinline__ void lit32(Wr& w, uint32_t bits, uint8_t want) {
  if (want == TY_INT) {
    int32_t v = (int32_t)bits;
    if (v == INT32_MIN) w.s("(-2147483647 - 1)");
    else w.i64(v);
  } else if (want == TY_FLOAT) {
    float_lit(w, bits, false);
  } else {
    w.u64(bits);
    w.c('u');
  }
}
__device__ __noinline__ void lit64(Wr& w, uint64_t bits, uint8_t want) {
  if (want == TY_LONG) {
    int64_t v = (int64_t)bits;
    if (v == INT64_MIN) w.s("(-9223372036854775807L - 1L)");
    else {
      w.i64(v);
      w.c('L');
    }
  } else if (want == TY_DOUBLE) {
    float_lit(w, bits, true);
  } else {
    w.u64(bits);
    w.s("UL");
  }
}

// How each operation is printed.  A template's characters are copied, except
// 1..3 (operand 0..2, converted to the type in ty: a TY_ value or kSelf, the
// node's own type) and 4..6 (the shift amount held by operand 0..2, masked
// with `mask`).  One template loop serves every operation, so lanes of a warp
// printing different operations run the same code.  Entry O_COUNT is a pair of
// 32-bit halves.
enum : uint8_t { F_NONE = 0, F_TPL, F_CARRY, F_LOAD4, F_LOAD8, F_BFE };
constexpr uint8_t kSelf = 0xFE;
struct Fmt {
  char tpl[64];
  uint8_t ty[3];
  uint8_t mask;
  uint8_t kind;
};
__device__ const Fmt g_fmt[O_COUNT + 1] = {
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"(\1 * \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 << \5)", {kSelf, TY_NONE, TY_NONE}, 31, F_TPL},
    {"(\1 + \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 == \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 != \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 > \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 < \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 >= \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 <= \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 == \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 != \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 > \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 < \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 >= \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 <= \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"(\1 + \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 - \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 * \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"mad24(\1, \2, \3)", {TY_UINT, TY_UINT, TY_UINT}, 0, F_TPL},
    {"mul24(\1, \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 & \2)", {kSelf, kSelf, TY_NONE}, 0, F_TPL},
    {"(\1 | \2)", {kSelf, kSelf, TY_NONE}, 0, F_TPL},
    {"(\1 ^ \2)", {kSelf, kSelf, TY_NONE}, 0, F_TPL},
    {"(\2 << \4)", {TY_NONE, kSelf, TY_NONE}, 31, F_TPL},
    {"(\2 >> \4)", {TY_NONE, TY_UINT, TY_NONE}, 31, F_TPL},
    {"(\2 >> \4)", {TY_NONE, TY_INT, TY_NONE}, 31, F_TPL},
    {"(\1 + \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 - \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 * \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"fma(\1, \2, \3)", {TY_FLOAT, TY_FLOAT, TY_FLOAT}, 0, F_TPL},
    {"(float)\1", {TY_INT, TY_NONE, TY_NONE}, 0, F_TPL},
    {"(float)\1", {TY_UINT, TY_NONE, TY_NONE}, 0, F_TPL},
    {"(double)\1", {TY_FLOAT, TY_NONE, TY_NONE}, 0, F_TPL},
    {"(double)\1", {TY_INT, TY_NONE, TY_NONE}, 0, F_TPL},
    {"(float)\1", {TY_DOUBLE, TY_NONE, TY_NONE}, 0, F_TPL},
    {"(\1 == \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 != \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 > \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 < \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 >= \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 <= \2)", {TY_INT, TY_INT, TY_NONE}, 0, F_TPL},
    {"(\1 == \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 != \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 > \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 < \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 >= \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 <= \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 == \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 != \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 > \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 < \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 >= \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 <= \2)", {TY_FLOAT, TY_FLOAT, TY_NONE}, 0, F_TPL},
    {"(\1 + \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 + \2)", {kSelf, kSelf, TY_NONE}, 0, F_CARRY},
    {"(\1 - \2)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"(\1 - \2)", {kSelf, kSelf, TY_NONE}, 0, F_CARRY},
    {"(\2 << \4)", {TY_NONE, kSelf, TY_NONE}, 63, F_TPL},
    {"(\1 + \2)", {TY_DOUBLE, TY_DOUBLE, TY_NONE}, 0, F_TPL},
    {"(\1 * \2)", {TY_DOUBLE, TY_DOUBLE, TY_NONE}, 0, F_TPL},
    {"fma(\1, \2, \3)", {TY_DOUBLE, TY_DOUBLE, TY_DOUBLE}, 0, F_TPL},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_LOAD4},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_LOAD8},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},
    {"(\3 ? \2 : \1)", {kSelf, kSelf, TY_NONE}, 0, F_TPL},
    {"(\1 >> \5)", {TY_UINT, TY_NONE, TY_NONE}, 31, F_TPL},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_BFE},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_LOAD4},  // flat_load_dword
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_LOAD8},  // flat_load_dwordx2
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},   // flat_store_dword (a statement, not a value)
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},   // flat_store_dwordx2
    // the high half of the 48-bit product of the operands' low 24 bits, zero- / sign-extended:
    // OpenCL's mul_hi of the operands reduced to 24 bits
    {"mul_hi((\1 & 16777215u), (\2 & 16777215u))", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"mul_hi(((int)(\1 << 8) >> 8), ((int)(\2 << 8) >> 8))", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_LOAD4},  // ds_read_b32 (an element of a __local buffer)
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_LOAD8},  // ds_read_b64
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},   // ds_write_b32 (a statement)
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},   // ds_write_b64
    {"", {TY_NONE, TY_NONE, TY_NONE}, 0, F_NONE},   // s_barrier (a statement)
    {"upsample(\2, \1)", {TY_UINT, TY_UINT, TY_NONE}, 0, F_TPL},
};

// Leaves: how a value reduced to a leaf kind (its class, or a variable) and a
// number is printed: pre, the number (or argument name, or literal), mid, the
// number again (NUM2), suf.  Every leaf goes through the same code.
enum : uint8_t { LF_F_NUM = 1, LF_F_NUM2 = 2, LF_F_NAME = 4, LF_F_LIT32 = 8, LF_F_LIT64 = 16, LF_F_PARTIAL = 32 };
constexpr uint8_t LF_VAR = 21, LF_EXPR = 22, LF_PART = 23;
struct LeafFmt {
  char pre[20];
  char mid[24];
  char suf[4];
  uint8_t flags;
};
static_assert(K_LID == 1 && K_UNDEF == 4 && K_GIDNO == 8 && K_ARGPTR == 10 && K_CONST64 == 14 && K_DISP == 15 &&
                  K_WDIM == 19 && K_LPTR == 20, "leaf table order");
__device__ const LeafFmt g_leaf[LF_VAR + 1] = {
    {"", "", "", 0},                                                   // K_NONE
    {"get_local_id(", "", ")", LF_F_NUM},                              // K_LID
    {"get_group_id(", "", ")", LF_F_NUM},                              // K_GRP
    {"0UL", "", "", LF_F_PARTIAL},                                     // K_KARG
    {"0u", "", "", LF_F_PARTIAL},                                      // K_UNDEF
    {"get_global_offset(", "", ")", LF_F_NUM},                         // K_GOFS64
    {"get_global_offset(", "", ")", LF_F_NUM},                         // K_GOFSLO
    {"", "", "", 0},                                                   // K_MULGRP (never a leaf)
    {"(get_global_id(", ") - get_global_offset(", "))", LF_F_NUM | LF_F_NUM2},  // K_GIDNO
    {"get_global_id(", "", ")", LF_F_NUM},                             // K_GID
    {"(ulong)", "", "", LF_F_NAME},                                    // K_ARGPTR
    {"", "", "", LF_F_NAME},                                           // K_ARG32
    {"", "", "", LF_F_NAME},                                           // K_ARG64
    {"", "", "", LF_F_LIT32},                                          // K_CONST32
    {"", "", "", LF_F_LIT64},                                          // K_CONST64
    {"0UL", "", "", LF_F_PARTIAL},                                     // K_DISP
    {"", "", "", 0},                                                   // K_DISP0 (never a leaf)
    {"get_global_size(", "", ")", LF_F_NUM},                           // K_GSIZE
    {"get_num_groups(", "", ")", LF_F_NUM},                            // K_NGRP
    {"get_work_dim()", "", "", 0},                                     // K_WDIM
    {"(uint)(ulong)", "", "", LF_F_NAME | LF_F_PARTIAL},               // K_LPTR (an LDS address, no element)
    {"var", "", "", LF_F_NUM},                                         // LF_VAR
};

// conversions: g_conv[want][from] is printed around a value of type `from` used as `want`
// (integer to integer and across widths a cast, same width otherwise as_T)
struct ConvFmt {
  char pre[12];
  char suf[2];
};
__device__ const ConvFmt g_conv[9][9] = {
    {{"", ""}, {"", ""}, {"", ""}, {"", ""}, {"", ""}, {"", ""}, {"", ""}, {"", ""}, {"", ""}},
    {{"as_int(", ")"}, {"", ""}, {"(int)", ""}, {"as_int(", ")"}, {"(int)", ""}, {"(int)", ""}, {"(int)", ""}, {"as_int(", ")"}, {"(int)", ""}},
    {{"as_uint(", ")"}, {"(uint)", ""}, {"", ""}, {"as_uint(", ")"}, {"(uint)", ""}, {"(uint)", ""}, {"(uint)", ""}, {"as_uint(", ")"}, {"(uint)", ""}},
    {{"as_float(", ")"}, {"as_float(", ")"}, {"as_float(", ")"}, {"", ""}, {"(float)", ""}, {"(float)", ""}, {"(float)", ""}, {"as_float(", ")"}, {"(float)", ""}},
    {{"(long)", ""}, {"(long)", ""}, {"(long)", ""}, {"(long)", ""}, {"", ""}, {"(long)", ""}, {"as_long(", ")"}, {"(long)", ""}, {"as_long(", ")"}},
    {{"(ulong)", ""}, {"(ulong)", ""}, {"(ulong)", ""}, {"(ulong)", ""}, {"(ulong)", ""}, {"", ""}, {"as_ulong(", ")"}, {"(ulong)", ""}, {"as_ulong(", ")"}},
    {{"(double)", ""}, {"(double)", ""}, {"(double)", ""}, {"(double)", ""}, {"as_double(", ")"}, {"as_double(", ")"}, {"", ""}, {"(double)", ""}, {"as_double(", ")"}},
    {{"as_uint(", ")"}, {"as_uint(", ")"}, {"as_uint(", ")"}, {"as_uint(", ")"}, {"(uint)", ""}, {"(uint)", ""}, {"(uint)", ""}, {"", ""}, {"(uint)", ""}},
    {{"(uint)", ""}, {"(uint)", ""}, {"(uint)", ""}, {"(uint)", ""}, {"as_uint(", ")"}, {"as_uint(", ")"}, {"as_uint(", ")"}, {"(uint)", ""}, {"", ""}},
};

// element type of load/store node id (slot 0 of its instruction): the argument's, else by width
__device__ __noinline__ uint8_t mem_elem_of(const KView& v, uint32_t id, uint32_t width) {
  Mem m = mem_of(v, id);
  if (m.ok) return v.A[m.arg].elem;
  return width == 8 ? TY_ULONG : TY_UINT;
}

// type of node id's own expression (nt: the kernel's node types)
__device__ __noinline__ uint8_t node_expr_type_of(const KView& v, const uint8_t* nt, uint32_t id) {
  const Node& n = v.node(id);
  uint8_t T = tresolve(nt[id], node_width(v, id));
  if (n.kind == N_PAIR) return TY_ULONG;
  if (n.kind != N_OP) return TY_UINT;
  uint16_t op = n.op;
  if (op_scmp(op) || op_vcmp(op)) return TY_INT;
  switch (op) {
    case O_S_ADD_U32: case O_V_ADD_U32: case O_V_SUB_U32: case O_V_MUL_LO_U32: case O_V_MAD_U32_U24:
    case O_V_MUL_U32_U24: case O_V_LSHRREV_B32: case O_V_ADD_CO_U32: case O_V_SUB_CO_U32: case O_S_LSHR_B32:
    case O_S_BFE_U32: return TY_UINT;
    case O_S_MUL_I32: case O_V_ASHRREV_I32: return TY_INT;
    case O_S_LSHL_B32: case O_V_AND_B32: case O_V_OR_B32: case O_V_XOR_B32: case O_V_LSHLREV_B32:
    case O_V_LSHLREV_B64: case O_V_CNDMASK_B32: return T;
    case O_V_ADD_F32: case O_V_SUB_F32: case O_V_MUL_F32: case O_V_FMA_F32: case O_V_CVT_F32_I32:
    case O_V_CVT_F32_U32: case O_V_CVT_F32_F64: return TY_FLOAT;
    case O_V_CVT_F64_F32: case O_V_CVT_F64_I32: case O_V_ADD_F64: case O_V_MUL_F64: case O_V_FMA_F64: return TY_DOUBLE;
    case O_V_ADDC_CO_U32: case O_V_SUBB_CO_U32: return n.fused ? T : TY_UINT;
    case O_GLOBAL_LOAD_DWORD: case O_GLOBAL_LOAD_DWORDX2: case O_FLAT_LOAD_DWORD: case O_FLAT_LOAD_DWORDX2:
    case O_DS_READ_B32: case O_DS_READ_B64:
      return mem_elem_of(v, id, op_mem_width(op));
    case O_V_MUL_HI_U32_U24: return TY_UINT;
    case O_V_MUL_HI_I32_I24: return TY_INT;
  }
  return T == TY_ULONG ? TY_ULONG : TY_UINT;
}

// What the printer reads of a node, in one 16-byte record per node slot,
// written after the analysis (k_print_records): one load per expression level
// instead of the node, its class, its variable and its types from six arrays.
struct PRec {
  uint16_t op;    // the node's operation
  uint8_t kind;   // N_*
  uint8_t fused;  // a fused 64-bit carry half
  uint8_t cls;    // class (K_*) and its number
  uint8_t clk;
  uint8_t nt;     // resolved node type
  uint8_t etype;  // type of the node's own expression
  int32_t var;    // its variable, or -1
  uint8_t vtype;  // the variable's type
  uint8_t pad[3];
};
static_assert(sizeof(PRec) == kPRecBytes, "PRec is 16 bytes");

struct Em {
  KView v;
  const PRec* pr;  // the kernel's print records (null: not built yet)
  const Batch* b;
  const KHdr* K;
  const uint32_t* uses;
  const uint8_t* fl;
  const uint8_t* nt;
  const int32_t* vo;
  const int32_t* pv;
  const uint8_t* vt;
  Wr w;
  bool partial;
  bool deep;

  __device__ uint8_t NT(uint32_t id) const { return tresolve(nt[id], node_width(v, id)); }
  __device__ int32_t phivar(uint32_t r) const {
    return pv[(size_t)((rid(r) >> 10) & 0x3FFFF) * K->R + (rid(r) & 0x3FF)];
  }

  // ---- conversions -----------------------------------------------------------
  __device__ __noinline__ void conv_open(uint8_t from, uint8_t want) {
    if (want == TY_NONE || from == want) return;
    if (tint(from) && tint(want)) {
      w.c('(');
      w.s(tname(want));
      w.c(')');
    } else if (twidth(from) == twidth(want)) {
      w.s("as_");
      w.s(tname(want));
      w.c('(');
    } else {
      w.c('(');
      w.s(tname(want));
      w.c(')');
    }
  }
  __device__ __noinline__ void conv_close(uint8_t from, uint8_t want) {
    if (want == TY_NONE || from == want) return;
    if (!(tint(from) && tint(want)) && twidth(from) == twidth(want)) w.c(')');
  }

  // ---- types of expressions (computed before printing) ------------------------
  __device__ __forceinline__ uint8_t mem_elem(const Node& n, uint32_t width) {
    return mem_elem_of(v, (uint32_t)(&n - v.N), width);
  }
  __device__ __forceinline__ uint8_t node_expr_type(uint32_t id) { return node_expr_type_of(v, nt, id); }

  __device__ __noinline__ uint8_t expr_type(uint32_t r, uint8_t want) {
    r = fwd(v, r);
    if (r_phi(r)) {
      int32_t x = phivar(r);
      return x < 0 ? TY_UINT : vt[x];
    }
    Cls c = classify(v, r);
    switch (c.c) {
      case K_UNDEF: case K_LID: case K_GRP: case K_GID: case K_GIDNO: case K_GOFSLO: case K_GSIZE: case K_NGRP:
      case K_WDIM: case K_LPTR: return TY_UINT;
      case K_GOFS64: case K_ARGPTR: case K_KARG: case K_DISP: return TY_ULONG;
      case K_ARG32: case K_ARG64: return v.A[c.k].elem;
      case K_CONST32: {
        uint8_t t = want == TY_NONE ? TY_UINT : want;
        return twidth(t) == 64 ? TY_UINT : t;
      }
      case K_CONST64: {
        uint8_t t = want == TY_NONE ? TY_ULONG : want;
        return twidth(t) == 32 ? TY_ULONG : t;
      }
    }
    if (!r_node(r)) return TY_UINT;
    uint32_t id = rid(r);
    if (rpart(r) != PART_ENTIRE) return TY_UINT;
    if (vo[id] >= 0) return vt[vo[id]];
    return node_expr_type(id);
  }

  // ---- printing -------------------------------------------------------------
  // P(r, want, d) prints value r for a use of type `want`: a conversion when the value's own type
  // differs, then the value (a join variable, a recovered system value or argument, a literal, a
  // variable, or the node's expression with its operands printed by P again).  With `top` set it
  // prints node rid(r)'s own expression, ignoring its variable, with no conversion (the right-hand
  // side of a statement, a branch condition).  The value is first reduced to a leaf kind and a
  // number, printed through the leaf table by one code path, or to an expression; the operand
  // helpers are inlined into P, so an expression level costs one call frame.
  __device__ __noinline__ void P(uint32_t r, uint8_t want, int d, bool top) {
    if (top) return body(rid(r), d);
    // the node's record answers forwarding, class, variable and types at once; a copy or a pair
    // goes the long way
    PRec rec;
    bool pre = false;  // rec belongs to node rid(r), and r needs no forwarding
    if (r_node(r)) {
      rec = pr[rid(r)];
      const bool copy = rec.kind == N_OP && (rec.op == O_V_MOV_B32 || rec.op == O_S_MOV_B32 ||
                                             rec.op == O_BUFFER_STORE_DWORD || rec.op == O_BUFFER_LOAD_DWORD);
      if ((copy && rpart(r) == PART_ENTIRE) || rec.kind == N_PAIR) r = fwd(v, r);
      else pre = true;
    } else if (r == kTop) {
      r = kUndef;  // what forwarding makes of it
    }
    uint8_t t, lk;  // the value's type; its leaf kind (a class, LF_VAR, or LF_EXPR / LF_PART)
    uint32_t num = 0, id = 0;
    if (r_phi(r)) {
      const int32_t x = phivar(r);
      t = x < 0 ? TY_UINT : vt[x];
      lk = x < 0 ? (uint8_t)K_UNDEF : LF_VAR;
      num = (uint32_t)x;
    } else {
      const Cls c = (pre && rpart(r) == PART_ENTIRE)                  ? Cls{rec.cls, rec.clk}
                    : (v.cc && r_node(r) && rpart(r) == PART_ENTIRE) ? Cls{v.cc[rid(r)], v.ck[rid(r)]}
                                                                     : classify(v, r);
      lk = c.c;
      num = c.k;
      switch (c.c) {
        case K_UNDEF: case K_LID: case K_GRP: case K_GID: case K_GIDNO: case K_GOFSLO: case K_GSIZE: case K_NGRP:
        case K_WDIM: case K_LPTR: t = TY_UINT; break;
        case K_GOFS64: case K_ARGPTR: case K_KARG: case K_DISP: t = TY_ULONG; break;
        case K_ARG32: case K_ARG64: t = v.A[c.k].elem; break;
        case K_CONST32: {
          const uint8_t u = want == TY_NONE ? TY_UINT : want;
          t = twidth(u) == 64 ? TY_UINT : u;
          break;
        }
        case K_CONST64: {
          const uint8_t u = want == TY_NONE ? TY_ULONG : want;
          t = twidth(u) == 32 ? TY_ULONG : u;
          break;
        }
        default:
          if (!r_node(r)) {
            t = TY_UINT;
            lk = K_UNDEF;
          } else if (rpart(r) != PART_ENTIRE) {
            t = TY_UINT;
            lk = LF_PART;
            id = rid(r);
          } else if ((pre ? rec.var : vo[rid(r)]) >= 0) {
            num = (uint32_t)(pre ? rec.var : vo[rid(r)]);
            t = pre ? rec.vtype : vt[num];
            lk = LF_VAR;
          } else {
            id = rid(r);
            t = pre ? rec.etype : node_expr_type(id);
            lk = LF_EXPR;
          }
      }
    }
    const bool conv = want != TY_NONE && t != want;
    // (a code beyond the lattice prints like top32: "uint", 32 bits wide, not an integer type)
    const ConvFmt& cf = g_conv[want > TY_TOP64 ? TY_TOP32 : want][t > TY_TOP64 ? TY_TOP32 : t];
    if (conv) w.s(cf.pre);
    if (d > 200) {
      deep = true;
      w.s("0u");
    } else if (lk == LF_EXPR) {
      body(id, d + 1);
    } else if (lk == LF_PART) {
      const uint32_t whole = mkref(id, PART_ENTIRE);
      const bool dbl = expr_type(whole, TY_NONE) == TY_DOUBLE;
      if (rpart(r) == PART_LO) {
        w.s(dbl ? "(uint)as_ulong(" : "(uint)");
        P(whole, TY_NONE, d + 1, false);
        if (dbl) w.c(')');
      } else {
        w.s(dbl ? "(uint)(as_ulong(" : "(uint)(");
        P(whole, TY_NONE, d + 1, false);
        w.s(dbl ? ") >> 32)" : " >> 32)");
      }
    } else {
      const LeafFmt& L = g_leaf[lk];
      const uint8_t f = L.flags;
      if (f & LF_F_PARTIAL) partial = true;
      w.s(L.pre);
      if (f & LF_F_NAME) name(num);
      else if (f & LF_F_NUM) w.u64(num);
      else if (f & LF_F_LIT32) {
        uint8_t u = want == TY_NONE ? TY_UINT : want;
        if (twidth(u) == 64) u = TY_UINT;
        lit32(w, v.node(rid(r)).cval, u);
      } else if (f & LF_F_LIT64) {
        const Node& p = v.node(rid(r));
        const uint64_t lo = v.node(rid(nsrc(v, p, 0))).cval, hi = v.node(rid(nsrc(v, p, 1))).cval;
        uint8_t u = want == TY_NONE ? TY_ULONG : want;
        if (twidth(u) == 32) u = TY_ULONG;
        lit64(w, lo | (hi << 32), u);
      }
      w.s(L.mid);
      if (f & LF_F_NUM2) w.u64(num);
      w.s(L.suf);
    }
    if (conv) w.s(cf.suf);
  }

  __device__ void name(uint32_t slot) { w.mem(b->text + v.A[slot].name_off, v.A[slot].name_len); }

  __device__ __forceinline__ void S(const Node& n, int q, uint8_t t, int d) { P(nsrc(v, n, q), t, d, false); }
  __device__ __forceinline__ void shamt(uint32_t f, uint32_t mask, int d) {
    if (r_node(f) && rpart(f) == PART_ENTIRE && v.node(rid(f)).kind == N_CONST) {
      w.u64(v.node(rid(f)).cval & mask);
      return;
    }
    w.c('(');
    P(f, TY_UINT, d, false);
    w.s(" & ");
    w.u64(mask);
    w.s("u)");
  }
  __device__ __noinline__ void memref(const Node& n, uint32_t width, int d) {
    Mem m = mem_of(v, (uint32_t)(&n - v.N));
    if (m.ok) {
      name(m.arg);
      w.c('[');
      if (m.idx == kTop) w.c('0');
      else P(m.idx, TY_NONE, d, false);
      w.c(']');
      return;
    }
    if (op_lds(n.op)) {  // an LDS address that is no buffer element: pseudo-code
      partial = true;
      w.s("*((__local ");
      w.s(width == 8 ? "ulong" : "uint");
      w.s(" *)(");
      P(nsrc(v, n, 0), TY_UINT, d, false);
      w.s("))");
      return;
    }
    w.s("*((__global ");
    w.s(width == 8 ? "ulong" : "uint");
    w.s(" *)(");
    P(nsrc(v, n, 0), TY_ULONG, d, false);
    w.s("))");
  }

  // a node's own expression (ignoring its variable), operands at depth d
  __device__ __noinline__ void node_expr(uint32_t id, int d) { P(mkref(id, PART_ENTIRE), TY_NONE, d, true); }
  __device__ __forceinline__ void body(uint32_t id, int d) {
    const Node& n = v.node(id);  // its sources and constants, where a template needs them
    const PRec rec = pr[id];
    const uint8_t T = rec.nt;
    if (rec.kind != N_OP && rec.kind != N_PAIR) {
      partial = true;
      w.s("0u");
      return;
    }
    const Fmt& f = g_fmt[rec.kind == N_PAIR ? O_COUNT : rec.op];
    const uint8_t fk = f.kind;
    if (fk == F_LOAD4 || fk == F_LOAD8) return memref(n, fk == F_LOAD8 ? 8 : 4, d);
    if (fk == F_BFE) {
      // field operand: offset bits [4:0], width bits [22:16]; (src >> offset) masked to
      // width bits.  A field that is not a constant, or 32 bits wide or more, is not written.
      const uint32_t fo = nsrc(v, n, 1);
      if (r_node(fo) && rpart(fo) == PART_ENTIRE && v.node(rid(fo)).kind == N_CONST) {
        const uint32_t c = v.node(rid(fo)).cval, off = c & 31u, wd = (c >> 16) & 0x7Fu;
        if (wd < 32) {
          if (wd == 0) {
            w.s("0u");
            return;
          }
          w.s("((");
          S(n, 0, TY_UINT, d);
          w.s(" >> ");
          w.u64(off);
          w.s(") & ");
          lit32(w, (1u << wd) - 1u, TY_UINT);
          w.c(')');
          return;
        }
      }
    }
    if (fk == F_NONE || fk == F_BFE) {
      partial = true;
      w.s(T == TY_ULONG ? "0UL" : "0u");
      return;
    }
    // a carry half not fused into a 64-bit operation keeps 32-bit operands and is not exact
    const bool lone = fk == F_CARRY && !rec.fused;
    if (lone) partial = true;
    for (int i = 0; i < (int)sizeof(f.tpl); ++i) {
      const char c = f.tpl[i];
      if (!c) break;
      if (c <= 3) {
        const uint8_t t = f.ty[c - 1];
        S(n, c - 1, t != kSelf ? t : (lone ? TY_UINT : T), d);
      } else if (c <= 6) {
        shamt(nsrc(v, n, c - 4), f.mask, d);
      } else {
        w.c(c);
      }
    }
  }

  // ---- statements ---------------------------------------------------------------
  // statements of instruction i: its operand-slot variables, then its result
  __device__ __noinline__ void instr_stmts(uint32_t i, int lvl) {
    {
      uint32_t gi = K->first_instr + i;
      const int order[4] = {1, 2, 3, 0};
      for (int q = 0; q < 4; ++q) {
        uint32_t id = 4 * i + (uint32_t)order[q];
        const Node& n = v.node(id);
        if (n.kind == N_OP && order[q] == 0 && n.op == O_UNKNOWN && (fl[id] & 1)) {
          w.indent(lvl);
          w.s("__asm__(\"");
          const uint8_t* p = b->text + b->line_start[b->instr_line[gi]];
          const uint8_t* e = b->text + b->line_start[b->instr_line[gi] + 1] - 1;
          while (p < e && is_space(*p)) ++p;
          while (e > p && is_space(e[-1])) --e;
          for (; p < e; ++p) {
            if (*p == '"' || *p == '\\') w.c('\\');
            w.c((char)*p);
          }
          w.s("\");\n");
          partial = true;
          continue;
        }
        if (n.kind == N_OP && order[q] == 0 && op_store(n.op) && (fl[id] & 1)) {
          uint32_t width = op_mem_width(n.op);
          uint8_t elem = mem_elem(n, width);
          w.indent(lvl);
          memref(n, width, 0);
          w.s(" = ");
          P(nsrc(v, n, 1), elem, 0, false);
          w.s(";\n");
          continue;
        }
        if (n.kind == N_OP && order[q] == 0 && n.op == O_S_BARRIER) {  // at its program point
          w.indent(lvl);
          w.s("barrier(CLK_LOCAL_MEM_FENCE);\n");
          continue;
        }
        if (vo[id] >= 0) {
          uint8_t t = node_expr_type(id), want = vt[vo[id]];
          w.indent(lvl);
          w.s("var");
          w.u64((uint64_t)vo[id]);
          w.s(" = ");
          conv_open(t, want);
          node_expr(id, 0);
          conv_close(t, want);
          w.s(";\n");
        }
      }
    }
  }

  // one assignment of the join version of register reg at block s along p -> s
  __device__ __noinline__ void one_copy(uint32_t s, uint32_t reg, uint32_t p, int lvl) {
    uint32_t dst = phiref(s, reg);
    uint32_t o = b->st_out[K->state_off + (size_t)p * K->R + reg];
    uint32_t src = fwd(v, o == kTop ? kUndef : o);
    int32_t x = phivar(dst);
    w.indent(lvl);
    w.s("var");
    w.u64((uint64_t)x);
    w.s(" = ");
    P(src, vt[x], 0, false);
    w.s(";\n");
  }


  // condition under which block t's terminator goes to block dst
  __device__ __noinline__ void cond_to(uint32_t t, uint32_t dst) {
    const BlockRec& B = b->lblocks[K->first_lblock + t];
    uint32_t i = b->lterm[K->first_lblock + t];
    uint32_t c = nsrc(v, v.node(4 * i), 0);
    bool sense = b->sense[K->first_instr + i] != 0;
    bool positive = (dst != B.succ0) ? sense : !sense;
    if (r_node(c) && rpart(c) == PART_ENTIRE) {
      const Node& n = v.node(rid(c));
      if (n.kind == N_OP && (op_scmp(n.op) || op_vcmp(n.op)) && vo[rid(c)] < 0) {
        if (!positive) {
          w.c('!');
          node_expr(rid(c), 0);
          return;
        }
        // the comparison without its outer parentheses
        const uint32_t start = w.n;
        node_expr(rid(c), 0);
        const uint32_t end = w.n;
        if (end <= w.cap) {
          for (uint32_t q = start; q + 2 < end; ++q) st_u8(w.p + q, (char)ld_u8(w.p + q + 1));
        } else {
          w.ovf = true;  // the text is redone with room for all of it
        }
        w.n = end - 2;
        return;
      }
    }
    if (!positive) w.s("!(");
    P(c, TY_NONE, 0, false);
    if (!positive) w.c(')');
  }
};


__device__ void print_args(Wr& w, const Batch& b, const KHdr& K, const ArgRec* A) {
  bool any = false;
  for (uint32_t q = 0; q < K.nargs; ++q) {
    const ArgRec& a = A[q];
    if (a.hidden) continue;
    if (any) w.s(", ");
    any = true;
    if (a.pointer) {
      w.s(a.space == 1 ? "__constant " : (a.space == 2 ? "__local " : "__global "));
      if (a.is_const) w.s("const ");
      w.s(tname(a.elem));
      w.s(" *");
    } else {
      w.s(tname(a.elem));
      w.c(' ');
    }
    w.mem(b.text + a.name_off, a.name_len);
  }
  if (!any) w.s("void");
}

// ---------------------------------------------------------------------------
// output items: a per-kernel walk lays them out in output order (count, then
// write at scanned offsets); one thread per item sizes it and, after a scan,
// writes it
// ---------------------------------------------------------------------------
enum : uint32_t { IT_NONE = 0, IT_HEAD, IT_DECLS, IT_BLOCK, IT_COPYSET, IT_IF, IT_ELSE, IT_CLOSE, IT_DO, IT_WHILE,
                  IT_TAIL, IT_FAIL, IT_BREAK };
// declarations per item: ten lines of at most 22 bytes ("    double var800000;") fit a
// staging slot, so declaration items are never printed twice
constexpr uint32_t kDeclChunk = 10;

// ---------------------------------------------------------------------------
// Copies on the edges into join blocks.  For CFG edge e = 2 * (global block p)
// + q (q = 0: succ0, 1: succ1) into block s: the used join versions of s
// whose incoming value along the edge differs from the version itself, in an
// order where no copy overwrites a version that a later copy still reads (a
// cycle marks the kernel partial when the edge is printed).  One thread per
// edge; the layout refers to an edge's copies as one item.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t next_used_bit(const uint32_t* pbits, uint64_t base, uint32_t reg, uint32_t R) {
  while (reg < R) {
    uint64_t g = base + reg;
    uint32_t w = pbits[g >> 5] >> (g & 31);
    if (w) {
      uint32_t r = reg + (uint32_t)(__ffs(w) - 1);
      return r < R ? r : R;
    }
    reg += 32 - (uint32_t)(g & 31);
  }
  return R;
}

// upper bound of the copies of each edge: the used join versions of its target
__global__ void k_copy_bound(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern,
                             const uint32_t* __restrict__ pbits, uint32_t* __restrict__ bound) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > 2 * b.NLB) return;
  if (e == 2 * b.NLB) {  // the end of the scanned array
    bound[e] = 0;
    return;
  }
  const uint32_t g = e >> 1;
  const KHdr& K = b.kh[blk_kern[g]];
  const BlockRec& B = b.lblocks[g];
  const uint32_t s = (e & 1) ? B.succ1 : B.succ0;
  uint32_t c = 0;
  if (!K.bad && s != kNone) {
    const uint64_t base = (uint64_t)K.state_off + (uint64_t)s * K.R;
    for (uint32_t r = next_used_bit(pbits, base, 0, K.R); r < K.R; r = next_used_bit(pbits, base, r + 1, K.R)) ++c;
  }
  bound[e] = c;
}

__global__ void k_copy_sets(const __grid_constant__ Batch b, const uint32_t* __restrict__ blk_kern,
                            const uint32_t* __restrict__ pbits, uint32_t* __restrict__ src_tmp) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * b.NLB) return;
  const uint32_t g = e >> 1;
  const uint32_t k = blk_kern[g];
  const KHdr& K = b.kh[k];
  const BlockRec& B = b.lblocks[g];
  const uint32_t s = (e & 1) ? B.succ1 : B.succ0;
  uint32_t m = 0;
  uint8_t cyc = 0;
  if (!K.bad && s != kNone) {
    const KView& v = b.kview[k];
    const uint32_t p = g - K.first_lblock, R = K.R, off = b.cs_off[e];
    uint32_t* reg_of = b.cs_reg + off;  // candidates, then the printing order
    uint32_t* src_of = src_tmp + off;
    const uint64_t base = (uint64_t)K.state_off + (uint64_t)s * R;
    for (uint32_t r = next_used_bit(pbits, base, 0, R); r < R; r = next_used_bit(pbits, base, r + 1, R)) {
      const uint32_t o = b.st_out[K.state_off + (size_t)p * R + r];
      const uint32_t src = fwd(v, o == kTop ? kUndef : o);
      if (src == phiref(s, r) || src == kUndef) continue;
      reg_of[m] = r;
      src_of[m] = src;
      ++m;
    }
    // sequentialise: repeatedly take the first copy whose destination no
    // other pending copy reads; the chosen order is written back in place
    uint32_t done = 0;
    while (done < m) {
      uint32_t pick = m;
      for (uint32_t q = done; q < m && pick == m; ++q) {
        const uint32_t dq = phiref(s, reg_of[q]);
        bool read = false;
        for (uint32_t x = done; x < m && !read; ++x)
          if (x != q && src_of[x] == dq) read = true;
        if (!read) pick = q;
      }
      if (pick == m) {
        cyc = 1;
        pick = done;
      }
      const uint32_t rr = reg_of[pick], ss = src_of[pick];
      for (uint32_t x = pick; x > done; --x) {  // keep the others in order
        reg_of[x] = reg_of[x - 1];
        src_of[x] = src_of[x - 1];
      }
      reg_of[done] = rr;
      src_of[done] = ss;
      ++done;
    }
  }
  b.cs_cnt[e] = m;
  b.cs_cyc[e] = cyc;
}

// ---------------------------------------------------------------------------
// Layout: one thread per kernel walks the region tree once and writes the
// kernel's items into its slice of a staging array (size bounded by
// layout_bound), counting them; a scan places the kernels and a copy compacts.
// ---------------------------------------------------------------------------
// items of a kernel: at most 4 per region (fewer than 3 per block) and 4 more per block for
// an early exit (if, copies, break, close)
__device__ __forceinline__ uint32_t layout_bound(const KHdr& K) {
  return 4 + (K.n_vars + kDeclChunk - 1) / kDeclChunk + (4 * kRegionsPerBlock + 4) * K.n_lblock;
}

__global__ void k_layout_bound(const __grid_constant__ Batch b, uint32_t* __restrict__ bound) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < b.K) bound[k] = layout_bound(b.kh[k]);
}

struct LayoutCtx {
  const Batch* b;
  KHdr* K;
  const BlockRec* BL;
  Item* items;
  uint32_t n, cap, k;
  bool over;
  __device__ void put(uint32_t kind, uint32_t lvl, uint32_t a, uint32_t bb) {
    if (n < cap) items[n] = Item{kind | (lvl << 8), k, a, bb};
    else over = true;
    ++n;
  }
  __device__ uint32_t edge(uint32_t p, uint32_t s) const {
    return 2 * (K->first_lblock + p) + (BL[p].succ0 == s ? 0u : 1u);
  }
  __device__ uint32_t ncopies(uint32_t p, uint32_t s) const { return b->cs_cnt[edge(p, s)]; }
  __device__ void copies(uint32_t p, uint32_t s, uint32_t lvl) {
    const uint32_t e = edge(p, s);
    if (!b->cs_cnt[e]) return;
    put(IT_COPYSET, lvl, e, 0);
    if (b->cs_cyc[e]) atomicOr(&K->partial, 1u);
  }
};

__global__ void k_layout(const __grid_constant__ Batch b, Item* __restrict__ stage, const uint32_t* __restrict__ stage_off,
                         uint32_t* __restrict__ item_cnt, uint32_t* __restrict__ stk_all) {
  uint32_t k = walk_kernel();
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  LayoutCtx L;
  L.b = &b;
  L.K = &K;
  L.BL = b.lblocks + K.first_lblock;
  L.items = stage + stage_off[k];
  L.n = 0;
  L.cap = layout_bound(K);
  L.k = k;
  L.over = false;
  K.partial = 0;
  if (K.bad) {
    L.put(IT_FAIL, 0, 0, 0);
    L.put(IT_TAIL, 0, 1, 0);
  } else if (K.capped) {
    L.put(IT_FAIL, 0, 1, 0);
    L.put(IT_TAIL, 0, 1, 0);
  } else if (K.n_lblock && K.root == kNone) {
    L.put(IT_FAIL, 0, 1, 0);
    L.put(IT_TAIL, 0, 1, 0);
  } else {
    L.put(IT_HEAD, 0, 0, 0);
    for (uint32_t x = 0; x < K.n_vars; x += kDeclChunk) L.put(IT_DECLS, 1, x, min(kDeclChunk, K.n_vars - x));
    if (K.n_lblock) {
      const uint32_t* RG = b.rg + (size_t)kRegionsPerBlock * K.first_lblock * RGW;
      const BlockRec* BL = L.BL;
      uint32_t* st = stk_all + kStackPerBlock * (size_t)K.first_lblock;
      uint32_t cap = kStackPerBlock * K.n_lblock, sp = 0;
      auto push = [&](uint32_t r, uint32_t lvl, uint32_t ph) {
        if (sp + 2 > cap) {
          atomicOr(b.err, ERR_STACK);
          return;
        }
        st[sp++] = r;
        st[sp++] = (lvl << 8) | ph;
      };
      push(K.root, 1, 0);
      while (sp >= 2) {
        uint32_t info = st[--sp];
        uint32_t r = st[--sp];
        uint32_t lvl = info >> 8, ph = info & 0xFF;
        const uint32_t* X = RG + (size_t)r * RGW;
        switch (X[RG_KIND]) {
          case R_BLOCK: {
            uint32_t bl = X[RG_BLOCK];
            const BlockRec& B = BL[bl];
            L.put(IT_BLOCK, lvl, bl, 0);
            uint32_t term = b.lterm[K.first_lblock + bl];
            bool cb = b.ctl[K.first_instr + term] == C_CBR && B.succ1 != kNone;
            const uint32_t lb = b.brk[K.first_lblock + bl];
            if (lb != kNone && lb != kBrkLatch) {  // an early exit: the join copies of each edge on its own path
              const uint32_t lh = BL[lb].succ0 <= lb ? BL[lb].succ0 : BL[lb].succ1;
              const uint32_t E = latch_exit(BL, lb, lh), xin = B.succ0 == E ? B.succ1 : B.succ0;
              L.put(IT_IF, lvl, bl, E);
              L.copies(bl, E, lvl + 1);
              L.put(IT_BREAK, lvl + 1, 0, 0);
              L.put(IT_CLOSE, lvl, 0, 0);
              L.copies(bl, xin, lvl);
            } else if (!cb && B.succ0 != kNone) {
              L.copies(bl, B.succ0, lvl);
            }
            break;
          }
          case R_SEQ:
            if (ph == 0) {
              push(r, lvl, 1);
              push(X[RG_CH], lvl, 0);
            } else {
              push(X[RG_CH + 1], lvl, 0);
            }
            break;
          case R_IF: {
            uint32_t t = RG[(size_t)X[RG_CH] * RGW + RG_TAIL];
            uint32_t th = RG[(size_t)X[RG_CH + 1] * RGW + RG_HEAD];
            if (ph == 0) {
              push(r, lvl, 1);
              push(X[RG_CH], lvl, 0);
            } else if (ph == 1) {
              L.put(IT_IF, lvl, t, th);
              push(r, lvl, 2);
              push(X[RG_CH + 1], lvl + 1, 0);
            } else {
              uint32_t other = BL[t].succ0 == th ? BL[t].succ1 : BL[t].succ0;
              if (L.ncopies(t, other)) {
                L.put(IT_ELSE, lvl, 0, 0);
                L.copies(t, other, lvl + 1);
              }
              L.put(IT_CLOSE, lvl, 0, 0);
              if (X[RG_NCH] == 3) push(X[RG_CH + 2], lvl, 0);
            }
            break;
          }
          case R_IFELSE: {
            uint32_t t = RG[(size_t)X[RG_CH] * RGW + RG_TAIL];
            uint32_t th = RG[(size_t)X[RG_CH + 1] * RGW + RG_HEAD];
            if (ph == 0) {
              push(r, lvl, 1);
              push(X[RG_CH], lvl, 0);
            } else if (ph == 1) {
              L.put(IT_IF, lvl, t, th);
              push(r, lvl, 2);
              push(X[RG_CH + 1], lvl + 1, 0);
            } else if (ph == 2) {
              L.put(IT_ELSE, lvl, 0, 0);
              push(r, lvl, 3);
              push(X[RG_CH + 2], lvl + 1, 0);
            } else {
              L.put(IT_CLOSE, lvl, 0, 0);
              if (X[RG_NCH] == 4) push(X[RG_CH + 3], lvl, 0);
            }
            break;
          }
          case R_LOOP: {
            uint32_t nch = X[RG_NCH];
            uint32_t h = RG[(size_t)X[RG_CH] * RGW + RG_HEAD];
            uint32_t t = RG[(size_t)X[RG_CH + nch - 1] * RGW + RG_TAIL];
            if (ph == 0) {
              L.put(IT_DO, lvl, 0, 0);
              push(r, lvl, 1);
              for (int q = (int)nch - 1; q >= 0; --q) push(X[RG_CH + q], lvl + 1, 0);
            } else {
              uint32_t exitb = BL[t].succ0 == h ? BL[t].succ1 : BL[t].succ0;
              // with an early exit the exit block's join versions are assigned before each
              // `break` too: the latch's exit copies go at the end of every iteration, before
              // the loop-carried ones (they assign only versions the loop does not read)
              const bool has_break = b.brk[K.first_lblock + t] == kBrkLatch;
              if (has_break && exitb != kNone) L.copies(t, exitb, lvl + 1);
              L.copies(t, h, lvl + 1);
              L.put(IT_WHILE, lvl, t, h);
              if (!has_break && exitb != kNone) L.copies(t, exitb, lvl);
            }
            break;
          }
        }
      }
    }
    L.put(IT_TAIL, 0, 0, 0);
  }
  if (L.over) atomicOr(b.err, ERR_CAPACITY);
  item_cnt[k] = min(L.n, L.cap);
}

// staged items -> their final places (thread per staging slot)
__global__ void k_items_place(const Item* __restrict__ stage, const uint32_t* __restrict__ stage_off, uint32_t K,
                              uint32_t total, const uint32_t* __restrict__ item_cnt,
                              const uint32_t* __restrict__ item_base, Item* __restrict__ items) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint32_t lo = 0, hi = K;  // last kernel with stage_off <= t
  while (lo + 1 < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (stage_off[mid] <= t) lo = mid;
    else hi = mid;
  }
  const uint32_t i = t - stage_off[lo];
  if (i < item_cnt[lo]) items[item_base[lo] + i] = stage[t];
}

// Sub-items.  Every instruction that may print a statement (a variable
// assignment of one of its four node slots, a store, inline asm) gets a rank
// among such instructions of the batch; a block item is split into one
// sub-item per such instruction of its range, every other item is one
// sub-item, so that a long block is printed by many threads instead of one.
__global__ void k_print_flag(const __grid_constant__ Batch b, uint32_t* __restrict__ flag) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi > b.I) return;
  uint32_t f = 0;
  if (gi < b.I && b.lblock_of[gi] != kNone) {
    const size_t id = 4 * (size_t)gi;
    const Node& n = b.nodes[id];
    if (n.kind == N_OP && (n.op == O_UNKNOWN || op_store(n.op)) && (b.nflag[id] & 1)) f = 1;
    if (n.kind == N_OP && n.op == O_S_BARRIER) f = 1;
    for (int q = 0; q < 4; ++q)
      if (b.var_of[id + q] >= 0) f = 1;
  }
  flag[gi] = f;
}

__global__ void k_print_list(uint32_t I, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank,
                             uint32_t* __restrict__ list) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi < I && flag[gi]) list[rank[gi]] = gi;
}

__global__ void k_item_weight(const __grid_constant__ Batch b, const Item* __restrict__ items, uint32_t NI,
                              const uint32_t* __restrict__ prank, uint32_t* __restrict__ weight) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NI) return;
  Item it = items[i];
  uint32_t w = 1;
  if ((it.kl & 0xFF) == IT_BLOCK) {
    const KHdr& K = b.kh[it.k];
    const BlockRec& B = b.lblocks[K.first_lblock + it.a];
    w = prank[K.first_instr + B.end] - prank[K.first_instr + B.first];
  } else if ((it.kl & 0xFF) == IT_COPYSET) {
    w = b.cs_cnt[it.a];
  }
  weight[i] = w;
}

// head of each non-empty item's sub-item range (the array is zeroed first; a
// max scan then gives every sub-item its item)
__global__ void k_sub_heads(const uint32_t* __restrict__ sub0, uint32_t NI, uint32_t* __restrict__ sub_item) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NI) return;
  if (sub0[i + 1] > sub0[i]) sub_item[sub0[i]] = i;
}

// Emission of sub-items.  Staging mode (stage != null): sub-item t prints into
// its own kEmitSlot-byte slot of `stage`, records its exact length, and
// appends itself to ovf_list when the text did not fit.  Direct mode
// (stage == null): sub-item list[t] prints straight into its final place in
// the output (used for the sub-items that overflowed their slot).
__global__ void __launch_bounds__(128, 12)
    k_items(const __grid_constant__ Batch b, const Item* __restrict__ items, const uint32_t* __restrict__ sub_item,
            const uint32_t* __restrict__ sub0, const uint32_t* __restrict__ prank, const uint32_t* __restrict__ pinstr,
            uint32_t N, const uint32_t* __restrict__ list, uint32_t* __restrict__ item_len,
            const uint32_t* __restrict__ item_off, uint8_t* stage, uint32_t* __restrict__ ovf_list,
            uint32_t* ovf_count, uint32_t lane_shift) {
  // with lane_shift 5 one warp handles one sub-item (lane 0 works): no
  // divergence between statements inside a warp
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt & ((1u << lane_shift) - 1u)) return;
  const uint32_t t = gt >> lane_shift;
  if (t >= N) return;
  const uint32_t sidx = list ? list[t] : t;
  const uint32_t i = sub_item[sidx];
  const uint32_t j = sidx - sub0[i];  // position inside the item
  Item it = items[i];
  uint32_t kind = it.kl & 0xFF, lvl = it.kl >> 8;
  uint32_t k = it.k;
  KHdr& K = b.kh[k];
  uint32_t q_stmt = 0;
  if (kind == IT_BLOCK) {
    const BlockRec& B = b.lblocks[K.first_lblock + it.a];
    const uint32_t gi = pinstr[prank[K.first_instr + B.first] + j];
    q_stmt = gi - K.first_instr;
    if (b.lblock_of[gi] != it.a) {
      if (stage) item_len[sidx] = 0;
      return;
    }
  }
  const ArgRec* A = b.args + (size_t)k * kMaxArgs;
  Em em;
  em.v = make_view(b, K, k);
  em.b = &b;
  em.K = &K;
  const size_t nb = 4 * (size_t)K.first_instr;
  em.uses = b.uses + nb;
  em.fl = b.nflag + nb;
  em.nt = b.ntype + nb;
  em.vo = b.var_of + nb;
  em.pv = b.phi_var + K.state_off;
  em.vt = b.var_type + nb + K.state_off;
  em.pr = b.prec + nb;
  if (stage) em.w = Wr{stage + (size_t)sidx * kEmitSlot, 0, kEmitSlot, false};
  else em.w = Wr{b.out + item_off[sidx], 0, item_len[sidx], false};
  em.partial = false;
  em.deep = false;
  Wr& w = em.w;
  switch (kind) {
    case IT_HEAD:
    case IT_FAIL:
      w.s("__kernel void ");
      w.mem(b.text + K.name_off, K.name_len);
      w.c('(');
      if (kind == IT_HEAD || it.a) print_args(w, b, K, A);
      w.s(")\n{\n");
      if (kind == IT_FAIL) {
        w.s("    /* not decompiled: ");
        w.s(K.bad ? "parse error" : K.capped ? "fixed-point limit" : "unstructured control flow");
        w.s(" */\n}\n");
      }
      break;
    case IT_DECLS:
      for (uint32_t x = it.a; x < it.a + it.b; ++x) {
        w.s("    ");
        w.s(tname(em.vt[x]));
        w.s(" var");
        w.u64(x);
        w.s(";\n");
      }
      break;
    case IT_BLOCK: em.instr_stmts(q_stmt, (int)lvl); break;
    case IT_COPYSET: {
      const uint32_t p = (it.a >> 1) - K.first_lblock;
      const BlockRec& B = b.lblocks[it.a >> 1];
      em.one_copy((it.a & 1) ? B.succ1 : B.succ0, b.cs_reg[b.cs_off[it.a] + j], p, (int)lvl);
      break;
    }
    case IT_IF:
      w.indent((int)lvl);
      w.s("if (");
      em.cond_to(it.a, it.b);
      w.s(") {\n");
      break;
    case IT_ELSE: w.indent((int)lvl); w.s("} else {\n"); break;
    case IT_CLOSE: w.indent((int)lvl); w.s("}\n"); break;
    case IT_BREAK: w.indent((int)lvl); w.s("break;\n"); break;
    case IT_DO: w.indent((int)lvl); w.s("do {\n"); break;
    case IT_WHILE:
      w.indent((int)lvl);
      w.s("} while (");
      em.cond_to(it.a, it.b);
      w.s(");\n");
      break;
    case IT_TAIL: {
      if (!it.a) w.s("}\n");
      bool last = k + 1 == b.K || b.kh[k + 1].file != K.file;
      if (!last) w.c('\n');
      break;
    }
  }
  if (stage) {
    item_len[sidx] = w.n;
    if (w.ovf) ovf_list[atomicAdd(ovf_count, 1u)] = sidx;
    if (em.partial) atomicOr(&K.partial, 1u);
  }
  if (em.deep) atomicOr(b.err, ERR_STACK);
}

__global__ void k_kernel_status(const __grid_constant__ Batch b, const uint32_t* __restrict__ item_base, const uint32_t* __restrict__ sub0,
                                const uint32_t* __restrict__ item_off) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.K) return;
  KHdr& K = b.kh[k];
  if (K.bad) K.status = ST_PARSE_ERROR;
  else if (K.capped) K.status = ST_FIXPOINT_CAP;
  else if (K.n_lblock && K.root == kNone) K.status = ST_PARTIAL;
  else K.status = K.partial ? ST_PARTIAL : ST_OK;
  b.kout_off[k] = item_off[sub0[item_base[k]]];
}

// per file: output offset and worst status of its kernels
__global__ void k_file_out(const __grid_constant__ Batch b, uint32_t total) {
  uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f > b.F) return;
  uint32_t lo = 0, hi = b.K;  // first kernel with file >= f
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (b.kh[mid].file < f) lo = mid + 1;
    else hi = mid;
  }
  b.file_out_off[f] = lo < b.K ? b.kout_off[lo] : total;
  if (f == b.F) return;
  int32_t st = 0;
  for (uint32_t k = lo; k < b.K && b.kh[k].file == f; ++k) st = max(st, (int32_t)b.kh[k].status);
  b.file_status[f] = st;
}

void launch_copy_sets(Batch& b, const uint32_t* blk_kern, const uint32_t* pbits, uint32_t* bound_or_tmp, int phase,
                      cudaStream_t s) {
  if (!b.NLB) return;
  const uint32_t ne = 2 * b.NLB;
  if (phase == 0) k_copy_bound<<<(ne + 1 + 255) / 256, 256, 0, s>>>(b, blk_kern, pbits, bound_or_tmp);
  else k_copy_sets<<<(ne + 127) / 128, 128, 0, s>>>(b, blk_kern, pbits, bound_or_tmp);
  ++launch_counter();
}

void launch_layout(Batch& b, Item* stage, uint32_t* stage_off, uint32_t* item_cnt, uint32_t* stk, int phase,
                   cudaStream_t s) {
  if (!b.K) return;
  if (phase == 0) k_layout_bound<<<(b.K + 127) / 128, 128, 0, s>>>(b, stage_off);
  else k_layout<<<walk_blocks(b.K), walk_threads(b.K), 0, s>>>(b, stage, stage_off, item_cnt, stk);
  ++launch_counter();
}

void launch_items_place(const Item* stage, const uint32_t* stage_off, uint32_t K, uint32_t total,
                        const uint32_t* item_cnt, const uint32_t* item_base, Item* items, cudaStream_t s) {
  if (!total || !K) return;
  k_items_place<<<(total + 255) / 256, 256, 0, s>>>(stage, stage_off, K, total, item_cnt, item_base, items);
  ++launch_counter();
}

void launch_print_list(Batch& b, uint32_t* flag, const uint32_t* rank, uint32_t* list, int phase, cudaStream_t s) {
  if (phase == 0) {
    k_print_flag<<<(b.I + 1 + 255) / 256, 256, 0, s>>>(b, flag);
  } else {
    if (!b.I) return;
    k_print_list<<<(b.I + 255) / 256, 256, 0, s>>>(b.I, flag, rank, list);
  }
  ++launch_counter();
}

void launch_subitems(Batch& b, const Item* items, uint32_t NI, const uint32_t* prank, uint32_t* weight,
                     const uint32_t* sub0, uint32_t* sub_item, uint32_t NS2, int phase, cudaStream_t s) {
  if (!NI) return;
  if (phase == 0) {
    k_item_weight<<<(NI + 255) / 256, 256, 0, s>>>(b, items, NI, prank, weight);
    ++launch_counter();
  } else {
    cudaMemsetAsync(sub_item, 0, sizeof(uint32_t) * ((size_t)NS2 + 1), s);
    k_sub_heads<<<(NI + 255) / 256, 256, 0, s>>>(sub0, NI, sub_item);
    ++launch_counter();
  }
}

// staged sub-item texts that fit their slot -> final place; a warp moves `per`
// consecutive sub-items (32, or 1 for a small batch, where the copies of one
// warp would be the critical path), its lanes copying the bytes of one
// sub-item at a time
__global__ void __launch_bounds__(256)
    k_compact(const uint8_t* __restrict__ stage, const uint32_t* __restrict__ item_len,
              const uint32_t* __restrict__ item_off, uint32_t N, uint8_t* __restrict__ out, uint32_t per) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t s0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * per;
  if (s0 >= N) return;
  const uint32_t mine = s0 + lane;
  const bool own = lane < per && mine < N;
  const uint32_t len = own ? item_len[mine] : 0;
  const uint32_t off = own ? item_off[mine] : 0;
  unsigned todo = __ballot_sync(0xFFFFFFFFu, len > 0 && len <= kEmitSlot);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const uint32_t l = __shfl_sync(0xFFFFFFFFu, len, src);
    const uint32_t o = __shfl_sync(0xFFFFFFFFu, off, src);
    const uint8_t* from = stage + (size_t)(s0 + src) * kEmitSlot;
    for (uint32_t q = lane; q < l; q += 32) out[o + q] = from[q];
  }
}

// Print records: one thread per instruction, its four node slots.
__global__ void __launch_bounds__(128, 12) k_print_records(const __grid_constant__ Batch b) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.I) return;
  // only reached nodes are ever printed (the reachability walk follows the printed operands)
  const uint32_t f4 = reinterpret_cast<const uint32_t*>(b.nflag)[gi];
  if (!(f4 & 0x01010101u)) return;
  const uint32_t k = b.ikern[gi];
  const KHdr& K = b.kh[k];
  if (K.bad) return;
  const size_t nb = 4 * (size_t)K.first_instr;
  const KView& v = b.kview[k];
  const uint8_t* nt = b.ntype + nb;
  const int32_t* vo = b.var_of + nb;
  const uint8_t* vt = b.var_type + nb + K.state_off;
  const uint32_t id0 = 4 * (gi - K.first_instr);
  for (uint32_t s = 0; s < 4; ++s) {
    if (!((f4 >> (8 * s)) & 1u)) continue;
    const uint32_t id = id0 + s;
    const Node& n = v.node(id);
    PRec r;
    r.op = n.op;
    r.kind = n.kind;
    r.fused = n.fused;
    r.cls = v.cc[id];
    r.clk = v.ck[id];
    r.nt = tresolve(nt[id], node_width(v, id));
    r.var = vo[id];
    // the expression's type is read for a node printed in place (no variable, no leaf class)
    r.etype = (r.var < 0 && !leaf_like(r.cls) && (n.kind == N_OP || n.kind == N_PAIR)) ? node_expr_type_of(v, nt, id)
                                                                                        : TY_UINT;
    r.vtype = r.var >= 0 ? vt[r.var] : 0;
    r.pad[0] = r.pad[1] = r.pad[2] = 0;
    b.prec[nb + id] = r;
  }
}

void launch_print_records(Batch& b, cudaStream_t s) {
  if (!b.I) return;
  k_print_records<<<(b.I + 127) / 128, 128, 0, s>>>(b);
  ++launch_counter();
}

// Printing order.  Lanes of a warp that print statements of different shapes
// walk different parts of the printer one after another (divergence, and an
// instruction working set larger than the instruction cache).  Sub-items are
// therefore printed in an order grouped by a shape key: the item kind, and for
// a block statement the printing node's operation and the shape of its first
// two operands (a variable, a recovered value, or the operation of an inlined
// expression).  The order only decides which thread prints which sub-item;
// every sub-item still prints into its own slot, so the output is unchanged.
constexpr uint32_t kShapeBuckets = 16384;

__device__ __forceinline__ uint32_t ref_shape(const KView& v, const int32_t* vo, uint32_t r) {
  if (r == kTop) return 1;
  if (r_phi(r)) return 2;
  if (!r_node(r)) return 3;
  const uint32_t id = rid(r);
  if (rpart(r) != PART_ENTIRE) return 4;
  if (vo[id] >= 0) return 5;
  const uint8_t c = v.cc[id];
  if (leaf_like(c)) return 8 + c;
  const Node& n = v.node(id);
  return n.kind == N_OP ? 32 + n.op : 28 + n.kind;
}

__global__ void __launch_bounds__(256)
    k_sub_key(const __grid_constant__ Batch b, const Item* __restrict__ items, const uint32_t* __restrict__ sub_item,
              const uint32_t* __restrict__ sub0, const uint32_t* __restrict__ prank, const uint32_t* __restrict__ pinstr,
              uint32_t N, uint32_t* __restrict__ key, uint32_t* __restrict__ hist) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t kk = kShapeBuckets;  // lanes past the end take no part
  if (t < N) {
    const uint32_t i = sub_item[t];
    const Item it = items[i];
    const uint32_t kind = it.kl & 0xFF;
    kk = kind;
    if (kind == IT_BLOCK) {
      const KHdr& K = b.kh[it.k];
      const BlockRec& B = b.lblocks[K.first_lblock + it.a];
      const uint32_t gi = pinstr[prank[K.first_instr + B.first] + (t - sub0[i])];
      if (b.lblock_of[gi] == it.a) {
        const KView& v = b.kview[it.k];
        const int32_t* vo = b.var_of + 4 * (size_t)K.first_instr;
        const uint32_t id = 4 * (gi - K.first_instr);
        const Node& n = v.node(id);
        uint32_t h = n.kind == N_OP ? n.op : 200u + n.kind, s0 = 0, s1 = 0;
        if (n.kind == N_OP && op_store(n.op)) {
          s0 = ref_shape(v, vo, nsrc(v, n, 1));
          const uint32_t x = v.midx[id / 4];
          s1 = v.marg[id / 4] == kNone ? 1 : (x == kTop ? 0 : ref_shape(v, vo, x));
        } else if (n.kind == N_OP && !op_gload(n.op)) {
          if (n.nsrc > 0) s0 = ref_shape(v, vo, nsrc(v, n, 0));
          if (n.nsrc > 1) s1 = ref_shape(v, vo, nsrc(v, n, 1));
        }
        h = h * 0x9E3779B1u ^ (s0 * 0x85EBCA77u) ^ (s1 * 0xC2B2AE3Du);
        h ^= h >> 15;
        kk = 16 + h % (kShapeBuckets - 16);
      }
    }
    key[t] = kk;
  }
  // one atomic per distinct key of the warp
  const unsigned grp = __match_any_sync(0xFFFFFFFFu, kk);
  if (kk < kShapeBuckets && (threadIdx.x & 31u) == (uint32_t)(__ffs(grp) - 1)) atomicAdd(&hist[kk], (uint32_t)__popc(grp));
}

__global__ void __launch_bounds__(256)
    k_sub_scatter(const uint32_t* __restrict__ key, uint32_t N, uint32_t* __restrict__ cursor,
                  uint32_t* __restrict__ order) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t kk = t < N ? key[t] : kShapeBuckets;
  const unsigned grp = __match_any_sync(0xFFFFFFFFu, kk);
  const uint32_t lane = threadIdx.x & 31u, leader = (uint32_t)(__ffs(grp) - 1);
  uint32_t base = 0;
  if (kk < kShapeBuckets && lane == leader) base = atomicAdd(&cursor[kk], (uint32_t)__popc(grp));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (kk < kShapeBuckets) order[base + __popc(grp & ((1u << lane) - 1u))] = t;
}

void launch_sub_order(Batch& b, const Item* items, const uint32_t* sub_item, const uint32_t* sub0,
                      const uint32_t* prank, const uint32_t* pinstr, uint32_t N, uint32_t* key, uint32_t* hist,
                      uint32_t* order, ScanScratch sc, cudaStream_t s) {
  if (!N) return;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kShapeBuckets, s);
  k_sub_key<<<(N + 255) / 256, 256, 0, s>>>(b, items, sub_item, sub0, prank, pinstr, N, key, hist);
  launch_scan(hist, hist, kShapeBuckets, 0, false, sc, nullptr, b.err, s);
  k_sub_scatter<<<(N + 255) / 256, 256, 0, s>>>(key, N, hist, order);
  launch_counter() += 2;
}
uint32_t shape_buckets() { return kShapeBuckets; }

void launch_items(Batch& b, const Item* items, const uint32_t* sub_item, const uint32_t* sub0, const uint32_t* prank,
                  const uint32_t* pinstr, uint32_t N, const uint32_t* list, uint32_t* item_len,
                  const uint32_t* item_off, uint8_t* stage, uint32_t* ovf_list, uint32_t* ovf_count,
                  uint32_t lane_shift, cudaStream_t s) {
  if (!N) return;
  const uint64_t threads = (uint64_t)N << lane_shift;
  k_items<<<(uint32_t)((threads + 127) / 128), 128, 0, s>>>(b, items, sub_item, sub0, prank, pinstr, N, list, item_len,
                                                          item_off, stage, ovf_list, ovf_count, lane_shift);
  ++launch_counter();
}

void launch_compact(const uint8_t* stage, const uint32_t* item_len, const uint32_t* item_off, uint32_t N,
                    uint8_t* out, cudaStream_t s) {
  if (!N) return;
  const uint32_t per = N <= kSmallBatchStmts ? 1u : 32u;
  const uint64_t warps = (N + per - 1) / per;
  k_compact<<<(uint32_t)((warps * 32 + 255) / 256), 256, 0, s>>>(stage, item_len, item_off, N, out, per);
  ++launch_counter();
}

void launch_finish(Batch& b, const uint32_t* item_base, const uint32_t* sub0, const uint32_t* item_off,
                   uint32_t total, cudaStream_t s) {
  if (b.K) {
    k_kernel_status<<<(b.K + 127) / 128, 128, 0, s>>>(b, item_base, sub0, item_off);
    ++launch_counter();
  }
  k_file_out<<<(b.F + 1 + 127) / 128, 128, 0, s>>>(b, total);
  ++launch_counter();
}

}  // namespace gd
