// gcngen — seeded synthetic AMD GCN (gfx9-syntax, CLRX-style) kernel generator.
//
// This is the shared INPUT module: the CPU oracle, the CUDA path, the tests and
// the benchmark all read the text it writes.  It holds none of the decompiler's
// arithmetic: it lowers a random typed program (expressions over work-item ids,
// buffer loads, a scalar argument and constants; stores; divergent and uniform
// if / if-else; counted loops) to GCN assembly text, the way a compiler would.
//
// Text layout follows the program-body structure of the paper's Listing 1 and
// the `.config`/`.arg` section of Listing 3 ("The body extraction", "Data type
// recovery").  Register conventions follow the ABI the paper describes in
// "Search for memory accesses": v0..v2 = local id, s6..s8 = group id (with
// .useargs), s[4:5] = pointer to the kernel settings (hidden global offsets at
// 0x0/0x8/0x10, user arguments from 0x30 in 8-byte slots).
//
// If-else lowering uses the exec-mask forms of "Search for control structures"
// (first form: two labels; second: label in the if part; third: label in the
// else part).  Loops (which the paper does not restore) are scalar-counter
// do-while loops, a project extension.
//
// Determinism: kernel k of a stream draws only from splitmix64 seeded with
// mix(seed, k); floating point is used only for the log-uniform length table,
// built by repeated IEEE multiplication (compile with -ffp-contract=off).

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace {

struct Rng {  // splitmix64
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
  bool chance(int pct) { return (int)below(100) < pct; }
  int range(int lo, int hi) { return lo + (int)below((uint32_t)(hi - lo + 1)); }
};

uint64_t mix(uint64_t a, uint64_t b) {
  Rng r{a ^ (b * 0xD1B54A32D192ED03ull) ^ 0x5851F42D4C957F2Dull};
  r.next();
  return r.next();
}

enum Ty { TI = 0, TU = 1, TF = 2, TD = 3, TL = 4 };
const char* kTyName[5] = {"int", "uint", "float", "double", "long"};
bool is64(int t) { return t == TD || t == TL; }

}  // namespace

extern "C" {
// Knobs of one synthetic workload (all fields plain integers).
struct gcngen_params {
  uint32_t min_len, max_len;   // target instruction count, log-uniform in [min,max]
  uint32_t type_mask;          // bit t set = value type t allowed (int,uint,float,double,long)
  int32_t w_if, w_ifelse, w_loop, w_uif;  // relative weights of control templates
  int32_t p_ctrl;              // percent chance that a statement opens a control structure
  int32_t max_depth;           // maximum nesting depth of control structures
  int32_t min_bufs, max_bufs;  // number of __global buffer arguments
  int32_t vgpr_budget, sgpr_budget;
  int32_t spills;              // 1 = locals beyond the VGPR budget live in scratch slots
  int32_t max_locals;
  int32_t expr_depth;          // maximum expression depth
  int32_t trip_max;            // loop trip counts drawn from [1, trip_max]
  int32_t dims;                // 0 = random 1 or 2, else fixed
  int32_t cws0, cws1;          // 0 = random work-group shape
  int32_t fixed_args;          // 1 = (__global int *a, __global float *b, uint n)
  int32_t one_ifelse;          // 1 = exactly one divergent if/else of the first form
  int32_t form_mask;           // bit f set = if-else form f+1 allowed
  int32_t p_select;            // percent chance that a 32-bit operation is a select (ternary); 0 = never
  int32_t p_sysval;            // percent chance that an integer leaf is a system value or a scalar
                               // bit field (s_load from the dispatch packet, s_lshr_b32, s_bfe_u32); 0 = never
  int32_t p_flat;              // percent chance that a buffer load or store is a FLAT instruction
                               // (flat_load_dword[x2] / flat_store_dword[x2]); 0 = never
  int32_t p_mulhi;             // percent chance that a 32-bit integer operation is a double-suffix
                               // high multiply (v_mul_hi_u32_u24 / v_mul_hi_i32_i24); 0 = never
  int32_t p_break;             // percent chance that a loop body has an early exit: a uniform
                               // test that jumps past the loop (break) or to its latch (continue)
  int32_t p_lds;               // percent chance that a top-level statement is an exchange through
                               // a __local buffer (ds_write_b32, s_barrier, ds_read_b32); 0 = never,
                               // and above 0 the kernel gets a __local argument and is 1-D
};
}

namespace {

struct Opd {
  enum K { VR, SR, IC, FI, LIT } k;
  int reg;
  uint32_t bits;
  std::string s() const {
    char b[32];
    switch (k) {
      case VR: snprintf(b, sizeof b, "v%d", reg); break;
      case SR: snprintf(b, sizeof b, "s%d", reg); break;
      case IC: snprintf(b, sizeof b, "%d", (int32_t)bits); break;
      case FI: {
        const char* t = "1.0";
        switch (bits) {
          case 0x3f000000u: t = "0.5"; break;
          case 0xbf000000u: t = "-0.5"; break;
          case 0x3f800000u: t = "1.0"; break;
          case 0xbf800000u: t = "-1.0"; break;
          case 0x40000000u: t = "2.0"; break;
          case 0xc0000000u: t = "-2.0"; break;
          case 0x40800000u: t = "4.0"; break;
          case 0xc0800000u: t = "-4.0"; break;
        }
        snprintf(b, sizeof b, "%s", t);
        break;
      }
      case LIT: snprintf(b, sizeof b, "0x%x", bits); break;
    }
    return b;
  }
};

Opd V(int r) { return Opd{Opd::VR, r, 0}; }
Opd S(int r) { return Opd{Opd::SR, r, 0}; }
Opd I(int32_t v) {
  if (v >= -16 && v <= 64) return Opd{Opd::IC, 0, (uint32_t)v};
  return Opd{Opd::LIT, 0, (uint32_t)v};
}

struct Local {
  int ty;
  int reg;    // home VGPR (pair base for 64-bit) or -1
  int slot;   // scratch byte offset when spilled, else -1
};

// log-uniform length table: 1024 points between 1 and 2^20 by repeated multiplication
struct LenTable {
  double r[1025];
  LenTable() {
    double f = 1.0, step = 1.0;
    // step = 2^(20/1024): computed by 10 square roots of 2^(20/1) via bisection-free
    // Newton iterations on IEEE arithmetic only.
    double x = 1.0 + 20.0 * 0.6931471805599453 / 1024.0;  // initial guess
    for (int it = 0; it < 60; ++it) {  // solve x^1024 = 2^20 by Newton on y = x^1024
      double y = x;
      for (int k = 0; k < 10; ++k) y = y * y;
      double dy = 1024.0 * y / x;
      x = x - (y - 1048576.0) / dy;
    }
    step = x;
    for (int i = 0; i <= 1024; ++i) { r[i] = f; f *= step; }
  }
};
const LenTable& lentab() { static LenTable t; return t; }

struct Gen {
  Rng rng;
  const gcngen_params& P;
  uint64_t kid;
  std::string body;
  uint32_t ninstr = 0, target = 0;
  int dims = 1, cws[3] = {64, 1, 1};
  int nbufs = 0;
  int buf_ty[8];
  bool buf_out[8];
  int s_buf[8];
  int s_n = 0;
  int s_lds = -1, lds_ty = TI;  // SGPR with the __local buffer's LDS address, its element type
  int vloc = 6, vtop = 6, vmax = 5, smax = 13;
  int label_ctr = 0, spill_next = 0;
  int ifelse_left = 0;
  std::vector<Local> locals;
  bool gid_ofs[2] = {true, true};
  uint32_t n_if = 0, n_else = 0, n_loop = 0;  // control statements emitted (ground truth)

  Gen(const gcngen_params& p, uint64_t seed, uint64_t k) : rng{mix(seed, k)}, P(p), kid(k) {}

  void ins(const std::string& s) {
    body += "        ";
    body += s;
    body += '\n';
    ++ninstr;
  }
  int label() { return label_ctr++; }
  void put_label(int l) {
    char b[32];
    snprintf(b, sizeof b, ".L%d:\n", l);
    body += b;
  }
  std::string lname(int l) {
    char b[32];
    snprintf(b, sizeof b, ".L%d", l);
    return b;
  }
  void touchv(int r, int n = 1) {
    if (r + n - 1 > vmax) vmax = r + n - 1;
  }
  void touchs(int r, int n = 1) {
    if (r + n - 1 > smax) smax = r + n - 1;
  }
  int tmp32() {
    int r = vtop++;
    touchv(r);
    return r;
  }
  int tmp64() {
    if (vtop & 1) ++vtop;
    int r = vtop;
    vtop += 2;
    touchv(r, 2);
    return r;
  }
  bool allowed(int t) const { return (P.type_mask >> t) & 1u; }
  int exec_pair(int depth) { return s_n + 2 + (s_n & 1) + 2 * depth; }  // even-aligned
  int loop_sreg(int depth) { return exec_pair(P.max_depth) + depth; }

  // ---- helpers ---------------------------------------------------------------
  std::string f(const char* fmt, ...) __attribute__((format(printf, 2, 3))) {
    char b[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    return b;
  }
  // make sure an operand sits in a VGPR
  Opd vgpr(Opd o) {
    if (o.k == Opd::VR) return o;
    int t = tmp32();
    ins(f("v_mov_b32 v%d, %s", t, o.s().c_str()));
    return V(t);
  }

  Opd const32(int t) {
    if (t == TF) {
      static const uint32_t inl[8] = {0x3f000000u, 0xbf000000u, 0x3f800000u, 0xbf800000u,
                                      0x40000000u, 0xc0000000u, 0x40800000u, 0xc0800000u};
      if (rng.chance(30)) return Opd{Opd::FI, 0, inl[rng.below(8)]};
      if (rng.chance(10)) {  // an arbitrary normal float
        uint32_t e = 120 + rng.below(16), m = rng.below(1u << 23);
        return Opd{Opd::LIT, 0, (rng.below(2) << 31) | (e << 23) | m};
      }
      int k = rng.range(-40, 40);  // k/4
      float v = (float)k * 0.25f;
      uint32_t b;
      memcpy(&b, &v, 4);
      if (b == 0x80000000u) b = 0;
      return Opd{Opd::LIT, 0, b};
    }
    if (rng.chance(70)) return I(rng.range(-16, 64));
    return Opd{Opd::LIT, 0, (uint32_t)rng.next()};
  }

  int const64(int t) {  // returns pair register
    int r = tmp64();
    uint64_t bits;
    if (t == TD) {
      if (rng.chance(85)) {
        double v = (double)rng.range(-64, 64) * 0.25;
        memcpy(&bits, &v, 8);
        if (bits == 0x8000000000000000ull) bits = 0;
      } else {
        bits = ((uint64_t)(1000 + rng.below(40)) << 52) | (rng.next() >> 12);
      }
    } else {
      int64_t v = rng.chance(80) ? (int64_t)rng.range(-100, 100) : (int64_t)rng.next();
      bits = (uint64_t)v;
    }
    ins(f("v_mov_b32 v%d, %s", r, I((int32_t)(uint32_t)bits).s().c_str()));
    ins(f("v_mov_b32 v%d, %s", r + 1, I((int32_t)(uint32_t)(bits >> 32)).s().c_str()));
    return r;
  }

  // address of buffer b at a 32-bit unsigned index held in `idx`; returns pair base
  int address(int b, Opd idx) {
    int ip = tmp64();
    if (idx.k == Opd::VR && idx.reg == ip) {
    } else {
      ins(f("v_mov_b32 v%d, %s", ip, idx.s().c_str()));
    }
    if (rng.chance(25))  // index is non-negative, so sign and zero extension agree
      ins(f("v_ashrrev_i32 v%d, 31, v%d", ip + 1, ip));
    else
      ins(f("v_mov_b32 v%d, 0", ip + 1));
    int a = tmp64();
    int sh = is64(buf_ty[b]) ? 3 : 2;
    ins(f("v_lshlrev_b64 v[%d:%d], %d, v[%d:%d]", a, a + 1, sh, ip, ip + 1));
    if (rng.chance(50)) {
      ins(f("v_add_co_u32 v%d, vcc, s%d, v%d", a, s_buf[b], a));
      ins(f("v_addc_co_u32 v%d, vcc, s%d, v%d, vcc", a + 1, s_buf[b] + 1, a + 1));
    } else {
      int t = tmp32();
      ins(f("v_mov_b32 v%d, s%d", t, s_buf[b] + 1));
      ins(f("v_add_co_u32 v%d, vcc, v%d, s%d", a, a, s_buf[b]));
      ins(f("v_addc_co_u32 v%d, vcc, v%d, v%d, vcc", a + 1, a + 1, t));
    }
    return a;
  }

  Opd lin() { return V(dims == 2 ? 5 : 3); }

  Opd index_for(int b, int d) {
    if (buf_out[b] || rng.chance(35)) return lin();
    Opd e = vgpr(gen32(TU, d < 2 ? d : 1));
    int t = tmp32();
    ins(f("v_and_b32 v%d, 0xff, %s", t, e.s().c_str()));
    return V(t);
  }

  // load element of buffer b (type known); returns VGPR (or pair base)
  int load(int b, int d) {
    int mark = vtop;
    Opd idx = index_for(b, d);
    int a = address(b, idx);
    int r;
    const bool flat = P.p_flat > 0 && rng.chance(P.p_flat);
    if (is64(buf_ty[b])) {
      r = mark + (mark & 1);
      if (flat) ins(f("flat_load_dwordx2 v[%d:%d], v[%d:%d]", r, r + 1, a, a + 1));
      else ins(f("global_load_dwordx2 v[%d:%d], v[%d:%d], off", r, r + 1, a, a + 1));
      vtop = r + 2;
    } else {
      r = mark;
      if (flat) ins(f("flat_load_dword v%d, v[%d:%d]", r, a, a + 1));
      else ins(f("global_load_dword v%d, v[%d:%d], off", r, a, a + 1));
      vtop = r + 1;
    }
    touchv(r, is64(buf_ty[b]) ? 2 : 1);
    ins("s_waitcnt vmcnt(0)");
    return r;
  }

  int pick_buf(int t) {
    int cand[8], n = 0;
    for (int b = 0; b < nbufs; ++b)
      if (buf_ty[b] == t || (t <= TU && buf_ty[b] <= TU)) cand[n++] = b;
    if (!n) return -1;
    return cand[rng.below(n)];
  }
  int pick_local(int t) {
    int cand[512], n = 0;
    for (int i = 0; i < (int)locals.size() && n < 512; ++i)
      if (locals[i].ty == t || (t <= TU && locals[i].ty <= TU)) cand[n++] = i;
    if (!n) return -1;
    return cand[rng.below(n)];
  }
  // read a local into an operand (unspills into a temp)
  Opd read_local(int li) {
    const Local& L = locals[li];
    if (L.slot < 0) return V(L.reg);
    if (is64(L.ty)) {
      int r = tmp64();
      ins(f("buffer_load_dword v%d, off, s[0:3], s9 offset:%d", r, L.slot));
      ins(f("buffer_load_dword v%d, off, s[0:3], s9 offset:%d", r + 1, L.slot + 4));
      ins("s_waitcnt vmcnt(0)");
      return V(r);
    }
    int r = tmp32();
    ins(f("buffer_load_dword v%d, off, s[0:3], s9 offset:%d", r, L.slot));
    ins("s_waitcnt vmcnt(0)");
    return V(r);
  }

  // ---- expressions -----------------------------------------------------------
  // a system value read through the dispatch packet pointer s[0:1] ("Search for memory
  // accesses": the global size at 0xc/0x10/0x14, the number of groups as global size /
  // work-group size, the dimension count as the field at bit 16, width 2, of the dword at
  // 0x0), or a bit field / logical shift of the scalar argument.  s15 is the scalar
  // temporary; the value moves to a VGPR at once, so s15 is free again for the next one.
  Opd sysval() {
    touchs(15);
    int d = (int)rng.below((uint32_t)dims);
    int k = (int)rng.below(5);
    int lg = 0;
    while ((1 << lg) < cws[d]) ++lg;
    if (k == 1 && (1 << lg) != cws[d]) k = 0;  // the shift form needs a power-of-two size
    switch (k) {
      case 0:  // get_global_size(d)
        ins(f("s_load_dword s15, s[0:1], 0x%x", 0xc + 4 * d));
        ins("s_waitcnt lgkmcnt(0)");
        break;
      case 1:  // get_num_groups(d)
        ins(f("s_load_dword s15, s[0:1], 0x%x", 0xc + 4 * d));
        ins("s_waitcnt lgkmcnt(0)");
        ins(f("s_lshr_b32 s15, s15, %d", lg));
        break;
      case 2:  // get_work_dim()
        ins("s_load_dword s15, s[0:1], 0x0");
        ins("s_waitcnt lgkmcnt(0)");
        ins("s_bfe_u32 s15, s15, 0x20010");
        break;
      case 3: {  // a bit field of the scalar argument
        int off = rng.range(0, 20), w = rng.range(1, 8);
        ins(f("s_bfe_u32 s15, s%d, 0x%x", s_n, (w << 16) | off));
        break;
      }
      default:  // a logical right shift of the scalar argument
        ins(f("s_lshr_b32 s15, s%d, %d", s_n, rng.range(1, 12)));
        break;
    }
    int r = tmp32();
    ins(f("v_mov_b32 v%d, s15", r));
    return V(r);
  }

  Opd leaf32(int t, int d) {
    if (t != TF && P.p_sysval > 0 && rng.chance(P.p_sysval)) return sysval();
    for (int attempt = 0; attempt < 6; ++attempt) {
      int c = rng.below(t == TF ? 6 : 7);
      if (t == TF) {
        switch (c) {
          case 0: { int li = pick_local(TF); if (li >= 0) return read_local(li); break; }
          case 1: { int b = pick_buf(TF); if (b >= 0) return V(load(b, d)); break; }
          case 2: return const32(TF);
          case 3: if (allowed(TI) || allowed(TU)) {
              int src = rng.below(2) ? TI : TU;
              Opd a = vgpr(gen32(src, d - 1));
              int r = tmp32();
              ins(f("v_cvt_f32_%s v%d, %s", src == TI ? "i32" : "u32", r, a.s().c_str()));
              return V(r);
            } break;
          case 4: if (allowed(TD) && d > 0) {
              int a = gen64(TD, d - 1);
              int r = tmp32();
              ins(f("v_cvt_f32_f64 v%d, v[%d:%d]", r, a, a + 1));
              return V(r);
            } break;
          default: { int li = pick_local(TF); if (li >= 0) return read_local(li); break; }
        }
      } else {
        switch (c) {
          case 0: return V(3);
          case 1: if (dims == 2) return V(4); return lin();
          case 2: { int li = pick_local(t); if (li >= 0) return read_local(li); break; }
          case 3: { int b = pick_buf(t); if (b >= 0) return V(load(b, d)); break; }
          case 4: return S(s_n);
          case 5: if (allowed(TL) && d > 0) {  // (int)long -> low dword
              int a = gen64(TL, d - 1);
              return V(a);
            } break;
          default: return const32(t);
        }
      }
    }
    return const32(t);
  }

  Opd gen32(int t, int d) {
    if (d <= 0 || rng.chance(30)) return leaf32(t, d);
    return gen32op(t, d);
  }

  // result register of an operation: the lowest temp of this subexpression
  int res32(int mark) {
    vtop = mark + 1;
    touchv(mark);
    return mark;
  }
  int res64(int mark) {
    int r = mark + (mark & 1);
    vtop = r + 2;
    touchv(r, 2);
    return r;
  }

  // ternary ("Search for control structures": one instruction, no template):
  //   v_cmp_<cc>_<ty> vcc, a, b;  v_cndmask_b32 vD, f, t, vcc   (vD = vcc ? t : f)
  // the values first: their code may itself write vcc
  Opd gen_select(int t, int d) {
    int mark = vtop;
    Opd fv = vgpr(gen32(t, d - 1));
    Opd tv = vgpr(gen32(t, d - 1));
    divergent_cond_depth(d - 1);
    int r = res32(mark);
    ins(f("v_cndmask_b32 v%d, %s, %s, vcc", r, fv.s().c_str(), tv.s().c_str()));
    return V(r);
  }

  Opd gen32op(int t, int d) {
    if (P.p_select > 0 && rng.chance(P.p_select)) return gen_select(t, d);
    int mark = vtop;
    int r;
    if (t == TF) {
      int op = rng.below(4);
      Opd a = gen32(TF, d - 1);
      Opd b = vgpr(gen32(TF, d - 1));
      if (op == 3) {
        Opd c = vgpr(gen32(TF, d - 1));
        r = res32(mark);
        ins(f("v_fma_f32 v%d, %s, %s, %s", r, a.s().c_str(), b.s().c_str(), c.s().c_str()));
        return V(r);
      }
      static const char* nm[3] = {"v_add_f32", "v_sub_f32", "v_mul_f32"};
      r = res32(mark);
      ins(f("%s v%d, %s, %s", nm[op], r, a.s().c_str(), b.s().c_str()));
      return V(r);
    }
    if (P.p_mulhi > 0 && rng.chance(P.p_mulhi)) {  // high half of a 24-bit multiply (double suffix)
      Opd a = gen32(t, d - 1);
      Opd b = vgpr(gen32(t, d - 1));
      r = res32(mark);
      ins(f("%s v%d, %s, %s", t == TI ? "v_mul_hi_i32_i24" : "v_mul_hi_u32_u24", r, a.s().c_str(), b.s().c_str()));
      return V(r);
    }
    int op = rng.below(t == TU ? 9 : 8);
    Opd a = gen32(t, d - 1);
    if (op == 6 || op == 7) {  // shifts by a constant
      Opd av = vgpr(a);
      r = res32(mark);
      int sh = rng.range(1, 12);
      const char* m = op == 6 ? "v_lshlrev_b32" : (t == TI ? "v_ashrrev_i32" : "v_lshrrev_b32");
      ins(f("%s v%d, %d, %s", m, r, sh, av.s().c_str()));
      return V(r);
    }
    if (op == 8) {  // 24-bit multiply-add (one literal at most: b and c in VGPRs)
      Opd b = vgpr(gen32(t, d - 1));
      Opd c = vgpr(gen32(t, d - 1));
      r = res32(mark);
      ins(f("v_mad_u32_u24 v%d, %s, %s, %s", r, a.s().c_str(), b.s().c_str(), c.s().c_str()));
      return V(r);
    }
    Opd b = vgpr(gen32(t, d - 1));
    static const char* nm[6] = {"v_add_u32", "v_sub_u32", "v_mul_lo_u32", "v_and_b32", "v_or_b32", "v_xor_b32"};
    r = res32(mark);
    ins(f("%s v%d, %s, %s", nm[op], r, a.s().c_str(), b.s().c_str()));
    return V(r);
  }

  int leaf64(int t, int d) {
    for (int attempt = 0; attempt < 6; ++attempt) {
      int c = rng.below(5);
      switch (c) {
        case 0: { int li = pick_local(t); if (li >= 0) return read_local(li).reg; break; }
        case 1: { int b = pick_buf(t); if (b >= 0) return load(b, d); break; }
        case 2: return const64(t);
        case 3:
          if (t == TD && allowed(TF)) {
            Opd a = vgpr(gen32(TF, d - 1));
            int r = tmp64();
            ins(f("v_cvt_f64_f32 v[%d:%d], %s", r, r + 1, a.s().c_str()));
            return r;
          }
          if (t == TL && (allowed(TI) || allowed(TU))) {  // (long)int: sign extension
            Opd a = gen32(TI, d - 1);
            int r = tmp64();
            ins(f("v_mov_b32 v%d, %s", r, a.s().c_str()));
            ins(f("v_ashrrev_i32 v%d, 31, v%d", r + 1, r));
            return r;
          }
          break;
        case 4:
          if (t == TD && (allowed(TI) || allowed(TU))) {
            Opd a = vgpr(gen32(TI, d - 1));
            int r = tmp64();
            ins(f("v_cvt_f64_i32 v[%d:%d], %s", r, r + 1, a.s().c_str()));
            return r;
          }
          if (t == TL) return const64(t);
          break;
      }
    }
    return const64(t);
  }

  int gen64(int t, int d) {
    if (d <= 0 || rng.chance(30)) return leaf64(t, d);
    int mark = vtop;
    int a = gen64(t, d - 1);
    int b = gen64(t, d - 1);
    int c = -1;
    if (t == TD && rng.below(3) == 2) c = gen64(t, d - 1);
    int r = res64(mark);
    if (t == TD) {
      int op = c >= 0 ? 2 : rng.below(2);
      if (op == 2) {
        ins(f("v_fma_f64 v[%d:%d], v[%d:%d], v[%d:%d], v[%d:%d]", r, r + 1, a, a + 1, b, b + 1, c, c + 1));
      } else {
        ins(f("%s v[%d:%d], v[%d:%d], v[%d:%d]", op ? "v_mul_f64" : "v_add_f64", r, r + 1, a, a + 1, b, b + 1));
      }
      return r;
    }
    if (rng.below(2)) {
      ins(f("v_add_co_u32 v%d, vcc, v%d, v%d", r, a, b));
      ins(f("v_addc_co_u32 v%d, vcc, v%d, v%d, vcc", r + 1, a + 1, b + 1));
    } else {
      ins(f("v_sub_co_u32 v%d, vcc, v%d, v%d", r, a, b));
      ins(f("v_subb_co_u32 v%d, vcc, v%d, v%d, vcc", r + 1, a + 1, b + 1));
    }
    return r;
  }

  int rand_type() {
    int c[5], n = 0;
    for (int t = 0; t < 5; ++t)
      if (allowed(t)) c[n++] = t;
    return c[rng.below(n)];
  }

  // ---- statements ------------------------------------------------------------
  void stmt_store() {
    int outs[8], n = 0;
    for (int b = 0; b < nbufs; ++b)
      if (buf_out[b]) outs[n++] = b;
    int b = outs[rng.below(n)];
    int t = buf_ty[b];
    int d = stmt_depth();
    if (is64(t)) {
      int v = gen64(t, d);
      int a = address(b, lin());
      if (P.p_flat > 0 && rng.chance(P.p_flat)) ins(f("flat_store_dwordx2 v[%d:%d], v[%d:%d]", a, a + 1, v, v + 1));
      else ins(f("global_store_dwordx2 v[%d:%d], v[%d:%d], off", a, a + 1, v, v + 1));
    } else {
      Opd v = vgpr(gen32(t, d));
      int a = address(b, lin());
      if (P.p_flat > 0 && rng.chance(P.p_flat)) ins(f("flat_store_dword v[%d:%d], %s", a, a + 1, v.s().c_str()));
      else ins(f("global_store_dword v[%d:%d], %s, off", a, a + 1, v.s().c_str()));
    }
  }

  // expression depth for the next statement: shallow near the end of the budget
  int stmt_depth() {
    int d = rng.range(1, P.expr_depth);
    uint32_t rem = target > ninstr ? target - ninstr : 0;
    if (rem < 40 && d > 2) d = 2;
    if (rem < 20) d = 1;
    return d;
  }

  void stmt_assign() {
    int li = -1;
    if (!locals.empty() && (rng.chance(45) || (int)locals.size() >= P.max_locals))
      li = (int)rng.below((uint32_t)locals.size());
    int t = li >= 0 ? locals[li].ty : rand_type();
    int d = stmt_depth();
    vtop = vloc + (vloc & 1) + 2;  // keep two registers free for a new home
    // the value first: a new local is not visible inside its own initialiser
    Opd v32{Opd::VR, 0, 0};
    int v64 = -1;
    if (is64(t)) v64 = gen64(t, d);
    else v32 = gen32(t, d);
    if (li < 0) {  // a new local: home register or scratch slot
      Local L{t, -1, -1};
      int need = is64(t) ? 2 : 1;
      int base = vloc + ((is64(t) && (vloc & 1)) ? 1 : 0);
      if (base + need + 24 <= P.vgpr_budget) {
        L.reg = base;
        vloc = base + need;
        touchv(L.reg, need);
      } else if (P.spills) {
        L.slot = spill_next;
        spill_next += 8;
      } else {
        return;  // no room: the value is computed and dropped
      }
      locals.push_back(L);
      li = (int)locals.size() - 1;
    }
    const Local L = locals[li];
    if (is64(t)) {
      if (L.slot >= 0) {
        ins(f("buffer_store_dword v%d, off, s[0:3], s9 offset:%d", v64, L.slot));
        ins(f("buffer_store_dword v%d, off, s[0:3], s9 offset:%d", v64 + 1, L.slot + 4));
      } else {
        ins(f("v_mov_b32 v%d, v%d", L.reg, v64));
        ins(f("v_mov_b32 v%d, v%d", L.reg + 1, v64 + 1));
      }
    } else {
      if (L.slot >= 0) {
        Opd vv = vgpr(v32);
        ins(f("buffer_store_dword %s, off, s[0:3], s9 offset:%d", vv.s().c_str(), L.slot));
      } else {
        ins(f("v_mov_b32 v%d, %s", L.reg, v32.s().c_str()));
      }
    }
  }

  // An exchange through the __local buffer (top level only: every work-item of the group reaches
  // both barriers): each work-item writes its element, and after the barrier reads a neighbour's,
  // which becomes a local.  The first barrier keeps this write from overtaking the reads of the
  // previous exchange.
  void stmt_lds() {
    int t = lds_ty;
    int d = stmt_depth();
    vtop = vloc + (vloc & 1) + 2;
    ins("s_barrier");
    Opd v = vgpr(gen32(t, d));
    int a = tmp32();
    ins(f("v_lshlrev_b32 v%d, 2, v0", a));
    ins(f("v_add_u32 v%d, s%d, v%d", a, s_lds, a));
    ins(f("ds_write_b32 v%d, %s", a, v.s().c_str()));
    ins("s_waitcnt lgkmcnt(0)");
    ins("s_barrier");
    int j = tmp32();
    const int c = cws[0];
    if ((c & (c - 1)) == 0) {
      ins(f("v_add_u32 v%d, %d, v0", j, rng.range(1, 7)));
      ins(f("v_and_b32 v%d, %s, v%d", j, I(c - 1).s().c_str(), j));
    } else {
      ins(f("v_xor_b32 v%d, 1, v0", j));
    }
    ins(f("v_lshlrev_b32 v%d, 2, v%d", j, j));
    ins(f("v_add_u32 v%d, s%d, v%d", j, s_lds, j));
    int r = tmp32();
    ins(f("ds_read_b32 v%d, v%d", r, j));
    ins("s_waitcnt lgkmcnt(0)");
    int base = vloc;
    if (base + 1 + 24 > P.vgpr_budget) return;  // no room for a new local: the value is dropped
    Local L{t, base, -1};
    vloc = base + 1;
    touchv(base);
    locals.push_back(L);
    ins(f("v_mov_b32 v%d, v%d", base, r));
  }

  void divergent_cond() { divergent_cond_depth(-1); }

  // a comparison into vcc (operand depth d, or a random shallow depth when d < 0)
  void divergent_cond_depth(int d) {
    int cands[3], n = 0;
    if (allowed(TI)) cands[n++] = TI;
    if (allowed(TU)) cands[n++] = TU;
    if (allowed(TF)) cands[n++] = TF;
    int t = n ? cands[rng.below(n)] : TU;
    if (d < 0) d = rng.range(0, P.expr_depth > 2 ? 2 : P.expr_depth);
    Opd a = gen32(t, d);
    Opd b = vgpr(gen32(t, d));
    static const char* cc[6] = {"lt", "gt", "le", "ge", "eq", "ne"};
    int k = rng.below(6);
    const char* c = (k == 5 && t == TF) ? "neq" : cc[k];
    ins(f("v_cmp_%s_%s vcc, %s, %s", c, t == TF ? "f32" : (t == TI ? "i32" : "u32"),
          a.s().c_str(), b.s().c_str()));
  }

  void block(int depth, uint32_t stop, int min_stmts) {
    size_t nloc = locals.size();
    int saved_vloc = vloc;
    int count = 0;
    while (count < min_stmts || ninstr < stop) {
      vtop = vloc + (vloc & 1);
      ++count;
      bool ctrl = depth < P.max_depth && stop > ninstr + 24 && rng.chance(P.p_ctrl);
      if (P.one_ifelse && ifelse_left && depth == 0 && ninstr * 5 >= target * 2) {
        ifelse_left = 0;
        stmt_ifelse(depth, stop, 1);
        continue;
      }
      if (s_lds >= 0 && depth == 0 && P.p_lds > 0 && rng.chance(P.p_lds)) {
        stmt_lds();
        continue;
      }
      if (ctrl && !P.one_ifelse) {
        int tot = P.w_if + P.w_ifelse + P.w_loop + P.w_uif;
        int c = (int)rng.below((uint32_t)tot);
        if ((c -= P.w_if) < 0) stmt_if(depth, stop);
        else if ((c -= P.w_ifelse) < 0) {
          int forms[3], nf = 0;
          for (int q = 0; q < 3; ++q)
            if ((P.form_mask >> q) & 1) forms[nf++] = q + 1;
          stmt_ifelse(depth, stop, nf ? forms[rng.below(nf)] : 1);
        } else if ((c -= P.w_loop) < 0) stmt_loop(depth, stop);
        else stmt_uif(depth, stop);
        continue;
      }
      if (rng.chance(50)) stmt_assign();
      else stmt_store();
    }
    locals.resize(nloc);
    vloc = saved_vloc;
  }

  uint32_t share(uint32_t stop, int pct) {
    uint32_t rem = stop > ninstr ? stop - ninstr : 0;
    return ninstr + rem * (uint32_t)pct / 100;
  }

  void stmt_if(int depth, uint32_t stop) {
    ++n_if;
    divergent_cond();
    int e = exec_pair(depth);
    touchs(e, 2);
    int l = label();
    ins(f("s_and_saveexec_b64 s[%d:%d], vcc", e, e + 1));
    ins(f("s_cbranch_execz %s", lname(l).c_str()));
    block(depth + 1, share(stop, rng.range(15, 45)), 1);
    put_label(l);
    ins(f("s_or_b64 exec, exec, s[%d:%d]", e, e + 1));
  }

  void stmt_ifelse(int depth, uint32_t stop, int form) {
    ++n_if;
    ++n_else;
    divergent_cond();
    int e = exec_pair(depth);
    touchs(e, 2);
    ins(f("s_and_saveexec_b64 s[%d:%d], vcc", e, e + 1));
    ins(f("s_xor_b64 s[%d:%d], exec, s[%d:%d]", e, e + 1, e, e + 1));
    int la = -1, lb = -1;
    if (form == 1 || form == 2) {
      la = label();
      ins(f("s_cbranch_execz %s", lname(la).c_str()));
    }
    block(depth + 1, share(stop, rng.range(10, 30)), 1);
    if (la >= 0) put_label(la);
    ins(f("s_or_saveexec_b64 s[%d:%d], s[%d:%d]", e, e + 1, e, e + 1));
    ins(f("s_xor_b64 exec, exec, s[%d:%d]", e, e + 1));
    if (form == 1 || form == 3) {
      lb = label();
      ins(f("s_cbranch_execz %s", lname(lb).c_str()));
    }
    block(depth + 1, share(stop, rng.range(10, 30)), 1);
    if (lb >= 0) put_label(lb);
    ins(f("s_or_b64 exec, exec, s[%d:%d]", e, e + 1));
  }

  void stmt_uif(int depth, uint32_t stop) {  // uniform if / if-else on the scalar argument
    ++n_if;
    static const char* cc[4] = {"gt", "lt", "eq", "lg"};
    ins(f("s_cmp_%s_u32 s%d, %s", cc[rng.below(4)], s_n, I(rng.range(0, 40)).s().c_str()));
    int l = label();
    ins(f("s_cbranch_scc0 %s", lname(l).c_str()));
    block(depth + 1, share(stop, rng.range(10, 35)), 1);
    if (rng.chance(40)) {
      ++n_else;
      int le = label();
      ins(f("s_branch %s", lname(le).c_str()));
      put_label(l);
      block(depth + 1, share(stop, rng.range(10, 30)), 1);
      put_label(le);
      // a join needs an instruction to start the next block: keep the stream going
    } else {
      put_label(l);
    }
  }

  void stmt_loop(int depth, uint32_t stop) {
    ++n_loop;
    int c = loop_sreg(depth);
    touchs(c);
    int trip = rng.range(1, P.trip_max);
    ins(f("s_mov_b32 s%d, 0", c));
    int l = label();
    put_label(l);
    // an early exit sits at the top level of the body, outside any divergent region, so that a
    // scalar branch leaves the loop (or skips to its latch) without touching the exec mask
    const bool early = P.p_break > 0 && rng.chance(P.p_break);
    if (early) {
      ++n_if;  // the exit's test
      block(depth + 1, share(stop, rng.range(8, 25)), 1);
      const bool brk = rng.chance(50);
      if (rng.chance(50)) ins(f("s_cmp_eq_u32 s%d, %s", c, I(rng.range(0, trip)).s().c_str()));
      else ins(f("s_cmp_gt_u32 s%d, %s", s_n, I(rng.range(0, 40)).s().c_str()));
      const int lx = label();
      ins(f("s_cbranch_scc1 %s", lname(lx).c_str()));
      block(depth + 1, share(stop, rng.range(8, 25)), 1);
      if (!brk) put_label(lx);  // continue: to the latch
      ins(f("s_add_u32 s%d, s%d, 1", c, c));
      ins(f("s_cmp_lt_u32 s%d, %s", c, I(trip).s().c_str()));
      ins(f("s_cbranch_scc1 %s", lname(l).c_str()));
      if (brk) put_label(lx);  // break: past the loop
      return;
    }
    block(depth + 1, share(stop, rng.range(15, 45)), 1);
    ins(f("s_add_u32 s%d, s%d, 1", c, c));
    ins(f("s_cmp_lt_u32 s%d, %s", c, I(trip).s().c_str()));
    ins(f("s_cbranch_scc1 %s", lname(l).c_str()));
  }

  // ---- whole kernel ----------------------------------------------------------
  std::string run() {
    const LenTable& LT = lentab();
    // log-uniform target length in [min_len, max_len]
    {
      double lo = P.min_len, hi = P.max_len;
      // find k range where lo * r[k] <= hi
      int kmax = 0;
      while (kmax < 1024 && lo * LT.r[kmax + 1] <= hi) ++kmax;
      int k = kmax > 0 ? (int)rng.below((uint32_t)kmax + 1) : 0;
      target = (uint32_t)(lo * LT.r[k] + 0.5);
      if (target < P.min_len) target = P.min_len;
      if (target > P.max_len) target = P.max_len;
    }
    dims = P.dims ? P.dims : (rng.chance(50) ? 1 : 2);
    if (P.p_lds > 0) dims = 1;  // the exchange indexes the buffer by get_local_id(0)
    if (P.cws0) {
      cws[0] = P.cws0;
      cws[1] = dims == 2 ? P.cws1 : 1;
    } else if (dims == 1) {
      static const int c1[4] = {64, 128, 256, 96};
      cws[0] = c1[rng.below(4)];
      cws[1] = 1;
    } else {
      static const int c2[4][2] = {{16, 16}, {8, 8}, {32, 4}, {16, 12}};
      int q = rng.below(4);
      cws[0] = c2[q][0];
      cws[1] = c2[q][1];
    }
    cws[2] = 1;
    if (P.fixed_args) {
      nbufs = 2;
      buf_ty[0] = TI;
      buf_ty[1] = TF;
      buf_out[0] = false;
      buf_out[1] = true;
    } else {
      nbufs = rng.range(P.min_bufs, P.max_bufs);
      bool any_out = false;
      for (int b = 0; b < nbufs; ++b) {
        buf_ty[b] = rand_type();
        buf_out[b] = rng.chance(50);
        any_out |= buf_out[b];
      }
      if (!any_out) buf_out[nbufs - 1] = true;
    }
    ifelse_left = P.one_ifelse;
    for (int b = 0; b < nbufs; ++b) s_buf[b] = 16 + 2 * b;
    s_n = 16 + 2 * nbufs;
    touchs(s_n);
    // prologue: hidden global offsets, argument pointers, scalar argument
    ins("s_load_dwordx2 s[10:11], s[4:5], 0x0");
    if (dims == 2) ins("s_load_dwordx2 s[12:13], s[4:5], 0x8");
    for (int b = 0; b < nbufs; b += 2) {
      if (b + 1 < nbufs && rng.chance(75))
        ins(f("s_load_dwordx4 s[%d:%d], s[4:5], 0x%x", s_buf[b], s_buf[b] + 3, 0x30 + 8 * b));
      else {
        ins(f("s_load_dwordx2 s[%d:%d], s[4:5], 0x%x", s_buf[b], s_buf[b] + 1, 0x30 + 8 * b));
        if (b + 1 < nbufs)
          ins(f("s_load_dwordx2 s[%d:%d], s[4:5], 0x%x", s_buf[b + 1], s_buf[b + 1] + 1, 0x30 + 8 * (b + 1)));
      }
    }
    ins(f("s_load_dword s%d, s[4:5], 0x%x", s_n, 0x30 + 8 * nbufs));
    if (P.p_lds > 0) {  // the __local buffer's LDS address: the low dword of the slot after n
      s_lds = s_n + 1;
      touchs(s_lds);
      int tys[3], nt = 0;
      for (int q = TI; q <= TF; ++q)
        if (allowed(q)) tys[nt++] = q;
      lds_ty = nt ? tys[rng.below(nt)] : TI;
      ins(f("s_load_dword s%d, s[4:5], 0x%x", s_lds, 0x30 + 8 * (nbufs + 1)));
    }
    ins("s_waitcnt lgkmcnt(0)");
    for (int d = 0; d < dims; ++d) {
      int g = 6 + d, l = d, dst = 3 + d, o = 10 + 2 * d, c = cws[d];
      gid_ofs[d] = !rng.chance(20);
      int var = rng.below(3);
      bool pow2 = (c & (c - 1)) == 0;
      if (var == 1 && !pow2) var = 0;
      if (var == 0) {
        ins(f("s_mul_i32 s14, s%d, %s", g, I(c).s().c_str()));
        ins(f("v_add_u32 v%d, s14, v%d", dst, l));
      } else if (var == 1) {
        int lg = 0;
        while ((1 << lg) < c) ++lg;
        ins(f("s_lshl_b32 s14, s%d, %d", g, lg));
        ins(f("v_add_u32 v%d, s14, v%d", dst, l));
      } else {
        ins(f("v_mov_b32 v%d, s%d", dst, g));
        ins(f("v_mad_u32_u24 v%d, v%d, %s, v%d", dst, dst, I(c).s().c_str(), l));
      }
      if (gid_ofs[d]) ins(f("v_add_u32 v%d, s%d, v%d", dst, o, dst));
    }
    if (dims == 2) {
      ins("v_lshlrev_b32 v5, 6, v4");
      ins("v_add_u32 v5, v3, v5");
    }
    touchv(5);
    vloc = 6;
    block(0, target > 12 ? target - 3 : 1, 1);
    if (P.one_ifelse && ifelse_left) {
      ifelse_left = 0;
      stmt_ifelse(0, ninstr + 40, 1);
    }
    // make sure at least one store exists
    vtop = vloc + (vloc & 1);
    stmt_store();
    ins("s_endpgm");

    // header
    std::string h;
    char b[256];
    snprintf(b, sizeof b, ".kernel k%llu\n", (unsigned long long)kid);
    h += b;
    h += "    .config\n";
    h += dims == 2 ? "        .dims xy\n" : "        .dims x\n";
    snprintf(b, sizeof b, "        .cws %d, %d, %d\n", cws[0], cws[1], cws[2]);
    h += b;
    int sg = smax + 1, vg = vmax + 1;
    snprintf(b, sizeof b, "        .sgprsnum %d\n        .vgprsnum %d\n", sg, vg);
    h += b;
    h += "        .floatmode 0xc0\n        .dx10clamp\n        .ieeemode\n        .useargs\n        .priority 0\n";
    h += "        .arg _.global_offset_0, \"size_t\", long\n";
    h += "        .arg _.global_offset_1, \"size_t\", long\n";
    h += "        .arg _.global_offset_2, \"size_t\", long\n";
    h += "        .arg _.printf_buffer, \"size_t\", void*, global, , rdonly\n";
    h += "        .arg _.vqueue_pointer, \"size_t\", long\n";
    h += "        .arg _.aqlwrap_pointer, \"size_t\", long\n";
    static const char* nm = "abcdefgh";
    for (int q = 0; q < nbufs; ++q) {
      snprintf(b, sizeof b, "        .arg %c, \"%s*\", %s*, global,%s\n", nm[q], kTyName[buf_ty[q]],
               kTyName[buf_ty[q]], buf_out[q] ? "" : " const");
      h += b;
    }
    h += "        .arg n, \"uint\", uint\n";
    if (s_lds >= 0) {
      snprintf(b, sizeof b, "        .arg tmp, \"%s*\", %s*, local,\n", kTyName[lds_ty], kTyName[lds_ty]);
      h += b;
    }
    h += "    .text\n";
    return h + body;
  }
};

gcngen_params preset(int cfg) {
  gcngen_params p;
  memset(&p, 0, sizeof p);
  p.type_mask = 0x1f;
  p.w_if = 50;
  p.w_ifelse = 30;
  p.w_loop = 20;
  p.w_uif = 0;
  p.p_ctrl = 12;
  p.max_depth = 3;
  p.min_bufs = 1;
  p.max_bufs = 8;
  p.vgpr_budget = 96;
  p.sgpr_budget = 64;
  p.max_locals = 12;
  p.expr_depth = 3;
  p.trip_max = 4;
  p.form_mask = 7;
  switch (cfg) {
    case 0:  // one kernel, ~200 instrs, (int *a, float *b, uint n), 2D (16,16,1), one if/else
      p.min_len = p.max_len = 200;
      p.type_mask = (1 << TI) | (1 << TU) | (1 << TF);
      p.fixed_args = 1;
      p.one_ifelse = 1;
      p.max_depth = 1;
      p.dims = 2;
      p.cws0 = 16;
      p.cws1 = 16;
      p.vgpr_budget = 64;
      p.sgpr_budget = 32;
      p.max_locals = 6;
      p.expr_depth = 4;
      p.form_mask = 1;
      break;
    case 1:
    case 2:  // 50..2000 instrs, all five value types, 50/30/20 if/if-else/loop, nesting <= 3
      p.min_len = 50;
      p.max_len = 2000;
      break;
    case 3:  // large CFGs: 200k instrs, int32/int64, nesting 6, spills
      p.min_len = p.max_len = 200000;
      p.type_mask = (1 << TI) | (1 << TU) | (1 << TL);
      p.max_depth = 6;
      p.p_ctrl = 28;
      p.vgpr_budget = 256;
      p.sgpr_budget = 104;
      p.spills = 1;
      p.max_locals = 300;
      p.expr_depth = 2;
      break;
    case 5:  // the batch mix with selects (v_cndmask_b32) in 15% of 32-bit operations
      p.min_len = 50;
      p.max_len = 2000;
      p.p_select = 15;
      break;
    case 4:  // serving requests: 100..50000 instrs, config-1 mix
      p.min_len = 100;
      p.max_len = 50000;
      break;
    case 6:  // the batch mix with system values and scalar bit fields in 10% of integer leaves
      p.min_len = 50;
      p.max_len = 2000;
      p.p_sysval = 10;
      break;
    case 7:  // the batch mix with FLAT loads/stores (30%) and double-suffix high multiplies (10%)
      p.min_len = 50;
      p.max_len = 2000;
      p.p_flat = 30;
      p.p_mulhi = 10;
      break;
    case 9:  // the batch mix (1-D) with exchanges through a __local buffer in 15% of top-level statements
      p.min_len = 50;
      p.max_len = 2000;
      p.p_lds = 15;
      break;
    case 8:  // mixed uniform and divergent nesting: divergent if / if-else (forms 1-3), uniform
             // if / if-else and loops interleaved, nesting <= 4; a third of the loops exit early
             // (break or continue)
      p.p_break = 35;
      p.min_len = 50;
      p.max_len = 2000;
      p.w_if = 30;
      p.w_ifelse = 30;
      p.w_loop = 15;
      p.w_uif = 25;
      p.max_depth = 4;
      p.p_ctrl = 18;
      break;
  }
  return p;
}

struct Result {
  std::string text;
  std::vector<uint64_t> off;
  std::vector<uint64_t> ninstr;
  std::vector<uint32_t> truth;  // per kernel 4 words: dims | gid_ofs[0] << 2 | gid_ofs[1] << 3, ifs, elses, loops
};

}  // namespace

extern "C" {

// Default knobs of workload `cfg` (0..9).  Returns 0, or -1 for an unknown index.
int gcngen_preset(int cfg, gcngen_params* out) {
  if (cfg < 0 || cfg > 9 || !out) return -1;
  *out = preset(cfg);
  return 0;
}

// Generate kernels [first, first+n) of the stream (params, seed) with `threads`
// host threads.  The kernels are concatenated; offsets[i] is where kernel i starts.
// Returns an opaque result (free with gcngen_free) or NULL.
void* gcngen_generate(const gcngen_params* p, uint64_t seed, uint64_t first, uint64_t n, int threads) {
  if (!p || n == 0) return nullptr;
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n) threads = (int)n;
  Result* R = new Result;
  std::vector<std::string> part(threads);
  std::vector<std::vector<uint64_t>> lens(threads), ni(threads);
  std::vector<std::vector<uint32_t>> tr(threads);
  auto work = [&](int t) {
    uint64_t a = n * t / threads, b = n * (t + 1) / threads;
    for (uint64_t k = a; k < b; ++k) {
      Gen g(*p, seed, first + k);
      std::string s = g.run();
      lens[t].push_back(s.size());
      ni[t].push_back(g.ninstr);
      tr[t].push_back((uint32_t)g.dims | ((uint32_t)g.gid_ofs[0] << 2) | ((uint32_t)g.gid_ofs[1] << 3));
      tr[t].push_back(g.n_if);
      tr[t].push_back(g.n_else);
      tr[t].push_back(g.n_loop);
      part[t] += s;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < threads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  size_t tot = 0;
  for (auto& s : part) tot += s.size();
  R->text.reserve(tot);
  R->off.push_back(0);
  for (int t = 0; t < threads; ++t) {
    R->text += part[t];
    std::string().swap(part[t]);
    for (size_t i = 0; i < lens[t].size(); ++i) {
      R->off.push_back(R->off.back() + lens[t][i]);
      R->ninstr.push_back(ni[t][i]);
      for (int q = 0; q < 4; ++q) R->truth.push_back(tr[t][4 * i + q]);
    }
  }
  return R;
}

uint64_t gcngen_size(void* r) { return r ? ((Result*)r)->text.size() : 0; }
// copy text into buf (cap bytes), offsets (n+1 entries) and per-kernel instruction counts (n)
int gcngen_copy(void* r, char* buf, uint64_t cap, uint64_t* offsets, uint64_t* ninstr) {
  Result* R = (Result*)r;
  if (!R) return -1;
  if (buf) {
    if (cap < R->text.size()) return -2;
    memcpy(buf, R->text.data(), R->text.size());
  }
  if (offsets) memcpy(offsets, R->off.data(), R->off.size() * 8);
  if (ninstr) memcpy(ninstr, R->ninstr.data(), R->ninstr.size() * 8);
  return 0;
}
// what the generator decided for each kernel, for ground-truth checks of the decompiled text, four
// words per kernel: bits 0-1 the number of NDRange dimensions and bit 2 + d set when the
// get_global_id(d) chain adds the global offset (clear: the offset-free idiom); then the numbers of
// ifs (divergent, uniform, and the tests of early exits), of else parts, and of counted loops
int gcngen_truth(void* r, uint32_t* out) {
  Result* R = (Result*)r;
  if (!R || !out) return -1;
  memcpy(out, R->truth.data(), R->truth.size() * 4);
  return 0;
}
void gcngen_free(void* r) { delete (Result*)r; }

}  // extern "C"
