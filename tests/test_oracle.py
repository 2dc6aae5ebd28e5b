"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: fixtures come from the paper's
worked examples (tests/golden, each cited), the structural-analysis trace of
Fig. 3, lattice laws, invariants of the dataflow, and brute force (a GCN
interpreter running the assembly against an evaluator running the decompiled
OpenCL on random buffers)."""
import os
import re
import struct

import numpy as np
import pytest

import brute
import gcngen
import ocl_eval
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return f.read()


# ---- "The body extraction", Listing 1 -------------------------------------
def test_listing1_dims_and_workgroup():
    r = oracle.decompile(gold("listing1_body.s"), with_ir=True)
    h = np.frombuffer(r.ir[0][oracle.IR_HEADER], np.uint32)
    dims, c0, c1, c2 = (int(x) for x in h[:4])
    assert dims == 3 and (c0, c1, c2) == (8, 8, 2) and c0 * c1 * c2 == 128


# ---- "Data type recovery", Listing 3 and its signature ---------------------
def test_listing3_signature():
    r = oracle.decompile(gold("listing3_copy.s"))
    assert r.status == [0]
    assert r.text.split("\n")[0] == "__kernel void copy(__global int *data, int x)"


# ---- "Search for memory accesses": system values ---------------------------
@pytest.mark.parametrize("name", ["p194_global_offset", "idiom_noofs", "gid_offset"])
def test_system_values(name):
    r = oracle.decompile(gold(name + ".s"))
    assert r.status == [0]
    assert r.text == gold(name + ".cl")


# ---- "Search for control structures": the ternary operator is one instruction ------
def test_ternary_is_one_instruction():
    """v_cndmask_b32 (vcc ? src1 : src0) becomes the conditional operator in place, with no
    control-flow template: ReLU written by hand, its expected text derived by hand."""
    r = oracle.decompile(gold("ternary_relu.s"))
    assert r.status == [0]
    assert r.text == gold("ternary_relu.cl")


# ---- "Search for memory accesses": global size, number of groups, dimension count ------
def test_dispatch_packet_system_values():
    """s_load_dword from the dispatch packet pointer s[0:1] at 0xc/0x10 is get_global_size(0/1),
    that shifted right by log2 of the work-group size of its dimension is get_num_groups (global
    size / work-group size), s_bfe_u32 with field 0x20010 of the dword at 0x0 is get_work_dim();
    other shifts and fields stay operators.  Written by hand, expected text derived by hand, and
    run: the interpreter reads a real packet for a 3x2-group range of 16x8 work-groups."""
    src = gold("sysvals_dispatch.s")
    r = oracle.decompile(src)
    assert r.status == [0]
    assert r.text == gold("sysvals_dispatch.cl")
    assert brute.check(src, r.text, groups=(3, 2)) is None
    # each value is told apart by the run: the other dimension's count, a constant 1
    # for the dimension count, the work-group size for the number of groups
    for a, b in (("get_num_groups(1)", "get_num_groups(0)"), ("get_work_dim()", "1u"),
                 ("get_global_size(0)", "get_global_size(1)")):
        assert brute.check(src, r.text.replace(a, b, 1), groups=(3, 2)) is not None, (a, b)


def test_brute_force_system_values():
    """The mix of workload 1 with system values read through the dispatch packet and scalar
    bit fields / shifts in 10% of integer leaves, on a 3x2-group range."""
    b = _batch(6, 30, cws0=8, cws1=4, max_len=400)
    seen = set()
    for i in range(len(b)):
        txt = b.kernel(i).decode()
        r = oracle.decompile(txt)
        assert r.status == [0]
        seen |= {f for f in ("get_global_size(", "get_num_groups(", "get_work_dim()") if f in r.text}
        seen |= {k for k, pat in (("field", r"s_bfe_u32 s15, s(?!15,)\d+,"), ("shift", r"s_lshr_b32 s15, s(?!15,)\d+,"))
                 if re.search(pat, txt)}
        assert brute.check(txt, r.text, seed=i, groups=(3, 2)) is None, f"kernel {i}"
    assert len(seen) == 5, seen


# ---- "Data type recovery": suffix typing -----------------------------------
def test_suffix_u32_is_unsigned_addition():
    r = oracle.decompile(gold("suffix_uint_add.s"))
    assert r.text == gold("suffix_uint_add.cl")


_SUFFIX_HEAD = """.kernel t
    .config
        .dims x
        .cws 64, 1, 1
        .sgprsnum 16
        .vgprsnum 12
        .useargs
        .arg _.global_offset_0, "size_t", long
        .arg _.global_offset_1, "size_t", long
        .arg _.global_offset_2, "size_t", long
        .arg _.printf_buffer, "size_t", void*, global, , rdonly
        .arg _.vqueue_pointer, "size_t", long
        .arg _.aqlwrap_pointer, "size_t", long
        .arg x, "int", int
        .arg y, "int", int
        .arg data, "int*", int*, global,
    .text
        s_load_dword s0, s[4:5], 0x30
        s_load_dword s1, s[4:5], 0x38
        s_load_dwordx2 s[8:9], s[4:5], 0x40
        s_waitcnt lgkmcnt(0)
        v_mov_b32 v2, v0
        v_mov_b32 v3, 0
        v_lshlrev_b64 v[4:5], 2, v[2:3]
        v_add_co_u32 v4, vcc, s8, v4
        v_addc_co_u32 v5, vcc, s9, v5, vcc
        v_mov_b32 v7, s0
        v_mov_b32 v8, s1
"""


def _suffix_kernel(op):
    # the result of `op` (in v6) is stored twice, so it becomes the kernel's one variable
    return (_SUFFIX_HEAD + "        " + op + "\n        global_store_dword v[4:5], v6, off\n"
            "        global_store_dword v[4:5], v6, off\n        s_endpgm\n")


@pytest.mark.parametrize("op,want", [
    ("v_add_f32 v6, v7, v8", "float"), ("v_sub_f32 v6, v7, v8", "float"), ("v_mul_f32 v6, v7, v8", "float"),
    ("v_fma_f32 v6, v7, v8, v7", "float"), ("v_cvt_f32_i32 v6, v7", "float"), ("v_cvt_f32_u32 v6, v7", "float"),
    ("v_add_u32 v6, v7, v8", "uint"), ("v_sub_u32 v6, v7, v8", "uint"), ("v_mul_lo_u32 v6, v7, v8", "uint"),
    ("v_mad_u32_u24 v6, v7, v8, v7", "uint"), ("v_mul_u32_u24 v6, v7, v8", "uint"),
    ("v_mul_hi_u32_u24 v6, v7, v8", "uint"), ("v_ashrrev_i32 v6, v7, v8", "int"),
    ("v_mul_hi_i32_i24 v6, v7, v8", "int"),
    ("s_mul_i32 s2, s0, s1\n        v_mov_b32 v6, s2", "int"),
    ("s_add_u32 s2, s0, s1\n        v_mov_b32 v6, s2", "uint"),
])
def test_result_type_follows_the_suffix(op, want):
    """"Data type recovery": an instruction's suffix (the first one for a conversion or a
    double-suffix operation) gives its result's type: f32 float, u32 uint, i32 int.  The result
    here is used twice, so it is declared once, with that type."""
    r = oracle.decompile(_suffix_kernel(op))
    assert r.worst == 0
    assert re.findall(r"^    (\w+) (var\d+);", r.text, re.M) == [(want, "var0")]


@pytest.mark.parametrize("op,stmt", [
    # an unsigned operation reads the inline constant -1 as 2^32 - 1
    ("v_add_u32 v6, -1, v8", "var0 = (4294967295u + (uint)y);"),
    ("v_add_u32 v6, 0xffffffff, v8", "var0 = (4294967295u + (uint)y);"),
    # a signed one keeps it signed
    ("s_mul_i32 s2, s0, -5\n        v_mov_b32 v6, s2", "var0 = (x * -5);"),
    ("s_mul_i32 s2, s0, 0x7fffffff\n        v_mov_b32 v6, s2", "var0 = (x * 2147483647);"),
    # a 32-bit shift uses the low five bits of its amount (33 & 31 = 1)
    ("v_lshlrev_b32 v6, 33, v8", "var0 = (y << 1);"),
    ("v_ashrrev_i32 v6, 3, v8", "var0 = (y >> 3);"),
    # an inline float constant in an integer operation is its bit pattern (1.0f = 0x3f800000)
    ("v_add_u32 v6, 1.0, v8", "var0 = (1065353216u + (uint)y);"),
])
def test_integer_literals(op, stmt):
    """Output format of integer literals (decimal, `u` for unsigned), with the values the GCN
    operation gives its constant operand."""
    r = oracle.decompile(_suffix_kernel(op))
    assert r.worst == 0
    assert "    " + stmt + "\n" in r.text


@pytest.mark.parametrize("op", [
    "v_add_f32 v6, v7, v8", "v_fma_f32 v6, v7, v8, v7", "v_cvt_f32_i32 v6, v7", "v_cvt_f32_u32 v6, v7",
    "v_sub_u32 v6, v7, v8", "v_mul_lo_u32 v6, v7, v8", "v_mad_u32_u24 v6, v7, v8, v7", "v_mul_hi_u32_u24 v6, v7, v8",
    "v_mul_hi_i32_i24 v6, v7, v8", "v_ashrrev_i32 v6, v7, v8", "v_lshrrev_b32 v6, v7, v8",
    "s_mul_i32 s2, s0, s1\n        v_mov_b32 v6, s2", "v_lshlrev_b32 v6, 33, v8", "v_add_u32 v6, 1.0, v8",
    "v_add_u32 v6, -1, v8", "v_add_f32 v6, 0x3dcccccd, v8", "v_add_f32 v9, v7, v8\n        v_and_b32 v6, v9, v7",
])
def test_brute_force_pin_kernels(op):
    """The hand-made kernels of the typing and literal pins compute, as decompiled, the same bits as
    their assembly (three seeded runs of the interpreter against the evaluator)."""
    src = _suffix_kernel(op)
    r = oracle.decompile(src)
    for seed in range(3):
        assert brute.check(src, r.text, seed=seed) is None


_SIG = "__kernel void t(int x, int y, __global int *data)\n{\n"


@pytest.mark.parametrize("body,want", [
    # used once: printed in place
    ("        v_add_u32 v6, v7, v8\n        global_store_dword v[4:5], v6, off\n",
     "    data[get_local_id(0)] = (int)((uint)x + (uint)y);\n"),
    # used twice: a variable
    ("        v_add_u32 v6, v7, v8\n        global_store_dword v[4:5], v6, off\n"
     "        global_store_dword v[4:5], v6, off\n",
     "    uint var0;\n    var0 = ((uint)x + (uint)y);\n    data[get_local_id(0)] = (int)var0;\n"
     "    data[get_local_id(0)] = (int)var0;\n"),
    # a global load: a variable at its program point, even when used once
    ("        global_load_dword v6, v[4:5], off\n        s_waitcnt vmcnt(0)\n        v_add_u32 v9, v6, v7\n"
     "        global_store_dword v[4:5], v9, off\n",
     "    int var0;\n    var0 = data[get_local_id(0)];\n    data[get_local_id(0)] = (int)((uint)var0 + (uint)x);\n"),
    # used in another block (the then-part of a uniform if): a variable
    ("        v_add_u32 v6, v7, v8\n        s_cmp_eq_u32 s0, 0\n        s_cbranch_scc1 .L1\n"
     "        global_store_dword v[4:5], v6, off\n.L1:\n",
     "    uint var0;\n    var0 = ((uint)x + (uint)y);\n    if (!((uint)x == 0u)) {\n"
     "        data[get_local_id(0)] = (int)var0;\n    }\n"),
])
def test_variables_by_the_materialisation_rule(body, want):
    """Variables are introduced only when needed: a value becomes a variable when it is a global
    load, is used twice or more, or is used in another block; otherwise it prints in place."""
    r = oracle.decompile(_SUFFIX_HEAD + body + "        s_endpgm\n")
    assert r.worst == 0
    assert r.text == _SIG + want + "}\n"


def _f32_bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


@pytest.mark.parametrize("lit,text", [
    (f"{_f32_bits(0.25):#x}", "0.25f"),       # two fraction bits: the exact decimal
    (f"{_f32_bits(1000.0):#x}", "1000.0f"),   # an integer value
    ("-4.0", "-4.0f"),                        # an inline float constant
    (f"{_f32_bits(0.1):#x}", f"as_float({_f32_bits(0.1)}u)"),              # 0.1 has no finite binary form
    (f"{_f32_bits(1.0) + 1:#x}", f"as_float({_f32_bits(1.0) + 1}u)"),      # 23 fraction bits
    ("0x7f800000", "as_float(2139095040u)"),  # infinity
    ("0x80000000", "as_float(2147483648u)"),  # negative zero
])
def test_float_literals(lit, text):
    """Output format of a float literal: its exact decimal when the value has at most 16 binary
    fraction digits, else its bit pattern reinterpreted, so that every literal reads back to the
    same bits."""
    r = oracle.decompile(_suffix_kernel(f"v_add_f32 v6, {lit}, v8"))
    assert f"    var0 = ({text} + as_float(y));\n" in r.text


@pytest.mark.parametrize("op,want,stmt", [
    # int and int join to int: no conversion
    ("v_and_b32 v6, v7, v8", "int", "var0 = (x & y);"),
    ("v_xor_b32 v6, v7, v8", "int", "var0 = (x ^ y);"),
    # float and int join to the top of the 32-bit chain, printed as uint: the float's bits are read
    # as an unsigned integer, the int is cast
    ("v_add_f32 v9, v7, v8\n        v_and_b32 v6, v9, v7", "uint",
     "var0 = (as_uint((as_float(x) + as_float(y))) & (uint)x);"),
    # uint and int join to top32 as well
    ("v_add_u32 v9, v7, v8\n        v_and_b32 v6, v9, v7", "uint", "var0 = (((uint)x + (uint)y) & (uint)x);"),
])
def test_bitwise_operations_take_the_join_of_their_operands(op, want, stmt):
    """"Data type recovery": a bitwise operation has no type of its own; its result takes the join
    of its operands' types in the lattice none < {int, uint, float} < top32, and top prints as
    uint."""
    r = oracle.decompile(_suffix_kernel(op))
    assert r.worst == 0
    assert re.findall(r"^    (\w+) (var\d+);", r.text, re.M) == [(want, "var0")]
    assert "    " + stmt + "\n" in r.text


@pytest.mark.parametrize("op,stmt", [
    # int arguments under a float operation: the register's bits are read as a float
    ("v_add_f32 v6, v7, v8", "var0 = (as_float(x) + as_float(y));"),
    # the paper's _u32 example: the signed arguments are read as unsigned
    ("v_add_u32 v6, v7, v8", "var0 = ((uint)x + (uint)y);"),
    # a conversion instruction converts the value
    ("v_cvt_f32_i32 v6, v7", "var0 = (float)x;"),
])
def test_operands_convert_to_the_suffix_type(op, stmt):
    """"Data type recovery": the arguments' types are fixed by the signature, so an operand of
    another type than the suffix asks for is converted: a cast between integers, a reinterpretation
    of the bits between an integer and a float, and a value conversion for a cvt instruction."""
    r = oracle.decompile(_suffix_kernel(op))
    assert "    " + stmt + "\n" in r.text


# ---- "Search for control structures", Fig. 3 --------------------------------
def test_fig3_region_trace():
    lines = [l.split() for l in gold("fig3_trace.txt").split("\n") if l and not l.startswith("#")]
    edges = [tuple(int(x) for x in e.split(">")) for e in lines[0][1:]]
    n = 6
    succ = {b: [] for b in range(1, n + 1)}
    for a, b in edges:
        succ[a].append(b)
    s0 = [succ[b][0] - 1 if succ[b] else -1 for b in range(1, n + 1)]
    s1 = [succ[b][1] - 1 if len(succ[b]) > 1 else -1 for b in range(1, n + 1)]
    log = oracle.reduce_graph(s0, s1)
    want = [(int(l[1]), sorted(int(x) for x in l[3:])) for l in lines[1:]]
    got = [(nid + 1, sorted(m + 1 for m in members)) for nid, members in log]
    assert got == want


def test_fig3_unstructured_graph_does_not_reduce():
    # two blocks jumping into each other's middle: an irreducible loop
    assert oracle.reduce_graph([1, 2, 1], [2, -1, -1]) is None


# ---- exec-mask if-else forms (Fig. 4, Fig. 5) --------------------------------
@pytest.mark.parametrize("form", [1, 2, 3])
def test_ifelse_forms_reduce_to_standard_form(form):
    r = oracle.decompile(gold(f"ifelse_form{form}.s"))
    assert r.status == [0]
    assert r.text == gold("ifelse.cl")


# ---- the type lattice: a join semilattice -----------------------------------
def test_type_join_is_a_semilattice():
    ts = range(9)
    j = oracle.type_join
    for a in ts:
        assert j(0, a) == a and j(a, 0) == a and j(a, a) == a
        for b in ts:
            assert j(a, b) == j(b, a)
            for c in ts:
                assert j(j(a, b), c) == j(a, j(b, c))
    # monotone: a <= b  =>  join(a, c) <= join(b, c), with x <= y iff join(x, y) == y
    for a in ts:
        for b in ts:
            if j(a, b) != b:
                continue
            for c in ts:
                assert j(j(a, c), j(b, c)) == j(b, c)


# ---- dataflow invariants on generated kernels --------------------------------
def _batch(cfg, n, **over):
    p = gcngen.preset(cfg, **over)
    return gcngen.generate(p, n, seed=gcngen.SEED_BASE + 7 + cfg)


def test_every_read_has_a_reaching_definition():
    b = _batch(1, 40, max_len=600)
    for i in range(len(b)):
        r = oracle.decompile(b.kernel(i), with_ir=True)
        stats = np.frombuffer(r.ir[0][oracle.IR_STATS], np.uint32)
        assert r.status == [0]
        assert stats[1] == 0, f"kernel {i}: {stats[1]} reads without a reaching definition"


def test_join_versions_are_minimal():
    # every used join version merges at least two different values (no trivial joins)
    b = _batch(1, 60, max_len=1500)
    used = 0
    for i in range(len(b)):
        r = oracle.decompile(b.kernel(i), with_ir=True)
        stats = np.frombuffer(r.ir[0][oracle.IR_STATS], np.uint32)
        used += int(stats[3])
        assert stats[4] == 0, f"kernel {i}: {stats[4]} trivial join versions"
    assert used > 0


@pytest.mark.parametrize("cfg", [1, 5, 6, 7, 8, 9])
def test_output_is_wellformed_opencl(cfg):
    b = _batch(cfg, 60, max_len=900)
    out, oo, st = oracle.decompile_batch(b.text, b.offsets)
    assert (st == 0).all()
    for i in range(len(b)):
        txt = out[oo[i]:oo[i + 1]].tobytes().decode()
        ks = ocl_eval.parse(txt)
        assert len(ks) == 1
        assert txt.count("{") == txt.count("}") and txt.count("(") == txt.count(")")


# ---- brute force: assembly vs decompiled OpenCL on random buffers -----------
@pytest.mark.parametrize("cfg,n,maxlen", [(0, 4, 0), (1, 40, 400), (4, 6, 1500), (5, 40, 400)])
def test_brute_force_semantics(cfg, n, maxlen):
    over = dict(cws0=8, cws1=4)
    if maxlen:
        over["max_len"] = maxlen
    b = _batch(cfg, n, **over)
    for i in range(len(b)):
        txt = b.kernel(i).decode()
        r = oracle.decompile(txt)
        assert r.status == [0]
        assert brute.check(txt, r.text, seed=i) is None, f"kernel {i}"


def test_brute_force_large_cfg_style():
    # the large-CFG workload's instruction mix (int/long, spills, deep loops) at a small size
    # a low VGPR budget forces locals into scratch slots
    b = _batch(3, 4, min_len=600, max_len=600, trip_max=2, max_depth=4, cws0=8, cws1=4,
               vgpr_budget=40, max_locals=40)
    spilled = 0
    for i in range(len(b)):
        txt = b.kernel(i).decode()
        spilled += "buffer_store_dword" in txt
        r = oracle.decompile(txt)
        assert r.status == [0]
        assert brute.check(txt, r.text, seed=i) is None, f"kernel {i}"
    assert spilled > 0


def test_brute_force_catches_planted_mistake():
    b = _batch(0, 1, cws0=8, cws1=4)
    txt = b.kernel(0).decode()
    good = oracle.decompile(txt).text
    bad = good.replace("get_global_id(0)", "get_local_id(0)", 1)
    assert bad != good and brute.check(txt, bad) is not None


# ---- files, kernels and failure statuses (Listing 2) --------------------------
def test_multi_kernel_file_equals_single_files():
    b = _batch(1, 5, max_len=300)
    whole = "junk before the first kernel\n" + "".join(b.kernel(i).decode() for i in range(5))
    r = oracle.decompile(whole)
    assert r.status == [0] * 5
    assert r.text == "\n".join(oracle.decompile(b.kernel(i)).text for i in range(5))


def test_kernel_with_empty_text_is_not_lost():
    src = ".kernel a\n    .config\n        .dims x\n.kernel b\n    .config\n        .dims x\n    .text\n        s_endpgm\n"
    r = oracle.decompile(src)
    assert r.text == "__kernel void a(void)\n{\n}\n\n__kernel void b(void)\n{\n}\n"


def test_unknown_instruction_is_inline_asm_and_partial():
    txt = gold("p194_global_offset.s").replace("        s_endpgm", "        v_frobnicate_b32 v7, v6\n        s_endpgm")
    r = oracle.decompile(txt)
    assert r.status == [1]
    assert '__asm__("v_frobnicate_b32 v7, v6");' in r.text


@pytest.mark.parametrize("mut", ["v_mov_b32 v6, s2x", "s_branch .Lnowhere", "v_mov_b32 v99, v0"])
def test_parse_errors(mut):
    txt = gold("p194_global_offset.s").replace("        v_mov_b32 v6, s2", "        " + mut)
    r = oracle.decompile(txt)
    assert r.status == [2]
    assert "not decompiled" in r.text


# ---- the type fixed point's sweep limit ("Data type recovery"; the paper gives no limit) ----
# A kernel whose every node is typed by its operation (no bitwise operation, select or
# type-keeping shift whose type comes from its operands, no join) has nothing to solve:
# the first sweep changes nothing, so even a limit of one sweep leaves it decompiled.
NO_OPERAND_TYPED = """.kernel plain_store
  .config
    .dims x
    .cws 64, 1, 1
    .sgprsnum 16
    .vgprsnum 8
    .floatmode 0xc0
    .useargs
    .priority 0
    .arg _.global_offset_0, "size_t", long
    .arg _.global_offset_1, "size_t", long
    .arg _.global_offset_2, "size_t", long
    .arg _.printf_buffer, "size_t", void*, global, , rdonly
    .arg _.vqueue_pointer, "size_t", long
    .arg _.aqlwrap_pointer, "size_t", long
    .arg out, "uint*", uint*, global,
    .arg n, "uint", uint
  .text
    s_load_dwordx2 s[8:9], s[4:5], 0x30
    s_load_dword s10, s[4:5], 0x38
    s_waitcnt lgkmcnt(0)
    v_mov_b32 v2, s8
    v_mov_b32 v3, s9
    v_add_u32 v1, s10, v0
    global_store_dword v[2:3], v1, off
    s_endpgm
"""


def _with_sweep_limit(n, texts):
    oracle.set_type_sweep_limit(n)
    try:
        return [oracle.decompile(t) for t in texts]
    finally:
        oracle.set_type_sweep_limit(0)


def test_sweep_limit_caps_kernels_that_still_change():
    """At a limit of one sweep, a kernel whose first sweep still raises a type (most generated
    kernels: their reached bitwise operations take the type of their operands) is capped: status
    3 and the not-decompiled text under the kernel's signature; a kernel whose first sweep
    changes nothing is printed as without a limit; the default limit caps nothing."""
    b = gcngen.generate(1, 6)
    texts = [b.kernel(i) for i in range(6)] + [NO_OPERAND_TYPED, gold("listing3_copy.s")]
    base = [oracle.decompile(t) for t in texts]
    assert all(r.worst != 3 for r in base)
    capped = _with_sweep_limit(1, texts)
    assert sum(r.status == [3] for r in capped[:6]) >= 3
    for r, full in zip(capped, base):
        if r.status == [3]:
            head = full.text.split("\n")[0]
            assert r.text == head + "\n{\n    /* not decompiled: fixed-point limit */\n}\n"
        else:
            assert r.text == full.text and r.status == full.status
    assert [r.status for r in capped[6:]] == [[0], [0]]


def test_sweep_limit_is_monotone_and_bounded_by_the_lattice_height():
    """A kernel capped at limit L is capped at every smaller limit; it is never capped at
    2 * (nodes + joins) + 1 sweeps, since every sweep that changes something raises one of
    them and each can rise at most twice (bottom, a type, top)."""
    b = gcngen.generate(gcngen.preset(1, w_if=0, w_ifelse=0, w_loop=1), 4, seed=gcngen.SEED_BASE + 41)
    for i in range(4):
        t = b.kernel(i)
        capped = [r.worst == 3 for r in (_with_sweep_limit(L, [t])[0] for L in range(1, 9))]
        first_ok = capped.index(False) if False in capped else None
        assert first_ok is not None and all(capped[:first_ok]) and not any(capped[first_ok:])
        n_nodes = 4 * len(t.split(b"\n"))
        assert _with_sweep_limit(2 * n_nodes + 1, [t])[0].worst != 3


# ---- "The body extraction": FLAT instructions and the double-suffix V_MUL_HI family ----------
def test_flat_and_mul_hi_golden():
    """flat_load/flat_store through a buffer address are that buffer's elements, like the GLOBAL
    instructions; v_mul_hi_u32_u24 / v_mul_hi_i32_i24 are the high half of the 24-bit products,
    typed by their first suffix (uint / int).  The expected text is derived by hand."""
    r = oracle.decompile(gold("flat_mulhi.s"))
    assert r.status == [0]
    assert r.text == gold("flat_mulhi.cl")


def test_brute_force_flat_and_mul_hi_golden():
    """The golden kernel and its text compute the same buffers on full-range operands, and three
    planted mistakes fail: no 24-bit mask, no sign extension, and the low half instead."""
    asm, good = gold("flat_mulhi.s"), gold("flat_mulhi.cl")
    for seed in range(3):
        assert brute.check(asm, good, seed=seed, wide=True) is None
    planted = [good.replace("(var0 & 16777215u)", "var0", 1),
               good.replace("((int)(var0 << 8) >> 8)", "(int)var0", 1),
               good.replace("(uint)mul_hi(", "(uint)mul24(", 1).replace(
                   "mul24(((int)(8388609u << 8) >> 8), ((int)(var0 << 8) >> 8))", "mul24(8388609u, var0)", 1)]
    for bad in planted:
        assert bad != good
        assert brute.check(asm, bad, seed=0, wide=True) is not None


def test_brute_force_flat_and_mul_hi_preset():
    """Generated kernels with FLAT accesses and high multiplies (preset 7): the decompiled text
    computes the assembly's buffers on full-range operands."""
    b = _batch(7, 30, max_len=400, cws0=8, cws1=4)
    seen = {"flat_load": 0, "flat_store": 0, "v_mul_hi_u32_u24": 0, "v_mul_hi_i32_i24": 0}
    for i in range(len(b)):
        txt = b.kernel(i).decode()
        for k in seen:
            seen[k] += txt.count(k)
        r = oracle.decompile(txt)
        assert r.status == [0]
        assert brute.check(txt, r.text, seed=i, wide=True) is None, f"kernel {i}"
    assert all(seen.values()), seen


# ---- early exits from counted loops (loops are a project extension; "Search for control
# structures" gives the templates they build on) ------------------------------------------------
@pytest.mark.parametrize("name", ["loop_break", "loop_continue"])
def test_early_exit_goldens(name):
    """A uniform test that leaves the loop prints `if (c) { <join copies> break; }` inside the
    do-while; one that skips to the latch is an if around the rest of the body.  The expected
    texts are derived by hand."""
    r = oracle.decompile(gold(name + ".s"))
    assert r.status == [0]
    assert r.text == gold(name + ".cl")


@pytest.mark.parametrize("name", ["loop_break", "loop_continue"])
def test_brute_force_early_exit_goldens(name):
    """The assembly and the text agree for an exit at every iteration (n = 0..3) and none (n = 4)."""
    for n in range(5):
        assert brute.check(gold(name + ".s"), gold(name + ".cl"), seed=n, scalars={"n": n}) is None


def test_brute_force_catches_misplaced_break_copy():
    good = gold("loop_break.cl")
    planted = [good.replace("            var5 = var2;\n", ""),               # the exit value not passed
               good.replace("        if (var1 == n) {", "        if (var1 != n) {"),  # the test inverted
               good.replace("            break;\n", "")]                      # no exit at all
    for bad in planted:
        assert bad != good
        assert any(brute.check(gold("loop_break.s"), bad, seed=n, scalars={"n": n}) is not None for n in range(4))


def test_exit_from_an_outer_loop_stays_unstructured():
    """A jump from an inner loop's body to the outer loop's exit would need a two-level break:
    the rule only cuts an exit of the innermost loop, so the graph does not reduce and the kernel
    is not decompiled (PARTIAL)."""
    src = gold("loop_break.s")
    nested = src.replace("LOOP:\n", "OUTER:\n    s_mov_b32 s13, 0\nLOOP:\n").replace(
        "    s_cbranch_scc1 LOOP\n", "    s_cbranch_scc1 LOOP\n    s_add_u32 s13, s13, 1\n"
        "    s_cmp_lt_u32 s13, 3\n    s_cbranch_scc1 OUTER\n")
    assert nested != src
    r = oracle.decompile(nested)
    assert r.status == [1]
    assert "/* not decompiled: unstructured control flow */" in r.text


def test_brute_force_mixed_nesting_and_early_exits():
    """Preset 8: divergent and uniform ifs of every form nested with loops, a third of the loops
    with a break or continue; the decompiled text computes the assembly's buffers."""
    b = _batch(8, 40, max_len=600, cws0=8, cws1=4)
    breaks = 0
    for i in range(len(b)):
        txt = b.kernel(i).decode()
        r = oracle.decompile(txt)
        assert r.status == [0]
        breaks += r.text.count("break;")
        assert brute.check(txt, r.text, seed=i, scalars={"n": i % 5}) is None, f"kernel {i}"
    assert breaks > 0


# ---- LDS ("The AMD GCN architecture": LDS is OpenCL local memory; "The body extraction":
# data share operations, prefix ds) ------------------------------------------------------------
def test_lds_golden():
    """A __local argument's slot holds its LDS address; ds_write / ds_read at that address plus
    the index shifted by the element size are elements of the buffer; s_barrier is the work-group
    barrier.  The expected text is derived by hand."""
    r = oracle.decompile(gold("lds_exchange.s"))
    assert r.status == [0]
    assert r.text == gold("lds_exchange.cl")


def test_brute_force_lds_golden_and_planted_mistakes():
    asm, good = gold("lds_exchange.s"), gold("lds_exchange.cl")
    for seed in range(3):
        assert brute.check(asm, good, seed=seed) is None
    planted = [good.replace("    barrier(CLK_LOCAL_MEM_FENCE);\n", ""),          # no barrier
               good.replace("(1u + get_local_id(0))", "(2u + get_local_id(0))"),   # another neighbour
               good.replace("tmp[get_local_id(0)] = var0;", "tmp[0] = var0;")]     # another element
    for bad in planted:
        assert bad != good
        assert brute.check(asm, bad, seed=0) is not None


def test_lds_address_that_is_no_element_is_partial():
    """An LDS address scaled by 8 for a buffer of 4-byte elements names no element: the access is
    printed as pseudo-code through a __local pointer and the kernel is PARTIAL."""
    src = gold("lds_exchange.s").replace("v_lshlrev_b32 v8, 2, v0", "v_lshlrev_b32 v8, 3, v0")
    r = oracle.decompile(src)
    assert r.status == [1]
    assert "*((__local uint *)(" in r.text


def test_brute_force_lds_preset():
    """Preset 9: exchanges through a __local buffer (write, barrier, read a neighbour) among the
    batch mix; the decompiled text computes the assembly's buffers."""
    b = _batch(9, 30, max_len=500, cws0=8)
    barriers = 0
    for i in range(len(b)):
        txt = b.kernel(i).decode()
        r = oracle.decompile(txt)
        assert r.status == [0]
        barriers += r.text.count("barrier(CLK_LOCAL_MEM_FENCE);")
        assert brute.check(txt, r.text, seed=i) is None, f"kernel {i}"
    assert barriers > 0


# ---- generator ground truth: the system values the generator built ("Search for memory
# accesses": the get_global_id chain with and without the global offset) -----------------------
@pytest.mark.parametrize("cfg", [0, 1, 2, 5, 6, 7, 8])
def test_global_ids_recovered_as_the_generator_built_them(cfg):
    """Every kernel computes get_global_id(d) once per dimension (group id times work-group size
    plus local id, the global offset added or not) and uses that register as an expression leaf.
    The decompiled text must show each use as exactly that value: get_global_id(d) when the chain
    adds the offset, the idiom (get_global_id(d) - get_global_offset(d)) when it does not, no
    get_global_id of a dimension the kernel does not have, and no raw group or local id."""
    b = gcngen.generate(cfg, 120, seed=gcngen.SEED_BASE + 300 + cfg)
    uses = 0
    for i in range(len(b)):
        t = oracle.decompile(b.kernel(i)).text
        truth = int(b.truth[i, 0])
        dims = truth & 3
        assert "get_group_id(" not in t and "get_local_id(" not in t, f"kernel {i}"
        for d in range(2):
            gid, idiom = f"get_global_id({d})", f"(get_global_id({d}) - get_global_offset({d}))"
            if d >= dims:
                assert gid not in t, f"kernel {i}: dimension {d} of a {dims}-D kernel"
                continue
            if truth & (4 << d):
                assert idiom not in t, f"kernel {i}: dimension {d} adds the offset"
            else:
                assert t.count(gid) == t.count(idiom), f"kernel {i}: dimension {d} is offset-free"
            uses += t.count(gid)
    assert uses >= 4 * len(b)  # the property is exercised (about 8 to 50 uses per kernel)


@pytest.mark.parametrize("cfg", [0, 1, 2, 5, 6, 7, 8, 9])
def test_control_structure_as_the_generator_built_it(cfg):
    """"Search for control structures" and the loop template, against what the generator emitted:
    every divergent if / if-else (in all three exec-mask forms), uniform if / if-else and
    early-exit test prints as exactly one `if (`, every counted loop as one `do {`; an else part
    the program has prints as `} else {`, and an if without one may still print an else part
    holding the join copies of its skip edge, so the generated else parts are a lower bound."""
    b = gcngen.generate(cfg, 120, seed=gcngen.SEED_BASE + 500 + cfg)
    stats = [0, 0, 0]
    for i in range(len(b)):
        r = oracle.decompile(b.kernel(i))
        assert r.status == [0], f"kernel {i}"
        n_if, n_else, n_loop = (int(x) for x in b.truth[i, 1:])
        assert r.text.count("if (") == n_if, f"kernel {i}: ifs"
        assert r.text.count("do {") == n_loop, f"kernel {i}: loops"
        assert r.text.count("} else {") >= n_else, f"kernel {i}: else parts"
        stats = [stats[0] + n_if, stats[1] + n_else, stats[2] + n_loop]
    assert stats[0] > 0 and (cfg == 0 or stats[2] > 0)


# ---- damaged input: the decompiler takes arbitrary disassembly text ---------------------------
def _damaged(n, seed, cws=False):
    import mutate

    texts = []
    for cfg in (0, 1, 5, 7, 8, 9):
        over = dict(max_len=400)
        if cws and cfg != 9:
            over.update(cws0=8, cws1=4)
        b = _batch(cfg, 30, **over)
        texts += [b.kernel(i) for i in range(len(b))]
    return mutate.mutants(texts, n, seed)


def test_damaged_files_decompile_to_balanced_text():
    """Generated files with lines missing, repeated or swapped, misspelled mnemonics and operands,
    registers out of range, undefined and doubled labels, bad configuration values, CRLF endings,
    comments and truncation: every file decompiles; a file whose worst kernel is a parse error says
    so; every output has balanced braces and parentheses.  (Whether an OK output also runs is the
    brute-force test's job below: the evaluator takes no buffer argument used as a value, which a
    damaged address computation can print.)"""
    st = [0, 0, 0]
    for k, m in enumerate(_damaged(800, 2107)):
        r = oracle.decompile(m)
        assert r.worst in (0, 1, 2), f"file {k}"
        st[r.worst] += 1
        assert r.text.count("{") == r.text.count("}") and r.text.count("(") == r.text.count(")"), f"file {k}"
        if r.worst == 2:
            assert "not decompiled: parse error" in r.text, f"file {k}"
    assert min(st) > 50  # every outcome is exercised


def test_brute_force_on_damaged_files():
    """Damaged files the oracle decompiles without inline assembly still compute what their
    (damaged) assembly computes, on every file the interpreter and the evaluator can run (the
    interpreter takes no comment rows and stops a program whose damaged address leaves every
    buffer, the evaluator takes no pointer arithmetic on buffer arguments)."""
    checked = 0
    for k, m in enumerate(_damaged(300, 99, cws=True)):
        r = oracle.decompile(m)
        if r.worst != 0:
            continue
        try:
            ocl_eval.parse(r.text)
        except ocl_eval.ParseError:
            continue
        try:
            err = brute.check(m.decode(errors="replace"), r.text, seed=k)
        except (AssertionError, NotImplementedError, IndexError):
            continue
        if err is not None and "vacuous" in err:
            continue
        assert err is None, f"file {k}: {err}"
        checked += 1
    assert checked >= 40


@pytest.mark.parametrize("cfg", [0, 1, 3, 5, 6, 7, 8, 9])
def test_class_depth_bound_changes_nothing(cfg):
    """Classification stops four levels below a value (a class comes from operands at most three
    levels down, and below that an operand can only keep a pattern from matching): with the bound
    raised to 1,000 levels every generated kernel decompiles to the same text."""
    b = _batch(cfg, 4 if cfg == 3 else 40, **({"max_len": 20000} if cfg == 3 else {}))
    texts = [b.kernel(i) for i in range(len(b))]
    want = [oracle.decompile(t).text for t in texts]
    oracle.set_class_depth(1000)
    try:
        got = [oracle.decompile(t).text for t in texts]
    finally:
        oracle.set_class_depth()
    assert got == want


def _fused_add(hi_sources):
    return f""".kernel k
    .text
        v_mov_b32 v2, 7
        s_mov_b32 s4, 9
        v_mov_b32 v3, 11
        v_add_co_u32 v0, vcc, v2, s4
        v_addc_co_u32 v1, vcc, {hi_sources}, vcc
        global_load_dword v5, v[0:1], off
        global_store_dword v[0:1], v5, off
        s_endpgm
"""


@pytest.mark.parametrize("hi,want", [
    # low halves 7 and 9 (v2, s4); high halves as written: the two 64-bit operands are
    # hi << 32 | lo, folded to their values
    ("0, v3", "(7UL + 47244640265UL)"),             # 0 << 32 | 7,  11 << 32 | 9
    ("v3, 5", "(47244640263UL + 21474836489UL)"),   # 11 << 32 | 7,  5 << 32 | 9
    ("s4, v3", "(38654705671UL + 47244640265UL)"),  # 9 << 32 | 7,  11 << 32 | 9
])
def test_fused_add_with_a_constant_high_source(hi, want):
    """A 64-bit add whose high half adds an inline constant (as compilers write for a 32-bit
    offset added to a pointer) fuses into one 64-bit add of the two register pairs; the value
    of each operand is fixed by its halves."""
    r = oracle.decompile(_fused_add(hi))
    assert r.worst == 0
    assert f"var0 = {want};" in r.text


def test_fused_add_with_two_constant_high_sources_stays_split():
    """Two constant high sources leave the carry half on its own (no slot is left for the second
    constant); the low half is still the 32-bit sum."""
    r = oracle.decompile(_fused_add("0, 1"))
    assert "(7u + 9u)" in r.text and "UL" not in r.text


def test_damaged_fused_add_is_not_self_referential():
    """A damaged file whose carry half adds an inline float constant to a low half that reads a
    register nothing wrote: every value is built from earlier ones (no variable is defined from
    itself), so the decompilation is finite."""
    asm = b""".kernel k37
    .text
        v_add_co_u32 v14, vcc, v14, s16
        v_addc_co_u32 v15, vcc, -4.0, v16, vcc
        global_load_dwordx2 v[12:13], v[14:15], off
        s_and_saveexec_b64 s[30:31], vcc
        s_xor_b64 s[30:31], exec, s[30:31]
        s_or_saveexec_b64 s[30:31], s[30:31]
        s_xor_b64 exec, exec, s[30:31]
        s_or_b64 exec, exec, s[30:31]"""
    oracle.set_class_depth(1000)
    try:
        r = oracle.decompile(asm)
    finally:
        oracle.set_class_depth()
    # -4.0 is 0xc0800000 = 3229614080; the unwritten registers read as 0
    assert "var0 = *((__global ulong *)((upsample(3229614080u, 0u) + upsample(0u, 0u))));" in r.text
