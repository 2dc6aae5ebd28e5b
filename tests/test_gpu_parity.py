"""GPU parity: the CUDA decompiler, called through the C ABI, against the CPU oracle.

Integer, byte and index work: every compared array and every byte of text must
be identical."""
import numpy as np
import pytest

import gcngen
import oracle
import paper_2107_07809_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dec():
    pkg.build()
    d = pkg.Decompiler(0)
    yield d
    d.close()


def _files(cfg, n, **over):
    p = gcngen.preset(cfg, **over)
    b = gcngen.generate(p, n, seed=gcngen.SEED_BASE + cfg)
    return [b.kernel(i) for i in range(n)]


def _check_ir(dec, files):
    ids = dec.submit_batch(files)
    assert len(ids) == len(files)
    for f, j in zip(files, ids):
        want = oracle.decompile(f, with_ir=True)
        for which in range(6):
            got = dec.fetch_ir(j, which)
            exp = b"".join(k[which] for k in want.ir)
            assert got == exp, f"IR array {which} differs"
        dec.fetch_opencl(j)


def test_ir_parity_small(dec):
    _check_ir(dec, _files(0, 1))


def test_ir_parity_config1_sample(dec):
    _check_ir(dec, _files(1, 300))


def test_ir_parity_ternary_mix(dec):
    _check_ir(dec, _files(5, 150))


def test_ir_parity_sysval_mix(dec):
    _check_ir(dec, _files(6, 150))


def test_ir_parity_flat_mulhi_mix(dec):
    _check_ir(dec, _files(7, 150))


def test_ir_parity_mixed_nesting(dec):
    _check_ir(dec, _files(8, 150))


def test_ir_parity_lds_mix(dec):
    _check_ir(dec, _files(9, 150))


def test_ir_parity_multi_kernel_files(dec):
    ks = _files(1, 12, max_len=400)
    files = [b"".join(ks[0:4]), b"leading junk\n" + b"".join(ks[4:9]), ks[9], b"", b"".join(ks[10:12])]
    _check_ir(dec, files)


def test_ir_parity_golden_fixtures(dec):
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    files = [open(os.path.join(g, f), "rb").read() for f in sorted(os.listdir(g)) if f.endswith(".s")]
    _check_ir(dec, files)


# ---- OpenCL text: byte-identical to the oracle -------------------------------
def _check_text(dec, files):
    ids = dec.submit_batch(files)
    assert len(ids) == len(files)
    for n, (f, j) in enumerate(zip(files, ids)):
        want = oracle.decompile(f)
        got, status = dec.fetch_opencl(j)
        assert got == want.text, f"file {n}: OpenCL text differs"
        assert status == want.worst, f"file {n}: status {status} vs {want.worst}"


def test_text_parity_config0(dec):
    _check_text(dec, _files(0, 1))


def test_text_parity_ternary_mix(dec):
    """the batch mix with selects (v_cndmask_b32) in 15% of 32-bit operations"""
    _check_text(dec, _files(5, 600))


def test_text_parity_sysval_mix(dec):
    """the batch mix with dispatch-packet system values and scalar bit fields in 10% of integer leaves"""
    _check_text(dec, _files(6, 600))


def test_text_parity_flat_mulhi_mix(dec):
    """the batch mix with FLAT loads/stores (30% of accesses) and double-suffix high multiplies
    (10% of 32-bit integer operations)"""
    _check_text(dec, _files(7, 600))


def test_text_parity_flat_mulhi_edge_cases(dec):
    """FLAT accesses whose address is not a buffer element (raw pointer arithmetic), a FLAT
    64-bit access, high multiplies of registers and of two literals"""
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    base = open(os.path.join(g, "flat_mulhi.s"), "rb").read()
    files = [
        base.replace(b"v_lshlrev_b64 v[4:5], 2, v[2:3]\n    v_mov_b32 v6, s9",
                     b"v_lshlrev_b64 v[4:5], 3, v[2:3]\n    v_mov_b32 v6, s9"),
        base.replace(b"v_mul_hi_u32_u24 v8, 0xfedcba, v7", b"v_mul_hi_u32_u24 v8, v7, v7"),
        base.replace(b"v_mul_hi_i32_i24 v9, 0x800001, v7", b"v_mul_hi_i32_i24 v9, v0, v7"),
        base.replace(b"flat_store_dword v[4:5], v8", b"flat_store_dwordx2 v[4:5], v[8:9]"),
        base.replace(b"flat_load_dword v7, v[4:5]", b"global_load_dword v7, v[4:5], off"),
        base.replace(b"flat_load_dword v7, v[4:5]", b"flat_load_dword v7, v[4:5] offset:8"),
    ]
    assert len(set(files)) == len(files)
    _check_text(dec, files)


def test_text_parity_mixed_nesting_and_early_exits(dec):
    """divergent if / if-else (three forms), uniform ifs and loops nested to depth 4, a third of
    the loops with a break or continue"""
    files = _files(8, 600)
    _check_text(dec, files)
    assert sum(oracle.decompile(f).text.count("break;") for f in files[:200]) > 0


def test_text_parity_early_exit_edge_cases(dec):
    """an exit from an inner loop to the outer loop's exit (unstructured), an exit whose other
    branch leaves the loop too, an exit at the loop's first block, and two exits of one loop"""
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    base = open(os.path.join(g, "loop_break.s"), "rb").read()
    files = [
        base.replace(b"LOOP:\n", b"OUTER:\n    s_mov_b32 s13, 0\nLOOP:\n").replace(
            b"    s_cbranch_scc1 LOOP\n", b"    s_cbranch_scc1 LOOP\n    s_add_u32 s13, s13, 1\n"
            b"    s_cmp_lt_u32 s13, 3\n    s_cbranch_scc1 OUTER\n"),
        base.replace(b"    s_cbranch_scc1 DONE\n    v_add_u32 v7, v7, 5\n",
                     b"    s_cbranch_scc1 DONE\n    s_branch DONE\n    v_add_u32 v7, v7, 5\n"),
        base.replace(b"LOOP:\n    v_add_u32 v7, v7, 3\n", b"LOOP:\n"),
        base.replace(b"    v_add_u32 v7, v7, 5\n", b"    v_add_u32 v7, v7, 5\n    s_cmp_eq_u32 s12, 2\n"
                     b"    s_cbranch_scc1 DONE\n    v_add_u32 v7, v7, 1\n"),
    ]
    assert len(set(files)) == len(files)
    _check_text(dec, files)


def test_text_parity_lds_mix(dec):
    """1-D kernels with a __local argument: ds writes of the own slot, a barrier, ds reads of
    a neighbour's slot (40% of kernels), among global accesses"""
    files = _files(9, 600)
    _check_text(dec, files)
    assert sum(oracle.decompile(f).text.count("barrier(") for f in files[:200]) > 0


def test_text_parity_lds_edge_cases(dec):
    """LDS addresses that are no element of the __local buffer (no base, a literal base, 64-bit
    accesses at a 4-byte stride), 64-bit accesses at their own stride, ds offsets (unsupported),
    no barrier and two barriers"""
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    base = open(os.path.join(g, "lds_exchange.s"), "rb").read()
    files = [
        base.replace(b"    v_add_u32 v9, s10, v9\n    ds_read_b32", b"    ds_read_b32"),
        base.replace(b"ds_read_b32 v9, v9\n", b"ds_read_b32 v9, v9 offset:4\n"),
        base.replace(b"ds_write_b32 v8, v7\n", b"ds_write_b32 v8, v7 offset:8\n"),
        base.replace(b"    s_waitcnt lgkmcnt(0)\n    s_barrier\n", b""),
        base.replace(b"ds_write_b32 v8, v7", b"ds_write_b64 v8, v[6:7]").replace(
            b"ds_read_b32 v9, v9", b"ds_read_b64 v[8:9], v9"),
        base.replace(b"ds_write_b32 v8, v7", b"ds_write_b64 v8, v[6:7]").replace(
            b"ds_read_b32 v9, v9", b"ds_read_b64 v[8:9], v9").replace(
            b"v_lshlrev_b32 v8, 2, v0", b"v_lshlrev_b32 v8, 3, v0").replace(
            b"v_lshlrev_b32 v9, 2, v9", b"v_lshlrev_b32 v9, 3, v9"),
        base.replace(b"    v_add_u32 v8, s10, v8\n", b"    v_add_u32 v8, 0x100, v8\n"),
        base.replace(b"    s_barrier\n", b"    s_barrier\n    s_barrier\n"),
    ]
    assert len(set(files)) == len(files)
    _check_text(dec, files)


def test_text_parity_sysval_edge_cases(dec):
    """dispatch packet loads and fields that are not system values: other offsets, a wide load,
    shifts by the other dimension's size, fields of width 0 and 32, a field and a shift amount
    held in registers"""
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    base = open(os.path.join(g, "sysvals_dispatch.s"), "rb").read()
    files = [
        base.replace(b"s_load_dword s10, s[0:1], 0xc", b"s_load_dword s10, s[0:1], 0x4"),
        base.replace(b"s_load_dword s10, s[0:1], 0xc", b"s_load_dword s10, s[0:1], 0x18"),
        base.replace(b"s_load_dword s12, s[0:1], 0x0", b"s_load_dword s12, s[0:1], 0x8"),
        base.replace(b"s_load_dword s11, s[0:1], 0x10", b"s_load_dwordx2 s[14:15], s[0:1], 0x10\n        s_mov_b32 s11, s14"),
        base.replace(b"s_lshr_b32 s11, s11, 3", b"s_lshr_b32 s11, s11, 4"),
        base.replace(b"s_lshr_b32 s11, s11, 3", b"s_lshr_b32 s11, s11, s13"),
        base.replace(b"s_bfe_u32 s12, s12, 0x20010", b"s_bfe_u32 s12, s12, 0x30010"),
        base.replace(b"s_bfe_u32 s13, s10, 0x40004", b"s_bfe_u32 s13, s10, 0x4"),
        base.replace(b"s_bfe_u32 s13, s10, 0x40004", b"s_bfe_u32 s13, s10, 0x200004"),
        base.replace(b"s_bfe_u32 s13, s10, 0x40004", b"s_bfe_u32 s13, s10, s11"),
        base.replace(b"s_load_dword s10, s[0:1], 0xc", b"s_load_dword s10, s[2:3], 0xc"),
        base.replace(b".dims xy", b".dims x").replace(b".cws 16, 8, 1", b".cws 16, 1, 1"),
    ]
    assert len(set(files)) == len(files)
    _check_text(dec, files)


def test_text_parity_golden(dec):
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    _check_text(dec, [open(os.path.join(g, f), "rb").read() for f in sorted(os.listdir(g)) if f.endswith(".s")])


def test_text_parity_config1(dec):
    _check_text(dec, _files(1, 2000))


def test_text_parity_multi_kernel_files(dec):
    ks = _files(1, 30, max_len=600)
    files = [b"".join(ks[0:10]), b"junk\n.text\n" + b"".join(ks[10:20]), b"", b"".join(ks[20:30])]
    _check_text(dec, files)


def test_text_parity_serving_sizes(dec):
    _check_text(dec, _files(4, 40))


def test_text_parity_large_cfg(dec):
    _check_text(dec, _files(3, 2))


def test_text_parity_edge_cases(dec):
    import os
    g = os.path.join(os.path.dirname(__file__), "golden")
    base = open(os.path.join(g, "p194_global_offset.s"), "rb").read()
    files = [
        base.replace(b"        s_endpgm", b"        v_frobnicate_b32 v7, v6\n        s_endpgm"),
        base.replace(b"        v_mov_b32 v6, s2", b"        v_mov_b32 v6, s2x"),
        base.replace(b"        v_mov_b32 v6, s2", b"        s_branch .Lnowhere"),
        base.replace(b"        v_mov_b32 v6, s2", b"        v_mov_b32 v99, v0"),
        base.replace(b".cws 64, 1, 1", b".cws 64, x, 1"),
        b".kernel empty\n    .config\n        .dims x\n",
        b"no kernel here\n",
    ]
    _check_text(dec, files)


def test_text_parity_label_cases(dec):
    """Label lookup through the batch-wide table: a label defined twice (the first definition
    wins), a longer label sharing the branch's name as a prefix, a branch to a name only the
    longer label has (parse error), and a branch to a label only another kernel of the file
    defines (parse error in that kernel only)."""
    t = gcngen.generate(0, 1).kernel(0)
    lines = t.split(b"\n")
    i0 = lines.index(b".L0:")
    dup = b"\n".join(lines[: i0 + 1] + [b".L1:"] + lines[i0 + 1:])
    pre = t.replace(b".L1:", b".L10:\n.L1:")
    only_long = t.replace(b".L1:", b".L10:")
    cross = t + t.replace(b".kernel k0", b".kernel k1").replace(b".L0:", b".M0:")
    _check_text(dec, [dup, pre, only_long, cross])


def test_parity_fused_add_constant_high_sources(dec):
    """64-bit adds whose carry half adds a constant: one constant high source fuses (the
    constant takes the instruction's last operand slot), two stay split; and a damaged file
    whose fused add reads unwritten registers."""
    files = []
    for hi in (b"0, v3", b"v3, 5", b"s4, v3", b"0, 1", b"-4.0, v3", b"0x12345, v3"):
        files.append(b""".kernel k
    .text
        v_mov_b32 v2, 7
        s_mov_b32 s4, 9
        v_mov_b32 v3, 11
        v_add_co_u32 v0, vcc, v2, s4
        v_addc_co_u32 v1, vcc, """ + hi + b""", vcc
        global_load_dword v5, v[0:1], off
        global_store_dword v[0:1], v5, off
        s_endpgm
""")
    files.append(b""".kernel k37
    .text
        v_add_co_u32 v14, vcc, v14, s16
        v_addc_co_u32 v15, vcc, -4.0, v16, vcc
        global_load_dwordx2 v[12:13], v[14:15], off
        s_and_saveexec_b64 s[30:31], vcc
        s_xor_b64 s[30:31], exec, s[30:31]
        s_or_saveexec_b64 s[30:31], s[30:31]
        s_xor_b64 exec, exec, s[30:31]
        s_or_b64 exec, exec, s[30:31]""")
    _check_ir(dec, files)
    _check_text(dec, files)
