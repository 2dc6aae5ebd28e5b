"""Seeded damage to generated kernel files, for parity on inputs the generator never writes: the
decompiler takes arbitrary disassembly text, so lines go missing or repeat, mnemonics and
operands are misspelled, registers fall outside the configured range, labels are undefined or
defined twice, configuration rows carry bad values, line endings are CRLF, and files end in the
middle of a line.  Holds none of the decompiler's arithmetic: it only edits text."""
import random
import re

_LITERALS = [b"0", b"-16", b"64", b"65", b"-17", b"0x10", b"0xffffffff", b"0x100000000", b"4294967296",
             b"1.0", b"-4.0", b"0.25", b"1e3", b"0x", b"-", b"--1", b"vcc", b"exec", b"off", b"v", b"s",
             b"v[1:0]", b"v[0:8]", b"s[3:4]", b"v[0x1:2]"]


def _instr_lines(lines):
    return [i for i, l in enumerate(lines) if l.strip() and not l.strip().startswith(b".") and not l.strip().endswith(b":")]


def _mutate_once(rng, text):
    lines = text.split(b"\n")
    ins = _instr_lines(lines)
    kind = rng.randrange(18)
    if kind == 0 and ins:  # a line goes missing
        del lines[rng.choice(ins)]
    elif kind == 1 and ins:  # a line repeats
        i = rng.choice(ins)
        lines.insert(i, lines[i])
    elif kind == 2 and len(ins) > 1:  # two neighbouring lines swap
        i = rng.randrange(len(ins) - 1)
        a, b = ins[i], ins[i + 1]
        lines[a], lines[b] = lines[b], lines[a]
    elif kind == 3 and ins:  # a register outside the configured range
        i = rng.choice(ins)
        lines[i] = re.sub(rb"\b([vs])(\d+)\b", lambda m: m.group(1) + rng.choice([b"255", b"1023", b"1024", b"99"]),
                          lines[i], count=1)
    elif kind == 4 and ins:  # a misspelled mnemonic
        i = rng.choice(ins)
        l = lines[i]
        j = len(l) - len(l.lstrip())
        k = j + rng.randrange(max(1, len(l.split()[0]) if l.split() else 1))
        if k < len(l):
            lines[i] = l[:k] + bytes([rng.choice(b"abxyz_0")]) + l[k + 1:]
    elif kind == 5 and ins:  # a comma lost, or an empty operand
        i = rng.choice(ins)
        lines[i] = lines[i].replace(b",", rng.choice([b"", b", ,", b",,"]), 1)
    elif kind == 6 and ins:  # an operand replaced by an odd literal or token
        i = rng.choice(ins)
        parts = lines[i].split(b",")
        if len(parts) > 1:
            q = rng.randrange(1, len(parts))
            parts[q] = b" " + rng.choice(_LITERALS)
            lines[i] = b",".join(parts)
    elif kind == 7:  # a garbage line
        lines.insert(rng.randrange(len(lines) + 1),
                     rng.choice([b"    garbage", b"@@@", b"    v_add_u32", b"    s_endpgm extra", b"\t\t", b"label with space:",
                                 b"    s_branch", b"    v_mov_b32 v1, v2, v3, v4, v5, v6"]))
    elif kind == 8 and ins:  # a branch to an undefined label, or a label defined twice
        labels = [i for i, l in enumerate(lines) if l.strip().endswith(b":")]
        if labels and rng.random() < 0.5:
            lines.insert(rng.choice(ins), lines[rng.choice(labels)])
        else:
            lines.insert(rng.choice(ins), b"    s_branch .Lnowhere")
    elif kind == 9 and ins:  # an extra operand
        i = rng.choice(ins)
        lines[i] = lines[i] + b", v1"
    elif kind == 10:  # a configuration value changed
        cfg = [i for i, l in enumerate(lines) if l.strip().startswith((b".cws", b".sgprsnum", b".vgprsnum", b".dims", b"dims"))]
        if cfg:
            i = rng.choice(cfg)
            key = lines[i].split()[0]
            lines[i] = b"    " + key + b" " + rng.choice([b"0", b"1", b"1025", b"xyz", b"", b"64, 0, 1", b"3", b"x"])
    elif kind == 11:  # no end of program
        lines = [l for l in lines if l.strip() != b"s_endpgm"]
    elif kind == 12 and ins:  # a constant offset on a memory access
        mem = [i for i in ins if re.search(rb"(global|flat|ds)_", lines[i])]
        if mem:
            i = rng.choice(mem)
            lines[i] = lines[i] + rng.choice([b" offset:8", b" offset:0", b" offset:-4", b" offset:x"])
    elif kind == 13:  # CRLF line endings
        lines = [l + b"\r" if l else l for l in lines]
    elif kind == 14:  # comment lines
        lines.insert(rng.randrange(len(lines) + 1), rng.choice([b"# note", b"; note", b"// note", b"    ; indented"]))
    elif kind == 15 and ins:  # tabs and trailing blanks
        i = rng.choice(ins)
        lines[i] = lines[i].replace(b" ", b"\t", 1) + b"  \t"
    elif kind == 16:  # the file ends in the middle of a line
        joined = b"\n".join(lines)
        return joined[: rng.randrange(len(joined) + 1)]
    elif kind == 17 and ins:  # a second kernel directive in the middle
        lines.insert(rng.choice(ins), b".kernel second")
    return b"\n".join(lines)


def mutants(texts, n, seed):
    """n damaged files made from the given kernel texts, one to three kinds of damage each."""
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        t = texts[rng.randrange(len(texts))]
        for _ in range(rng.randint(1, 3)):
            t = _mutate_once(rng, t)
        out.append(t)
    return out
