"""The ctypes binding agrees with include/msp.h, on the CPU.

A mismatch between the header and ``msp.py`` (a struct field out of order,
a wrong width, a renumbered option or status) would silently corrupt what
the binding reads, so the header text is parsed here and compared with the
binding's constants and ``Stats`` layout.
"""
import ctypes
import os
import re

from paper_2507_05045_gb300 import msp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = open(os.path.join(ROOT, "include", "msp.h")).read()
CODE = re.sub(r"/\*.*?\*/", "", HEADER, flags=re.S)  # comments out


def enum_values(prefix):
    return {name: int(v) for name, v in re.findall(rf"\b({prefix}\w*)\s*=\s*(-?\d+)", CODE)}


def test_status_codes():
    want = {v: k for k, v in enum_values("MSP_E").items()}
    want.update({v: k for k, v in enum_values("MSP_OK").items()})
    want.update({v: k for k, v in enum_values("MSP_PENDING").items()})
    assert msp.STATUS == want


def test_option_codes():
    opts = enum_values("MSP_OPT_")
    assert msp.OPT_EXACT_PATH == opts["MSP_OPT_EXACT_PATH"]
    assert msp.OPT_CLASS_PART == opts["MSP_OPT_CLASS_PART"]
    assert msp.OPT_CLASS_PARTS == opts["MSP_OPT_CLASS_PARTS"]
    assert msp.OPT_FIRST == opts["MSP_OPT_FIRST"]
    assert msp.OPT_WAIT_LIMIT_US == opts["MSP_OPT_WAIT_LIMIT_US"]
    assert msp.OPT_WAIT_CHECK == opts["MSP_OPT_WAIT_CHECK"]
    for key, code in msp.PLAN_KEYS.items():
        assert opts["MSP_OPT_" + key.upper()] == code
    # exact path, part, parts, first, wait limit, wait check
    assert len(opts) == len(msp.PLAN_KEYS) + 6


def test_kernel_kinds_in_index_order():
    kinds = enum_values("MSP_K_")
    by_index = sorted(kinds.items(), key=lambda kv: kv[1])
    assert [v for _, v in by_index] == list(range(len(by_index)))
    assert tuple(name[len("MSP_K_"):].lower() for name, _ in by_index) == msp.Stats.KINDS


CTYPES = {"int": ctypes.c_int, "uint64_t": ctypes.c_uint64, "double": ctypes.c_double}


def header_stats_fields():
    body = re.search(r"typedef struct \{(.*?)\}\s*msp_stats;", CODE, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        for nm in names.split(","):
            nm = nm.strip()
            m = re.fullmatch(r"(\w+)\[(\d+)\]", nm)
            if m:
                fields.append((m.group(1), CTYPES[ctype] * int(m.group(2))))
            else:
                fields.append((nm, CTYPES[ctype]))
    return fields


def test_stats_struct_layout():
    want = header_stats_fields()
    got = msp.Stats._fields_
    assert [n for n, _ in got] == [n for n, _ in want]
    for (n, t), (_, u) in zip(got, want):
        assert ctypes.sizeof(t) == ctypes.sizeof(u), n
        assert getattr(t, "_type_", t) == getattr(u, "_type_", u), n
        assert getattr(t, "_length_", 1) == getattr(u, "_length_", 1), n
    assert len(msp.Stats.KINDS) == msp.Stats.kernel_ms.size // ctypes.sizeof(ctypes.c_double)
