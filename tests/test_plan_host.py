"""msp_plan: the default plan of an (m, n) instance, computed on the host.

The expected plans follow the formulas of the two passes: the direct pass
splits each half into an outer quarter of at most 9 columns and an inner
quarter of B + 4 columns, B = max(0, log2 |half| - 13), whenever both halves
have at most 40 columns; otherwise the streaming pass takes
B = min(23, log2 |half| - 21) classes (log2 |half| - 21 for halves of 44 to
47 columns, min(27, log2 |half| - 20) for halves of 48 or more), inner
quarters of B + 4 columns (B + 5 for halves of 44 to 47 columns; at most 27,
or 30 past 2^23 classes or for halves of 44 columns or more) and
D = min(12, log2 |half| - B - 12) digit bits.
"""
import ctypes

import pytest

import paper_2507_05045_gb300 as msp


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2507_05045_gb300 import build
    build.build()


def test_headline_shapes():
    p = msp.plan_info(9, 80)
    assert (p["path"], p["class_bits"], p["class_rows"], p["quarter"], p["table_bits"]) == \
        ("direct", 27, 4, [9, 9, 31, 31], 14)
    assert p["records_left"] == p["records_right"] == 1 << 40
    # inner lists of 2 x 2^31 keys and masks, plus offsets and scratch
    assert 2 * (1 << 31) * 8 < p["device_bytes"] < 60 << 30

    p = msp.plan_info(10, 90)
    assert (p["path"], p["class_bits"], p["class_rows"], p["quarter"], p["digit_bits"]) == \
        ("streaming", 24, 4, [16, 16, 29, 29], 9)
    assert p["records_left"] == p["records_right"] == 1 << 45

    p = msp.plan_info(4, 30)
    assert (p["path"], p["class_bits"], p["class_rows"], p["quarter"]) == ("direct", 2, 1, [9, 9, 6, 6])


@pytest.mark.parametrize("m", [1, 3, 9, 16])
def test_every_shape(m):
    for n in range(1, 101):
        p = msp.plan_info(m, n)
        q = p["quarter"]
        assert sum(q) == n
        assert p["records_left"] == 1 << (q[0] + q[2]) and p["records_right"] == 1 << (q[1] + q[3])
        assert 1 <= p["class_rows"] <= m
        half = (n + 1) // 2
        if 2 <= n and half <= 40:
            B = max(0, half - 13)
            assert p["path"] == "direct" and p["class_bits"] == B
            for s, cols in ((0, half), (1, n - half)):
                qi = min(cols, B + 4)
                qo = cols - qi
                if qo > 9:
                    qo, qi = 9, cols - 9
                assert (q[s], q[s + 2]) == (qo, qi)
        else:
            assert p["path"] == "streaming"
            lg = max(q[0] + q[2], q[1] + q[3])
            B = min(23, max(0, lg - 21))
            if lg >= 44:
                B = min(27, lg - 20 if lg >= 48 else lg - 21)
            assert p["class_bits"] == B
            assert p["digit_bits"] == min(12, max(0, lg - B - 12))
            cap = 30 if B > 23 or lg >= 44 else 27
            assert max(q[2], q[3]) <= cap
            for s in (0, 1):
                tot = q[s] + q[s + 2]
                target = B + (5 if 44 <= lg < 48 else 4)
                assert q[s + 2] == max(n // 4 + (s + 2 < n % 4), min(target, cap, tot - 1))


@pytest.mark.parametrize("m,n", [(0, 30), (17, 30), (4, 0), (4, 101)])
def test_out_of_range(m, n):
    with pytest.raises(msp.MspError) as e:
        msp.plan_info(m, n)
    assert e.value.code == -2


def test_null_output_is_rejected():
    lib = msp.load_library()
    assert lib.msp_plan(4, 30, ctypes.POINTER(msp.msp.PlanInfo)()) == -1


def test_large_plans_fit_the_device():
    # the streaming plans of the largest shapes keep their lists and per-class
    # tables well inside a GB300's memory, leaving room for the pass buffers
    for m, n, B, inner in [(10, 90, 24, 29), (11, 100, 27, 30)]:
        p = msp.plan_info(m, n)
        assert p["path"] == "streaming" and p["class_bits"] == B
        assert max(p["quarter"][2], p["quarter"][3]) == inner
        assert p["digit_bits"] == max(0, (max(p["quarter"][0] + p["quarter"][2],
                                               p["quarter"][1] + p["quarter"][3])) - B - 12)
        assert p["device_bytes"] < 150 << 30
