"""Byte counts of the device-memory budget ($MSP_MEMORY_BUDGET), on the CPU."""
import pytest

from paper_2507_05045_gb300 import msp


@pytest.mark.parametrize("text,want", [
    ("4096", 4096), ("0", 0), ("1K", 1024), ("1500M", 1500 << 20), ("1500MB", 1500 << 20),
    ("150G", 150 << 30), ("150g", 150 << 30), (" 2T ", 2 << 40), ("0.5G", 1 << 29), ("64kb", 64 << 10),
])
def test_parse_bytes(text, want):
    assert msp.parse_bytes(text) == want


@pytest.mark.parametrize("text", ["", "G", "abc", "-1G", "1.5X", "nan", "inf", "1e30", "12 GB extra"])
def test_parse_bytes_rejects(text):
    with pytest.raises(msp.MspError):
        msp.parse_bytes(text)


def test_default_budget_from_environment(monkeypatch):
    monkeypatch.delenv(msp.BUDGET_ENV, raising=False)
    assert msp.default_budget() == 0
    monkeypatch.setenv(msp.BUDGET_ENV, "")
    assert msp.default_budget() == 0
    monkeypatch.setenv(msp.BUDGET_ENV, "150G")
    assert msp.default_budget() == 150 << 30
    monkeypatch.setenv(msp.BUDGET_ENV, "lots")
    with pytest.raises(msp.MspError):
        msp.default_budget()
