"""The serving warm-up's page-in of the process's mapped files (host only)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.skipif(not os.path.exists("/proc/self/maps"), reason="needs /proc")
def test_page_in_reads_the_mapped_files_once(monkeypatch):
    from paper_1712_09407_gb300 import serving
    monkeypatch.setattr(serving, "_PAGED_IN", False)
    mapped = set()
    for line in open("/proc/self/maps"):
        parts = line.split()
        if len(parts) >= 6 and parts[5].startswith("/") and os.path.isfile(parts[5]):
            mapped.add(parts[5])
    expect = sum(os.path.getsize(f) for f in mapped)
    got = serving.page_in_mapped_files()
    # every mapped file is read whole (files mapped after the listing above only add to it)
    assert got >= expect > 0
    assert serving.page_in_mapped_files() == 0
