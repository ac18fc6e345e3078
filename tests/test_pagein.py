"""The serving warm-up's page-in of the process's mapped files (host only)."""
import mmap
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _mapped_regular_files():
    out = set()
    for line in open("/proc/self/maps"):
        parts = line.split()
        if len(parts) >= 6 and parts[5].startswith("/") and os.path.isfile(parts[5]):
            out.add(parts[5])
    return out


@pytest.mark.skipif(not os.path.exists("/proc/self/maps"), reason="needs /proc")
@pytest.mark.timeout(60)
def test_page_in_reads_the_mapped_files_once_and_skips_devices(monkeypatch):
    from paper_1712_09407_gb300 import serving
    monkeypatch.setattr(serving, "_PAGED_IN", False)
    # a device mapping that would read without end (the GPU driver maps its device files too)
    fd = os.open("/dev/zero", os.O_RDONLY)
    m = mmap.mmap(fd, 1 << 20, mmap.MAP_PRIVATE, mmap.PROT_READ)
    try:
        assert any("/dev/zero" in l for l in open("/proc/self/maps"))
        expect = sum(os.path.getsize(f) for f in _mapped_regular_files())
        got = serving.page_in_mapped_files()
        # every mapped regular file is read whole, once; files mapped after the listing only add
        assert got >= expect > 0
        assert serving.page_in_mapped_files() == 0
    finally:
        m.close()
        os.close(fd)
