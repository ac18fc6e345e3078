"""The oracle and its stage pieces under AddressSanitizer and UndefinedBehaviorSanitizer (host only):
a driver built with -fsanitize=address,undefined runs the float and double tracker with and
without global tracking and the merger on a small 36-sector event and on an empty one."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1712_09407_gb300 import eventgen

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")


def _dump(path, ev_y, ev_z, row, counts, row_x, n_sectors):
    with open(path, "wb") as f:
        f.write(np.int64(len(ev_y)).tobytes())
        f.write(np.int32(len(row_x)).tobytes())
        f.write(np.int32(n_sectors).tobytes())
        f.write(np.asarray(row_x, np.float64).tobytes())
        f.write(np.asarray(ev_y, np.float64).tobytes())
        f.write(np.asarray(ev_z, np.float64).tobytes())
        f.write(np.asarray(row, np.uint8).tobytes())
        f.write(np.asarray(counts, np.int32).tobytes())


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    d = tmp_path_factory.mktemp("asan")
    exe = str(d / "oracle_driver")
    flags = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
             "-fno-omit-frame-pointer", "-ffp-contract=off", "-std=c11", "-fopenmp", "-I", ORACLE]
    objs = []
    for src, extra, obj in [("common.c", [], "common.o"), ("tracker.c", [], "t64.o"), ("tracker.c", ["-DORC_F32"], "t32.o")]:
        o = str(d / obj)
        subprocess.check_call(["gcc", *flags, *extra, "-c", os.path.join(ORACLE, src), "-o", o])
        objs.append(o)
    subprocess.check_call(["gcc", *flags, os.path.join(HERE, "native", "oracle_driver.c"), *objs, "-o", exe, "-lm"])
    return exe, d


def _run(exe, path):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    p = subprocess.run([exe, path], capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    assert "runtime error" not in p.stderr and "AddressSanitizer" not in p.stderr, p.stderr[-3000:]
    return p.stdout


def test_oracle_clean_under_sanitizers(driver):
    exe, d = driver
    spec = eventgen.EventSpec(n_primaries=150, n_secondaries=20, pt_cut=0.08, noise_frac=0.1)
    ev = eventgen.generate_event(spec, eventgen.Geometry(), seed=4)
    path = str(d / "ev.bin")
    _dump(path, ev.y, ev.z, ev.row, ev.counts, ev.geometry.row_x, 36)
    out = _run(exe, path)
    assert out.count("tracks") == 8


def test_empty_event_clean_under_sanitizers(driver):
    exe, d = driver
    geo = eventgen.Geometry()
    path = str(d / "empty.bin")
    _dump(path, np.zeros(0), np.zeros(0), np.zeros(0, np.uint8), np.zeros(36 * geo.n_rows, np.int32), geo.row_x, 36)
    out = _run(exe, path)
    assert "tracks 0 merged 0" in out
