"""The launch-shape autotuner's host side (no GPU): its cache round-trips,
its shape buckets follow the library's TAM classes, and the header's tuning
struct matches the binding's layout."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def relo():
    from paper_2511_01219_gb300 import _build
    _build.build()
    import paper_2511_01219_gb300 as relo
    relo.lib()
    return relo


def test_cache_round_trip(relo, tmp_path):
    from paper_2511_01219_gb300 import autotune
    entries = [(relo.TUNE_TAM, (34, 360, 256), (16, 4)), (relo.TUNE_CAST, (1440, 0, 0), (5, 0)),
               (relo.TUNE_TAM_ONE, (46, 720, 1024), (48, 4))]
    path = str(tmp_path / "t" / "dev.json")
    autotune.save(path, entries, {"device": "test"})
    assert autotune.load(path) == entries
    assert autotune.load(str(tmp_path / "missing.json")) == []
    assert autotune.cache_path("NVIDIA GB300").endswith(os.path.join("tuning", "NVIDIA_GB300.json"))


def test_buckets_follow_the_tam_classes(relo):
    from paper_2511_01219_gb300 import autotune
    # values per lane: ceil(n / 32) rounded up to even, at least 8
    assert [relo.tam_class(n) for n in (1, 256, 257, 1081, 1440, 2048)] == [8, 8, 10, 34, 46, 64]
    assert relo.tam_class(2049) == -1 and relo.tam_class(0) == -1
    b = autotune.buckets([(1081, 360, 256), (1081, 360, 256), (1440, 720, 1024), (541, 360, 256)])
    assert b == [(18, 360, 256), (34, 360, 256), (46, 720, 1024)]


def test_tune_entry_layout_matches_header(relo, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "relo.h"\n'
                   "int main(void){printf(\"%zu %zu %zu\\n\", sizeof(relo_tune_entry),"
                   " offsetof(relo_tune_entry, key), offsetof(relo_tune_entry, val)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    E = relo.TuneEntry
    assert got == [ctypes.sizeof(E), E.key.offset, E.val.offset]
