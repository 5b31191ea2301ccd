"""Host-side pieces of bench.py that need no GPU: the source hash that keeps
a committed DRAM-traffic record tied to the code it was measured on, and the
choice of the dominant kernel class from the library's timers."""
import os
from types import SimpleNamespace

import bench


def test_code_hash_ignores_comments_and_spacing(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "a.cu").write_text("int f(int x) {\n    return x + 1;  // one more\n}\n/* note */\n")
    (tmp_path / "b.cu").write_text("/* reworded\n   note */ int  f(int x) { return x + 1; }\n\n")
    (tmp_path / "c.cu").write_text("int f(int x) {\n    return x + 2;  // one more\n}\n")
    assert bench.code_sha256(["a.cu"]) == bench.code_sha256(["b.cu"])
    assert bench.code_sha256(["a.cu"]) != bench.code_sha256(["c.cu"])
    # file boundaries count: two files are not their concatenation
    (tmp_path / "d.cu").write_text("int g;")
    (tmp_path / "e.cu").write_text("int f(int x) { return x + 1; } int g;")
    assert bench.code_sha256(["a.cu", "d.cu"]) != bench.code_sha256(["e.cu"])


def test_traffic_records_name_existing_sources():
    prof = os.path.join(bench.ROOT, "profiles")
    for name in os.listdir(prof):
        if not name.endswith(".traffic.txt"):
            continue
        rec, srcs = {}, []
        for line in open(os.path.join(prof, name)):
            if line.startswith("# valid while these sources hash"):
                srcs = line.split(":", 1)[1].split()
            elif ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        assert srcs and all(os.path.exists(os.path.join(bench.ROOT, s)) for s in srcs), name
        assert int(rec["dram_bytes_per_launch"]) > 0 and len(rec["sources_sha256"]) == 64, name


def test_dominant_class_skips_stream_spans():
    # a frame step's timers: the record pass beside the cache pass spans about as long as it
    timing = {"path_trace": (1.3, 2), "cache": (2.79, 1), "train_records": (2.80, 1), "train_fwd": (0.15, 1),
              "train_bwd": (0.0, 0), "train_gradw": (1.06, 1), "adam": (0.10, 7), "query": (9.0, 0)}
    piped = SimpleNamespace(overlap_records=1, pipeline_trace=1)
    assert bench.dominant_class(timing, piped) == "cache"
    serial = SimpleNamespace(overlap_records=0, pipeline_trace=0)
    assert bench.dominant_class(timing, serial) == "train_records"  # on one stream a span is device time
    # classes that launched nothing never count
    assert bench.dominant_class({"cache": (1.0, 1), "query": (5.0, 0)}, serial) == "cache"
