"""Host-side logic of bench.py: the DRAM traffic figure of a kernel is taken from the
committed ncu summary only while the kernel's source files are the ones captured."""
import hashlib
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tree(tmp_path, files):
    csrc = tmp_path / "paper_1105_3505_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in files.items():
        (csrc / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    return csrc


def _hash(csrc, names):
    h = hashlib.sha256()
    for n in names:
        h.update((csrc / n).read_bytes())
    return h.hexdigest()[:16]


def test_traffic_follows_the_source_hash(tmp_path):
    bench = _bench()
    csrc = _tree(tmp_path, {"k.cu": "kernel v1", "common.h": "helpers v1", "other.cu": "x"})
    entries = {
        "_note": "test",
        "multi": {"source": ["k.cu", "common.h"], "source_sha256_16": _hash(csrc, ["k.cu", "common.h"]),
                  "bytes_per_launch": 123},
        "single": {"source": "other.cu", "source_sha256_16": _hash(csrc, ["other.cu"]), "bytes_per_launch": 7},
    }
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entries))
    bench.ROOT = str(tmp_path)
    assert bench.traffic_for("multi") == 123
    assert bench.traffic_for("single") == 7
    assert bench.traffic_for("absent") is None
    (csrc / "common.h").write_text("helpers v2")  # a header the kernel includes changed
    assert bench.traffic_for("multi") is None
    assert bench.traffic_for("single") == 7


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    for kernel, e in d.items():
        if kernel.startswith("_"):
            continue
        names = e["source"] if isinstance(e["source"], list) else [e["source"]]
        for n in names:
            assert os.path.exists(os.path.join(ROOT, "paper_1105_3505_gb300", "csrc", n)), (kernel, n)
        assert e["bytes_per_launch"] > 0
