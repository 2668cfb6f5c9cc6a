"""The bench's traffic records (no GPU): a record holds for a kernel only
while neither its source file nor any library header it includes changed."""
import json
import os

import bench


def _tree(tmp_path, files):
    csrc = tmp_path / "paper_1302_4332_b300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in files.items():
        (csrc / name).write_text(text)
    return csrc


def test_digest_follows_included_headers(tmp_path, monkeypatch):
    csrc = _tree(tmp_path, {
        "k.cu": '#include "a.cuh"\n#include <cuda.h>\n__global__ void k() {}\n',
        "a.cuh": '#include "b.cuh"\nint a;\n',
        "b.cuh": "int b;\n",
        "other.cuh": "int unrelated;\n",
    })
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest("k.cu")
    (csrc / "other.cuh").write_text("int unrelated = 1;\n")  # not included: no change
    assert bench.source_digest("k.cu") == d0
    (csrc / "b.cuh").write_text("int b = 2;\n")  # included through a.cuh
    d1 = bench.source_digest("k.cu")
    assert d1 != d0
    (csrc / "k.cu").write_text('#include "a.cuh"\n#include <cuda.h>\n__global__ void k() { }\n')
    assert bench.source_digest("k.cu") not in (d0, d1)


def test_kernel_traffic_only_for_the_recorded_source(tmp_path, monkeypatch):
    _tree(tmp_path, {"k.cu": '#include "a.cuh"\n', "a.cuh": "int a;\n"})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    rec = {"p/t": {"source": "k.cu", "sha256_16": bench.source_digest("k.cu"), "dram_bytes": 123}}
    (tmp_path / "profiles" / "traffic_per_launch.json").write_text(json.dumps(rec))
    assert bench.kernel_traffic("p", "t") == 123
    assert bench.kernel_traffic("p", "other") is None
    (tmp_path / "paper_1302_4332_b300" / "csrc" / "a.cuh").write_text("int a = 1;\n")
    assert bench.kernel_traffic("p", "t") is None


def test_committed_records_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic_per_launch.json")) as f:
        recs = json.load(f)
    for key, rec in recs.items():
        assert os.path.exists(os.path.join(bench.ROOT, "paper_1302_4332_b300", "csrc", rec["source"])), key
        assert rec["dram_bytes"] > 0 and len(rec["sha256_16"]) == 16, key
        assert "--clock-control none" in rec["command"], key
