"""Host logic of bench.py that needs no GPU: the kernel-source hash that
decides whether a committed DRAM-traffic capture still describes the kernel
(comments and blank lines do not count, code does), and the traffic lookup
that reports nothing once the hash no longer matches."""
import json
import os

import bench

SRC = """// header comment
#include "x.cuh"

/* block
   comment */
__global__ void k(float* a)   // trailing
{
    a[threadIdx.x] += 1.f;
}
"""


def _tree(tmp_path, files):
    d = tmp_path / "paper_1907_00908_gb300" / "csrc"
    d.mkdir(parents=True, exist_ok=True)
    for name, text in files.items():
        (d / name).write_text(text)
    return str(tmp_path)


def test_code_hash_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "a", {"k.cu": SRC}))
    h0 = bench._code_hash(["k.cu"])
    edited = SRC.replace("// header comment", "// another header\n\n// two lines").replace("// trailing", "")
    edited = edited.replace("/* block\n   comment */", "/* reworded */") + "\n\n"
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "b", {"k.cu": edited}))
    assert bench._code_hash(["k.cu"]) == h0


def test_code_hash_sees_code_changes(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "a", {"k.cu": SRC}))
    h0 = bench._code_hash(["k.cu"])
    for change in (("+= 1.f", "+= 2.f"), ("threadIdx.x", "threadIdx.y"), ("float*", "double*")):
        monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / change[1].replace("*", "p"),
                                                 {"k.cu": SRC.replace(*change)}))
        assert bench._code_hash(["k.cu"]) != h0, change


def test_traffic_lookup_follows_the_hash(tmp_path, monkeypatch):
    files = {f: SRC for f in ("sweep_tma.cu", "sweep_common.cuh", "tma_common.cuh", "lbmbt_internal.cuh")}
    root = _tree(tmp_path, files)
    monkeypatch.setattr(bench, "ROOT", root)
    os.makedirs(os.path.join(root, "profiles"))
    rec = {"source_hash": bench.sweep_source_hash(), "bytes_per_site_member": 120.0}
    with open(os.path.join(root, "profiles", "sweep_traffic.json"), "w") as fh:
        json.dump(rec, fh)
    assert bench.traffic_per_launch() == 120.0 * bench.N_EDGE ** 3 * 3
    (tmp_path / "paper_1907_00908_gb300" / "csrc" / "sweep_tma.cu").write_text(SRC.replace("1.f", "3.f"))
    assert bench.traffic_per_launch() is None
