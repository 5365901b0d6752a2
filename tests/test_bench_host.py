"""Host logic of bench.py that needs no GPU: the kernel-source hash that
decides whether a committed DRAM-traffic capture still describes the kernel
(comments and blank lines do not count, code does), the traffic lookup
that reports nothing once the hash no longer matches, and the achieved phase
fractions reported with the tissue workload."""
import json
import os

import numpy as np

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
    rec = {"source_hash": bench.sweep_source_hash(),
           "by_form": {"z-marching": {"bytes_per_site_member": 113.5}, "staged": {"bytes_per_site_member": 120.0}}}
    with open(os.path.join(root, "profiles", "sweep_traffic.json"), "w") as fh:
        json.dump(rec, fh)
    n = bench.N_EDGE ** 3 * 3
    assert bench.traffic_per_launch(n, "staged") == 120.0 * n
    assert bench.traffic_per_launch(n, "z-marching") == 113.5 * n
    assert bench.traffic_per_launch(n, "prefetched") is None    # not captured
    (tmp_path / "paper_1907_00908_gb300" / "csrc" / "sweep_tma.cu").write_text(SRC.replace("1.f", "3.f"))
    assert bench.traffic_per_launch(1000, "staged") is None


def test_phase_fractions_of_a_known_geometry():
    from paper_1907_00908_gb300 import synth
    lab = np.zeros((2, 4, 5), np.int32)
    lab[:, :, :2] = 1                      # label 1: 16 of 40 sites
    lab[0, 0, 4] = 2                       # label 2: 1 site, same phase as label 0
    g = synth.Geometry(lab, np.array([0, 1, 0], np.uint8), 0.5)
    assert bench.phase_fractions(g) == [0.6, 0.4]


def test_tissue_fractions_follow_the_recipe():
    """The tissue's extracellular band (phase 1) is the 0.2 quantile of
    d2 - d1 over all sites, and the vessel tubes (phase 2) then overwrite
    sites regardless of the band, so the band keeps about 0.2 of what the
    vessels leave (128^3, same recipe as the 512^3 workload)."""
    fr = bench.phase_fractions(bench.geometry(128))
    assert len(fr) == 3 and abs(sum(fr) - 1.0) < 1e-4, fr
    assert abs(fr[1] - 0.2 * (1.0 - fr[2])) < 0.01, fr
    assert 0.0 < fr[2] < 0.2 and fr[0] > 0.6, fr


def test_clock_samplers_keep_their_own_records():
    """Regions timed one after another in one process each get their own
    nvidia-smi record, so a line's clocks are those of its own region."""
    a, b = bench.Clocks(0), bench.Clocks(0)
    assert a.path != b.path
