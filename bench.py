"""Benchmark of the fused hybrid-LBM Bloch-Torrey sweep on GB300.

Workload (large tissue model): 512^3 lattice, dx = 0.25 um, seeded Voronoi
cell tessellation (mean cell diameter 10 um) with ~20 % extracellular band and
4 vessel tubes, 3 phases (cells D = 1.0, extracellular D = 2.5, vessels
D = 3.0 um^2/ms; T2 50/80/80 ms), permeable membranes on every compartment
boundary (kappa = 0.01 um/ms), mirroring outer boundaries, PGSE b = 1000
s/mm^2, delta = 10 ms, Delta = 30 ms, dt = 0.0015625 ms, three orthogonal
gradient directions run as one batch (one launch per time step).

A "step" is one time step of the whole batch: every site of the lattice
updated once for each of the 3 directions.  value = MLUPS = sites x members x
steps / s.  Inputs (15 GB of state per direction) are far larger than L2.

The same JSON line carries, each timed on its own on the same GPU, the
forms the metric compares: ``plain_single_direction`` (one member on the
128^3 permeable cylinders), ``batched`` (528 members on 17 geometries, one
launch per step), ``adjoint`` (the gradient of S for 60 members of a 96^3
sphere pack over a 400-step prefix of its schedule, against a forward run)
and ``adjoint_full_schedule`` (the same over all 6400 steps, with the
member groups the checkpoints needed).

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "tissue512_voronoi_mirror_3dir"
N_EDGE = 512
DX = 0.25
DT = 0.0015625
B = 1000.0
DELTA, BIG_DELTA = 10.0, 30.0
D = [1.0, 2.5, 3.0]
T2 = [50.0, 80.0, 80.0]
KAPPA = 0.01
BYTES_PER_SITE = 113  # 7 complex64 read + 7 written + 1 mask byte (algorithmic)
METRIC = "MLUPS (fused sweep, FP32, 3-direction batch)"


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


TISSUE_SEED = 2024


def phase_fractions(geom):
    """Achieved (voxelised) volume fraction of each phase of a geometry."""
    counts = np.bincount(np.asarray(geom.phase_of_label)[geom.labels.ravel()],
                         minlength=int(np.max(geom.phase_of_label)) + 1)
    return [round(float(c) / geom.labels.size, 5) for c in counts]


def geometry(n=N_EDGE, seed=TISSUE_SEED):
    from paper_1907_00908_gb300 import synth
    return synth.voronoi_tissue(n, DX, cell_diam=10.0, ecs_fraction=0.2, n_vessels=4, vessel_radius=3.0, seed=seed)


def sequences():
    from paper_1907_00908_gb300 import lbmbt
    out = []
    for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        gG, f = lbmbt.pgse(B, DELTA, BIG_DELTA, DT, d)
        out.append((gG, f))
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_hash(files):
    """Hash of the sources' code: comments, blank lines and trailing blanks
    left out, so an edit of a comment keeps a capture valid."""
    h = hashlib.sha256()
    for f in files:
        text = open(os.path.join(ROOT, "paper_1907_00908_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def sweep_source_hash():
    return _code_hash(("sweep_tma.cu", "sweep_common.cuh", "tma_common.cuh", "lbmbt_internal.cuh"))


def links_source_hash():
    return _code_hash(("sweep.cu", "links.cuh", "sweep_common.cuh", "lbmbt_internal.cuh"))


def links_traffic_per_launch(n):
    """DRAM bytes per launch of the membrane-position sweep on the n^3
    cylinders (3 members) from the committed ncu summary, or None when the
    kernel source changed since, or the capture was of another size."""
    p = os.path.join(ROOT, "profiles", "links_traffic.json")
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    if j.get("source_hash") != links_source_hash() or j.get("n") != n:
        return None
    return j["dram_bytes_read"] + j["dram_bytes_write"]


def traffic_per_launch(site_updates, form):
    """DRAM bytes per sweep launch of `site_updates` site-member updates in
    the own-z form `form` ("z-marching", "staged", "prefetched"), from the
    bytes per update in the committed ncu summary, or None when the kernel
    source changed since it was captured or the form was not captured."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    if j.get("source_hash") != sweep_source_hash():
        return None
    f = j.get("by_form", {}).get(form)
    return None if f is None else float(f["bytes_per_site_member"]) * site_updates


class Clocks:
    """nvidia-smi sampler running during the timed region (one file per
    sampler, so regions timed one after the other keep their own records)."""

    _count = 0

    def __init__(self, index):
        self.index = index
        self.proc = None
        Clocks._count += 1
        self.path = f"/tmp/lbmbt_clocks_{os.getpid()}_{Clocks._count}.csv"

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(geom, seqs, steps=24):
    """The FP64 oracle on a 128^3 corner crop of the same tissue, the first
    `steps` steps of each of the 3 PGSE sequences, all host cores."""
    import oracle
    from paper_1907_00908_gb300 import synth
    crop = synth.crop(geom, 128)
    cores = os.cpu_count() or 1
    oracle.build()
    t0 = time.perf_counter()
    for gG, f in seqs:
        oracle.run(crop.labels, DX, crop.phase_of_label, [1, 1, 1], D, T2, KAPPA, DT, f[:steps], gG, threads=cores)
    t = time.perf_counter() - t0
    sites = crop.n_sites * len(seqs) * steps
    # one core, on a 64^3 crop (an eighth of the work)
    small = synth.crop(geom, 64)
    t1 = time.perf_counter()
    for gG, f in seqs:
        oracle.run(small.labels, DX, small.phase_of_label, [1, 1, 1], D, T2, KAPPA, DT, f[:steps], gG, threads=1)
    t1 = time.perf_counter() - t1
    return {"value": sites / t / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"128^3 corner crop of the tissue, {steps} steps x 3 directions, FP64, {t:.1f} s",
            "single_core": {"value": small.n_sites * len(seqs) * steps / t1 / 1e6, "unit": "MLUPS", "cores": 1,
                            "sample": f"64^3 corner crop, {steps} steps x 3 directions, FP64, {t1:.1f} s"}}


def run_reference(args):
    rank, world, _ = _rank()
    if rank != 0:
        return 0
    import oracle
    from paper_1907_00908_gb300 import synth
    oracle.build()
    geom = synth.crop(geometry(), 128)
    from oracle import pgse
    seqs = [pgse(B, DELTA, BIG_DELTA, DT, d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    cores = os.cpu_count() or 1
    per_step = 24   # lattice steps per oracle call, as in the cpu_baseline leg (set-up amortised)

    def one():
        for gG, f in seqs:
            oracle.run(geom.labels, DX, geom.phase_of_label, [1, 1, 1], D, T2, KAPPA, DT, f[:per_step], gG,
                       threads=cores)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    t = time.perf_counter() - t0
    sites = geom.n_sites * 3 * per_step * args.steps
    v = sites / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"128^3 crop, {per_step} lattice steps x 3 directions per "
                                                      "step"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"128^3 corner crop of the 512^3 tissue, {per_step} lattice steps x 3 "
                                       "directions per bench step"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- batched (c3)
C2_D, C2_T2, C2_KAPPA = [2.0, 1.0], [80.0, 50.0], 0.02   # phase 0 extracellular, 1 intracellular
C2_DT, C2_DELTA, C2_BIG_DELTA = 0.00625, 10.0, 30.0


def batch_workload(seed=7):
    """64 directions x 8 b-values on one 128^3 cylinder pack (dx 0.5 um) plus
    16 sphere packs of uneven edges (multiples of 16 in 48..160, radii
    U(2, 6) um, fraction 0.5, kappa U(0, 0.05) um/ms), one member each."""
    from paper_1907_00908_gb300 import lbmbt, synth
    rng = np.random.Generator(np.random.PCG64(seed))
    cyl = synth.cylinders(128, 0.5, seed=1)
    dirs = synth.directions_on_sphere(64, seed=seed)
    bvals = np.linspace(0.0, 3000.0, 8)
    members = []
    for d in dirs:
        for b in bvals:
            gG, _ = lbmbt.pgse(float(b), C2_DELTA, C2_BIG_DELTA, C2_DT, d)
            members.append((gG, 0, C2_KAPPA))
    sizes = rng.choice(np.arange(48, 161, 16), size=16)
    packs = []
    for j, n in enumerate(sizes):
        g = synth.spheres(int(n), 0.5, rmin=2.0, rmax=6.0, fraction=0.5, seed=100 + j)
        packs.append(g)
        gG, _ = lbmbt.pgse(float(bvals[j % 8]), C2_DELTA, C2_BIG_DELTA, C2_DT, dirs[j])
        members.append((gG, 1 + j, float(rng.uniform(0.0, 0.05))))
    _, f = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, C2_DT, (1, 0, 0))
    return cyl, packs, members, f


def _timed_advance(solver, stream, members, steps, warmup, want_signal=True):
    """Prepare ``members``, advance ``warmup`` steps, then time ``steps``
    steps with CUDA events on ``stream`` (nvidia-smi sampling around them).
    Returns (ms per step, clocks summary, signals)."""
    import torch
    solver.prepare(members)
    solver.advance(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        sig = solver.advance(steps, want_signal=want_signal, n_members=len(members))
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, clk.summary(), sig


def _launch_shape(s, lbmbt):
    return {"kernel": "bulk-copy" if s.get_option(lbmbt.OPT_KERNEL_USED) == 2 else "register",
            "tma_shape": s.get_option(lbmbt.OPT_TMA_SHAPE), "stages": s.get_option(lbmbt.OPT_STAGES),
            "block": s.get_option(lbmbt.OPT_BLOCK), "spt": s.get_option(lbmbt.OPT_SPT)}


def _hbm_roofline(mlups, bytes_per_site, kernel):
    peak, peak_kind = peaks()
    achieved = mlups * 1e6 * bytes_per_site / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "bytes_per_site_member": bytes_per_site, "kernel": kernel}


PLAIN_C2_STEPS, PLAIN_C2_WARMUP = 4000, 50   # 0.2 s timed: a 56 us step needs many for a stable figure


def measure_plain_c2(args, stream):
    """The plain single-direction sweep on the two-phase permeable-cylinder
    workload: 128^3 at dx 0.5 um, D 2.0/1.0, T2 80/50, kappa 0.02 um/ms,
    PGSE b 1000 s/mm^2 along x, delta 10 / Delta 30 ms, one member,
    autotuned launch, timed over 4000 of its 6400 steps (a step takes
    about 50 us, so a 20-step region is dominated by fixed costs)."""
    from paper_1907_00908_gb300 import lbmbt, synth
    geom = synth.cylinders(128, 0.5, seed=1)
    gG, f = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, C2_DT, (1, 0, 0))
    s = lbmbt.Solver(0, stream)
    s.set_option(lbmbt.OPT_AUTOTUNE, 0 if args.no_autotune else 1)
    s.set_geometry(geom.labels, geom.phase_of_label, 0.5)
    s.set_phases(C2_D, C2_T2)
    s.set_sequence(C2_DT, f, gG)
    ms, clk, _ = _timed_advance(s, stream, lbmbt.Solver.members([gG], 0, C2_KAPPA), PLAIN_C2_STEPS,
                                PLAIN_C2_WARMUP)
    shape = _launch_shape(s, lbmbt)
    s.close()
    v = geom.n_sites / (ms * 1e-3) / 1e6
    return {"value": v, "unit": "MLUPS", "ms_per_step": ms, "steps": PLAIN_C2_STEPS, "warmup": PLAIN_C2_WARMUP,
            "workload": "128^3 permeable cylinders, dx 0.5 um, 1 member (PGSE b 1000 along x)",
            "l2": "state of 235 MB per time level pair, larger than L2; no flush needed",
            "launch": shape, "roofline": _hbm_roofline(v, BYTES_PER_SITE, "sweep (" + shape["kernel"] + ")"),
            "clocks": clk}


def measure_batch(args, stream):
    """The batched workload: 64 directions x 8 b-values on the 128^3
    cylinders plus 16 sphere packs of uneven edges, 528 members in one
    launch per step, autotuned launch."""
    from paper_1907_00908_gb300 import lbmbt
    t0 = time.perf_counter()
    cyl, packs, members, f = batch_workload()
    t_gen = time.perf_counter() - t0
    s = lbmbt.Solver(0, stream)
    s.set_option(lbmbt.OPT_STAGE_OWN_Z, args.stage_own_z)
    s.set_option(lbmbt.OPT_COLUMN_PLANES, args.column_planes)
    s.set_option(lbmbt.OPT_AUTOTUNE, 0 if args.no_autotune else 1)
    s.set_geometry(cyl.labels, cyl.phase_of_label, 0.5)
    for g in packs:
        s.add_geometry(g.labels, g.phase_of_label, 0.5)
    s.set_phases(C2_D, C2_T2)
    s.set_sequence(C2_DT, f, members[0][0])
    mem = lbmbt.Solver.members([m[0] for m in members], [m[1] for m in members], [m[2] for m in members])
    total_sites = float(cyl.n_sites * 512 + sum(g.n_sites for g in packs))
    ms, clk, _ = _timed_advance(s, stream, mem, args.steps, args.warmup)
    shape = _launch_shape(s, lbmbt)
    s.close()
    v = total_sites / (ms * 1e-3) / 1e6
    return {"value": v, "unit": "MLUPS", "ms_per_step": ms, "steps": args.steps,
            "workload": "batch_528: 64 directions x 8 b-values on the 128^3 cylinders + 16 sphere packs "
                        "(edges 48-160, dx 0.5 um, kappa U(0, 0.05) um/ms)",
            "members": len(members), "sites_per_step": total_sites,
            "pack_edges": [int(g.shape[0]) for g in packs], "geometry_gen_s": round(t_gen, 1),
            "launch": shape, "roofline": _hbm_roofline(v, BYTES_PER_SITE, "sweep (" + shape["kernel"] + ")"),
            "clocks": clk}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    b = measure_batch(args, stream)
    p = measure_plain_c2(args, stream)
    line = {"metric": "MLUPS (batched sweep, FP32, 528 members)", "value": b["value"], "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_c3_128cyl_64dirx8b_plus_16_packs", "members": b["members"],
                       "sites_per_step": b["sites_per_step"], "pack_edges": b["pack_edges"],
                       "launch": b["launch"]},
            "plain_single_direction": p, "batched_over_plain": b["value"] / p["value"],
            "roofline": b["roofline"], "clocks": b["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- adjoint (c4)
def adjoint_workload(n_members=60):
    """96^3 two-phase sphere pack (dx 0.5 um, radii U(2, 6) um, fraction
    0.5), 30 seeded directions x b in {1000, 2500} s/mm^2, PGSE delta 10 /
    Delta 30 ms."""
    from paper_1907_00908_gb300 import lbmbt, synth
    geom = synth.spheres(96, 0.5, rmin=2.0, rmax=6.0, fraction=0.5, seed=4)
    dirs = synth.directions_on_sphere(30, seed=11)
    gGs = [lbmbt.pgse(b, C2_DELTA, C2_BIG_DELTA, C2_DT, d)[0] for b in (1000.0, 2500.0) for d in dirs]
    _, f = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, C2_DT, (1, 0, 0))
    return geom, gGs[:n_members], f


def measure_adjoint(args, stream, K=None):
    """Gradient of S with respect to D, T2 and kappa for every member of the
    adjoint workload (forward with checkpoints every 64 steps, recomputed
    segments, reverse sweep), over the first K steps of the 6400-step
    schedule (all of it when K is None), against a forward run of the same
    members and steps.  Both timed with CUDA events on ``stream``.  On a
    prefix the untimed warm-up is the same gradient call, so the checkpoint
    and segment buffers (about 3.6 GB per member at 400 steps) are allocated
    before the timed region; on the full schedule a 2-member warm-up, and the
    first member group's allocation falls in the timed region."""
    import torch
    from paper_1907_00908_gb300 import lbmbt
    geom, gGs, f = adjoint_workload(args.members)
    if K is not None:
        f = f[:K]
    K = len(f)
    s = lbmbt.Solver(0, stream)
    s.set_geometry(geom.labels, geom.phase_of_label, 0.5)
    s.set_phases(C2_D, C2_T2)
    s.set_sequence(C2_DT, f, gGs[0])
    s.set_option(lbmbt.OPT_ADJOINT_SHAPE, args.adj_shape)
    s.set_option(lbmbt.OPT_ADJOINT_KERNEL, args.adjoint_kernel)
    mem = lbmbt.Solver.members(gGs, 0, C2_KAPPA)
    warm = mem if K < 6400 else lbmbt.Solver.members(gGs[:2], 0, C2_KAPPA)
    s.grad_batch(warm, checkpoint_every=64)   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        g = s.grad_batch(mem, checkpoint_every=64)
        e1.record(stream)
        torch.cuda.synchronize()
    t_grad = e0.elapsed_time(e1) * 1e-3
    groups = s.get_option(lbmbt.OPT_GRAD_GROUPS)
    torch.cuda.synchronize()
    e0.record(stream)
    s.run_batch(mem)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) * 1e-3
    s.close()
    work = geom.n_sites * len(gGs) * K
    return {"value": work / t_grad / 1e6, "unit": "MLUPS-equivalent", "seconds": t_grad, "steps": K,
            "ms_per_step": 1e3 * t_grad / K,
            "workload": f"adjoint_60: 96^3 sphere pack, {len(gGs)} members (30 directions x b 1000, 2500), "
                        "checkpoint every 64 steps",
            "members": len(gGs), "member_groups": groups,
            "plain_forward": {"value": work / t_fwd / 1e6, "unit": "MLUPS", "seconds": t_fwd},
            "gradient_over_forward_time": t_grad / t_fwd,
            "sample_gradient_member0": {"S": float(g["S"][0]), "dS_dD": g["dD"][0].tolist(),
                                        "dS_dT2": g["dT2"][0].tolist(), "dS_dkappa": float(g["dkappa"][0])},
            "clocks": clk.summary()}


def run_adjoint(args):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    a = measure_adjoint(args, stream, args.adj_steps)
    line = {"metric": "MLUPS-equivalent (gradient of S wrt D, T2, kappa; forward + checkpointed adjoint)",
            "value": a["value"], "unit": "MLUPS", "n_gpus": 1, "steps": a["steps"], "warmup": 1,
            "ms_per_step": a["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "adjoint_c4_96pack_30dirx2b", "members": a["members"], "checkpoint_every": 64,
                       "steps_of_schedule": a["steps"], "member_groups": a["member_groups"]},
            "plain_forward": a["plain_forward"], "gradient_over_forward_time": a["gradient_over_forward_time"],
            "sample_gradient_member0": a["sample_gradient_member0"], "clocks": a["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- membrane positions
def run_links(args):
    """Membranes at their exact positions on the links (theta = 0 rule,
    Eqs. B4a-B4c, register sweep) against the half-link rule on the same
    grid: z-aligned cylinders (the c2 generator) at twice its resolution,
    256^3 at dx 0.25 um, 3 gradient directions, PGSE b = 1000."""
    import torch
    from paper_1907_00908_gb300 import lbmbt, synth
    torch.cuda.set_device(0)
    n = min(args.n, 256)
    t0 = time.perf_counter()
    geom = synth.cylinders(n, 0.25, seed=1)
    dl = synth.link_distances(geom, (0, 0, 0))
    t_geo = time.perf_counter() - t0
    dt = 0.0015625
    gGs = [lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, dt, d)[0] for d in ((1, 0, 0), (0, 1, 0), (1, 1, 1))]
    _, f = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, dt, (1, 0, 0))
    members = lbmbt.Solver.members(gGs, 0, C2_KAPPA)
    stream = torch.cuda.current_stream()
    n_memb_links = int((dl != 0.5).sum())
    res = {}
    for name, kernel, use_dl in (("links_register", 1, True), ("half_link_register", 1, False),
                                 ("half_link_bulk_copy", 2, False)):
        s = lbmbt.Solver(0, stream)
        s.set_option(lbmbt.OPT_KERNEL, kernel)
        s.set_option(lbmbt.OPT_AUTOTUNE, 0 if args.no_autotune else 1)
        if args.no_autotune and use_dl:   # the tuner's usual choice for this kernel
            s.set_option(lbmbt.OPT_BLOCK, 128)
            s.set_option(lbmbt.OPT_SPT, 2)
        s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, (0, 0, 0))
        if use_dl:
            s.set_link_distances(dl)
        s.set_phases(C2_D, C2_T2)
        s.set_sequence(dt, f, gGs[0])
        s.prepare(members)
        s.advance(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(0) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            sig = s.advance(args.steps, want_signal=True, n_members=len(gGs))
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"MLUPS": geom.n_sites * len(gGs) / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                     "launch": {"block": s.get_option(lbmbt.OPT_BLOCK), "spt": s.get_option(lbmbt.OPT_SPT)},
                     "S_after": (np.abs(sig[:, 0] + 1j * sig[:, 1]) / geom.n_sites).tolist(), "clocks": clk.summary()}
        s.close()
    peak, peak_kind = peaks()
    v = res["links_register"]["MLUPS"]
    # algorithmic bytes: 113 per site update + 4 per membrane link (its position)
    bytes_site = BYTES_PER_SITE + 4.0 * n_memb_links / geom.n_sites
    achieved = bytes_site * v * 1e6 / 1e9
    traffic = links_traffic_per_launch(n)
    line = {"metric": "MLUPS (fused sweep with membrane positions on the links, FP32)", "value": v, "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["links_register"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"cylinders{n}_dx0.25_links_3dir", "grid": [n] * 3, "membrane_link_fraction":
                       n_memb_links / (6.0 * geom.n_sites), "geometry_gen_s": round(t_geo, 1)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_source": peak_kind, "bytes_per_site_member": bytes_site,
                         "kernel": "sweep_links_kernel (register)"},
            "compare": res}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- membrane-rule study
def run_membrane_study(args):
    """The paper's four-variant membrane study (Sec. 3.6) on the GPU: a 40 um
    disc at intracellular fraction 0.5 in a periodic square (D 2.3 um^2/ms
    on both sides, kappa 0.05 um/ms, PGSE delta 5 / Delta 20 ms, b 1000
    s/mm^2 along x, tau 0.8, D2Q5 on one plane), S at the echo for the full
    general-angle rule, Delta_m = 1/2 with the angles, theta = 0 with the
    positions, and the half-link rule, on grids of 100^2 to 800^2.  The
    reported throughput is the full rule's sweep on the finest grid."""
    import torch
    from paper_1907_00908_gb300 import lbmbt, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    D, kap, b, delta, Delta, R = 2.3, 0.05, 1000.0, 5.0, 20.0, 20.0
    Lb = math.sqrt(math.pi * R * R / 0.5)
    study, timing = {}, {}
    grids = (100, 200, 400, 800)
    with Clocks(0) as clk:
        for n in grids:
            dx = Lb / n
            dt = delta / math.ceil(delta / (0.3 * (1.0 / 3.0) * dx * dx / D))   # tau <= 0.8
            g = synth.disks(n, dx, [[Lb / 2 + 0.123, Lb / 2 - 0.071]], [R])
            dl, th = synth.link_distances(g, (0, 0, 0)), synth.link_angles(g, (0, 0, 0))
            gG, f = lbmbt.pgse(b, delta, Delta, dt, (1, 0, 0))
            row = {}
            for name, pos, ang in (("full", dl, th), ("delta_half", np.full_like(dl, 0.5), th),
                                   ("theta_zero", dl, None), ("half_link", None, None)):
                s = lbmbt.Solver(0, stream)
                s.set_option(lbmbt.OPT_LATTICE, 1)
                s.set_geometry(g.labels, g.phase_of_label, dx, (0, 0, 0))
                if pos is not None:
                    s.set_link_distances(pos)
                if ang is not None:
                    s.set_link_angles(ang)
                s.set_phases([D, D], [math.inf, math.inf])
                s.set_sequence(dt, f, gG)
                s.prepare(lbmbt.Solver.members([gG], 0, kap))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                sig = s.advance(len(f), want_signal=True, n_members=1)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                row[name] = float(abs(sig[0, 0] + 1j * sig[0, 1]) / g.n_sites)
                if n == grids[-1]:
                    timing[name] = {"MLUPS": g.n_sites * len(f) / (ms * 1e-3) / 1e6, "ms_run": ms, "steps": len(f)}
                s.close()
            study[str(n)] = {"dx_um": dx, "dt_ms": dt, "steps": len(f), "S": row}
    v = timing["full"]["MLUPS"]
    fin = study[str(grids[-1])]["S"]
    line = {"metric": "MLUPS (2-D sweep, membrane positions and angles, FP32)", "value": v, "unit": "MLUPS",
            "n_gpus": 1, "steps": timing["full"]["steps"], "warmup": 0,
            "ms_per_step": timing["full"]["ms_run"] / timing["full"]["steps"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "disc40um_fraction0.5_four_membrane_variants", "grids": list(grids),
                       "kappa_um_ms": kap, "D": D, "b_s_mm2": b, "lattice": "D2Q5"},
            "study": study,
            "finest_grid_relative_to_full": {k: (val - fin["full"]) / fin["full"] for k, val in fin.items()},
            "timing_finest_grid": timing, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- scheme variants
def run_variants(args):
    """The paper's cheap variants, each timed against its plain counterpart:
    the 2-D D2Q5 lattice (Sec. 2.3) on a 4096^2 cell pattern, and reaction
    sub-steps (dt = 4 dt', an OGSE-like sine waveform, so every step takes
    the general rotation) on the 256^3 cylinders."""
    import torch
    from paper_1907_00908_gb300 import lbmbt, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = {}

    def timed(s, n_sites, members, steps):
        s.set_option(lbmbt.OPT_AUTOTUNE, 1)
        s.prepare(members)
        s.advance(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.advance(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        return {"MLUPS": n_sites * len(members) / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                "kernel": "bulk-copy" if s.get_option(lbmbt.OPT_KERNEL_USED) == 2 else "register"}

    # D2Q5 vs D3Q7 on the same one-plane grid (cells of ~10 um in a 1 mm square)
    n2 = 4096
    cell = 40
    lab = (np.arange(n2)[:, None] // cell * (n2 // cell) + np.arange(n2)[None, :] // cell).astype(np.int64)
    lab = (lab * 2654435761 % 97).astype(np.int32)[None]   # neighbouring cells get different labels
    pol = (np.arange(97) % 2).astype(np.uint8)
    gG, f = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, 0.005, (1, 1, 0))
    mem = lbmbt.Solver.members([gG], 0, C2_KAPPA)
    for lat in (1, 0):
        s = lbmbt.Solver(0, stream)
        s.set_option(lbmbt.OPT_LATTICE, lat)
        s.set_geometry(lab, pol, 0.25, (0, 0, 0))
        s.set_phases(C2_D, C2_T2)
        s.set_sequence(0.005, f, gG)
        out["D2Q5_4096sq" if lat else "D3Q7_same_grid"] = timed(s, lab.size, mem, args.steps)
        s.close()
    # reaction sub-steps on the cylinders
    geom = synth.cylinders(256, 0.25, seed=1)
    dt, k, K = 0.0015625, 4, 2000
    t = (np.arange(K * k) + 0.5) * dt / k
    f_fine = np.sin(2 * np.pi * t / 1.0)
    gG3 = [0.2 * np.asarray(d, float) / np.linalg.norm(d) for d in ((1, 0, 0), (0, 1, 0), (1, 1, 1))]
    mem3 = lbmbt.Solver.members(gG3, 0, C2_KAPPA)
    for name, sub in (("substeps4_sine", k), ("pgse_one_reaction", 1)):
        s = lbmbt.Solver(0, stream)
        s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, (0, 0, 0))
        s.set_phases(C2_D, C2_T2)
        if sub > 1:
            s.set_sequence_substeps(dt, f_fine, gG3[0], sub)
        else:
            _, fp = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, dt, (1, 0, 0))
            s.set_sequence(dt, fp, gG3[0])
        out[name] = timed(s, geom.n_sites, mem3, args.steps)
        s.close()
    line = {"metric": "MLUPS (scheme variants, FP32)", "value": out["D2Q5_4096sq"]["MLUPS"], "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "variants_d2q5_4096sq_and_substeps_cyl256"}, "compare": out}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- classical scheme (Appendix A)
def run_classical(args):
    """The paper's comparison scheme, the classical LBM with the reaction as a
    collision source (Appendix A, Eq. A12), on the GPU.

    Throughput: the 256^3 cylinders (dx 0.25 um, c2 phases, 3 gradient
    directions, PGSE b = 1000) with the classical pass (autotuned; and on
    each sweep) against the hybrid pass on the same sweeps.

    Accuracy (Sec. 3.2, Fig. 5): a uniform initial field in periodic squares
    of side L = 20 and 100 um (D2Q5, D = 2.0, T2 = inf, tau = 0.6, PGSE
    b = 1000, delta 3 / Delta 6 ms, run to the echo), relative L2 error of
    the field at the echo against the continuum exp(-bD), for dx = 1, 0.5
    and 0.25 um: the hybrid's does not depend on L, the classical one's does."""
    import torch
    from paper_1907_00908_gb300 import lbmbt, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = min(args.n, 256)
    geom = synth.cylinders(n, 0.25, seed=1)
    dt = 0.0015625
    gGs = [lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, dt, d)[0] for d in ((1, 0, 0), (0, 1, 0), (1, 1, 1))]
    _, f = lbmbt.pgse(1000.0, C2_DELTA, C2_BIG_DELTA, dt, (1, 0, 0))
    members = lbmbt.Solver.members(gGs, 0, C2_KAPPA)
    timing = {}
    clocks = None
    for name, scheme, kernel in (("classical", 1, 0), ("classical_register", 1, 1),
                                 ("classical_bulk_copy", 1, 2), ("hybrid_register", 0, 1),
                                 ("hybrid_bulk_copy", 0, 2)):
        s = lbmbt.Solver(0, stream)
        s.set_option(lbmbt.OPT_SCHEME, scheme)
        s.set_option(lbmbt.OPT_KERNEL, kernel)
        s.set_option(lbmbt.OPT_AUTOTUNE, 0 if args.no_autotune else 1)
        s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, (0, 0, 0))
        s.set_phases(C2_D, C2_T2)
        s.set_sequence(dt, f, gGs[0])
        s.prepare(members)
        s.advance(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(0) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            s.advance(args.steps, want_signal=True, n_members=len(gGs))
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        timing[name] = {"MLUPS": geom.n_sites * len(gGs) / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                        "launch": _launch_shape(s, lbmbt)}
        if name == "classical":
            clocks = clk.summary()
        s.close()

    # Sec. 3.2 / Fig. 5: uniform initial field, L-dependence
    Dfree, b, delta, Delta, tau = 2.0, 1000.0, 3.0, 6.0, 0.6
    ex = math.exp(-b * 1e-3 * Dfree)
    study = {}
    for L in (20.0, 100.0):
        for dx in (1.0, 0.5, 0.25):
            m = math.ceil(delta / ((tau - 0.5) * (1.0 / 3.0) * dx * dx / Dfree))
            while abs(Delta * m / delta - round(Delta * m / delta)) > 1e-9:
                m += 1
            dts = delta / m
            gG, fs = lbmbt.pgse(b, delta, Delta, dts, (1, 0, 0))
            nn = int(round(L / dx))
            lab = np.zeros((1, nn, nn), np.int32)
            row = {"dt_ms": dts, "steps": len(fs)}
            for scheme in (0, 1):
                s = lbmbt.Solver(0, stream)
                s.set_option(lbmbt.OPT_SCHEME, scheme)
                s.set_option(lbmbt.OPT_LATTICE, 1)
                s.set_geometry(lab, [0], dx, (0, 0, 0))
                s.set_phases([Dfree], [math.inf])
                s.set_sequence(dts, fs, gG)
                fld = torch.zeros(lab.size, dtype=torch.complex64, device="cuda")
                r = s.run(field=fld)
                torch.cuda.synchronize()
                err = float(torch.sqrt(torch.mean(torch.abs(fld.to(torch.complex128) - ex) ** 2)) / ex)
                fin = lambda x: x if math.isfinite(x) else None   # a diverged run has no error to report
                row["classical" if scheme else "hybrid"] = {"S": fin(r["S"]), "field_L2_rel_err": fin(err)}
                s.close()
            study[f"L{int(L)}_dx{dx}"] = row
    peak, peak_kind = peaks()
    v = timing["classical"]["MLUPS"]
    achieved = BYTES_PER_SITE * v * 1e6 / 1e9
    line = {"metric": "MLUPS (classical LBM with reaction source, FP32)", "value": v, "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": timing["classical"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"cylinders{n}_dx0.25_classical_3dir", "grid": [n] * 3},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                         "bytes_per_site_member": BYTES_PER_SITE,
                         "kernel": "classical pass, " + timing["classical"]["launch"]["kernel"] + " sweep"},
            "compare": timing, "uniform_ic_study": study, "exact_exp_minus_bD": ex, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- slabs (strips)
def run_slab(args):
    """The 512^3 tissue batch cut into z slabs on one GPU (one context per
    slab, faces exchanged before every step), against the same grid in one
    piece, both timed with CUDA events over the same steps."""
    import torch
    from paper_1907_00908_gb300 import lbmbt, slab
    torch.cuda.set_device(0)
    geom = geometry(args.n)
    seqs = sequences()
    nm = len(seqs)
    members = lbmbt.Solver.members([g for g, _ in seqs], 0, KAPPA)
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        # whole grid, stepped one launch at a time like the slabs
        s = lbmbt.Solver(0, stream)
        s.set_geometry(geom.labels, geom.phase_of_label, DX, (1, 1, 1))
        s.set_phases(D, T2)
        s.set_sequence(DT, seqs[0][1], seqs[0][0])
        s.prepare(members)
        for _ in range(args.warmup):
            s.advance(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            sig_whole = s.advance(1, want_signal=(k == args.steps - 1), n_members=nm)
        e1.record(stream)
        torch.cuda.synchronize()
        out["whole"] = e0.elapsed_time(e1) / args.steps
        s.close()
        g = slab.SlabGroup(geom.labels, geom.phase_of_label, DX, (1, 1, 1), args.slabs, D, T2, DT, seqs[0][1],
                           members, stream)
        for _ in range(args.warmup):
            g.step()
        with Clocks(0) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for k in range(args.steps):
                Z = g.step(want_signal=(k == args.steps - 1))
            e1.record(stream)
            torch.cuda.synchronize()
        out["slabs"] = e0.elapsed_time(e1) / args.steps
        g.close()
    Zw = sig_whole[:, 0] + 1j * sig_whole[:, 1]
    v = geom.n_sites * nm / (out["slabs"] * 1e-3) / 1e6
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["slabs"], "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"tissue512_voronoi_mirror_3dir_{args.slabs}slabs", "grid": [args.n] * 3,
                       "slabs": slab.split(args.n, args.slabs), "exchange": "one plane of one population per "
                       "face, member and step, device copies on one stream"},
            "whole_grid_one_step_per_call": {"value": geom.n_sites * nm / (out["whole"] * 1e-3) / 1e6,
                                             "unit": "MLUPS", "ms_per_step": out["whole"]},
            "slab_over_whole_time": out["slabs"] / out["whole"],
            "signal_rel_diff_vs_whole": float(np.max(np.abs(Z - Zw) / np.abs(Zw))),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use the default launch shape")
    ap.add_argument("--adj-shape", type=int, default=2, help="bulk-copy adjoint consumer shape (0, 1 or 2)")
    ap.add_argument("--adjoint-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="adjoint sweep: 0 auto, 1 register, 2 bulk copy")
    ap.add_argument("--stage-own-z", type=int, default=0, choices=[0, 1, 2, 3],
                    help="bulk-copy sweep: own z values 0 auto, 1 prefetched into registers, 2 staged, "
                         "3 z-marching columns")
    ap.add_argument("--column-planes", type=int, default=0,
                    help="bulk-copy sweep, z-marching form: planes per column (0 auto, else a power of two)")
    ap.add_argument("--members", type=int, default=60, help="adjoint workload: number of members (<= 60)")
    ap.add_argument("--adj-steps", type=int, default=400,
                    help="adjoint workload: steps of the 6400-step schedule timed (the prefix)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the plain 128^3, batched and adjoint figures")
    ap.add_argument("--no-adjoint-full", action="store_true",
                    help="skip the full-schedule (6400-step) adjoint figure of the default run")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--spt", type=int, default=0)
    ap.add_argument("--n", type=int, default=N_EDGE, help="lattice edge (default 512)")
    ap.add_argument("--slabs", type=int, default=4, help="slab workload: number of z slabs")
    ap.add_argument("--nz", type=int, default=0,
                    help="default workload: run only the tissue's first NZ planes (a small case for counters)")
    ap.add_argument("--workload", default="tissue512",
                    choices=["tissue512", "batch", "adjoint", "slab", "links", "variants", "membrane_study",
                             "classical"],
                    help="tissue512 (default): the 512^3 tissue batch of 3 directions; batch: 528 members on "
                         "17 geometries; adjoint: gradient of 60 members on a 96^3 sphere pack; slab: the "
                         "tissue batch cut into --slabs z slabs with a face exchange per step; links: membranes at "
                         "their exact positions on the links (256^3 cylinders) against the half-link rule; variants: "
                         "D2Q5 and reaction sub-steps against their plain counterparts; membrane_study: the "
                         "paper's four membrane-rule variants on a 40 um disc, 100^2 to 800^2; classical: the "
                         "classical LBM with a reaction source against the hybrid scheme (throughput on 256^3 "
                         "cylinders, and the domain-size study of Sec. 3.2)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "slab":
        return run_slab(args)
    if args.workload == "links":
        return run_links(args)
    if args.workload == "membrane_study":
        return run_membrane_study(args)
    if args.workload == "variants":
        return run_variants(args)
    if args.workload == "classical":
        return run_classical(args)

    import torch
    import torch.distributed as dist
    from paper_1907_00908_gb300 import lbmbt

    rank, world, local = _rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    t_geo = time.perf_counter()
    geom = geometry(args.n)
    if args.nz and args.nz < args.n:
        # the tissue's first nz planes (same planes, staging form and faces;
        # a small case for counter captures)
        from paper_1907_00908_gb300 import synth
        geom = synth.Geometry(np.ascontiguousarray(geom.labels[:args.nz]), geom.phase_of_label, geom.dx)
    t_geo = time.perf_counter() - t_geo
    nz_run = int(geom.labels.shape[0])
    fractions = phase_fractions(geom)
    seqs = sequences()
    K_total = len(seqs[0][1])
    assert args.warmup + args.steps <= K_total
    n_sites = geom.n_sites
    nm = len(seqs)

    s = lbmbt.Solver(local, stream)
    s.set_option(lbmbt.OPT_STAGE_OWN_Z, args.stage_own_z)
    s.set_option(lbmbt.OPT_COLUMN_PLANES, args.column_planes)
    if not args.no_autotune:
        s.set_option(lbmbt.OPT_AUTOTUNE, 1)
    if args.block:
        s.set_option(lbmbt.OPT_BLOCK, args.block)
    if args.spt:
        s.set_option(lbmbt.OPT_SPT, args.spt)
    s.set_geometry(geom.labels, geom.phase_of_label, DX, (1, 1, 1))
    s.set_phases(D, T2)
    s.set_sequence(DT, seqs[0][1], seqs[0][0])
    members = lbmbt.Solver.members([g for g, _ in seqs], 0, KAPPA)
    s.prepare(members)
    s.advance(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = s.launch_count()
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        sig = s.advance(args.steps, want_signal=True, n_members=nm)
        e1.record(stream)
        torch.cuda.synchronize()
    clocks_main = clk.summary()
    launches = s.launch_count() - l0
    shape = {"kernel": "bulk-copy" if s.get_option(lbmbt.OPT_KERNEL_USED) == 2 else "register",
             "tma_shape": s.get_option(lbmbt.OPT_TMA_SHAPE), "stages": s.get_option(lbmbt.OPT_STAGES),
             "block": s.get_option(lbmbt.OPT_BLOCK), "spt": s.get_option(lbmbt.OPT_SPT),
             "own_z": {0: None, 1: "prefetched", 2: "staged", 3: "z-marching"}[s.get_option(lbmbt.OPT_STAGE_OWN_Z_USED)],
             "autotuned": not args.no_autotune}
    from paper_1907_00908_gb300 import shard
    ms = shard.max_over_ranks(e0.elapsed_time(e1), dist if world > 1 else None, dev)
    if world > 1:
        dist.barrier()
    value = n_sites * nm * args.steps * world / (ms * 1e-3) / 1e6
    per_launch_s = ms * 1e-3 / args.steps
    achieved = BYTES_PER_SITE * n_sites * nm / per_launch_s / 1e9
    peak, peak_kind = peaks()

    # end to end through the public API: host labels (pinned) -> mask,
    # sequence upload, batch set-up and the same K steps, signal to the host.
    e2e = None
    if not args.no_e2e:
        lab_pinned = torch.from_numpy(geom.labels).pin_memory()
        s2 = lbmbt.Solver(local, stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        h0 = time.perf_counter()
        s2.set_geometry(lab_pinned.numpy(), geom.phase_of_label, DX, (1, 1, 1))
        s2.set_phases(D, T2)
        s2.set_sequence(DT, seqs[0][1], seqs[0][0])
        s2.prepare(members)
        sig2 = s2.advance(args.steps, want_signal=True, n_members=nm)
        torch.cuda.synchronize()
        te = shard.max_over_ranks(time.perf_counter() - h0, dist if world > 1 else None, dev)
        s2.close()
        h2d = n_sites * 4 + geom.phase_of_label.size + K_total * (4 + 8) + nm * 200
        d2h = nm * 16
        e2e = {"value": n_sites * nm * args.steps * world / te / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": te, "includes": "label upload + mask build + sequence upload + set-up + K steps + signal"}
        del sig2
    s.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(geom, seqs)

    # the other forms the metric compares on the same GPU, each timed on its
    # own: the plain single-direction sweep on the 128^3 cylinders, the
    # 528-member batch, and the adjoint (a 400-step prefix and the full
    # 6400-step schedule of its 60 members)
    extras = {}
    if world == 1 and not args.no_extras:
        del geom
        extras["plain_single_direction"] = measure_plain_c2(args, stream)
        b = measure_batch(args, stream)
        b["batched_over_plain"] = b["value"] / extras["plain_single_direction"]["value"]
        extras["batched"] = b
        extras["adjoint"] = measure_adjoint(args, stream, args.adj_steps)
        if not args.no_adjoint_full:
            extras["adjoint_full_schedule"] = measure_adjoint(args, stream, None)

    if rank == 0:
        tr = traffic_per_launch(n_sites * nm, shape["own_z"])
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if nz_run == args.n else
                       f"tissue512_first{nz_run}planes_voronoi_mirror_3dir",
                       "grid": [args.n, args.n, nz_run], "dx_um": DX, "dt_ms": DT, "members": nm,
                       "bc": "mirror", "phases": 3, "kappa_um_ms": KAPPA, "b_s_mm2": B,
                       "l2": f"state of {2 * 7 * 8 * n_sites / 1e9:.2f} GB per direction, larger than L2; "
                             "no flush needed",
                       "sites_per_step": n_sites * nm, "geometry_gen_s": round(t_geo, 1), "launch": shape,
                       "seed": TISSUE_SEED, "phase_fractions": fractions},
            "signal_after_timed_steps": [float(x) for x in sig[:, 2]],
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": tr, "peak_source": peak_kind,
                         "traffic_gbs": tr / per_launch_s / 1e9 if tr is not None else None,
                         "traffic_source": ("ncu DRAM bytes of the " + str(shape["own_z"]) + " form on the tissue's "
                                            "first 128 planes, scaled by site updates (profiles/sweep_traffic.json)"
                                            + ("" if shape["own_z"] == "z-marching" else
                                               "; bytes per update rise with the planes, so a lower bound for "
                                               "the full grid")) if tr is not None else None,
                         "bytes_per_site_member": BYTES_PER_SITE, "kernel": "sweep_tma_kernel"},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks_main,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
