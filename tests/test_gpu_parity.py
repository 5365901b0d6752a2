"""GPU parity: the CUDA sweep through the C ABI against the FP64 oracle.

Tolerances (the FP32 sweep against the FP64 scheme): signal S within 1e-5
relative; field within 1e-4 of max|M| (max_x |M_gpu - M_ref| / max_x |M_ref|);
the mask byte bit-exact.  Inputs are seeded synthetic geometries of the
workloads' kinds (free diffusion, z-aligned cylinders, sphere packs, Voronoi
tissue with vessels), at sizes the oracle finishes in seconds plus full-size
grids on shortened schedules.
"""
import math

import numpy as np
import pytest

import oracle
import refs
from paper_1907_00908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S_TOL = 1e-5
FIELD_TOL = 1e-4
INF = math.inf


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _solver(lb, geom, bc, D, T2, kappa, dt, f, gG):
    s = lb.Solver(0)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
    s.set_phases(D, T2)
    s.set_permeability(kappa)
    s.set_sequence(dt, f, gG)
    return s


def _oracle(geom, bc, D, T2, kappa, dt, f, gG, **kw):
    return oracle.run(geom.labels, geom.dx, geom.phase_of_label, bc, D, T2, kappa, dt, f, gG, **kw)


def _field_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _gpu_field(s, n):
    fld = torch.zeros(n, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    return r, fld.cpu().numpy()


# ------------------------------------------------------------------ mask
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (1, 0, 1), (0, 1, 0)])
def test_mask_bit_exact(lb, bc):
    rng = np.random.default_rng(42)
    cases = [
        synth.Geometry(rng.integers(0, 5, size=(7, 9, 13)).astype(np.int32), np.array([0, 1, 2, 3, 1], np.uint8), 1.0),
        synth.cylinders(40, 0.5, seed=3),
        synth.crop(synth.voronoi_tissue(64, 0.25, seed=5), 37),
        synth.planes((3, 4, 50), 1.0, [7, 5], axis=0, phases=[0, 1]),
    ]
    for g in cases:
        with lb.Solver(0) as s:
            s.set_geometry(g.labels, g.phase_of_label, g.dx, bc)
            m = s.get_mask(0, g.labels.shape)
        ref = oracle.mask(g.labels, g.phase_of_label, bc)
        assert np.array_equal(m, ref)


def test_mask_from_device_labels(lb):
    g = synth.spheres(30, 0.5, seed=8)
    lab = torch.from_numpy(g.labels).cuda()
    with lb.Solver(0) as s:
        s.set_geometry(lab, g.phase_of_label, g.dx, (0, 0, 0))
        m = s.get_mask(0, g.labels.shape)
    assert np.array_equal(m, oracle.mask(g.labels, g.phase_of_label, (0, 0, 0)))


# ------------------------------------------------------ free diffusion (c1)
@pytest.mark.parametrize("b", [0.0, 250.0, 500.0, 1000.0, 2000.0])
def test_free_diffusion_32cubed(lb, b):
    """32^3 periodic, dx = 1, D = 2, T2 = inf, PGSE delta 5 / Delta 20 along x,
    dt = 0.0125 (tau = 0.6), run to the echo (2000 steps)."""
    geom = synth.uniform(32, 1.0)
    dt = 0.0125
    gG, f = oracle.pgse(b, 5.0, 20.0, dt, (1, 0, 0))
    s = _solver(lb, geom, (0, 0, 0), [2.0], [INF], INF, dt, f, gG)
    r = s.run()
    s.close()
    o = _oracle(geom, (0, 0, 0), [2.0], [INF], INF, dt, f, gG)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    # the same number from the plane-wave closed form of the scheme
    assert abs(r["S"] - refs.planewave_signal(32, 1.0, 2.0, INF, dt, f, gG)) <= S_TOL * o["S"]
    # and close to the continuum exp(-bD): the lattice's dispersion error at
    # q dx = 0.33 (b = 2000) is about 4 % of S
    assert r["S"] == pytest.approx(math.exp(-b * 1e-3 * 2.0), rel=0.05)


# --------------------------------------------------- cylinders (c2 kind)
@pytest.mark.parametrize("direction", [(1, 0, 0), (0.6, 0.8, 0), (1, 1, 1)])
def test_cylinders_signal_and_field(lb, direction):
    geom = synth.cylinders(48, 0.5, seed=21)
    dt = 0.025
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    gG, f = oracle.pgse(3000.0, 2.0, 6.0, dt, direction)
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert abs(r["Z"] - o["Z"]) <= S_TOL * abs(o["Z"])
    assert _field_err(fld.reshape(geom.shape), o["field"]) < FIELD_TOL


def test_c2_geometry_full_size_short_schedule(lb):
    """128^3 at dx = 0.5 with the c2 cylinder pack and c2 physics
    (D 1/2, T2 50/80, kappa 0.02, dt 0.00625), the first 64 steps of the
    PGSE (b = 3000, oblique G), with the field."""
    geom = synth.cylinders(128, 0.5, seed=1)
    dt = 0.00625
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    gG, f = oracle.pgse(3000.0, 10.0, 30.0, dt, (0.48, -0.6, 0.64))
    f = f[:64]
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.reshape(geom.shape), o["field"]) < FIELD_TOL


# ----------------------------------------------------- mirror (c5 kind)
@pytest.mark.parametrize("direction", [(1, 0, 0), (0, 1, 0), (0, 0, 1)])
def test_voronoi_mirror_parity(lb, direction):
    geom = synth.crop(synth.voronoi_tissue(64, 0.5, cell_diam=8.0, vessel_radius=2.0, seed=7), 40)
    dt = 0.025
    D, T2, kap = [1.0, 2.5, 3.0], [50.0, 80.0, 80.0], 0.01
    gG, f = oracle.pgse(1000.0, 2.0, 5.0, dt, direction)
    s = _solver(lb, geom, (1, 1, 1), D, T2, kap, dt, f, gG)
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    o = _oracle(geom, (1, 1, 1), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.reshape(geom.shape), o["field"]) < FIELD_TOL


def test_mixed_bc_parity(lb):
    """Mirror on x and z, periodic on y, G normal to x (conjugate rule on x,
    plain swap on z)."""
    geom = synth.spheres((33, 20, 17), 0.5, rmin=1.5, rmax=3.0, fraction=0.4, seed=12)
    dt = 0.02
    D, T2, kap = [2.0, 1.2], [70.0, 40.0], 0.05
    gG, f = oracle.pgse(2000.0, 1.0, 3.0, dt, (1, 0, 0))
    s = _solver(lb, geom, (1, 0, 1), D, T2, kap, dt, f, gG)
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    o = _oracle(geom, (1, 0, 1), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.reshape(geom.shape), o["field"]) < FIELD_TOL


# ------------------------------------------------------ series and edges
def test_series_parity(lb):
    geom = synth.cylinders(24, 1.0, fraction=0.5, seed=2)
    dt = 0.05
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.05
    gG, f = oracle.pgse(1500.0, 2.0, 5.0, dt, (1, 2, 0))
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    r = s.run(series=True)
    s.close()
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG, want_series=True)
    scale = np.abs(o["series"]).max()
    assert np.abs(r["series"] - o["series"]).max() <= S_TOL * scale
    assert r["Z"] == r["series"][-1]


@pytest.mark.parametrize("shape,bc,kappa", [
    ((1, 1, 1), (0, 0, 0), INF),
    ((1, 1, 37), (1, 0, 0), 0.0),
    ((3, 5, 37), (0, 1, 0), 0.1),
    ((2, 65, 3), (1, 1, 1), INF),
    ((17, 1, 1), (0, 0, 1), 0.3),
])
def test_edge_shapes(lb, shape, bc, kappa):
    """Ragged and degenerate grids: single node, 1-wide axes, sizes that leave
    a partial tile, every BC combination, kappa = 0 / finite / inf."""
    rng = np.random.default_rng(sum(shape))
    lab = rng.integers(0, 3, size=shape).astype(np.int32)
    geom = synth.Geometry(lab, np.array([0, 1, 0], np.uint8), 0.7)
    dt = 0.04
    D, T2 = [1.5, 0.8], [60.0, 30.0]
    # a gradient normal to the first mirror axis is parallel to the others;
    # without mirror axes an oblique gradient is allowed
    ax = [a for a in range(3) if bc[a] == 1]
    d = [0.0, 0.0, 0.0]
    if ax:
        d[ax[0]] = 1.0
    else:
        d = [1.0, 0.5, 0.25]
    gG, f = oracle.pgse(1000.0, 1.0, 2.0, dt, d)
    s = _solver(lb, geom, bc, D, T2, kappa, dt, f, gG)
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    o = _oracle(geom, bc, D, T2, kappa, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.reshape(shape), o["field"]) < FIELD_TOL


def test_gradient_free_conservation_on_gpu(lb):
    """G = 0, T2 = inf: M = 1 is a fixed point on the GPU too (FP32: the
    weights 1/4, 1/8 are exact and r + s = 1 up to one rounding)."""
    geom = synth.spheres(20, 1.0, rmin=2.0, rmax=4.0, fraction=0.4, seed=5)
    s = _solver(lb, geom, (1, 0, 1), [1.0, 2.5], [INF, INF], 0.03, 0.05, np.zeros(200), [0, 0, 0])
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    assert abs(r["S"] - 1.0) < 1e-6
    assert np.abs(fld - 1.0).max() < 1e-5


# ------------------------------------------------------------ options
def test_graph_and_launch_shapes_do_not_change_results(lb):
    geom = synth.cylinders(32, 0.5, seed=9)
    dt = 0.025
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    gG, f = oracle.pgse(2000.0, 1.0, 3.0, dt, (1, 1, 0))
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    base = s.run()["S"]
    for graph, block, spt, kern in [(0, 256, 2, 1), (1, 128, 1, 1), (1, 512, 1, 1), (1, 256, 4, 1), (0, 64, 4, 1),
                                    (1, 256, 2, 2), (0, 256, 2, 2)]:
        s.set_option(lb.OPT_GRAPH, graph)
        s.set_option(lb.OPT_BLOCK, block)
        s.set_option(lb.OPT_SPT, spt)
        s.set_option(lb.OPT_KERNEL, kern)
        # the fields are bit-identical across shapes and kernels; the signal's
        # per-thread FP32 partial sums group sites differently, ~1e-9 relative
        assert s.run()["S"] == pytest.approx(base, rel=1e-7)
    s.set_option(lb.OPT_AUTOTUNE, 1)
    assert s.run()["S"] == pytest.approx(base, rel=1e-7)
    s.close()


# -------------------------------------------------------------- batch
def test_batch_matches_plain_runs(lb):
    """Members with different directions, b-values, permeabilities and two
    geometries of different sizes in one batched launch per step equal the
    corresponding plain runs."""
    g1 = synth.cylinders(32, 0.5, seed=4)
    g2 = synth.spheres(27, 0.5, rmin=2.0, rmax=3.0, fraction=0.4, seed=6)
    dt = 0.025
    D, T2 = [2.0, 1.0], [80.0, 50.0]
    _, f = oracle.pgse(1000.0, 1.0, 3.0, dt, (1, 0, 0))
    dirs = synth.directions_on_sphere(5, seed=1)
    bvals = [0.0, 800.0, 1600.0, 2400.0, 3000.0]
    members = []
    for i in range(5):
        gG, _ = oracle.pgse(bvals[i], 1.0, 3.0, dt, dirs[i])
        members.append((gG, 0 if i < 3 else 1, [0.02, 0.0, INF, 0.05, 0.01][i]))
    s = lb.Solver(0)
    s.set_geometry(g1.labels, g1.phase_of_label, g1.dx)
    s.add_geometry(g2.labels, g2.phase_of_label, g2.dx)
    s.set_phases(D, T2)
    s.set_sequence(dt, f, members[0][0])
    mem = lb.Solver.members([m[0] for m in members], [m[1] for m in members], [m[2] for m in members])
    rb = s.run_batch(mem)
    s.close()
    for i, (gG, gi, kap) in enumerate(members):
        geom = g1 if gi == 0 else g2
        o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG)
        assert abs(rb["S"][i] - o["S"]) <= S_TOL * o["S"], i
        with _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG) as sp:
            assert sp.run()["S"] == pytest.approx(rb["S"][i], rel=1e-7)


# -------------------------------------------------------------- errors
def test_error_codes(lb):
    geom = synth.uniform(8, 1.0)
    s = lb.Solver(0)
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -7  # ESTATE
    bad = geom.labels.copy()
    bad[0, 0, 3] = 5
    with pytest.raises(lb.LbmbtError) as e:
        s.set_geometry(bad, [0], 1.0)
    assert e.value.code == -6  # EDEVICE: label outside the table
    s.set_geometry(geom.labels, [0], 1.0, (1, 0, 0))
    s.set_phases([1e-30], [INF])
    s.set_sequence(0.05, np.zeros(4), [0, 0, 0])
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -4  # EUNSTABLE: tau rounds to 1/2
    s.set_phases([1.0], [INF])
    s.set_sequence(0.05, np.ones(4), [0.1, 0.1, 0])
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -5  # EUNSUPPORTED: mirror x with oblique G
    s.set_sequence(0.05, np.ones(4), [0.1, 0, 0])
    assert math.isfinite(s.run()["S"])
    with pytest.raises(lb.LbmbtError):
        s.set_option(lb.OPT_SPT, 3)
    # sizes: an empty axis and a grid beyond 2^28 sites are refused before
    # any label is read (the buffer passed is deliberately tiny)
    tiny = np.zeros(8, np.int32)
    pol = np.zeros(1, np.uint8)
    bcv = np.zeros(3, np.int32)
    for dims in [(0, 4, 4), (4, 0, 4), (1024, 1024, 257)]:
        rc = lb.lib().lbmbt_set_geometry(s.h, dims[0], dims[1], dims[2], 1.0, lb._p(tiny), 0, 1, lb._p(pol),
                                         lb._p(bcv))
        assert rc == -1, dims
    # an empty sequence and a non-finite waveform sample are refused (host checks)
    for f_bad in (np.zeros(0), np.array([1.0, math.nan])):
        with pytest.raises(lb.LbmbtError) as e:
            s.set_sequence(0.05, f_bad, [0.1, 0, 0])
        assert e.value.code == -1
    s.close()


# --------------------------------------------- bulk-copy (TMA) sweep
TMA_CASES = [
    ((8, 20, 16), (1, 1, 1), (1, 0, 0)),      # one 20-row unit per plane: both y faces in one unit
    ((6, 37, 32), (1, 0, 0), (1, 0, 0)),      # 16-row units, ragged last unit, periodic y
    ((5, 9, 48), (0, 1, 1), (0, 0, 1)),       # mirror y/z, G normal to z
    ((3, 4, 512), (1, 0, 0), (0, 0.6, 0.8)),  # one row per unit, oblique G parallel to the x mirror
    ((1, 1, 64), (0, 0, 0), (1, 1, 1)),       # single row, every axis wraps onto itself
    ((2, 1, 16), (0, 1, 0), (1, 0, 0)),       # ny = 1 with a mirror on y
]


@pytest.mark.parametrize("case", range(len(TMA_CASES)))
def test_bulk_copy_sweep_parity(lb, case):
    """The bulk-copy sweep equals the register sweep bit for bit on the field
    and both match the oracle, on grids whose row units cover faces, ragged
    units, degenerate axes and membranes on most links."""
    shape, bc, d = TMA_CASES[case]
    rng = np.random.default_rng(100 + case)
    lab = rng.integers(0, 3, size=shape).astype(np.int32)
    geom = synth.Geometry(lab, np.array([0, 1, 2], np.uint8), 0.5)
    dt = 0.02
    D, T2, kap = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.04
    gG, f = oracle.pgse(1500.0, 1.0, 2.0, dt, d)
    out = {}
    for kern, tshape in ((1, 0), (2, 0), (2, 1), (2, 2), (2, 3)):
        s = _solver(lb, geom, bc, D, T2, kap, dt, f, gG)
        s.set_option(lb.OPT_KERNEL, kern)
        s.set_option(lb.OPT_TMA_SHAPE, tshape)
        r, fld = _gpu_field(s, geom.n_sites)
        assert s.get_option(lb.OPT_KERNEL_USED) == kern
        s.close()
        out[(kern, tshape)] = (r, fld)
    for key in out:
        assert np.array_equal(out[(1, 0)][1], out[key][1]), key
    o = _oracle(geom, bc, D, T2, kap, dt, f, gG, want_field=True)
    for kern in out:
        assert abs(out[kern][0]["S"] - o["S"]) <= S_TOL * o["S"]
        assert _field_err(out[kern][1].reshape(shape), o["field"]) < FIELD_TOL


def test_bulk_copy_sweep_rejects_ineligible_grid(lb):
    geom = synth.uniform((4, 4, 24), 1.0)
    s = _solver(lb, geom, (0, 0, 0), [2.0], [INF], INF, 0.05, np.zeros(4), [0, 0, 0])
    s.set_option(lb.OPT_KERNEL, 2)
    with pytest.raises(lb.LbmbtError):
        s.run()
    s.set_option(lb.OPT_KERNEL, 0)
    s.run()
    assert s.get_option(lb.OPT_KERNEL_USED) == 1
    s.close()


def test_signal_partials_do_not_leak_between_runs(lb):
    """Runs with different kernels and launch shapes in one context reuse the
    per-tile signal buffer: every shape must reduce only its own slots."""
    geom = synth.cylinders(32, 0.5, seed=4)
    dt = 0.025
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    gG, f = oracle.pgse(2000.0, 1.0, 3.0, dt, (1, 1, 0))
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    for kern, shape, block, spt in [(1, 0, 64, 1), (2, 0, 256, 2), (2, 1, 256, 2), (2, 2, 256, 2), (1, 0, 512, 4),
                                    (2, 3, 256, 2), (2, 1, 128, 1)]:
        s.set_option(lb.OPT_KERNEL, kern)
        s.set_option(lb.OPT_TMA_SHAPE, shape)
        s.set_option(lb.OPT_BLOCK, block)
        s.set_option(lb.OPT_SPT, spt)
        r = s.run()
        assert abs(r["S"] - o["S"]) <= S_TOL * o["S"], (kern, shape, block, spt)
    s.close()


# --------------------------------------------- full size (benchmark workload)
def test_full_size_tissue_sampled_parity(lb):
    """The benchmark workload at full size (512^3 tissue, mirror faces, three
    directions, default launch configuration = bulk-copy sweep): the field
    after 8 steps at sampled interior, face, edge and corner sites (at the
    low and the high faces) equals the oracle (crop method, cropcheck.py,
    pinned against full oracle runs), and
    the batched signal equals the per-direction runs."""
    import bench
    import cropcheck
    geom = bench.geometry(512)
    seqs = bench.sequences()
    k = 8
    rng = np.random.default_rng(5)
    sites = [tuple(int(v) for v in rng.integers(20, 490, size=3)) for _ in range(6)]
    sites += [(0, 0, 0), (0, 250, 17), (300, 0, 0), (77, 1, 400), (5, 480, 0), (0, 3, 255)]
    sites += [(511, 511, 511), (511, 250, 3), (100, 509, 506), (508, 0, 511), (2, 511, 300), (510, 7, 0)]
    idx = torch.tensor([(z * 512 + y) * 512 + x for (z, y, x) in sites], device="cuda")
    S_plain = []
    for gG, f in seqs:
        s = lb.Solver(0)
        s.set_geometry(geom.labels, geom.phase_of_label, bench.DX, (1, 1, 1))
        s.set_phases(bench.D, bench.T2)
        s.set_permeability(bench.KAPPA)
        s.set_sequence(bench.DT, f[:k], gG)
        fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
        r = s.run(field=fld)
        assert s.get_option(lb.OPT_KERNEL_USED) == 2
        s.close()
        got = fld[idx].cpu().numpy()
        del fld
        ref = cropcheck.sample_values(geom.labels, geom.phase_of_label, (1, 1, 1), bench.DX, bench.D, bench.T2,
                                      bench.KAPPA, bench.DT, f, gG, sites, k)
        assert np.abs(got - ref).max() <= FIELD_TOL * np.abs(ref).max()
        S_plain.append(r["S"])
    s = lb.Solver(0)
    s.set_geometry(geom.labels, geom.phase_of_label, bench.DX, (1, 1, 1))
    s.set_phases(bench.D, bench.T2)
    s.set_sequence(bench.DT, seqs[0][1][:k], seqs[0][0])
    rb = s.run_batch(lb.Solver.members([g for g, _ in seqs], 0, bench.KAPPA))
    s.close()
    np.testing.assert_allclose(rb["S"], S_plain, rtol=1e-7)


# ------------------------------------------------ long schedules (FP32 drift)
def test_full_schedule_cylinders_6400_steps(lb):
    """The cylinder configuration's full PGSE schedule (delta 10, Delta 30,
    dt 0.00625: 6400 steps) at b = 3000 with an oblique gradient, on a 64^3
    pack: the FP32 sweep stays within 1e-5 of the FP64 oracle at the echo."""
    geom = synth.cylinders(64, 0.5, seed=2)
    dt = 0.00625
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    gG, f = oracle.pgse(3000.0, 10.0, 30.0, dt, (0.48, -0.6, 0.64))
    assert len(f) == 6400
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    r = s.run()
    s.close()
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]


@pytest.mark.parametrize("direction", [(1, 0, 0), (0, 0, 1)])
def test_full_schedule_tissue_25600_steps(lb, direction):
    """The tissue configuration's full schedule (dt 0.0015625: 25,600 steps,
    b = 1000, mirror faces, 3 phases) on a 32^3 corner of the 512^3 tissue:
    the FP32 sweep stays within 1e-5 of the FP64 oracle at the echo."""
    import bench
    geom = synth.crop(bench.geometry(128), 32)
    gG, f = oracle.pgse(1000.0, 10.0, 30.0, bench.DT, direction)
    assert len(f) == 25600
    s = _solver(lb, geom, (1, 1, 1), bench.D, bench.T2, bench.KAPPA, bench.DT, f, gG)
    r = s.run()
    s.close()
    o = _oracle(geom, (1, 1, 1), bench.D, bench.T2, bench.KAPPA, bench.DT, f, gG)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"], (r["S"], o["S"])


# ------------------------------------------------------- reaction sub-steps
@pytest.mark.parametrize("bc, gdir", [((0, 0, 0), (0.6, 0.0, 0.8)), ((1, 1, 1), (0.0, 0.0, 1.0))])
def test_reaction_substeps_match_oracle(lb, bc, gdir):
    """dt = k dt' (Sec. 2.3): a fine waveform (a sine-modulated gradient plus
    a PGSE whose edges fall inside diffusion steps) through
    lbmbt_set_sequence_substeps against the oracle's literal k reaction
    sub-steps."""
    geom = synth.cylinders(32, 0.5, seed=4) if bc == (0, 0, 0) else synth.crop(synth.voronoi_tissue(48, 0.5, seed=3), 32)
    n_ph = int(geom.phase_of_label.max()) + 1
    D, T2 = [2.0, 1.0, 1.5][:n_ph], [80.0, 50.0, 60.0][:n_ph]
    dt, k = 0.02, 3
    K = 90
    t = (np.arange(K * k) + 0.5) * dt / k
    f_fine = np.sin(2 * np.pi * t / 0.9)
    f_fine[(t > 0.55) & (t < 0.61)] = 1.0
    gG = 0.08 * np.asarray(gdir) / np.linalg.norm(gdir)
    s = lb.Solver(0)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
    s.set_phases(D, T2)
    s.set_permeability(0.03)
    s.set_sequence_substeps(dt, f_fine, gG, k)
    fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    s.close()
    o = _oracle(geom, bc, D, T2, 0.03, dt, f_fine, gG, want_field=True, substeps=k)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.cpu().numpy().reshape(geom.shape), o["field"]) < FIELD_TOL


# ------------------------------------------------------------- D2Q5 lattice
@pytest.mark.parametrize("bc, gdir", [((0, 0, 0), (0.6, 0.8, 0.0)), ((1, 1, 0), (1.0, 0.0, 0.0))])
def test_d2q5_matches_oracle(lb, bc, gdir):
    """The 2-D D2Q5 lattice (Sec. 2.3, eps_D = 1/3) on one z plane with dense
    membranes, against the oracle's D2Q5 run."""
    rng = np.random.default_rng(17)
    lab = rng.integers(0, 3, size=(1, 40, 48)).astype(np.int32)
    geom = synth.Geometry(lab, np.array([0, 1, 2], np.uint8), 0.5)
    D, T2, kap, dt = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.04, 0.01
    gG, f = oracle.pgse(1500.0, 0.3, 0.6, dt, gdir)
    s = _solver(lb, geom, bc, D, T2, kap, dt, f, gG)
    s.set_option(lb.OPT_LATTICE, 1)
    r, fld = _gpu_field(s, geom.n_sites)
    assert s.get_option(lb.OPT_KERNEL_USED) == 1
    s.close()
    o = _oracle(geom, bc, D, T2, kap, dt, f, gG, want_field=True, lattice="D2Q5")
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.reshape(geom.shape), o["field"]) < FIELD_TOL


def test_d2q5_needs_one_plane(lb):
    geom = synth.uniform((2, 16, 16), 1.0)
    s = _solver(lb, geom, (0, 0, 0), [2.0], [INF], INF, 0.05, np.zeros(4), [0, 0, 0])
    s.set_option(lb.OPT_LATTICE, 1)
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -1
    s.set_option(lb.OPT_LATTICE, 0)
    s.run()
    s.close()


@pytest.mark.parametrize("n_steps", [1, 3, 40])
def test_autotuned_runs_of_any_length_match_the_oracle(lb, n_steps):
    """The autotuner times batches of steps from k = 0 and never beyond the
    schedule, so a schedule shorter than a timing batch is tuned and run
    like any other; the result matches the oracle."""
    geom = synth.cylinders(32, 0.5, seed=4)
    dt = 0.025
    f = np.resize([1.0, 0.0, -1.0, 0.5], n_steps)
    gG = [0.05, 0.03, 0.0]
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    s = _solver(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG)
    s.set_option(lb.OPT_AUTOTUNE, 1)
    r, fld = _gpu_field(s, geom.n_sites)
    s.close()
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"]
    assert _field_err(fld.reshape(geom.labels.shape), o["field"]) < FIELD_TOL
