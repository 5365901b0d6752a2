"""GPU: the three forms of the bulk-copy sweep for geometries with membranes
-- the own-site values of the z populations (needed at membrane links in z,
Eq. B5) prefetched into registers (option 1), staged with the unit (2), or
carried from unit to unit by z-marching columns (3).  All do the same
arithmetic on the same values, so their fields and signals must agree bit
for bit, and each must match the FP64 oracle (S within 1e-5, field within
1e-4 of max|M|).  The automatic choice marches (or, where the grid gives
too few columns, stages) on large planes with membranes only."""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = math.inf


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _run(lb, labels, pol, bc, D, T2, kap, dt, f, gG, oz):
    s = lb.Solver(0)
    s.set_option(lb.OPT_KERNEL, 2)
    s.set_option(lb.OPT_STAGE_OWN_Z, oz)
    s.set_geometry(labels, pol, 0.5, bc)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    fld = torch.zeros(labels.size, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    used = (s.get_option(lb.OPT_KERNEL_USED), s.get_option(lb.OPT_STAGE_OWN_Z_USED))
    s.close()
    return r, fld.cpu().numpy().reshape(labels.shape), used


# a mirror face needs G normal or parallel to it (Sec. 2.4.4)
@pytest.mark.parametrize("bc,gdir", [((0, 0, 0), (0.3, -0.5, 0.81)), ((1, 1, 1), (0.0, 0.0, 1.0)),
                                     ((0, 1, 1), (1.0, 0.0, 0.0))])
def test_forms_agree_and_match_oracle(lb, bc, gdir):
    rng = np.random.default_rng(21)
    labels = rng.integers(0, 3, size=(8, 12, 32)).astype(np.int32)   # z-marching: one column of 8 planes
    pol = np.array([0, 1, 2], np.uint8)
    D, T2, kap, dt = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.05, 0.02
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, dt, gdir)
    out = {}
    for oz in (1, 2, 3):
        r, fld, used = _run(lb, labels, pol, bc, D, T2, kap, dt, f, gG, oz)
        assert used == (2, oz)
        out[oz] = (r, fld)
    for oz in (2, 3):
        assert np.array_equal(out[1][1], out[oz][1])
        assert out[1][0]["S"] == out[oz][0]["S"]
    o = oracle.run(labels, 0.5, pol, bc, D, T2, kap, dt, f, gG, want_field=True)
    assert abs(out[2][0]["S"] - o["S"]) <= 1e-5 * o["S"]
    assert np.abs(out[2][1] - o["field"]).max() < 1e-4 * np.abs(o["field"]).max()


def test_auto_stages_large_planes_with_membranes(lb):
    """A 512 x 256 plane (2^17 sites) with membranes: auto stages, and equals
    the prefetching form bit for bit and the oracle within tolerance; the
    same plane without membranes and a small plane with them prefetch."""
    rng = np.random.default_rng(4)
    nz, ny, nx = 3, 256, 512
    labels = (rng.random((nz, ny // 8, nx // 8)) < 0.4).astype(np.int32)
    labels = np.repeat(np.repeat(labels, 8, axis=1), 8, axis=2)
    pol = np.array([0, 1], np.uint8)
    D, T2, kap, dt = [2.0, 1.0], [80.0, 50.0], 0.05, 0.02
    gG, f = oracle.pgse(1500.0, 0.06, 0.1, dt, (0.3, 0.5, 0.81))
    ra, fa, used = _run(lb, labels, pol, (0, 0, 0), D, T2, kap, dt, f, gG, 0)
    assert used == (2, 2)
    rb, fb, used = _run(lb, labels, pol, (0, 0, 0), D, T2, kap, dt, f, gG, 1)
    assert used == (2, 1)
    assert np.array_equal(fa, fb)
    o = oracle.run(labels, 0.5, pol, (0, 0, 0), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(ra["S"] - o["S"]) <= 1e-5 * o["S"]
    assert np.abs(fa - o["field"]).max() < 1e-4 * np.abs(o["field"]).max()
    _, _, used = _run(lb, np.zeros_like(labels), pol, (0, 0, 0), D, T2, kap, dt, f[:4], gG, 0)
    assert used == (2, 1)
    _, _, used = _run(lb, labels[:, :128], pol, (0, 0, 0), D, T2, kap, dt, f[:4], gG, 0)
    assert used == (2, 1)


def test_auto_marches_tall_large_planes(lb):
    """320 planes of 512 x 256 with membranes: enough columns of 8 planes for
    the automatic choice to march; the same bits as the staging form."""
    rng = np.random.default_rng(5)
    nz, ny, nx = 320, 256, 512
    labels = (rng.random((nz // 4, ny // 8, nx // 8)) < 0.4).astype(np.int32)
    labels = np.repeat(np.repeat(np.repeat(labels, 4, axis=0), 8, axis=1), 8, axis=2)
    pol = np.array([0, 1], np.uint8)
    gG, f = oracle.pgse(1500.0, 0.04, 0.06, 0.02, (0.6, 0.8, 0.0))   # parallel to the mirror z faces
    ra, fa, used = _run(lb, labels, pol, (0, 0, 1), [2.0, 1.0], [80.0, 50.0], 0.05, 0.02, f, gG, 0)
    assert used == (2, 3)
    rb, fb, used = _run(lb, labels, pol, (0, 0, 1), [2.0, 1.0], [80.0, 50.0], 0.05, 0.02, f, gG, 2)
    assert used == (2, 2)
    assert np.array_equal(fa, fb)
    assert ra["S"] == rb["S"]


def test_tuner_picks_staging_or_marching_on_large_planes(lb):
    """With the autotuner on, a grid of large planes with membranes runs in
    whichever of the staging and z-marching forms timed faster, with the
    prefetching form's bits."""
    rng = np.random.default_rng(5)
    nz, ny, nx = 64, 256, 512
    labels = (rng.random((nz // 4, ny // 8, nx // 8)) < 0.4).astype(np.int32)
    labels = np.repeat(np.repeat(np.repeat(labels, 4, axis=0), 8, axis=1), 8, axis=2)
    pol = np.array([0, 1], np.uint8)
    gG, f = oracle.pgse(1500.0, 0.04, 0.06, 0.02, (0.6, 0.8, 0.0))
    args = (labels, pol, (0, 0, 1), [2.0, 1.0], [80.0, 50.0], 0.05, 0.02, f, gG)
    _, ref, _ = _run(lb, *args, 1)
    s = lb.Solver(0)
    s.set_option(lb.OPT_AUTOTUNE, 1)
    s.set_geometry(labels, pol, 0.5, (0, 0, 1))
    s.set_phases([2.0, 1.0], [80.0, 50.0])
    s.set_permeability(0.05)
    s.set_sequence(0.02, f, gG)
    fld = torch.zeros(labels.size, dtype=torch.complex64, device="cuda")
    s.run(field=fld)
    torch.cuda.synchronize()
    used = (s.get_option(lb.OPT_KERNEL_USED), s.get_option(lb.OPT_STAGE_OWN_Z_USED))
    s.close()
    assert used in ((2, 2), (2, 3), (1, 0)), used   # the register sweep may win on a short schedule
    assert np.array_equal(fld.cpu().numpy().reshape(labels.shape), ref)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_marching_batch_of_geometries(lb, bc):
    """Columns over a batch: geometries of 32 and 48 planes (columns of 16
    planes), members with their own directions and kappa, against the
    prefetching form bit for bit and each member's oracle run."""
    geoms = [synth.spheres(32, 0.5, rmin=1.5, rmax=3.0, fraction=0.4, seed=7),
             synth.spheres(48, 0.5, rmin=2.0, rmax=4.0, fraction=0.45, seed=8)]
    dt = 0.025
    _, f = oracle.pgse(1000.0, 0.5, 1.0, dt, (1, 0, 0))
    spec = [(0, 1200.0, (0.0, 0.0, 1.0), 0.02), (1, 2000.0, (0.0, 0.0, 1.0), 0.05), (1, 800.0, (0.0, 0.0, 1.0), 0.0)]
    if bc == (0, 0, 0):
        spec += [(0, 1500.0, (0.6, 0.0, 0.8), INF)]
    gGs = [oracle.pgse(b, 0.5, 1.0, dt, d)[0] for _, b, d, _ in spec]
    out = {}
    for oz in (1, 3):
        s = lb.Solver(0)
        s.set_option(lb.OPT_KERNEL, 2)
        s.set_option(lb.OPT_STAGE_OWN_Z, oz)
        s.set_geometry(geoms[0].labels, geoms[0].phase_of_label, 0.5, bc)
        s.add_geometry(geoms[1].labels, geoms[1].phase_of_label, 0.5, bc)
        s.set_phases([2.0, 1.0], [80.0, 50.0])
        s.set_sequence(dt, f, gGs[0])
        mem = lb.Solver.members(gGs, [g for g, *_ in spec], [k for *_, k in spec])
        flds = [torch.zeros(geoms[g].n_sites, dtype=torch.complex64, device="cuda") for g, *_ in spec]
        r = s.run_batch(mem, fields=flds)
        torch.cuda.synchronize()
        assert s.get_option(lb.OPT_STAGE_OWN_Z_USED) == oz
        s.close()
        out[oz] = (r, [fl.cpu().numpy() for fl in flds])
    for i, (gi, _, _, kap) in enumerate(spec):
        assert np.array_equal(out[1][1][i], out[3][1][i]), i
        assert out[1][0]["S"][i] == out[3][0]["S"][i], i
        g = geoms[gi]
        o = oracle.run(g.labels, g.dx, g.phase_of_label, bc, [2.0, 1.0], [80.0, 50.0], kap, dt, f, gGs[i],
                       want_field=True)
        assert abs(out[3][0]["S"][i] - o["S"]) <= 1e-5 * o["S"], i
        assert np.abs(out[3][1][i].reshape(g.labels.shape) - o["field"]).max() < 1e-4 * np.abs(o["field"]).max()


def test_column_planes_option(lb):
    """Columns of 1, 2 and 4 of the 8 planes give the same bits as the
    prefetching form; a length that does not divide nz is refused."""
    rng = np.random.default_rng(23)
    labels = rng.integers(0, 3, size=(8, 12, 32)).astype(np.int32)
    pol = np.array([0, 1, 2], np.uint8)
    args = ([2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.05, 0.02)
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, 0.02, (0.3, -0.5, 0.81))
    _, ref, _ = _run(lb, labels, pol, (0, 0, 0), *args, f, gG, 1)
    for zc in (1, 2, 4):
        s = lb.Solver(0)
        s.set_option(lb.OPT_KERNEL, 2)
        s.set_option(lb.OPT_STAGE_OWN_Z, 3)
        s.set_option(lb.OPT_COLUMN_PLANES, zc)
        s.set_geometry(labels, pol, 0.5, (0, 0, 0))
        s.set_phases(args[0], args[1])
        s.set_permeability(args[2])
        s.set_sequence(args[3], f, gG)
        fld = torch.zeros(labels.size, dtype=torch.complex64, device="cuda")
        s.run(field=fld)
        torch.cuda.synchronize()
        assert s.get_option(lb.OPT_STAGE_OWN_Z_USED) == 3
        s.close()
        assert np.array_equal(fld.cpu().numpy().reshape(labels.shape), ref), zc
    s = lb.Solver(0)
    for bad in (-1, 3, 128):
        with pytest.raises(lb.LbmbtError):
            s.set_option(lb.OPT_COLUMN_PLANES, bad)
    s.set_option(lb.OPT_KERNEL, 2)
    s.set_option(lb.OPT_STAGE_OWN_Z, 3)
    s.set_option(lb.OPT_COLUMN_PLANES, 16)
    s.set_geometry(labels, pol, 0.5, (0, 0, 0))
    s.set_phases(args[0], args[1])
    s.set_sequence(args[3], f, gG)
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -1
    s.close()


def test_option_range(lb):
    s = lb.Solver(0)
    with pytest.raises(lb.LbmbtError):
        s.set_option(lb.OPT_STAGE_OWN_Z, 4)
    with pytest.raises(lb.LbmbtError):
        s.set_option(lb.OPT_STAGE_OWN_Z, -1)
    assert s.get_option(lb.OPT_STAGE_OWN_Z) == 0
    assert s.get_option(lb.OPT_STAGE_OWN_Z_USED) == 0
    s.close()
