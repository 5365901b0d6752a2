"""GPU batches through the C ABI against per-member FP64 oracle runs.

* A batch over several geometries whose edges are multiples of 16, so that
  the whole launch runs on the bulk-copy sweep (the configuration the
  batched benchmark times): each member's signal and field against its own
  oracle run, and the register sweep's fields bit for bit.
* A batch whose members carry their own PGSE waveforms with different
  diffusion times (delta, Delta) and so different echo times (Sec. 2.1,
  Fig. 2), through lbmbt_run_batch_ex: each member's signal and field at
  its own echo against its own oracle run, on both sweeps, with and
  without the per-step series.

Tolerances: S within 1e-5 relative, the field within 1e-4 of max|M|.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S_TOL = 1e-5
FIELD_TOL = 1e-4
INF = math.inf
D, T2 = [2.0, 1.0], [80.0, 50.0]


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _geoms():
    return [synth.cylinders(32, 0.5, seed=4),
            synth.spheres(48, 0.5, rmin=2.0, rmax=4.0, fraction=0.45, seed=12),
            synth.spheres(16, 0.5, rmin=1.0, rmax=1.8, fraction=0.3, seed=13),
            synth.cylinders(64, 0.5, seed=2)]


def _field_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _solver(lb, geoms, bcs, dt, f, gG0, kernel):
    s = lb.Solver(0)
    s.set_option(lb.OPT_KERNEL, kernel)
    for i, (g, bc) in enumerate(zip(geoms, bcs)):
        if i == 0:
            s.set_geometry(g.labels, g.phase_of_label, g.dx, bc)
        else:
            s.add_geometry(g.labels, g.phase_of_label, g.dx, bc)
    s.set_phases(D, T2)
    s.set_sequence(dt, f, gG0)
    return s


def test_multi_geometry_batch_on_the_bulk_copy_sweep(lb):
    """Four geometries (32^3, 48^3, 16^3, 64^3 at dx 0.5 um; periodic and
    mirror faces), seven members with different directions, b-values and
    kappa (0, finite, infinite), in one launch per step."""
    geoms = _geoms()
    bcs = [(0, 0, 0), (1, 1, 1), (0, 0, 0), (0, 1, 0)]
    dt = 0.025
    _, f = oracle.pgse(1000.0, 1.0, 3.0, dt, (1, 0, 0))
    spec = [  # geometry, b, direction, kappa
        (0, 1500.0, (0.6, 0.0, 0.8), 0.02), (0, 800.0, (0.0, 1.0, 0.0), 0.0),
        (1, 2000.0, (0.0, 0.0, 1.0), 0.05), (1, 1200.0, (1.0, 0.0, 0.0), INF),
        (2, 3000.0, (0.3, -0.5, 0.8), 0.01), (3, 2500.0, (0.6, 0.0, 0.8), 0.03),
        (3, 1000.0, (0.8, 0.0, 0.6), 0.02)]
    gGs = [oracle.pgse(b, 1.0, 3.0, dt, d)[0] for _, b, d, _ in spec]
    out = {}
    for kernel in (2, 1):
        s = _solver(lb, geoms, bcs, dt, f, gGs[0], kernel)
        mem = lb.Solver.members(gGs, [g for g, *_ in spec], [k for *_, k in spec])
        flds = [torch.zeros(geoms[g].n_sites, dtype=torch.complex64, device="cuda") for g, *_ in spec]
        r = s.run_batch(mem, fields=flds)
        torch.cuda.synchronize()
        assert s.get_option(lb.OPT_KERNEL_USED) == kernel
        s.close()
        out[kernel] = (r, [fl.cpu().numpy() for fl in flds])
    for i, (gi, _, _, kap) in enumerate(spec):
        geom = geoms[gi]
        o = oracle.run(geom.labels, geom.dx, geom.phase_of_label, bcs[gi], D, T2, kap, dt, f, gGs[i],
                       want_field=True)
        r, flds = out[2]
        assert abs(r["S"][i] - o["S"]) <= S_TOL * o["S"], i
        assert _field_err(flds[i].reshape(geom.labels.shape), o["field"]) < FIELD_TOL, i
        assert np.array_equal(flds[i], out[1][1][i]), i


# (delta, Delta) pairs in ms at dt = 0.025 ms: echo times 3, 4, 6 and 3.5 ms
TIMINGS = [(1.0, 2.0), (1.0, 3.0), (2.0, 4.0), (0.5, 3.0)]


@pytest.mark.parametrize("kernel,series", [(2, False), (1, False), (2, True)])
def test_batch_mixes_diffusion_times(lb, kernel, series):
    """Members with their own PGSE timings (and so their own echoes) in one
    batch: each member's signal and field at its echo equal its own oracle
    run; members without a waveform take the set one."""
    geoms = _geoms()[:2]
    bcs = [(0, 0, 0), (0, 0, 0)]
    dt = 0.025
    waves, gGs, geo, kaps = [], [], [], []
    dirs = synth.directions_on_sphere(len(TIMINGS) + 1, seed=3)
    for j, (dl, Dl) in enumerate(TIMINGS):
        gG, fj = oracle.pgse(1500.0 + 300.0 * j, dl, Dl, dt, dirs[j])
        waves.append(fj)
        gGs.append(gG)
        geo.append(j % 2)
        kaps.append([0.02, 0.05, 0.0, 0.01][j])
    longest = max(waves, key=len)
    # one more member with no waveform of its own: it takes the set one
    gGs.append(oracle.pgse(1000.0, 2.0, 4.0, dt, dirs[-1])[0])
    waves.append(None)
    geo.append(1)
    kaps.append(0.02)
    s = _solver(lb, geoms, bcs, dt, longest, gGs[0], kernel)
    mem = lb.Solver.members(gGs, geo, kaps)
    flds = [torch.zeros(geoms[g].n_sites, dtype=torch.complex64, device="cuda") for g in geo]
    r = s.run_batch(mem, series=series, waveforms=waves, fields=flds)
    torch.cuda.synchronize()
    assert s.get_option(lb.OPT_KERNEL_USED) == kernel
    s.close()
    for i in range(len(gGs)):
        geom = geoms[geo[i]]
        fi = longest if waves[i] is None else waves[i]
        o = oracle.run(geom.labels, geom.dx, geom.phase_of_label, bcs[geo[i]], D, T2, kaps[i], dt, fi, gGs[i],
                       want_field=True, want_series=series)
        assert abs(r["S"][i] - o["S"]) <= S_TOL * o["S"], i
        assert _field_err(flds[i].cpu().numpy().reshape(geom.labels.shape), o["field"]) < FIELD_TOL, i
        if series:
            ser = r["series"][i][:len(fi)]
            np.testing.assert_allclose(ser, o["series"], rtol=0, atol=S_TOL * np.abs(o["series"]).max())


def test_member_waveform_refusals(lb):
    geom = synth.cylinders(32, 0.5, seed=4)
    gG, f = oracle.pgse(1000.0, 1.0, 2.0, 0.025, (1, 0, 0))
    s = _solver(lb, [geom], [(0, 0, 0)], 0.025, f, gG, 0)
    mem = lb.Solver.members([gG], 0, 0.02)
    for bad in (np.ones(len(f) + 1), np.array([1.0, math.nan])):
        with pytest.raises(lb.LbmbtError) as e:
            s.run_batch(mem, waveforms=[bad])
        assert e.value.code == -1
    with pytest.raises(ValueError):
        s.run_batch(mem, fields=[torch.zeros(geom.n_sites - 1, dtype=torch.complex64, device="cuda")])
    r = s.run_batch(mem, waveforms=[f[:40]])
    assert math.isfinite(r["S"][0])
    s.close()
