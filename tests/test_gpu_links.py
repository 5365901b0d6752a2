"""GPU parity of the membrane rule with per-link membrane positions (theta =
0, Eqs. B4a-B4c) against the FP64 oracle: S within 1e-5 relative, field
within 1e-4 of max|M|.  Random compartments with random consistent
positions (dense membranes, periodic / mirror / mixed faces, finite and zero
permeability, second neighbours across the faces), spheres and walls with
their exact positions, the half-position and infinite-permeability limits,
and the calls that must refuse positions."""
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
AXES = [(2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1)]   # numpy axis, sign of +x -x +y -y +z -z


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _random_positions(shape, seed, lo=0.05, hi=0.95):
    rng = np.random.default_rng(seed)
    dl = np.empty((6,) + shape, np.float32)
    for j, (ax, sg) in enumerate(AXES):
        if sg > 0:
            dl[j] = rng.uniform(lo, hi, size=shape)
    for j, (ax, sg) in enumerate(AXES):
        if sg < 0:
            dl[j] = 1.0 - np.roll(dl[j - 1], 1, axis=ax)
    return dl


def _gpu(lb, labels, pol, dx, bc, D, T2, kap, dt, f, gG, dl, kernel=0):
    s = lb.Solver(0)
    s.set_option(lb.OPT_KERNEL, kernel)
    s.set_geometry(labels, pol, dx, bc)
    s.set_link_distances(dl)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    fld = torch.zeros(labels.size, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    used = s.get_option(lb.OPT_KERNEL_USED)
    s.close()
    return r, fld.cpu().numpy().reshape(labels.shape), used


def _check(lb, labels, pol, dx, bc, D, T2, kap, dt, f, gG, dl):
    r, fld, used = _gpu(lb, labels, pol, dx, bc, D, T2, kap, dt, f, gG, dl)
    assert used == 1
    o = oracle.run(labels, dx, pol, bc, D, T2, kap, dt, f, gG, want_field=True, delta=dl.astype(np.float64))
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"], (r["S"], o["S"])
    err = np.abs(fld - o["field"]).max() / np.abs(o["field"]).max()
    assert err < FIELD_TOL, err
    return r, fld, o


CASES = {
    "periodic_oblique": dict(bc=(0, 0, 0), d=(0.6, -0.5, 0.62), kap=0.05),
    "periodic_impermeable": dict(bc=(0, 0, 0), d=(0.0, 0.8, 0.6), kap=0.0),
    "mirror_Gz": dict(bc=(1, 1, 1), d=(0.0, 0.0, 1.0), kap=0.05),
    "mixed_Gx": dict(bc=(0, 1, 1), d=(1.0, 0.0, 0.0), kap=0.2),
}


@pytest.mark.parametrize("shape", [(7, 9, 12), (5, 7, 32)])
@pytest.mark.parametrize("name", list(CASES))
def test_random_positions_match_oracle(lb, name, shape):
    c = CASES[name]
    rng = np.random.default_rng(5)
    labels = rng.integers(0, 3, size=shape).astype(np.int32)
    pol = np.array([0, 1, 2], np.uint8)
    dl = _random_positions(shape, 6)
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, 0.02, c["d"])
    _check(lb, labels, pol, 0.5, c["bc"], [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], c["kap"], 0.02, f, gG, dl)


@pytest.mark.parametrize("n", [20, 32])
def test_sphere_pack_exact_positions(lb, n):
    g = synth.spheres(n, 0.5, rmin=1.2, rmax=2.5, fraction=0.35, seed=9)
    dl = synth.link_distances(g, (0, 0, 0))
    gG, f = oracle.pgse(2000.0, 0.4, 0.8, 0.02, (0.3, 0.5, 0.81))
    _check(lb, g.labels, g.phase_of_label, g.dx, (0, 0, 0), [2.0, 1.0], [80.0, 50.0], 0.03, 0.02, f, gG, dl)


@pytest.mark.parametrize("n", [24, 32])
def test_walls_exact_positions_mirror(lb, n):
    g = synth.walls(n, 0.5, [2.13, 5.61, 9.02], axis=0, cross=(4, 6), periodic=False, phases=[0, 1])
    dl = synth.link_distances(g, (1, 0, 0))
    gG, f = oracle.pgse(1500.0, 0.4, 0.8, 0.02, (1.0, 0.0, 0.0))
    _check(lb, g.labels, g.phase_of_label, g.dx, (1, 0, 0), [2.0, 1.0], [80.0, 50.0], 0.05, 0.02, f, gG, dl)


def test_half_positions_equal_half_link_rule(lb):
    shape = (6, 8, 10)
    rng = np.random.default_rng(7)
    labels = rng.integers(0, 3, size=shape).astype(np.int32)
    pol = np.array([0, 1, 2], np.uint8)
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, 0.02, (0.6, 0.8, 0.0))
    args = (labels, pol, 0.5, (0, 0, 0), [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.05, 0.02, f, gG)
    a, fa, _ = _gpu(lb, *args, np.full((6,) + shape, 0.5, np.float32))
    b, fb, _ = _gpu(lb, *args, None, kernel=1)
    assert np.abs(fa - fb).max() < 1e-6 * np.abs(fb).max()
    assert abs(a["S"] - b["S"]) < 1e-6 * b["S"]


def test_infinite_permeability_ignores_positions(lb):
    shape = (6, 8, 16)
    rng = np.random.default_rng(8)
    labels = rng.integers(0, 3, size=shape).astype(np.int32)
    pol = np.array([0, 1, 2], np.uint8)
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, 0.02, (0.6, 0.8, 0.0))
    args = (labels, pol, 0.5, (0, 0, 0), [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], INF, 0.02, f, gG)
    _, fa, _ = _gpu(lb, *args, _random_positions(shape, 9), kernel=1)
    _, fb, _ = _gpu(lb, *args, None, kernel=1)
    assert np.array_equal(fa, fb)


def test_positions_refused_where_unsupported(lb):
    shape = (4, 4, 16)
    labels = (np.arange(np.prod(shape)).reshape(shape) % 2).astype(np.int32)
    pol = np.array([0, 1], np.uint8)
    s = lb.Solver(0)
    s.set_geometry(labels, pol, 0.5, (0, 0, 0))
    with pytest.raises(lb.LbmbtError) as e:
        s.set_link_distances(np.full((6,) + shape, 1.5, np.float32))
    assert e.value.code == -1
    s.set_link_distances(_random_positions(shape, 1))
    s.set_phases([2.0, 1.0], [INF, INF])
    s.set_permeability(0.05)
    gG, f = oracle.pgse(500.0, 0.2, 0.4, 0.02, (1, 0, 0))
    s.set_sequence(0.02, f, gG)
    s.set_option(lb.OPT_KERNEL, 2)
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -1
    s.set_option(lb.OPT_KERNEL, 0)
    s.run()
    assert s.get_option(lb.OPT_KERNEL_USED) == 1
    with pytest.raises(lb.LbmbtError) as e:
        s.grad()
    assert e.value.code == -5
    s.set_link_distances(None)
    s.run()
    assert s.get_option(lb.OPT_KERNEL_USED) == 2
    s.close()


def test_batch_mixes_members_with_and_without_positions(lb):
    """One launch over three members: a sphere pack with its exact positions,
    the same pack without (half-link rule), and random compartments with
    random positions and a finite kappa of their own; each member against its
    own oracle run, and the per-step series of the first against the
    oracle's."""
    g1 = synth.spheres(16, 0.5, rmin=1.2, rmax=2.2, fraction=0.35, seed=4)
    dl1 = synth.link_distances(g1, (0, 0, 0))
    rng = np.random.default_rng(12)
    lab2 = rng.integers(0, 3, size=(6, 8, 12)).astype(np.int32)
    g2 = synth.Geometry(lab2, np.array([0, 1, 1], np.uint8), 0.5)
    dl2 = _random_positions(lab2.shape, 13)
    D, T2, dt = [2.0, 1.0], [80.0, 50.0], 0.02
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, dt, (0.3, 0.5, 0.81))
    gG2 = np.array([0.0, 0.0, 1.0]) * np.linalg.norm(gG)
    s = lb.Solver(0)
    s.set_geometry(g1.labels, g1.phase_of_label, g1.dx, (0, 0, 0))
    s.add_geometry(g1.labels, g1.phase_of_label, g1.dx, (0, 0, 0))
    s.add_geometry(g2.labels, g2.phase_of_label, g2.dx, (0, 0, 0))
    s.set_link_distances(dl1, index=0)
    s.set_link_distances(dl2, index=2)
    s.set_phases(D, T2)
    s.set_sequence(dt, f, gG)
    mem = lb.Solver.members([gG, gG, gG2], [0, 1, 2], [0.03, 0.03, 0.1])
    r = s.run_batch(mem, series=True)
    s.close()
    cases = [(g1, dl1, gG, 0.03), (g1, None, gG, 0.03), (g2, dl2, gG2, 0.1)]
    for m, (g, dl, gv, kap) in enumerate(cases):
        o = oracle.run(g.labels, g.dx, g.phase_of_label, (0, 0, 0), D, T2, kap, dt, f, gv, want_series=(m == 0),
                       delta=None if dl is None else dl.astype(np.float64))
        assert abs(r["S"][m] - o["S"]) <= S_TOL * o["S"], (m, r["S"][m], o["S"])
        if m == 0:
            err = np.abs(r["series"][0] - o["series"]).max() / np.abs(o["series"]).max()
            assert err < 1e-5, err


def test_uniform_field_stays_uniform_over_a_long_run(lb):
    """G = 0, T2 = inf: M = 1 is a fixed point of the rule (its coefficients
    sum to one); in FP32 over 6400 steps on cylinders with their exact
    positions the field must stay within 1e-6 of 1 (no systematic drift from
    the rounded coefficients)."""
    g = synth.cylinders(48, 0.5, seed=1)
    dl = synth.link_distances(g, (0, 0, 0))
    for kap in (0.0, 0.02, 1.0):
        s = lb.Solver(0)
        s.set_option(lb.OPT_KERNEL, 1)
        s.set_geometry(g.labels, g.phase_of_label, g.dx, (0, 0, 0))
        s.set_link_distances(dl)
        s.set_phases([2.0, 1.0], [INF, INF])
        s.set_permeability(kap)
        s.set_sequence(0.00625, np.zeros(6400), [0.0, 0.0, 0.0])
        fld = torch.zeros(g.n_sites, dtype=torch.complex64, device="cuda")
        r = s.run(field=fld)
        torch.cuda.synchronize()
        s.close()
        assert np.abs(fld.cpu().numpy() - 1).max() < 1e-6, kap
        assert abs(r["S"] - 1.0) < 1e-8, kap
