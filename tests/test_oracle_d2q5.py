"""Pins of the oracle's 2-D D2Q5 lattice (Sec. 2.3: velocities 0, +-x, +-y,
eps_D = 1/3, omega_0 = 1/3, omega_1..4 = 1/6): the plane-wave closed form of
the five-velocity scheme, convergence of free diffusion to exp(-b D) (which
fails for a wrong eps_D), conservation of the summed magnetisation with
membranes, restricted diffusion between impermeable planes converging to
the continuum Neumann-mode propagator, and equality with the five-velocity
operator assembled link by link on random tiny grids."""
import math

import numpy as np
import pytest

import oracle
import refs
from paper_1907_00908_gb300 import synth

INF = math.inf


@pytest.mark.parametrize("b", [0.0, 500.0, 2000.0])
@pytest.mark.parametrize("direction", [(1, 0, 0), (0.6, -0.8, 0.0)])
def test_d2q5_free_diffusion_equals_planewave_recurrence(b, direction):
    n, dx, D, T2, dt = (1, 10, 12), 1.0, 2.0, 60.0, 0.05
    gG, f = oracle.pgse(b, 2.0, 5.0, dt, direction)
    geom = synth.uniform(n, dx)
    o = oracle.run(geom.labels, dx, geom.phase_of_label, (0, 0, 0), [D], [T2], INF, dt, f, gG, lattice="D2Q5",
                   want_series=True)
    S_ref, ser = refs.planewave_signal((12, 10, 1), dx, D, T2, dt, f, gG, series=True, lattice="D2Q5")
    assert o["S"] == pytest.approx(S_ref, rel=1e-12, abs=1e-15)
    np.testing.assert_allclose(o["series"] / geom.n_sites, ser, rtol=0, atol=1e-12)


def test_d2q5_converges_to_exp_bD():
    """tau = 0.8 fixed, dx halved, dt = (tau - 1/2) eps_D dx^2 / D with
    eps_D = 1/3: S -> exp(-b D) (G along the diagonal of the plane)."""
    D, b, delta, Delta = 2.0, 1000.0, 2.0, 6.0
    errs = []
    for m in (1, 2, 4):
        dx = 1.0 / m
        dt = 0.3 * (1 / 3) * dx * dx / D
        dt = delta / round(delta / dt)
        gG, f = oracle.pgse(b, delta, Delta, dt, (1, 1, 0))
        geom = synth.uniform((1, 16 * m, 16 * m), dx)
        o = oracle.run(geom.labels, dx, geom.phase_of_label, (0, 0, 0), [D], [INF], INF, dt, f, gG, lattice="D2Q5")
        errs.append(abs(o["S"] - math.exp(-b * 1e-3 * D)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 2e-3


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0)])
def test_d2q5_conservation_with_membranes(bc):
    rng = np.random.default_rng(3)
    lab = rng.integers(0, 3, size=(1, 9, 11)).astype(np.int32)
    o = oracle.run(lab, 0.5, np.array([0, 1, 2], np.uint8), bc, [2.0, 1.0, 1.5], [INF] * 3, 0.05, 0.02,
                   np.zeros(40), [0, 0, 0], lattice="D2Q5", want_field=True)
    assert abs(o["Z"] - lab.size) < 1e-10 * lab.size
    # and M = 1 is a fixed point
    np.testing.assert_allclose(o["field"], 1.0, rtol=0, atol=1e-12)


def test_d2q5_impermeable_planes_converge_to_continuum():
    a, D, b, delta, Delta = 8.0, 2.0, 2000.0, 2.0, 6.0
    errs = []
    for m in (8, 16, 32):
        dx = a / m
        dt = 0.4 * (1 / 3) * dx * dx / D
        dt = delta / round(delta / dt)
        gG, f = oracle.pgse(b, delta, Delta, dt, (1, 0, 0))
        geom = synth.planes((1, 3, 2 * m), dx, [m], axis=0)
        o = oracle.run(geom.labels, dx, geom.phase_of_label, (0, 0, 0), [D], [INF], 0.0, dt, f, gG, lattice="D2Q5")
        errs.append(abs(o["S"] - refs.slab_signal(a, D, gG[0], f, dt)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 2e-3


def test_d2q5_needs_one_plane():
    with pytest.raises(ValueError):
        oracle.run(np.zeros((2, 4, 4), np.int32), 1.0, np.zeros(1, np.uint8), (0, 0, 0), [1.0], [INF], INF, 0.05,
                   np.zeros(3), [0, 0, 0], lattice="D2Q5")


@pytest.mark.parametrize("seed", range(16))
def test_d2q5_matches_brute_force_operator_on_random_grids(seed):
    """The oracle's D2Q5 mode equals the five-velocity operator assembled
    link by link (refs.brute_state with lattice="D2Q5") on seeded random
    one-plane grids, to 1e-13. The grids have 1 to 5 nodes per in-plane axis,
    periodic or mirror faces, random labels and phases, and kappa of 0,
    finite or infinite. Gradients lie in the plane as the mirror rule
    allows. The oracle's z slots stay exactly zero."""
    rng = np.random.default_rng(2000 + seed)
    shape = (1,) + tuple(int(v) for v in rng.integers(1, 6, size=2))
    n_lab = int(rng.integers(2, 4))
    lab = rng.integers(0, n_lab, size=shape).astype(np.int32)
    pol = rng.integers(0, 2, size=n_lab).astype(np.uint8)
    bc = [int(v) for v in rng.integers(0, 2, size=3)]
    mirror = [a for a in range(2) if bc[a] == 1]
    gG = np.zeros(3)
    if mirror and rng.random() < 0.5:
        gG[int(rng.choice(mirror))] = rng.uniform(-0.4, 0.4)
    else:
        gG[:2] = rng.uniform(-0.4, 0.4, size=2)
        gG[mirror] = 0.0
    kappa = [0.0, float(rng.uniform(0.05, 1.0)), INF][int(rng.integers(0, 3))]
    D, T2 = list(rng.uniform(0.3, 2.0, size=2)), [float(rng.uniform(5.0, 50.0)), INF]
    f = np.round(rng.uniform(-1.5, 1.5, size=int(rng.integers(4, 11))), 2)
    f[rng.random(f.size) < 0.2] = 0.0
    o = oracle.run(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, want_state=True, lattice="D2Q5")
    ref = refs.brute_state(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, lattice="D2Q5")
    np.testing.assert_allclose(o["state"][..., :5], ref, rtol=0, atol=1e-13)
    assert not np.any(o["state"][..., 5:])
