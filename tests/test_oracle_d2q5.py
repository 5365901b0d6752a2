"""Pins of the oracle's 2-D D2Q5 lattice (Sec. 2.3: velocities 0, +-x, +-y,
eps_D = 1/3, omega_0 = 1/3, omega_1..4 = 1/6): the plane-wave closed form of
the five-velocity scheme, convergence of free diffusion to exp(-b D) (which
fails for a wrong eps_D), conservation of the summed magnetisation with
membranes, and restricted diffusion between impermeable planes converging to
the continuum Neumann-mode propagator."""
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
