"""Pins of the oracle's theta = 0 membrane rule with a per-link membrane
position (Eqs. B4a-B4c with the coefficients of Eqs. c_n and c_d), against
what the paper and the mathematics fix: the reduction to the half-link rule
(Eq. B5) at Delta_m = 1/2, the impermeable limit (Li et al.'s Neumann rule,
B = 0), a uniform magnetisation staying uniform, the mirror symmetry of the
rule, and second-order convergence to the continuum for walls that do not
sit on half-links (where the half-link rule, which moves each wall to the
nearest half-link, converges only at first order)."""
import math

import numpy as np
import pytest

import oracle
import refs
from paper_1907_00908_gb300 import synth

INF = math.inf


def _cn(d):
    return np.array([1.0, -(2 * d - 1) / (2 * d + 1), (2 * d - 1) / (2 * d + 1), 2 / (2 * d + 1)])


def test_coefficients_reduce_to_half_link_and_neumann():
    dt, dx = 0.02, 0.5
    for kap in (0.0, 0.01, 0.3, 7.0):
        _, r, s = oracle.params(1.0, dt, dx, kap)
        A, B = oracle.link_coefficients(0.5, kap, dt, dx)
        np.testing.assert_allclose(A, [r, 0, 0], atol=1e-15)
        np.testing.assert_allclose(B, [s, 0, 0], atol=1e-15)
    # impermeable: Li et al.'s Neumann (bounce-back) rule, nothing crosses
    for d in (0.1, 0.37, 0.8):
        A, B = oracle.link_coefficients(d, 0.0, dt, dx)
        np.testing.assert_allclose(A, _cn(d)[:3], atol=1e-15)
        np.testing.assert_allclose(B, 0.0, atol=1e-15)


def test_coefficients_keep_a_uniform_field():
    """sum_j A_j + sum_j B_j = 1 for any position and permeability (a uniform
    magnetisation carries no flux, so it must pass the membrane unchanged)."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = rng.uniform(0.01, 0.99)
        kap = 10 ** rng.uniform(-3, 1)
        A, B = oracle.link_coefficients(d, kap, 0.01, 0.5)
        assert abs(A.sum() + B.sum() - 1.0) < 1e-13


def _random_case(shape, seed):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 3, size=shape).astype(np.int32)
    nz, ny, nx = shape
    # consistent positions: delta_j(x) = 1 - delta_jbar(x + e_j)
    dl = np.empty((6,) + shape)
    for j, (ax, sg) in enumerate([(2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1)]):
        if sg > 0:
            dl[j] = rng.uniform(0.05, 0.95, size=shape)
    for j, (ax, sg) in enumerate([(2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1)]):
        if sg < 0:
            dl[j] = 1.0 - np.roll(dl[j - 1], 1, axis=ax)
    return lab, np.array([0, 1, 2], np.uint8), dl


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (0, 1, 0)])
def test_half_position_equals_half_link_rule(bc):
    lab, pol, _ = _random_case((5, 4, 6), 1)
    dl = np.full((6,) + lab.shape, 0.5)
    gdir = {(0, 0, 0): (0.6, 0.8, 0.0), (1, 1, 1): (0, 0, 1), (0, 1, 0): (1, 0, 0)}[bc]
    gG, f = oracle.pgse(1200.0, 0.2, 0.4, 0.02, gdir)
    args = (lab, 0.5, pol, bc, [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.05, 0.02, f, gG)
    a = oracle.run(*args, want_field=True)
    b = oracle.run(*args, want_field=True, delta=dl)
    np.testing.assert_allclose(b["field"], a["field"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
@pytest.mark.parametrize("kappa", [0.0, 0.02, 1.0])
def test_uniform_field_is_a_fixed_point(bc, kappa):
    """G = 0, T2 = inf: M = 1 stays 1 everywhere, whatever the membrane
    positions (every compartment boundary carries no flux)."""
    lab, pol, dl = _random_case((5, 6, 4), 2)
    o = oracle.run(lab, 0.5, pol, bc, [2.0, 1.0, 1.5], [INF] * 3, kappa, 0.02, np.zeros(30), [0, 0, 0],
                   want_field=True, delta=dl)
    np.testing.assert_allclose(o["field"], 1.0, rtol=0, atol=1e-12)


def test_mirror_image_geometry_gives_mirror_image_field():
    """Reflecting labels and membrane positions in x (x -> -x on a periodic
    axis, G along y) reflects the field: the rule treats both sides alike."""
    lab, pol, dl = _random_case((3, 4, 7), 3)
    gG, f = oracle.pgse(1500.0, 0.2, 0.4, 0.02, (0, 1, 0))
    args = (pol, (0, 0, 0), [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.05, 0.02, f, gG)
    a = oracle.run(lab, 0.5, *args, want_field=True, delta=dl)
    # node x -> (-x) mod n: roll so node 0 stays node 0
    flip = lambda v: np.roll(v[..., ::-1], 1, axis=-1)
    dlr = dl.copy()
    dlr[0], dlr[1] = flip(dl[1]), flip(dl[0])
    for j in range(2, 6):
        dlr[j] = flip(dl[j])
    b = oracle.run(flip(lab), 0.5, *args, want_field=True, delta=dlr)
    np.testing.assert_allclose(b["field"], flip(a["field"]), rtol=0, atol=1e-12)


def test_impermeable_slab_field_with_wall_positions():
    """Two impermeable walls at 3.17 um and 10.47 um (a slab 7.3 um wide, off
    the half-links) on a 20 um periodic axis, PGSE normal to them: the field
    at the echo inside the slab against the continuum Neumann-mode propagator
    (refs.slab_field, sampled at the nodes) -- with the walls' positions the
    error falls with dx and ends well below the half-link rule's, which moves
    each wall to the nearest half-link."""
    L, a, D, b, delta, Delta = 20.0, 7.3, 2.0, 1000.0, 2.0, 6.0
    w0 = 3.17
    el, eh = [], []
    for N in (20, 40, 80):
        dx = L / N
        dt = 0.25 * dx * dx * 0.4 / D
        dt = delta / round(delta / dt)
        gG, f = oracle.pgse(b, delta, Delta, dt, (1, 0, 0))
        g = synth.walls(N, dx, [w0, w0 + a], axis=0)
        dl = synth.link_distances(g, (0, 0, 0))
        xk = np.arange(N) * dx
        ins = (xk >= w0) & (xk < w0 + a)
        Mref = refs.slab_field(a, D, gG[0], f, dt, xk[ins] - w0)
        args = (g.labels, dx, g.phase_of_label, [0, 0, 0], [D], [INF], 0.0, dt, f, gG)
        o = oracle.run(*args, delta=dl, want_field=True)
        h = oracle.run(*args, want_field=True)
        el.append(np.abs(o["field"][0, 0][ins] - Mref).max())
        eh.append(np.abs(h["field"][0, 0][ins] - Mref).max())
    assert el[2] < 0.5 * el[1] < 0.5 * el[0]
    assert el[2] < 0.25 * eh[2]


def test_exchange_field_with_membrane_position():
    """One permeable membrane (kappa = 0.1 um/ms) 4.23 um from the left mirror
    wall (off the half-links), compartments with different D and T2, G = 0:
    the field at t = 10 ms against a fine finite-volume solution of the
    continuum flux condition (Eq. permeability_flux, refs.exchange_field) --
    the error with the membrane's position falls at about 2nd order and is a
    small fraction of the half-link rule's."""
    a1, D1, D2, T21, T22, kap, t_end = 4.23, 1.0, 2.0, 20.0, 80.0, 0.1, 10.0
    el, eh = [], []
    for m in (4, 8, 16, 32):
        dx = 4.0 / m
        n = int(round(10.0 / dx))
        a2 = n * dx - a1
        dt = 0.25 * dx * dx * 0.4 / D2
        dt = t_end / math.ceil(t_end / dt)
        # mirror wall at -dx/2: the membrane sits at x = a1 - dx/2
        g = synth.walls(n, dx, [a1 - dx / 2], axis=0, periodic=False)
        dl = synth.link_distances(g, (1, 0, 0))
        pol = np.array([0, 1], np.uint8)
        f = np.zeros(int(round(t_end / dt)))
        Mref = refs.exchange_field(a1, a2, D1, D2, T21, T22, kap, t_end, np.arange(n) * dx + dx / 2)
        args = (g.labels, dx, pol, [1, 0, 0], [D1, D2], [T21, T22], kap, dt, f, [0, 0, 0])
        o = oracle.run(*args, delta=dl, want_field=True)
        h = oracle.run(*args, want_field=True)
        el.append(np.abs(o["field"][0, 0] - Mref).max())
        eh.append(np.abs(h["field"][0, 0] - Mref).max())
    assert el[0] / el[2] > 16.0 and el[3] < el[2]
    assert el[2] < 0.1 * eh[2] and el[3] < 0.1 * eh[3]
