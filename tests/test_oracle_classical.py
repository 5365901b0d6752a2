"""Pins of the oracle's classical LBM scheme (the paper's comparison scheme:
the reaction as a source term in the collision, Appendix A, Eq. A12; no
reaction step), checked against things other than the oracle itself:

* the operator assembled link by link (refs.brute_state, scheme
  "classical") on tiny grids, to 1e-13;
* the exact discrete decay of a uniform field without gradient: the source
  is a forward-Euler step of dM/dt = -M/T2, so S = (1 - dt/T2)^K;
* without gradient and T2 the source vanishes and the scheme is the hybrid
  scheme bit for bit;
* the paper's comparison (Sec. 3.2, Fig. 5): from a uniform initial field
  in a periodic square, the hybrid scheme's result does not depend on the
  square's size L, the classical scheme's error grows with L (Eqs. A14,
  A15: the source's truncation scales with (gamma L |G0|)^2), and at equal
  resolution the hybrid is the more accurate;
* the classical scheme converges to the continuum exp(-bD) under refinement
  (dt ~ dx^2).
"""
import math

import numpy as np
import pytest

import oracle
import refs

INF = math.inf


def _pattern(shape, kind):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(range(nz), range(ny), range(nx), indexing="ij")
    if kind == "split_x":
        return (x >= nx // 2).astype(np.int32)
    if kind == "split_z":
        return (z >= 1).astype(np.int32)
    return ((x + y + z) % 3).astype(np.int32)


BRUTE = [
    ((2, 2, 3), "split_x", [0, 0, 0], (0.3, 0.2, -0.1), 0.5, "D3Q7"),
    ((2, 3, 4), "checker", [0, 0, 0], (0.2, -0.4, 0.3), 0.2, "D3Q7"),
    ((2, 2, 4), "split_x", [1, 0, 0], (0.4, 0.0, 0.0), 0.3, "D3Q7"),
    ((3, 2, 2), "split_z", [0, 1, 1], (0.0, 0.0, -0.35), 0.0, "D3Q7"),
    ((2, 2, 4), "split_x", [0, 1, 0], (0.3, 0.0, 0.2), INF, "D3Q7"),
    ((1, 3, 4), "checker", [0, 0, 0], (0.25, -0.3, 0.0), 0.4, "D2Q5"),
    ((1, 4, 3), "split_x", [1, 1, 0], (0.0, 0.3, 0.0), 0.6, "D2Q5"),
]


@pytest.mark.parametrize("case", range(len(BRUTE)))
def test_classical_oracle_matches_brute_force_operator(case):
    """Membranes, periodic wraps, mirror faces (normal and parallel
    gradient), oblique gradients, both lattices, arbitrary waveforms."""
    shape, kind, bc, gG, kappa, lattice = BRUTE[case]
    lab = _pattern(shape, kind)
    pol = np.array([0, 1, 1], np.uint8)[: lab.max() + 1]
    D, T2 = [1.3, 0.6], [30.0, 12.0]
    f = np.array([1, 1, 0.5, 0, 0, -1, -1.5, 0.25, -0.25, 1, -1, 0.7])
    o = oracle.run(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, want_state=True, lattice=lattice,
                   scheme="classical")
    ref = refs.brute_state(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, lattice=lattice, scheme="classical")
    q = 5 if lattice == "D2Q5" else 7
    np.testing.assert_allclose(o["state"][..., :q], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", range(12))
def test_classical_oracle_matches_brute_force_on_random_grids(seed):
    """Seeded random tiny grids: axes of 1-4 nodes, random faces, labels,
    phases, kappa and waveform; the gradient as the mirror rule allows."""
    rng = np.random.default_rng(5000 + seed)
    shape = tuple(int(v) for v in rng.integers(1, 5, size=3))
    n_lab = int(rng.integers(1, 4))
    lab = rng.integers(0, n_lab, size=shape).astype(np.int32)
    pol = rng.integers(0, 2, size=n_lab).astype(np.uint8)
    bc = [int(v) for v in rng.integers(0, 2, size=3)]
    mirror = [a for a in range(3) if bc[a] == 1]
    if mirror and rng.random() < 0.5:
        gG = np.zeros(3)
        gG[int(rng.choice(mirror))] = rng.uniform(-0.4, 0.4)
    else:
        gG = rng.uniform(-0.4, 0.4, size=3)
        gG[mirror] = 0.0
    kappa = [0.0, float(rng.uniform(0.05, 1.0)), INF][int(rng.integers(0, 3))]
    D, T2 = list(rng.uniform(0.3, 2.0, size=2)), [float(rng.uniform(5.0, 50.0)), INF]
    f = np.round(rng.uniform(-1.5, 1.5, size=int(rng.integers(4, 11))), 2)
    o = oracle.run(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, want_state=True, scheme="classical")
    ref = refs.brute_state(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, scheme="classical")
    np.testing.assert_allclose(o["state"], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 1, 1]])
def test_classical_uniform_decay_is_the_euler_step(bc):
    """G = 0, one phase (several compartments, permeable membranes): the
    field stays uniform and each collision multiplies it by 1 - dt/T2, the
    forward-Euler step of the source (Eq. A12 with R = -1/T2)."""
    rng = np.random.default_rng(3)
    lab = rng.integers(0, 4, size=(4, 5, 6)).astype(np.int32)
    pol = np.zeros(4, np.uint8)
    dt, T2, K = 0.05, 7.0, 40
    o = oracle.run(lab, 0.7, pol, bc, [1.1], [T2], 0.08, dt, np.zeros(K), [0.0, 0.0, 0.0], scheme="classical",
                   want_field=True)
    want = (1.0 - dt / T2) ** K
    assert o["S"] == pytest.approx(want, rel=1e-13)
    np.testing.assert_allclose(o["field"], want, rtol=1e-13, atol=0)
    # and the hybrid scheme decays by the exact exp(-dt/T2) per step instead
    h = oracle.run(lab, 0.7, pol, bc, [1.1], [T2], 0.08, dt, np.zeros(K), [0.0, 0.0, 0.0])
    assert h["S"] == pytest.approx(math.exp(-K * dt / T2), rel=1e-13)


@pytest.mark.parametrize("lattice", ["D3Q7", "D2Q5"])
def test_classical_equals_hybrid_without_gradient_and_t2(lattice):
    """R = 0: the source vanishes, so the two schemes are the same scheme."""
    rng = np.random.default_rng(11)
    shape = (3, 5, 4) if lattice == "D3Q7" else (1, 6, 5)
    lab = rng.integers(0, 3, size=shape).astype(np.int32)
    pol = np.array([0, 1, 0], np.uint8)
    args = (lab, 0.9, pol, [0, 1, 0], [1.4, 0.7], [INF, INF], 0.05, 0.07, np.ones(20), [0.0, 0.0, 0.0])
    a = oracle.run(*args, want_state=True, lattice=lattice)
    b = oracle.run(*args, want_state=True, lattice=lattice, scheme="classical")
    assert np.array_equal(a["state"], b["state"])


# ------------------------------------------- the paper's L-dependence (Fig. 5)
D_FREE = 2.0


def _uniform_square(L, dx, scheme, b=1000.0, delta=3.0, Delta=6.0, tau=0.6):
    """Uniform initial field in a periodic square of side L (D2Q5), PGSE
    along x run to the echo; returns (S, relative L2 error of the field
    against the continuum exp(-bD), which is uniform at the echo)."""
    n = int(round(L / dx))
    m = math.ceil(delta / ((tau - 0.5) * (1.0 / 3.0) * dx * dx / D_FREE))
    while abs(Delta * m / delta - round(Delta * m / delta)) > 1e-9:
        m += 1
    dt = delta / m
    gG, f = oracle.pgse(b, delta, Delta, dt, (1.0, 0.0, 0.0))
    lab = np.zeros((1, n, n), np.int32)
    o = oracle.run(lab, dx, [0], [0, 0, 0], [D_FREE], [INF], INF, dt, f, gG, lattice="D2Q5", scheme=scheme,
                   want_field=True)
    ex = math.exp(-b * 1e-3 * D_FREE)
    return o["S"], float(np.sqrt(np.mean(np.abs(o["field"] - ex) ** 2)) / ex)


def test_hybrid_is_independent_of_domain_size_and_classical_is_not():
    """Sec. 3.2: with a uniform initial condition the hybrid scheme's error
    does not depend on L; the classical scheme's grows with L (at L = 100 um
    this time step violates Eq. A15 and the classical run is far off)."""
    S20h, e20h = _uniform_square(20.0, 1.0, "hybrid")
    S100h, e100h = _uniform_square(100.0, 1.0, "hybrid")
    assert S100h == pytest.approx(S20h, rel=1e-12)
    assert e100h == pytest.approx(e20h, rel=1e-9)
    _, e20c = _uniform_square(20.0, 1.0, "classical")
    _, e100c = _uniform_square(100.0, 1.0, "classical")
    assert e100c > 100.0 * e20c
    assert e20h < e20c / 5.0


def test_classical_converges_under_refinement():
    """At L = 20 um, halving dx (dt ~ dx^2 at fixed tau) cuts the classical
    scheme's error by about 4 (second order in dx, first order in dt); the
    hybrid's falls alike and stays below it."""
    _, ec1 = _uniform_square(20.0, 1.0, "classical")
    _, ec2 = _uniform_square(20.0, 0.5, "classical")
    _, eh1 = _uniform_square(20.0, 1.0, "hybrid")
    _, eh2 = _uniform_square(20.0, 0.5, "hybrid")
    assert 3.0 < ec1 / ec2 < 6.0
    assert 3.0 < eh1 / eh2 < 6.0
    assert eh2 < ec2
