"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: a number printed in the paper
(``tests/golden``), a closed form of the scheme, an invariant, a limit that
reduces to a textbook solution, or an independent implementation of the same
equations (``refs.py``).  All run on the CPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import refs
from paper_1907_00908_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = math.inf


def _run(geom, bc, D, T2, kappa, dt, f, gG, **kw):
    return oracle.run(geom.labels, geom.dx, geom.phase_of_label, bc, D, T2, kappa, dt, f, gG, **kw)


# ------------------------------------------------------------------ golden
def test_tau_matches_paper_3d_run():
    """Sec. 3.7 (Fig. 14 caption): the paper's 3-D D3Q7 code ran with
    D = 2.0 um^2/ms, dt = 0.010 ms, dx = 1.0 um and tau = 0.58.  This pins
    eps_D = 1/4 for D3Q7 (eps_D = 1/3 would give 0.56)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    c = g["tau_3d_scaling_run"]
    tau, _, _ = oracle.params(c["D"], c["dt"], c["dx"], 1.0)
    assert tau == pytest.approx(c["tau"], abs=5e-3)
    assert abs(tau - c["tau"]) < abs(0.5 + c["dt"] * c["D"] / (c["dx"] ** 2 / 3.0) - c["tau"])


def test_membrane_shares_limits():
    """Eq. B5 / P_def: r + s = 1; kappa -> inf gives streaming (s = 1),
    kappa -> 0 gives bounce-back (r = 1); P = eps_D dx/(2 kappa dt)."""
    _, r, s = oracle.params(1.0, 0.00625, 0.5, 0.02)
    P = 0.25 * 0.5 / (2 * 0.02 * 0.00625)
    assert P == pytest.approx(500.0)
    assert r == pytest.approx(P / (1 + P), rel=1e-15) and s == pytest.approx(1 / (1 + P), rel=1e-15)
    assert oracle.params(1.0, 0.01, 1.0, INF)[1:] == (0.0, 1.0)
    assert oracle.params(1.0, 0.01, 1.0, 0.0)[1:] == (1.0, 0.0)


def test_pgse_b_value():
    """Sec. 2.1: b = gamma^2 |G0|^2 delta^2 (Delta - delta/3); f = +1, then -1."""
    gG, f = oracle.pgse(1000.0, 5.0, 20.0, 0.0125, (1, 0, 0))
    assert len(f) == 2000 and f.sum() == 0.0
    assert f[:400].min() == 1 and f[1600:].max() == -1 and not f[400:1600].any()
    b = gG[0] ** 2 * 25.0 * (20.0 - 5.0 / 3.0)
    assert b == pytest.approx(1.0, rel=1e-14)
    assert gG[0] == pytest.approx(0.04671, abs=1e-5)
    with pytest.raises(ValueError):
        oracle.pgse(1000.0, 5.003, 20.0, 0.0125)


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("b", [0.0, 250.0, 1000.0, 2000.0])
@pytest.mark.parametrize("direction", [(1, 0, 0), (1, 2, -2)])
def test_free_diffusion_equals_planewave_recurrence(b, direction):
    """Uniform periodic medium: the lattice solution is exactly a plane wave,
    so the oracle's S equals the 7-vector recurrence (refs.planewave_signal)."""
    n, dx, D, T2, dt = 8, 1.0, 2.0, 60.0, 0.05
    gG, f = oracle.pgse(b, 2.0, 5.0, dt, direction)
    geom = synth.uniform(n, dx)
    o = _run(geom, [0, 0, 0], [D], [T2], INF, dt, f, gG, want_series=True)
    S_ref, ser_ref = refs.planewave_signal(n, dx, D, T2, dt, f, gG, series=True)
    assert o["S"] == pytest.approx(S_ref, rel=1e-12, abs=1e-15)
    np.testing.assert_allclose(o["series"] / geom.n_sites, ser_ref, rtol=0, atol=1e-12)


def test_b0_gives_pure_t2_decay():
    """G = 0: M(t) = exp(-t/T2) everywhere (Sec. 3.1 uniform-IC case)."""
    geom = synth.cylinders(32, 1.0, fraction=0.5, seed=3)
    gG, f = oracle.pgse(0.0, 2.0, 6.0, 0.05)
    o = _run(geom, [0, 0, 0], [1.0, 2.0], [40.0, 40.0], 0.05, 0.05, f, gG, want_field=True)
    np.testing.assert_allclose(o["field"], math.exp(-len(f) * 0.05 / 40.0), rtol=1e-12)


def test_free_diffusion_converges_to_exp_bD():
    """Sec. 3.1 (Fig. 5): with a uniform IC the exact Bloch-Torrey solution is
    S = exp(-bD); the hybrid scheme is 2nd order in dx and 1st in dt, so
    refining dx by 2 at fixed tau (dt by 4) cuts the error about 4x.
    Uses the recurrence (pinned to the oracle above) for the fine grids."""
    D, b = 2.0, 1000.0
    errs = []
    for dx in (2.0, 1.0, 0.5):
        dt = 0.1 * (dx / 2.0) ** 2 / 1.0
        dt = 5.0 / round(5.0 / dt)
        gG, f = oracle.pgse(b, 5.0, 20.0, dt, (1, 0, 0))
        S = refs.planewave_signal(int(round(40 / dx)), dx, D, INF, dt, f, gG)
        errs.append(abs(S - math.exp(-b * 1e-3 * D)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 2e-3


# ----------------------------------------------------------- brute force
CASES = [
    # (shape nz,ny,nx), labels pattern, bc, gG, kappa
    ((2, 2, 3), "split_x", [0, 0, 0], (0.3, 0.2, -0.1), 0.5),
    ((2, 3, 4), "checker", [0, 0, 0], (0.2, -0.4, 0.3), 0.2),
    ((2, 2, 4), "split_x", [1, 0, 0], (0.4, 0.0, 0.0), 0.3),
    ((2, 3, 3), "checker", [1, 1, 0], (0.0, 0.0, 0.25), 0.7),
    ((3, 2, 2), "split_z", [0, 1, 1], (0.0, 0.0, -0.35), 0.0),
    ((2, 2, 4), "split_x", [0, 1, 0], (0.3, 0.0, 0.2), INF),
]


def _pattern(shape, kind):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(range(nz), range(ny), range(nx), indexing="ij")
    if kind == "split_x":
        lab = (x >= nx // 2).astype(np.int32)
    elif kind == "split_z":
        lab = (z >= 1).astype(np.int32)
    else:
        lab = ((x + y + z) % 3).astype(np.int32)
    return lab


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_matches_brute_force_operator(case):
    """The oracle's final state equals the operator assembled link by link
    (refs.brute_state) on tiny grids with membranes, periodic wraps, mirror
    faces (normal and parallel gradient) and oblique G, to 1e-13."""
    shape, kind, bc, gG, kappa = CASES[case]
    lab = _pattern(shape, kind)
    pol = np.array([0, 1, 1], np.uint8)[: lab.max() + 1]
    D, T2 = [1.3, 0.6], [30.0, 12.0]
    dt, dx = 0.1, 0.8
    f = np.array([1, 1, 0.5, 0, 0, -1, -1.5, 0.25, -0.25, 1, -1, 0.7])
    o = oracle.run(lab, dx, pol, bc, D, T2, kappa, dt, f, gG, want_state=True)
    ref = refs.brute_state(lab, dx, pol, bc, D, T2, kappa, dt, f, gG)
    np.testing.assert_allclose(o["state"], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", range(24))
def test_oracle_matches_brute_force_operator_on_random_grids(seed):
    """The same comparison on seeded random tiny grids.
    * Axes of 1 to 4 nodes, each face periodic or mirror.
    * 1 to 3 labels with random phases, so membranes fall anywhere, including
      across a wrap.
    * kappa of 0, finite or infinite.
    * Arbitrary waveform values.
    * A gradient drawn as the mirror rule (Sec. 2.4.4) allows: either along
      one mirror normal, or anywhere in the periodic axes."""
    rng = np.random.default_rng(1000 + seed)
    shape = tuple(int(v) for v in rng.integers(1, 5, size=3))
    n_lab = int(rng.integers(1, 4)) if seed % 4 == 0 else int(rng.integers(2, 4))
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
    f[rng.random(f.size) < 0.2] = 0.0
    o = oracle.run(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG, want_state=True)
    ref = refs.brute_state(lab, 0.8, pol, bc, D, T2, kappa, 0.1, f, gG)
    np.testing.assert_allclose(o["state"], ref, rtol=0, atol=1e-13)


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 1, 1], [1, 0, 1]])
@pytest.mark.parametrize("kappa", [0.0, 0.03, INF])
def test_conservation_without_gradient_and_t2(bc, kappa):
    """G = 0, T2 = inf: BGK keeps sum_i g_i per site (sum w = 1) and the
    membrane split r + s = 1 keeps the total, so sum_x M is conserved, and
    M = 1 everywhere is a fixed point (Eq. g_eq, Eq. B5)."""
    geom = synth.spheres(16, 1.0, rmin=2.0, rmax=4.0, fraction=0.4, seed=5)
    f = np.zeros(60)
    o = _run(geom, bc, [1.0, 2.5], [INF, INF], kappa, 0.05, f, [0, 0, 0], want_field=True)
    assert abs(o["Z"] - geom.n_sites) < 1e-11 * geom.n_sites
    np.testing.assert_allclose(o["field"], 1.0, atol=1e-13)


def test_g0_impermeable_compartment_decay():
    """kappa = 0, G = 0: compartments do not exchange and stay uniform, so
    S = sum_p f_p exp(-TE/T2_p) exactly (f_p: lattice volume fractions)."""
    geom = synth.cylinders(24, 1.0, fraction=0.5, seed=11)
    f = np.zeros(200)
    dt = 0.05
    o = _run(geom, [0, 0, 0], [1.0, 2.0], [50.0, 80.0], 0.0, dt, f, [0, 0, 0])
    fr = geom.phase_fractions(2)
    TE = len(f) * dt
    expect = fr[0] * math.exp(-TE / 50.0) + fr[1] * math.exp(-TE / 80.0)
    assert o["S"] == pytest.approx(expect, rel=1e-12)


def test_infinite_permeability_equals_no_membrane():
    """Eq. permeability_BC: kappa -> inf (P -> 0) reduces to plain streaming,
    so a multi-label geometry at kappa = inf with equal phases equals the
    single-label run bit for bit."""
    geom = synth.cylinders(16, 1.0, fraction=0.5, seed=2)
    gG, f = oracle.pgse(800.0, 2.0, 4.0, 0.05, (1, 1, 0))
    a = _run(geom, [0, 0, 0], [1.5, 1.5], [70.0, 70.0], INF, 0.05, f, gG, want_field=True)
    one = synth.uniform(16, 1.0)
    b = _run(one, [0, 0, 0], [1.5], [70.0], INF, 0.05, f, gG, want_field=True)
    assert np.array_equal(a["field"], b["field"])


def test_periodic_translation_invariance():
    """A periodic shift of the geometry only multiplies M by a global phase
    exp(-i gG.s F(t)), which is 1 at the echo: Z is unchanged."""
    geom = synth.cylinders(20, 1.0, fraction=0.5, seed=4)
    gG, f = oracle.pgse(1500.0, 2.0, 5.0, 0.05, (0.6, 0.8, 0.0))
    a = _run(geom, [0, 0, 0], [1.0, 2.0], [50.0, 80.0], 0.03, 0.05, f, gG)
    shifted = synth.Geometry(np.roll(geom.labels, (3, 5, 7), axis=(0, 1, 2)), geom.phase_of_label, 1.0)
    b = _run(shifted, [0, 0, 0], [1.0, 2.0], [50.0, 80.0], 0.03, 0.05, f, gG)
    assert abs(a["Z"] - b["Z"]) < 1e-12 * abs(a["Z"])


def test_z_invariance_for_z_aligned_cylinders():
    """Sec. 3.5 (Fig. 13): z-aligned cylinders with periodic BCs give no z
    dependence at TE even for an oblique gradient."""
    geom = synth.cylinders(20, 1.0, fraction=0.5, seed=9)
    geom = synth.Geometry(np.ascontiguousarray(geom.labels[:5]), geom.phase_of_label, 1.0)
    gG, f = oracle.pgse(1000.0, 2.0, 5.0, 0.05, (1, 1, 1))
    o = _run(geom, [0, 0, 0], [1.5, 2.0], [30.0, 10.0], 0.01, 0.05, f, gG, want_field=True)
    M = o["field"]
    assert np.abs(M - M[0:1]).max() < 1e-12 * np.abs(M).max()


@pytest.mark.parametrize("gdir", [(1, 0, 0), (0, 1, 0)])
def test_mirror_equals_doubled_periodic_domain(gdir):
    """Sec. 2.4.4: a mirror boundary reflects the domain across the face.
    The run on N with mirror faces along x must equal, on its N nodes, the
    modified-periodic run on the explicitly mirrored 2N domain, for G normal
    (conjugate rule) and parallel (plain swap) to the face."""
    geom = synth.cylinders(12, 1.0, fraction=0.5, seed=13)
    lab = np.ascontiguousarray(np.roll(geom.labels, 2, axis=2)[:4])
    doubled = np.ascontiguousarray(np.concatenate([lab, lab[:, :, ::-1]], axis=2))
    gG, f = oracle.pgse(1200.0, 2.0, 5.0, 0.05, gdir)
    pol = geom.phase_of_label
    a = oracle.run(lab, 1.0, pol, [1, 0, 0], [1.0, 2.0], [50.0, 80.0], 0.04, 0.05, f, gG, want_field=True)
    b = oracle.run(doubled, 1.0, pol, [0, 0, 0], [1.0, 2.0], [50.0, 80.0], 0.04, 0.05, f, gG, want_field=True)
    np.testing.assert_allclose(a["field"], b["field"][:, :, :12], rtol=0, atol=1e-12)


# ----------------------------------------------------- restricted diffusion
@pytest.mark.parametrize("Delta", [3.0, 12.0])
def test_impermeable_slabs_converge_to_continuum(Delta):
    """Impermeable planes a = 8 um apart (kappa = 0, G normal): the oracle
    converges at 2nd order in dx to the continuum Neumann-mode propagator
    (refs.slab_signal)."""
    a, D, b, delta = 8.0, 2.0, 2000.0, 2.0
    errs = []
    for m in (8, 16, 32):
        dx = a / m
        dt = 0.25 * dx * dx * 0.4 / D     # tau = 0.9
        dt = delta / round(delta / dt)
        gG, f = oracle.pgse(b, delta, Delta, dt, (1, 0, 0))
        geom = synth.planes((1, 1, 2 * m), dx, [m], axis=0)
        o = _run(geom, [0, 0, 0], [D], [INF], 0.0, dt, f, gG)
        S_ref = refs.slab_signal(a, D, gG[0], f, dt)
        errs.append(abs(o["S"] - S_ref))
    assert errs[2] < 0.02 * errs[0] + 1e-9 or (errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0)
    assert errs[2] < 2e-3


def test_slab_reference_matches_sgp_diffraction():
    """Pin of the continuum reference itself: narrow pulses and long Delta
    give the SGP diffraction formula E = 2(1 - cos qa)/(qa)^2 (Sec. 3.6)."""
    a, D = 5.0, 2.3
    dt = 0.001
    delta, Delta = 0.002, 40.0
    for qa in (1.0, 3.0, 2 * math.pi):
        q = qa / a
        gG = q / delta
        f = np.zeros(int(round((Delta + delta) / dt)))
        f[:2] = 1.0
        f[int(round(Delta / dt)):int(round(Delta / dt)) + 2] = -1.0
        E = refs.slab_signal(a, D, gG, f, dt, n_modes=60)
        expect = 2 * (1 - math.cos(qa)) / qa ** 2
        assert E == pytest.approx(expect, abs=2e-3)


def test_slab_reference_matches_mitra_short_time_limit():
    """Pin of the continuum reference at short times: narrow pulses, low q,
    sqrt(D Delta) << a -- the apparent diffusivity -ln E / (q^2 (Delta -
    delta/3)) follows Mitra's surface-to-volume law 1 - D_app/D =
    4/(3 sqrt(pi)) (S/V) sqrt(D Delta) with S/V = 2/a for a slab (flat walls:
    no curvature term at the next order)."""
    a, D, q, dt, nd = 20.0, 2.0, 0.01, 0.0005, 2
    for Delta in (0.25, 1.0, 4.0):
        gG = q / (nd * dt)
        n = int(round(Delta / dt))
        f = np.zeros(n + nd)
        f[:nd] = 1.0
        f[n:n + nd] = -1.0
        E = refs.slab_signal(a, D, gG, f, dt, n_modes=300)
        dev = 1.0 - (-math.log(E) / (q * q * (Delta - nd * dt / 3))) / D
        mitra = 4.0 / (3.0 * math.sqrt(math.pi)) * (2.0 / a) * math.sqrt(D * Delta)
        assert dev == pytest.approx(mitra, rel=3e-3)


def test_slab_reference_matches_gaussian_phase_long_pulse_limit():
    """Pin of the continuum reference in the motional-narrowing regime: pulses
    much longer than a^2/D, with little phase per correlation time (gG a^3/D
    small), give a Gaussian phase whose variance follows from the slab's
    position autocorrelation C(tau) = sum over odd n of 8 a^2/(n pi)^4
    exp(-(n pi)^2 D tau/a^2), so that int C = a^4/(120 D) and
    int tau C = 17 a^6/(20160 D^2).  For PGSE with Delta - delta >> a^2/D
    the two pulses decorrelate and -ln E = 2 gG^2 (delta int C - int tau C).
    The next cumulant is smaller by (gG a^3/D)^2: the deviation must fall
    with it."""
    a, D, dt = 2.0, 2.0, 1.0
    i0, i1 = a ** 4 / (120 * D), 17 * a ** 6 / (20160 * D ** 2)
    devs, pars = [], []
    for delta, gG in ((500.0, 0.06), (2000.0, 0.03), (2000.0, 0.015)):
        n = int(round(delta / dt))
        f = np.zeros(3 * n)
        f[:n] = 1.0
        f[2 * n:] = -1.0
        E = refs.slab_signal(a, D, gG, f, dt, n_modes=60)
        expect = -2 * gG ** 2 * (delta * i0 - i1)
        devs.append(abs(math.log(E) / expect - 1))
        pars.append(gG * a ** 3 / D)
    assert max(devs) < 1e-4
    for j in (1, 2):   # quadratic fall-off with the narrowing parameter
        ratio = (devs[0] / devs[j]) / (pars[0] / pars[j]) ** 2
        assert 0.5 < ratio < 2.0, (devs, pars)


def test_exchange_reference_matches_karger_limit():
    """Pin of the exchange reference: for kappa a/D << 1 the compartments are
    well mixed and the Karger two-compartment ODE holds."""
    S = refs.exchange_signal(4.0, 6.0, 2.0, 1.0, 30.0, 80.0, 0.005, 40.0)
    K = refs.karger_signal(4.0, 6.0, 2.0, 1.0, 30.0, 80.0, 0.005, 40.0)
    assert S == pytest.approx(K, rel=2e-4)


def test_two_compartment_exchange_converges():
    """One planar permeable membrane between compartments of widths a1, a2
    (mirror walls outside, G = 0, different T2 and D): the oracle's S
    converges at 2nd order to the continuum flux condition of
    Eq. permeability_flux (refs.exchange_signal)."""
    a1, a2, D1, D2, T21, T22, kap = 4.0, 6.0, 1.0, 2.0, 20.0, 80.0, 0.1
    t_end = 10.0
    S_ref = refs.exchange_signal(a1, a2, D1, D2, T21, T22, kap, t_end, n_cells=2000)
    errs = []
    for m in (4, 8, 16):
        dx = a1 / m
        dt = 0.25 * dx * dx * 0.4 / D2
        dt = t_end / math.ceil(t_end / dt)
        n1, n2 = m, int(round(a2 / dx))
        lab = np.zeros((1, 1, n1 + n2), np.int32)
        lab[..., n1:] = 1
        pol = np.array([0, 1], np.uint8)
        f = np.zeros(int(round(t_end / dt)))
        o = oracle.run(lab, dx, pol, [1, 0, 0], [D1, D2], [T21, T22], kap, dt, f, [0, 0, 0])
        errs.append(abs(o["S"] - S_ref))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


# ------------------------------------------------------------------- mask
def test_oracle_mask_matches_numpy_definition():
    """Bit (i-1) set iff the neighbour across +e_i exists (periodic wraps,
    mirror faces do not) and carries a different label; bits 6-7 = phase."""
    rng = np.random.default_rng(0)
    lab = rng.integers(0, 4, size=(5, 6, 7)).astype(np.int32)
    pol = np.array([0, 1, 2, 3], np.uint8)
    for bc in ([0, 0, 0], [1, 0, 1], [1, 1, 1]):
        m = oracle.mask(lab, pol, bc)
        exp = (pol[lab].astype(np.uint16) << 6)
        for i, (ax, sh) in enumerate([(2, -1), (2, 1), (1, -1), (1, 1), (0, -1), (0, 1)]):
            nb = np.roll(lab, sh, axis=ax)
            diff = nb != lab
            a = {2: 0, 1: 1, 0: 2}[ax]
            if bc[a] == 1:
                idx = [slice(None)] * 3
                idx[ax] = -1 if sh == -1 else 0
                diff[tuple(idx)] = False
            exp |= diff.astype(np.uint16) << i
        assert np.array_equal(m, exp.astype(np.uint8))


# ------------------------------------------------------ sampled checking
@pytest.mark.parametrize("gdir,bc", [((1, 0, 0), (1, 1, 1)), ((0, 0, 1), (1, 1, 1)), ((0.6, 0.8, 0.0), (0, 0, 0))])
def test_crop_sampling_reproduces_full_run(gdir, bc):
    """The crop method used for full-size GPU checks (cropcheck.py) gives
    the full run's values at interior, face and corner sites."""
    import cropcheck
    geom = synth.crop(synth.voronoi_tissue(64, 0.5, cell_diam=6.0, vessel_radius=2.0, seed=21), 36)
    dt, k = 0.025, 6
    gG, f = oracle.pgse(1500.0, 1.0, 2.0, dt, gdir)
    D, T2, kap = [1.0, 2.5, 3.0], [50.0, 80.0, 80.0], 0.03
    full = oracle.run(geom.labels, geom.dx, geom.phase_of_label, bc, D, T2, kap, dt, f[:k], gG, want_field=True)
    sites = [(18, 17, 16), (0, 0, 0), (0, 20, 11), (12, 0, 25), (20, 19, 0), (2, 28, 3),
             (35, 35, 35), (35, 10, 0), (4, 34, 17), (0, 35, 33), (30, 2, 35)]
    vals = cropcheck.sample_values(geom.labels, geom.phase_of_label, bc, geom.dx, D, T2, kap, dt, f, gG, sites, k)
    ref = np.array([full["field"][s] for s in sites])
    np.testing.assert_allclose(vals, ref, rtol=0, atol=1e-13)
