"""Pins of the oracle's general-angle membrane rule (Appendix B: Eqs.
dirichlet_1-neumann_2, phi_1, phi_2, B1, B1.5, solved per link), 2-D D2Q5,
against what the paper and the mathematics fix:

* the printed closed forms of the coefficients (Eqs. B3a, B3c), which the
  oracle never evaluates (it solves the relations as a linear system);
* theta = 0 gives the Eqs. B4a-B4c rule, kappa = 0 decouples the far side;
* the coefficients sum to one (a uniform magnetisation passes unchanged);
* the rule is exact for the lattice's steady linear fields tangential to the
  membrane (hat g_i = w_i (M - (tau - 1) dx e_i . grad M)), and a flipped
  beta or a flipped x'_ii breaks that;
* runs: G = 0 keeps M = 1; on stripes at 45 degrees with a gradient along
  them the field approaches free diffusion closer than with theta = 0; the
  paper's four-variant study on a packed disc (Sec. 3.6): the full rule and
  Delta_m = 1/2 approach each other under refinement, the two theta = 0
  variants move away from them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import synth

INF = math.inf
EPS2 = 1.0 / 3.0


def _cn(d):
    return np.array([1.0, -(2 * d - 1) / (2 * d + 1), (2 * d - 1) / (2 * d + 1), 2 / (2 * d + 1)])


def _cd(d):
    return np.array([2 * (d - 1), -(2 * d - 1) ** 2 / (2 * d + 1), 2 * (2 * d - 1) / (2 * d + 1),
                     (3 - 2 * d) / (2 * d + 1)])


def _b3(dl, th, kap, dt, dx, eps=EPS2):
    """Eqs. B3a and B3c as printed (intracellular coefficients)."""
    c_n, c_d = _cn(dl), _cd(dl)
    s_n, s_d = _cn(1 - dl), _cd(1 - dl)
    p_n, p_d = _cn(0.0), _cd(0.0)
    ct, st = math.cos(th), abs(math.sin(th))
    E, K = eps * dx, kap * dt
    cd4, cn4, sd4, sn4, pd4, pn4 = c_d[3], c_n[3], s_d[3], s_n[3], p_d[3], p_n[3]
    F = (cd4 * pn4 * ct * (ct * pn4 * sd4 * E + pn4 * sn4 * K + pd4 * sn4 * E * st)
         + cn4 * (ct * pn4 * sd4 * (pn4 * K + pd4 * E * st) + pd4 * sn4 * st * (2 * pn4 * K + pd4 * E * st)))
    A = [(cd4 * pn4 * ct * (pn4 * sd4 * c_n[j] * E * ct + pn4 * sn4 * c_n[j] * K + pd4 * sn4 * c_n[j] * E * st)
          + cn4 * (ct * pn4 * sd4 * c_d[j] * (pn4 * K + pd4 * E * st)
                   + pd4 * sn4 * c_d[j] * st * (2 * pn4 * K + pd4 * E * st))) / F for j in range(3)]
    B = [cd4 * cn4 * pn4 ** 2 * K * ct * (s_n[j] - s_d[j]) / F for j in range(3)]
    C = [cd4 * cn4 * st * (p_n[j] - p_d[j]) * (pn4 * sd4 * E * ct + pn4 * sn4 * K + pd4 * sn4 * E * st) / F
         for j in range(3)]
    D = [cd4 * cn4 * sn4 * pn4 * K * st * (p_n[j] - p_d[j]) / F for j in range(3)]
    return [np.array(v) for v in (A, B, C, D)]


@pytest.mark.parametrize("dl,th,kap", [(0.3, 0.5, 0.05), (0.7, -0.9, 0.0), (0.5, 0.3, 1.0), (0.2, 1.2, 0.01),
                                       (0.93, 0.785, 0.2), (0.05, -0.2, 3.0)])
def test_coefficients_match_printed_closed_forms(dl, th, kap):
    got = oracle.angled_coefficients(dl, th, kap, 0.01, 0.5)
    want = _b3(dl, th, kap, 0.01, 0.5)
    for g, w in zip(got, want):
        np.testing.assert_allclose(g, w, rtol=1e-12, atol=1e-14)


def test_theta_zero_and_impermeable_limits():
    dt, dx = 0.01, 0.5
    for dl in (0.15, 0.5, 0.8):
        for kap in (0.0, 0.04, 2.0):
            A, B, C, D = oracle.angled_coefficients(dl, 0.0, kap, dt, dx)
            c_n, c_d, s_n, s_d = _cn(dl), _cd(dl), _cn(1 - dl), _cd(1 - dl)
            rho = kap * dt / (EPS2 * dx)
            F = c_d[3] * s_d[3] + (c_d[3] * s_n[3] + c_n[3] * s_d[3]) * rho
            A0 = (c_d[3] * s_d[3] * c_n[:3] + (s_d[3] * c_n[3] * c_d[:3] + s_n[3] * c_d[3] * c_n[:3]) * rho) / F
            B0 = c_d[3] * c_n[3] * (s_n[:3] - s_d[:3]) * rho / F
            np.testing.assert_allclose(A, A0, atol=1e-14)
            np.testing.assert_allclose(B, B0, atol=1e-14)
            np.testing.assert_allclose(C, 0.0, atol=1e-15)
            np.testing.assert_allclose(D, 0.0, atol=1e-15)
        A, B, C, D = oracle.angled_coefficients(dl, 0.6, 0.0, dt, dx)
        np.testing.assert_allclose(B, 0.0, atol=1e-15)
        np.testing.assert_allclose(D, 0.0, atol=1e-15)


def test_coefficients_sum_to_one():
    rng = np.random.default_rng(4)
    for _ in range(40):
        dl, th, kap = rng.uniform(0.02, 0.98), rng.uniform(-1.5, 1.5), 10 ** rng.uniform(-3, 1)
        A, B, C, D = oracle.angled_coefficients(dl, th, kap, 0.01, 0.5)
        assert abs(A.sum() + B.sum() + C.sum() + D.sum() - 1.0) < 1e-12


E2 = {1: (1, 0), 2: (-1, 0), 3: (0, 1), 4: (0, -1)}
OPP2 = {1: 2, 2: 1, 3: 4, 4: 3}


@pytest.mark.parametrize("flip", [None, "beta", "x_ii"])
def test_exact_for_tangential_linear_fields(flip):
    """Steady linear field M = M0 + t.x with t along the membrane: the
    lattice's populations are w (M - (tau - 1) dx e_i.t) after collision and
    w (M - tau dx e_i.t) on arrival; the rule (kappa = 0) must return the
    arriving one exactly.  The planted variants must not."""
    w, tau, dx = EPS2 / 2, 0.8, 1.0
    worst = 0.0
    for dl in (0.1, 0.3, 0.5, 0.9):
        for th in (0.4, -0.4, 1.1, -0.7):
            n = np.array([math.cos(th), math.sin(th)])      # from x's side, alpha = +x, perp = +y
            t = np.array([-n[1], n[0]]) * 0.37
            gh = lambda i, p: w * (1.0 + t @ p - (tau - 1) * dx * (np.array(E2[i]) @ t))
            i, ib = 2, 1                                     # arriving along -x at x = 0
            bet = 3 if th > 0 else 4
            if flip == "beta":
                bet = OPP2[bet]
            bb = OPP2[bet]
            ei, eb = np.array(E2[i], float), np.array(E2[bet], float)
            x = np.zeros(2)
            xm = x - dl * ei
            sg = -1.0 if flip == "x_ii" else 1.0
            a = [gh(ib, x), gh(ib, x + ei), gh(i, x)]
            y = x - ei
            b = [gh(i, y), gh(i, y - ei), gh(ib, y)]
            p = [gh(bet, xm), gh(bet, xm - sg * eb), gh(bb, xm)]
            q = [gh(bb, xm), gh(bb, xm + sg * eb), gh(bet, xm)]
            A, B, C, D = oracle.angled_coefficients(dl, th, 0.0, 0.01, dx)
            X = A @ a + B @ b + C @ p + D @ q
            exact = w * (1.0 - tau * dx * (ei @ t))
            worst = max(worst, abs(X - exact))
    if flip is None:
        assert worst < 1e-14
    else:
        assert worst > 1e-3


def _stripes(N, mode, slope=(1, 1)):
    L, D, b, delta, Delta = 20.0, 2.0, 1000.0, 2.0, 6.0
    dx = L / N
    dt = 0.1 * dx * dx / D
    dt = delta / round(delta / dt)
    g = synth.stripes(N, dx, slope, 0.45, 0.37)
    Nn = np.asarray(g.info["normal"])
    d = (Nn[1], -Nn[0], 0.0) if mode == "tan" else (0.0, 0.0, 0.0)
    gG, f = oracle.pgse(b, delta, Delta, dt, d) if mode == "tan" else (np.zeros(3), np.zeros(int(8.0 / dt)))
    dl = synth.link_distances(g, (0, 0, 0))
    th = synth.link_angles(g, (0, 0, 0))
    args = (g.labels, dx, g.phase_of_label, [0, 0, 0], [D, D], [INF, INF], 0.0, dt, f, gG)
    return args, dl, th, math.exp(-b * 1e-3 * D)


def test_uniform_field_is_a_fixed_point():
    args, dl, th, _ = _stripes(20, "zero")
    o = oracle.run(*args, delta=dl, theta=th, want_field=True, lattice="D2Q5")
    np.testing.assert_allclose(o["field"], 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("slope,ratio", [((1, 1), 0.4), ((2, 1), 0.6)])
def test_stripes_tangential_gradient_beats_theta_zero(slope, ratio):
    """Impermeable stripes at 45 degrees and at slope 1/2 (links at 26.6 and
    63.4 degrees from the normal), gradient along them: the field at the
    echo is free diffusion's exp(-bD); with the angles the error is a
    fraction of the theta = 0 rule's (which treats the staircase as walls
    normal to each link)."""
    args, dl, th, ref = _stripes(80, "tan", slope)
    full = oracle.run(*args, delta=dl, theta=th, want_field=True, lattice="D2Q5")["field"]
    t0 = oracle.run(*args, delta=dl, want_field=True, lattice="D2Q5")["field"]
    e_full, e_t0 = np.abs(full - ref).max(), np.abs(t0 - ref).max()
    assert e_full < ratio * e_t0, (e_full, e_t0)


def _disk(N):
    D, kap, b, delta, Delta, R = 2.3, 0.05, 1000.0, 5.0, 20.0, 20.0
    Lb = math.sqrt(math.pi * R * R / 0.5)
    dx = Lb / N
    dt = 0.1 * dx * dx / D
    dt = delta / math.ceil(delta / dt)
    g = synth.disks(N, dx, [[Lb / 2 + 0.123, Lb / 2 - 0.071]], [R])
    gG, f = oracle.pgse(b, delta, Delta, dt, (1, 0, 0))
    dl = synth.link_distances(g, (0, 0, 0))
    th = synth.link_angles(g, (0, 0, 0))
    args = (g.labels, dx, g.phase_of_label, [0, 0, 0], [D, D], [INF, INF], kap, dt, f, gG)
    S = {"full": oracle.run(*args, delta=dl, theta=th, lattice="D2Q5")["S"],
         "dl05": oracle.run(*args, delta=np.full_like(dl, 0.5), theta=th, lattice="D2Q5")["S"],
         "theta0": oracle.run(*args, delta=dl, lattice="D2Q5")["S"],
         "half": oracle.run(*args, lattice="D2Q5")["S"]}
    return S


def test_four_variant_disc_study():
    """Sec. 3.6's study on a 40 um disc at intracellular fraction 0.5 (D 2.3,
    kappa 0.05 um/ms, PGSE delta 5 / Delta 20, b 1000) at dx ~ 1 and 0.5 um:
    the full rule and Delta_m = 1/2 draw together, both theta = 0 variants
    draw away, and all four stay within 2 % of each other."""
    c, f = _disk(50), _disk(100)
    assert abs(f["full"] - f["dl05"]) < 0.6 * abs(c["full"] - c["dl05"])
    for k in ("theta0", "half"):
        assert abs(f["full"] - f[k]) > 1.5 * abs(c["full"] - c[k])
    vals = list(f.values())
    assert (max(vals) - min(vals)) / f["full"] < 0.02
