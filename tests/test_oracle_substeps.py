"""Pins of the oracle's reaction sub-steps (Sec. 2.3: dt = k dt', one
diffusion step then k reaction steps): a waveform constant over each
diffusion step gives the plain run; in a uniform periodic medium the lattice
solution stays a plane wave whose wave vector advances by gG * sum_j f_j dt'
per step, so the oracle equals the 7-vector recurrence (refs.planewave_signal)
driven by the step-mean waveform -- the equivalence the library relies on;
and a PGSE whose pulse edges fall inside a diffusion step (delta = 2.5 dt)
converges to exp(-b D) as dt shrinks."""
import math

import numpy as np
import pytest

import oracle
import refs
from paper_1907_00908_gb300 import synth

INF = math.inf


def test_step_constant_waveform_equals_plain_run():
    g = synth.cylinders(16, 1.0, fraction=0.5, seed=2)
    gG, f = oracle.pgse(1500.0, 1.0, 2.0, 0.05, (0.6, 0.0, 0.8))
    args = (g.labels, g.dx, g.phase_of_label, (0, 0, 0), [1.0, 2.0], [50.0, 80.0], 0.05, 0.05)
    a = oracle.run(*args, f, gG, want_field=True)
    for k in (2, 3):
        b = oracle.run(*args, np.repeat(f, k), gG, want_field=True, substeps=k)
        np.testing.assert_allclose(b["field"], a["field"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [2, 4])
def test_substeps_equal_planewave_recurrence_with_step_mean(k):
    n, dx, D, T2, dt = 8, 1.0, 2.0, 60.0, 0.05
    rng = np.random.default_rng(k)
    K = 60
    f_fine = np.sin(np.linspace(0, 3 * np.pi, K * k)) + 0.3 * rng.standard_normal(K * k)
    gG = np.array([0.05, -0.02, 0.03])
    geom = synth.uniform(n, dx)
    o = oracle.run(geom.labels, dx, geom.phase_of_label, (0, 0, 0), [D], [T2], INF, dt, f_fine, gG, substeps=k,
                   want_series=True)
    f_mean = f_fine.reshape(K, k).mean(axis=1)
    S_ref, ser_ref = refs.planewave_signal(n, dx, D, T2, dt, f_mean, gG, series=True)
    assert o["S"] == pytest.approx(S_ref, rel=1e-12, abs=1e-15)
    np.testing.assert_allclose(o["series"] / geom.n_sites, ser_ref, rtol=0, atol=1e-12)


def test_pulse_edges_inside_a_step_converge_to_exp_bD():
    """delta = 1 ms, Delta = 4 ms with dt = delta / (n + 1/2): the pulse edges
    fall inside diffusion steps, and with k = 2 sub-steps the PGSE is exact on
    the dt' grid; S -> exp(-b D) at first order as dt -> 0 (b from the
    continuum formula, tau = 0.8 at every resolution)."""
    D, b, delta = 2.0, 1000.0, 1.0
    errs = []
    for n in (5, 11, 23):
        dt = delta / (n + 0.5)
        gG, f = oracle.pgse(b, delta, 4.0 * delta, dt / 2, (1, 0, 0))
        f = np.concatenate([f, np.zeros(len(f) % 2)])   # end on a whole step (the field is uniform by then)
        dx = math.sqrt(dt * D / (0.25 * 0.3))
        geom = synth.uniform((1, 1, 16), dx)
        o = oracle.run(geom.labels, dx, geom.phase_of_label, (0, 0, 0), [D], [INF], INF, dt, f, gG, substeps=2)
        errs.append(abs(o["S"] - math.exp(-b * 1e-3 * D)))
    assert errs[0] > 1.8 * errs[1] and errs[1] > 1.8 * errs[2]     # first order in time (Sec. 3.1)
    assert errs[2] < 0.04 * math.exp(-b * 1e-3 * D)
