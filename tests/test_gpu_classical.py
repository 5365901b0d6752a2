"""GPU parity of the classical LBM scheme (the paper's comparison scheme:
the reaction as a source term in the collision, Appendix A, Eq. A12)
through the C ABI, against the FP64 oracle's classical scheme.

Tolerances as for the hybrid scheme: S within 1e-5 relative, the field
within 1e-4 of max|M|.  Cases: both lattices, periodic, mirror (gradient
normal and parallel to the faces) and mixed faces, membranes with kappa 0,
finite and infinite, ragged tile tails, several launch shapes, and a
128^3 cylinder pack on a short schedule.  Grids the bulk-copy sweep takes
(nx a multiple of 16) run on both sweeps, whose fields agree bit for bit.
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


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _gpu(lb, geom, bc, D, T2, kap, dt, f, gG, lattice=0, block=None, spt=None, series=False, kernel=1):
    s = lb.Solver(0)
    s.set_option(lb.OPT_SCHEME, 1)
    s.set_option(lb.OPT_LATTICE, lattice)
    s.set_option(lb.OPT_KERNEL, kernel)
    if block:
        s.set_option(lb.OPT_BLOCK, block)
    if spt:
        s.set_option(lb.OPT_SPT, spt)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld, series=series)
    torch.cuda.synchronize()
    used = s.get_option(lb.OPT_KERNEL_USED)
    assert used == kernel if kernel else used == (2 if geom.labels.shape[2] % 16 == 0 and lattice == 0 else 1)
    s.close()
    return r, fld.cpu().numpy().reshape(geom.labels.shape)


def _oracle(geom, bc, D, T2, kap, dt, f, gG, lattice="D3Q7", **kw):
    return oracle.run(geom.labels, geom.dx, geom.phase_of_label, bc, D, T2, kap, dt, f, gG, want_field=True,
                      lattice=lattice, scheme="classical", **kw)


def _check(r, fld, o):
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"], (r["S"], o["S"])
    err = float(np.abs(fld - o["field"]).max() / np.abs(o["field"]).max())
    assert err < FIELD_TOL, err


CASES = [
    # geometry, bc, gradient direction, kappa
    (lambda: synth.cylinders(24, 1.0, fraction=0.5, seed=3), (0, 0, 0), (1, 1, 0), 0.05),
    (lambda: synth.spheres(20, 1.0, rmin=2.0, rmax=3.5, fraction=0.45, seed=4), (0, 0, 0), (0.3, -0.5, 0.8), 0.02),
    (lambda: synth.crop(synth.voronoi_tissue(40, 0.5, cell_diam=6.0, vessel_radius=1.5, seed=2), 22), (1, 1, 1),
     (0, 0, 1), 0.01),
    (lambda: synth.crop(synth.voronoi_tissue(40, 0.5, cell_diam=6.0, vessel_radius=1.5, seed=2), 22), (1, 1, 1),
     (1, 0, 0), 0.0),
    (lambda: synth.spheres(18, 1.0, rmin=2.0, rmax=3.0, fraction=0.4, seed=9), (1, 0, 0), (0, 0.6, 0.8), INF),
    # nx a multiple of 16: both sweeps
    (lambda: synth.cylinders(32, 1.0, fraction=0.5, seed=6), (0, 0, 0), (0.6, -0.48, 0.64), 0.05),
    (lambda: synth.crop(synth.voronoi_tissue(48, 0.5, cell_diam=6.0, vessel_radius=1.5, seed=8), 32), (1, 1, 1),
     (0, 0, 1), 0.01),
    (lambda: synth.crop(synth.voronoi_tissue(48, 0.5, cell_diam=6.0, vessel_radius=1.5, seed=8), 32), (1, 0, 1),
     (0, 1, 0), 0.02),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_classical_matches_oracle_d3q7(lb, case):
    mk, bc, d, kap = CASES[case]
    geom = mk()
    nph = int(geom.phase_of_label.max()) + 1
    D = [2.0, 1.0, 3.0][:max(nph, 2)]
    T2 = [80.0, 50.0, 80.0][:max(nph, 2)]
    gG, f = oracle.pgse(1500.0, 2.0, 5.0, 0.05, d)
    r, fld = _gpu(lb, geom, bc, D, T2, kap, 0.05, f, gG)
    _check(r, fld, _oracle(geom, bc, D, T2, kap, 0.05, f, gG))
    if geom.labels.shape[2] % 16 == 0:   # the bulk-copy sweep: the same bits
        r2, fld2 = _gpu(lb, geom, bc, D, T2, kap, 0.05, f, gG, kernel=2)
        assert np.array_equal(fld, fld2)
        assert r2["S"] == pytest.approx(r["S"], rel=1e-7)


@pytest.mark.parametrize("bc,d", [((0, 0, 0), (0.6, 0.8, 0.0)), ((1, 1, 0), (1.0, 0.0, 0.0)),
                                  ((0, 1, 0), (1.0, 0.0, 0.0))])
def test_classical_matches_oracle_d2q5(lb, bc, d):
    geom = synth.disks(40, 0.5, [[5.3, 6.1], [14.8, 13.2], [4.9, 15.7]], [3.6, 4.1, 2.4])
    D, T2, kap, dt = [2.0, 1.0], [80.0, 50.0], 0.05, 0.02
    gG, f = oracle.pgse(2000.0, 0.4, 1.0, dt, d)
    r, fld = _gpu(lb, geom, bc, D, T2, kap, dt, f, gG, lattice=1)
    _check(r, fld, _oracle(geom, bc, D, T2, kap, dt, f, gG, lattice="D2Q5"))


@pytest.mark.parametrize("block,spt", [(64, 1), (128, 4), (512, 2)])
def test_classical_launch_shapes_and_ragged_tails(lb, block, spt):
    """A grid whose site count is not a multiple of any tile, random labels
    (membranes on most links), an arbitrary waveform, the signal after every
    step against the oracle's series."""
    rng = np.random.default_rng(44)
    lab = rng.integers(0, 3, size=(5, 7, 13)).astype(np.int32)
    geom = synth.Geometry(lab, np.array([0, 1, 0], np.uint8), 0.6)
    f = np.round(rng.uniform(-1.0, 1.0, size=60), 3)
    gG = [0.09, -0.05, 0.04]
    D, T2, kap, dt = [1.5, 0.8], [40.0, 25.0], 0.1, 0.04
    r, fld = _gpu(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG, block=block, spt=spt, series=True)
    o = _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG, want_series=True)
    _check(r, fld, o)
    ser = np.asarray(r["series"])
    np.testing.assert_allclose(ser, o["series"], rtol=0, atol=S_TOL * np.abs(o["series"]).max())


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_classical_own_z_forms_agree(lb, bc):
    """The classical pass on the bulk-copy sweep in its three own-z forms
    (prefetched, staged, z-marching): the same bits, and the oracle."""
    geom = synth.crop(synth.voronoi_tissue(48, 0.5, cell_diam=6.0, vessel_radius=1.5, seed=8), 32)
    D, T2, kap, dt = [2.0, 1.0, 3.0], [80.0, 50.0, 80.0], 0.02, 0.05
    gG, f = oracle.pgse(1500.0, 2.0, 5.0, dt, (0, 0, 1))
    out = {}
    for oz in (1, 2, 3):
        s = lb.Solver(0)
        s.set_option(lb.OPT_SCHEME, 1)
        s.set_option(lb.OPT_KERNEL, 2)
        s.set_option(lb.OPT_STAGE_OWN_Z, oz)
        s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
        s.set_phases(D, T2)
        s.set_permeability(kap)
        s.set_sequence(dt, f, gG)
        fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
        r = s.run(field=fld)
        torch.cuda.synchronize()
        assert s.get_option(lb.OPT_STAGE_OWN_Z_USED) == oz
        s.close()
        out[oz] = (r, fld.cpu().numpy().reshape(geom.labels.shape))
    for oz in (2, 3):
        assert np.array_equal(out[1][1], out[oz][1]), oz
        assert out[1][0]["S"] == out[oz][0]["S"], oz
    _check(out[3][0], out[3][1], _oracle(geom, bc, D, T2, kap, dt, f, gG))


def test_classical_equals_hybrid_bitwise_without_gradient_and_t2(lb):
    """R = 0: the source adds exact zeros, so the classical pass gives the
    hybrid pass's field bit for bit (both on the register sweep)."""
    geom = synth.cylinders(32, 0.5, seed=4)
    f = np.ones(40)
    out = []
    for scheme in (0, 1):
        s = lb.Solver(0)
        s.set_option(lb.OPT_SCHEME, scheme)
        s.set_option(lb.OPT_KERNEL, 1)
        s.set_geometry(geom.labels, geom.phase_of_label, geom.dx)
        s.set_phases([2.0, 1.0], [INF, INF])
        s.set_permeability(0.02)
        s.set_sequence(0.025, f, [0.0, 0.0, 0.0])
        fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
        s.run(field=fld)
        torch.cuda.synchronize()
        out.append(fld.cpu().numpy())
        s.close()
    assert np.array_equal(out[0], out[1])


def test_classical_cylinders_128_short_schedule(lb):
    """The 128^3 permeable-cylinder workload (dx 0.5 um, c2 phases) on the
    first 64 steps of its PGSE, G oblique, against the oracle."""
    geom = synth.cylinders(128, 0.5, seed=1)
    dt = 0.00625
    gG, f = oracle.pgse(3000.0, 10.0, 30.0, dt, (0.6, 0.0, 0.8))
    f = f[:64]
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    r, fld = _gpu(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG, kernel=0)   # auto: the bulk-copy sweep
    _check(r, fld, _oracle(geom, (0, 0, 0), D, T2, kap, dt, f, gG))


def test_classical_refusals(lb):
    geom = synth.cylinders(32, 0.5, seed=4)
    gG, f = oracle.pgse(1000.0, 1.0, 3.0, 0.025, (1, 0, 0))
    s = lb.Solver(0)
    s.set_option(lb.OPT_SCHEME, 1)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx)
    s.set_phases([2.0, 1.0], [80.0, 50.0])
    s.set_permeability(0.02)
    s.set_sequence(0.025, f, gG)
    with pytest.raises(lb.LbmbtError) as e:             # adjoint: hybrid only
        s.grad()
    assert e.value.code == -5
    s.set_link_distances(synth.link_distances(geom, (0, 0, 0)))
    with pytest.raises(lb.LbmbtError) as e:             # membrane positions: half-link rule only
        s.run()
    assert e.value.code == -5
    s.set_link_distances(None)
    s.set_sequence_substeps(0.025, np.repeat(f, 2), gG, 2)
    with pytest.raises(lb.LbmbtError) as e:             # no reaction step to sub-step
        s.run()
    assert e.value.code == -1
    s.set_sequence(0.025, f, gG)
    assert math.isfinite(s.run()["S"])
    with pytest.raises(lb.LbmbtError):
        s.set_option(lb.OPT_SCHEME, 2)
    s.close()
