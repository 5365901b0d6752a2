"""GPU parity of the general-angle membrane rule (2-D, Appendix B; D2Q5 on
one z plane) against the FP64 oracle: S within 1e-5 relative, field within
1e-4 of max|M|.  Oblique stripes (slopes 1/1 and 2/1, permeable and
impermeable, gradients along and across them), disc packs with exact
positions and angles (periodic, and mirror faces where the stencil falls
back to the theta = 0 rule), random labels with random consistent
positions and angles (most links fall back: every branch runs), zero
angles equal to no angles bit for bit, and the calls that must refuse
angles."""
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
DT = 0.025   # dx 0.5, eps_D 1/3: tau = 0.5 + 0.3 D >= 0.8 for D >= 1 (the angle rule needs tau >= 0.75)
AXES = [(2, 1), (2, -1), (1, 1), (1, -1)]   # numpy axis, sign of +x -x +y -y


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _gpu(lb, geom, bc, D, T2, kap, dt, f, gG, dl, th):
    s = lb.Solver(0)
    s.set_option(lb.OPT_LATTICE, 1)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
    if dl is not None:
        s.set_link_distances(dl)
    if th is not None:
        s.set_link_angles(th)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    used = s.get_option(lb.OPT_KERNEL_USED)
    s.close()
    return r, fld.cpu().numpy().reshape(geom.shape), used


def _check(lb, geom, bc, D, T2, kap, dt, f, gG, dl, th):
    r, fld, used = _gpu(lb, geom, bc, D, T2, kap, dt, f, gG, dl, th)
    assert used == 1
    o = oracle.run(geom.labels, geom.dx, geom.phase_of_label, bc, D, T2, kap, dt, f, gG, want_field=True,
                   delta=dl.astype(np.float64), theta=th.astype(np.float64), lattice="D2Q5")
    assert abs(r["S"] - o["S"]) <= S_TOL * o["S"], (r["S"], o["S"])
    err = np.abs(fld - o["field"]).max() / np.abs(o["field"]).max()
    assert err < FIELD_TOL, err
    return r, fld, o


STRIPES = {
    "s11_perm_oblique": dict(n=32, slope=(1, 1), kap=0.05, d=(0.6, 0.8, 0.0)),
    "s11_imperm_normal": dict(n=32, slope=(1, 1), kap=0.0, d=(-0.7071, 0.7071, 0.0)),
    "s21_perm_along": dict(n=40, slope=(2, 1), kap=0.2, d=(1.0, 2.0, 0.0)),
}


@pytest.mark.parametrize("name", list(STRIPES))
def test_stripes_match_oracle(lb, name):
    c = STRIPES[name]
    g = synth.stripes(c["n"], 0.5, c["slope"], 0.45, 0.37, phases=[0, 1])
    dl, th = synth.link_distances(g, (0, 0, 0)), synth.link_angles(g, (0, 0, 0))
    assert np.count_nonzero(th) > 0
    gG, f = oracle.pgse(1500.0, 0.5, 1.0, DT, c["d"])
    _check(lb, g, (0, 0, 0), [2.0, 1.0], [80.0, 50.0], c["kap"], DT, f, gG, dl, th)


@pytest.mark.parametrize("bc,d", [((0, 0, 0), (1.0, 0.0, 0.0)), ((1, 1, 0), (0.0, 1.0, 0.0)),
                                  ((1, 0, 0), (1.0, 0.0, 0.0))])
def test_discs_match_oracle(lb, bc, d):
    n, dx = 48, 0.5
    g = synth.disks(n, dx, [[6.1, 7.3], [17.2, 15.9], [4.4, 19.5], [20.9, 3.2]], [4.2, 5.1, 2.7, 2.3])
    dl, th = synth.link_distances(g, bc), synth.link_angles(g, bc)
    gG, f = oracle.pgse(2000.0, 0.5, 1.0, DT, d)
    _check(lb, g, bc, [2.0, 1.0], [80.0, 50.0], 0.03, DT, f, gG, dl, th)


def _random_links(shape, seed):
    rng = np.random.default_rng(seed)
    dl = np.full((6,) + shape, 0.5, np.float32)
    th = np.zeros((6,) + shape, np.float32)
    for j, (ax, sg) in enumerate(AXES):
        if sg > 0:
            dl[j] = rng.uniform(0.05, 0.95, size=shape)
            th[j] = rng.uniform(-1.4, 1.4, size=shape)
    for j, (ax, sg) in enumerate(AXES):
        if sg < 0:
            dl[j] = 1.0 - np.roll(dl[j - 1], 1, axis=ax)
            th[j] = -np.roll(th[j - 1], 1, axis=ax)
    return dl, th


@pytest.mark.parametrize("bc", [(0, 0, 0), (0, 1, 0)])
def test_random_links_match_oracle(lb, bc):
    """Blocky random compartments (5x5 blocks, so many links keep the angle
    rule) with random positions and angles on every link."""
    rng = np.random.default_rng(21)
    blocks = rng.integers(0, 3, size=(8, 8))
    lab = np.kron(blocks, np.ones((5, 5), np.int64))[None].astype(np.int32)
    g = synth.Geometry(lab, np.array([0, 1, 2], np.uint8), 0.5)
    dl, th = _random_links(lab.shape, 22)
    gd = (0.6, 0.8, 0.0) if bc == (0, 0, 0) else (1.0, 0.0, 0.0)
    gG, f = oracle.pgse(1500.0, 0.5, 1.0, DT, gd)
    _check(lb, g, bc, [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.05, DT, f, gG, dl, th)


def test_zero_angles_equal_no_angles(lb):
    g = synth.disks(40, 0.5, [[9.0, 10.0]], [5.5])
    dl = synth.link_distances(g, (0, 0, 0))
    gG, f = oracle.pgse(1500.0, 0.5, 1.0, DT, (1, 0, 0))
    args = (g, (0, 0, 0), [2.0, 1.0], [80.0, 50.0], 0.03, DT, f, gG, dl)
    a, fa, _ = _gpu(lb, *args, np.zeros_like(dl))
    b, fb, _ = _gpu(lb, *args, None)
    assert np.array_equal(fa, fb) and a["S"] == b["S"]


def test_angles_refused_where_unsupported(lb):
    g = synth.disks(16, 0.5, [[4.0, 4.0]], [2.2])
    dl, th = synth.link_distances(g, (0, 0, 0)), synth.link_angles(g, (0, 0, 0))
    s = lb.Solver(0)
    s.set_geometry(g.labels, g.phase_of_label, g.dx, (0, 0, 0))
    with pytest.raises(lb.LbmbtError) as e:            # positions first
        s.set_link_angles(th)
    assert e.value.code == -1
    s.set_link_distances(dl)
    bad = th.copy()
    bad[0, 0, 0, 0] = 1.6
    with pytest.raises(lb.LbmbtError) as e:
        s.set_link_angles(bad)
    assert e.value.code == -1
    s.set_link_angles(th)
    s.set_phases([2.0, 1.0], [INF, INF])
    s.set_permeability(0.05)
    gG, f = oracle.pgse(500.0, 0.2, 0.4, 0.02, (1, 0, 0))
    s.set_sequence(0.02, f, gG)
    with pytest.raises(lb.LbmbtError) as e:            # D3Q7 lattice
        s.run()
    assert e.value.code == -5
    s.set_option(lb.OPT_LATTICE, 1)
    with pytest.raises(lb.LbmbtError) as e:            # tau = 0.74 in phase 1
        s.run()
    assert e.value.code == -4
    gG, f = oracle.pgse(500.0, 0.5, 1.0, DT, (1, 0, 0))
    s.set_sequence(DT, f, gG)
    s.run()
    with pytest.raises(lb.LbmbtError) as e:
        s.grad()
    assert e.value.code == -5
    s.set_link_distances(None)                          # removes the angles too
    s.set_link_distances(dl)
    r1 = s.run()
    s.close()
    g3 = synth.uniform((2, 8, 8), 0.5)
    s = lb.Solver(0)
    s.set_geometry(g3.labels, g3.phase_of_label, g3.dx, (0, 0, 0))
    s.set_link_distances(np.full((6, 2, 8, 8), 0.5, np.float32))
    with pytest.raises(lb.LbmbtError) as e:            # one plane only
        s.set_link_angles(np.zeros((6, 2, 8, 8), np.float32))
    assert e.value.code == -1
    s.close()
    assert r1["S"] > 0


def test_batch_mixes_members_with_and_without_angles(lb):
    """One launch of the angle kernel over a disc pack with angles, the same
    pack with positions only, and oblique stripes with angles, each against
    its own oracle run."""
    g1 = synth.disks(40, 0.5, [[6.1, 7.3], [14.2, 13.9]], [4.2, 3.6])
    g2 = synth.stripes(32, 0.5, (1, 2), 0.4, 0.21, phases=[0, 1])
    dl1, th1 = synth.link_distances(g1, (0, 0, 0)), synth.link_angles(g1, (0, 0, 0))
    dl2, th2 = synth.link_distances(g2, (0, 0, 0)), synth.link_angles(g2, (0, 0, 0))
    D, T2 = [2.0, 1.0], [80.0, 50.0]
    gG, f = oracle.pgse(1500.0, 0.5, 1.0, DT, (1.0, 0.0, 0.0))
    gG2 = np.array([0.6, 0.8, 0.0]) * np.linalg.norm(gG)
    s = lb.Solver(0)
    s.set_option(lb.OPT_LATTICE, 1)
    s.set_geometry(g1.labels, g1.phase_of_label, g1.dx, (0, 0, 0))
    s.add_geometry(g1.labels, g1.phase_of_label, g1.dx, (0, 0, 0))
    s.add_geometry(g2.labels, g2.phase_of_label, g2.dx, (0, 0, 0))
    s.set_link_distances(dl1, index=0)
    s.set_link_angles(th1, index=0)
    s.set_link_distances(dl1, index=1)
    s.set_link_distances(dl2, index=2)
    s.set_link_angles(th2, index=2)
    s.set_phases(D, T2)
    s.set_sequence(DT, f, gG)
    r = s.run_batch(lb.Solver.members([gG, gG, gG2], [0, 1, 2], [0.03, 0.03, 0.2]))
    s.close()
    cases = [(g1, dl1, th1, gG, 0.03), (g1, dl1, None, gG, 0.03), (g2, dl2, th2, gG2, 0.2)]
    for m, (g, dl, th, gv, kap) in enumerate(cases):
        o = oracle.run(g.labels, g.dx, g.phase_of_label, (0, 0, 0), D, T2, kap, DT, f, gv,
                       delta=dl.astype(np.float64), theta=None if th is None else th.astype(np.float64),
                       lattice="D2Q5")
        assert abs(r["S"][m] - o["S"]) <= S_TOL * o["S"], (m, r["S"][m], o["S"])


def test_device_inputs_equal_host_inputs(lb):
    """Positions and angles given as CUDA tensors (device-to-device copies)
    give the same run, bit for bit, as the same values from host memory."""
    g = synth.disks(40, 0.5, [[6.1, 7.3], [14.2, 13.9]], [4.2, 3.6])
    dl, th = synth.link_distances(g, (0, 0, 0)), synth.link_angles(g, (0, 0, 0))
    gG, f = oracle.pgse(1500.0, 0.5, 1.0, DT, (0.6, 0.8, 0.0))
    outs = []
    for dev in (False, True):
        s = lb.Solver(0)
        s.set_option(lb.OPT_LATTICE, 1)
        s.set_geometry(g.labels, g.phase_of_label, g.dx, (0, 0, 0))
        if dev:
            s.set_link_distances(torch.from_numpy(dl).cuda())
            s.set_link_angles(torch.from_numpy(th).cuda())
        else:
            s.set_link_distances(dl)
            s.set_link_angles(th)
        s.set_phases([2.0, 1.0], [80.0, 50.0])
        s.set_permeability(0.03)
        s.set_sequence(DT, f, gG)
        fld = torch.zeros(g.n_sites, dtype=torch.complex64, device="cuda")
        r = s.run(field=fld)
        torch.cuda.synchronize()
        s.close()
        outs.append((r["S"], fld.cpu().numpy()))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])


def test_removing_angles_keeps_positions(lb):
    """set_link_angles(None) returns to the theta = 0 rule with the same
    positions: the run equals a positions-only run bit for bit."""
    g = synth.disks(32, 0.5, [[7.3, 8.1]], [4.4])
    dl, th = synth.link_distances(g, (0, 0, 0)), synth.link_angles(g, (0, 0, 0))
    gG, f = oracle.pgse(1500.0, 0.5, 1.0, DT, (1.0, 0.0, 0.0))
    res = []
    for drop in (True, False):
        s = lb.Solver(0)
        s.set_option(lb.OPT_LATTICE, 1)
        s.set_geometry(g.labels, g.phase_of_label, g.dx, (0, 0, 0))
        s.set_link_distances(dl)
        if drop:
            s.set_link_angles(th)
            s.set_link_angles(None)
        s.set_phases([2.0, 1.0], [80.0, 50.0])
        s.set_permeability(0.03)
        s.set_sequence(DT, f, gG)
        fld = torch.zeros(g.n_sites, dtype=torch.complex64, device="cuda")
        s.run(field=fld)
        torch.cuda.synchronize()
        s.close()
        res.append(fld.cpu().numpy())
    assert np.array_equal(res[0], res[1])
