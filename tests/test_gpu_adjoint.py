"""GPU adjoint sweep: dS/d(D_p, T2_p, kappa) against central finite
differences (h = 1e-3 relative) of the FP64 oracle and of the GPU forward.

Tolerance against the oracle's differences: 1e-4 of the largest
log-parameter gradient component (theta dS/dtheta).  The differences' own
truncation error is O(h^2) ~ 1e-6 of that scale; the rest is the FP32
forward and adjoint arithmetic."""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
INF = math.inf
H = 1e-3
ADJ_TOL = 1e-4   # of the largest log-parameter gradient component


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _setup(lb, geom, bc, D, T2, kap, dt, f, gG):
    s = lb.Solver(0)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    return s


def _fd(fun, D, T2, kap):
    """Central differences of S in every parameter (relative step H)."""
    out = {"dD": [], "dT2": [], "dkappa": None}
    for p in range(len(D)):
        Dp, Dm = list(D), list(D)
        Dp[p] *= 1 + H
        Dm[p] *= 1 - H
        out["dD"].append((fun(Dp, T2, kap) - fun(Dm, T2, kap)) / (2 * H * D[p]))
    for p in range(len(T2)):
        if math.isinf(T2[p]):
            out["dT2"].append(0.0)
            continue
        Tp, Tm = list(T2), list(T2)
        Tp[p] *= 1 + H
        Tm[p] *= 1 - H
        out["dT2"].append((fun(D, Tp, kap) - fun(D, Tm, kap)) / (2 * H * T2[p]))
    out["dkappa"] = (fun(D, T2, kap * (1 + H)) - fun(D, T2, kap * (1 - H))) / (2 * H * kap)
    return out


def _logvec(g, D, T2, kap):
    """Gradient in log-parameters, theta * dS/dtheta, as one vector."""
    return np.concatenate([np.asarray(g["dD"]) * D,
                           np.asarray(g["dT2"]) * np.where(np.isinf(T2), 0.0, T2),
                           [g["dkappa"] * kap]])


CASES = {
    "cylinders_periodic": dict(geom=lambda: synth.cylinders(24, 1.0, fraction=0.5, seed=3), bc=(0, 0, 0),
                               D=[2.0, 1.0], T2=[80.0, 50.0], kap=0.05, dt=0.05, b=1500.0,
                               delta=2.0, Delta=6.0, d=(1, 1, 0)),
    "spheres_oblique": dict(geom=lambda: synth.spheres(20, 1.0, rmin=2.0, rmax=3.5, fraction=0.45, seed=4),
                            bc=(0, 0, 0), D=[2.0, 1.0], T2=[80.0, 50.0], kap=0.02, dt=0.05, b=2500.0,
                            delta=2.0, Delta=5.0, d=(0.3, -0.5, 0.8)),
    "cylinders32_bulk": dict(geom=lambda: synth.cylinders(32, 1.0, fraction=0.5, seed=6), bc=(0, 0, 0),
                             D=[2.0, 1.0], T2=[80.0, 50.0], kap=0.05, dt=0.05, b=1500.0,
                             delta=2.0, Delta=5.0, d=(0.6, -0.48, 0.64)),
    "voronoi32_mirror_bulk": dict(geom=lambda: synth.crop(synth.voronoi_tissue(48, 0.5, cell_diam=6.0,
                                                                               vessel_radius=1.5, seed=8), 32),
                                  bc=(1, 1, 1), D=[1.0, 2.5, 3.0], T2=[50.0, 80.0, 80.0], kap=0.01, dt=0.025,
                                  b=1000.0, delta=1.0, Delta=3.0, d=(0, 0, 1)),
    "voronoi_mirror": dict(geom=lambda: synth.crop(synth.voronoi_tissue(40, 0.5, cell_diam=6.0, vessel_radius=1.5,
                                                                        seed=2), 22),
                           bc=(1, 1, 1), D=[1.0, 2.5, 3.0], T2=[50.0, 80.0, 80.0], kap=0.01, dt=0.025,
                           b=1000.0, delta=1.0, Delta=3.0, d=(1, 0, 0)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_oracle_finite_differences(lb, name):
    c = CASES[name]
    geom = c["geom"]()
    gG, f = oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], c["d"])
    s = _setup(lb, geom, c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, gG)
    g = s.grad(checkpoint_every=16)
    s.close()

    def S(D, T2, kap):
        return oracle.run(geom.labels, geom.dx, geom.phase_of_label, c["bc"], D, T2, kap, c["dt"], f, gG)["S"]

    fd = _fd(S, c["D"], c["T2"], c["kap"])
    a = _logvec(g, c["D"], c["T2"], c["kap"])
    b = _logvec(fd, c["D"], c["T2"], c["kap"])
    err = np.abs(a - b).max() / np.abs(b).max()
    print(name, "adjoint", a, "fd", b, "err", err)
    assert err < ADJ_TOL
    assert abs(g["S"] - S(c["D"], c["T2"], c["kap"])) < 1e-5 * g["S"]


def test_adjoint_matches_gpu_forward_finite_differences(lb):
    c = CASES["cylinders_periodic"]
    geom = c["geom"]()
    gG, f = oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], c["d"])
    s = _setup(lb, geom, c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, gG)
    g = s.grad()

    def S(D, T2, kap):
        s.set_phases(D, T2)
        s.set_permeability(kap)
        return s.run()["S"]

    fd = _fd(S, c["D"], c["T2"], c["kap"])
    s.close()
    a = _logvec(g, c["D"], c["T2"], c["kap"])
    b = _logvec(fd, c["D"], c["T2"], c["kap"])
    assert np.abs(a - b).max() / np.abs(b).max() < 2e-2


def test_checkpoint_interval_does_not_change_gradients(lb):
    c = CASES["spheres_oblique"]
    geom = c["geom"]()
    gG, f = oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], c["d"])
    s = _setup(lb, geom, c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, gG)
    ref = s.grad(checkpoint_every=64)
    for ck in (1, 7, 1000):
        g = s.grad(checkpoint_every=ck)
        np.testing.assert_array_equal(g["dD"], ref["dD"])
        np.testing.assert_array_equal(g["dT2"], ref["dT2"])
        assert g["dkappa"] == ref["dkappa"]
    s.close()


def test_grad_batch_matches_single(lb):
    c = CASES["cylinders_periodic"]
    geom = c["geom"]()
    _, f = oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], c["d"])
    dirs = synth.directions_on_sphere(3, seed=5)
    gGs = [oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], d)[0] for d in dirs]
    s = _setup(lb, geom, c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, gGs[0])
    mem = lb.Solver.members(gGs, 0, c["kap"])
    gb = s.grad_batch(mem, checkpoint_every=32)
    # the members' units fall on other CTAs than in a run of one member, so
    # the FP32 partial sums group differently (FP32-rounding agreement only)
    for i, gG in enumerate(gGs):
        s.set_sequence(c["dt"], f, gG)
        g = s.grad(checkpoint_every=32)
        a = np.concatenate([g["dD"], g["dT2"], [g["dkappa"]]])
        b = np.concatenate([gb["dD"][i], gb["dT2"][i], [gb["dkappa"][i]]])
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max(), i
        assert gb["S"][i] == pytest.approx(g["S"], rel=1e-12)
    s.close()


def test_autograd_function(lb):
    from paper_1907_00908_gb300.autograd import signal
    c = CASES["cylinders_periodic"]
    geom = c["geom"]()
    gG, f = oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], c["d"])
    s = _setup(lb, geom, c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, gG)
    D = torch.tensor(c["D"], dtype=torch.float64, requires_grad=True)
    T2 = torch.tensor(c["T2"], dtype=torch.float64, requires_grad=True)
    kap = torch.tensor(c["kap"], dtype=torch.float64, requires_grad=True)
    S = signal(s, D, T2, kap)
    (2.0 * S).backward()
    g = s.grad()
    s.close()
    np.testing.assert_allclose(D.grad.numpy(), 2.0 * g["dD"], rtol=1e-12)
    np.testing.assert_allclose(T2.grad.numpy(), 2.0 * g["dT2"], rtol=1e-12)
    assert float(kap.grad) == pytest.approx(2.0 * g["dkappa"], rel=1e-12)


@pytest.mark.parametrize("name", ["cylinders32_bulk", "voronoi32_mirror_bulk"])
def test_bulk_copy_adjoint_matches_register_adjoint(lb, name):
    """The bulk-copy adjoint sweep and the register adjoint sweep give the
    same gradients (they differ only in the grouping of FP32 partial sums)."""
    c = CASES[name]
    geom = c["geom"]()
    gG, f = oracle.pgse(c["b"], c["delta"], c["Delta"], c["dt"], c["d"])
    s = _setup(lb, geom, c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, gG)
    out = {}
    for kern, shape in ((1, 0), (2, 0), (2, 1), (2, 2)):
        s.set_option(lb.OPT_ADJOINT_KERNEL, kern)
        s.set_option(lb.OPT_ADJOINT_SHAPE, shape)
        out[(kern, shape)] = s.grad(checkpoint_every=16)
    s.close()
    a = _logvec(out[(1, 0)], c["D"], c["T2"], c["kap"])
    for key in ((2, 0), (2, 1), (2, 2)):
        b = _logvec(out[key], c["D"], c["T2"], c["kap"])
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max(), key
        assert out[(1, 0)]["S"] == out[key]["S"]


@pytest.mark.parametrize("bc,d", [((0, 0, 0), (0.6, 0.8, 0.0)), ((1, 1, 0), (1.0, 0.0, 0.0))])
def test_adjoint_d2q5_matches_oracle_finite_differences(lb, bc, d):
    """The register adjoint on the 2-D D2Q5 lattice (weights 1/3, 1/6 and
    eps_D = 1/3 in the chain rule) against central differences of the
    oracle's D2Q5 runs; a forced bulk-copy adjoint is refused."""
    geom = synth.disks(40, 0.5, [[5.3, 6.1], [14.8, 13.2], [4.9, 15.7]], [3.6, 4.1, 2.4])
    D, T2, kap, dt = [2.0, 1.0], [80.0, 50.0], 0.05, 0.02
    gG, f = oracle.pgse(2000.0, 0.4, 1.0, dt, d)
    s = _setup(lb, geom, bc, D, T2, kap, dt, f, gG)
    s.set_option(lb.OPT_LATTICE, 1)
    g = s.grad(checkpoint_every=8)
    s.set_option(lb.OPT_ADJOINT_KERNEL, 2)
    with pytest.raises(lb.LbmbtError) as e:
        s.grad()
    assert e.value.code == -5
    s.close()

    def S(D_, T2_, kap_):
        return oracle.run(geom.labels, geom.dx, geom.phase_of_label, bc, D_, T2_, kap_, dt, f, gG,
                          lattice="D2Q5")["S"]

    fd = _fd(S, D, T2, kap)
    a, b = _logvec(g, D, T2, kap), _logvec(fd, D, T2, kap)
    err = np.abs(a - b).max() / np.abs(b).max()
    print("d2q5", bc, d, "adjoint", a, "fd", b, "err", err)
    assert err < ADJ_TOL, (a, b, err)
    assert abs(g["S"] - S(D, T2, kap)) < 1e-5 * g["S"]


def test_bulk_copy_adjoint_shape_falls_back_for_wide_rows(lb):
    """The default bulk-copy adjoint shape takes units of <= 480 sites; a grid
    with nx = 496 runs on the 512-site shape instead, and its gradients equal
    the register adjoint's."""
    rng = np.random.default_rng(31)
    lab = rng.integers(0, 2, size=(3, 4, 496)).astype(np.int32)
    geom = synth.Geometry(lab, np.array([0, 1], np.uint8), 0.5)
    gG, f = oracle.pgse(1500.0, 0.4, 0.8, 0.02, (1.0, 0.0, 0.0))
    s = _setup(lb, geom, (0, 0, 0), [2.0, 1.0], [80.0, 50.0], 0.05, 0.02, f, gG)
    out = {}
    for kern in (1, 2):
        s.set_option(lb.OPT_ADJOINT_KERNEL, kern)
        out[kern] = s.grad(checkpoint_every=8)
    assert s.get_option(lb.OPT_ADJOINT_SHAPE) == 2
    s.close()
    a = _logvec(out[1], [2.0, 1.0], [80.0, 50.0], 0.05)
    b = _logvec(out[2], [2.0, 1.0], [80.0, 50.0], 0.05)
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
