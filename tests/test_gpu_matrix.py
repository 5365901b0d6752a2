"""GPU parity over a seeded matrix of random configurations, each against
the FP64 oracle (S within 1e-5 relative, field within 1e-4 of max|M|):
ragged grid shapes, periodic / mirror faces per axis, gradient directions
allowed by the faces, kappa 0, finite or infinite, three compartments, with
or without membrane positions, both sweeps (the bulk-copy sweep where the
grid allows it), graphs on or off, launch shapes, 1 or 4 reaction sub-steps,
and the D2Q5 lattice on one-plane grids; the classical scheme over the same
kind of configurations; random batches of members on different geometries
(some with positions), and random batches whose members carry their own
waveforms and field outputs, each member against its own oracle run.  Every
configuration is a pure function of its seed."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S_TOL = 1e-5
FIELD_TOL = 1e-4
AXES = [(2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1)]


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _positions(shape, rng):
    dl = np.empty((6,) + shape, np.float32)
    for j, (ax, sg) in enumerate(AXES):
        if sg > 0:
            dl[j] = rng.uniform(0.05, 0.95, size=shape)
    for j, (ax, sg) in enumerate(AXES):
        if sg < 0:
            dl[j] = 1.0 - np.roll(dl[j - 1], 1, axis=ax)
    return dl


def _config(seed):
    rng = np.random.default_rng(1000 + seed)
    d2q5 = seed % 6 == 5
    nz = 1 if d2q5 else int(rng.integers(1, 9))
    ny = int(rng.integers(1, 13))
    nx = int(rng.choice([16, 32])) if rng.random() < 0.4 else int(rng.integers(1, 21))
    shape = (nz, ny, nx)
    bc = [int(rng.integers(0, 2)) for _ in range(3)]
    if d2q5:
        bc[2] = 0
    # gradient: free direction, except that on a mirror axis it must be
    # normal to that face (and then zero on the others) or parallel to it
    mir = [a for a in range(3) if bc[a] == 1]
    g = np.array([rng.normal(), rng.normal(), 0.0 if d2q5 else rng.normal()])
    if mir and (len(mir) == 3 or rng.random() < 0.5):
        g = np.zeros(3)
        g[int(rng.choice(mir))] = 1.0
    else:
        g[mir] = 0.0
    n_lab = int(rng.integers(1, 4))
    block = int(rng.integers(1, 4))
    lab = rng.integers(0, n_lab, size=(max(1, nz // block + 1), max(1, ny // block + 1), max(1, nx // block + 1)))
    lab = np.kron(lab, np.ones((block, block, block), np.int64))[:nz, :ny, :nx].astype(np.int32)
    pol = np.array([0, 1, 2], np.uint8)[:max(1, n_lab)]
    kap = float(rng.choice([0.0, 0.03, 0.3, math.inf]))
    use_dl = (not d2q5) and n_lab > 1 and math.isfinite(kap) and rng.random() < 0.35
    dt = 0.02
    D = [2.0, 1.0, 1.5][:len(pol)]
    T2 = [80.0, 50.0, math.inf][:len(pol)]
    substeps = 4 if rng.random() < 0.2 else 1
    K = int(rng.integers(5, 30))
    if substeps == 1:
        f = rng.choice([-1.0, 0.0, 1.0, 0.5], size=K)
    else:
        f = np.sin(np.arange(K * substeps) * 0.37)
    gG = g * 0.08
    opts = dict(kernel=int(rng.choice([0, 1, 2])), graph=int(rng.integers(0, 2)),
                block=int(rng.choice([64, 128, 256])), spt=int(rng.choice([1, 2, 4])))
    return dict(shape=shape, bc=tuple(bc), lab=lab, pol=pol, kap=kap, dl=_positions(shape, rng) if use_dl else None,
                dt=dt, D=D, T2=T2, f=f, gG=gG, substeps=substeps, d2q5=d2q5, opts=opts)


@pytest.mark.parametrize("seed", list(range(64)))
def test_random_configuration_matches_oracle(lb, seed):
    c = _config(seed)
    s = lb.Solver(0)
    s.set_option(lb.OPT_GRAPH, c["opts"]["graph"])
    s.set_option(lb.OPT_BLOCK, c["opts"]["block"])
    s.set_option(lb.OPT_SPT, c["opts"]["spt"])
    if c["d2q5"]:
        s.set_option(lb.OPT_LATTICE, 1)
    kernel = c["opts"]["kernel"]
    tma_ok = c["shape"][2] % 16 == 0 and c["dl"] is None and not c["d2q5"]
    if kernel == 2 and not tma_ok:
        kernel = 1
    s.set_option(lb.OPT_KERNEL, kernel)
    # the bulk-copy sweep's own-z form, drawn apart so the configurations stay as they were
    own_z = int(np.random.default_rng(1000 + seed).integers(0, 4)) if kernel == 2 else 0
    s.set_option(lb.OPT_STAGE_OWN_Z, own_z)
    s.set_geometry(c["lab"], c["pol"], 0.5, c["bc"])
    if c["dl"] is not None:
        s.set_link_distances(c["dl"])
    s.set_phases(c["D"], c["T2"])
    s.set_permeability(c["kap"])
    if c["substeps"] > 1:
        s.set_sequence_substeps(c["dt"], c["f"], c["gG"], c["substeps"])
    else:
        s.set_sequence(c["dt"], c["f"], c["gG"])
    n = int(np.prod(c["shape"]))
    fld = torch.zeros(n, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    if own_z:
        assert s.get_option(lb.OPT_STAGE_OWN_Z_USED) == own_z
    s.close()
    o = oracle.run(c["lab"], 0.5, c["pol"], c["bc"], c["D"], c["T2"], c["kap"], c["dt"], c["f"], c["gG"],
                   want_field=True, delta=None if c["dl"] is None else c["dl"].astype(np.float64),
                   substeps=c["substeps"], lattice="D2Q5" if c["d2q5"] else "D3Q7")
    assert abs(r["S"] - o["S"]) <= S_TOL * max(o["S"], 1e-30) + 1e-12, (c["shape"], c["bc"], r["S"], o["S"])
    ref = o["field"]
    err = np.abs(fld.cpu().numpy().reshape(c["shape"]) - ref).max() / max(np.abs(ref).max(), 1e-30)
    assert err < FIELD_TOL, (c["shape"], c["bc"], c["opts"], err)


@pytest.mark.parametrize("seed", list(range(16)))
def test_random_batch_matches_oracle(lb, seed):
    """2 to 4 members on different random geometries of the D3Q7 lattice
    (faces shared by the batch, kappa and gradient per member), one launch
    per step; each member's S against its own oracle run."""
    rng = np.random.default_rng(5000 + seed)
    bc = tuple(int(v) for v in rng.integers(0, 2, size=3))
    n_mem = int(rng.integers(2, 5))
    s = lb.Solver(0)
    s.set_option(lb.OPT_GRAPH, int(rng.integers(0, 2)))
    geoms, cases = [], []
    dt, K = 0.02, int(rng.integers(5, 25))
    f = rng.choice([-1.0, 0.0, 1.0], size=K)
    for m in range(n_mem):
        shape = (int(rng.integers(1, 7)), int(rng.integers(1, 9)), int(rng.choice([16, 32, 7, 12])))
        lab = rng.integers(0, 3, size=shape).astype(np.int32)
        pol = np.array([0, 1, 1], np.uint8)
        (s.set_geometry if m == 0 else s.add_geometry)(lab, pol, 0.5, bc)
        kap = float(rng.choice([0.0, 0.05, math.inf]))
        dl = _positions(shape, rng) if (math.isfinite(kap) and rng.random() < 0.4) else None
        if dl is not None:
            s.set_link_distances(dl, index=m)
        mir = [a for a in range(3) if bc[a] == 1]
        g = rng.normal(size=3)
        if mir and (len(mir) == 3 or rng.random() < 0.5):
            g = np.zeros(3)
            g[int(rng.choice(mir))] = 1.0
        else:
            g[mir] = 0.0
        cases.append((lab, pol, kap, dl, g * 0.08))
    s.set_phases([2.0, 1.0], [80.0, 50.0])
    s.set_sequence(dt, f, cases[0][4])
    mem = lb.Solver.members([c[4] for c in cases], list(range(n_mem)), [c[2] for c in cases])
    r = s.run_batch(mem)
    s.close()
    for m, (lab, pol, kap, dl, gG) in enumerate(cases):
        o = oracle.run(lab, 0.5, pol, bc, [2.0, 1.0], [80.0, 50.0], kap, dt, f, gG,
                       delta=None if dl is None else dl.astype(np.float64))
        assert abs(r["S"][m] - o["S"]) <= S_TOL * o["S"], (seed, m, lab.shape, bc, kap, dl is not None)


@pytest.mark.parametrize("seed", list(range(32)))
def test_random_classical_configuration_matches_oracle(lb, seed):
    """The classical scheme (Appendix A, Eq. A12) over the same kind of
    random configurations (no membrane positions and no sub-steps, which it
    refuses), either sweep, both lattices."""
    c = _config(700 + seed)
    rng = np.random.default_rng(9000 + seed)
    f = rng.choice([-1.0, 0.0, 1.0, 0.5], size=int(rng.integers(5, 30)))
    s = lb.Solver(0)
    s.set_option(lb.OPT_SCHEME, 1)
    s.set_option(lb.OPT_GRAPH, c["opts"]["graph"])
    s.set_option(lb.OPT_BLOCK, c["opts"]["block"])
    s.set_option(lb.OPT_SPT, c["opts"]["spt"])
    if c["d2q5"]:
        s.set_option(lb.OPT_LATTICE, 1)
    kernel = c["opts"]["kernel"]
    if kernel == 2 and not (c["shape"][2] % 16 == 0 and not c["d2q5"]):
        kernel = 1
    s.set_option(lb.OPT_KERNEL, kernel)
    s.set_option(lb.OPT_STAGE_OWN_Z, int(np.random.default_rng(2000 + seed).integers(0, 4)) if kernel == 2 else 0)
    s.set_geometry(c["lab"], c["pol"], 0.5, c["bc"])
    s.set_phases(c["D"], c["T2"])
    s.set_permeability(c["kap"])
    s.set_sequence(c["dt"], f, c["gG"])
    n = int(np.prod(c["shape"]))
    fld = torch.zeros(n, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    s.close()
    o = oracle.run(c["lab"], 0.5, c["pol"], c["bc"], c["D"], c["T2"], c["kap"], c["dt"], f, c["gG"],
                   want_field=True, lattice="D2Q5" if c["d2q5"] else "D3Q7", scheme="classical")
    assert abs(r["S"] - o["S"]) <= S_TOL * max(o["S"], 1e-30) + 1e-12, (c["shape"], c["bc"], r["S"], o["S"])
    ref = o["field"]
    err = np.abs(fld.cpu().numpy().reshape(c["shape"]) - ref).max() / max(np.abs(ref).max(), 1e-30)
    assert err < FIELD_TOL, (c["shape"], c["bc"], c["opts"], err)


@pytest.mark.parametrize("seed", list(range(12)))
def test_random_batch_with_member_waveforms_matches_oracle(lb, seed):
    """Random batches through lbmbt_run_batch_ex: each member with its own
    random waveform of its own length (or the set one) and its own field
    output, against its own oracle run at its own end."""
    rng = np.random.default_rng(7000 + seed)
    bc = tuple(int(v) for v in rng.integers(0, 2, size=3))
    n_mem = int(rng.integers(2, 5))
    kernel = int(rng.choice([0, 1, 2]))
    dt, K = 0.02, int(rng.integers(8, 25))
    f_set = rng.choice([-1.0, 0.0, 1.0], size=K)
    cases = []
    nx_all = []
    for m in range(n_mem):
        shape = (int(rng.integers(1, 7)), int(rng.integers(1, 9)), int(rng.choice([16, 32, 7, 12])))
        nx_all.append(shape[2])
        lab = rng.integers(0, 3, size=shape).astype(np.int32)
        kap = float(rng.choice([0.0, 0.05, math.inf]))
        mir = [a for a in range(3) if bc[a] == 1]
        g = rng.normal(size=3)
        if mir and (len(mir) == 3 or rng.random() < 0.5):
            g = np.zeros(3)
            g[int(rng.choice(mir))] = 1.0
        else:
            g[mir] = 0.0
        wave = None if rng.random() < 0.3 else rng.choice([-1.0, 0.0, 1.0, 0.5], size=int(rng.integers(1, K + 1)))
        cases.append((lab, kap, g * 0.08, wave))
    if kernel == 2 and any(v % 16 for v in nx_all):
        kernel = 1
    pol = np.array([0, 1, 1], np.uint8)
    s = lb.Solver(0)
    s.set_option(lb.OPT_KERNEL, kernel)
    s.set_option(lb.OPT_GRAPH, int(rng.integers(0, 2)))
    for m, (lab, _, _, _) in enumerate(cases):
        (s.set_geometry if m == 0 else s.add_geometry)(lab, pol, 0.5, bc)
    s.set_phases([2.0, 1.0], [80.0, 50.0])
    s.set_sequence(dt, f_set, cases[0][2])
    mem = lb.Solver.members([c[2] for c in cases], list(range(n_mem)), [c[1] for c in cases])
    flds = [torch.zeros(c[0].size, dtype=torch.complex64, device="cuda") for c in cases]
    r = s.run_batch(mem, waveforms=[c[3] for c in cases], fields=flds)
    torch.cuda.synchronize()
    s.close()
    for m, (lab, kap, gG, wave) in enumerate(cases):
        fm = f_set if wave is None else wave
        o = oracle.run(lab, 0.5, pol, bc, [2.0, 1.0], [80.0, 50.0], kap, dt, fm, gG, want_field=True)
        assert abs(r["S"][m] - o["S"]) <= S_TOL * o["S"], (seed, m, lab.shape, bc, kap)
        err = np.abs(flds[m].cpu().numpy().reshape(lab.shape) - o["field"]).max() / np.abs(o["field"]).max()
        assert err < FIELD_TOL, (seed, m, err)
