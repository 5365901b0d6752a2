"""GPU: one grid cut into z slabs (the strips of Sec. 2.5), each slab its own
context, faces exchanged before every step.  Each cell of the decomposed run
performs the same FP32 arithmetic as the whole-grid run, so the field at the
echo must agree bit for bit; the summed signal differs only in how the sweep
groups its FP32 per-thread partial sums (1e-7).  The whole-grid run itself is
checked against the FP64 oracle (S within 1e-5).  Covered: periodic z with an
oblique gradient (wrap factor at the global face, reaction phase of global
planes), mirror z with G normal and parallel to the faces, membranes on links
that cross the cuts, ragged slab sizes, both sweep kernels, a waveform with
values other than +-1 (the general rotation), the slab mask against the
whole-grid mask, the one-rank distributed driver, and the calls a slab must
refuse."""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import slab, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = math.inf


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


def _labels(kind, n):
    if kind == "random":
        rng = np.random.default_rng(11)
        lab = rng.integers(0, 3, size=(n[0], n[1], n[2])).astype(np.int32)
        return synth.Geometry(lab, np.array([0, 1, 2], np.uint8), 0.5)
    if kind == "spheres":
        return synth.spheres(n[2], 0.5, rmin=1.0, rmax=2.5, fraction=0.4, seed=6)
    raise ValueError(kind)


def _whole(lb, geom, bc, D, T2, kap, dt, f, gG, kernel):
    s = lb.Solver(0, torch.cuda.current_stream())
    s.set_option(lb.OPT_KERNEL, kernel)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    s.close()
    return r, fld.cpu().numpy()


def _slabs(lb, geom, bc, D, T2, kap, dt, f, gG, kernel, n_slabs, options=None):
    mem = lb.Solver.members([gG], 0, kap)
    g = slab.SlabGroup(geom.labels, geom.phase_of_label, geom.dx, bc, n_slabs, D, T2, dt, f, mem,
                       torch.cuda.current_stream(), kernel=kernel, field=True, options=options)
    r = g.run(len(f))
    fld = g.field().cpu().numpy()
    for s in g.solvers:
        assert s.get_option(lb.OPT_KERNEL_USED) == kernel
        if options and lb.OPT_STAGE_OWN_Z in options:
            assert s.get_option(lb.OPT_STAGE_OWN_Z_USED) == options[lb.OPT_STAGE_OWN_Z]
    g.close()
    return r, fld


CASES = {
    # periodic z, oblique G: wrap factors on x, y and z, three-axis rotation
    "random_periodic_oblique": dict(kind="random", n=(20, 16, 32), bc=(0, 0, 0), d=(0.6, -0.5, 0.62)),
    # mirror z, G normal to the z faces (conjugating mirror with global positions)
    "random_mirror_Gz": dict(kind="random", n=(19, 16, 16), bc=(1, 1, 1), d=(0.0, 0.0, 1.0)),
    # mirror z, G parallel to the z faces
    "spheres_mirror_Gx": dict(kind="spheres", n=(32, 32, 32), bc=(0, 0, 1), d=(1.0, 0.0, 0.0)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kernel", [1, 2])
def test_slabs_match_whole_grid_bit_for_bit(lb, name, kernel):
    c = CASES[name]
    geom = _labels(c["kind"], c["n"])
    if c["kind"] == "random":
        assert geom.labels.shape == c["n"]
    D, T2, kap, dt = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.04, 0.02
    gG, f = oracle.pgse(1500.0, 0.3, 0.5, dt, c["d"])
    ref, ref_fld = _whole(lb, geom, c["bc"], D, T2, kap, dt, f, gG, kernel)
    o = oracle.run(geom.labels, geom.dx, geom.phase_of_label, c["bc"], D, T2, kap, dt, f, gG)
    assert abs(ref["S"] - o["S"]) <= 1e-5 * o["S"]
    for n_slabs in (1, 2, 3):
        if n_slabs == 1 and c["bc"][2] == 1:
            continue   # a mirror grid in one piece is a plain geometry
        r, fld = _slabs(lb, geom, c["bc"], D, T2, kap, dt, f, gG, kernel, n_slabs)
        assert np.array_equal(fld, ref_fld), (name, n_slabs)
        assert abs(r["Z"][0] - ref["Z"]) <= 1e-7 * abs(ref["Z"]), (name, n_slabs)


@pytest.mark.parametrize("name", list(CASES))
def test_marching_slabs_match_whole_grid_bit_for_bit(lb, name):
    """The bulk-copy sweep's z-marching form on slabs: a column that starts
    at a cut takes its +z pull from the halo plane (2 slabs of 16 planes
    march in columns of 16), and the fields equal the whole grid's."""
    c = CASES[name]
    geom = _labels(c["kind"], c["n"])
    D, T2, kap, dt = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.04, 0.02
    gG, f = oracle.pgse(1500.0, 0.3, 0.5, dt, c["d"])
    ref, ref_fld = _whole(lb, geom, c["bc"], D, T2, kap, dt, f, gG, 2)
    for n_slabs in (2, 3):
        r, fld = _slabs(lb, geom, c["bc"], D, T2, kap, dt, f, gG, 2, n_slabs, {lb.OPT_STAGE_OWN_Z: 3})
        assert np.array_equal(fld, ref_fld), (name, n_slabs)
        assert abs(r["Z"][0] - ref["Z"]) <= 1e-7 * abs(ref["Z"]), (name, n_slabs)


def test_slab_general_waveform_and_offsets(lb):
    """Waveform values other than +-1 take the general rotation (sincos of the
    global plane index); four uneven slabs of a periodic grid."""
    geom = _labels("random", (23, 16, 16))
    D, T2, kap, dt = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.04, 0.02
    gG, _ = oracle.pgse(1500.0, 0.3, 0.5, dt, (0.3, 0.4, 0.87))
    f = np.array([1.0, 0.7, -0.35, 0.0, 0.5, -1.0, 0.25, 1.0] * 5)
    for kernel in (1, 2):
        ref, ref_fld = _whole(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG, kernel)
        r, fld = _slabs(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG, kernel, 4)
        assert np.array_equal(fld, ref_fld)
        assert abs(r["Z"][0] - ref["Z"]) <= 1e-7 * abs(ref["Z"])
    o = oracle.run(geom.labels, geom.dx, geom.phase_of_label, (0, 0, 0), D, T2, kap, dt, f, gG)
    assert abs(r["S"][0] - o["S"]) <= 1e-5 * o["S"]


def test_slab_mask_matches_whole_grid(lb):
    geom = _labels("random", (20, 16, 16))
    for bc in [(0, 0, 0), (1, 1, 1)]:
        with lb.Solver(0) as s:
            s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
            whole = s.get_mask(0, geom.labels.shape)
        parts = []
        for z0, z1 in slab.split(20, 3):
            lo, hi = slab.face_kinds(z0, z1, 20, bc[2])
            with lb.Solver(0) as s:
                s.set_geometry_slab(slab.ghost_labels(geom.labels, z0, z1, bc[2]), geom.phase_of_label, geom.dx,
                                    bc, z0, 20, lo, hi)
                parts.append(s.get_mask(0, (z1 - z0, 16, 16)))
        assert np.array_equal(np.concatenate(parts), whole)


def test_distributed_driver_one_rank(lb):
    """``run_distributed`` with one rank on a periodic axis: the slab is its own
    neighbour across the wrap, the result equals the whole-grid run."""
    geom = _labels("random", (12, 16, 16))
    D, T2, kap, dt = [2.0, 1.0, 1.5], [80.0, 50.0, 60.0], 0.04, 0.02
    gG, f = oracle.pgse(1500.0, 0.3, 0.5, dt, (0.0, 0.6, 0.8))
    ref, _ = _whole(lb, geom, (0, 0, 0), D, T2, kap, dt, f, gG, 0)
    mem = lb.Solver.members([gG], 0, kap)
    made = []

    def make(z0, z1, lo, hi):
        s = lb.Solver(0, torch.cuda.current_stream())
        s.set_geometry_slab(slab.ghost_labels(geom.labels, z0, z1, 0), geom.phase_of_label, geom.dx, (0, 0, 0),
                            z0, 12, lo, hi)
        s.set_phases(D, T2)
        s.set_sequence(dt, f, gG)
        s.prepare(mem)
        made.append(s)
        return s

    Z = slab.run_distributed(make, 12, 0, len(f), 1, (16, 16), 0, 1, device=torch.device("cuda"))
    made[0].close()
    assert abs(Z[0] - ref["Z"]) <= 1e-7 * abs(ref["Z"])


def test_slab_refuses_whole_run_calls(lb):
    geom = _labels("random", (8, 16, 16))
    s = lb.Solver(0)
    with pytest.raises(lb.LbmbtError):   # a wrapping face needs a periodic axis
        s.set_geometry_slab(slab.ghost_labels(geom.labels, 0, 4, 1), geom.phase_of_label, 0.5, (1, 1, 1), 0, 8,
                            lb.FACE_HALO_WRAP, lb.FACE_HALO)
    with pytest.raises(lb.LbmbtError):   # an interior face cannot be the slab's own
        s.set_geometry_slab(slab.ghost_labels(geom.labels, 2, 6, 1), geom.phase_of_label, 0.5, (1, 1, 1), 2, 8,
                            lb.FACE_OWN, lb.FACE_HALO)
    s.set_geometry_slab(slab.ghost_labels(geom.labels, 0, 4, 0), geom.phase_of_label, 0.5, (0, 0, 0), 0, 8,
                        lb.FACE_HALO_WRAP, lb.FACE_HALO)
    s.set_phases([2.0, 1.0, 1.5], [INF] * 3)
    gG, f = oracle.pgse(500.0, 0.3, 0.5, 0.02, (1, 0, 0))
    s.set_sequence(0.02, f, gG)
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -7
    with pytest.raises(lb.LbmbtError) as e:
        s.grad()
    assert e.value.code == -5
    s.prepare()
    with pytest.raises(lb.LbmbtError) as e:
        s.advance(2)
    assert e.value.code == -1
    s.advance(1)
    s.close()
