"""The seeded synthetic geometries behind every workload: each holds the
recipe it states.
* Cylinders are z-aligned and non-overlapping (periodic minimum image), fill
  their area fraction, and take gamma radii of mean 3 um.
* Sphere packs are non-overlapping, fill their volume fraction, keep radii in
  [rmin, rmax], and give every sphere at least one site.
* Gradient directions are unit vectors, isotropic and seeded.
* Crops keep the label partition and phases.
* The tissue is reproducible from its seed.
* The exact membrane positions on the links of sphere and cylinder packs lie
  on the bodies' surfaces and agree from both ends of a link."""
import numpy as np

import bench
from paper_1907_00908_gb300 import synth


def _min_gap(centers, radii, box):
    d = centers[:, None, :] - centers[None, :, :]
    d -= box * np.round(d / box)
    gap = np.linalg.norm(d, axis=2) - (radii[:, None] + radii[None, :])
    np.fill_diagonal(gap, np.inf)
    return gap.min()


def test_cylinder_pack_recipe():
    g = synth.cylinders(128, 0.5, seed=1)
    assert all(np.array_equal(g.labels[0], g.labels[z]) for z in range(g.labels.shape[0]))
    c, r = np.asarray(g.info["centers"]), np.asarray(g.info["radii"])
    assert _min_gap(c[:, :2], r, 128 * 0.5) > -1e-6
    assert abs((g.phase_of_label[g.labels] == 1).mean() - 0.6) < 0.02
    assert len(np.unique(g.labels)) == len(r) + 1
    assert abs(r.mean() - 3.0) < 0.3 and 0.15 < r.std() / r.mean() < 0.45


def test_sphere_pack_recipe():
    g = synth.spheres(96, 0.5, rmin=2.0, rmax=6.0, fraction=0.5, seed=4)
    c, r = np.asarray(g.info["centers"]), np.asarray(g.info["radii"])
    assert r.min() >= 2.0 and r.max() <= 6.0
    assert _min_gap(c, r, 96 * 0.5) > -1e-6
    assert abs((g.phase_of_label[g.labels] == 1).mean() - 0.5) < 0.02
    assert len(np.unique(g.labels)) == len(r) + 1


def test_directions_are_unit_isotropic_and_seeded():
    d = synth.directions_on_sphere(4000, seed=3)
    assert np.abs(np.linalg.norm(d, axis=1) - 1.0).max() < 1e-12
    assert np.linalg.norm(d.mean(0)) < 0.05
    assert np.abs(d.T @ d / len(d) - np.eye(3) / 3).max() < 0.02
    assert np.array_equal(synth.directions_on_sphere(8, seed=3), d[:8])
    assert not np.array_equal(synth.directions_on_sphere(8, seed=4), d[:8])


def test_crop_keeps_the_label_partition_and_phases():
    g = bench.geometry(96)
    cr = synth.crop(g, 40)
    orig = g.labels[:40, :40, :40]
    assert np.array_equal(cr.phase_of_label[cr.labels], g.phase_of_label[orig])
    pairs = np.unique(np.stack([orig.ravel(), cr.labels.ravel()]), axis=1)
    assert len(np.unique(pairs[0])) == pairs.shape[1] == len(np.unique(pairs[1]))
    assert cr.labels.max() == pairs.shape[1] - 1


def test_tissue_is_reproducible_from_its_seed():
    a, b = bench.geometry(48), bench.geometry(48)
    assert np.array_equal(a.labels, b.labels) and np.array_equal(a.phase_of_label, b.phase_of_label)
    c = bench.geometry(48, seed=bench.TISSUE_SEED + 1)
    assert not np.array_equal(a.labels, c.labels)


_DIRS = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def _check_link_positions(g, ndim):
    """Every membrane position from synth.link_distances lies on the surface
    of the body its link crosses. The tolerance is the documented clip to
    [1e-4, 1 - 1e-4] of a link. Both ends of a link see the same cut:
    Delta_j(s) + Delta_jbar(s + e_j) = 1 exactly."""
    lab, dx = g.labels, g.dx
    nz, ny, nx = lab.shape
    dl = synth.link_distances(g, (0, 0, 0))
    cen, rad = np.asarray(g.info["centers"]), np.asarray(g.info["radii"])
    box = np.array([nx, ny, nz]) * dx
    n = 0
    for j, e in enumerate(_DIRS):
        a = j // 2
        nb = np.roll(lab, -e[a], axis=2 - a)
        idx = np.nonzero(nb != lab)
        if len(idx[0]) == 0:
            continue
        la, lb = lab[idx], nb[idx]
        k = np.where((la > 0) & (lb > 0), np.minimum(la, lb), np.where(la > 0, la, lb)) - 1
        p = np.stack([idx[2], idx[1], idx[0]], 1) * dx + dl[j][idx][:, None] * dx * np.array(e)
        c = np.zeros((len(k), 3))
        c[:, :ndim] = cen[k][:, :ndim]
        dv = p - c
        dv[:, ndim:] = 0.0
        dv -= box * np.round(dv / box)
        assert np.abs(np.linalg.norm(dv, axis=1) - rad[k]).max() <= 1e-4 * dx + 1e-6, j
        jb = j + 1 if j % 2 == 0 else j - 1
        assert np.array_equal(dl[j][idx] + np.roll(dl[jb], -e[a], axis=2 - a)[idx], np.ones(len(k), np.float32))
        n += len(k)
    assert n > 1000


def test_sphere_link_positions_lie_on_the_spheres():
    _check_link_positions(synth.spheres(48, 0.5, rmin=2.0, rmax=6.0, fraction=0.5, seed=4), 3)


def test_cylinder_link_positions_lie_on_the_cylinders():
    _check_link_positions(synth.cylinders(64, 0.5, seed=1), 2)


def test_disc_link_angles_are_consistent_and_mirror_antisymmetric():
    """synth.link_angles on a disc whose centre lies on a node row. The two
    ends of a link carry opposite angles. Reflecting y about that row maps
    the disc onto itself: the x links' angles change sign, and the +y and -y
    links swap with equal angles (the normal's y part flips while e_j does
    too)."""
    n, dx = 40, 0.5
    c = (n // 2) * dx
    g = synth.disks(n, dx, [[c + 0.137, c]], [6.3])
    th = synth.link_angles(g, (0, 0, 0))[:, 0]
    assert np.count_nonzero(th) > 100 and not np.any(th[4:])
    for j, (ex, ey) in enumerate([(1, 0), (-1, 0), (0, 1), (0, -1)]):
        jb = j + 1 if j % 2 == 0 else j - 1
        far = np.roll(np.roll(th[jb], -ey, axis=0), -ex, axis=1)
        assert np.array_equal(th[j], -far), j
    refl = lambda a: np.roll(a[::-1], 1, axis=0)
    assert np.array_equal(refl(g.labels[0]), g.labels[0])
    assert np.array_equal(refl(th[0]), -th[0]) and np.array_equal(refl(th[1]), -th[1])
    assert np.array_equal(refl(th[2]), th[3]) and np.array_equal(refl(th[3]), th[2])
