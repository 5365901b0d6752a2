"""Seeded synthetic tissue geometries and gradient-direction sets.

This module only makes inputs: int32 compartment-label volumes (x fastest,
shape [nz, ny, nx]) with a phase id per label, and direction / b-value lists.
It holds none of the lattice scheme's arithmetic, so the CUDA path and the
FP64 oracle can both be fed from it.  Every generator is deterministic in its
seed (numpy PCG64).

Node n of an axis sits at x_n = n*dx, the lattice convention of the solver.

Geometries follow the tissue models of the paper (Sec. 2.1: fibres in an
extracellular matrix; Sec. 3.5: z-aligned cylinders; Sec. 3.8: cells from a
micrograph, here replaced by a Voronoi tessellation):

* ``planes``     -- parallel slabs normal to one axis (restricted-diffusion tests)
* ``cylinders``  -- non-overlapping z-aligned cylinders, gamma-distributed radii
* ``spheres``    -- non-overlapping sphere pack, uniform radii
* ``voronoi_tissue`` -- Voronoi cells + extracellular band + vessel tubes
* ``walls``      -- planes at arbitrary positions (membranes off the half-links)
* ``stripes``    -- 2-D periodic stripes oblique to the lattice (one z plane)
* ``disks``      -- 2-D discs at given centres and radii (one z plane)

``link_distances`` gives, for the analytic geometries (walls, stripes,
spheres, cylinders, discs), where each membrane cuts its lattice link: the
input of the membrane rule with a per-link distance (Eqs. B4a-B4c);
``link_angles`` gives, for the 2-D ones, the angle between the membrane
normal and each cut link (the general-angle rule of Appendix B).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PHASE_EX = 0  # extracellular
PHASE_IN = 1  # intracellular


@dataclass
class Geometry:
    labels: np.ndarray            # int32 [nz, ny, nx]
    phase_of_label: np.ndarray    # uint8 [n_labels]
    dx: float
    info: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.labels.shape

    @property
    def n_sites(self):
        return int(self.labels.size)

    def phase_fractions(self, n_phases=None):
        ph = self.phase_of_label[self.labels]
        n = n_phases or int(self.phase_of_label.max()) + 1
        return np.bincount(ph.ravel(), minlength=n) / ph.size


def uniform(n, dx=1.0):
    """Single compartment, single phase: free diffusion."""
    nz, ny, nx = (n, n, n) if np.isscalar(n) else n
    return Geometry(np.zeros((nz, ny, nx), np.int32), np.zeros(1, np.uint8), dx, {"kind": "uniform"})


def planes(shape, dx, widths, axis=0, phases=None):
    """Slabs normal to ``axis`` (0 = x); slab j has ``widths[j]`` nodes and label j.

    The walls sit at the half-links between slabs, so slab j is
    ``widths[j]*dx`` thick.  The widths repeat to fill the axis.
    """
    nz, ny, nx = shape
    n_ax = (nx, ny, nz)[axis]
    lab1 = np.empty(n_ax, np.int32)
    pos, j = 0, 0
    while pos < n_ax:
        w = widths[j % len(widths)]
        lab1[pos:pos + w] = j
        pos += w
        j += 1
    n_labels = j
    if axis == 0:
        labels = np.broadcast_to(lab1[None, None, :], shape)
    elif axis == 1:
        labels = np.broadcast_to(lab1[None, :, None], shape)
    else:
        labels = np.broadcast_to(lab1[:, None, None], shape)
    if phases is None:
        pol = np.zeros(n_labels, np.uint8)
    else:
        pol = np.array([phases[i % len(phases)] for i in range(n_labels)], np.uint8)
    return Geometry(np.ascontiguousarray(labels, np.int32), pol, dx, {"kind": "planes", "widths": list(widths)})


def walls(n, dx, positions, axis=0, cross=(1, 1), phases=None, periodic=True):
    """Planes normal to ``axis`` at the given positions (um, increasing, inside
    [0, n*dx)), not tied to the half-links.  Node k (at k*dx) gets label j =
    the number of walls at or below it; on a periodic axis the segment after
    the last wall continues into the first (label 0).  ``cross`` = sizes of
    the two other axes (in z, y, x order without ``axis``)."""
    pos = np.asarray(positions, np.float64)
    xk = np.arange(n) * dx
    lab1 = np.searchsorted(pos, xk, side="right").astype(np.int32)
    n_labels = len(pos) + 1
    if periodic and len(pos) > 0:
        lab1 %= len(pos)
        n_labels = len(pos)
    if axis == 0:
        labels = np.broadcast_to(lab1[None, None, :], (cross[0], cross[1], n))
    elif axis == 1:
        labels = np.broadcast_to(lab1[None, :, None], (cross[0], n, cross[1]))
    else:
        labels = np.broadcast_to(lab1[:, None, None], (n, cross[0], cross[1]))
    if phases is None:
        pol = np.zeros(n_labels, np.uint8)
    else:
        pol = np.array([phases[i % len(phases)] for i in range(n_labels)], np.uint8)
    return Geometry(np.ascontiguousarray(labels, np.int32), pol, dx,
                    {"kind": "walls", "positions": pos.tolist(), "axis": axis})


def stripes(n, dx, slope=(1, 1), width=0.5, offset=0.0, phases=None):
    """Periodic stripes on an n x n grid of one z plane, running along
    (q, p) for ``slope`` = (p, q) (coprime integers): with the unit normal
    N = (-p, q) / sqrt(p^2 + q^2) and the pattern period Lam = n dx /
    sqrt(p^2 + q^2) (so the pattern is periodic on the box), label 1 where
    (N.x - offset) mod Lam < width * Lam, label 0 elsewhere; the walls are the
    lines N.x = offset + m Lam and N.x = offset + width Lam + m Lam."""
    p, q = slope
    h = math.hypot(p, q)
    N = np.array([-p / h, q / h])
    lam = n * dx / h
    xk = np.arange(n) * dx
    u = N[0] * xk[None, :] + N[1] * xk[:, None]
    lab2 = (np.mod(u - offset, lam) < width * lam).astype(np.int32)
    labels = np.ascontiguousarray(lab2[None], np.int32)
    pol = np.zeros(2, np.uint8) if phases is None else np.array(phases[:2], np.uint8)
    return Geometry(labels, pol, dx, {"kind": "stripes", "normal": N.tolist(), "period": lam,
                                      "walls": [offset, offset + width * lam]})


def disks(n, dx, centers, radii, phases=None):
    """Discs (x, y centres in um, radii in um) on an n x n periodic grid of one
    z plane: label j >= 1 inside disc j (minimum image; the first disc wins
    where two overlap), label 0 outside."""
    L = n * dx
    xk = np.arange(n) * dx
    lab2 = np.zeros((n, n), np.int32)
    for j, (c, r) in enumerate(zip(centers, radii)):
        dxv = xk[None, :] - c[0]
        dyv = xk[:, None] - c[1]
        dxv -= L * np.round(dxv / L)
        dyv -= L * np.round(dyv / L)
        lab2[(dxv * dxv + dyv * dyv < r * r) & (lab2 == 0)] = j + 1
    pol = np.full(len(radii) + 1, PHASE_IN, np.uint8)
    pol[0] = PHASE_EX
    if phases is not None:
        pol[:] = phases[1]
        pol[0] = phases[0]
    g = Geometry(np.ascontiguousarray(lab2[None], np.int32), pol, dx,
                 {"kind": "cylinders", "centers": np.asarray(centers, float).tolist(),
                  "radii": np.asarray(radii, float).tolist()})
    g.info["intra_fraction"] = float((lab2 > 0).mean())
    return g


_DIRS = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))   # +x -x +y -y +z -z


def _membrane_links(lab, bc, j):
    """Nodes whose link along direction j carries a membrane (periodic wrap;
    none across a mirror face)."""
    nz, ny, nx = lab.shape
    dims = (nx, ny, nz)
    e = _DIRS[j]
    a = j // 2
    nb = np.roll(lab, -e[a], axis=2 - a)
    memb = nb != lab
    if bc[a] != 0:
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        node = (xx, yy, zz)[a]
        memb &= node != (dims[a] - 1 if e[a] > 0 else 0)
    return memb, nb


def _stripe_cut(geom, idx, j):
    """Distance (um) along direction j from the nodes idx to the first stripe
    wall, for a ``stripes`` geometry."""
    N = np.asarray(geom.info["normal"])
    lam = geom.info["period"]
    e = np.array(_DIRS[j][:2], float)
    ne = N @ e
    px = np.stack([idx[2] * geom.dx, idx[1] * geom.dx], 1)
    u = px @ N
    best = np.full(len(u), np.inf)
    for w in geom.info["walls"]:
        for m in range(-3, 4):
            # N.(x + t e) = w + (k + m) Lam with k the period index near x
            k = np.floor((u - w) / lam)
            t = (w + (k + m) * lam - u) / ne
            ok = (t > 0) & (t <= geom.dx * (1 + 1e-12))
            best = np.where(ok & (t < best), t, best)
    return best


def link_angles(geom: Geometry, bc=(0, 0, 0)):
    """Angle between the membrane normal and each cut link, for the 2-D
    analytic geometries (stripes, discs).

    Returns float32 [6, 1, ny, nx]: entry j at node s is theta such that the
    unit normal of the membrane on the link from s to s + e_j, pointing from
    s's compartment to the other, is cos(theta) e_j + sin(theta) e_perp, with
    e_perp = +y for the x links and +x for the y links (so the two ends of a
    link carry opposite angles); 0 where the link carries no membrane and on
    the z links.  |theta| is kept below pi/2 - 1e-3.
    """
    lab = geom.labels
    nz, ny, nx = lab.shape
    if nz != 1:
        raise ValueError("membrane angles are defined for one-plane (2-D) geometries")
    kind = geom.info.get("kind")
    if kind not in ("stripes", "cylinders"):
        raise ValueError(f"no membrane angles for a '{kind}' geometry")
    out = np.zeros((6, 1, ny, nx), np.float32)
    dl = link_distances(geom, bc)
    L = np.array([nx, ny], float) * geom.dx
    for j in range(4):
        memb, nb = _membrane_links(lab, bc, j)
        if not memb.any():
            continue
        idx = np.nonzero(memb)
        e = np.array(_DIRS[j][:2], float)
        perp = np.array([0.0, 1.0]) if j < 2 else np.array([1.0, 0.0])
        if kind == "stripes":
            N = np.asarray(geom.info["normal"], float)
            n_out = np.sign(N @ e) * np.tile(N, (len(idx[0]), 1))
        else:
            cen = np.asarray(geom.info["centers"], float)[:, :2]
            la, lb = lab[idx], nb[idx]
            k = np.where((la > 0) & (lb > 0), np.minimum(la, lb), np.where(la > 0, la, lb)) - 1
            px = np.stack([idx[2] * geom.dx, idx[1] * geom.dx], 1)
            cut = px + (dl[j][idx].astype(np.float64) * geom.dx)[:, None] * e[None, :]
            r = cut - cen[k]
            r -= L * np.round(r / L)
            r /= np.linalg.norm(r, axis=1)[:, None]
            # outward from the disc; from s's side towards the other
            n_out = np.where((la == k + 1)[:, None], r, -r)
        c = n_out @ e
        sn = n_out @ perp
        th = np.arctan2(sn, np.maximum(c, 1e-12))
        out[j][idx] = np.clip(th, -(math.pi / 2 - 1e-3), math.pi / 2 - 1e-3)
    return out


def link_distances(geom: Geometry, bc=(0, 0, 0)):
    """Where membranes cut the lattice links, for the analytic geometries.

    Returns float32 [6, nz, ny, nx]: entry j at node s is the distance, in
    units of dx, from s to the membrane on its link to s + e_j (directions
    +x, -x, +y, -y, +z, -z), 0.5 where the link carries no membrane.  Walls
    are exact; for spheres and cylinders the link is cut where it leaves the
    sphere (cylinder) of whichever end node lies inside one (periodic minimum
    image).  Values are clipped to [1e-4, 1 - 1e-4].
    """
    lab = geom.labels
    nz, ny, nx = lab.shape
    dims = (nx, ny, nz)
    dx = geom.dx
    out = np.full((6, nz, ny, nx), 0.5, np.float32)
    kind = geom.info.get("kind")
    if kind not in ("walls", "spheres", "cylinders", "stripes"):
        raise ValueError(f"no sub-voxel membrane positions for a '{kind}' geometry")
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    node = [xx, yy, zz]
    for j, e in enumerate(_DIRS):
        a = j // 2
        nb = lab
        # neighbour label (periodic wrap; none across a mirror face)
        nb = np.roll(lab, -e[a], axis=2 - a)
        exists = np.ones(lab.shape, bool)
        if bc[a] != 0:
            edge = node[a] == (dims[a] - 1 if e[a] > 0 else 0)
            exists &= ~edge
        memb = exists & (nb != lab)
        if not memb.any():
            continue
        idx = np.nonzero(memb)
        if kind == "stripes":
            if a == 2:
                continue
            d = _stripe_cut(geom, idx, j) / dx
        elif kind == "walls":
            if geom.info["axis"] != a:
                continue
            pos = np.asarray(geom.info["positions"])
            x0 = node[a][idx] * dx
            L = dims[a] * dx
            # the wall between x0 and x0 + e dx (periodic: positions repeat with L)
            cand = np.concatenate([pos - L, pos, pos + L])
            t = (cand[None, :] - x0[:, None]) * e[a]
            t[(t < 0) | (t > dx)] = np.inf
            d = t.min(axis=1) / dx
        else:
            cen = np.asarray(geom.info["centers"], np.float64)
            rad = np.asarray(geom.info["radii"], np.float64)
            box = np.array([nx, ny, nz], np.float64) * dx
            la, lb = lab[idx], nb[idx]
            # the body one end lies in; between two bodies the lower label's,
            # so both ends of a link see the same membrane
            k = np.where((la > 0) & (lb > 0), np.minimum(la, lb), np.where(la > 0, la, lb)) - 1
            p = np.stack([node[c][idx] * dx for c in range(3)], 1)
            ndim = 3 if kind == "spheres" else 2
            c3 = np.zeros((len(k), 3))
            c3[:, :ndim] = cen[k][:, :ndim]
            dv = p - c3
            if ndim == 2:
                dv[:, 2] = 0.0
            dv -= box * np.round(dv / box)
            ev = np.array(e, np.float64)
            if ndim == 2:
                ev[2] = 0.0
            bq = dv @ ev
            cq = (dv * dv).sum(1) - rad[k] ** 2
            disc = np.sqrt(np.maximum(bq * bq - cq, 0.0))
            r1, r2 = -bq - disc, -bq + disc
            t = np.where((r1 > 0) & (r1 < dx), r1, r2)
            d = t / dx
        out[j][idx] = np.clip(d, 1e-4, 1 - 1e-4)
    return out


def _relax_periodic(centers, radii, box, gap, max_iter=4000, rng=None):
    """Place discs/spheres without overlap in a periodic box.

    Radii are grown from 60 % to full size in steps; after each growth step
    overlapping pairs (found with a periodic KD-tree) are pushed apart along
    their centre line (minimum image) until none overlap.  Returns the
    centres and the iterations used.
    """
    from scipy.spatial import cKDTree

    c = np.array(centers, dtype=np.float64) % box
    dim = c.shape[1]
    boxv = np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,)).copy()
    total = 0
    for scale in np.linspace(0.6, 1.0, 9):
        rad = radii * scale
        reach = 2.0 * float(rad.max()) + gap
        for it in range(max_iter):
            tree = cKDTree(c, boxsize=boxv)
            pairs = tree.query_pairs(reach, output_type="ndarray")
            if len(pairs) == 0:
                break
            i, j = pairs[:, 0], pairs[:, 1]
            d = c[i] - c[j]
            d -= boxv * np.round(d / boxv)
            dist = np.sqrt((d * d).sum(-1))
            need = rad[i] + rad[j] + gap
            bad = dist < need
            if not bad.any():
                break
            i, j, d, dist, need = i[bad], j[bad], d[bad], dist[bad], need[bad]
            ov = need + 1e-6 - dist  # push slightly past contact
            safe = np.where(dist > 1e-12, dist, 1.0)
            u = d / safe[:, None]
            coinc = dist <= 1e-12
            if coinc.any():
                rnd = (rng or np.random.default_rng(0)).normal(size=(int(coinc.sum()), dim))
                u[coinc] = rnd / np.linalg.norm(rnd, axis=1, keepdims=True)
            wi = rad[j] ** dim / (rad[i] ** dim + rad[j] ** dim)
            push = 0.55 * ov[:, None] * u
            np.add.at(c, i, push * wi[:, None])
            np.add.at(c, j, -push * (1.0 - wi)[:, None])
            c %= boxv
            total += 1
        else:
            raise RuntimeError("packing relaxation did not converge; lower the target fraction")
    return c, total


def cylinders(n, dx, mean_radius=3.0, cv=0.3, fraction=0.6, seed=0, gap=None):
    """z-aligned non-overlapping cylinders in a periodic n x n x n box.

    Radii ~ Gamma(shape 1/cv^2, scale mean*cv^2), sampled until the summed
    cross-section reaches ``fraction`` of the box area, then placed at random
    and relaxed until no two overlap (periodic).  Label 0 = extracellular,
    label j >= 1 = cylinder j (phase 1).  The achieved voxel fraction is in
    ``info``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n * dx
    gap = 0.0 if gap is None else gap
    k = 1.0 / (cv * cv)
    radii = []
    area = 0.0
    while area < fraction * L * L:
        r = float(rng.gamma(k, mean_radius / k))
        r = min(max(r, 2.0 * dx), 0.3 * L)
        radii.append(r)
        area += math.pi * r * r
    radii = np.array(sorted(radii, reverse=True))
    # trim the last disc so the analytic fraction is not overshot by much
    centers = rng.uniform(0, L, size=(len(radii), 2))
    centers, iters = _relax_periodic(centers, radii, L, gap, rng=rng)
    ys = np.arange(n) * dx
    lab2 = np.zeros((n, n), np.int32)
    for j, (c, r) in enumerate(zip(centers, radii)):
        dxv = ys[None, :] - c[0]
        dyv = ys[:, None] - c[1]
        dxv -= L * np.round(dxv / L)
        dyv -= L * np.round(dyv / L)
        inside = dxv * dxv + dyv * dyv < r * r
        lab2[inside & (lab2 == 0)] = j + 1
    labels = np.ascontiguousarray(np.broadcast_to(lab2[None], (n, n, n)), np.int32)
    pol = np.full(len(radii) + 1, PHASE_IN, np.uint8)
    pol[0] = PHASE_EX
    g = Geometry(labels, pol, dx, {"kind": "cylinders", "n_cyl": len(radii), "seed": seed,
                                   "target_fraction": fraction, "relax_iters": iters,
                                   "centers": np.asarray(centers).tolist(), "radii": radii.tolist()})
    g.info["intra_fraction"] = float((lab2 > 0).mean())
    return g


def spheres(n, dx, rmin=2.0, rmax=6.0, fraction=0.5, seed=0, gap=None):
    """Non-overlapping sphere pack in a periodic n^3 box, radii ~ U(rmin, rmax).

    Label 0 = extracellular, label j >= 1 = sphere j (phase 1).  Radii are drawn
    until the summed volume reaches ``fraction`` of the box, positions relaxed
    until no overlap (periodic).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    box = np.array([nx, ny, nz], np.float64) * dx
    vol = float(np.prod(box))
    gap = 0.0 if gap is None else gap
    radii = []
    v = 0.0
    rcap = 0.45 * float(box.min())
    while v < fraction * vol:
        r = min(float(rng.uniform(rmin, rmax)), rcap)
        radii.append(r)
        v += 4.0 / 3.0 * math.pi * r ** 3
    radii = np.array(sorted(radii, reverse=True))
    centers = rng.uniform(0, 1, size=(len(radii), 3)) * box
    centers, iters = _relax_periodic(centers, radii, box, gap, rng=rng)
    labels = np.zeros((nz, ny, nx), np.int32)
    ax = [np.arange(m) * dx for m in (nx, ny, nz)]
    for j, (c, r) in enumerate(zip(centers, radii)):
        lo = [int(math.floor((c[a] - r) / dx)) for a in range(3)]
        hi = [int(math.ceil((c[a] + r) / dx)) + 1 for a in range(3)]
        idx = [np.arange(lo[a], hi[a]) for a in range(3)]
        d = []
        for a in range(3):
            p = idx[a] * dx - c[a]
            d.append(p)
        rr = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
        inside = rr < r * r
        zi = idx[2] % nz
        yi = idx[1] % ny
        xi = idx[0] % nx
        sub = labels[np.ix_(zi, yi, xi)]
        sub = np.where(inside & (sub == 0), j + 1, sub)
        labels[np.ix_(zi, yi, xi)] = sub
    pol = np.full(len(radii) + 1, PHASE_IN, np.uint8)
    pol[0] = PHASE_EX
    g = Geometry(labels, pol, dx, {"kind": "spheres", "n_spheres": len(radii), "seed": seed,
                                   "target_fraction": fraction, "relax_iters": iters,
                                   "centers": np.asarray(centers).tolist(), "radii": radii.tolist()})
    g.info["intra_fraction"] = float((labels > 0).mean())
    return g


def voronoi_tissue(n, dx, cell_diam=10.0, ecs_fraction=0.2, n_vessels=4, vessel_radius=3.0,
                   seed=0, chunk=1 << 22):
    """Voronoi cells with an extracellular band and straight vessel tubes.

    Seeds have density 1/(pi/6 d^3) so the mean cell volume matches a sphere
    of diameter ``cell_diam``; ties go to the lowest seed index.  A site is
    extracellular where (d2 - d1) < w, with w the ``ecs_fraction`` quantile of
    d2 - d1 (d1, d2: distances to the nearest and second-nearest seed).
    Vessels are z-aligned tubes of ``vessel_radius`` at seeded (x, y).
    Labels: 0 = extracellular (phase 1), 1..n_cells = cells (phase 0),
    n_cells+1.. = vessels (phase 2).
    """
    from scipy.spatial import cKDTree

    rng = np.random.Generator(np.random.PCG64(seed))
    L = n * dx
    n_cells = max(2, int(round(L ** 3 / (math.pi / 6.0 * cell_diam ** 3))))
    seeds = rng.uniform(0, L, size=(n_cells, 3))
    tree = cKDTree(seeds)
    coords = np.arange(n, dtype=np.float64) * dx
    N = n ** 3
    near = np.empty(N, np.int32)
    gapd = np.empty(N, np.float32)
    plane = n * n
    zs_per = max(1, chunk // plane)
    X, Y = np.meshgrid(coords, coords, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    for z0 in range(0, n, zs_per):
        z1 = min(n, z0 + zs_per)
        pts = np.concatenate([np.concatenate([xy, np.full((plane, 1), coords[z])], 1) for z in range(z0, z1)])
        d, i = tree.query(pts, k=2, workers=-1)
        near[z0 * plane:z1 * plane] = i[:, 0]
        gapd[z0 * plane:z1 * plane] = d[:, 1] - d[:, 0]
    w = float(np.quantile(gapd, ecs_fraction))
    labels = (near + 1).astype(np.int32)
    labels[gapd < w] = 0
    labels = labels.reshape(n, n, n)
    vx = rng.uniform(0, L, size=(n_vessels, 2))
    lab2 = np.full((n, n), -1, np.int32)
    for j, c in enumerate(vx):
        inside = (coords[None, :] - c[0]) ** 2 + (coords[:, None] - c[1]) ** 2 < vessel_radius ** 2
        lab2[inside & (lab2 < 0)] = n_cells + 1 + j
    vmask = lab2 >= 0
    labels[:, vmask] = lab2[vmask][None, :]
    pol = np.zeros(n_cells + 1 + n_vessels, np.uint8)
    pol[0] = 1
    pol[n_cells + 1:] = 2
    g = Geometry(np.ascontiguousarray(labels), pol, dx, {"kind": "voronoi", "n_cells": n_cells,
                                                          "n_vessels": n_vessels, "ecs_width_um": w,
                                                          "seed": seed})
    return g


def directions_on_sphere(n, seed=0):
    """``n`` unit vectors, normalised Gaussian triples (uniform on the sphere)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def crop(geom: Geometry, n):
    """Corner crop n^3 of a geometry (labels renumbered compactly)."""
    lab = geom.labels[:n, :n, :n]
    uniq, inv = np.unique(lab, return_inverse=True)
    return Geometry(inv.reshape(lab.shape).astype(np.int32), geom.phase_of_label[uniq].copy(), geom.dx,
                    dict(geom.info, cropped=n))
