"""Oracle values at sampled sites of a large run, from small crops.

After k steps the value at a site depends only on sites within distance k
(D3Q7 moves one site per step).  A crop of edge w around the site, with its
far edges more than k away, therefore gives the same value, up to the global
phase exp(-i gamma x0.G F_k) of the crop offset x0 (the reaction uses
absolute positions; the mirror rule with G normal to the face keeps that
relation, its rewind being conjugated with the field).  On a periodic axis
the crop is centred on the sample with wrapped indices (the offset may be
negative: the modified periodic condition is exactly that quasi-periodic
extension).  On a mirror axis a crop that reaches the low face starts
there, one that reaches the high face ends there, and either keeps the
mirror on both of its ends (the far one lies more than k sites from the
sample).  Elsewhere the crop's own edges are periodic; they never
influence the sample.
"""
import numpy as np

import oracle


def sample_values(labels, pol, bc, dx, D, T2, kappa, dt, f, gG, sites, k_steps):
    nz, ny, nx = labels.shape
    h = k_steps + 1
    w = 2 * h + 1
    F = float(np.sum(f[:k_steps]) * dt)
    out = []
    for (z, y, x) in sites:
        start, idx, cbc = [], [], []
        for a, (c, n) in enumerate(zip((x, y, z), (nx, ny, nz))):
            if bc[a] == 0:
                # periodic axis: centred crop with wrapped indices; the
                # unwrapped offset may be negative (quasi-periodic extension)
                s0 = c - h
                cbc.append(0)
            elif c - h <= 0:
                s0 = 0            # low mirror face inside the crop
                cbc.append(1)
            elif c + h >= n:
                assert n >= w, "axis shorter than the crop"
                s0 = n - w        # high mirror face inside the crop
                cbc.append(1)
            else:
                s0 = c - h
                cbc.append(0)
            start.append(s0)
            idx.append((s0 + np.arange(w)) % n)
        sub = labels[np.ix_(idx[2], idx[1], idx[0])]
        uniq, inv = np.unique(sub, return_inverse=True)
        sub = np.ascontiguousarray(inv.reshape(sub.shape).astype(np.int32))
        o = oracle.run(sub, dx, np.asarray(pol)[uniq], cbc, D, T2, kappa, dt, f[:k_steps], gG, want_field=True)
        ph = np.exp(-1j * (np.array(start, float) * dx) @ np.asarray(gG, float) * F)
        out.append(o["field"][z - start[2], y - start[1], x - start[0]] * ph)
    return np.array(out)
