"""Slab decomposition of one grid along z (the paper's strip decomposition,
Sec. 2.5, with the cut along z).

A grid of ``nz`` planes is split into slabs of consecutive planes.  Each slab
is one library context (``lbmbt_set_geometry_slab``); per time step a slab
needs, from each neighbour, one plane of one population: the lower neighbour's
hat g_5 of its last plane (moving +z) and the upper neighbour's hat g_6 of its
first plane (moving -z).  Across the periodic global face the receiving slab
applies the wrap factor itself (face kind ``FACE_HALO_WRAP``); a mirror
global face is the slab's own (``FACE_OWN``).

Two drivers share the same face bookkeeping:

* ``SlabGroup`` -- several slabs on one GPU in one process (all contexts on one
  stream, never the legacy default stream; faces move by device copies).  No kernel waits on another: each step
  is faces -> halos -> one sweep per slab, issued in that order.
* ``run_distributed`` -- one slab per rank of a ``torch.distributed`` group;
  faces move by point-to-point send/recv between neighbouring ranks.

Argument marshalling and bookkeeping only: every sweep runs in the CUDA
library.
"""
from __future__ import annotations

import numpy as np

from . import lbmbt

FACE_OWN, FACE_HALO, FACE_HALO_WRAP = lbmbt.FACE_OWN, lbmbt.FACE_HALO, lbmbt.FACE_HALO_WRAP


def split(nz: int, n_slabs: int):
    """Plane ranges [(z0, z1), ...] of ``n_slabs`` slabs, sizes differing by at most one."""
    if not 1 <= n_slabs <= nz:
        raise ValueError(f"cannot cut {nz} planes into {n_slabs} slabs")
    q, r = divmod(nz, n_slabs)
    out, z = [], 0
    for i in range(n_slabs):
        n = q + (1 if i < r else 0)
        out.append((z, z + n))
        z += n
    return out


def face_kinds(z0: int, z1: int, nz: int, bc_z: int):
    """(lo_kind, hi_kind) of slab [z0, z1) of a grid of nz planes."""
    def kind(at_face):
        if not at_face:
            return FACE_HALO
        return FACE_HALO_WRAP if bc_z == lbmbt.BC_PERIODIC else FACE_OWN
    return kind(z0 == 0), kind(z1 == nz)


def ghost_labels(labels: np.ndarray, z0: int, z1: int, bc_z: int) -> np.ndarray:
    """Labels of slab [z0, z1) with the plane below and the plane above
    (wrapped across a periodic global face; at a mirror global face the face
    plane itself, which the library ignores)."""
    nz = labels.shape[0]
    below = z0 - 1 if z0 > 0 else (nz - 1 if bc_z == lbmbt.BC_PERIODIC else 0)
    above = z1 if z1 < nz else (0 if bc_z == lbmbt.BC_PERIODIC else nz - 1)
    return np.ascontiguousarray(np.concatenate([labels[below:below + 1], labels[z0:z1], labels[above:above + 1]]),
                                np.int32)


def neighbours(i: int, n: int, lo_kind: int, hi_kind: int):
    """Indices of the slabs across the low and high face (None at an own face)."""
    lo = None if lo_kind == FACE_OWN else (i - 1) % n
    hi = None if hi_kind == FACE_OWN else (i + 1) % n
    return lo, hi


class SlabGroup:
    """``n_slabs`` slabs of one grid on one GPU, one context each, one stream."""

    def __init__(self, labels, phase_of_label, dx, bc, n_slabs, D, T2, dt, f, members, stream, kernel=0,
                 field=False, options=None):
        import torch
        labels = np.ascontiguousarray(labels, np.int32)
        nz, ny, nx = labels.shape
        self.shape = (nz, ny, nx)
        self.ranges = split(nz, n_slabs)
        self.n_members = len(members)
        # every context must issue on the same stream, so faces, halos and
        # sweeps of different slabs stay ordered; the legacy default stream
        # (handle 0) would give each context a stream of its own
        if stream is None or getattr(stream, "cuda_stream", stream) == 0:
            stream = torch.cuda.Stream()
        self.stream = stream
        self.solvers, self.kinds = [], []
        self.fields = []
        for (z0, z1) in self.ranges:
            s = lbmbt.Solver(torch.cuda.current_device(), stream)
            if kernel:
                s.set_option(lbmbt.OPT_KERNEL, kernel)
            for opt, val in (options or {}).items():   # further per-context options
                s.set_option(opt, val)
            lo, hi = face_kinds(z0, z1, nz, bc[2])
            s.set_geometry_slab(ghost_labels(labels, z0, z1, bc[2]), phase_of_label, dx, bc, z0, nz, lo, hi)
            s.set_phases(D, T2)
            s.set_sequence(dt, f, list(members[0].gamma_G0))
            if field:
                fld = torch.empty((z1 - z0) * ny * nx, dtype=torch.complex64, device="cuda")
                s.set_field(fld)
                self.fields.append(fld)
            s.prepare(members)
            self.solvers.append(s)
            self.kinds.append((lo, hi))
        dev = torch.device("cuda", torch.cuda.current_device())
        mk = lambda: torch.empty((ny, nx), dtype=torch.complex64, device=dev)
        self.lo_face = [[mk() for _ in range(self.n_members)] for _ in self.ranges]
        self.hi_face = [[mk() for _ in range(self.n_members)] for _ in self.ranges]

    def exchange(self):
        """Move every slab's faces into its neighbours' halos (device copies on the stream)."""
        n = len(self.solvers)
        for i, s in enumerate(self.solvers):
            for m in range(self.n_members):
                s.slab_faces(m, self.lo_face[i][m], self.hi_face[i][m])
        for i, s in enumerate(self.solvers):
            lo, hi = neighbours(i, n, *self.kinds[i])
            for m in range(self.n_members):
                s.slab_set_halos(m, None if lo is None else self.hi_face[lo][m],
                                 None if hi is None else self.lo_face[hi][m])

    def step(self, want_signal=False):
        """One time step of the whole grid; with want_signal the summed Z per member."""
        self.exchange()
        Z = np.zeros(self.n_members, np.complex128)
        for s in self.solvers:
            sig = s.advance(1, want_signal=want_signal, n_members=self.n_members)
            if want_signal:
                Z += sig[:, 0] + 1j * sig[:, 1]
        return Z if want_signal else None

    def run(self, n_steps):
        """``n_steps`` steps; returns {Z, S} per member at the end (S = |Z| / N of the whole grid)."""
        Z = None
        for k in range(n_steps):
            Z = self.step(want_signal=(k == n_steps - 1))
        n = float(np.prod(self.shape))
        return {"Z": Z, "S": np.abs(Z) / n}

    def field(self):
        """M(x, t_end) of the whole grid (member 0), when built with field=True."""
        import torch
        return torch.cat(self.fields)

    def close(self):
        for s in self.solvers:
            s.close()
        self.solvers = []


def exchange_faces(lo_face, hi_face, rank, world, lo_kind, hi_kind, group=None):
    """Point-to-point face exchange between neighbouring ranks of a slab run.

    lo_face / hi_face: this rank's outgoing faces (tensors [ny, nx] complex64,
    on the device the group's backend works with).  Returns (lo_halo,
    hi_halo): the lower neighbour's hi_face and the upper neighbour's lo_face
    (None at an own face).  A single rank across a periodic face is its own
    neighbour.  Sends and receives are posted together, so the ring cannot
    deadlock.  A face moving down carries tag 0, one moving up tag 1, and
    every rank posts its sends (down, up) and receives (from above, from
    below) in that order, so two ranks that are each other's upper and lower
    neighbour (two ranks on a periodic axis) still pair the messages right
    on backends that match by order."""
    import torch
    import torch.distributed as dist
    lo, hi = neighbours(rank, world, lo_kind, hi_kind)
    lo_halo = None if lo is None else torch.empty_like(hi_face)
    hi_halo = None if hi is None else torch.empty_like(lo_face)
    if world == 1:
        if lo is not None:
            lo_halo.copy_(hi_face)
        if hi is not None:
            hi_halo.copy_(lo_face)
        return lo_halo, hi_halo
    # complex tensors travel as real views (not every backend sends complex)
    r = torch.view_as_real
    ops = []
    if lo is not None:
        ops.append(dist.P2POp(dist.isend, r(lo_face).contiguous(), lo, group, 0))
    if hi is not None:
        ops.append(dist.P2POp(dist.isend, r(hi_face).contiguous(), hi, group, 1))
    if hi is not None:
        ops.append(dist.P2POp(dist.irecv, r(hi_halo), hi, group, 0))
    if lo is not None:
        ops.append(dist.P2POp(dist.irecv, r(lo_halo), lo, group, 1))
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    return lo_halo, hi_halo


def run_distributed(make_solver, nz, bc_z, n_steps, n_members, face_shape, rank, world, device=None, group=None):
    """One slab per rank: ``make_solver(z0, z1, lo_kind, hi_kind)`` returns a
    prepared solver of slab [z0, z1) (``lbmbt.Solver`` or any object with
    ``slab_faces``, ``slab_set_halos`` and ``advance``).  Runs ``n_steps``
    steps with a face exchange before each and returns the summed Z per member
    (all-reduced over the ranks) at the end."""
    import torch
    import torch.distributed as dist
    z0, z1 = split(nz, world)[rank]
    lo_kind, hi_kind = face_kinds(z0, z1, nz, bc_z)
    s = make_solver(z0, z1, lo_kind, hi_kind)
    dev = device if device is not None else torch.device("cpu")
    lo_f = [torch.empty(face_shape, dtype=torch.complex64, device=dev) for _ in range(n_members)]
    hi_f = [torch.empty(face_shape, dtype=torch.complex64, device=dev) for _ in range(n_members)]
    Z = torch.zeros(n_members, 2, dtype=torch.float64, device=dev)
    for k in range(n_steps):
        for m in range(n_members):
            s.slab_faces(m, lo_f[m], hi_f[m])
        if dev.type == "cuda":
            torch.cuda.synchronize(dev)   # the face copies run on the solver's stream
        for m in range(n_members):
            lo_h, hi_h = exchange_faces(lo_f[m], hi_f[m], rank, world, lo_kind, hi_kind, group)
            s.slab_set_halos(m, lo_h, hi_h)
        last = k == n_steps - 1
        sig = s.advance(1, want_signal=last, n_members=n_members)
        if last:
            Z += torch.as_tensor(np.asarray(sig)[:, :2], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(Z, group=group)
    return Z[:, 0].cpu().numpy() + 1j * Z[:, 1].cpu().numpy()
