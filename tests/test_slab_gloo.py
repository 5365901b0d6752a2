"""Slab decomposition along z (the strips of Sec. 2.5): the host-side
bookkeeping (plane ranges, face kinds, ghost labels, neighbours) and the
multi-rank face exchange on CPU ranks (gloo, world sizes 2 and 3), checked
bit for bit against a one-rank run.  The per-rank sweep is a stand-in with
the same face contract as the library (hat g_5 leaves through the high face,
hat g_6 through the low face, a wrap factor on the periodic global face, a
reflection at a mirror face) and a dependence on the global plane index, so
a wrong neighbour, a missing wrap or a wrong offset changes the result."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1907_00908_gb300 import lbmbt, slab


def test_split_covers_the_grid():
    for nz in (1, 5, 17, 64):
        for n in range(1, min(nz, 6) + 1):
            r = slab.split(nz, n)
            assert r[0][0] == 0 and r[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        slab.split(3, 4)


def test_face_kinds_and_neighbours():
    P, M = lbmbt.BC_PERIODIC, lbmbt.BC_MIRROR
    assert slab.face_kinds(0, 4, 12, P) == (slab.FACE_HALO_WRAP, slab.FACE_HALO)
    assert slab.face_kinds(4, 8, 12, P) == (slab.FACE_HALO, slab.FACE_HALO)
    assert slab.face_kinds(8, 12, 12, P) == (slab.FACE_HALO, slab.FACE_HALO_WRAP)
    assert slab.face_kinds(0, 4, 12, M) == (slab.FACE_OWN, slab.FACE_HALO)
    assert slab.face_kinds(8, 12, 12, M) == (slab.FACE_HALO, slab.FACE_OWN)
    assert slab.face_kinds(0, 12, 12, P) == (slab.FACE_HALO_WRAP, slab.FACE_HALO_WRAP)
    assert slab.neighbours(0, 3, slab.FACE_HALO_WRAP, slab.FACE_HALO) == (2, 1)
    assert slab.neighbours(2, 3, slab.FACE_HALO, slab.FACE_HALO_WRAP) == (1, 0)
    assert slab.neighbours(0, 3, slab.FACE_OWN, slab.FACE_HALO) == (None, 1)
    assert slab.neighbours(0, 1, slab.FACE_HALO_WRAP, slab.FACE_HALO_WRAP) == (0, 0)


def test_ghost_labels():
    lab = np.arange(5 * 2 * 2, dtype=np.int32).reshape(5, 2, 2)
    g = slab.ghost_labels(lab, 1, 3, lbmbt.BC_PERIODIC)
    assert np.array_equal(g, lab[[0, 1, 2, 3]])
    g = slab.ghost_labels(lab, 0, 2, lbmbt.BC_PERIODIC)
    assert np.array_equal(g, lab[[4, 0, 1, 2]])
    g = slab.ghost_labels(lab, 3, 5, lbmbt.BC_PERIODIC)
    assert np.array_equal(g, lab[[2, 3, 4, 0]])
    g = slab.ghost_labels(lab, 0, 5, lbmbt.BC_MIRROR)
    assert g.shape == (7, 2, 2) and np.array_equal(g[1:6], lab)


WRAP = np.complex64(np.exp(0.3j))


class FakeSlab:
    """Stand-in sweep on planes [z0, z1): a5 streams +z, a6 streams -z, then
    the two mix with a phase of the global plane index."""

    def __init__(self, z0, z1, lo_kind, hi_kind, n_members, shape, seed=3):
        ny, nx = shape
        rng = np.random.default_rng(seed)
        nzg = FakeSlab.nzg
        full5 = (rng.standard_normal((n_members, nzg, ny, nx)) + 1j * rng.standard_normal((n_members, nzg, ny, nx)))
        full6 = (rng.standard_normal((n_members, nzg, ny, nx)) + 1j * rng.standard_normal((n_members, nzg, ny, nx)))
        self.a5 = full5[:, z0:z1].astype(np.complex64)
        self.a6 = full6[:, z0:z1].astype(np.complex64)
        self.z0, self.z1, self.kinds = z0, z1, (lo_kind, hi_kind)
        self.halo = [[None, None] for _ in range(n_members)]
        self.ph = np.exp(0.1j * np.arange(z0, z1)).astype(np.complex64)[:, None, None]

    def slab_faces(self, m, lo_out, hi_out):
        lo_out.copy_(torch.from_numpy(self.a6[m, 0].copy()))
        hi_out.copy_(torch.from_numpy(self.a5[m, -1].copy()))

    def slab_set_halos(self, m, lo, hi):
        self.halo[m] = [None if lo is None else lo.numpy().copy(), None if hi is None else hi.numpy().copy()]

    def advance(self, n, want_signal=False, n_members=1):
        assert n == 1
        out = np.zeros((n_members, 3))
        for m in range(n_members):
            a5, a6 = self.a5[m], self.a6[m]
            n5 = np.empty_like(a5)
            n6 = np.empty_like(a6)
            n5[1:] = a5[:-1]
            n6[:-1] = a6[1:]
            lo, hi = self.kinds
            n5[0] = a6[0] if lo == slab.FACE_OWN else self.halo[m][0] * (WRAP if lo == slab.FACE_HALO_WRAP else 1)
            n6[-1] = a5[-1] if hi == slab.FACE_OWN else self.halo[m][1] * (np.conj(WRAP) if hi == slab.FACE_HALO_WRAP
                                                                          else 1)
            self.a5[m] = np.complex64(0.75) * n5 + np.complex64(0.25) * n6 * self.ph
            self.a6[m] = np.complex64(0.75) * n6 + np.complex64(0.25) * n5 * np.conj(self.ph)
            z = (self.a5[m].astype(np.complex128) + self.a6[m]).sum()
            out[m] = [z.real, z.imag, abs(z)]
        return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(rank, world, port, nzg, bc_z, steps, n_members, shape, outdir):
    if world > 1:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
    FakeSlab.nzg = nzg
    made = {}

    def make(z0, z1, lo, hi):
        made["s"] = FakeSlab(z0, z1, lo, hi, n_members, shape)
        return made["s"]

    Z = slab.run_distributed(make, nzg, bc_z, steps, n_members, shape, rank, world)
    s = made["s"]
    np.savez(os.path.join(outdir, f"w{world}_r{rank}.npz"), a5=s.a5, a6=s.a6, z0=s.z0, Z=Z)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("bc_z", [lbmbt.BC_PERIODIC, lbmbt.BC_MIRROR])
@pytest.mark.parametrize("world", [2, 3])
def test_gloo_slab_exchange_matches_one_rank(world, bc_z):
    nzg, steps, n_members, shape = 11, 9, 2, (3, 4)
    with tempfile.TemporaryDirectory() as d:
        _run(0, 1, 0, nzg, bc_z, steps, n_members, shape, d)
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_run, args=(r, world, port, nzg, bc_z, steps, n_members, shape, d))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        ref = np.load(os.path.join(d, "w1_r0.npz"))
        parts = [np.load(os.path.join(d, f"w{world}_r{r}.npz")) for r in range(world)]
        a5 = np.concatenate([p["a5"] for p in parts], axis=1)
        a6 = np.concatenate([p["a6"] for p in parts], axis=1)
        assert np.array_equal(a5, ref["a5"]) and np.array_equal(a6, ref["a6"])
        for p in parts:   # every rank holds the all-reduced signal
            np.testing.assert_allclose(p["Z"], ref["Z"], rtol=1e-12)
