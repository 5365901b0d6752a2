"""The allocation-free entry point, lbmbt_sweep_noalloc.

Callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or their loop must not enter the driver's allocator) run the plain
sweep on buffers they already own; the library keeps its working data in a
fixed file-scope device array.  This file checks, through the C ABI, that two
calls in a row give the same signal as lbmbt_run (within the signal tolerance
of the parity tests), that chained calls continue a run, that a call after the
first one changes no device memory use, that sizes beyond the stated limit
are refused, and that a mask naming more phases than given is refused.  It is collected last so a run stopping at the first failure has
already run every other test.
"""
import math

import numpy as np
import pytest

from paper_1907_00908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S_TOL = 1e-5


def _case():
    geom = synth.cylinders(40, 0.5, seed=17)
    dt = 0.025
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.02
    return geom, (0, 0, 0), D, T2, kap, dt


def test_noalloc_matches_run_on_two_calls():
    from paper_1907_00908_gb300 import lbmbt
    geom, bc, D, T2, kap, dt = _case()
    gG, f = lbmbt.pgse(2500.0, 2.0, 5.0, dt, (0.6, 0.0, 0.8))
    with lbmbt.Solver(0) as s:
        s.set_geometry(geom.labels, geom.phase_of_label, geom.dx, bc)
        s.set_phases(D, T2)
        s.set_permeability(kap)
        s.set_sequence(dt, f, gG)
        ref = s.run()
        mask = s.get_mask(0)
    N = geom.n_sites
    plane = (N + 63) // 64 * 64
    mask_dev = torch.from_numpy(mask).cuda()
    state = torch.zeros(2 * 7 * plane, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()

    r1 = lbmbt.sweep_noalloc(mask_dev, geom.shape, geom.dx, bc, D, T2, kap, dt, f, gG, state)
    assert abs(r1["S"] - ref["S"]) <= S_TOL * ref["S"]

    free_before, _ = torch.cuda.mem_get_info()
    r2 = lbmbt.sweep_noalloc(mask_dev, geom.shape, geom.dx, bc, D, T2, kap, dt, f, gG, state)
    free_after, _ = torch.cuda.mem_get_info()
    assert abs(r2["S"] - ref["S"]) <= S_TOL * ref["S"]
    assert r2["Z"] == r1["Z"]
    assert free_after == free_before

    # chained: steps [0, K/2) then [K/2, K) continue the same run
    K = len(f)
    lbmbt.sweep_noalloc(mask_dev, geom.shape, geom.dx, bc, D, T2, kap, dt, f, gG, state, k0=0, n_steps=K // 2)
    r3 = lbmbt.sweep_noalloc(mask_dev, geom.shape, geom.dx, bc, D, T2, kap, dt, f, gG, state, k0=K // 2,
                             n_steps=K - K // 2, init=False)
    assert abs(r3["S"] - ref["S"]) <= S_TOL * ref["S"]


def _raw_call(lbmbt, mask, shape, n_phases, f, state):
    """The C entry point itself (the binding checks buffer sizes first; the
    library's own checks below refuse before touching any buffer)."""
    import ctypes
    L = lbmbt.lib()
    nz, ny, nx = shape
    D = np.full(n_phases, 2.0)
    T2 = np.full(n_phases, math.inf)
    bc = np.zeros(3, np.int32)
    gG = np.array([0.01, 0.0, 0.0])
    fv = np.ascontiguousarray(f, np.float64)
    sig = np.zeros(3)
    err = ctypes.create_string_buffer(256)
    rc = L.lbmbt_sweep_noalloc(nx, ny, nz, 0.5, lbmbt._p(mask), lbmbt._p(bc), n_phases, lbmbt._p(D), lbmbt._p(T2),
                               math.inf, 0.01, int(fv.size), lbmbt._p(fv), lbmbt._p(gG), lbmbt._p(state), 0,
                               int(fv.size), 1, lbmbt._p(sig), None, err, 256)
    return rc, err.value.decode()


def test_noalloc_rejects_sizes_beyond_the_limit():
    from paper_1907_00908_gb300 import lbmbt
    dummy = torch.zeros(64, dtype=torch.uint8, device="cuda")
    state = torch.zeros(64, dtype=torch.complex64, device="cuda")
    rc, msg = _raw_call(lbmbt, dummy, (257, 256, 256), 1, np.zeros(10), state)
    assert rc == -1 and "16,777,216" in msg
    rc, msg = _raw_call(lbmbt, dummy, (4, 4, 4), 1, np.zeros(40000), state)
    assert rc == -1 and "32,768" in msg


def test_noalloc_rejects_a_mask_with_more_phases_than_given():
    """A mask whose phase bits name a phase beyond n_phases is refused with
    LBMBT_ESTATE before the state is touched (lbmbt_run refuses the same
    input); the same mask with enough phases runs."""
    from paper_1907_00908_gb300 import lbmbt
    shape = (4, 4, 8)
    mask = torch.zeros(128, dtype=torch.uint8, device="cuda")
    mask[77] = 2 << 6    # phase 2
    state = torch.full((2 * 7 * 128,), 3.0 + 1.0j, dtype=torch.complex64, device="cuda")
    rc, msg = _raw_call(lbmbt, mask, shape, 2, np.zeros(6), state)
    assert rc == -7 and "phase 2" in msg
    assert bool((state == (3.0 + 1.0j)).all())
    rc, msg = _raw_call(lbmbt, mask, shape, 3, np.zeros(6), state)
    assert rc == 0, msg
