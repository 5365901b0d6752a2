"""The allocation-free entry point, lbmbt_sweep_noalloc.

Callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or their loop must not enter the driver's allocator) run the plain
sweep on buffers they already own; the library keeps its working data in a
fixed file-scope device array.  This file checks, through the C ABI, that two
calls in a row give the same signal as lbmbt_run (within the signal tolerance
of the parity tests), that chained calls continue a run, that a call after the
first one changes no device memory use, and that sizes beyond the stated limit
are refused.  It is collected last so a run stopping at the first failure has
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


def test_noalloc_rejects_sizes_beyond_the_limit():
    from paper_1907_00908_gb300 import lbmbt
    dummy = torch.zeros(64, dtype=torch.uint8, device="cuda")
    state = torch.zeros(64, dtype=torch.complex64, device="cuda")
    gG = [0.01, 0.0, 0.0]
    with pytest.raises(lbmbt.LbmbtError) as e:
        lbmbt.sweep_noalloc(dummy, (257, 256, 256), 0.5, (0, 0, 0), [2.0], [math.inf], math.inf, 0.01,
                            np.zeros(10), gG, state)
    assert e.value.code == -1 and "16,777,216" in str(e.value)
    with pytest.raises(lbmbt.LbmbtError) as e:
        lbmbt.sweep_noalloc(dummy, (4, 4, 4), 0.5, (0, 0, 0), [2.0], [math.inf], math.inf, 0.01,
                            np.zeros(40000), gG, state)
    assert e.value.code == -1 and "32,768" in str(e.value)
