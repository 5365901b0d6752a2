"""The bulk-copy sweep's device-side failure path, exercised without a fault.

Every mbarrier wait of the bulk-copy sweep is bounded; a wait that runs out
sets the step control's error word, the CTA's producer waits (bounded) for
its own copies in flight, and the call returns LBMBT_EDEVICE.  The test-only
option LBMBT_OPT_TEST_WAIT_NS makes each consumer warp first wait, with a
short limit, on a shared-memory barrier that nothing completes, so the wait
runs out as one for a lost copy would.  The grid is tiny (one unit per CTA),
so the producer never waits for a stage to be released.  The next run on the
same context, with the option off, matches the oracle.
"""
import math
import time

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    from paper_1907_00908_gb300 import lbmbt
    lbmbt.lib()
    return lbmbt


@pytest.mark.parametrize("n_steps", [4, 20])   # 20: the steps replay as a captured graph
def test_wait_timeout_reports_edevice_and_the_context_recovers(lb, n_steps):
    rng = np.random.default_rng(9)
    geom = synth.Geometry(rng.integers(0, 2, size=(2, 4, 16)).astype(np.int32), np.array([0, 1], np.uint8), 0.5)
    dt = 0.02
    gG = [0.05, 0.0, 0.03]
    f = np.ones(n_steps)
    D, T2, kap = [2.0, 1.0], [80.0, 50.0], 0.04
    s = lb.Solver(0)
    s.set_option(lb.OPT_KERNEL, 2)
    s.set_geometry(geom.labels, geom.phase_of_label, geom.dx)
    s.set_phases(D, T2)
    s.set_permeability(kap)
    s.set_sequence(dt, f, gG)
    assert s.get_option(lb.OPT_TEST_WAIT_NS) == 0          # off unless a test sets it
    s.set_option(lb.OPT_TEST_WAIT_NS, 1_000_000)           # 1 ms
    t0 = time.perf_counter()
    with pytest.raises(lb.LbmbtError) as e:
        s.run()
    assert e.value.code == -6 and "timed out" in str(e.value)
    assert time.perf_counter() - t0 < 5.0
    s.set_option(lb.OPT_TEST_WAIT_NS, 0)
    fld = torch.zeros(geom.n_sites, dtype=torch.complex64, device="cuda")
    r = s.run(field=fld)
    torch.cuda.synchronize()
    assert s.get_option(lb.OPT_KERNEL_USED) == 2
    s.close()
    o = oracle.run(geom.labels, geom.dx, geom.phase_of_label, (0, 0, 0), D, T2, kap, dt, f, gG, want_field=True)
    assert abs(r["S"] - o["S"]) <= 1e-5 * o["S"]
    err = np.abs(fld.cpu().numpy().reshape(geom.labels.shape) - o["field"]).max() / np.abs(o["field"]).max()
    assert err < 1e-4 and math.isfinite(r["S"])


def test_test_wait_option_bounds(lb):
    s = lb.Solver(0)
    for bad in (-1, 1_000_000_001):
        with pytest.raises(lb.LbmbtError):
            s.set_option(lb.OPT_TEST_WAIT_NS, bad)
    s.close()
