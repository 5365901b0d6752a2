"""GPU: the binding refuses device tensors that the library would read or
write with the wrong layout -- wrong dtype, not contiguous, too small, on the
host -- with a Python error before any library call, and accepts the right
ones."""
import math

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


def test_field_and_input_tensors_are_checked(lb):
    g = synth.spheres(30, 0.5, seed=8)
    n = g.n_sites
    gG, f = oracle.pgse(1000.0, 0.1, 0.2, 0.02, (1.0, 0.0, 0.0))
    with lb.Solver(0) as s:
        with pytest.raises(TypeError):
            s.set_geometry(torch.from_numpy(g.labels.astype(np.int64)).cuda(), g.phase_of_label, g.dx)
        s.set_geometry(torch.from_numpy(g.labels).cuda(), g.phase_of_label, g.dx)
        s.set_phases([2.0, 1.0], [80.0, 50.0])
        s.set_permeability(0.02)
        s.set_sequence(0.02, f, gG)
        with pytest.raises(TypeError):
            s.set_link_distances(torch.full((6, n), 0.5, dtype=torch.float64, device="cuda"))
        with pytest.raises(ValueError):
            s.set_link_distances(torch.full((6, n - 1), 0.5, dtype=torch.float32, device="cuda"))
        bad = {
            TypeError: [torch.zeros(n, dtype=torch.complex64), torch.zeros(n, dtype=torch.complex128, device="cuda")],
            ValueError: [torch.zeros(2 * n, dtype=torch.complex64, device="cuda")[::2],
                         torch.zeros(n - 1, dtype=torch.complex64, device="cuda")],
        }
        for err, tensors in bad.items():
            for t in tensors:
                with pytest.raises(err):
                    s.run(field=t)
                with pytest.raises(err):
                    s.set_field(t)
        fld = torch.zeros(n, dtype=torch.complex64, device="cuda")
        r = s.run(field=fld)
        torch.cuda.synchronize()
    o = oracle.run(g.labels, g.dx, g.phase_of_label, (0, 0, 0), [2.0, 1.0], [80.0, 50.0], 0.02, 0.02, f, gG)
    assert abs(r["S"] - o["S"]) <= 1e-5 * o["S"]
    assert float(fld.abs().max()) > 0.0 and not math.isnan(float(fld.abs().sum()))
