"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/lbmbt.h, and its host-only helpers agree with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1907_00908_gb300 import lbmbt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbmbt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmbt_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = lbmbt.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lbmbt.EXPORTS)


def test_binding_constants_match_the_header():
    """Every status code, face kind, boundary kind and option number of the
    header has the same value in the Python binding, and the binding names
    no option the header lacks."""
    txt = open(os.path.join(ROOT, "include", "lbmbt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\bLBMBT_([A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    assert len(consts) >= 25
    for name, v in consts.items():
        if name == "OK":
            assert lbmbt.LBMBT_OK == v
        elif name.startswith("E"):
            assert lbmbt.STATUS[v] == name, name
        else:
            assert getattr(lbmbt, name) == v, name
    opts = {n for n in dir(lbmbt) if n.startswith("OPT_")}
    assert opts == {n for n in consts if n.startswith("OPT_")}


def test_version_string():
    assert b"sm_103a" in lbmbt.lib().lbmbt_version()


@pytest.mark.parametrize("b,delta,Delta,dt,d", [
    (1000.0, 5.0, 20.0, 0.0125, (1, 0, 0)),
    (3000.0, 10.0, 30.0, 0.00625, (0.3, -0.5, 0.8)),
    (0.0, 2.0, 6.0, 0.05, (0, 0, 1)),
])
def test_pgse_matches_oracle(b, delta, Delta, dt, d):
    g1, f1 = lbmbt.pgse(b, delta, Delta, dt, d)
    g2, f2 = oracle.pgse(b, delta, Delta, dt, d)
    assert np.array_equal(f1, f2)
    np.testing.assert_allclose(g1, g2, rtol=1e-15, atol=0)


def test_pgse_rejects_non_integer_timing():
    with pytest.raises(lbmbt.LbmbtError):
        lbmbt.pgse(1000.0, 5.003, 20.0, 0.0125)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(lbmbt.LbmbtError) as e:
        lbmbt.Solver(0)
    assert e.value.code in (-1, -3)


def test_null_arguments_rejected():
    L = lbmbt.lib()
    assert L.lbmbt_create(None, 0, None) == -1
    assert L.lbmbt_destroy(None) == 0
    assert L.lbmbt_run(None, None, None, None) == -1


def test_device_tensor_check_rejects_host_data():
    """Tensors the library reads or writes in place must be CUDA tensors: a
    host tensor or a numpy array is refused before any library call, and
    None or a raw device pointer passes through."""
    torch = pytest.importorskip("torch")
    for bad in (torch.zeros(4, dtype=torch.complex64), np.zeros(4, np.complex64), [0.0] * 4):
        with pytest.raises(TypeError):
            lbmbt._device_tensor(bad, "complex64", "field")
    assert lbmbt._device_tensor(None, "complex64", "field") is None
    assert lbmbt._device_tensor(12345, "complex64", "field") == 12345


class _FakeLib:
    """Stands in for the library: every entry point succeeds and records its call."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append(name)
            return 0
        return fn


def _fake_solver(shape):
    s = object.__new__(lbmbt.Solver)
    s.L, s.h, s.shape = _FakeLib(), 1, shape
    s.n_sites, s.n_steps, s.n_phases = [int(np.prod(shape))], 0, 0
    return s


def test_buffer_checks_follow_each_call_contract():
    """Slab faces and halos accept host or device buffers (the C calls take
    either); a field output must be a CUDA tensor. Wrong dtype, layout or
    size is refused before the library is called."""
    torch = pytest.importorskip("torch")
    s = _fake_solver((4, 3, 5))
    s.slab_faces(0, torch.zeros(15, dtype=torch.complex64), np.zeros((3, 5), np.complex64))
    s.slab_set_halos(0, None, torch.zeros((3, 5), dtype=torch.complex64))
    assert s.L.calls == ["lbmbt_slab_faces", "lbmbt_slab_set_halos"]
    for bad, err in ((torch.zeros(15, dtype=torch.float32), TypeError), (np.zeros(15, np.complex128), TypeError),
                     (torch.zeros(14, dtype=torch.complex64), ValueError),
                     (np.zeros((5, 3), np.complex64).T, ValueError)):
        with pytest.raises(err):
            s.slab_faces(0, bad, None)
        with pytest.raises(err):
            s.slab_set_halos(0, bad, None)
    with pytest.raises(TypeError):
        s.run(field=torch.zeros(60, dtype=torch.complex64))
    with pytest.raises(TypeError):
        s.set_field(np.zeros(60, np.complex64))
    assert s.L.calls == ["lbmbt_slab_faces", "lbmbt_slab_set_halos"]
    s.h = None   # nothing to destroy


def test_noalloc_buffers_are_checked_before_any_launch(monkeypatch):
    """lbmbt_sweep_noalloc cannot see the sizes of the caller's buffers, so
    the binding checks them against the shape first: an undersized state
    (2 x 7 x plane complex64, plane = N rounded up to 64) or mask (N bytes)
    raises before the library is called; right-sized host tensors are then
    refused as not being on the GPU, again before any call."""
    torch = pytest.importorskip("torch")
    fake = _FakeLib()
    monkeypatch.setattr(lbmbt, "lib", lambda: fake)
    shape = (3, 4, 5)   # N = 60, plane = 64
    args = ((3, 4, 5), 0.5, (0, 0, 0), [2.0], [math.inf], math.inf, 0.01, np.zeros(4), [0.0, 0.0, 0.0])
    ok_mask, ok_state = torch.zeros(60, dtype=torch.uint8), torch.zeros(2 * 7 * 64, dtype=torch.complex64)
    for mask, state in ((ok_mask, torch.zeros(2 * 7 * 64 - 1, dtype=torch.complex64)),
                        (ok_mask, torch.zeros(2 * 7 * 60, dtype=torch.complex64)),
                        (torch.zeros(59, dtype=torch.uint8), ok_state)):
        with pytest.raises(ValueError):
            lbmbt.sweep_noalloc(mask, args[0], *args[1:-1], args[-1], state)
    with pytest.raises(TypeError):
        lbmbt.sweep_noalloc(ok_mask, shape, *args[1:-1], args[-1], ok_state)
    assert fake.calls == []


def test_member_struct_layout_matches_the_c_compiler(tmp_path):
    """The binding's lbmbt_member has the size and field offsets that the C
    compiler gives the header's struct."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbmbt.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(lbmbt_member), '
                   'offsetof(lbmbt_member, gamma_G0), offsetof(lbmbt_member, geometry), '
                   'offsetof(lbmbt_member, kappa_um_ms)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    size, o_g, o_geo, o_k = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                     text=True).stdout.split())
    M = lbmbt.Member
    assert ctypes.sizeof(M) == size
    assert (M.gamma_G0.offset, M.geometry.offset, M.kappa_um_ms.offset) == (o_g, o_geo, o_k)


def test_binding_signatures_match_the_header_prototypes():
    """Every entry point's ctypes signature has as many arguments as its
    prototype in the header (a miscount would shift every later argument)."""
    txt = open(os.path.join(ROOT, "include", "lbmbt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = dict(re.findall(r"\b(lbmbt_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt))
    L = lbmbt.lib()
    assert set(protos) == set(lbmbt.EXPORTS)
    for name, params in protos.items():
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        argtypes = getattr(L, name).argtypes
        assert argtypes is not None and len(argtypes) == n, (name, n, argtypes)


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++11")])
def test_header_compiles_cleanly_as_c_and_cxx(tmp_path, lang, std):
    """include/lbmbt.h is a plain C ABI: it compiles on its own, warning-free
    under -Wall -Wextra -Wpedantic, as C99 and as C++11."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no compiler")
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "lbmbt.h"\nint main(void) { return 0; }\n')
    subprocess.run([cc, std, "-Wall", "-Wextra", "-Wpedantic", "-Werror", "-fsyntax-only",
                    "-I", os.path.join(ROOT, "include"), str(src)], check=True)


def test_member_ex_struct_layout_matches_the_c_compiler(tmp_path):
    """The binding's lbmbt_member_ex (per-member waveform and field) has the
    size and field offsets that the C compiler gives the header's struct."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = ["gamma_G0", "geometry", "kappa_um_ms", "f", "n_steps", "field_dev"]
    src = tmp_path / "layout_ex.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbmbt.h"\n'
                   'int main(void) { printf("%zu' + ' %zu' * len(names) + '\\n", sizeof(lbmbt_member_ex)' +
                   "".join(f", offsetof(lbmbt_member_ex, {n})" for n in names) + "); return 0; }\n")
    exe = tmp_path / "layout_ex"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()))
    M = lbmbt.MemberEx
    assert ctypes.sizeof(M) == vals[0]
    assert [getattr(M, n).offset for n in names] == vals[1:]
