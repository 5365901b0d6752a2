"""ctypes binding of ``liblbmbt.so`` (C ABI in ``include/lbmbt.h``).

Argument marshalling only: every step of the sweep runs in the CUDA library.
Loading fails loudly if the library is missing -- there is no CPU fallback.
The low-level functions keep the C names; ``Solver`` is a thin convenience
wrapper that owns one context and accepts numpy arrays / torch tensors.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbmbt.so")

LBMBT_OK = 0
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSTABLE", -5: "EUNSUPPORTED",
          -6: "EDEVICE", -7: "ESTATE"}
BC_PERIODIC = 0
BC_MIRROR = 1
FACE_OWN, FACE_HALO, FACE_HALO_WRAP = 0, 1, 2
OPT_GRAPH, OPT_AUTOTUNE, OPT_BLOCK, OPT_SPT, OPT_KERNEL, OPT_KERNEL_USED, OPT_STAGES, OPT_TMA_SHAPE = 1, 2, 3, 4, 5, 6, 7, 8
OPT_ADJOINT_KERNEL, OPT_ADJOINT_SHAPE, OPT_LATTICE = 9, 10, 11
OPT_STAGE_OWN_Z, OPT_STAGE_OWN_Z_USED, OPT_SCHEME, OPT_GRAD_GROUPS, OPT_TEST_WAIT_NS = 12, 13, 14, 15, 16
OPT_COLUMN_PLANES = 17

# every entry point declared in include/lbmbt.h
EXPORTS = [
    "lbmbt_create", "lbmbt_destroy", "lbmbt_last_error", "lbmbt_version", "lbmbt_set_geometry",
    "lbmbt_add_geometry", "lbmbt_get_mask", "lbmbt_set_phases", "lbmbt_set_permeability",
    "lbmbt_set_sequence", "lbmbt_pgse", "lbmbt_run", "lbmbt_run_batch", "lbmbt_grad",
    "lbmbt_grad_batch", "lbmbt_set_option", "lbmbt_get_option", "lbmbt_prepare", "lbmbt_advance",
    "lbmbt_launch_count", "lbmbt_sweep_noalloc", "lbmbt_set_geometry_slab", "lbmbt_slab_faces",
    "lbmbt_slab_set_halos", "lbmbt_set_field", "lbmbt_set_link_distances", "lbmbt_set_sequence_substeps",
    "lbmbt_set_link_angles", "lbmbt_run_batch_ex",
]


class LbmbtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Member(ctypes.Structure):
    """``lbmbt_member``: gradient, geometry index, permeability of one batch member."""
    _fields_ = [("gamma_G0", ctypes.c_double * 3), ("geometry", ctypes.c_int), ("kappa_um_ms", ctypes.c_double)]


class MemberEx(ctypes.Structure):
    """``lbmbt_member_ex``: a batch member with its own waveform (f, n_steps)
    and field output (device pointer), each optional (NULL)."""
    _fields_ = [("gamma_G0", ctypes.c_double * 3), ("geometry", ctypes.c_int), ("kappa_um_ms", ctypes.c_double),
                ("f", ctypes.c_void_p), ("n_steps", ctypes.c_int64), ("field_dev", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load ``liblbmbt.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"liblbmbt.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
            sig = {
                "lbmbt_create": [ctypes.POINTER(P), I, P],
                "lbmbt_destroy": [P],
                "lbmbt_set_geometry": [P, I, I, I, D, P, I, I, P, P],
                "lbmbt_add_geometry": [P, I, I, I, D, P, I, I, P, P, ctypes.POINTER(I)],
                "lbmbt_get_mask": [P, I, P],
                "lbmbt_set_phases": [P, I, P, P],
                "lbmbt_set_permeability": [P, D],
                "lbmbt_set_sequence": [P, D, I64, P, P],
                "lbmbt_pgse": [D, D, D, D, P, P, ctypes.POINTER(I64), P],
                "lbmbt_run": [P, P, P, P],
                "lbmbt_run_batch": [P, I, P, P, P],
                "lbmbt_run_batch_ex": [P, I, P, P, P],
                "lbmbt_grad": [P, I, P, P, P, P],
                "lbmbt_grad_batch": [P, I, P, I, P, P, P, P],
                "lbmbt_set_option": [P, I, I64],
                "lbmbt_get_option": [P, I, ctypes.POINTER(I64)],
                "lbmbt_prepare": [P, I, P],
                "lbmbt_advance": [P, I64, I, P],
                "lbmbt_launch_count": [P, ctypes.POINTER(I64)],
                "lbmbt_set_geometry_slab": [P, I, I, I, D, P, I, I, P, P, I, I, I, I],
                "lbmbt_slab_faces": [P, I, P, P],
                "lbmbt_slab_set_halos": [P, I, P, P],
                "lbmbt_set_field": [P, P],
                "lbmbt_set_link_distances": [P, I, P, I],
                "lbmbt_set_link_angles": [P, I, P, I],
                "lbmbt_set_sequence_substeps": [P, D, I64, I, P, P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = I
            L.lbmbt_sweep_noalloc.argtypes = [I, I, I, D, P, P, I, P, P, D, D, I64, P, P, P, I64, I64, I, P, P,
                                              ctypes.c_char_p, ctypes.c_size_t]
            L.lbmbt_sweep_noalloc.restype = I
            L.lbmbt_last_error.argtypes = [P]
            L.lbmbt_last_error.restype = ctypes.c_char_p
            L.lbmbt_version.argtypes = []
            L.lbmbt_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _p(a):
    """Host numpy array, torch tensor (host or device) or raw int -> void*."""
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(type(a))


def _device_tensor(t, dtype, what, numel=None, host_ok=False):
    """Check a buffer that the library reads or writes in place through its
    data pointer alone: a torch CUDA tensor (with ``host_ok`` also a host
    tensor or numpy array, for calls that accept host memory) of the
    expected dtype (``"int32"``, ``"uint8"``, ``"float32"``,
    ``"complex64"``), contiguous, and with at least ``numel`` elements when
    given.  None and raw integer pointers pass unchecked."""
    if t is None or isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        if not host_ok:
            raise TypeError(f"{what}: expected a torch CUDA tensor, got a numpy array")
        if t.dtype != np.dtype(dtype):
            raise TypeError(f"{what}: expected dtype {dtype}, got {t.dtype}")
        if not t.flags.c_contiguous:
            raise ValueError(f"{what}: the array must be C-contiguous")
        if numel is not None and t.size < numel:
            raise ValueError(f"{what}: {t.size} elements, at least {numel} needed")
        return t
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch CUDA tensor, got {type(t).__name__}")
    if not t.is_cuda and not host_ok:
        raise TypeError(f"{what}: expected a CUDA tensor, got one on {t.device}")
    if t.dtype != getattr(torch, dtype):
        raise TypeError(f"{what}: expected dtype torch.{dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: the tensor must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{what}: {t.numel()} elements, at least {numel} needed")
    return t


def pgse(b_s_mm2, delta, Delta, dt, direction=(1.0, 0.0, 0.0)):
    """``lbmbt_pgse``: returns (gamma_G0[3], f[K])."""
    L = lib()
    d = np.ascontiguousarray(direction, np.float64)
    g = np.zeros(3)
    n = ctypes.c_int64(0)
    rc = L.lbmbt_pgse(b_s_mm2, delta, Delta, dt, _p(d), _p(g), ctypes.byref(n), None)
    if rc:
        raise LbmbtError(rc, "lbmbt_pgse: invalid PGSE parameters")
    f = np.empty(n.value)
    L.lbmbt_pgse(b_s_mm2, delta, Delta, dt, _p(d), _p(g), ctypes.byref(n), _p(f))
    return g, f


def sweep_noalloc(mask_dev, shape, dx, bc, D, T2, kappa, dt, f, gG, state_dev, k0=0, n_steps=None, init=True,
                  stream=None):
    """``lbmbt_sweep_noalloc``: plain sweep on caller-owned device buffers
    (mask uint8 [N], state complex64 [2*7*plane]) with no device allocation
    inside the library.  Returns {Z, S} after step k0 + n_steps."""
    L = lib()
    nz, ny, nx = shape
    # the library cannot see the buffers' sizes: check them here against the
    # shape (mask N bytes, state 2 x 7 x plane complex64, plane = N rounded
    # up to 64), before anything is launched, and that both are on the
    # current device
    N = int(nx) * int(ny) * int(nz)
    plane = (N + 63) // 64 * 64
    for t, need, what in ((mask_dev, N, "mask"), (state_dev, 2 * 7 * plane, "state")):
        if hasattr(t, "numel") and t.numel() < need:
            raise ValueError(f"sweep_noalloc {what}: {t.numel()} elements, at least {need} needed for shape "
                             f"{tuple(shape)}")
    _device_tensor(mask_dev, "uint8", "sweep_noalloc mask", numel=N)
    _device_tensor(state_dev, "complex64", "sweep_noalloc state", numel=2 * 7 * plane)
    import torch
    cur = torch.cuda.current_device()
    for t, what in ((mask_dev, "mask"), (state_dev, "state")):
        if t.device.index != cur:
            raise ValueError(f"sweep_noalloc {what}: on {t.device}, but the current device is cuda:{cur}")
    bcv = np.ascontiguousarray(bc, np.int32)
    Dv = np.ascontiguousarray(np.atleast_1d(D), np.float64)
    T2v = np.ascontiguousarray(np.atleast_1d(T2), np.float64)
    fv = np.ascontiguousarray(f, np.float64)
    gv = np.ascontiguousarray(gG, np.float64)
    n = fv.size - k0 if n_steps is None else n_steps
    sig = np.zeros(3)
    err = ctypes.create_string_buffer(256)
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    rc = L.lbmbt_sweep_noalloc(nx, ny, nz, float(dx), _p(mask_dev), _p(bcv), int(Dv.size), _p(Dv), _p(T2v),
                               float(kappa), float(dt), int(fv.size), _p(fv), _p(gv), _p(state_dev), int(k0), int(n),
                               int(bool(init)), _p(sig), s, err, 256)
    if rc:
        raise LbmbtError(rc, "lbmbt_sweep_noalloc: " + err.value.decode())
    return {"Z": complex(sig[0], sig[1]), "S": float(sig[2])}


class Solver:
    """One library context (device + stream) with numpy/torch marshalling."""

    def __init__(self, device: int = 0, stream=None):
        self.L = lib()
        h = ctypes.c_void_p()
        s = None
        if stream is not None:
            s = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        rc = self.L.lbmbt_create(ctypes.byref(h), int(device), s)
        if rc:
            raise LbmbtError(rc, self.L.lbmbt_last_error(None).decode())
        self.h = h
        self.n_sites = []
        self.n_steps = 0
        self.n_phases = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.lbmbt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, rc, what):
        if rc:
            raise LbmbtError(rc, f"{what}: {self.L.lbmbt_last_error(self.h).decode()}")

    # --- set-up -------------------------------------------------------------
    def set_geometry(self, labels, phase_of_label, dx, bc=(0, 0, 0), add=False):
        """labels: int32 [nz, ny, nx] numpy (host) or torch CUDA tensor (device)."""
        on_dev = hasattr(labels, "is_cuda") and labels.is_cuda
        if on_dev:
            _device_tensor(labels, "int32", "labels")
            nz, ny, nx = labels.shape
        else:
            labels = np.ascontiguousarray(labels, np.int32)
            nz, ny, nx = labels.shape
        pol = np.ascontiguousarray(phase_of_label, np.uint8)
        bcv = np.ascontiguousarray(bc, np.int32)
        if add:
            idx = ctypes.c_int(0)
            self._chk(self.L.lbmbt_add_geometry(self.h, nx, ny, nz, float(dx), _p(labels), int(on_dev),
                                                int(pol.size), _p(pol), _p(bcv), ctypes.byref(idx)),
                      "add_geometry")
            self.n_sites.append(nx * ny * nz)
            return idx.value
        self._chk(self.L.lbmbt_set_geometry(self.h, nx, ny, nz, float(dx), _p(labels), int(on_dev),
                                            int(pol.size), _p(pol), _p(bcv)), "set_geometry")
        self.n_sites = [nx * ny * nz]
        self.shape = (nz, ny, nx)
        return 0

    def set_geometry_slab(self, labels_ext, phase_of_label, dx, bc, z0, nz_global, lo_kind, hi_kind):
        """``lbmbt_set_geometry_slab``: labels_ext int32 [nz + 2, ny, nx] (ghost
        plane below, the slab's planes, ghost plane above), numpy or torch CUDA."""
        on_dev = hasattr(labels_ext, "is_cuda") and labels_ext.is_cuda
        if on_dev:
            _device_tensor(labels_ext, "int32", "labels_ext")
        else:
            labels_ext = np.ascontiguousarray(labels_ext, np.int32)
        nz2, ny, nx = labels_ext.shape
        pol = np.ascontiguousarray(phase_of_label, np.uint8)
        bcv = np.ascontiguousarray(bc, np.int32)
        self._chk(self.L.lbmbt_set_geometry_slab(self.h, nx, ny, nz2 - 2, float(dx), _p(labels_ext), int(on_dev),
                                                 int(pol.size), _p(pol), _p(bcv), int(z0), int(nz_global),
                                                 int(lo_kind), int(hi_kind)), "set_geometry_slab")
        self.n_sites = [nx * ny * (nz2 - 2)]
        self.shape = (nz2 - 2, ny, nx)
        return 0

    def slab_faces(self, member, lo_out, hi_out):
        """Copy the faces leaving the slab (complex64 [ny, nx], host or CUDA, or None)."""
        n = self._face_sites()
        _device_tensor(lo_out, "complex64", "slab_faces lo_out", n, host_ok=True)
        _device_tensor(hi_out, "complex64", "slab_faces hi_out", n, host_ok=True)
        self._chk(self.L.lbmbt_slab_faces(self.h, int(member), _p(lo_out), _p(hi_out)), "slab_faces")

    def slab_set_halos(self, member, lo_in, hi_in):
        """Set the halo planes read by the next step (complex64 [ny, nx], host or CUDA, or None)."""
        n = self._face_sites()
        _device_tensor(lo_in, "complex64", "slab_set_halos lo_in", n, host_ok=True)
        _device_tensor(hi_in, "complex64", "slab_set_halos hi_in", n, host_ok=True)
        self._chk(self.L.lbmbt_slab_set_halos(self.h, int(member), _p(lo_in), _p(hi_in)), "slab_set_halos")

    def _face_sites(self):
        shape = getattr(self, "shape", None)
        return None if shape is None else shape[1] * shape[2]

    def add_geometry(self, labels, phase_of_label, dx, bc=(0, 0, 0)):
        return self.set_geometry(labels, phase_of_label, dx, bc, add=True)

    def set_link_distances(self, delta, index=0):
        """Membrane positions on the links (float32 [6, nz, ny, nx], numpy or
        torch CUDA), or None to return to the half-link rule."""
        if delta is None:
            self._chk(self.L.lbmbt_set_link_distances(self.h, int(index), None, 0), "set_link_distances")
            return
        on_dev = hasattr(delta, "is_cuda") and delta.is_cuda
        if on_dev:
            _device_tensor(delta, "float32", "link distances", self._sites(index, 6))
        else:
            delta = np.ascontiguousarray(delta, np.float32)
        self._chk(self.L.lbmbt_set_link_distances(self.h, int(index), _p(delta), int(on_dev)), "set_link_distances")

    def set_link_angles(self, theta, index=0):
        """Membrane angles on the links of a one-plane geometry (float32
        [6, 1, ny, nx], numpy or torch CUDA), or None to remove them."""
        if theta is None:
            self._chk(self.L.lbmbt_set_link_angles(self.h, int(index), None, 0), "set_link_angles")
            return
        on_dev = hasattr(theta, "is_cuda") and theta.is_cuda
        if on_dev:
            _device_tensor(theta, "float32", "link angles", self._sites(index, 6))
        else:
            theta = np.ascontiguousarray(theta, np.float32)
        self._chk(self.L.lbmbt_set_link_angles(self.h, int(index), _p(theta), int(on_dev)), "set_link_angles")

    def _sites(self, index=0, per_site=1):
        """Sites of geometry ``index`` times ``per_site``, None if unknown."""
        return self.n_sites[index] * per_site if 0 <= index < len(self.n_sites) else None

    def get_mask(self, index=0, shape=None):
        n = self.n_sites[index]
        out = np.empty(n, np.uint8)
        self._chk(self.L.lbmbt_get_mask(self.h, index, _p(out)), "get_mask")
        return out.reshape(shape) if shape is not None else out

    def set_phases(self, D, T2):
        Dv = np.ascontiguousarray(np.atleast_1d(D), np.float64)
        T2v = np.ascontiguousarray(np.atleast_1d(T2), np.float64)
        self._chk(self.L.lbmbt_set_phases(self.h, int(Dv.size), _p(Dv), _p(T2v)), "set_phases")
        self.n_phases = int(Dv.size)

    def set_permeability(self, kappa):
        self._chk(self.L.lbmbt_set_permeability(self.h, float(kappa)), "set_permeability")

    def set_sequence(self, dt, f, gG):
        fv = np.ascontiguousarray(f, np.float64)
        gv = np.ascontiguousarray(gG, np.float64)
        self._chk(self.L.lbmbt_set_sequence(self.h, float(dt), int(fv.size), _p(fv), _p(gv)), "set_sequence")
        self.n_steps = int(fv.size)

    def set_sequence_substeps(self, dt, f_fine, gG, substeps):
        """Waveform sampled on the dt/substeps grid (Sec. 2.3, dt = k dt')."""
        fv = np.ascontiguousarray(f_fine, np.float64)
        gv = np.ascontiguousarray(gG, np.float64)
        if fv.size % substeps:
            raise ValueError("len(f_fine) must be a multiple of substeps")
        n = fv.size // substeps
        self._chk(self.L.lbmbt_set_sequence_substeps(self.h, float(dt), int(n), int(substeps), _p(fv), _p(gv)),
                  "set_sequence_substeps")
        self.n_steps = n

    def set_option(self, opt, value):
        self._chk(self.L.lbmbt_set_option(self.h, int(opt), int(value)), "set_option")

    def get_option(self, opt):
        v = ctypes.c_int64(0)
        self._chk(self.L.lbmbt_get_option(self.h, int(opt), ctypes.byref(v)), "get_option")
        return v.value

    # --- runs ---------------------------------------------------------------
    def run(self, field=None, series=False):
        """Plain run.  ``field``: torch complex64 CUDA tensor [N] (or None).
        Returns dict(Z, S[, series])."""
        _device_tensor(field, "complex64", "run field", self._sites(0))
        sig = np.zeros(3)
        ser = np.zeros(2 * self.n_steps) if series else None
        self._chk(self.L.lbmbt_run(self.h, _p(sig), _p(field), _p(ser)), "run")
        out = {"Z": complex(sig[0], sig[1]), "S": float(sig[2])}
        if series:
            out["series"] = ser[0::2] + 1j * ser[1::2]
        return out

    @staticmethod
    def members(gGs, geometry=0, kappa=math.inf):
        gGs = np.atleast_2d(np.asarray(gGs, np.float64))
        n = gGs.shape[0]
        geo = np.broadcast_to(np.asarray(geometry), (n,))
        kap = np.broadcast_to(np.asarray(kappa, np.float64), (n,))
        arr = (Member * n)()
        for i in range(n):
            arr[i].gamma_G0[:] = [float(v) for v in gGs[i]]
            arr[i].geometry = int(geo[i])
            arr[i].kappa_um_ms = float(kap[i])
        return arr

    def run_batch(self, members, series=False, waveforms=None, fields=None):
        """Batched run.  ``waveforms`` (optional, one per member): the
        member's own waveform (1-D array, at most the set sequence's length;
        its signal is taken at its end) or None for the set one.  ``fields``
        (optional, one per member): torch complex64 CUDA tensor [N of the
        member's geometry] receiving M(x) at the member's end, or None.
        Either selects ``lbmbt_run_batch_ex``."""
        n = len(members)
        sig = np.zeros(3 * n)
        ser = np.zeros(2 * n * self.n_steps) if series else None
        if waveforms is None and fields is None:
            self._chk(self.L.lbmbt_run_batch(self.h, n, members, _p(sig), _p(ser)), "run_batch")
        else:
            waveforms = [None] * n if waveforms is None else list(waveforms)
            fields = [None] * n if fields is None else list(fields)
            if len(waveforms) != n or len(fields) != n:
                raise ValueError("one waveform and one field entry per member")
            ex = (MemberEx * n)()
            keep = []
            for i in range(n):
                m = members[i]
                ex[i].gamma_G0[:] = list(m.gamma_G0)
                ex[i].geometry = m.geometry
                ex[i].kappa_um_ms = m.kappa_um_ms
                if waveforms[i] is not None:
                    w = np.ascontiguousarray(waveforms[i], np.float64)
                    if w.ndim != 1 or w.size < 1:
                        raise ValueError(f"member {i}: waveform must be a non-empty 1-D array")
                    keep.append(w)
                    ex[i].f = w.ctypes.data
                    ex[i].n_steps = w.size
                fl = _device_tensor(fields[i], "complex64", f"member {i} field", self._sites(m.geometry))
                ex[i].field_dev = None if fl is None else (fl if isinstance(fl, int) else fl.data_ptr())
            self._chk(self.L.lbmbt_run_batch_ex(self.h, n, ex, _p(sig), _p(ser)), "run_batch_ex")
            del keep
        sig = sig.reshape(n, 3)
        out = {"Z": sig[:, 0] + 1j * sig[:, 1], "S": sig[:, 2].copy()}
        if series:
            s = ser.reshape(n, self.n_steps, 2)
            out["series"] = s[..., 0] + 1j * s[..., 1]
        return out

    def grad(self, checkpoint_every=64):
        sig = np.zeros(3)
        dD = np.zeros(self.n_phases)
        dT2 = np.zeros(self.n_phases)
        dk = np.zeros(1)
        self._chk(self.L.lbmbt_grad(self.h, int(checkpoint_every), _p(sig), _p(dD), _p(dT2), _p(dk)), "grad")
        return {"Z": complex(sig[0], sig[1]), "S": float(sig[2]), "dD": dD, "dT2": dT2, "dkappa": float(dk[0])}

    def grad_batch(self, members, checkpoint_every=64):
        n = len(members)
        sig = np.zeros(3 * n)
        dD = np.zeros(n * self.n_phases)
        dT2 = np.zeros(n * self.n_phases)
        dk = np.zeros(n)
        self._chk(self.L.lbmbt_grad_batch(self.h, n, members, int(checkpoint_every), _p(sig), _p(dD), _p(dT2),
                                          _p(dk)), "grad_batch")
        sig = sig.reshape(n, 3)
        return {"Z": sig[:, 0] + 1j * sig[:, 1], "S": sig[:, 2].copy(),
                "dD": dD.reshape(n, -1), "dT2": dT2.reshape(n, -1), "dkappa": dk}

    # --- timing hooks -------------------------------------------------------
    def set_field(self, field):
        """Field buffer (torch complex64 CUDA [N] or None) for the next prepare()."""
        _device_tensor(field, "complex64", "set_field", self._sites(0))
        self._field_keep = field
        self._chk(self.L.lbmbt_set_field(self.h, _p(field)), "set_field")

    def prepare(self, members=None):
        if members is None:
            self._chk(self.L.lbmbt_prepare(self.h, 0, None), "prepare")
        else:
            self._chk(self.L.lbmbt_prepare(self.h, len(members), members), "prepare")

    def advance(self, n_steps, want_signal=False, n_members=1):
        sig = np.zeros(3 * n_members) if want_signal else None
        self._chk(self.L.lbmbt_advance(self.h, int(n_steps), int(bool(want_signal)), _p(sig)), "advance")
        return sig.reshape(n_members, 3) if want_signal else None

    def launch_count(self):
        v = ctypes.c_int64(0)
        self._chk(self.L.lbmbt_launch_count(self.h, ctypes.byref(v)), "launch_count")
        return v.value
