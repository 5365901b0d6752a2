"""FP64 CPU oracle of the hybrid lattice Boltzmann Bloch-Torrey scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_1907_00908_gb300/`` and never imports
it.  The scheme itself lives in ``lbm_oracle.c`` (plain C, FP64), compiled on
first use with the system C compiler; this module adds the PGSE waveform
(Sec. 2.1, Fig. 2) and the b-value relation, plus ctypes marshalling.

Every function follows a passage of Naughton, Tennyson & Georgiadis,
arXiv 1907.00908:

* ``pgse``      -- Sec. 2.1 (b = gamma^2 |G0|^2 delta^2 (Delta - delta/3)),
                   effective gradient f(t) of Fig. 2 sampled at t^k = k dt.
* ``run``       -- Eq. LBM_process_list_2 with Eqs. collision_LBM,
                   streaming_LBM, reaction_LBM, permeability_BC/B5,
                   collision_BC (modified periodic) and Sec. 2.4.4 (mirror).
* ``mask``      -- half-link membrane links on label changes (Sec. 2.4.2).
* ``run(..., scheme="classical")`` -- the paper's comparison scheme, the
                   classical LBM with the reaction as a collision source
                   (Appendix A, Eqs. A2 and A12).
* ``link_coefficients`` / ``angled_coefficients`` -- the membrane rule with
                   positions (Eqs. B4a-B4c) and its general-angle form
                   (Appendix B, Eqs. B2a, phi_1, phi_2, B1, B1.5).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC = 0
BC_MIRROR = 1
EPS_D = 0.25  # D3Q7: omega_0 = eps_D, omega_i = eps_D/2 (Sec. 2.3 pattern)


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``liblbm_oracle.so`` (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.lbm_oracle_run.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                P, ctypes.c_int, P, P, ctypes.c_int, P, P,
                ctypes.c_double, ctypes.c_double, ctypes.c_long, P, P, ctypes.c_int,
                P, P, P, P]
            lib.lbm_oracle_run.restype = ctypes.c_int
            lib.lbm_oracle_run_links.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                P, ctypes.c_int, P, P, ctypes.c_int, P, P,
                ctypes.c_double, ctypes.c_double, ctypes.c_long, P, P, ctypes.c_int, P,
                P, P, P, P]
            lib.lbm_oracle_run_links.restype = ctypes.c_int
            lib.lbm_oracle_run_ex.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                P, ctypes.c_int, P, P, ctypes.c_int, P, P,
                ctypes.c_double, ctypes.c_double, ctypes.c_long, P, P, ctypes.c_int, P, P, ctypes.c_int,
                ctypes.c_int, P, P, P, P]
            lib.lbm_oracle_run_ex.restype = ctypes.c_int
            lib.lbm_oracle_run_scheme.argtypes = lib.lbm_oracle_run_ex.argtypes[:21] + [ctypes.c_int] + [P] * 4
            lib.lbm_oracle_run_scheme.restype = ctypes.c_int
            lib.lbm_oracle_angled_coefficients.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, P, P, P, P]
            lib.lbm_oracle_angled_coefficients.restype = None
            lib.lbm_oracle_link_coefficients.argtypes = [ctypes.c_double] * 4 + [P, P]
            lib.lbm_oracle_link_coefficients.restype = None
            lib.lbm_oracle_mask.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P]
            lib.lbm_oracle_mask.restype = ctypes.c_int
            lib.lbm_oracle_params.argtypes = [ctypes.c_double] * 4 + [P]
            lib.lbm_oracle_params.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def pgse(b_s_mm2: float, delta: float, Delta: float, dt: float, direction=(1.0, 0.0, 0.0)):
    """PGSE sequence (Sec. 2.1, Fig. 2) on the time grid t^k = k dt.

    Returns ``(gG, f)``: gG = gamma*G0 (rad/(um ms), 3-vector along the unit
    ``direction``) from b = gamma^2 |G0|^2 delta^2 (Delta - delta/3) with b in
    ms/um^2 (= 1e-3 * s/mm^2); f[k] is the effective waveform (the 180-degree
    pulse folded in) sampled at the left end of step k: +1 on [0, delta),
    -1 on [Delta, Delta + delta), 0 elsewhere.  The run lasts to the echo,
    TE = Delta + delta, i.e. K = (Delta + delta)/dt steps; delta/dt and
    Delta/dt must be integers.
    """
    nd = delta / dt
    nD = Delta / dt
    if abs(nd - round(nd)) > 1e-9 * max(1.0, nd) or abs(nD - round(nD)) > 1e-9 * max(1.0, nD):
        raise ValueError("delta/dt and Delta/dt must be integers")
    nd, nD = int(round(nd)), int(round(nD))
    if nd < 1 or nD < nd:
        raise ValueError("need 0 < delta <= Delta")
    K = nD + nd
    f = np.zeros(K, dtype=np.float64)
    f[:nd] = 1.0
    f[nD:nD + nd] = -1.0
    d = np.asarray(direction, dtype=np.float64)
    nrm = math.sqrt(float(d @ d))
    if nrm == 0.0:
        raise ValueError("zero gradient direction")
    b = b_s_mm2 * 1e-3
    gmag = math.sqrt(b / (delta * delta * (Delta - delta / 3.0))) if b > 0 else 0.0
    return gmag * d / nrm, f


def params(D, dt, dx, kappa):
    """(tau, r, s): Eq. tau_def and the Eq. B5 shares r = P/(1+P), s = 1/(1+P)."""
    out = np.zeros(3)
    _load().lbm_oracle_params(float(D), float(dt), float(dx), float(kappa), _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def link_coefficients(delta_m, kappa, dt, dx):
    """(A[3], B[3]) of the theta = 0 membrane rule, Eqs. B4a-B4c."""
    A, B = np.zeros(3), np.zeros(3)
    _load().lbm_oracle_link_coefficients(float(delta_m), float(kappa), float(dt), float(dx), _ptr(A), _ptr(B))
    return A, B


def angled_coefficients(delta_m, theta, kappa, dt, dx, lattice="D2Q5"):
    """(A[3], B[3], C[3], D[3]) of the general-angle membrane rule (Appendix
    B, Eq. B2a), obtained by linearity from the oracle's solve of Eqs.
    dirichlet_1-neumann_2, phi_1, phi_2, B1 and B1.5."""
    A, B, C, D = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3)
    _load().lbm_oracle_angled_coefficients(float(delta_m), float(theta), float(kappa), float(dt), float(dx),
                                           int(lattice == "D2Q5"), _ptr(A), _ptr(B), _ptr(C), _ptr(D))
    return A, B, C, D


def mask(labels, phase_of_label, bc):
    """Bit-packed membrane/phase byte per site (see ``lbm_oracle_mask``)."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    nz, ny, nx = labels.shape
    pol = np.ascontiguousarray(phase_of_label, dtype=np.uint8)
    bcv = np.ascontiguousarray(bc, dtype=np.int32)
    out = np.empty(labels.shape, dtype=np.uint8)
    rc = _load().lbm_oracle_mask(nx, ny, nz, _ptr(labels), int(pol.size), _ptr(pol), _ptr(bcv), _ptr(out))
    if rc != 0:
        raise ValueError("oracle mask: invalid input")
    return out


def run(labels, dx, phase_of_label, bc, D, T2, kappa, dt, f, gG,
        want_field=False, want_series=False, want_state=False, threads=0, delta=None, substeps=1,
        lattice="D3Q7", theta=None, scheme="hybrid"):
    """Run the scheme from M = 1 to t = len(f)*dt.

    ``labels``: int32 [nz, ny, nx] compartment ids; ``phase_of_label``: phase
    id per label; ``bc``: per-axis (x, y, z) 0 = modified periodic, 1 = mirror.
    Returns a dict with ``Z`` (complex sum of M over sites at the end),
    ``S`` = |Z|/N, and optionally ``field`` (complex [nz, ny, nx]),
    ``series`` (complex [K], Z after each step) and ``state`` (complex
    [nz, ny, nx, 7]).  ``delta``: optional [6, nz, ny, nx] membrane positions
    on the links (distance in dx from the node along +x, -x, +y, -y, +z, -z),
    which selects the theta = 0 rule of Eqs. B4a-B4c.  ``substeps`` = k > 1:
    k reaction steps of dt/k after each diffusion step (Sec. 2.3, dt = k dt'),
    ``f`` then sampled on the dt/k grid (len(f) = k * number of steps).
    ``lattice`` = "D2Q5": the 2-D lattice of Sec. 2.3 (eps_D = 1/3, nz = 1).
    ``theta`` (D2Q5, with ``delta``): [6, 1, ny, nx] signed angles between the
    membrane normal and each link (see ``angled_arrival`` in the C source),
    which selects the general-angle rule of Appendix B.
    ``scheme`` = "classical": the classical LBM of Appendix A (Eq. A12), the
    reaction as the collision source dt omega_i R M with R = -i gamma x.G0
    f(t^k) - 1/T2 and no reaction step (``substeps`` must be 1); the outer
    faces then take F_(k+1), the phase the source has already given the
    streamed populations.
    """
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    nz, ny, nx = labels.shape
    N = labels.size
    pol = np.ascontiguousarray(phase_of_label, dtype=np.uint8)
    bcv = np.ascontiguousarray(bc, dtype=np.int32)
    Dv = np.ascontiguousarray(np.atleast_1d(D), dtype=np.float64)
    T2v = np.ascontiguousarray(np.atleast_1d(T2), dtype=np.float64)
    fv = np.ascontiguousarray(f, dtype=np.float64)
    gv = np.ascontiguousarray(gG, dtype=np.float64)
    if fv.size % substeps:
        raise ValueError("len(f) must be a multiple of substeps")
    K = fv.size // substeps
    Z = np.zeros(2)
    field = np.empty(2 * N) if want_field else None
    series = np.empty(2 * K) if want_series else None
    state = np.empty(2 * 7 * N) if want_state else None
    if lattice not in ("D3Q7", "D2Q5"):
        raise ValueError("lattice must be D3Q7 or D2Q5")
    if theta is not None and (delta is None or lattice != "D2Q5"):
        raise ValueError("membrane angles need positions and the D2Q5 lattice")
    if scheme not in ("hybrid", "classical"):
        raise ValueError("scheme must be hybrid or classical")
    if scheme == "classical":
        if substeps != 1:
            raise ValueError("the classical scheme has no reaction step to sub-step")
        dl = None if delta is None else np.ascontiguousarray(np.asarray(delta, dtype=np.float64).reshape(6, N).T)
        th = None if theta is None else np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(6, N).T)
        rc = _load().lbm_oracle_run_scheme(
            nx, ny, nz, float(dx), _ptr(labels), int(pol.size), _ptr(pol), _ptr(bcv),
            int(Dv.size), _ptr(Dv), _ptr(T2v), float(kappa), float(dt), K, _ptr(fv), _ptr(gv),
            int(threads), _ptr(dl), _ptr(th), 1, int(lattice == "D2Q5"), 1, _ptr(Z), _ptr(field),
            _ptr(series), _ptr(state))
    elif substeps != 1 or lattice == "D2Q5":
        dl = None if delta is None else np.ascontiguousarray(np.asarray(delta, dtype=np.float64).reshape(6, N).T)
        th = None if theta is None else np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(6, N).T)
        rc = _load().lbm_oracle_run_ex(
            nx, ny, nz, float(dx), _ptr(labels), int(pol.size), _ptr(pol), _ptr(bcv),
            int(Dv.size), _ptr(Dv), _ptr(T2v), float(kappa), float(dt), K, _ptr(fv), _ptr(gv),
            int(threads), _ptr(dl), _ptr(th), int(substeps), int(lattice == "D2Q5"), _ptr(Z), _ptr(field),
            _ptr(series), _ptr(state))
    elif delta is None:
        rc = _load().lbm_oracle_run(
            nx, ny, nz, float(dx), _ptr(labels), int(pol.size), _ptr(pol), _ptr(bcv),
            int(Dv.size), _ptr(Dv), _ptr(T2v), float(kappa), float(dt), K, _ptr(fv), _ptr(gv),
            int(threads), _ptr(Z), _ptr(field), _ptr(series), _ptr(state))
    else:
        dl = np.ascontiguousarray(np.asarray(delta, dtype=np.float64).reshape(6, N).T)
        rc = _load().lbm_oracle_run_links(
            nx, ny, nz, float(dx), _ptr(labels), int(pol.size), _ptr(pol), _ptr(bcv),
            int(Dv.size), _ptr(Dv), _ptr(T2v), float(kappa), float(dt), K, _ptr(fv), _ptr(gv),
            int(threads), _ptr(dl), _ptr(Z), _ptr(field), _ptr(series), _ptr(state))
    if rc != 0:
        raise ValueError("oracle run: invalid input")
    out = {"Z": complex(Z[0], Z[1])}
    out["S"] = abs(out["Z"]) / N
    if field is not None:
        out["field"] = (field[0::2] + 1j * field[1::2]).reshape(nz, ny, nx)
    if series is not None:
        out["series"] = series[0::2] + 1j * series[1::2]
    if state is not None:
        out["state"] = (state[0::2] + 1j * state[1::2]).reshape(nz, ny, nx, 7)
    return out
