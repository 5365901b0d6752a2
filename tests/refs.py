"""Independent references that pin the FP64 oracle (test helpers only).

None of these shares code with ``oracle/`` or with the CUDA library; each is
a different route to a number the oracle must reproduce:

* ``planewave_signal`` -- exact closed form of the lattice scheme itself for a
  uniform periodic medium: a plane wave g_i = a_i exp(-i k.x) stays a plane
  wave, so one 7-vector recurrence replaces the whole lattice.
* ``brute_state`` -- the one-step operator assembled link by link as a pair of
  complex matrices (out = A g + B conj(g)), applied K times; a second,
  matrix-form implementation of the same equations for tiny grids.
* ``slab_signal`` -- continuum PGSE signal between impermeable parallel planes
  by the Neumann cosine-mode ("matrix formalism") propagator, exact for a
  piecewise-constant gradient up to mode truncation.
* ``exchange_signal`` -- continuum two-compartment 1-D problem with a
  permeable membrane (flux D dM/dn = kappa (M_2 - M_1)), fine finite-volume
  grid, matrix exponential in time.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

# D3Q7 velocity set and the weights eps_D = 1/4, w0 = 1/4, w_i = 1/8
E = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
WTS = np.array([0.25] + [0.125] * 6)
EPS = 0.25


# D2Q5 (Sec. 2.3): eps_D = 1/3, w0 = 1/3, w_i = 1/6
E2 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]])
WTS2 = np.array([1 / 3] + [1 / 6] * 4)
EPS2 = 1 / 3


def tau(D, dt, dx, eps=EPS):
    return 0.5 + dt * D / (eps * dx * dx)


# ---------------------------------------------------------------- plane wave
def planewave_signal(n, dx, D, T2, dt, f, gG, series=False, lattice="D3Q7"):
    """S(t^K) (and optionally Z(t^k)/N for all k) of a uniform periodic n^3 box.

    State g_i(x) = a_i exp(-i kv.x).  Collision acts on a; streaming from
    x - e_i dx multiplies a_i by exp(+i kv.e_i dx); the reaction adds
    gG f_k dt to kv and damps by exp(-dt/T2).  ``lattice`` = "D2Q5": the
    five-velocity 2-D set (the box then has one z plane).
    """
    nxyz = np.array([n, n, n]) if np.isscalar(n) else np.array(n)
    Ev, Wv, eps = (E, WTS, EPS) if lattice == "D3Q7" else (E2, WTS2, EPS2)
    om = 1.0 / tau(D, dt, dx, eps)
    dec = math.exp(-dt / T2)
    a = Wv.astype(np.complex128).copy()
    kv = np.zeros(3)
    gG = np.asarray(gG, float)
    out = []
    for fk in f:
        M = a.sum()
        a = a - om * (a - Wv * M)
        a = a * np.exp(1j * (Ev @ kv) * dx)
        kv = kv + gG * fk * dt
        a = a * dec
        if series:
            geo = 1.0 + 0j
            for ax in range(3):
                m = np.arange(nxyz[ax])
                geo *= np.exp(-1j * kv[ax] * m * dx).sum() / nxyz[ax]
            out.append(a.sum() * geo)
    geo = 1.0 + 0j
    for ax in range(3):
        m = np.arange(nxyz[ax])
        geo *= np.exp(-1j * kv[ax] * m * dx).sum() / nxyz[ax]
    S = abs(a.sum() * geo)
    return (S, np.array(out)) if series else S


# --------------------------------------------------------------- brute force
def _site(x, y, z, nx, ny):
    return (z * ny + y) * nx + x


def brute_state(labels, dx, phase_of_label, bc, D, T2, kappa, dt, f, gG, lattice="D3Q7", scheme="hybrid"):
    """Final state g_i(x) [nz, ny, nx, Q] from operator matrices (tiny grids).

    Each step: collision block per site; a link map that routes every arriving
    population from its source (neighbour, periodic image with its phase
    factor, or the mirror image) and mixes in the membrane shares; a diagonal
    reaction.  Real-linear maps are kept as (A, B): v -> A v + B conj(v).
    lattice "D3Q7" (Q = 7) or "D2Q5" (Q = 5, one z plane, eps_D = 1/3).
    scheme "classical" (Appendix A, Eq. A12): the collision block gains the
    source column dt R(x, t^k) w (a rank-one block, w times the row of ones,
    scaled by R = -i x.gG f_k - 1/T2), the reaction is the identity, and the
    face phases use the waveform integral after step k, F + f_k dt.
    """
    labels = np.asarray(labels)
    nz, ny, nx = labels.shape
    dims = (nx, ny, nz)
    N = labels.size
    if lattice == "D2Q5":
        assert nz == 1
        Q, vel, wts, eps = 5, E2, WTS2, EPS2
    else:
        Q, vel, wts, eps = 7, E, WTS, EPS
    opp = [0, 2, 1, 4, 3, 6, 5][:Q]
    ph = np.asarray(phase_of_label)[labels].ravel()
    Dv = np.atleast_1d(D)
    T2v = np.atleast_1d(T2)
    if kappa == 0:
        r, s = 1.0, 0.0
    elif math.isinf(kappa):
        r, s = 0.0, 1.0
    else:
        P = eps * dx / (2 * kappa * dt)
        r, s = P / (1 + P), 1 / (1 + P)
    gG = np.asarray(gG, float)
    conj_axis = [bc[a] == 1 and gG[a] != 0 for a in range(3)]

    # collision matrix (real coefficients)
    C = np.zeros((N * Q, N * Q))
    for x in range(N):
        om = 1.0 / tau(Dv[ph[x]], dt, dx, eps)
        blk = (1 - om) * np.eye(Q) + om * np.outer(wts, np.ones(Q))
        C[x * Q:(x + 1) * Q, x * Q:(x + 1) * Q] = blk

    lab = labels.ravel()
    g = np.tile(wts.astype(complex), N)
    F = 0.0
    classical = scheme == "classical"
    assert scheme in ("hybrid", "classical")
    for fk in f:
        if classical:
            Cs = C.astype(complex)
            for z in range(nz):
                for y in range(ny):
                    for x in range(nx):
                        t = _site(x, y, z, nx, ny)
                        Rt = -1j * (x * gG[0] + y * gG[1] + z * gG[2]) * dx * fk - 1.0 / T2v[ph[t]]
                        Cs[t * Q:(t + 1) * Q, t * Q:(t + 1) * Q] += dt * Rt * np.outer(wts, np.ones(Q))
            Fl = F + fk * dt   # faces: the source of this step is in the streamed values
        else:
            Cs, Fl = C, F
        A = np.zeros((N * Q, N * Q), complex)
        B = np.zeros((N * Q, N * Q), complex)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    t = _site(x, y, z, nx, ny)
                    A[t * Q, t * Q] = 1.0
                    for i in range(1, Q):
                        src = [x - vel[i][0], y - vel[i][1], z - vel[i][2]]
                        fac, mirror, mconj = 1.0 + 0j, False, 0j
                        for a in range(3):
                            if src[a] < 0 or src[a] >= dims[a]:
                                low = src[a] < 0
                                if bc[a] == 0:
                                    src[a] %= dims[a]
                                    fac = np.exp((1j if low else -1j) * gG[a] * dims[a] * dx * Fl)
                                else:
                                    mirror = True
                                    if conj_axis[a]:
                                        xn = 0 if low else dims[a] - 1
                                        xm = -1 if low else dims[a]
                                        mconj = np.exp(-1j * gG[a] * (xn + xm) * dx * Fl)
                        row = t * Q + i
                        if mirror:
                            col = t * Q + opp[i]
                            if any(conj_axis[a] and (src[a] < 0 or src[a] >= dims[a]) for a in range(3)):
                                B[row, col] += mconj
                            else:
                                A[row, col] += 1.0
                            continue
                        u = _site(src[0], src[1], src[2], nx, ny)
                        if lab[u] != lab[t]:
                            A[row, u * Q + i] += s * fac
                            A[row, t * Q + opp[i]] += r
                        else:
                            A[row, u * Q + i] += fac
        # reaction
        R = np.zeros(N * Q, complex)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    t = _site(x, y, z, nx, ny)
                    xg = (x * gG[0] + y * gG[1] + z * gG[2]) * dx
                    R[t * Q:(t + 1) * Q] = 1.0 if classical else np.exp(-1j * xg * fk * dt) * math.exp(-dt / T2v[ph[t]])
        h = Cs @ g
        g = R * (A @ h + B @ np.conj(h))
        F += fk * dt
    return g.reshape(nz, ny, nx, Q)


# ------------------------------------------------------- slab (matrix form)
def slab_signal(a, D, gG, f, dt, T2=math.inf, n_modes=80):
    """|E| for one impermeable slab of width a, gradient normal to it.

    Basis: Neumann cosines phi_0 = 1/sqrt(a), phi_n = sqrt(2/a) cos(n pi x/a).
    dM/dt = -(D Lam + i gG f X + 1/T2) M with X_mn = <phi_m, (x - a/2) phi_n>;
    the offset a/2 only adds a global phase that vanishes when sum f = 0.
    Piecewise-constant f is integrated exactly with matrix exponentials.
    """
    n = np.arange(n_modes)
    lam = (n * math.pi / a) ** 2
    X = np.zeros((n_modes, n_modes))
    xs, wq = np.polynomial.legendre.leggauss(400)
    xs = (xs + 1) * a / 2
    wq = wq * a / 2
    phi = np.array([np.full_like(xs, 1 / math.sqrt(a)) if m == 0 else math.sqrt(2 / a) * np.cos(m * math.pi * xs / a)
                    for m in n])
    X = (phi * (xs - a / 2) * wq) @ phi.T
    v = np.zeros(n_modes, complex)
    v[0] = 1.0
    # group consecutive equal f values
    f = np.asarray(f, float)
    k = 0
    cache = {}
    while k < len(f):
        j = k
        while j < len(f) and f[j] == f[k]:
            j += 1
        key = (f[k], j - k)
        if key not in cache:
            Hm = -(D * np.diag(lam) + 1j * gG * f[k] * X + np.eye(n_modes) / T2)
            cache[key] = sla.expm(Hm * (j - k) * dt)
        v = cache[key] @ v
        k = j
    return abs(v[0])


def slab_field(a, D, gG, f, dt, xi, T2=math.inf, n_modes=120):
    """M(xi, t_end) inside one impermeable slab [0, a] (gradient normal to it,
    coordinate measured from the slab's centre for the reaction, so the field
    carries the global phase of the centre when sum f != 0), at positions xi in
    [0, a], from the same Neumann-mode propagator as ``slab_signal``."""
    n = np.arange(n_modes)
    lam = (n * math.pi / a) ** 2
    xs, wq = np.polynomial.legendre.leggauss(600)
    xs = (xs + 1) * a / 2
    wq = wq * a / 2
    basis = lambda x: np.array([np.full_like(x, 1 / math.sqrt(a)) if m == 0 else
                                math.sqrt(2 / a) * np.cos(m * math.pi * x / a) for m in n])
    phi = basis(xs)
    X = (phi * (xs - a / 2) * wq) @ phi.T
    v = np.zeros(n_modes, complex)
    v[0] = math.sqrt(a)          # M = 1 projected on phi_0
    f = np.asarray(f, float)
    k = 0
    while k < len(f):
        j = k
        while j < len(f) and f[j] == f[k]:
            j += 1
        Hm = -(D * np.diag(lam) + 1j * gG * f[k] * X + np.eye(n_modes) / T2)
        v = sla.expm(Hm * (j - k) * dt) @ v
        k = j
    return basis(np.asarray(xi, float)).T @ v


def exchange_field(a1, a2, D1, D2, T21, T22, kappa, t_end, xq, n_cells=2000):
    """M at positions xq (from the left wall) at t_end for the set-up of
    ``exchange_signal``, by linear interpolation of the cell values."""
    n1 = max(2, int(round(n_cells * a1 / (a1 + a2))))
    n2 = max(2, n_cells - n1)
    h1, h2 = a1 / n1, a2 / n2
    n = n1 + n2
    h = np.array([h1] * n1 + [h2] * n2)
    Dc = np.array([D1] * n1 + [D2] * n2)
    rate = np.array([1 / T21] * n1 + [1 / T22] * n2)
    Amat = np.zeros((n, n))
    for j in range(n - 1):
        if j == n1 - 1:
            res = h1 / (2 * D1) + (1 / kappa if kappa > 0 else math.inf) + h2 / (2 * D2)
            g = 0.0 if math.isinf(res) else 1.0 / res
        else:
            g = 1.0 / (h[j] / (2 * Dc[j]) + h[j + 1] / (2 * Dc[j + 1]))
        Amat[j, j] -= g / h[j]
        Amat[j, j + 1] += g / h[j]
        Amat[j + 1, j + 1] -= g / h[j + 1]
        Amat[j + 1, j] += g / h[j + 1]
    Amat -= np.diag(rate)
    M = sla.expm(Amat * t_end) @ np.ones(n)
    xc = np.concatenate([(np.arange(n1) + 0.5) * h1, a1 + (np.arange(n2) + 0.5) * h2])
    xq = np.asarray(xq, float)
    out = np.empty(xq.shape)
    left = xq < a1
    out[left] = np.interp(xq[left], xc[:n1], M[:n1])
    out[~left] = np.interp(xq[~left], xc[n1:], M[n1:])
    return out


# --------------------------------------------------- two-compartment exchange
def exchange_signal(a1, a2, D1, D2, T21, T22, kappa, t_end, n_cells=400):
    """Mean M over [0, a1 + a2] at t_end, M(0) = 1, Neumann outer walls,
    membrane at x = a1 with flux kappa (M_2 - M_1), no gradient."""
    n1 = max(2, int(round(n_cells * a1 / (a1 + a2))))
    n2 = max(2, n_cells - n1)
    h1, h2 = a1 / n1, a2 / n2
    n = n1 + n2
    h = np.array([h1] * n1 + [h2] * n2)
    Dc = np.array([D1] * n1 + [D2] * n2)
    rate = np.array([1 / T21] * n1 + [1 / T22] * n2)
    Amat = np.zeros((n, n))
    for j in range(n - 1):
        if j == n1 - 1:
            res = h1 / (2 * D1) + (1 / kappa if kappa > 0 else math.inf) + h2 / (2 * D2)
            g = 0.0 if math.isinf(res) else 1.0 / res
        else:
            g = 1.0 / (h[j] / (2 * Dc[j]) + h[j + 1] / (2 * Dc[j + 1]))
        Amat[j, j] -= g / h[j]
        Amat[j, j + 1] += g / h[j]
        Amat[j + 1, j + 1] -= g / h[j + 1]
        Amat[j + 1, j] += g / h[j + 1]
    Amat -= np.diag(rate)
    M = sla.expm(Amat * t_end) @ np.ones(n)
    return float((M * h).sum() / (a1 + a2))


def karger_signal(a1, a2, D1, D2, T21, T22, kappa, t_end):
    """Slow-exchange (well-mixed compartments) limit of ``exchange_signal``."""
    A = np.array([[-1 / T21 - kappa / a1, kappa / a1],
                  [kappa / a2, -1 / T22 - kappa / a2]])
    m = sla.expm(A * t_end) @ np.ones(2)
    return float((m[0] * a1 + m[1] * a2) / (a1 + a2))
