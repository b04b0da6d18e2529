"""Plain FP64 CPU oracle of the SCF gravity step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is the slow, obviously-correct
definition of what the CUDA path computes, written from the paper:

* Eq. 1-3 (basis expansion, coefficients as a mass-weighted particle sum),
* Eq. 4, the Zhao (1996) radial family of exponent ``alpha`` (every basis
  function takes it; the default 1 is the Hernquist-Ostriker Gegenbauer basis),
* Sec. 2.1 (accelerating, non-rotating cluster frame; COM test particle),
* App. A (Hernquist, NFW, Miyamoto-Nagai host components).

The arithmetic lives in ``scf_oracle.c`` (plain C, double precision, long
double for the host tidal difference).  This module compiles it with gcc on
first use and wraps it with ctypes; numpy arrays in, numpy arrays out.

Array conventions (shared with the CUDA path by specification, not by code):
positions ``(N, 4)`` = (x, y, z, m); velocities ``(N, 4)`` = (vx, vy, vz, 0);
accelerations ``(N, 4)`` = (ax, ay, az, potential); coefficients ``A`` =
``[S | T]`` with ``(nmax+1) * (lmax+1)(lmax+2)/2`` entries each, index
``n * N_lm + l(l+1)/2 + m``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

HOST_HERNQUIST = 1
HOST_NFW = 2
HOST_MN = 3


class _HostComp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("M", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double)]


class _Host(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("G", ctypes.c_double), ("c", _HostComp * 8)]


def build(force: bool = False) -> str:
    """Compile ``scf_oracle.c`` into ``liboracle.so`` (gcc, -O2, no fast-math)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "or_gegenbauer": (d, [i, d, d]),
        "or_plm": (d, [i, i, d]),
        "or_dplm_dtheta": (d, [i, i, d]),
        "or_mplm_over_sin": (d, [i, i, d]),
        "or_nlm2": (d, [i, i]),
        "or_knl": (d, [i, i, d]),
        "or_inl": (d, [i, i, d, d]),
        "or_phi_nl": (d, [i, i, d, d, d]),
        "or_phi_nl_over_r": (d, [i, i, d, d, d]),
        "or_dphi_nl_dr": (d, [i, i, d, d, d]),
        "or_rho_nl": (d, [i, i, d, d, d]),
        "or_coeffs": (None, [i64, p, p, i, i, d, d, p]),
        "or_field": (None, [i64, p, p, i, i, d, d, d, p]),
        "or_density": (None, [i64, p, p, i, i, d, d, p]),
        "or_host_accel": (None, [p, p, p, p]),
        "or_tidal": (None, [p, p, p, p]),
        "or_tidal_tensor": (None, [p, i64, p, p]),
        "or_host_accel_many": (None, [p, i64, p, p]),
        "or_tidal_many": (None, [p, p, i64, p, p]),
        "or_forces": (None, [i64, p, p, p, p, i, i, d, d, d, p]),
        "or_energy": (None, [i64, p, p, p, p, p, i, i, d, d, d, p]),
        "or_step": (None, [i64, p, p, p, p, p, i, i, d, d, d, d, i, p, p, p]),
        "or_direct": (None, [i64, p, i64, p, d, p]),
        "or_power_l": (None, [p, i, i, d, d, p]),
        "or_num_threads": (i, []),
        "or_lower_gamma": (d, [d, d]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def n_lm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def n_coef(nmax: int, lmax: int) -> int:
    """Length of one of the S or T halves of a coefficient vector."""
    return (nmax + 1) * n_lm(lmax)


def idx(n: int, l: int, m: int, lmax: int) -> int:
    return n * n_lm(lmax) + l * (l + 1) // 2 + m


def host_struct(components, G: float = 1.0):
    """``components``: iterable of ``(kind, M, a, b)`` tuples (b unused except MN)."""
    h = _Host()
    comps = list(components)
    if len(comps) > 8:
        raise ValueError("at most 8 host components")
    h.n = len(comps)
    h.G = G
    for k, (kind, M, a, b) in enumerate(comps):
        h.c[k].kind, h.c[k].M, h.c[k].a, h.c[k].b = int(kind), float(M), float(a), float(b)
    return h


# ---------------------------------------------------------------- scalars
def gegenbauer(n, alpha, xi):
    return _load().or_gegenbauer(int(n), float(alpha), float(xi))


def plm(l, m, x):
    return _load().or_plm(int(l), int(m), float(x))


def dplm_dtheta(l, m, costh):
    return _load().or_dplm_dtheta(int(l), int(m), float(costh))


def mplm_over_sin(l, m, costh):
    return _load().or_mplm_over_sin(int(l), int(m), float(costh))


def nlm2(l, m):
    return _load().or_nlm2(int(l), int(m))


# ``alpha``: the exponent of the Zhao (1996) radial family (Eq. 4); 1 is the
# Hernquist-Ostriker basis, 1/2 the Clutton-Brock one.
def knl(n, l, alpha=1.0):
    return _load().or_knl(int(n), int(l), float(alpha))


def inl(n, l, b, alpha=1.0):
    return _load().or_inl(int(n), int(l), float(b), float(alpha))


def phi_nl(n, l, b, r, alpha=1.0):
    return _load().or_phi_nl(int(n), int(l), float(b), float(alpha), float(r))


def phi_nl_over_r(n, l, b, r, alpha=1.0):
    return _load().or_phi_nl_over_r(int(n), int(l), float(b), float(alpha), float(r))


def dphi_nl_dr(n, l, b, r, alpha=1.0):
    return _load().or_dphi_nl_dr(int(n), int(l), float(b), float(alpha), float(r))


def rho_nl(n, l, b, r, alpha=1.0):
    return _load().or_rho_nl(int(n), int(l), float(b), float(alpha), float(r))


# ---------------------------------------------------------------- arrays
def coeffs(pos, nmax, lmax, b, mask=None, alpha=1.0):
    """Real-form coefficients ``[S | T]`` of Eq. 3b for ``pos`` (N, 4)."""
    pos = _f64(pos)
    n = pos.shape[0]
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    A = np.zeros(2 * n_coef(nmax, lmax))
    _load().or_coeffs(n, _ptr(pos), _ptr(m), int(nmax), int(lmax), float(b), float(alpha), _ptr(A))
    return A


def field(pos, A, nmax, lmax, b, G=1.0, alpha=1.0):
    """(N, 4) = (ax, ay, az, potential) of the expansion at ``pos[:, :3]``."""
    pos = _f64(pos)
    A = _f64(A)
    out = np.zeros((pos.shape[0], 4))
    _load().or_field(pos.shape[0], _ptr(pos), _ptr(A), int(nmax), int(lmax), float(b), float(alpha), float(G),
                     _ptr(out))
    return out


def density(pos, A, nmax, lmax, b, alpha=1.0):
    """Mass density of the expansion (Eq. 1b) at ``pos[:, :3]`` -> (N,)."""
    pos = _f64(pos)
    A = _f64(A)
    out = np.zeros(pos.shape[0])
    _load().or_density(pos.shape[0], _ptr(pos), _ptr(A), int(nmax), int(lmax), float(b), float(alpha), _ptr(out))
    return out


def lower_gamma(a, x):
    """Lower incomplete gamma function gamma(a, x) (unregularised), long double
    series / continued fraction of the oracle (App. A bulge)."""
    return _load().or_lower_gamma(float(a), float(x))


def host_accel(host, x):
    x = _f64(x)
    a = np.zeros(3)
    pot = np.zeros(1)
    _load().or_host_accel(ctypes.byref(host), _ptr(x), _ptr(a), _ptr(pot))
    return a, float(pot[0])


def tidal(host, R, x):
    R = _f64(R)
    x = _f64(x)
    a = np.zeros(3)
    _load().or_tidal(ctypes.byref(host), _ptr(R), _ptr(x), _ptr(a))
    return a


def tidal_tensor(host, P):
    """Tidal tensors d a_host / dx (App. A) at points ``P`` (n, 3) -> (n, 3, 3)."""
    P = _f64(np.atleast_2d(P))
    T = np.zeros((P.shape[0], 3, 3))
    _load().or_tidal_tensor(ctypes.byref(host), P.shape[0], _ptr(P), _ptr(T))
    return T


def host_accel_many(host, P):
    """Host acceleration at points ``P`` (n, 3) -> (n, 3)."""
    P = _f64(np.atleast_2d(P))
    a = np.zeros((P.shape[0], 3))
    _load().or_host_accel_many(ctypes.byref(host), P.shape[0], _ptr(P), _ptr(a))
    return a


def tidal_many(host, R, pos):
    """a_host(R + x_k) - a_host(R) for particles ``pos`` (n, 4) -> (n, 3)."""
    R = _f64(R)[:3].copy()
    pos = _f64(pos)
    a = np.zeros((pos.shape[0], 3))
    _load().or_tidal_many(ctypes.byref(host), _ptr(R), pos.shape[0], _ptr(pos), _ptr(a))
    return a


def forces(pos, A, nmax, lmax, b, G=1.0, com=None, host=None, alpha=1.0):
    pos = _f64(pos)
    A = _f64(A)
    out = np.zeros((pos.shape[0], 4))
    c = None if com is None else _f64(com)
    hp = None if host is None else ctypes.byref(host)
    _load().or_forces(pos.shape[0], _ptr(pos), _ptr(A), _ptr(c), hp, int(nmax), int(lmax), float(b), float(alpha),
                      float(G), _ptr(out))
    return out


def energy(pos, vel, A, nmax, lmax, b, G=1.0, com=None, host=None, alpha=1.0):
    """(K, W, U, K + W + U): kinetic, self (1/2 sum m psi_SCF) and tidal
    energy of the particles in the cluster frame (see or_energy)."""
    pos = _f64(pos)
    vel = _f64(vel)
    A = _f64(A)
    out = np.zeros(4)
    c = None if com is None else _f64(com)
    hp = None if host is None else ctypes.byref(host)
    _load().or_energy(pos.shape[0], _ptr(pos), _ptr(vel), _ptr(A), _ptr(c), hp, int(nmax), int(lmax), float(b),
                      float(alpha), float(G), _ptr(out))
    return out


def step(pos, vel, acc, nmax, lmax, b, dt, nsteps, G=1.0, com=None, host=None, A_frozen=None, mask=None,
         alpha=1.0):
    """Kick-drift-kick leapfrog; returns new ``(pos, vel, acc, com, A_last)``.

    ``acc`` must hold the acceleration at ``pos`` (from :func:`forces`);
    ``mask`` (optional, per particle) is the coefficient set of Eq. 3b."""
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    acc = _f64(acc).copy()
    com = np.zeros(6) if com is None else _f64(com).copy()
    A_out = np.zeros(2 * n_coef(nmax, lmax))
    hp = None if host is None else ctypes.byref(host)
    Af = None if A_frozen is None else _f64(A_frozen)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    _load().or_step(pos.shape[0], _ptr(pos), _ptr(vel), _ptr(acc), _ptr(com), hp, int(nmax), int(lmax), float(b),
                    float(alpha), float(G), float(dt), int(nsteps), _ptr(Af), _ptr(mk), _ptr(A_out))
    return pos, vel, acc, com, A_out


def direct(src, tgt, G=1.0):
    """Unsoftened direct-summation (ax, ay, az, potential) at ``tgt`` from ``src``."""
    src = _f64(src)
    tgt = _f64(tgt)
    out = np.zeros((tgt.shape[0], 4))
    _load().or_direct(src.shape[0], _ptr(src), tgt.shape[0], _ptr(tgt), float(G), _ptr(out))
    return out


# ---------------------------------------------------------------- escape physics
def boundedness(pos, vel, G=1.0, kin=0.5, frac=0.999):
    """Energy-based boundedness and the radius of the coefficient set (Sec. 2.2).

    Particle i is bound when its cluster-frame energy
    ``E_i = kin |v_i|^2 - sum_{j != i} G m_j / |r_i - r_j|`` is negative, the
    sum being the unsoftened direct summation over every particle of the
    progenitor (coincident pairs are skipped like the self term).  The
    footnote of Sec. 2.2 prints ``kin = 1``; the standard specific energy
    has ``kin = 1/2`` (the default).  ``r_x`` is the smallest radius that
    encloses the fraction ``frac`` of the bound particles, i.e. the k-th
    smallest cluster-frame radius among them with ``k = ceil(frac n_bound)``;
    the particles that enter Eq. 3b are those with ``r <= r_x``.  With no
    bound particle ``r_x = 0``.  Radii are compared through
    ``r^2 = (x x + y y) + z z`` in double precision.

    Returns ``(E, bound, r_x^2, mask, M_bound)``.
    """
    pos = _f64(pos)
    vel = _f64(vel)
    n = pos.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros(0, bool), 0.0, np.zeros(0, bool), 0.0
    v2 = vel[:, 0] * vel[:, 0] + vel[:, 1] * vel[:, 1] + vel[:, 2] * vel[:, 2]
    E = kin * v2 + direct(pos, pos, G)[:, 3]
    bound = E < 0.0
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    r2 = x * x + y * y + z * z
    nb = int(bound.sum())
    if nb == 0:
        rx2 = 0.0
    else:
        k = max(1, int(np.ceil(frac * float(nb))))
        rx2 = float(np.sort(r2[bound])[min(k, nb) - 1])
    mask = r2 <= rx2
    return E, bound, rx2, mask, float(pos[bound, 3].sum())


def tidal_scales(host, R, M_c, eta=1.0 / 400.0, G=1.0):
    """Tidal tensor, its eigenvalues, the tidal radius and the integration
    timestep at centre positions ``R`` (n, 3) for cluster masses ``M_c`` (n,).

    * ``T_ij = -d^2 psi_host / dx_i dx_j`` (Sec. 2.2, App. A), here the
      derivative of the host acceleration (``tidal_tensor``);
    * eigenvalues ``l1 >= l2 >= l3`` (numpy's symmetric eigensolver);
    * tidal radius ``r_t = (G M_c / l1e)^(1/3)`` with
      ``l1e = l1 - (l2 + l3)/2`` (Sec. 3.1, footnote on generic orbits);
      infinite when ``l1e <= 0``;
    * integration timestep ``dt_int = sqrt(eta) (|T|_F^2 / 6)^(-1/4)``
      (Sec. 2.2, with the Frobenius norm).

    Returns an (n, 16) array laid out as ``T`` (row-major, 9), ``l1, l2, l3``,
    ``|T|_F``, ``l1e``, ``r_t``, ``dt_int``.
    """
    R = _f64(np.atleast_2d(R))[:, :3].copy()
    M_c = _f64(np.atleast_1d(M_c))
    T = tidal_tensor(host, R)
    out = np.zeros((R.shape[0], 16))
    for i in range(R.shape[0]):
        Ts = 0.5 * (T[i] + T[i].T)
        lam = np.sort(np.linalg.eigvalsh(Ts))[::-1]
        fro = float(np.sqrt(np.sum(T[i] * T[i])))
        l1e = lam[0] - 0.5 * (lam[1] + lam[2])
        r_t = (G * M_c[i] / l1e) ** (1.0 / 3.0) if l1e > 0 else np.inf
        dt_int = np.sqrt(eta) * (fro * fro / 6.0) ** (-0.25) if fro > 0 else np.inf
        out[i, :9] = T[i].reshape(9)
        out[i, 9:12] = lam
        out[i, 12] = fro
        out[i, 13] = l1e
        out[i, 14] = r_t
        out[i, 15] = dt_int
    return out


def zhao_half_mass_scale(r50, alpha=1.0):
    """Scale b of the lowest-order density of the Zhao family (Eq. 4) whose
    half-mass radius is ``r50``.  The enclosed mass of rho_00, from
    M(r) = r^2 dU_00/dr, is (t / (1 + t))^(alpha + 1) with t = (r/b)^(1/alpha),
    so M = 1/2 at t = 1 / (2^(1/(alpha+1)) - 1) and
    ``b = r50 (2^(1/(alpha+1)) - 1)^alpha`` (alpha = 1: r50 / (1 + sqrt 2),
    the Hernquist scale; alpha = 1/2: r50 sqrt(2^(2/3) - 1), the Plummer one)."""
    if alpha == 1.0:
        return float(r50) / (1.0 + np.sqrt(2.0))
    return float(r50) * (2.0 ** (1.0 / (alpha + 1.0)) - 1.0) ** alpha


def evolve(pos, vel, acc, nmax, lmax, b, dt, nsteps, G=1.0, com=None, host=None, kin=0.5, frac=0.999,
           eta=1.0 / 400.0, max_steps=1000, retune_every=0, alpha=1.0, recentre=False, retune_rule="half_mass",
           alpha_range=(0.25, 2.0), return_alpha=False):
    """Leapfrog with the escape physics of Sec. 2.2.  At the start of every
    integration timestep: the boundedness test and the coefficient set
    r <= r_x (:func:`boundedness`); at every ``retune_every``-th integration
    timestep (the first included; 0 = never) a complete refresh, which (with
    ``recentre``) first moves the frame to the SCF centre and core velocity
    (:func:`recentre`, over the coefficient set) and takes the boundedness
    again in it, then
    retunes the basis scale b (alpha fixed): with ``retune_rule="a000"`` to
    the maximum of a_000 (:func:`a000_scale`, over the coefficient set); with
    ``"alpha_a000"`` alpha and b together at the joint maximum of a_000
    (:func:`a000_alpha_scale`, alpha in ``alpha_range``); else
    to the scale of the lowest-order
    density whose half-mass radius is the bound stars' energy-based one,
    :func:`zhao_half_mass_scale` (alpha = 1: b = r_50 / (1 + sqrt 2)); the field
    of the coefficient set at the current positions; and the length of the
    integration timestep, dt_int of :func:`tidal_scales` at the current
    centre with the bound mass as M_c, taken as
    ``clamp(floor(dt_int / dt), 1, max_steps)`` leapfrog steps (``max_steps``
    without a host; fewer at the end).

    Returns ``(pos, vel, acc, com, bound, mask, stats, n_int, b)`` with
    ``bound``, ``mask`` and ``stats = (n_bound, M_bound, r_x, set size)`` as
    of the start of the last integration timestep and ``b`` the scale in use
    (``return_alpha``: and then the exponent in use)."""
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    com = np.zeros(6) if com is None else _f64(com).copy()
    has_host = host is not None and host.n > 0
    done, n_int = 0, 0
    bound = mask = None
    stats = np.zeros(4)
    b = float(b)
    while done < nsteps:
        E, bound, rx2, mask, Mb = boundedness(pos, vel, G, kin, frac)
        stats = np.array([bound.sum(), Mb, np.sqrt(rx2), mask.sum()], dtype=np.float64)
        if retune_every > 0 and n_int % retune_every == 0:
            if recentre:   # the frame to the SCF centre and core velocity, boundedness again in it
                pos, vel, com, _, _, _, _ = _recentre_frame(pos, vel, com, nmax, lmax, b, alpha, mask=mask)
                E, bound, rx2, mask, Mb = boundedness(pos, vel, G, kin, frac)
                stats = np.array([bound.sum(), Mb, np.sqrt(rx2), mask.sum()], dtype=np.float64)
            if retune_rule == "a000":   # b maximising a_000 of the coefficient set
                b = a000_scale(pos, b, alpha, mask=mask)
            elif retune_rule == "alpha_a000":   # alpha and b at the joint maximum
                alpha, bs = a000_alpha_scale(pos, alpha, b, mask=mask, alpha_range=alpha_range)
                b = float(bs[0])
            elif bound.any():
                r50 = np.sqrt(boundedness(pos, vel, G, kin, 0.5)[2])
                b = zhao_half_mass_scale(r50, alpha)
        A = coeffs(pos, nmax, lmax, b, mask=mask, alpha=alpha)
        acc = forces(pos, A, nmax, lmax, b, G, com=com if has_host else None, host=host if has_host else None,
                     alpha=alpha)
        k = max_steps
        if has_host:
            dt_int = tidal_scales(host, com[:3], np.array([Mb]), eta, G)[0, 15]
            ks = np.floor(dt_int / dt)
            if ks < k:
                k = 1 if ks < 1 else int(ks)
        k = min(k, nsteps - done)
        pos, vel, acc, c2, _ = step(pos, vel, acc, nmax, lmax, b, dt, k, G, com=com if has_host else None,
                                    host=host if has_host else None, mask=mask, alpha=alpha)
        if has_host:    # without a host the centre is not integrated (it keeps the re-centring offsets)
            com = c2
        done += k
        n_int += 1
    if return_alpha:
        return pos, vel, acc, com, bound, mask, stats, n_int, b, alpha
    return pos, vel, acc, com, bound, mask, stats, n_int, b


# ---------------------------------------------------------------- re-centring (Sec. 2.1)
def a000_profile(s, alpha=1.0):
    """g(s) = (1 + s^(1/alpha))^-alpha = -b U_00(r): the radial profile of the
    lowest-order potential (Eq. 4), s = r/b."""
    s = np.asarray(s, dtype=np.float64)
    return (1.0 + s ** (1.0 / alpha)) ** -alpha


def expansion_centre(pos, b, alpha=1.0, mask=None, tol=1e-12, max_iter=100):
    """The point x_c at which a_000 of the particles' expansion is largest
    (Sec. 2.1: the SCF centre), the expansion taken about x_c with alpha and b
    fixed, over the coefficient set (``mask``; all particles if None).

    a_000 is a positive multiple of F(x_c) = sum_k m_k g(|x_k - x_c| / b) (the
    lowest basis function is -g/b times a constant, its normalisation I_00 < 0),
    so x_c solves grad F = 0, i.e. sum_k m_k w_k (x_k - x_c) = 0 with
    w_k = -g'(s_k)/s_k = t_k (1 + t_k)^(-alpha-1) / s_k^2, t = s^(1/alpha).  The
    iteration x_c <- sum m w x / sum m w from x_c = 0 (the current centre)
    climbs F (a mean-shift step); it stops when the step is below tol * b or
    after max_iter steps.  s_k^2 is floored at 1e-300 (a particle on x_c: the
    iteration has arrived there).  Returns (x_c, iterations)."""
    pos = _f64(pos)
    sel = np.ones(pos.shape[0], bool) if mask is None else np.asarray(mask, bool)
    x, m = pos[sel, :3], pos[sel, 3]
    xc = np.zeros(3)
    it = 0
    if not (m.sum() > 0.0):     # an empty set (or no mass): the centre stays
        return xc, 0
    for it in range(1, max_iter + 1):
        d = x - xc
        s2 = np.maximum((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) / (b * b), 1e-300)
        s = np.sqrt(s2)
        t = s ** (1.0 / alpha)
        w = m * t * (1.0 + t) ** (-alpha - 1.0) / s2
        new = (w[:, None] * x).sum(axis=0) / w.sum()
        step = np.sqrt(np.sum((new - xc) ** 2))
        xc = new
        if step <= tol * b:
            break
    return xc, it


def core_frame(pos, vel, A, nmax, lmax, b, alpha=1.0):
    """Core radius and core velocity about the current centre (Sec. 2.1):
    r_core^2 = sum_i rho_i^2 r_i^2 / sum_i rho_i^2 with rho_i the expansion's
    density at each particle (:func:`density`; particles at r = 0, where a
    cusped rho is infinite, are left out of both sums), and the frame velocity
    = the mass-weighted mean velocity of the particles with r < r_core.
    Returns (r_core, V_core)."""
    pos = _f64(pos)
    vel = _f64(vel)
    rho = density(pos, A, nmax, lmax, b, alpha)
    r2 = pos[:, 0] * pos[:, 0] + pos[:, 1] * pos[:, 1] + pos[:, 2] * pos[:, 2]
    ok = r2 > 0.0
    w = rho[ok] * rho[ok]
    rc2 = float((w * r2[ok]).sum() / w.sum()) if w.sum() > 0 else 0.0
    core = r2 < rc2
    mc = pos[core, 3]
    V = (mc[:, None] * vel[core, :3]).sum(axis=0) / mc.sum() if mc.sum() > 0 else np.zeros(3)
    return float(np.sqrt(rc2)), V


def recentre(pos, vel, com, nmax, lmax, b, alpha=1.0, mask=None, tol=1e-12, max_iter=100):
    """Moves the cluster frame to the SCF centre with the core velocity
    (Sec. 2.1): x_c of :func:`expansion_centre`, then the coefficients of the
    set about x_c, then :func:`core_frame` about x_c; particles are shifted by
    (-x_c, -V_core) and the centre by (+x_c, +V_core), so host-frame positions
    and velocities are unchanged.  Returns (pos, vel, com, x_c, V_core, r_core,
    iterations)."""
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    com = np.zeros(6) if com is None else _f64(com).copy()
    xc, it = expansion_centre(pos, b, alpha, mask, tol, max_iter)
    pos[:, :3] -= xc
    com[:3] += xc
    A = coeffs(pos, nmax, lmax, b, mask=mask, alpha=alpha)
    rc, V = core_frame(pos, vel, A, nmax, lmax, b, alpha)
    vel[:, :3] -= V
    com[3:] += V
    return pos, vel, com, xc, V, rc, it


_recentre_frame = recentre   # (evolve's keyword of the same name shadows it there)


def a000_biorth(pos, b, alpha=1.0, mask=None):
    """a_000 of the particles about the origin in the bi-orthonormal
    normalisation of Eq. 3a (the lowest pair scaled to unit self-energy,
    psi_000 = U_00 Y_00 / sqrt|I_00(b)|), as a function of b (alpha fixed):
    a_000 = Y_00 / sqrt(|I_00(1)| b) sum_k m_k g(r_k / b)."""
    pos = _f64(pos)
    sel = np.ones(pos.shape[0], bool) if mask is None else np.asarray(mask, bool)
    r = np.sqrt(np.sum(pos[sel, :3] ** 2, axis=1))
    y00 = 1.0 / np.sqrt(4.0 * np.pi)
    return y00 / np.sqrt(abs(inl(0, 0, 1.0, alpha)) * b) * float(np.sum(pos[sel, 3] * a000_profile(r / b, alpha)))


def a000_scale_slope(pos, lnb, alpha=1.0, mask=None):
    """d ln a_000 / d ln b at b = exp(lnb) (alpha and the centre fixed).
    With t_k = (r_k / b)^(1/alpha), g = (1 + t)^-alpha and -s g'(s) = t (1 + t)^(-alpha-1):
    d ln h / d ln b = -1/2 + sum m t (1+t)^(-alpha-1) / sum m (1+t)^-alpha,
    h(b) = b^(-1/2) sum m g(r/b) the b-dependent factor of a_000."""
    pos = _f64(pos)
    sel = np.ones(pos.shape[0], bool) if mask is None else np.asarray(mask, bool)
    r = np.sqrt(np.sum(pos[sel, :3] ** 2, axis=1))
    m = pos[sel, 3]
    t = (r / np.exp(lnb)) ** (1.0 / alpha)
    return -0.5 + float(np.sum(m * t * (1.0 + t) ** (-alpha - 1.0))) / float(np.sum(m * (1.0 + t) ** -alpha))


def a000_scale(pos, b0, alpha=1.0, mask=None, span=8.0, points=257):
    """The basis scale that maximises :func:`a000_biorth` (Sec. 2: b tuned so
    that the lowest mode approximates the cluster; Sec. 2.1: the same
    criterion as the centre), over b in [b0/span, b0 span].  The largest of
    the b-dependent factor h(b) = b^(-1/2) sum m g(r/b) on ``points`` values
    of ln b brackets the maximum; inside the bracket the maximum is the root of
    :func:`a000_scale_slope`, found by bisection to the last bit of ln b.  A
    maximum at an end of the range returns that end; an empty set keeps b0."""
    pos = _f64(pos)
    sel = np.ones(pos.shape[0], bool) if mask is None else np.asarray(mask, bool)
    if not sel.any():
        return float(b0)
    r = np.sqrt(np.sum(pos[sel, :3] ** 2, axis=1))
    m = pos[sel, 3]

    def h(lnb):
        bb = np.exp(lnb)
        return bb ** -0.5 * float(np.sum(m * a000_profile(r / bb, alpha)))

    xs = np.linspace(np.log(b0) - np.log(span), np.log(b0) + np.log(span), points)
    j = int(np.argmax([h(x) for x in xs]))
    if j == 0 or j == points - 1:
        return float(np.exp(xs[j]))
    lo, hi = xs[j - 1], xs[j + 1]
    slope = lambda x: a000_scale_slope(pos, x, alpha, mask)
    if not (slope(lo) > 0.0 > slope(hi)):
        return float(np.exp(xs[j]))
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if slope(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return float(np.exp(0.5 * (lo + hi)))


def dln_i00_dalpha(alpha):
    """d ln|I_00| / d alpha of the lowest pair's normalisation (at b = 1),
    I_00 = -(alpha + 1) Gamma(2 alpha + 1) / (2^(4 alpha + 3) (alpha + 1/2) Gamma(alpha + 1/2)^2)
    (the n = l = 0 case of the closed form in the Zhao family):
    1/(alpha+1) + 2 psi(2 alpha + 1) - 4 ln 2 - 1/(alpha + 1/2) - 2 psi(alpha + 1/2)."""
    from scipy.special import digamma
    a = float(alpha)
    return 1.0 / (a + 1.0) + 2.0 * digamma(2.0 * a + 1.0) - 4.0 * np.log(2.0) - 1.0 / (a + 0.5) - 2.0 * digamma(a + 0.5)


def a000_alpha_slope(pos, alpha, b, mask=None):
    """d ln a_000 / d alpha at fixed b and centre (bi-orthonormal normalisation):
    -1/2 d ln|I_00|/d alpha + sum m g d ln g/d alpha / sum m g, with g = (1 + t)^-alpha,
    t = (r/b)^(1/alpha) and d ln g / d alpha = -ln(1 + t) + t ln(r/b) / (alpha (1 + t))."""
    pos = _f64(pos)
    sel = np.ones(pos.shape[0], bool) if mask is None else np.asarray(mask, bool)
    r = np.sqrt(np.sum(pos[sel, :3] ** 2, axis=1))
    m = pos[sel, 3]
    s = r / b
    t = s ** (1.0 / alpha)
    g = (1.0 + t) ** -alpha
    with np.errstate(divide="ignore", invalid="ignore"):
        tls = np.where(s > 0.0, t * np.log(np.where(s > 0.0, s, 1.0)), 0.0)
    dlng = -np.log1p(t) + tls / (alpha * (1.0 + t))
    return -0.5 * dln_i00_dalpha(alpha) + float(np.sum(m * g * dlng)) / float(np.sum(m * g))


def a000_alpha_scale(pos, alpha0, b0, offsets=None, mask=None, alpha_range=(0.25, 2.0), points=33, span=8.0):
    """The exponent alpha of the radial family (Eq. 4) and the scales b_p that
    maximise a_000 (the same criterion as b alone; Secs. 2 and 2.2: a complete
    refresh retunes alpha and b).  One alpha is shared by the progenitors
    (``offsets``, as in a batched handle): it maximises the product of their
    a_000, each at its own maximising b_p(alpha) (:func:`a000_scale`).  By the
    envelope theorem d/d alpha of sum_p ln a_000,p(alpha, b_p(alpha)) is the sum
    of :func:`a000_alpha_slope` at b_p(alpha).  ``points`` values of ln alpha over
    ``alpha_range`` bracket the maximum of that sum; bisection on its slope
    finds it to the last bit (an end of the range returns that end).
    Progenitors with an empty set keep b0 and take no part.  Returns
    ``(alpha, b)`` with b an array of the progenitors' scales."""
    pos = _f64(pos)
    offsets = [0, pos.shape[0]] if offsets is None else [int(o) for o in offsets]
    b0 = np.broadcast_to(np.asarray(b0, dtype=np.float64), (len(offsets) - 1,)).copy()
    sel = np.ones(pos.shape[0], bool) if mask is None else np.asarray(mask, bool)
    live = [p for p in range(len(offsets) - 1) if sel[offsets[p]:offsets[p + 1]].any()]
    if not live:
        return float(alpha0), b0

    def parts(p):
        lo, hi = offsets[p], offsets[p + 1]
        return pos[lo:hi], sel[lo:hi]

    def scales(al):
        b = b0.copy()
        for p in live:
            q, m = parts(p)
            b[p] = a000_scale(q, b0[p], al, mask=m, span=span)
        return b

    def H(al):
        b = scales(al)
        return sum(np.log(a000_biorth(*parts(p)[:1], b[p], al, mask=parts(p)[1])) for p in live)

    def dH(al):
        b = scales(al)
        return sum(a000_alpha_slope(parts(p)[0], al, b[p], mask=parts(p)[1]) for p in live)

    xs = np.linspace(np.log(alpha_range[0]), np.log(alpha_range[1]), points)
    j = int(np.argmax([H(np.exp(x)) for x in xs]))
    if j == 0 or j == points - 1:
        al = float(np.exp(xs[j]))
        return al, scales(al)
    lo, hi = xs[j - 1], xs[j + 1]
    if not (dH(np.exp(lo)) > 0.0 > dH(np.exp(hi))):
        al = float(np.exp(xs[j]))
        return al, scales(al)
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if dH(np.exp(mid)) > 0.0:
            lo = mid
        else:
            hi = mid
    al = float(np.exp(0.5 * (lo + hi)))
    return al, scales(al)


def power_l(A, nmax, lmax, b, alpha=1.0):
    """E_l = sum_{n,m} |a_nlm|^2 in the bi-orthonormal normalisation of Eq. 3a."""
    A = _f64(A)
    El = np.zeros(lmax + 1)
    _load().or_power_l(_ptr(A), int(nmax), int(lmax), float(b), float(alpha), _ptr(El))
    return El


def num_threads() -> int:
    return int(_load().or_num_threads())
