"""Reverse-mode (adjoint) oracle of the SCF leapfrog, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY: imported by the test suite, never by the CUDA
package.  It differentiates the oracle's own forward step (``oracle.step``:
kick-drift-kick of Sec. 2.1 with the centre orbit stepped in the host of
App. A) and shares nothing with the GPU adjoint but the mathematics.

The forward map of one step, for particles x, v (cluster frame) and the
centre R, V, with h = dt/2:

    v' = v + h a(x, R)         V' = V + h g(R)
    x1 = x + dt v'              R1 = R + dt V'
    v1 = v' + h a(x1, R1)       V1 = V' + h g(R1)

where g is the host acceleration, T = dg/dx its tidal tensor (App. A), and

    a_k(x, R) = f(x_k; A(x)) + g(R + x_k) - g(R),   A(x) = sum_j m_j B(x_j),

f(y; A) = -grad psi(y; A) is the field of Eq. 1a and B the vector of basis
functions whose mass-weighted sum is Eq. 3b.  Reversing the six assignments
gives, at every level t (states x_t, R_t), a pull-back of a(x_t, R_t) along
d_k = w_t vbar_k with w_t = h at t = 0 and t = T and dt in between (the
closing kick of step t and the opening kick of step t+1 see the same a):

    xbar_k += sum_i d_i . da_i/dx_k
    Rbar   += sum_k (T(R+x_k) - T(R)) d_k + w_t T(R) Vbar
    thbar  += sum_k d_k . (dg/dth(R+x_k) - dg/dth(R)) + w_t dg/dth(R) . Vbar

followed, for t > 0, by the reversed drift vbar += dt xbar, Vbar += dt Rbar.

The particle term splits into the particle's own position (coefficients held
fixed) and the path through A:

    sum_i d_i . da_i/dx_k = (df/dy)(x_k; A) d_k + T(R+x_k) d_k
                            + m_k (dB/dy)(x_k)^T sum_i (df/dA)(x_i)^T d_i,

and since psi(y; A) = sum_c A_c Psi_c(y) with Psi_c proportional to B_c
(the basis is its own dual up to a constant per coefficient, Eq. 3a), the
last term equals m_k f(x_k; A^J) with A^J = sum_i (dB/dy)(x_i) d_i: the
coefficients of the directional derivative of the particle set.  This
oracle evaluates those directional derivatives by fourth-order central
differences of ``oracle.field`` and ``oracle.coeffs`` (steps of 1e-3 of
min(r, b) per particle), the tidal tensor by the closed forms of App. A
(``oracle.tidal_tensor``), d g / d GM_c = g_c / GM_c exactly, and
d g / d a_c by fourth-order differences of the tidal difference in a_c.
The decomposition itself is pinned against brute-force differences of
sum_i d_i . a_i(x) in the tests.
"""
from __future__ import annotations

import numpy as np

from . import coeffs, field, host_accel_many, host_struct, step, tidal_many, tidal_tensor, forces

_FD = ((-2, 1.0), (-1, -8.0), (1, 8.0), (2, -1.0))   # 4th-order central first derivative, / (12 e)


def _steps(x, d, b, rel=1e-3):
    """Per-particle parameter step e_k with |e_k d_k| = rel * min(r_k, b)."""
    r = np.linalg.norm(x[:, :3], axis=1)
    dn = np.linalg.norm(d, axis=1)
    scale = rel * np.minimum(np.where(r > 0, r, b), b)
    e = np.where(dn > 0, scale / np.where(dn > 0, dn, 1.0), 0.0)
    return e, dn > 0


def jvp_field(x, A, d, nmax, lmax, b, G=1.0):
    """(df/dy)(x_k; A) d_k for every particle: the own-position term."""
    e, live = _steps(x, d, b)
    out = np.zeros((x.shape[0], 3))
    if not live.any():
        return out
    xl, dl, el = x[live], d[live], e[live]
    acc = np.zeros((xl.shape[0], 3))
    for j, c in _FD:
        pts = xl.copy()
        pts[:, :3] += (j * el)[:, None] * dl
        acc += c * field(pts, A, nmax, lmax, b, G)[:, :3]
    out[live] = acc / (12.0 * el)[:, None]
    return out


def jvp_coeffs(x, d, nmax, lmax, b):
    """A^J = sum_i (dB/dy)(x_i) d_i: Eq. 3b is linear in the masses, so the
    four stencil points of every particle enter one coefficient sum with the
    stencil weights / (12 e_i) as masses."""
    e, live = _steps(x, d, b)
    if not live.any():
        return np.zeros(2 * (nmax + 1) * (lmax + 1) * (lmax + 2) // 2)
    xl, dl, el = x[live], d[live], e[live]
    pts = []
    for j, c in _FD:
        p = np.zeros((xl.shape[0], 4))
        p[:, :3] = xl[:, :3] + (j * el)[:, None] * dl
        p[:, 3] = c / (12.0 * el)
        pts.append(p)
    return coeffs(np.concatenate(pts), nmax, lmax, b)


def _single(comp, G, M=None, a=None):
    kind, M0, a0, b0 = comp
    return host_struct([(kind, M0 if M is None else M, a0 if a is None else a, b0)], G)


def level(x, R, V_bar, d, w, nmax, lmax, b, G=1.0, host_components=()):
    """Pull-back of a(x, R) along d at one level.  Returns (dx, dR, dth):
    the increments of xbar (n, 3), of Rbar (3,), and of the host-parameter
    adjoint (n_host, 2) = (d/dGM_c, d/da_c); V_bar is the centre's velocity
    adjoint at this level."""
    A = coeffs(x, nmax, lmax, b)
    dx = jvp_field(x, A, d, nmax, lmax, b, G)                       # own position
    AJ = jvp_coeffs(x, d, nmax, lmax, b)
    dx += x[:, 3:4] * field(x, AJ, nmax, lmax, b, G)[:, :3]         # through the coefficients
    dR = np.zeros(3)
    dth = np.zeros((len(host_components), 2))
    if host_components:
        host = host_struct(host_components, G)
        P = R[None, :3] + x[:, :3]
        TP = tidal_tensor(host, P)
        TR = tidal_tensor(host, R[:3])[0]
        dx += np.einsum("kij,kj->ki", TP, d)
        dR = np.einsum("kij,kj->i", TP - TR[None], d) + w * TR @ V_bar
        for c, comp in enumerate(host_components):
            one = _single(comp, G, M=1.0 / G)                        # the component with GM = 1
            dth[c, 0] = np.sum(d * tidal_many(one, R, x)) + w * host_accel_many(one, R[:3])[0] @ V_bar

            def D(a):
                hc = _single(comp, G, a=a)
                return np.sum(d * tidal_many(hc, R, x)) + w * host_accel_many(hc, R[:3])[0] @ V_bar

            da = 1e-3 * comp[2]
            dth[c, 1] = sum(cf * D(comp[2] + j * da) for j, cf in _FD) / (12.0 * da)
    return dx, dR, dth


def forward(pos0, vel0, com0, nmax, lmax, b, dt, nsteps, G=1.0, host_components=()):
    """States x_t, com_t for t = 0..nsteps of the oracle's leapfrog, and the
    final (pos, vel, com)."""
    host = host_struct(host_components, G) if host_components else None
    com = np.asarray(com0, dtype=np.float64).copy()
    A = coeffs(pos0, nmax, lmax, b)
    acc = forces(pos0, A, nmax, lmax, b, G, com=com if host else None, host=host)
    X, C = [np.array(pos0, dtype=np.float64)], [com.copy()]
    p, v = X[0].copy(), np.array(vel0, dtype=np.float64)
    for _ in range(nsteps):
        p, v, acc, com, _ = step(p, v, acc, nmax, lmax, b, dt, 1, G, com=com if host else None, host=host)
        X.append(p.copy())
        C.append(com.copy())
    return X, C, p, v, com


def sweep(X, C, xbar, vbar, combar, nmax, lmax, b, dt, G=1.0, host_components=()):
    """Reverse sweep over the stored states.  xbar, vbar (n, 3) and combar (6,)
    are dL/d of the final state; returns dL/d(x_0, v_0, com_0) and the host
    parameters (n_host, 2) = (d/dGM_c, d/da_c)."""
    T = len(X) - 1
    h = 0.5 * dt
    xbar = np.array(xbar, dtype=np.float64)[:, :3].copy()
    vbar = np.array(vbar, dtype=np.float64)[:, :3].copy()
    Rbar = np.array(combar[:3], dtype=np.float64)
    Vbar = np.array(combar[3:6], dtype=np.float64)
    th = np.zeros((len(host_components), 2))
    for t in range(T, -1, -1):
        w = h if t in (0, T) else dt
        d = w * vbar
        dx, dR, dth = level(X[t], C[t], Vbar, d, w, nmax, lmax, b, G, host_components)
        xbar += dx
        Rbar += dR
        th += dth
        if t > 0:
            vbar += dt * xbar
            Vbar += dt * Rbar
    return xbar, vbar, np.concatenate([Rbar, Vbar]), th
