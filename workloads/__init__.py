"""Seeded synthetic inputs for the SCF gravity step.

This module is shared by the tests, the benchmark and the oracle scripts.  It
holds input generators only — particle samplers, unit conversions and host
parameter presets — and none of the method's arithmetic (no basis functions,
coefficients, forces or integrators).

Units: every cluster is expressed in Henon units (G = M = 1, E = -1/4, so the
virial radius is 1).  Host potentials are converted into the same units.

Samplers:
* :func:`plummer`  — Aarseth, Henon & Wielen (1974) Plummer sphere.
* :func:`king`     — King (1966) lowered isothermal model of depth W0, by
  integrating its Poisson equation and rejection-sampling speeds from the DF.
  (The paper's clusters come from COSMIC King models, Sec. 3; COSMIC is not
  available, so this sampler stands in for it.)
* :func:`hernquist_positions` — Hernquist (1990) sphere (inverse CDF).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

# Physical constants (App. B: 1 km/s = 1.022712165045695 pc/Myr).
KMS_TO_PC_MYR = 1.022712165045695
G_PC_KMS2_MSUN = 4.30091727e-3                       # pc (km/s)^2 / Msun
G_PC3_MSUN_MYR2 = G_PC_KMS2_MSUN * KMS_TO_PC_MYR**2   # pc^3 / (Msun Myr^2)
H0_KMS_MPC = 70.0

HOST_HERNQUIST = 1
HOST_NFW = 2
HOST_MN = 3
HOST_POWCUT = 4      # power-law bulge with an exponential cut-off (b holds the index alpha)

_HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------
# particle samplers (all return float64 arrays in Henon units)
# --------------------------------------------------------------------------
def _isotropic(rng, n):
    u = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2 * np.pi, n)
    s = np.sqrt(1 - u * u)
    return np.stack([s * np.cos(ph), s * np.sin(ph), u], axis=1)


def _centre(pos, vel, m):
    pos = pos - (m[:, None] * pos).sum(0) / m.sum()
    vel = vel - (m[:, None] * vel).sum(0) / m.sum()
    return pos, vel


def _pack(pos, vel, m):
    p4 = np.zeros((len(m), 4))
    p4[:, :3] = pos
    p4[:, 3] = m
    v4 = np.zeros((len(m), 4))
    v4[:, :3] = vel
    return p4, v4


def plummer(n: int, seed: int, rmax_over_a: float = 22.8):
    """Equal-mass Plummer sphere in Henon units (scale a = 3 pi / 16).

    Returns ``(pos (n,4) = x,y,z,m ; vel (n,4))``."""
    rng = np.random.default_rng(seed)
    a = 3 * np.pi / 16
    r = np.empty(n)
    k = 0
    while k < n:
        x = rng.uniform(0, 1, n)
        rr = 1.0 / np.sqrt(np.maximum(x, 1e-300) ** (-2.0 / 3.0) - 1.0)
        rr = rr[rr < rmax_over_a]
        take = min(n - k, rr.size)
        r[k:k + take] = rr[:take]
        k += take
    pos = _isotropic(rng, n) * (a * r)[:, None]
    # speeds: q = v / v_esc from g(q) = q^2 (1 - q^2)^(7/2) by rejection
    q = np.empty(n)
    k = 0
    while k < n:
        x = rng.uniform(0, 1, 2 * n)
        y = rng.uniform(0, 0.1, 2 * n)
        ok = x[y < x * x * (1 - x * x) ** 3.5]
        take = min(n - k, ok.size)
        q[k:k + take] = ok[:take]
        k += take
    vesc = np.sqrt(2.0) * (1.0 + r * r) ** (-0.25) / np.sqrt(a)
    vel = _isotropic(rng, n) * (q * vesc)[:, None]
    m = np.full(n, 1.0 / n)
    pos, vel = _centre(pos, vel, m)
    return _pack(pos, vel, m)


def hernquist_positions(n: int, b: float, seed: int, rmax_over_b: float = 1e4):
    """Equal-mass Hernquist sphere of total mass 1 and scale ``b`` (positions only).

    M(<r) = s^2/(1+s)^2, so s = sqrt(u)/(1 - sqrt(u)) for u ~ U(0,1)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1, n)
    su = np.sqrt(u)
    s = np.minimum(su / (1 - su), rmax_over_b)
    pos = _isotropic(rng, n) * (b * s)[:, None]
    p4 = np.zeros((n, 4))
    p4[:, :3] = pos
    p4[:, 3] = 1.0 / n
    return p4


@dataclass
class KingModel:
    W0: float
    r: np.ndarray          # radius in King units (core radius r0 = 1)
    W: np.ndarray          # dimensionless potential depth W(r) >= 0
    M: np.ndarray          # enclosed mass (King units, G = 1 scaled by 9/(4 pi) convention below)
    rt: float


def _king_rho(W):
    W = np.maximum(W, 0.0)
    from scipy.special import erf
    return np.exp(W) * erf(np.sqrt(W)) - np.sqrt(4 * W / np.pi) * (1 + 2 * W / 3)


def king_model(W0: float) -> KingModel:
    """Integrate the King (1966) Poisson equation W'' + 2 W'/r = -9 rho(W)/rho(W0)."""
    from scipy.integrate import solve_ivp
    rho0 = _king_rho(W0)

    def rhs(r, y):
        W, dW = y
        return [dW, -9.0 * _king_rho(W) / rho0 - 2.0 * dW / r]

    r0 = 1e-6
    y0 = [W0 - 1.5 * r0 * r0, -3.0 * r0]

    def hit(r, y):
        return y[0]
    hit.terminal = True
    hit.direction = -1
    sol = solve_ivp(rhs, [r0, 1e4], y0, events=hit, rtol=1e-11, atol=1e-13, dense_output=True, max_step=0.01)
    rt = float(sol.t_events[0][0])
    r = np.concatenate([[0.0], np.geomspace(r0, rt, 20000)])
    W = np.concatenate([[W0], sol.sol(r[1:])[0]])
    dW = np.concatenate([[0.0], sol.sol(r[1:])[1]])
    W = np.maximum(W, 0.0)
    # Poisson: (1/r^2)(r^2 W')' = -9 rho/rho0 => M(r) proportional to -r^2 W'
    M = -r * r * dW
    M[-1] = max(M[-1], M[-2])
    return KingModel(W0=W0, r=r, W=W, M=M, rt=rt)


def king(n: int, W0: float, seed: int):
    """Equal-mass King (1966) model of depth W0 in Henon units.

    Positions from the enclosed-mass profile, speeds from the lowered
    isothermal DF f(eps) ~ exp(eps) - 1 (eps = W - v^2/2 in units of sigma^2).
    The sample is then scaled so that G = M = 1 and the model's total energy
    is -1/4.  Returns ``(pos (n,4), vel (n,4))``."""
    km = king_model(W0)
    rng = np.random.default_rng(seed)
    Mt = km.M[-1]
    u = rng.uniform(0, 1, n) * Mt
    r = np.interp(u, km.M, km.r)
    Wr = np.interp(r, km.r, km.W)
    # speed v in units of sigma: p(v) ~ v^2 (exp(W - v^2/2) - 1), 0 <= v <= sqrt(2W)
    v = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        W = Wr[todo]
        vmax = np.sqrt(2 * W)
        x = rng.uniform(0, 1, todo.size) * vmax
        # envelope: p(v) <= vmax^2 (exp(W) - 1)
        p = x * x * (np.exp(W - 0.5 * x * x) - 1.0)
        env = vmax * vmax * (np.exp(W) - 1.0)
        ok = rng.uniform(0, 1, todo.size) * env <= p
        v[todo[ok]] = x[ok]
        todo = todo[~ok]
    pos = _isotropic(rng, n) * r[:, None]
    vel = _isotropic(rng, n) * v[:, None]
    # Model units: r0 = 1, sigma = 1 and G = 1, so the Poisson equation above
    # fixes 4 pi rho0 = 9 and the enclosed mass is M(r) = -r^2 W'(r) (km.M).
    # Potential energy U = -int M dM / r over the model.
    M = km.M
    rm = 0.5 * (km.r[1:] + km.r[:-1])
    U = -np.sum(0.5 * (M[1:] + M[:-1]) * np.diff(M) / np.maximum(rm, 1e-30))
    Mt = M[-1]
    # Henon units: mass / Mt, length / L, G = 1, so U_H = U L / Mt^2; an
    # equilibrium model has E = U/2, and E = -1/4 needs U_H = -1/2.
    L = Mt * Mt / (2.0 * abs(U))
    vscale = math.sqrt(L / Mt)      # speeds scale as sqrt(G M / length)
    pos = pos / L
    vel = vel * vscale
    m = np.full(n, 1.0 / n)
    pos, vel = _centre(pos, vel, m)
    return _pack(pos, vel, m)


def half_mass_radius(pos4) -> float:
    r = np.sqrt((pos4[:, :3] ** 2).sum(1))
    order = np.argsort(r)
    cm = np.cumsum(pos4[order, 3])
    return float(r[order][np.searchsorted(cm, 0.5 * cm[-1])])


def basis_scale(r_half: float, alpha: float = 1.0) -> float:
    """Basis scale b of the lowest-order density of the radial family (Eq. 4)
    with the same half-mass radius: its enclosed mass is (t/(1+t))^(alpha+1),
    t = (r/b)^(1/alpha), so b = r_h (2^(1/(alpha+1)) - 1)^alpha -- a Hernquist
    sphere's r_h = (1 + sqrt 2) b at alpha = 1, a Plummer sphere's scale at
    alpha = 1/2.  The paper retunes b at each complete refresh (Sec. 2)."""
    if alpha == 1.0:
        return r_half / (1.0 + math.sqrt(2.0))
    return r_half * (2.0 ** (1.0 / (alpha + 1.0)) - 1.0) ** alpha


# --------------------------------------------------------------------------
# symmetric inputs for the coefficient pins
# --------------------------------------------------------------------------
def mirror8(pos4):
    """Each particle with its 8 reflections (+-x, +-y, +-z); mass split evenly."""
    out = []
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                q = pos4.copy()
                q[:, 0] *= sx
                q[:, 1] *= sy
                q[:, 2] *= sz
                q[:, 3] /= 8
                out.append(q)
    return np.concatenate(out)


def rotate_copies(pos4, K: int):
    """K copies rotated about z by 2 pi j / K; mass split evenly."""
    out = []
    for j in range(K):
        c, s = math.cos(2 * math.pi * j / K), math.sin(2 * math.pi * j / K)
        q = pos4.copy()
        q[:, 0] = c * pos4[:, 0] - s * pos4[:, 1]
        q[:, 1] = s * pos4[:, 0] + c * pos4[:, 1]
        q[:, 3] /= K
        out.append(q)
    return np.concatenate(out)


# --------------------------------------------------------------------------
# units and host presets
# --------------------------------------------------------------------------
@dataclass
class Units:
    """Henon units of a cluster of mass ``M_msun`` and virial radius ``rv_pc``."""
    M_msun: float
    rv_pc: float

    @property
    def T_myr(self) -> float:
        return math.sqrt(self.rv_pc**3 / (G_PC3_MSUN_MYR2 * self.M_msun))

    @property
    def V_pc_myr(self) -> float:
        return self.rv_pc / self.T_myr

    def length(self, pc):
        return pc / self.rv_pc

    def mass(self, msun):
        return msun / self.M_msun

    def velocity_kms(self, kms):
        return kms * KMS_TO_PC_MYR / self.V_pc_myr


def nfw_scale_mass(Mvir_msun: float, rs_pc: float, H0=H0_KMS_MPC, overdensity=200.0) -> float:
    """Scale mass M_NFW of App. A from a virial mass: rho_crit = 3 H0^2/(8 pi G),
    M_vir = (4 pi/3) 200 rho_crit R_vir^3, c = R_vir/r_s, M_NFW = M_vir/g(c)."""
    H = H0 * 1e-6  # km/s/pc
    rho_crit = 3 * H * H / (8 * math.pi * G_PC_KMS2_MSUN)
    Rvir = (3 * Mvir_msun / (4 * math.pi * overdensity * rho_crit)) ** (1 / 3)
    c = Rvir / rs_pc
    g = math.log1p(c) - c / (1 + c)
    return Mvir_msun / g


def galaxy_host_physical():
    """The host of the multi-cluster workloads: NFW halo (M_vir = 1e12 Msun,
    r_s = 20 kpc), Miyamoto-Nagai disk (6.8e10 Msun, a = 3 kpc, b = 0.28 kpc),
    Hernquist bulge (5e9 Msun, a = 0.5 kpc).  Returns (kind, M_msun, a_pc, b_pc)."""
    return [
        (HOST_NFW, nfw_scale_mass(1e12, 20e3), 20e3, 0.0),
        (HOST_MN, 6.8e10, 3e3, 280.0),
        (HOST_HERNQUIST, 5e9, 500.0, 0.0),
    ]


def mw2022_physical():
    """MilkyWayPotential2022 as tabulated in App. A (kind, M_msun, a_kpc, b_kpc);
    lengths in kpc for use with G in kpc (km/s)^2 / Msun."""
    return [
        (HOST_HERNQUIST, 1.8142e9, 68.8867e-3, 0.0),
        (HOST_HERNQUIST, 5e9, 1.0, 0.0),
        (HOST_MN, 7.872306998700792e9, 1.5259431976529216, 0.20663742603550295),
        (HOST_MN, -2.7562522194433154e11, 6.782764436261113, 0.20663742603550295),
        (HOST_MN, 3.206184188979487e11, 5.894799616164217, 0.20663742603550295),
        (HOST_NFW, 5.5427e11, 15.626, 0.0),
    ]


# MWPotential2014 (App. A "MWPotential2014" subsection and its table): the
# components contribute f_b, f_d, f_h of the centripetal acceleration
# f_cent = G M_s / r0^2 of a circular disk orbit at r0 = 8 kpc.
MW2014_R0_KPC = 8.0
MW2014_MS = 9.00273072e10         # scale mass M_s, Msun
MW2014_F_CENT_PC_MYR2 = 6.32793804994


def mw2014_physical():
    """MWPotential2014 recast as in App. A (kind, M_msun, a_kpc, b): the
    exponentially cut-off power-law bulge (alpha = 1.8, r_c = 1.9 kpc; b holds
    alpha), the Miyamoto-Nagai disk (a = 3 kpc, b = 0.28 kpc) and the NFW halo
    (R_s = 16 kpc, scale mass), with the masses that give each component its
    fraction (0.05, 0.6, 0.35) of f_cent at r0 = 8 kpc:
    M_b = f_b M_s Gamma(s)/gamma(s, (r0/r_c)^2), s = (3 - alpha)/2;
    M_d = f_d M_s (r0^2 + (a + b)^2)^(3/2) / r0^3;  M_h = f_h M_s / g(r0/R_s),
    g(u) = ln(1 + u) - u/(1 + u).  Lengths in kpc for G in kpc (km/s)^2/Msun."""
    from scipy.special import gammainc      # regularised lower incomplete gamma
    r0, alpha, rc, a, b, Rs = MW2014_R0_KPC, 1.8, 1.9, 3.0, 0.28, 16.0
    s = 0.5 * (3.0 - alpha)
    Mb = 0.05 * MW2014_MS / gammainc(s, (r0 / rc) ** 2)
    Md = 0.6 * MW2014_MS * (r0 * r0 + (a + b) ** 2) ** 1.5 / r0 ** 3
    u = r0 / Rs
    Mh = 0.35 * MW2014_MS / (math.log1p(u) - u / (1.0 + u))
    return [(HOST_POWCUT, Mb, rc, alpha), (HOST_MN, Md, a, b), (HOST_NFW, Mh, Rs, 0.0)]


def host_in_units(components_phys, units: Units):
    """Host components in the cluster's Henon units (b is a length except for
    the cut-off bulge, whose b is its dimensionless power-law index)."""
    return [(k, units.mass(M), units.length(a), b if k == HOST_POWCUT else units.length(b))
            for (k, M, a, b) in components_phys]


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    pos: np.ndarray                 # (N, 4) x, y, z, m   (cluster frame, Henon units)
    vel: np.ndarray                 # (N, 4)
    nmax: int
    lmax: int
    b: float
    dt: float
    nsteps: int
    host: list = field(default_factory=list)   # [(kind, M, a, b)] in Henon units, G = 1
    com: np.ndarray = field(default_factory=lambda: np.zeros(6))
    units: Units | None = None
    offsets: np.ndarray | None = None          # progenitor boundaries (batched workloads)
    b_per_prog: np.ndarray | None = None
    com_per_prog: np.ndarray | None = None
    alpha: float = 1.0                         # exponent of the radial family (Eq. 4)

    @property
    def n(self) -> int:
        return self.pos.shape[0]


def _orbit_ics():
    path = os.path.join(_HERE, "orbit_ics.json")
    with open(path) as f:
        return json.load(f)


def _com_from_orbit(orbit, units: Units):
    R = np.array(orbit["R_kpc"]) * 1e3 / units.rv_pc
    V = np.array([units.velocity_kms(v) for v in orbit["V_kms"]])
    return np.concatenate([R, V])


# The validation orbits of Table A3 in MWPotential2014: position [kpc], velocity [km/s].
MW2014_ORBITS = {
    "circular_5kpc": ([5.0, 0.0, 0.0], [0.0, 225.55900747, 0.0]),
    "circular_20kpc": ([20.0, 0.0, 0.0], [0.0, 197.61111164, 0.0]),
    "eccentric": ([4.04231677, 0.0, 19.58670971], [0.0, 81.49205330, 0.0]),
}


def mw2014_validation(orbit: str = "circular_5kpc", n: int = 50_000, seed: int = 80, nsteps: int = 1000) -> Workload:
    """The paper's validation progenitor (Sec. 3: King W0 = 5, 1e5 Msun,
    r_h = 10 pc; N = 5e4 in the validation runs) on one of the three
    validation orbits of Table A3 in MWPotential2014 (App. A), Henon units of
    the cluster; nmax = 10, lmax = 5, dt = 0.01."""
    pos, vel = king(n, 5.0, seed)
    rh = half_mass_radius(pos)
    units = Units(1e5, 10.0 / rh)
    comps = [(k, M, a * 1e3, b if k == HOST_POWCUT else b * 1e3) for (k, M, a, b) in mw2014_physical()]
    host = host_in_units(comps, units)
    R, V = MW2014_ORBITS[orbit]
    com = np.concatenate([np.array(R) * 1e3 / units.rv_pc, [units.velocity_kms(v) for v in V]])
    return Workload(f"king5_n{n}_mw2014_{orbit}", pos, vel, 10, 5, basis_scale(rh), 0.01, nsteps, host, com, units)


def plummer_isolated(n: int = 4096, seed: int = 1) -> Workload:
    """Isolated Plummer sphere, nmax = 10, lmax = 6, dt = 0.01, 100 steps, no host."""
    pos, vel = plummer(n, seed)
    return Workload("plummer_n4096_isolated", pos, vel, 10, 6, basis_scale(half_mass_radius(pos)), 0.01, 100)


def king_circular(n: int = 100_000, seed: int = 2, nsteps: int = 2000) -> Workload:
    """King W0 = 6 cluster (1e5 Msun, r_h = 3 pc) on a circular orbit at R = 8 kpc
    in the NFW + MN + Hernquist host; nmax = 20, lmax = 8."""
    pos, vel = king(n, 6.0, seed)
    rh = half_mass_radius(pos)
    units = Units(1e5, 3.0 / rh)
    host = host_in_units(galaxy_host_physical(), units)
    com = _com_from_orbit(_orbit_ics()["circular_8kpc"], units)
    return Workload(f"king_w6_n{n}_circular8kpc", pos, vel, 20, 8, basis_scale(rh), 0.01, nsteps, host, com, units)


def plummer_eccentric(n: int = 1_000_000, seed: int = 3, nsteps: int = 2000) -> Workload:
    """Plummer cluster (2e5 Msun, r_h = 4 pc) on the 5-20 kpc eccentric orbit;
    nmax = 20, lmax = 10."""
    pos, vel = plummer(n, seed)
    rh = half_mass_radius(pos)
    units = Units(2e5, 4.0 / rh)
    host = host_in_units(galaxy_host_physical(), units)
    com = _com_from_orbit(_orbit_ics()["eccentric_5_20kpc"], units)
    return Workload(f"plummer_n{n}_eccentric", pos, vel, 20, 10, basis_scale(rh), 0.01, nsteps, host, com, units)


def plummer_eccentric_cb(n: int = 1_000_000, seed: int = 3, nsteps: int = 2000) -> Workload:
    """The same Plummer cluster and orbit expanded in the alpha = 1/2 member of
    the radial family (Eq. 4; the Clutton-Brock basis, whose lowest-order pair
    is the Plummer sphere), b = the sample's Plummer scale; nmax = 20, lmax = 10."""
    wl = plummer_eccentric(n, seed, nsteps)
    rh = half_mass_radius(wl.pos)
    wl.name = f"plummer_n{n}_eccentric_alpha0.5"
    wl.alpha = 0.5
    wl.b = basis_scale(rh, 0.5)
    return wl


def plummer_stream(n: int = 100_000, seed: int = 6, nsteps: int = 6000) -> Workload:
    """Stream-forming run: a tidally filling Plummer cluster (2e5 Msun, r_h =
    20 pc, so about a tenth of its mass lies beyond the Jacobi radius at the
    5 kpc pericentre) on the 5-20 kpc eccentric orbit, starting at apocentre;
    nmax = 10, lmax = 5 (the paper's fiducial stream model), dt = 0.01."""
    pos, vel = plummer(n, seed)
    rh = half_mass_radius(pos)
    units = Units(2e5, 20.0 / rh)
    host = host_in_units(galaxy_host_physical(), units)
    com = _com_from_orbit(_orbit_ics()["eccentric_5_20kpc"], units)
    return Workload(f"plummer_rh20_n{n}_stream", pos, vel, 10, 5, basis_scale(rh), 0.01, nsteps, host, com, units)


def king_eccentric(n: int = 100_000, seed: int = 5, nsteps: int = 500) -> Workload:
    """The differentiable run: King W0 = 6 cluster (1e5 Msun, r_h = 3 pc) on
    the 5-20 kpc eccentric orbit in the NFW + MN + Hernquist host; nmax = 20,
    lmax = 8, dt = 0.01, 500 steps (checkpointed every 50 by the caller)."""
    pos, vel = king(n, 6.0, seed)
    rh = half_mass_radius(pos)
    units = Units(1e5, 3.0 / rh)
    host = host_in_units(galaxy_host_physical(), units)
    com = _com_from_orbit(_orbit_ics()["eccentric_5_20kpc"], units)
    return Workload(f"king_w6_n{n}_eccentric", pos, vel, 20, 8, basis_scale(rh), 0.01, nsteps, host, com, units)


def reference_track(R, V, n_points: int = 256, half_length: float = 50.0, sigma: float = 2.0, seed: int = 50):
    """Seeded synthetic reference track for the stream-track loss: ``n_points``
    points along the direction of motion V through R, spanning
    +-``half_length`` (length units), each displaced by seeded Gaussian
    offsets of width ``sigma`` perpendicular to V.  Returns (n_points, 3)."""
    rng = np.random.default_rng(seed)
    R = np.asarray(R, dtype=np.float64)[:3]
    t = np.asarray(V, dtype=np.float64)[:3]
    t = t / np.linalg.norm(t)
    e1 = np.cross(t, [0.0, 0.0, 1.0])
    if np.linalg.norm(e1) < 1e-8:
        e1 = np.cross(t, [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(t, e1)
    s = np.linspace(-half_length, half_length, n_points)
    off = rng.normal(0.0, sigma, size=(n_points, 2))
    return R[None] + s[:, None] * t[None] + off[:, :1] * e1[None] + off[:, 1:] * e2[None]


# Table A3: initial positions (kpc) and velocities (km/s) of Orbits 0-9 in
# the host frame of MilkyWayPotential2022.
PAPER_ORBITS_A3 = [
    (-8.26114834, 4.31927900, -6.25723160, -74.46836937, 14.72551502, -137.10220626),
    (6.65417846, -6.77625060, -6.89249860, 131.88487388, -54.38017150, 4.34224828),
    (7.90677816, 19.00502796, -7.29228303, -38.33588368, -66.85081211, 111.04181836),
    (9.73591969, 8.80768907, 0.73284850, -59.71003689, 91.24008328, -39.80505238),
    (-7.75511077, 6.32704860, 23.10803486, 1.54688377, -69.83998228, 18.65659155),
    (-9.14496546, -2.86774379, 4.55846674, 25.93998870, -146.50950043, -246.21359733),
    (-20.83691936, -15.77790335, -20.69545845, -13.04785291, -35.40337893, -181.82805977),
    (-18.82672221, 27.56963834, 27.40177203, 25.20438668, -112.02637209, 29.55096514),
    (22.45554180, 35.25629955, -2.75494642, -10.73021364, -7.94047313, -128.19547342),
    (-23.95107022, 9.24097888, -14.06736155, 27.31176344, -167.54952847, -128.11428538),
]


def paper_orbits(n_per: int = 20_000, seed: int = 60, nsteps: int = 4000) -> Workload:
    """The paper's stream progenitors on its ten orbits: King W0 = 5 clusters of
    1e5 Msun and r_h = 10 pc (Sec. 3), one per orbit of Table A3, in
    MilkyWayPotential2022 (Table A2); nmax = 10, lmax = 5 (the paper's
    fiducial stream model), dt = 0.01.  The paper samples N = 5e4 or 2e5 stars
    per cluster; ``n_per`` sets it here.  All clusters share one unit system."""
    ref = king(20000, 5.0, seed)
    units = Units(1e5, 10.0 / half_mass_radius(ref[0]))
    host = host_in_units([(k, M, a * 1e3, b * 1e3) for (k, M, a, b) in mw2022_physical()], units)
    pos_l, vel_l, bs, coms = [], [], [], []
    for p, ic in enumerate(PAPER_ORBITS_A3):
        pos, vel = king(int(n_per), 5.0, seed + 1 + p)
        lam = (10.0 / units.rv_pc) / half_mass_radius(pos)     # exactly r_h = 10 pc
        pos[:, :3] *= lam
        vel[:, :3] /= math.sqrt(lam)
        pos_l.append(pos)
        vel_l.append(vel)
        bs.append(basis_scale(half_mass_radius(pos)))
        coms.append(_com_from_orbit({"R_kpc": ic[:3], "V_kms": ic[3:]}, units))
    offsets = np.concatenate([[0], np.cumsum([len(q) for q in pos_l])]).astype(np.int64)
    return Workload(f"paper_orbits10_king5_n{n_per}", np.concatenate(pos_l), np.concatenate(vel_l), 10, 5,
                    float(bs[0]), 0.01, nsteps, host, coms[0], units, offsets, np.array(bs), np.array(coms))


def progenitor_batch(n_prog: int = 10, seed: int = 40, n_range=(2e4, 5e5), nsteps: int = 2000,
                     scale: float = 1.0) -> Workload:
    """Batch of progenitors with N log-uniform in ``n_range`` (times ``scale``)
    and W0 ~ U(4, 8), each on its own seeded orbit; nmax = 20, lmax = 10.
    All clusters share the unit system of a 1e5 Msun, r_h = 3 pc King W0 = 6
    cluster (so one dt and one host serve the batch)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), n_prog)) * scale
    ns = np.maximum(ns.astype(np.int64), 1)
    w0s = rng.uniform(4.0, 8.0, n_prog)
    ref = king(20000, 6.0, seed)
    units = Units(1e5, 3.0 / half_mass_radius(ref[0]))
    host = host_in_units(galaxy_host_physical(), units)
    orbits = _orbit_ics()["batch"]
    pos_l, vel_l, bs, coms = [], [], [], []
    for p in range(n_prog):
        pos, vel = king(int(ns[p]), float(w0s[p]), seed + 1 + p)
        rh_h = half_mass_radius(pos)
        # every cluster has M = 1e5 Msun and r_h = 3 pc: rescale to the shared units
        lam = (3.0 / units.rv_pc) / rh_h
        pos[:, :3] *= lam
        vel[:, :3] /= math.sqrt(lam)
        pos_l.append(pos)
        vel_l.append(vel)
        bs.append(basis_scale(half_mass_radius(pos)))
        coms.append(_com_from_orbit(orbits[p % len(orbits)], units))
    offsets = np.concatenate([[0], np.cumsum([len(p) for p in pos_l])]).astype(np.int64)
    wl = Workload(f"batch{n_prog}_king", np.concatenate(pos_l), np.concatenate(vel_l), 20, 10, float(bs[0]), 0.01,
                  nsteps, host, coms[0], units, offsets, np.array(bs), np.array(coms))
    return wl
