"""Seeded synthetic workloads for the grey IMEX radiation step.

This module only builds inputs: a problem description (a plain dict) and the
initial state.  It holds none of the step's arithmetic and imports neither the
CUDA library nor the CPU oracle, so both can be fed the same bytes.

State arrays have shape (10, nz, ny, nx), float64, field-major with x fastest;
the field order is ``FIELDS``.  F is the physical lab-frame radiation flux and
``kappa`` the specific opacity (chi = kappa * rho).  Code units: a_r = 1,
k_B/mu = 1.

The paper has no public dataset; the workloads restate the problem classes of
its Sec. 5 (static diffusion of a Gaussian pulse, the streaming / diffusion /
dynamic-diffusion regimes, a uniformly advected medium) on synthetic fields:
  * static_diffusion_1d -- Gaussian temperature pulse, rho = 1, gas at rest,
    tau_cell = 10, reflecting walls, chat = c;
  * regime_sweep_1d -- three bands with tau_cell = 1e-3, 1, 1e3 and a Gaussian
    pulse in each, uniform v = 1e-3 c, chat = c/10, periodic;
  * turbulent_box_3d -- log-normal density (k^-4 Gaussian random field,
    sigma_ln rho = 1), kappa proportional to rho with tau_cell clipped to
    [1e-3, 1e3], log-uniform T over one decade, k^-4 random velocity with rms
    Mach 1, chat = 30 max|v|, c = 10 chat.
Radiation starts in comoving equilibrium with the gas (Sec. 5.5):
E = a T^4 (1 + 4/3 beta^2) for v/c order 2 (a T^4 for order 1), F = 4/3 v a T^4.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("rho", "mx", "my", "mz", "egas", "erad", "fx", "fy", "fz", "kappa")
NFIELD = len(FIELDS)
F_RHO, F_MX, F_MY, F_MZ, F_EGAS, F_ERAD, F_FX, F_FY, F_FZ, F_KAPPA = range(10)


def gas_state(prob: dict, rho, v, p, kappa=0.0) -> np.ndarray:
    """State of a gas given by density, velocity (3, nz, ny, nx) and pressure,
    with radiation in comoving equilibrium at the gas temperature
    T = p / (rho kB_over_mu) (ideal gas) and specific opacity kappa."""
    kB = prob.get("kB_over_mu", 1.0)
    rho = np.asarray(rho, dtype=np.float64)
    T = np.asarray(p, dtype=np.float64) / (rho * kB)
    kap = np.broadcast_to(np.asarray(kappa, dtype=np.float64), rho.shape)
    return equilibrium_state(prob, rho, T, v, kap)


def riemann_problem_1d(n: int, left, right, x0: float = 0.5, gamma: float = 1.4,
                       bc: str = "reflect", **kw):
    """Shock-tube initial state on [0, 1]: primitive states left = (rho, u, p)
    for x < x0 and right beyond; no radiation coupling (kappa = 0).  Returns
    (problem, state)."""
    prob = base_problem(1, [n], [1.0 / n], gamma=gamma, bc=bc, **kw)
    x = (np.arange(n) + 0.5) / n
    sh = (1, 1, n)
    L = x < x0
    rho = np.where(L, left[0], right[0]).reshape(sh)
    u = np.where(L, left[1], right[1]).reshape(sh)
    pr = np.where(L, left[2], right[2]).reshape(sh)
    v = np.zeros((3,) + sh)
    v[0] = u
    return prob, gas_state(prob, rho, v, pr)


def base_problem(ndim, n, dx, **kw) -> dict:
    """Problem dict with the library defaults filled in."""
    prob = {
        "ndim": int(ndim),
        "n": [int(v) for v in n] + [1] * (3 - len(n)),
        "dx": [float(v) for v in dx] + [1.0] * (3 - len(dx)),
        "bc": "periodic",
        "gamma": 5.0 / 3.0,
        "c": 1.0,
        "chat": 1.0,
        "a_rad": 1.0,
        "kB_over_mu": 1.0,
        "cfl": 0.4,
        "closure": "m1",
        "vc_order": 2,
        "hll_mode": "tau",
        "newton_rtol": 1e-13,
        "outer_rtol": 1e-13,
        "newton_max_iter": 64,
        "outer_max_iter": 32,
    }
    prob.update(kw)
    return prob


def shape_of(prob: dict):
    n = prob["n"]
    return (NFIELD, n[2], n[1], n[0])


def equilibrium_state(prob: dict, rho, T, v, kappa) -> np.ndarray:
    """Initial state with radiation in comoving equilibrium with the gas.

    rho, T, kappa: arrays of shape (nz, ny, nx); v: (3, nz, ny, nx)."""
    a = prob.get("a_rad", 1.0)
    c = prob["c"]
    cv = prob.get("kB_over_mu", 1.0) / (prob["gamma"] - 1.0)
    rho = np.asarray(rho, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    beta2 = (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) / c ** 2
    aT4 = a * T ** 4
    U = np.zeros(shape_of(prob), dtype=np.float64)
    U[F_RHO] = rho
    for d in range(3):
        U[F_MX + d] = rho * v[d]
        U[F_FX + d] = (4.0 / 3.0) * v[d] * aT4
    U[F_EGAS] = rho * cv * T + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    if prob.get("vc_order", 2) == 2:
        U[F_ERAD] = aT4 * (1.0 + (4.0 / 3.0) * beta2)
    else:
        U[F_ERAD] = aT4
    U[F_KAPPA] = kappa
    return np.ascontiguousarray(U)


def cell_centres(prob: dict):
    """Cell-centre coordinates on [0, n dx) per axis, broadcastable to (nz, ny, nx)."""
    n, dx = prob["n"], prob["dx"]
    x = (np.arange(n[0]) + 0.5) * dx[0]
    y = (np.arange(n[1]) + 0.5) * dx[1]
    z = (np.arange(n[2]) + 0.5) * dx[2]
    return x[None, None, :], y[None, :, None], z[:, None, None]


def gaussian_random_field(shape, slope: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field with power
    spectrum P(k) ~ k^slope (k = 0 mode removed)."""
    white = rng.standard_normal(shape)
    fk = np.fft.rfftn(white)
    ks = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    grids = np.meshgrid(*ks, indexing="ij", sparse=True)
    k2 = sum(g * g for g in grids)
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P) = k^(slope/2)
    field = np.fft.irfftn(fk * amp, s=shape, axes=tuple(range(len(shape))))
    field -= field.mean()
    sd = field.std()
    return field / sd if sd > 0 else field


# ---------------------------------------------------------------- workloads

def static_diffusion_1d(n: int = 256, tau_cell: float = 10.0, c: float = 1e5,
                        **kw):
    """1-D static diffusion: T = 1 + 10 exp(-((x-0.5)/0.05)^2), rho = 1, v = 0,
    E = T^4, F = 0, kappa rho dx = tau_cell, reflecting walls, chat = c.
    Returns (problem, state, nsteps)."""
    dx = 1.0 / n
    prob = base_problem(1, [n], [dx], bc="reflect", c=c, chat=c, **kw)
    x, _, _ = cell_centres(prob)
    T = 1.0 + 10.0 * np.exp(-(((x - 0.5) / 0.05) ** 2))
    T = np.broadcast_to(T, (1, 1, n))
    rho = np.ones((1, 1, n))
    v = np.zeros((3, 1, 1, n))
    kappa = np.full((1, 1, n), tau_cell / dx)
    return prob, equilibrium_state(prob, rho, T, v, kappa), 1000


def regime_sweep_1d(n: int = 4096, c: float = 1e3, beta: float = 1e-3, **kw):
    """1-D regime sweep: bands [0,1/3), [1/3,2/3), [2/3,1] with tau_cell =
    1e-3, 1, 1e3, a pulse T = 1 + exp(-((x-x_b)/0.02)^2) at each band centre,
    uniform v = beta c, chat = c/10, periodic.  Returns (problem, state, nsteps)."""
    dx = 1.0 / n
    prob = base_problem(1, [n], [dx], bc="periodic", c=c, chat=c / 10.0, **kw)
    x, _, _ = cell_centres(prob)
    x = x.reshape(-1)
    tau = np.where(x < 1.0 / 3.0, 1e-3, np.where(x < 2.0 / 3.0, 1.0, 1e3))
    T = np.ones(n)
    for xb in (1.0 / 6.0, 0.5, 5.0 / 6.0):
        T += np.exp(-(((x - xb) / 0.02) ** 2))
    rho = np.ones((1, 1, n))
    v = np.zeros((3, 1, 1, n))
    v[0] = beta * c
    kappa = (tau / dx).reshape(1, 1, n)
    return prob, equilibrium_state(prob, rho, T.reshape(1, 1, n), v, kappa), 2000


def turbulent_box_3d(n: int = 256, seed_rho: int = 3, seed_v: int = 4,
                     seed_T: int = 5, shape=None, **kw):
    """3-D bandwidth workload on a periodic n^3 box (or ``shape`` = (nx, ny, nz)).
    Returns (problem, state, nsteps)."""
    if shape is None:
        shape = (n, n, n)
    nx, ny, nz = shape
    dx = 1.0 / nx
    arr_shape = (nz, ny, nx)
    lnrho = gaussian_random_field(arr_shape, -4.0, np.random.default_rng(seed_rho))
    rho = np.exp(lnrho)
    rho /= rho.mean()
    # kappa ~ rho (chi ~ rho^2) with tau_cell(rho = 1) = 1, clipped to [1e-3, 1e3]
    tau = np.clip(rho * rho, 1e-3, 1e3)
    kappa = tau / (rho * dx)
    T = 10.0 ** np.random.default_rng(seed_T).uniform(0.0, 1.0, arr_shape)
    rng_v = np.random.default_rng(seed_v)
    u = np.stack([gaussian_random_field(arr_shape, -4.0, rng_v) for _ in range(3)])
    gamma = kw.get("gamma", 5.0 / 3.0)
    cs = np.sqrt(gamma * T)
    mach = np.sqrt((u * u).sum(axis=0)) / cs
    v = u / np.sqrt((mach * mach).mean())
    vmax = float(np.sqrt((v * v).sum(axis=0)).max())
    chat = 30.0 * vmax
    prob = base_problem(3, [nx, ny, nz], [dx, dx, dx], bc="periodic",
                        c=10.0 * chat, chat=chat, **kw)
    return prob, equilibrium_state(prob, rho, T, v, kappa), 100


def random_state(prob: dict, seed: int, tau_range=(1e-3, 1e3), T_range=(1.0, 3.0),
                 beta_max: float = 1e-3, flux_frac: float = 0.1) -> np.ndarray:
    """Generic out-of-equilibrium random state (iid per cell) for parity tests:
    log-uniform tau_cell and T, random v with |v|/c <= beta_max, E = a T_r^4
    with an independent radiation temperature, F a random fraction of c E.

    Cell-to-cell contrasts are kept moderate: with iid data, piecewise-linear
    faces and CFL 0.4 in 3-D, E can turn negative after the explicit transport
    once the contrast and |F|/cE are both large."""
    rng = np.random.default_rng(seed)
    n = prob["n"]
    sh = (n[2], n[1], n[0])
    dxmin = min(prob["dx"][: prob["ndim"]])
    rho = 10.0 ** rng.uniform(-0.5, 0.5, sh)
    tau = 10.0 ** rng.uniform(np.log10(tau_range[0]), np.log10(tau_range[1]), sh)
    kappa = tau / (rho * dxmin)
    lo, hi = np.log10(T_range[0]), np.log10(T_range[1])
    T = 10.0 ** rng.uniform(lo, hi, sh)
    Tr = 10.0 ** rng.uniform(lo, hi, sh)
    c = prob["c"]
    v = rng.uniform(-1.0, 1.0, (3,) + sh) * beta_max * c / np.sqrt(3.0)
    for d in range(prob["ndim"], 3):
        v[d] = 0.0
    U = equilibrium_state(prob, rho, T, v, kappa)
    a = prob.get("a_rad", 1.0)
    U[F_ERAD] = a * Tr ** 4
    fdir = rng.standard_normal((3,) + sh)
    for d in range(prob["ndim"], 3):
        fdir[d] = 0.0
    norm = np.sqrt((fdir * fdir).sum(axis=0)) + 1e-300
    mag = flux_frac * rng.uniform(0.0, 1.0, sh) * c * U[F_ERAD]
    for d in range(3):
        U[F_FX + d] = fdir[d] / norm * mag
    return np.ascontiguousarray(U)


def batched_problems(nprob: int = 512, seed: int = 11, c: float = 1e3,
                     chat: float = 1e2, **kw):
    """Independent problems of uneven size for the batched form: each is 1-D
    with N ~ U{64..4096} or 2-D with side ~ U{32..256} (probability 1/2 each),
    periodic on [0, 1]^d, rho = 1, log10 tau_cell iid U[-3, 3] per cell, a
    Gaussian temperature pulse T = 1 + exp(-(r/0.05)^2) at the centre, and a
    uniform velocity of random direction with |v|/c ~ U[0, 1e-3].
    Returns a list of (problem, state)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nprob):
        if rng.uniform() < 0.5:
            n = [int(rng.integers(64, 4097))]
        else:
            side = int(rng.integers(32, 257))
            n = [side, side]
        ndim = len(n)
        dx = [1.0 / v for v in n]
        prob = base_problem(ndim, n, dx, bc="periodic", c=c, chat=chat, **kw)
        sh = (1, n[1] if ndim == 2 else 1, n[0])
        x, y, _ = cell_centres(prob)
        r2 = (x - 0.5) ** 2 + ((y - 0.5) ** 2 if ndim == 2 else 0.0)
        T = np.broadcast_to(1.0 + np.exp(-r2 / 0.05 ** 2), sh)
        tau = 10.0 ** rng.uniform(-3.0, 3.0, sh)
        rho = np.ones(sh)
        kappa = tau / (rho * dx[0])
        direction = rng.standard_normal(3)
        if ndim == 1:
            direction[1:] = 0.0
        else:
            direction[2] = 0.0
        direction /= np.linalg.norm(direction)
        speed = rng.uniform(0.0, 1e-3) * c
        v = np.zeros((3,) + sh)
        for d in range(3):
            v[d] = speed * direction[d]
        out.append((prob, equilibrium_state(prob, rho, T, v, kappa)))
    return out


def pulse_inverse_problem_2d(n: int = 512, seed_chi: int = 7, seed_target: int = 8,
                             seed_T: int = 9, T_ripple: float = 0.2, c: float = 1e3,
                             nsteps: int = 200, **kw):
    """Differentiation workload: a radiation pulse on a periodic n^2 grid
    through a log-normal opacity field, with a target radiation field.

    rho = 1, gas at rest; ln chi is a k^-4 Gaussian random field (sigma = 1,
    seed ``seed_chi``) scaled so that the median tau_cell = chi dx is 1;
    T = (1 + 9 exp(-r^2 / (2 0.05^2))) (1 + T_ripple u) about the centre, with u
    iid uniform on [-1, 1] per cell (seed ``seed_T``); radiation in
    equilibrium (E = a T^4, F = 0); chat = c.  The cell-to-cell ripple keeps
    every neighbourhood away from the limiter's branch points: on uniform data
    the limited slopes sit at a kink (one-sided derivatives only), and on
    smooth data |d-| and |d+| nearly tie, so that a perturbation of relative
    size h switches branches in a fraction ~h/(ripple (k dx)^2) of the cells
    (finite differences then converge only linearly in h).  The target is
    E_tgt = a (1 + 9 exp(-|x - x1|^2 / (2 0.08^2)))^4 with x1 uniform in
    [0.25, 0.75]^2 (seed ``seed_target``).  The loss is
    L = sum (E(nsteps) - E_tgt)^2 over cells.

    Returns (problem, T0 (1, n, n), log_kappa (1, n, n), E_tgt (1, n, n), nsteps)."""
    dx = 1.0 / n
    prob = base_problem(2, [n, n], [dx, dx], bc="periodic", c=c, chat=c, **kw)
    sh = (1, n, n)
    lnchi = gaussian_random_field(sh, -4.0, np.random.default_rng(seed_chi))
    chi = np.exp(lnchi)
    chi *= 1.0 / (np.median(chi) * dx)
    x, y, _ = cell_centres(prob)
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    ripple = np.random.default_rng(seed_T).uniform(-1.0, 1.0, sh)
    T0 = np.ascontiguousarray((1.0 + 9.0 * np.exp(-r2 / (2 * 0.05 ** 2))) *
                              (1.0 + T_ripple * ripple))
    x1 = np.random.default_rng(seed_target).uniform(0.25, 0.75, 2)
    r2t = (x - x1[0]) ** 2 + (y - x1[1]) ** 2
    a = prob.get("a_rad", 1.0)
    E_tgt = np.ascontiguousarray(
        np.broadcast_to(a * (1.0 + 9.0 * np.exp(-r2t / (2 * 0.08 ** 2))) ** 4, sh))
    log_kappa = np.log(chi)  # rho = 1
    return prob, T0, np.ascontiguousarray(log_kappa), E_tgt, nsteps


def rest_state(prob: dict, T, log_kappa) -> np.ndarray:
    """State of gas at rest (rho = 1) with radiation in equilibrium at T and
    opacity exp(log_kappa): the map from the differentiation workload's
    parameters to the step's input."""
    T = np.asarray(T, dtype=np.float64)
    sh = T.shape
    return equilibrium_state(prob, np.ones(sh), T, np.zeros((3,) + sh),
                             np.exp(np.asarray(log_kappa, dtype=np.float64)))


# Asymptotic Marshak wave (Sec. 5.2) in cgs with temperatures in keV.
A_RAD_KEV = 7.5657e-15 * 1.160451812e7 ** 4  # radiation constant, erg cm^-3 keV^-4
C_CGS = 2.99792458e10                         # cm s^-1


def marshak_wave_1d(n: int = 60, L: float = 0.66, scheme: str = "imex", cfl: float = 0.9,
                    T_source: float = 1.0, T0: float = 1e-3, **kw):
    """Radiation from a T_source (keV) source entering a cold medium through the
    x = 0 face: chi = 300 cm^-1 (T/keV)^-3, volumetric heat capacity
    3e15 erg cm^-3 keV^-1 (rho = 1 g cm^-3, gamma = 5/3), T = T0 and
    E = a T0^4 initially, gas at rest, chat = c, HLL NONE (the paper's IMEX
    method), reflecting far wall.  The inflow face holds E = a T_source^4,
    F = 0.  Returns (problem, state)."""
    dx = L / n
    cv = 3e15
    prob = base_problem(
        1, [n], [dx], c=C_CGS, chat=C_CGS, a_rad=A_RAD_KEV, kB_over_mu=cv * (2.0 / 3.0),
        gamma=5.0 / 3.0, hll_mode="none", kappa_T_exp=-3.0, kappa_T_ref=1.0,
        bc=[["inflow", "reflect"], ["periodic", "periodic"], ["periodic", "periodic"]],
        bc_state={(0, 0): (A_RAD_KEV * T_source ** 4, 0.0, 0.0, 0.0)},
        scheme=scheme, cfl=cfl, **kw)
    sh = (1, 1, n)
    U = equilibrium_state(prob, np.ones(sh), np.full(sh, T0), np.zeros((3,) + sh),
                          np.full(sh, 300.0))
    return prob, U


A_RAD_CGS = 7.5657e-15   # radiation constant, erg cm^-3 K^-4
K_B_CGS = 1.380649e-16   # erg K^-1


def advecting_pulse_1d(v0: float = 1e6, n: int = 512, kappa: float = 100.0,
                       T0: float = 1e7, T1: float = 2e7, rho0: float = 1.2, w: float = 24.0,
                       mu: float = 3.9e-24, gamma: float = 5.0 / 3.0, **kw):
    """The advecting radiation pulse of Sec. 5.3: a Gaussian temperature pulse
    T = T0 + (T1 - T0) exp(-x^2 / 2w^2) on (-512, 512) cm (periodic, n cells),
    the density rho = rho0 T0/T + (a mu / 3 k_B)(T0^4/T - T^3) that balances
    gas and radiation pressure, gas and radiation at the same temperature
    (radiation in comoving equilibrium), grey kappa = 100 cm^2 g^-1, the
    Eddington closure, chat = c, uniform velocity v0 (0: the comoving run).
    Returns (problem, state)."""
    L = 1024.0
    dx = L / n
    prob = base_problem(1, [n], [dx], c=C_CGS, chat=C_CGS, a_rad=A_RAD_CGS,
                        kB_over_mu=K_B_CGS / mu, gamma=gamma, closure="eddington",
                        hll_mode="none", bc="periodic", **kw)
    x = -0.5 * L + (np.arange(n) + 0.5) * dx
    T = T0 + (T1 - T0) * np.exp(-x ** 2 / (2.0 * w * w))
    rho = rho0 * T0 / T + A_RAD_CGS * mu / (3.0 * K_B_CGS) * (T0 ** 4 / T - T ** 3)
    sh = (1, 1, n)
    v = np.zeros((3,) + sh)
    v[0] = v0
    U = equilibrium_state(prob, rho.reshape(sh), T.reshape(sh), v, np.full(sh, kappa))
    return prob, U
