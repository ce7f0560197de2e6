"""Pins of the oracle's hydrodynamic subsystem and operator split (Sec. 3.1):
the Euler equations by a method of lines with RK2-SSP, primitives
reconstructed with the transport's option, HLLC fluxes; then the radiation
step subcycled within the hydrodynamic step.

Each pin checks the oracle against something other than itself: the exact
Riemann solution (itself pinned to Toro's printed star values), the exact
preservation of a stationary contact that HLLC (not HLL) guarantees, the
translation of a contact in uniform flow, the acoustic speed, conservation,
mirror and axis symmetries, and the order of the split.  A dropped term in
the HLLC star energy leaves the shock-tube errors almost unchanged (they
measure wave positions and plateaus) but breaks the mirror pin.
"""
import os

import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from riemann_exact import sample, star

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toro_riemann_star.txt")


def prims(prob, U):
    rho = U[I.F_RHO]
    v = U[I.F_MX:I.F_MZ + 1] / rho
    p = (prob["gamma"] - 1.0) * (U[I.F_EGAS] - 0.5 * rho * (v * v).sum(axis=0))
    return rho, v, p


def test_exact_solver_reproduces_the_printed_star_values():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        rL, uL, pL, rR, uR, pR, ps, us, rsl, rsr = map(float, r[1:])
        p_, u_ = star((rL, uL, pL), (rR, uR, pR), 1.4)
        W = sample((rL, uL, pL), (rR, uR, pR), 1.4, [u_ - 1e-9, u_ + 1e-9])
        assert abs(p_ - ps) <= 6e-6 * max(ps, 1.0) + 5e-6, r
        assert abs(u_ - us) <= 6e-5, r
        assert abs(W[0, 0] - rsl) <= 6e-6 and abs(W[0, 1] - rsr) <= 6e-6, r


def _sod(O, n, rec):
    prob, U = I.riemann_problem_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1),
                                   reconstruction=rec)
    nsteps = int(np.ceil(0.2 / (0.3 / n / 2.0)))
    O.hydro_step(prob, U, nsteps, 0.2 / nsteps)
    x = (np.arange(n) + 0.5) / n
    W = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, (x - 0.5) / 0.2)
    rho, v, p = prims(prob, U)
    return [np.abs(rho[0, 0] - W[0]).mean(), np.abs(v[0, 0, 0] - W[1]).mean(),
            np.abs(p[0, 0] - W[2]).mean()]


@pytest.mark.parametrize("rec", ["plm", "ppm"])
def test_sod_converges_to_the_exact_solution(oracle_mod, rec):
    """Sod's shock tube at t = 0.2 (100, 200, 400 cells): the L1 errors of
    rho, u and p fall by at least 1.7 per doubling (first order at the shock
    and the contact) and are below 5e-3 (rho), 1e-2 (u), 3.5e-3 (p) on 100
    cells (measured PLM 4.9e-3, 9.4e-3, 3.4e-3; PPM lower)."""
    errs = [_sod(oracle_mod, n, rec) for n in (100, 200, 400)]
    for k in range(3):
        assert errs[0][k] > 1.7 * errs[1][k] > 1.7 * 1.7 * errs[2][k] * 0.999, errs
    assert errs[0][0] < 5e-3 and errs[0][1] < 1e-2 and errs[0][2] < 3.5e-3, errs


@pytest.mark.parametrize("rec", ["plm", "ppm"])
def test_strong_blast_converges(oracle_mod, rec):
    """Toro's test 3 (pressure ratio 1e5) at t = 0.012: positive throughout,
    L1 error of rho below 0.09 on 200 cells and falling by 1.9 per doubling
    (measured PLM 0.079 -> 0.038)."""
    WL, WR, t = (1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 0.012
    errs = []
    for n in (200, 400):
        prob, U = I.riemann_problem_1d(n, WL, WR, reconstruction=rec)
        nsteps = int(np.ceil(t / (0.3 / n / 45.0)))
        oracle_mod.hydro_step(prob, U, nsteps, t / nsteps)
        x = (np.arange(n) + 0.5) / n
        W = sample(WL, WR, 1.4, (x - 0.5) / t)
        errs.append(np.abs(U[I.F_RHO, 0, 0] - W[0]).mean())
    assert errs[0] < 0.09 and errs[0] > 1.9 * errs[1], errs


def test_stationary_contact_is_exact(oracle_mod):
    """A density jump at rest in uniform pressure: HLLC's middle wave
    resolves it exactly (zero mass and energy flux, flux p of momentum),
    where HLL would smear it; 50 steps leave the state unchanged."""
    n = 64
    prob, U = I.riemann_problem_1d(n, (1.0, 0.0, 1.0), (0.1, 0.0, 1.0), bc="periodic")
    U0 = U.copy()
    oracle_mod.hydro_step(prob, U, 50, 0.3 / n / np.sqrt(1.4 / 0.1))
    for f in (I.F_RHO, I.F_MX, I.F_EGAS):
        assert np.max(np.abs(U[f] - U0[f])) <= 1e-14 * np.max(np.abs(U0[I.F_EGAS])), f


def test_contact_advects_with_the_flow(oracle_mod):
    """rho = 1 + 0.2 sin(2 pi x) carried by u = 1 at p = 1 once around a
    periodic box returns to itself: second-order convergent (error ratio
    above 3.2 per doubling, against 2 at first order; the limiters clip the
    extrema: measured 3.3-3.7), PPM below PLM at every resolution."""
    errs = {}
    for rec in ("plm", "ppm"):
        errs[rec] = []
        for n in (32, 64, 128):
            prob = I.base_problem(1, [n], [1.0 / n], gamma=1.4, reconstruction=rec)
            x = (np.arange(n) + 0.5) / n
            sh = (1, 1, n)
            rho0 = (1.0 + 0.2 * np.sin(2 * np.pi * x)).reshape(sh)
            v = np.zeros((3,) + sh)
            v[0] = 1.0
            U = I.gas_state(prob, rho0, v, np.ones(sh))
            nsteps = 4 * n
            oracle_mod.hydro_step(prob, U, nsteps, 1.0 / nsteps)
            errs[rec].append(np.abs(U[I.F_RHO, 0, 0] - rho0[0, 0]).mean())
        e = errs[rec]
        assert e[0] / e[1] > 3.2 and e[1] / e[2] > 3.2, errs
    assert all(a < b for a, b in zip(errs["ppm"], errs["plm"])), errs


def test_acoustic_pulse_moves_at_the_sound_speed(oracle_mod):
    """A small right-going simple wave (d rho = eps f, du = a d rho / rho,
    dp = a^2 d rho) travels at a = sqrt(gamma p / rho): its centroid moves
    by a t (to 1e-3 of the distance)."""
    n, g = 400, 1.4
    prob = I.base_problem(1, [n], [1.0 / n], gamma=g, bc="periodic")
    x = (np.arange(n) + 0.5) / n
    sh = (1, 1, n)
    a = np.sqrt(g)
    drho = 1e-4 * np.exp(-((x - 0.3) / 0.03) ** 2)
    v = np.zeros((3,) + sh)
    v[0] = (a * drho).reshape(sh)
    U = I.gas_state(prob, (1.0 + drho).reshape(sh), v, (1.0 + a * a * drho).reshape(sh))
    t = 0.25
    nsteps = 400
    oracle_mod.hydro_step(prob, U, nsteps, t / nsteps)
    d = U[I.F_RHO, 0, 0] - 1.0
    shift = (x * d).sum() / d.sum() - 0.3
    assert abs(shift / (a * t) - 1.0) < 1e-3, shift / (a * t)


def _random_gas(prob, seed, mach=0.5):
    rng = np.random.default_rng(seed)
    sh = I.shape_of(prob)[1:]
    rho = 1.0 + 0.3 * rng.uniform(-1, 1, sh)
    p = 1.0 + 0.3 * rng.uniform(-1, 1, sh)
    v = mach * rng.uniform(-1, 1, (3,) + sh)
    for d in range(prob["ndim"], 3):
        v[d] = 0.0
    return rho, v, p


@pytest.mark.parametrize("rec", ["plm", "ppm"])
def test_hydro_conserves_mass_momentum_energy(oracle_mod, rec):
    prob = I.base_problem(2, [24, 20], [1 / 24, 1 / 20], gamma=1.4, reconstruction=rec)
    rho, v, p = _random_gas(prob, 3)
    U = I.gas_state(prob, rho, v, p)
    tot0 = [U[f].sum() for f in (I.F_RHO, I.F_MX, I.F_MY, I.F_EGAS)]
    oracle_mod.hydro_step(prob, U, 10)
    tot1 = [U[f].sum() for f in (I.F_RHO, I.F_MX, I.F_MY, I.F_EGAS)]
    scale = [U[I.F_RHO].sum(), np.abs(U[I.F_MX]).sum(), np.abs(U[I.F_MY]).sum(),
             U[I.F_EGAS].sum()]
    for a, b, s in zip(tot0, tot1, scale):
        assert abs(a - b) <= 1e-13 * s


def test_uniform_flow_is_preserved(oracle_mod):
    prob = I.base_problem(3, [6, 5, 4], [0.1, 0.2, 0.3], gamma=1.4)
    sh = I.shape_of(prob)[1:]
    v = np.zeros((3,) + sh)
    v[0], v[1], v[2] = 0.3, -0.2, 0.1
    U = I.gas_state(prob, np.full(sh, 2.0), v, np.full(sh, 3.0))
    U0 = U.copy()
    oracle_mod.hydro_step(prob, U, 5)
    for f in (I.F_RHO, I.F_MX, I.F_MY, I.F_MZ, I.F_EGAS):
        assert np.max(np.abs(U[f] - U0[f])) <= 1e-14 * np.max(np.abs(U0[I.F_EGAS]))


@pytest.mark.parametrize("ndim,rec", [(1, "plm"), (2, "plm"), (1, "ppm"), (2, "ppm")])
def test_reflecting_walls_equal_the_mirrored_periodic_box(oracle_mod, ndim, rec):
    """A wall mirrors the cell and negates the normal velocity: n cells
    between walls = the left half of a periodic box of 2n holding the state
    and its mirror image (1e-13)."""
    n = 11
    shape = (n,) if ndim == 1 else (n, 6)
    kw = dict(gamma=1.4, reconstruction=rec)
    bc_w = [["reflect", "reflect"], ["periodic", "periodic"], ["periodic", "periodic"]]
    pw = I.base_problem(ndim, shape, tuple(1.0 / s for s in shape), bc=bc_w, **kw)
    pp = I.base_problem(ndim, (2 * n,) + shape[1:], tuple(1.0 / s for s in shape),
                        bc="periodic", **kw)
    rho, v, p = _random_gas(pw, 5)
    U = I.gas_state(pw, rho, v, p)
    M = U[..., ::-1].copy()
    M[I.F_MX] *= -1.0
    M[I.F_FX] *= -1.0
    U2 = np.concatenate([U, M], axis=-1)
    dt = 0.2 * oracle_mod.hydro_dt(pw, U)
    oracle_mod.hydro_step(pw, U, 4, dt)
    oracle_mod.hydro_step(pp, U2, 4, dt)
    for f in (I.F_RHO, I.F_MX, I.F_MY, I.F_EGAS):
        s = np.max(np.abs(U2[f]))
        assert np.max(np.abs(U[f] - U2[f][..., :n])) <= 1e-13 * s, I.FIELDS[f]


def test_flow_along_y_equals_1d(oracle_mod):
    """Sod along the second axis of a 2-D grid, uniform along the first: every
    column evolves bit for bit as the 1-D tube (the first axis's faces carry
    exactly the pressure)."""
    n = 64
    p1, U1 = I.riemann_problem_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    p2 = I.base_problem(2, [4, n], [1.0 / n, 1.0 / n], gamma=1.4, bc="reflect")
    sh = (1, n, 4)
    rho = np.broadcast_to(U1[I.F_RHO, 0, 0][None, :, None], sh)
    rho1, v1, pr1 = prims(p1, U1)
    v = np.zeros((3,) + sh)
    U2 = I.gas_state(p2, rho, v, np.broadcast_to(pr1[0, 0][None, :, None], sh))
    dt = 0.3 / n / 2.0
    oracle_mod.hydro_step(p1, U1, 30, dt)
    oracle_mod.hydro_step(p2, U2, 30, dt)
    for i in range(4):
        assert np.array_equal(U2[I.F_RHO, 0, :, i], U1[I.F_RHO, 0, 0])
        assert np.array_equal(U2[I.F_MY, 0, :, i], U1[I.F_MX, 0, 0])
        assert np.array_equal(U2[I.F_EGAS, 0, :, i], U1[I.F_EGAS, 0, 0])


def test_hydro_dt_is_the_cfl_bound(oracle_mod):
    prob = I.base_problem(2, [12, 10], [0.1, 0.05], gamma=1.4, cfl_hydro=0.35)
    rho, v, p = _random_gas(prob, 9)
    U = I.gas_state(prob, rho, v, p)
    a = np.sqrt(1.4 * p / rho)
    s = (np.abs(v[0]) + a) / 0.1 + (np.abs(v[1]) + a) / 0.05
    assert oracle_mod.hydro_dt(prob, U) == pytest.approx(0.35 / s.max(), rel=1e-14)


def test_inflow_axis_is_refused(oracle_mod):
    prob, U = I.marshak_wave_1d(16)
    with pytest.raises(RuntimeError, match="arg"):
        oracle_mod.hydro_rate(prob, U)


def test_split_runs_hydro_then_subcycled_radiation(oracle_mod):
    """Sec. 3.1: one split step = the hydrodynamic step of dt_h, then
    nsub = ceil(dt_h / dt_rad) radiation steps of dt_h / nsub; bit for bit
    against the two subsystems called in that order (coupled gas)."""
    prob = I.base_problem(2, [12, 10], [1 / 12, 1 / 10], gamma=5 / 3, c=30.0, chat=10.0)
    rho, v, p = _random_gas(prob, 11, mach=0.3)
    U = I.gas_state(prob, rho, v, p, kappa=2.0)
    A, B = U.copy(), U.copy()
    dt_h = oracle_mod.hydro_dt(prob, U)
    subs = oracle_mod.split_step(prob, A, 1)
    nsub = int(np.ceil(dt_h / oracle_mod.dt(prob) - 1e-12))
    assert subs == [nsub] and nsub > 3
    oracle_mod.hydro_step(prob, B, 1, dt_h)
    oracle_mod.step(prob, B, nsub, dt_h / nsub)
    assert np.array_equal(A, B)


@pytest.mark.parametrize("kappa", [0.5, 20.0])
def test_split_error_is_first_order_in_the_hydro_step(oracle_mod, kappa):
    """Sec. 3.1 splits the hydrodynamic step from the radiation update once per
    step (first order): on a fixed grid, with every radiation substep the same
    dt_rad (t_end = 512 dt_rad, dt_h = t_end/m), the state at t_end moves
    toward the m = 512 result in proportion to dt_h (error ratio 2 per halving;
    a symmetric split would give 4, a split that loses or misplaces a substep
    would not converge).  A smooth coupled gas, optically thin and thick."""
    n = 48
    prob = I.base_problem(1, [n], [1.0 / n], gamma=5 / 3, c=300.0, chat=100.0, bc="periodic")
    x = (np.arange(n) + 0.5) / n
    sh = (1, 1, n)
    rho = (1 + 0.2 * np.sin(2 * np.pi * x)).reshape(sh)
    p = (1 + 0.2 * np.cos(2 * np.pi * x)).reshape(sh)
    v = np.zeros((3,) + sh)
    v[0] = 0.3 * np.sin(2 * np.pi * x + 1).reshape(sh)
    U0 = I.gas_state(prob, rho, v, p, kappa=kappa)
    t_end = 512 * oracle_mod.dt(prob)
    assert t_end / 16 < oracle_mod.hydro_dt(prob, U0)
    out = {}
    for m in (16, 32, 64, 512):
        U = U0.copy()
        subs = oracle_mod.split_step(prob, U, m, t_end / m)
        assert subs == [512 // m] * m
        out[m] = U
    fields = (I.F_RHO, I.F_MX, I.F_EGAS, I.F_ERAD, I.F_FX)
    err = [max(np.max(np.abs(out[m][f] - out[512][f])) / np.max(np.abs(out[512][f]))
               for f in fields) for m in (16, 32, 64)]
    for a, b in zip(err, err[1:]):
        assert 1.8 < a / b < 2.5, err


def test_split_conserves_total_energy_and_momentum(oracle_mod):
    """Hydrodynamics conserves E_gas and m, the radiation step E_gas +
    (c/chat) E and m + F/(c chat): the split conserves the latter (1e-13)."""
    prob = I.base_problem(2, [12, 10], [1 / 12, 1 / 10], gamma=5 / 3, c=30.0, chat=10.0,
                          hll_mode="none")
    rho, v, p = _random_gas(prob, 13, mach=0.3)
    U = I.gas_state(prob, rho, v, p, kappa=3.0)
    r = prob["c"] / prob["chat"]
    cc = prob["c"] * prob["chat"]

    def tot(U):
        return [(U[I.F_EGAS] + r * U[I.F_ERAD]).sum(),
                (U[I.F_MX] + U[I.F_FX] / cc).sum(), (U[I.F_MY] + U[I.F_FY] / cc).sum()]
    t0 = tot(U)
    oracle_mod.split_step(prob, U, 3)
    t1 = tot(U)
    scale = [t0[0], np.abs(U[I.F_MX]).sum(), np.abs(U[I.F_MY]).sum()]
    for a, b, s in zip(t0, t1, scale):
        assert abs(a - b) <= 1e-13 * s


def test_colella_sekora_keeps_the_pulse_density_dip(oracle_mod):
    """The density of the dynamic-diffusion pulse of Sec. 5.4 (a 17:1 dip 24
    cells wide) carried 128 cells by uniform flow at uniform pressure: CW84's
    constraint flattens the smooth minimum every step (> 2 % lost), the
    Colella-Sekora limiter keeps it (< 1e-4)."""
    prob0, U0 = I.advecting_pulse_1d(3e7, n=1024, kappa=500.0)
    rho = U0[I.F_RHO, 0, 0]
    n = 1024
    loss = {}
    for rec in ("ppm", "ppm_cs"):
        prob = I.base_problem(1, [n], [1.0], gamma=5 / 3, bc="periodic", reconstruction=rec,
                              kB_over_mu=prob0["kB_over_mu"])
        sh = (1, 1, n)
        v = np.zeros((3,) + sh)
        v[0] = 3e7
        U = I.gas_state(prob, rho.reshape(sh).copy(), v, np.full(sh, 6.0e14))
        t_end = 128 / 3e7
        nh = int(np.ceil(t_end / (0.9 * oracle_mod.hydro_dt(prob, U))))
        oracle_mod.hydro_step(prob, U, nh, t_end / nh)
        loss[rec] = np.max(np.abs(np.roll(U[I.F_RHO, 0, 0], -128) - rho) / rho)
    assert loss["ppm"] > 2e-2 and loss["ppm_cs"] < 1e-4, loss


def test_sod_ppm_rounding_floor(oracle_mod):
    """Conditioning of Sod's tube with PPM faces (100 cells, 134 steps), the
    basis of the GPU parity bound of that case: half-ulp noise added to rho,
    m and E_gas after every step moves the oracle's own end state by more
    than 1e-10 (the constraint's switches at the shock and contact feed
    rounding back), and by less than the bound the GPU test applies (1e-9);
    with PLM faces the same noise stays below 1e-13."""
    from parity import field_errors
    O = oracle_mod
    spread = {}
    for rec in ("plm", "ppm"):
        prob, U = I.riemann_problem_1d(100, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1),
                                       reconstruction=rec)
        A = U.copy()
        O.hydro_step(prob, A, 134, 0.2 / 134)
        worst = 0.0
        for seed in (1, 2):
            rng = np.random.default_rng(seed)
            B = U.copy()
            for _ in range(134):
                O.hydro_step(prob, B, 1, 0.2 / 134)
                for f in (I.F_RHO, I.F_MX, I.F_EGAS):
                    B[f] *= 1.0 + 1.1e-16 * rng.choice([-1.0, 1.0], B.shape[1:])
            worst = max(worst, max(field_errors(B, A).values()))
        spread[rec] = worst
    assert 1e-10 < spread["ppm"] <= 1e-9, spread
    assert spread["plm"] < 1e-13, spread
