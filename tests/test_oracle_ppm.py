"""Pins of the oracle's PPM face states (the paper's reconstruction, Sec.
3.3; Colella & Woodward 1984 base scheme as method-of-lines interface
values): a free-streaming beam against a textbook PPM advection code, the
order on a smooth wave, and the asymptotic diffusion limit against PLM."""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from diffusion_ref import front, marshak_diffusion


def _mc(um, u0, up):
    dm, dp = u0 - um, up - u0
    mag = np.minimum(np.minimum(2 * np.abs(dm), 2 * np.abs(dp)), 0.5 * np.abs(dm + dp))
    return np.where(dm * dp > 0, np.sign(dm) * mag, 0.0)


def ppm_advect(u, a, dt, dx, nsteps):
    """Textbook u_t + a u_x = 0 (a > 0), periodic: PPM interface values
    a_{j+1/2} = (u_j + u_{j+1})/2 - (dm_{j+1} - dm_j)/6 (MC slopes dm), the
    monotonicity constraint on each cell's edge pair, the upwind edge value
    at each face, Heun (SSP-RK2) steps."""
    def rhs(u):
        s = _mc(np.roll(u, 1), u, np.roll(u, -1))
        ah = 0.5 * (u + np.roll(u, -1)) - (np.roll(s, -1) - s) / 6.0
        aL, aR = np.roll(ah, 1), ah
        ext = (aR - u) * (u - aL) <= 0
        dd, m6 = aR - aL, 6.0 * (u - 0.5 * (aL + aR))
        c1 = dd * m6 > dd * dd
        c2 = -dd * dd > dd * m6
        aR2 = np.where(ext, u, np.where(~c1 & c2, 3 * u - 2 * aL, aR))
        flux = a * aR2                      # face j+1/2
        return -(flux - np.roll(flux, 1)) / dx

    for _ in range(nsteps):
        u1 = u + dt * rhs(u)
        u = 0.5 * (u + u1) + 0.5 * dt * rhs(u1)
    return u


def _beam(n, profile, reconstruction, cfl=0.3):
    prob = I.base_problem(1, [n], [1.0 / n], c=1.0, chat=1.0, reconstruction=reconstruction,
                          cfl=cfl)
    sh = (1, 1, n)
    U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh), np.zeros((3,) + sh), np.zeros(sh))
    x = I.cell_centres(prob)[0].reshape(-1)
    E = profile(x)
    U[I.F_ERAD] = E.reshape(sh)
    U[I.F_FX] = E.reshape(sh)
    return prob, U, x, E


@pytest.mark.parametrize("nsteps,tol", [(10, 1e-13), (60, 1e-8)])
def test_ppm_beam_is_textbook_ppm_advection(oracle_mod, nsteps, tol):
    """chi = 0 and F = c E: HLL is exact upwinding at chat, so E follows the
    textbook PPM scheme (a Gaussian and a step, CFL 0.3: an edge value may
    reach three times the cell mean, so each forward-Euler stage keeps E > 0
    only for CFL <= 1/3; above that the step's foot goes negative and the
    next face state is refused as nonphysical).

    The two codes round in different orders (HLL's flux formula against a
    plain upwind product), and where the parabola is monotone the scheme is
    the centred fourth-order flux, which Heun steps amplify (|G|^2 = 1 +
    z^4/4); switches of the monotonicity constraint on the pulse's flanks
    then feed the difference back: 1e-16 for 11 steps, ~4e-10 after 60.
    Rounding-level agreement over 10 steps, 1e-8 over 60."""
    O = oracle_mod
    n = 96
    for prof in (lambda x: 1e-3 + np.exp(-((x - 0.3) / 0.05) ** 2),
                 lambda x: 1e-3 + (np.abs(x - 0.4) < 0.1)):
        prob, U, x, E = _beam(n, prof, "ppm")
        dt = O.dt(prob)
        O.step(prob, U, nsteps=nsteps, dt=dt)
        ref = ppm_advect(E.copy(), 1.0, dt, 1.0 / n, nsteps)
        assert np.max(np.abs(U[I.F_ERAD, 0, 0] - ref)) <= tol * np.max(np.abs(ref))


def test_ppm_rate_is_fourth_order_away_from_extrema(oracle_mod):
    """Where the profile is monotone the PPM interface value is the centred
    fourth-order one (CW84 eq. 1.6 with unlimited slopes), so the transport
    rate of a free-streaming smooth wave converges as dx^4 (error ratio 16 per
    doubling), against dx^2 for PLM; near the extrema the monotonicity
    constraint flattens the cell and is left out of the measure."""
    O = oracle_mod
    for rec, ratio in (("plm", 4.0), ("ppm", 16.0)):
        errs = []
        for n in (32, 64, 128, 256):
            prob, U, x, E = _beam(n, lambda x: 2.0 + np.sin(2 * np.pi * x), rec)
            rate = O.transport(prob, U)[0].reshape(-1)
            exact = -2 * np.pi * np.cos(2 * np.pi * x)
            away = np.abs(np.sin(2 * np.pi * x)) < 0.7
            errs.append(np.abs(rate - exact)[away].max())
        for e0, e1 in zip(errs, errs[1:]):
            assert abs(e0 / e1 / ratio - 1.0) < 0.03, (rec, errs)


def test_ppm_diffusion_limit(oracle_mod):
    """The asymptotic diffusion limit with PPM faces (tau_cell = 10, negligible
    gas heat capacity): a Gaussian spreads as sigma^2 + 2 D t with
    D = c/(3 chi) to the same accuracy as with PLM (Sec. 4.1: the limit is a
    property of the time integration, not of the face states)."""
    O = oracle_mod
    c, rho, chi, n, s0 = 1e3, 1e3, 1280.0, 128, 0.05
    out = {}
    for rec in ("plm", "ppm"):
        prob = I.base_problem(1, [n], [1.0 / n], bc="periodic", c=c, chat=c, kB_over_mu=1e-6,
                              hll_mode="none", reconstruction=rec)
        x = I.cell_centres(prob)[0].reshape(-1)
        E0 = 1.0 + np.exp(-((x - 0.5) ** 2) / (2 * s0 ** 2))
        sh = (1, 1, n)
        U = I.equilibrium_state(prob, np.full(sh, rho), (E0 ** 0.25).reshape(sh),
                                np.zeros((3,) + sh), np.full(sh, chi / rho))
        dt = O.dt(prob)
        nsteps = int(round(s0 ** 2 / (2 * c / (3 * chi)) / dt))
        O.step(prob, U, nsteps=nsteps, dt=dt)
        t = nsteps * dt
        s2 = s0 ** 2 + 2 * c / (3 * chi) * t
        exact = 1.0 + np.sqrt(s0 ** 2 / s2) * np.exp(-((x - 0.5) ** 2) / (2 * s2))
        out[rec] = np.abs(U[I.F_ERAD, 0, 0] - exact).max()
    assert out["ppm"] < 2.5e-2 and out["ppm"] < 1.5 * out["plm"], out


def test_ppm_refuses_a_negative_stage_state(oracle_mod):
    """Beyond CFL 1/3 a free-streaming step undershoots in the first stage;
    the oracle reports that instead of carrying E < 0 into the faces."""
    O = oracle_mod
    prob, U, x, E = _beam(96, lambda x: 1e-3 + (np.abs(x - 0.4) < 0.1), "ppm", cfl=0.4)
    with pytest.raises(RuntimeError, match="nonphysical"):
        O.step(prob, U, nsteps=10)


T_MARSHAK = 3e-9


def _marshak_front(O, n, cfl, rec):
    prob, U = I.marshak_wave_1d(n, scheme="imex", cfl=cfl, reconstruction=rec)
    dt = O.dt(prob)
    O.step(prob, U, nsteps=int(round(T_MARSHAK / dt)), dt=dt)
    x = I.cell_centres(prob)[0].reshape(-1)
    return front(x, U[I.F_EGAS, 0, 0] / 3e15)


def test_marshak_with_ppm_is_closer_to_diffusion(oracle_mod):
    """Sec. 5.2 runs the asymptotic Marshak wave with PPM faces: on 60 cells
    the T = 0.5 keV front lies within 2 % of the equilibrium-diffusion front
    (measured 1.1 %, against 11 % with PLM), and the same within 1 % at CFL
    10."""
    O = oracle_mod
    ref = front(*marshak_diffusion(T_MARSHAK, I.A_RAD_KEV, I.C_CGS, 3e15))
    f_ppm = _marshak_front(O, 60, 0.9, "ppm")
    f_plm = _marshak_front(O, 60, 0.9, "plm")
    assert abs(f_ppm / ref - 1.0) < 0.02, (f_ppm, ref)
    assert abs(f_ppm / ref - 1.0) < 0.5 * abs(f_plm / ref - 1.0), (f_ppm, f_plm, ref)
    f10 = _marshak_front(O, 60, 10.0, "ppm")
    assert abs(f10 / f_ppm - 1.0) < 1e-2, (f10, f_ppm)


def test_ppm_along_y_equals_1d(oracle_mod):
    """A beam along the second axis of a 2-D grid, uniform along the first:
    the first axis's PPM faces are exact (interface value = cell value), so
    every column evolves bit for bit as the 1-D problem."""
    O = oracle_mod
    n = 48
    prof = lambda x: 1e-2 + np.exp(-((x - 0.5) / 0.08) ** 2)
    p1, U1, x, E = _beam(n, prof, "ppm")
    p2 = I.base_problem(2, [5, n], [1.0 / n, 1.0 / n], c=1.0, chat=1.0, reconstruction="ppm",
                        cfl=0.3)
    sh = (1, n, 5)
    U2 = I.equilibrium_state(p2, np.ones(sh), np.ones(sh), np.zeros((3,) + sh), np.zeros(sh))
    U2[I.F_ERAD] = E[None, :, None]
    U2[I.F_FY] = E[None, :, None]
    dt = O.dt(p1) * 0.5
    O.step(p1, U1, nsteps=8, dt=dt)
    O.step(p2, U2, nsteps=8, dt=dt)
    for i in range(5):
        assert np.array_equal(U2[I.F_ERAD, 0, :, i], U1[I.F_ERAD, 0, 0])
        assert np.array_equal(U2[I.F_FY, 0, :, i], U1[I.F_FX, 0, 0])


@pytest.mark.parametrize("ndim", [1, 2])
def test_ppm_reflecting_walls_equal_the_mirrored_periodic_box(oracle_mod, ndim):
    """A reflecting wall mirrors E and flips the normal F, three cells deep
    for the PPM stencil.  A coupled random state on n cells between two walls
    (axis 0) equals, to rounding, the left half of a periodic box of 2n cells
    holding the state and its mirror image."""
    O = oracle_mod
    n = 11
    shape = (n,) if ndim == 1 else (n, 6)
    bc_w = [["reflect", "reflect"], ["periodic", "periodic"], ["periodic", "periodic"]]
    kw = dict(c=1e3, chat=2e2, reconstruction="ppm", cfl=0.2, hll_mode="tau")
    pw = I.base_problem(ndim, shape, tuple(1.0 / v for v in shape), bc=bc_w, **kw)
    shape2 = (2 * n,) + shape[1:]
    pp = I.base_problem(ndim, shape2, tuple(1.0 / v for v in shape), bc="periodic", **kw)
    U = I.random_state(pw, seed=77, tau_range=(1e-2, 1e1), beta_max=1e-2)
    M = U[..., ::-1].copy()
    M[I.F_MX] *= -1.0
    M[I.F_FX] *= -1.0
    U2 = np.concatenate([U, M], axis=-1)
    dt = O.dt(pw)
    O.step(pw, U, nsteps=3, dt=dt)
    O.step(pp, U2, nsteps=3, dt=dt)
    for f in range(I.NFIELD):
        a, b = U[f], U2[f][..., :n]
        scale = np.max(np.abs(U2[f])) + 1e-300
        assert np.max(np.abs(a - b)) <= 1e-13 * scale, I.FIELDS[f]


# ---------------------------------------- the Colella-Sekora (2008) limiter

def _cs_edges(u, C=1.25):
    """Textbook PPM edges with the limiter of Colella & Sekora (2008) on a
    periodic array: the fourth-order interface value, limited through its
    second difference where it leaves [u_j, u_j+1]; at a local extremum the
    parabola's curvature limited against C times the neighbouring second
    differences; elsewhere the overshoot correction."""
    um1, up1, up2, um2 = np.roll(u, 1), np.roll(u, -1), np.roll(u, -2), np.roll(u, 2)
    a = 7.0 / 12.0 * (u + up1) - 1.0 / 12.0 * (um1 + up2)
    bad = (a - u) * (up1 - a) < 0
    d2a, d2l, d2r = 3.0 * (u - 2 * a + up1), um1 - 2 * u + up1, u - 2 * up1 + up2
    same = (np.sign(d2a) == np.sign(d2l)) & (np.sign(d2a) == np.sign(d2r))
    lim = np.where(same, np.sign(d2a) * np.minimum(C * np.abs(d2a),
                                                   np.minimum(np.abs(d2l), np.abs(d2r))), 0.0)
    a = np.where(bad, 0.5 * (u + up1) - lim / 6.0, a)
    l, r = np.roll(a, 1), a.copy()
    ext = ((r - u) * (u - l) <= 0) | ((um1 - u) * (u - up1) <= 0)
    d2 = -12.0 * u + 6.0 * (l + r)
    d2c, d2L, d2R = um1 - 2 * u + up1, um2 - 2 * um1 + u, u - 2 * up1 + up2
    same = (np.sign(d2) == np.sign(d2c)) & (np.sign(d2) == np.sign(d2L)) & \
        (np.sign(d2) == np.sign(d2R))
    lim = np.where(same, np.sign(d2) * np.minimum(
        np.minimum(C * np.abs(d2c), C * np.abs(d2L)), np.minimum(C * np.abs(d2R), np.abs(d2))),
        0.0)
    fac = np.where(d2 != 0, lim / np.where(d2 != 0, d2, 1.0), 0.0)
    le, re = np.where(ext, u + (l - u) * fac, l), np.where(ext, u + (r - u) * fac, r)
    dl, dr = u - le, re - u
    big_r = (~ext) & (np.abs(dr) >= 2 * np.abs(dl))
    big_l = (~ext) & (np.abs(dl) >= 2 * np.abs(dr))
    return np.where(big_l, u - 2 * dr, le), np.where(big_r, u + 2 * dl, re)


def _cs_advect(u, nu, nsteps):
    def rhs(u):
        r = _cs_edges(u)[1]
        return -(r - np.roll(r, 1)) * nu
    for _ in range(nsteps):
        u1 = u + rhs(u)
        u = 0.5 * (u + u1) + 0.5 * rhs(u1)
    return u


@pytest.mark.parametrize("nsteps", [10, 60])
def test_ppm_cs_beam_is_textbook_colella_sekora_advection(oracle_mod, nsteps):
    """The reconstruction option ppm_cs on a free-streaming beam (a Gaussian
    and a step) = a textbook Colella-Sekora PPM advection with Heun steps, to
    rounding (1e-14) over 10 and 60 steps: without CW84's switch at every
    smooth extremum the rounding difference does not grow."""
    O = oracle_mod
    n = 96
    for prof in (lambda x: 1e-3 + np.exp(-((x - 0.3) / 0.05) ** 2),
                 lambda x: 1e-3 + (np.abs(x - 0.4) < 0.1)):
        prob, U, x, E = _beam(n, prof, "ppm_cs")
        dt = O.dt(prob)
        O.step(prob, U, nsteps=nsteps, dt=dt)
        ref = _cs_advect(E.copy(), dt * n, nsteps)
        assert np.max(np.abs(U[I.F_ERAD, 0, 0] - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_ppm_cs_keeps_fourth_order_at_extrema(oracle_mod):
    """The transport rate of a free-streaming sine over every cell, extrema
    included: with CW84's constraint the max error halves per doubling (the
    flat extremum cells are first order), with Colella-Sekora it falls 16x."""
    O = oracle_mod
    for rec, ratio in (("ppm", 2.0), ("ppm_cs", 16.0)):
        errs = []
        for n in (32, 64, 128, 256):
            prob, U, x, E = _beam(n, lambda x: 2.0 + np.sin(2 * np.pi * x), rec)
            rate = O.transport(prob, U)[0].reshape(-1)
            errs.append(np.abs(rate + 2 * np.pi * np.cos(2 * np.pi * x)).max())
        for e0, e1 in zip(errs, errs[1:]):
            assert abs(e0 / e1 / ratio - 1.0) < 0.03, (rec, errs)


def test_ppm_cs_reflecting_walls_equal_the_mirrored_periodic_box(oracle_mod):
    """Mirror ghosts three cells deep under the Colella-Sekora limiter (which
    reads the second differences of cells two away): walls = the mirrored
    periodic box, 1e-13 (1-D and 2-D).  The limiter keeps a cell's curvature
    at an extremum, so on rough data an edge can leave the range of its
    neighbours (and E go negative): the random state here has a temperature
    contrast of 1.3, not 3."""
    O = oracle_mod
    n = 11
    for ndim in (1, 2):
        shape = (n,) if ndim == 1 else (n, 6)
        bc_w = [["reflect", "reflect"], ["periodic", "periodic"], ["periodic", "periodic"]]
        kw = dict(c=1e3, chat=2e2, reconstruction="ppm_cs", cfl=0.2, hll_mode="tau")
        pw = I.base_problem(ndim, shape, tuple(1.0 / v for v in shape), bc=bc_w, **kw)
        pp = I.base_problem(ndim, (2 * n,) + shape[1:], tuple(1.0 / v for v in shape),
                            bc="periodic", **kw)
        U = I.random_state(pw, seed=78, tau_range=(1e-2, 1e1), beta_max=1e-2,
                           T_range=(1.0, 1.3))
        M = U[..., ::-1].copy()
        M[I.F_MX] *= -1.0
        M[I.F_FX] *= -1.0
        U2 = np.concatenate([U, M], axis=-1)
        dt = O.dt(pw)
        O.step(pw, U, nsteps=3, dt=dt)
        O.step(pp, U2, nsteps=3, dt=dt)
        for f in range(I.NFIELD):
            scale = np.max(np.abs(U2[f])) + 1e-300
            assert np.max(np.abs(U[f] - U2[f][..., :n])) <= 1e-13 * scale, I.FIELDS[f]
