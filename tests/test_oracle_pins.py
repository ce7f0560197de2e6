"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a textbook
scheme it must reduce to, a closed form, a conservation law, a limiting
regime, or the paper's equations solved by a generic root finder.
"""
import os

import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def scalar_advect(u, a, dt, dx, nsteps, axis):
    """Textbook linear advection u_t + a u_x = 0 (a > 0): piecewise-linear
    reconstruction with the monotonised-central limiter, upwind face value and
    Heun's (SSP-RK2) time stepping, periodic."""
    def rhs(u):
        dm = u - np.roll(u, 1, axis)
        dp = np.roll(u, -1, axis) - u
        mag = np.minimum(np.minimum(2 * np.abs(dm), 2 * np.abs(dp)),
                         0.5 * np.abs(dm + dp))
        slope = np.where(dm * dp > 0, np.sign(dm) * mag, 0.0)
        flux = a * (u + 0.5 * slope)
        return -(flux - np.roll(flux, 1, axis)) / dx

    for _ in range(nsteps):
        u1 = u + dt * rhs(u)
        u = 0.5 * (u + u1) + 0.5 * dt * rhs(u1)
    return u


def beam_problem(axis, n_axis=64, n_other=4):
    """Free-streaming beam along `axis` with chi = 0 and c = chat = 1."""
    n = [n_other] * 3
    n[axis] = n_axis
    dx = [1.0 / v for v in n]
    prob = I.base_problem(3, n, dx, c=1.0, chat=1.0)
    sh = (n[2], n[1], n[0])
    coord = I.cell_centres(prob)[axis]
    E = 1e-3 + np.exp(-((coord - 0.3) / 0.05) ** 2) * np.ones(sh)
    U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh), np.zeros((3,) + sh),
                            np.zeros(sh))
    U[I.F_ERAD] = E
    U[I.F_FX + axis] = E  # F = c E: every photon moves along +axis
    return prob, U


# ---------------------------------------------- P1: streaming limit (chi = 0)

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_free_streaming_beam_is_textbook_advection(oracle_mod, axis):
    """With chi = 0 the PD-ARS stages reduce to SSP-RK2 (Sec. 3.2 footnote) and,
    for a beam with F = c E, the M1 closure gives f = 1, D_dd = 1, S = chat and
    the HLL flux is exact upwinding: E must follow the scalar scheme."""
    O = oracle_mod
    prob, U = beam_problem(axis)
    dx = prob["dx"][axis]
    dt = 0.4 * dx
    nsteps = 40
    E0 = U[I.F_ERAD].copy()
    O.step(prob, U, nsteps=nsteps, dt=dt)
    ref = scalar_advect(E0, 1.0, dt, dx, nsteps, axis=2 - axis)
    err = np.abs(U[I.F_ERAD] - ref).max() / np.abs(ref).max()
    assert err < 1e-13, err
    # the beam stays a beam: F = c E, transverse flux and gas untouched
    assert np.abs(U[I.F_FX + axis] - U[I.F_ERAD]).max() < 1e-13
    for d in range(3):
        if d != axis:
            assert np.all(U[I.F_FX + d] == 0.0)
        assert np.all(U[I.F_MX + d] == 0.0)


def test_beam_centroid_moves_at_chat(oracle_mod):
    """Streaming radiation moves at the reduced speed of light."""
    O = oracle_mod
    n = 400
    chat = 2.0
    prob = I.base_problem(1, [n], [1.0 / n], c=4.0, chat=chat)
    x = I.cell_centres(prob)[0].reshape(-1)
    E = 1e-9 + np.exp(-((x - 0.3) / 0.03) ** 2)
    sh = (1, 1, n)
    U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh), np.zeros((3,) + sh),
                            np.zeros(sh))
    U[I.F_ERAD, 0, 0] = E
    U[I.F_FX, 0, 0] = prob["c"] * E
    dt = O.dt(prob)
    nsteps = 200
    O.step(prob, U, nsteps=nsteps)
    w0 = E - 1e-9
    w1 = U[I.F_ERAD, 0, 0] - 1e-9
    shift = (x * w1).sum() / w1.sum() - (x * w0).sum() / w0.sum()
    assert abs(shift / (chat * nsteps * dt) - 1.0) < 1e-3


def test_streaming_second_order_convergence(oracle_mod):
    """IMEX PD-ARS is second-order accurate in the streaming limit (Sec. 1,
    Sec. 3.2): the error of a smooth advected wave falls ~4x per refinement."""
    O = oracle_mod
    errs = []
    for n in (32, 64, 128):
        prob = I.base_problem(1, [n], [1.0 / n], c=1.0, chat=1.0, hll_mode="none")
        x = I.cell_centres(prob)[0].reshape(-1)
        E = 1.0 + 0.5 * np.sin(2 * np.pi * x)
        sh = (1, 1, n)
        U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh),
                                np.zeros((3,) + sh), np.zeros(sh))
        U[I.F_ERAD, 0, 0] = E
        U[I.F_FX, 0, 0] = E
        dt = 0.4 / n
        nsteps = int(round(1.0 / dt))  # one period
        O.step(prob, U, nsteps=nsteps, dt=dt)
        errs.append(np.abs(U[I.F_ERAD, 0, 0] - E).mean())
    order1 = np.log2(errs[0] / errs[1])
    order2 = np.log2(errs[1] / errs[2])
    assert order1 > 1.6 and order2 > 1.6, errs


# -------------------------------------- the M1 closure (Sec. 2.1 leaves it free)

def test_m1_closure_matches_boosted_isotropic_radiation(oracle_mod):
    """The M1 closure is exact for radiation isotropic in a frame moving at
    speed b: f = 4b/(3+b^2), Eddington factor (1+3b^2)/(3+b^2).  Trace 1,
    symmetric, eigenvector F/|F|, transverse eigenvalue (1-xi)/2."""
    O = oracle_mod
    prob = I.base_problem(3, [1, 1, 1], [1, 1, 1], c=3.0, chat=3.0)
    rng = np.random.default_rng(0)
    for b in (0.0, 0.1, 0.5, 0.9, 0.999, 1.0):
        f = 4 * b / (3 + b * b)
        xi = (1 + 3 * b * b) / (3 + b * b)
        E = 2.5
        nhat = rng.standard_normal(3)
        nhat /= np.linalg.norm(nhat)
        F = f * prob["c"] * E * nhat
        D = O.eddington_tensor(prob, E, F)
        assert np.allclose(D, D.T, rtol=0, atol=1e-15)
        assert abs(np.trace(D) - 1.0) < 1e-14
        if b > 0:
            assert np.allclose(D @ nhat, xi * nhat, rtol=0, atol=1e-14)
            t = np.cross(nhat, [1.0, 0.0, 0.0])
            t /= np.linalg.norm(t)
            assert np.allclose(D @ t, 0.5 * (1 - xi) * t, rtol=0, atol=1e-14)
        else:
            assert np.allclose(D, np.eye(3) / 3, rtol=0, atol=1e-16)
    # fluxes above the free-streaming limit are treated as f = 1
    D = O.eddington_tensor(prob, 1.0, [10.0, 0.0, 0.0])
    assert np.allclose(D, np.diag([1.0, 0.0, 0.0]), atol=1e-15)
    De = O.eddington_tensor(dict(prob, closure="eddington"), 1.0, [2.0, 1.0, 0.0])
    assert np.allclose(De, np.eye(3) / 3, atol=0)


# --------------------------------- P2: closed-form local solve (v = 0, F = 0)

def _quartic_T(mp, A, Cv, C):
    """Positive real root of A T^4 + Cv T - C = 0 (unique for A, Cv, C > 0)."""
    roots = mp.polyroots([A, 0, 0, Cv, -C], maxsteps=200, extraprec=200)
    real = [r.real for r in roots if abs(r.imag) < mp.mpf(10) ** -30 * abs(r) and r.real > 0]
    assert len(real) == 1
    return real[0]


@pytest.mark.parametrize("k", [1e-3, 1.0, 1e3, 1e8])
@pytest.mark.parametrize("ratio", [1e-6, 1.0, 1e6])
@pytest.mark.parametrize("chat_frac", [1.0, 0.1])
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_local_solve_equals_energy_quartic(oracle_mod, k, ratio, chat_frac, theta):
    """With v = 0 and F = 0, eq. (egupdate)/(eupdate) with G0 of eq. (G0) give
    Egas = Cv T, E = E0 + R, R = k (aT^4 - E), k = chat chi theta dt, so T is the
    positive root of (c/chat) k a/(1+k) T^4 + Cv T - [Eg0 + (c/chat) k E0/(1+k)]
    and E = (E0 + k a T^4)/(1 + k).  The Newton test of Sec. 3.3 bounds the
    error by ~1e-13 E_tot; we allow 1e-12 E_tot for conditioning."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    O = oracle_mod
    c = 1.0
    chat = chat_frac * c
    prob = I.base_problem(1, [1], [1.0], c=c, chat=chat)
    rho = 1.0
    Cv = rho / (prob["gamma"] - 1.0)
    Eg0 = Cv * 2.0
    E0 = ratio * Eg0
    dt = 1.0
    chi = k / (chat * theta * dt)
    st, y, nn, no = O.local_solve(prob, theta, dt, rho, chi,
                                  [Eg0, 0, 0, 0, E0, 0, 0, 0])
    assert st == 0
    kk = mp.mpf(chat) * mp.mpf(chi) * theta * dt
    cr = mp.mpf(c) / mp.mpf(chat)
    A = cr * kk / (1 + kk)
    C = mp.mpf(Eg0) + cr * kk * mp.mpf(E0) / (1 + kk)
    T = _quartic_T(mp, A, mp.mpf(Cv), C)
    Eg_ex = Cv * T
    E_ex = (E0 + kk * T ** 4) / (1 + kk)
    Etot = Eg0 + (c / chat) * E0
    assert abs(float(y[0] - Eg_ex)) <= 1e-12 * Etot
    assert abs(float((y[4] - E_ex) * cr)) <= 1e-12 * Etot
    assert np.all(y[1:4] == 0) and np.all(y[5:8] == 0)


def test_local_solve_without_coupling_is_identity(oracle_mod):
    """chi = 0: every right-hand side of eq. (egupdate)-(fupdate) vanishes."""
    O = oracle_mod
    prob = I.base_problem(1, [1], [1.0], c=10.0, chat=2.0)
    y0 = [3.0, 0.1, -0.2, 0.3, 7.0, 5.0, -1.0, 2.0]
    st, y, nn, no = O.local_solve(prob, 1.0, 0.3, 1.0, 0.0, y0)
    assert st == 0 and np.array_equal(y, np.array(y0))


# -------------------------------------------------- P3: conservation (Sec. 3.3)

@pytest.mark.parametrize("chat_frac", [1.0, 0.1])
@pytest.mark.parametrize("order", [1, 2])
def test_conservation_periodic_box(oracle_mod, chat_frac, order):
    """Egas + (c/chat) E and m + F/(c chat) are conserved to rounding in a
    periodic box (the energy closure and the momentum update of Sec. 3.3 make
    each cell exact; transport fluxes telescope)."""
    O = oracle_mod
    n = [8, 6, 5]
    prob = I.base_problem(3, n, [1.0 / v for v in n], c=1e3, chat=1e3 * chat_frac,
                          vc_order=order)
    U = I.random_state(prob, seed=11, beta_max=1e-2)
    t0 = O.totals(prob, U)
    O.step(prob, U, nsteps=3)
    t1 = O.totals(prob, U)
    V = np.prod(prob["dx"])
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(U[I.F_MX + d]).sum() + np.abs(U[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= 1e-13 * scale


def test_reflecting_walls_equal_mirrored_periodic_box(oracle_mod):
    """A reflecting wall is a mirror plane: a periodic box of 2n cells holding
    mirror-symmetric data evolves its left half exactly like a reflecting box
    of n cells."""
    O = oracle_mod
    n = 24
    pr = I.base_problem(1, [n], [1.0 / n], bc="reflect", c=1e3, chat=1e3)
    pp = I.base_problem(1, [2 * n], [1.0 / n], bc="periodic", c=1e3, chat=1e3)
    Ur = I.random_state(pr, seed=5, beta_max=1e-2)
    Up = np.zeros(I.shape_of(pp))
    for f in range(I.NFIELD):
        a = Ur[f, 0, 0]
        mirror = a[::-1].copy()
        if f in (I.F_MX, I.F_FX):
            mirror = -mirror
        Up[f, 0, 0] = np.concatenate([a, mirror])
    dt = O.dt(pr)
    O.step(pr, Ur, nsteps=5, dt=dt)
    O.step(pp, Up, nsteps=5, dt=dt)
    assert np.array_equal(Ur[:, 0, 0, :], Up[:, 0, 0, :n])


def test_x_only_data_in_2d_equals_1d(oracle_mod):
    """Transverse faces of data that varies along x only carry no divergence,
    so a 2-D box must reproduce the 1-D run bit for bit (same dt)."""
    O = oracle_mod
    n = 32
    p1 = I.base_problem(1, [n], [1.0 / n], c=1e3, chat=2e2)
    p2 = I.base_problem(2, [n, 3], [1.0 / n, 0.5], c=1e3, chat=2e2)
    U1 = I.random_state(p1, seed=9, beta_max=1e-2)
    for f in (I.F_MY, I.F_MZ, I.F_FY, I.F_FZ):
        U1[f] = 0.0
    U2 = np.ascontiguousarray(np.repeat(U1, 3, axis=2))
    dt = O.dt(p2)
    O.step(p1, U1, nsteps=4, dt=dt)
    O.step(p2, U2, nsteps=4, dt=dt)
    for j in range(3):
        assert np.array_equal(U2[:, :, j, :], U1[:, :, 0, :])


# --------------------------- P4/P5: static diffusion limit (Sec. 2.2, Sec. 4.1)

def _diffusion_run(O, n, chi, t_end, hll_mode="none"):
    """Gaussian E pulse in a uniform thick medium.  Heavy gas (rho = 1e3) with
    a tiny heat capacity (C_v = 1.5e-3 << 4 a T^3) so that the radiation force
    barely moves it and D_eff = c/(3 chi) / (1 + C_v/(4 a T^3)) -> c/(3 chi)."""
    c = 1e3
    rho = 1e3
    prob = I.base_problem(1, [n], [1.0 / n], bc="periodic", c=c, chat=c,
                          kB_over_mu=1e-6, hll_mode=hll_mode)
    x = I.cell_centres(prob)[0].reshape(-1)
    s0 = 0.05
    E0 = 1.0 + np.exp(-((x - 0.5) ** 2) / (2 * s0 ** 2))
    sh = (1, 1, n)
    U = I.equilibrium_state(prob, np.full(sh, rho), (E0 ** 0.25).reshape(sh),
                            np.zeros((3,) + sh), np.full(sh, chi / rho))
    dt = O.dt(prob)
    nsteps = int(round(t_end / dt))
    O.step(prob, U, nsteps=nsteps, dt=dt)
    t = nsteps * dt
    D = prob["c"] / (3.0 * chi)
    s2 = s0 ** 2 + 2 * D * t
    exact = 1.0 + np.sqrt(s0 ** 2 / s2) * np.exp(-((x - 0.5) ** 2) / (2 * s2))
    return prob, U, x, exact, D


def test_static_diffusion_spreads_with_fick_coefficient(oracle_mod):
    """Thick medium with negligible gas heat capacity: E obeys dE/dt =
    D d2E/dx2 with D = c/(3 chi) (eq. diffu, Sec. 5.4), so a Gaussian spreads
    as sigma^2 = sigma0^2 + 2 D t.  The error must be small and shrink as the
    grid is refined."""
    O = oracle_mod
    chi = 1280.0
    t_end = 0.05 ** 2 / (2 * (1e3 / (3 * chi)))  # doubles sigma^2
    errs = []
    for n in (128, 256):
        prob, U, x, exact, D = _diffusion_run(O, n, chi, t_end)
        errs.append(np.abs(U[I.F_ERAD, 0, 0] - exact).max())
    # sigma0 = 6.4 cells at n = 128; the error must fall at least 4x (2nd order)
    assert errs[0] < 2.5e-2 and errs[1] < errs[0] / 4, errs


def test_thick_flux_obeys_ficks_law(oracle_mod):
    """In thick cells the stage flux tends to -c grad E / (3 chi) (eq. f1,
    eq. flux_nhalf) up to O(1/tau)."""
    O = oracle_mod
    chi = 1280.0
    prob, U, x, exact, D = _diffusion_run(O, 128, chi, 2e-3)
    E = U[I.F_ERAD, 0, 0]
    dx = prob["dx"][0]
    grad = (np.roll(E, -1) - np.roll(E, 1)) / (2 * dx)
    fick = -prob["c"] * grad / (3 * chi)
    F = U[I.F_FX, 0, 0]
    # away from the extremum, where the limiter flattens the face slopes
    bulk = np.abs(fick) > 0.2 * np.abs(fick).max()
    assert np.abs(F - fick)[bulk].max() < 0.02 * np.abs(fick).max()


def test_tau_correction_limits(oracle_mod):
    """The optical-depth correction of the HLL energy flux (Sec. 4.3) is 1 in
    thin cells, so it must leave a thin problem unchanged, and in a coarse
    thick problem it must remove numerical diffusion, not add it."""
    O = oracle_mod
    n = 48
    prob = I.base_problem(1, [n], [1.0 / n], c=1e3, chat=1e3, hll_mode="none")
    U = I.random_state(prob, seed=2, tau_range=(1e-19, 1e-18))
    U2 = U.copy()
    O.step(prob, U, nsteps=3)
    O.step(dict(prob, hll_mode="tau"), U2, nsteps=3)
    assert np.array_equal(U, U2)
    # coarse, very thick Gaussian: compare spreading error of both modes
    chi = 2e4
    t_end = 0.05 ** 2 / (2 * (1e3 / (3 * chi)))
    e = {}
    for mode in ("none", "tau"):
        prob, U, x, exact, D = _diffusion_run(O, 40, chi, t_end, hll_mode=mode)
        e[mode] = np.abs(U[I.F_ERAD, 0, 0] - exact).max()
    assert e["tau"] < e["none"]


def _jump_face_energy_flux(O, mode, chi_l, chi_r, dx, axis=0, ndim=1,
                           dxs=None, chat=3.0):
    """Energy flux through the one face where E jumps, F = 0 everywhere.

    E is E_L on the first half of the axis and E_R on the second; the MC
    limiter gives zero slopes next to a step (one of its two differences is
    zero), so both face states are the cell values, F = 0 gives D = I/3 and
    S_R = -S_L = chat/sqrt(3), and the HLL energy flux of Sec. 4.3 is its
    dissipative term alone: eps S_R S_L (E_R - E_L)/(S_R - S_L).  The face
    above the first E_R cell sees uniform data and carries no energy flux,
    so that cell's rate is the jump face's flux divided by dx.  chi is
    chi_l on the left half and chi_r on the right (rho = 1)."""
    n_ax = 8
    n = [1, 1, 1]
    n[axis] = n_ax
    if dxs is None:
        dxs = [dx] * 3
    dxs = list(dxs)
    dxs[axis] = dx
    prob = I.base_problem(ndim, n[:ndim], dxs[:ndim], c=10.0, chat=chat,
                          hll_mode=mode)
    sh = (n[2], n[1], n[0])
    U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh),
                            np.zeros((3,) + sh), np.ones(sh))
    E_l, E_r = 1.0, 5.0
    idx = [slice(None)] * 3
    half = [slice(None)] * 3
    half[2 - axis] = slice(0, n_ax // 2)
    U[I.F_ERAD] = E_r
    U[(I.F_ERAD,) + tuple(half)] = E_l
    U[I.F_KAPPA] = chi_r
    U[(I.F_KAPPA,) + tuple(half)] = chi_l
    for d in range(3):
        U[I.F_FX + d] = 0.0
    rate = O.transport(prob, U)[0]
    idx[2 - axis] = n_ax // 2
    j = tuple(i if isinstance(i, int) else 0 for i in idx)
    flux = rate[j] * dx            # rate = -(0 - flux)/dx
    # the NONE flux of this face, from the formula (eps = 1)
    none = -chat / np.sqrt(3.0) * (E_r - E_l) / 2.0
    return flux, none


def test_tau_factor_thin_and_thick_limits(oracle_mod):
    """Sec. 4.3: the factor on the energy-flux dissipation goes to 1 in thin
    faces and to 1/tau in thick ones, tau the face's optical depth.  With the
    face's dissipative term isolated, tau * eps -> 1 for tau >> 1 and
    eps -> 1 for tau << 1; doubling chi on both sides of a thick face halves
    the term.  NONE carries exactly the formula's flux."""
    O = oracle_mod
    dx = 1.0 / 8
    f_none, ref = _jump_face_energy_flux(O, "none", 400.0, 400.0, dx)
    assert abs(f_none / ref - 1.0) < 1e-14
    for chi in (200.0, 800.0, 8e4):           # tau = chi dx = 25 .. 1e4
        tau = chi * dx
        f_tau, ref = _jump_face_energy_flux(O, "tau", chi, chi, dx)
        assert abs(f_tau * tau / ref - 1.0) < 1e-3, (chi, f_tau * tau / ref)
        f_2, _ = _jump_face_energy_flux(O, "tau", 2 * chi, 2 * chi, dx)
        assert abs(f_2 / f_tau - 0.5) < 1e-3
    for chi in (8e-6, 8e-8):                  # tau = 1e-6, 1e-8
        f_tau, ref = _jump_face_energy_flux(O, "tau", chi, chi, dx)
        assert abs(f_tau / ref - 1.0) < 2 * chi * dx
    # between the limits eps falls monotonically from 1 towards 1/tau
    epss = [_jump_face_energy_flux(O, "tau", t / dx, t / dx, dx)[0] / ref
            for t in (1e-3, 0.1, 1.0, 3.0, 10.0)]
    assert all(0 < b < a <= 1 for a, b in zip(epss, epss[1:]))


def test_tau_factor_face_optical_depth(oracle_mod):
    """The face's optical depth is the mean of its two cells' chi times the
    cell width along the face normal, tau = (chi_L + chi_R) dx_d / 2: with a
    contrast chi_L != chi_R a thick face's term is 1/tau of NONE's for that
    tau (a one-sided chi, a dropped 1/2 or a dropped dx each miss it by a
    factor >= 1.5), halving dx at fixed chi halves tau, and in 3-D each
    axis takes its own dx."""
    O = oracle_mod
    dx = 1.0 / 8
    for chi_l, chi_r in ((400.0, 1200.0), (1200.0, 400.0), (100.0, 2900.0)):
        tau = 0.5 * (chi_l + chi_r) * dx
        f_tau, ref = _jump_face_energy_flux(O, "tau", chi_l, chi_r, dx)
        assert abs(f_tau * tau / ref - 1.0) < 1e-3, (chi_l, chi_r, f_tau * tau / ref)
    chi = 800.0
    f1, ref = _jump_face_energy_flux(O, "tau", chi, chi, dx)
    f2, ref2 = _jump_face_energy_flux(O, "tau", chi, chi, dx / 2)
    assert ref == ref2
    assert abs(f2 / f1 - 2.0) < 2e-3          # eps = 1/tau doubles
    dxs = [1.0 / 8, 1.0 / 32, 1.0 / 128]
    for axis in range(3):
        chi_l, chi_r = 3000.0, 9000.0
        tau = 0.5 * (chi_l + chi_r) * dxs[axis]
        f_tau, ref = _jump_face_energy_flux(O, "tau", chi_l, chi_r, dxs[axis],
                                            axis=axis, ndim=3, dxs=dxs)
        assert abs(f_tau * tau / ref - 1.0) < 1e-3, (axis, f_tau * tau / ref)


# ------------------------------ P6: uniform advecting medium (Sec. 5.5, Table 1)

def _uniform(order, beta, closure="m1", tau_cell=1e3, c=1e3, ratio=1.0):
    n = 8
    prob = I.base_problem(1, [n], [1.0 / n], c=c, chat=c, vc_order=order,
                          closure=closure)
    sh = (1, 1, n)
    v = np.zeros((3,) + sh)
    v[0] = beta * c
    Cv = 1.0 / (prob["gamma"] - 1.0)
    T = np.ones(sh)
    # radiation-to-gas energy ratio aT^4/(Cv T) = ratio  ->  a = ratio * Cv
    prob["a_rad"] = ratio * Cv
    U = I.equilibrium_state(prob, np.ones(sh), T, v, np.full(sh, tau_cell * n))
    return prob, U


def test_uniform_medium_has_zero_transport(oracle_mod):
    O = oracle_mod
    prob, U = _uniform(2, 1e-2)
    assert np.all(O.transport(prob, U) == 0.0)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("beta", [1e-3, 1e-2])
def test_uniform_medium_solve_matches_implicit_system(oracle_mod, order, beta):
    """One implicit solve of the advected equilibrium (Sec. 5.5) against the
    8 implicit equations (egupdate)-(fupdate) solved by a generic root finder,
    with the four-force of eq. (G0), (G1) kept to the v/c order in use."""
    O = oracle_mod
    prob, U = _uniform(order, beta, closure="eddington")
    rho = 1.0
    chi = U[I.F_KAPPA, 0, 0, 0] * rho
    dt = O.dt(prob)
    y0 = [U[f, 0, 0, 0] for f in (I.F_EGAS, I.F_MX, I.F_MY, I.F_MZ, I.F_ERAD,
                                  I.F_FX, I.F_FY, I.F_FZ)]
    _check_against_root_finder(O, prob, 1.0, dt, rho, chi, y0, order)


def _table1_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table1_uniform_advection.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                b, bt, o, e = line.split()
                rows.append((float(b), float(bt), int(o), float(e)))
    return rows


def test_uniform_medium_drift_pattern_of_table1(oracle_mod):
    """Table 1's pattern: with the order-matched initial state the temperature
    drift of the advected uniform medium is O(beta^2) at v/c order 1 and
    O(beta^4) at order 2 (the four-force of the order-2 state vanishes to
    O(v^4/c^4), Sec. 5.5)."""
    O = oracle_mod
    rows = _table1_rows()
    assert len(rows) == 3
    beta = max(r[0] for r in rows)

    def drift(order, b):
        prob, U = _uniform(order, b, tau_cell=rows[1][1] / rows[1][0] / 8)
        Cv = 1.0 / (prob["gamma"] - 1.0)
        T0 = (U[I.F_EGAS] - 0.5 * U[I.F_MX] ** 2) / Cv
        O.step(prob, U, nsteps=2)
        T1 = (U[I.F_EGAS] - 0.5 * U[I.F_MX] ** 2 / U[I.F_RHO]) / Cv
        return float(np.abs(T1 / T0 - 1.0).max())

    d1, d1b = drift(1, beta), drift(1, 2 * beta)
    d2, d2b = drift(2, beta), drift(2, 2 * beta)
    assert abs(d1b / d1 / 4.0 - 1.0) < 0.05
    assert abs(d2b / d2 / 16.0 - 1.0) < 0.05
    assert d2 < 10 * beta ** 2 * d1


# ---------------------- P8: the paper's implicit equations, solved independently

def _G_general(mp, chiP, chiE, chiF, aT4, E, F, v, P, c, order=2):
    """Radiation four-force of eq. (G0), (G1) to O(v^2/c^2) (order 2), or to
    O(v/c) (order 1: the (1 + beta^2/2) factors and the O(v^2/c^2) terms of
    the non-grey parts dropped, as eq. numF1 does); returns (cG0, G)."""
    o2 = 1 if order == 2 else 0
    b2 = sum(vi * vi for vi in v) / c ** 2 * o2
    vF = sum(v[i] * F[i] for i in range(3))
    vvP = sum(v[i] * v[j] * P[i][j] for i in range(3) for j in range(3)) * o2
    minus_cG0 = (c * (chiP * aT4 - chiE * E) * (1 + b2 / 2) + (2 * chiE - chiF) * vF / c
                 + c * (chiF - chiE) * (b2 * E + vvP / c ** 2))
    G = []
    for i in range(3):
        vP = sum(v[j] * P[j][i] for j in range(3))
        minus_Gi = (-chiF * F[i] / c * (1 + b2 / 2) + chiP * aT4 * v[i] / c
                    + chiF * vP / c + (chiF - chiE) * (E - 2 * o2 * vF / c ** 2) * v[i] / c)
        G.append(-minus_Gi)
    return -minus_cG0, G


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("chat_frac", [1.0, 0.1])
def test_energy_equations_hold_at_solution(oracle_mod, theta, chat_frac):
    """After a local solve, eq. (egupdate) and (eupdate) with G0 of eq. (G0)
    evaluated at the final state must hold to the convergence tolerances of
    Sec. 3.3 (inner 1e-13 E_tot, outer 1e-13 of the v,F terms)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    O = oracle_mod
    n = [6, 5, 4]
    prob = I.base_problem(3, n, [1.0 / v for v in n], c=1e3, chat=1e3 * chat_frac)
    U = I.random_state(prob, seed=21, beta_max=1e-2)
    dt = O.dt(prob)
    c, chat, a = mp.mpf(prob["c"]), mp.mpf(prob["chat"]), mp.mpf(prob["a_rad"])
    worst = 0.0
    for idx in np.ndindex(U.shape[1:]):
        rho = U[(I.F_RHO,) + idx]
        chi = U[(I.F_KAPPA,) + idx] * rho
        y0 = [U[(f,) + idx] for f in (I.F_EGAS, I.F_MX, I.F_MY, I.F_MZ, I.F_ERAD,
                                      I.F_FX, I.F_FY, I.F_FZ)]
        st, y, nn, no = O.local_solve(prob, theta, dt, rho, chi, y0)
        assert st == 0
        Cv = mp.mpf(rho) / (mp.mpf(prob["gamma"]) - 1)
        m = [mp.mpf(y[1 + i]) for i in range(3)]
        v = [mi / rho for mi in m]
        T = (mp.mpf(y[0]) - sum(mi * mi for mi in m) / (2 * rho)) / Cv
        F = [mp.mpf(y[5 + i]) for i in range(3)]
        zero3 = [[0] * 3] * 3
        cG0, _ = _G_general(mp, chi, chi, chi, a * T ** 4, mp.mpf(y[4]), F, v, zero3, c)
        Etot = y0[0] + (prob["c"] / prob["chat"]) * y0[4]
        rg = mp.mpf(y[0]) - y0[0] - cG0 * theta * dt
        re = (mp.mpf(y[4]) - y0[4] + (chat / c) * cG0 * theta * dt) * c / chat
        # The inner test bounds F_G and (c/chat) F_R by 1e-13 E_tot; G0 taken
        # again at the final E multiplies the F_R part by k g = theta dt chat
        # chi (1 + beta^2/2), k g <= 1.01 k here.
        k = prob["chat"] * chi * theta * dt
        bound = 3e-13 * (1.0 + 1.01 * k) * Etot
        worst = max(worst, float(abs(rg)) / bound, float(abs(re)) / bound)
    assert worst < 1.0, worst


def _check_against_root_finder(O, prob, theta, dt, rho, chi, y0, order=2):
    """Solve eq. (egupdate)-(fupdate) (Eddington closure) with mpmath's
    findroot and compare with the oracle's local solve; chi is chi_0E and the
    problem's kappa ratios give chi_0P and chi_0F."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    st, y, nn, no = O.local_solve(prob, theta, dt, rho, chi, y0)
    assert st == 0
    c = mp.mpf(prob["c"])
    chat = mp.mpf(prob["chat"])
    a = mp.mpf(prob["a_rad"])
    tdt = mp.mpf(theta) * dt
    Cvm = mp.mpf(rho) * mp.mpf(prob["kB_over_mu"]) / (mp.mpf(prob["gamma"]) - 1)

    def eqs(*x):
        Eg, m1, m2, m3, E, F1, F2, F3 = x
        mm = [m1, m2, m3]
        FF = [F1, F2, F3]
        v = [mi / rho for mi in mm]
        T = (Eg - sum(mi * mi for mi in mm) / (2 * rho)) / Cvm
        P = [[E / 3 if i == j else 0 for j in range(3)] for i in range(3)]
        rP = mp.mpf(prob.get("kappa_P_ratio", 1.0))
        rF = mp.mpf(prob.get("kappa_F_ratio", 1.0))
        cG0, G = _G_general(mp, rP * chi, chi, rF * chi, a * T ** 4, E, FF, v, P, c, order)
        out = [Eg - y0[0] - cG0 * tdt, E - y0[4] + (chat / c) * cG0 * tdt]
        out += [mm[i] - y0[1 + i] - G[i] * tdt for i in range(3)]
        out += [FF[i] - y0[5 + i] + chat * c * G[i] * tdt for i in range(3)]
        return out

    sol = mp.findroot(eqs, [mp.mpf(v) for v in y], tol=mp.mpf(10) ** -25)
    sol = [float(s) for s in sol]
    Fs = np.abs(y0[5:8]).max() + 1e-300
    ms = np.abs(y0[1:4]).max() + Fs / (prob["c"] * prob["chat"])
    Etot = y0[0] + prob["c"] / prob["chat"] * y0[4]
    assert abs(y[0] - sol[0]) <= 1e-12 * Etot
    assert abs(y[4] - sol[4]) * prob["c"] / prob["chat"] <= 1e-12 * Etot
    for i in range(3):
        assert abs(y[5 + i] - sol[5 + i]) <= 1e-11 * Fs
        assert abs(y[1 + i] - sol[1 + i]) <= 1e-11 * ms


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_full_implicit_system_by_generic_root_finder(oracle_mod, theta):
    """eq. (egupdate)-(fupdate) form 8 equations in 8 unknowns.  Solved by a
    generic multidimensional root finder (Eddington closure P = E I/3, heavy
    gas so the outer iteration's lag is negligible) they must agree with the
    oracle's inner/outer solve, flux and momentum included."""
    O = oracle_mod
    prob = I.base_problem(1, [1], [1.0], c=10.0, chat=10.0, closure="eddington",
                          a_rad=1e4)
    rng = np.random.default_rng(4)
    for trial in range(6):
        rho = 1e6
        Cv = rho / (prob["gamma"] - 1)
        T0 = 10 ** rng.uniform(0, 1)
        v0 = rng.uniform(-1, 1, 3) * 0.05 * prob["c"]
        E0 = prob["a_rad"] * (10 ** rng.uniform(0, 1)) ** 4
        F0 = rng.uniform(-1, 1, 3) * 0.3 * prob["c"] * E0
        Eg0 = Cv * T0 + 0.5 * rho * (v0 ** 2).sum()
        y0 = [Eg0, *(rho * v0), E0, *F0]
        chi = 10 ** rng.uniform(-1, 2)
        _check_against_root_finder(O, prob, theta, 0.1, rho, chi, y0)


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("delta", [1e-4, 1e-8, 0.0])
def test_outer_stop_with_cancelling_exchange_terms(oracle_mod, theta, delta):
    """The outer iteration stops on the change of Q, the part of the exchange
    that depends on v and F (Sec. 3.3).  With v = (u, u, 0) and F = (f,
    -f (1 - delta), 0), v.F cancels to a fraction delta of its terms and
    radiation starts in equilibrium, so Q is far smaller than its terms.
    The solve must still stop within a few passes (the cap is 32) and on the
    root of eq. (egupdate)-(fupdate) that a generic root finder gives: a stop
    taken on rounding noise of the cancelled Q would leave F and m off that
    root.  (Here |R| is large enough that the paper's own two tests stop
    too: a copy of the oracle without the test against the terms' magnitude
    takes the same passes.)"""
    O = oracle_mod
    prob = I.base_problem(1, [1], [1.0], c=10.0, chat=10.0, closure="eddington",
                          a_rad=1e4)
    rho = 1e6
    Cv = rho / (prob["gamma"] - 1)
    T0 = 3.0
    E0 = prob["a_rad"] * T0 ** 4
    u, f = 0.05 * prob["c"], 0.3 * prob["c"] * E0
    v0 = np.array([u, u, 0.0])
    F0 = np.array([f, -f * (1.0 - delta), 0.0])
    y0 = [Cv * T0 + 0.5 * rho * (v0 ** 2).sum(), *(rho * v0), E0, *F0]
    for chi in (0.1, 10.0, 100.0):
        st, _, _, n_outer = O.local_solve(prob, theta, 0.1, rho, chi, y0)
        assert st == 0 and n_outer <= 10
        _check_against_root_finder(O, prob, theta, 0.1, rho, chi, y0)


@pytest.mark.parametrize("order", [2, 1])
@pytest.mark.parametrize("rP,rF", [(0.5, 0.3), (3.0, 1.5), (1.0, 4.0)])
def test_nongrey_implicit_system_by_generic_root_finder(oracle_mod, order, rP, rF):
    """Non-grey material (chi_0P = rP chi_0E, chi_0F = rF chi_0E): the oracle's
    solve -- eq. (Rnew) with every (chi_0F - chi_0E) term, the 3 x 3 flux
    update that eq. (G1)'s v (v.F) term makes of eq. (fupdate) at
    O(v^2/c^2), eq. (numF1) at O(v/c) -- against eq. (egupdate)-(fupdate)
    with the four-force of eq. (G0)/(G1) solved by a generic root finder.
    (chi_0F = 2 chi_0E is avoided: at O(v/c) eq. (Rnew) then has no term in v
    or F, the outer test of Sec. 3.3 stops after one pass and m keeps the
    lagged velocity.)"""
    O = oracle_mod
    prob = I.base_problem(1, [1], [1.0], c=10.0, chat=10.0, closure="eddington",
                          a_rad=1e4, kappa_P_ratio=rP, kappa_F_ratio=rF, vc_order=order,
                          newton_max_iter=400, outer_max_iter=200)
    # at beta = 0.05 the paper's lagged outer iteration converges slowly for
    # non-grey material (up to 84 passes here): the cap is raised
    rng = np.random.default_rng(44)
    for trial in range(4):
        rho = 1e6
        Cv = rho / (prob["gamma"] - 1)
        T0 = 10 ** rng.uniform(0, 1)
        v0 = rng.uniform(-1, 1, 3) * 0.05 * prob["c"]
        E0 = prob["a_rad"] * (10 ** rng.uniform(0, 1)) ** 4
        F0 = rng.uniform(-1, 1, 3) * 0.3 * prob["c"] * E0
        Eg0 = Cv * T0 + 0.5 * rho * (v0 ** 2).sum()
        y0 = [Eg0, *(rho * v0), E0, *F0]
        chi = 10 ** rng.uniform(-1, 2)
        _check_against_root_finder(O, prob, 1.0, 0.1, rho, chi, y0, order=order)


@pytest.mark.parametrize("rP,rF", [(0.5, 0.3), (3.0, 2.0)])
def test_nongrey_conservation_periodic_box(oracle_mod, rP, rF):
    """The energy closure and the momentum update conserve sum(Egas + (c/chat)
    E) and sum(m + F/(c chat)) whatever the opacities (Sec. 3.3)."""
    O = oracle_mod
    prob = I.base_problem(2, [12, 10], [1 / 12, 1 / 10], c=1e3, chat=1e2,
                          kappa_P_ratio=rP, kappa_F_ratio=rF)
    U = I.random_state(prob, seed=17, beta_max=1e-2)
    t0 = O.totals(prob, U)
    O.step(prob, U, 5)
    t1 = O.totals(prob, U)
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    scale = np.abs(U[I.F_MX:I.F_MZ + 1]).sum() + np.abs(U[I.F_FX:I.F_FZ + 1]).sum() / (1e3 * 1e2)
    assert np.max(np.abs(t1[1:] - t0[1:])) <= 1e-13 * scale / U[0].size
