"""Pins of the oracle's adjoint (reverse-mode derivative of one IMEX step).

The adjoint is checked against things other than itself: central finite
differences of the forward oracle, the conservation laws of Sec. 3.3 (whose
totals are exact left null-vectors of the step's Jacobian), and the closed-form
derivative of the local solve's energy quartic.

Finite differences use per-cell relative perturbations.  The step is only
piecewise smooth (the slope limiter, the max in the HLL speed and the flux
rescale have kinks), so a difference step that straddles a kink is off by a
term proportional to the step; single steps use a step small enough that the
seeded cases straddle none, trajectories the best of a short ladder.
"""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I


def _slots(O):
    return list(O.SLOT_INDEX)


def _fd_directional(O, prob, U, D, W, h, dt):
    """Central difference of sum(W * y(n+1)) along the state direction D."""
    vals = []
    for sgn in (1.0, -1.0):
        V = U + sgn * h * D
        O.step(prob, V, 1, dt)
        vals.append(sum((W[k] * V[i]).sum() for k, i in enumerate(_slots(O))))
    return (vals[0] - vals[1]) / (2.0 * h)


CASES = [(ndim, bc, hll, clo, order)
         for ndim in (1, 2, 3)
         for bc in ("periodic", "reflect")
         for hll in ("tau", "none")
         for clo in ("m1", "eddington")
         for order in (2, 1)]


@pytest.mark.parametrize("ndim,bc,hll,clo,order", CASES)
def test_step_adjoint_matches_central_differences(oracle_mod, ndim, bc, hll, clo, order):
    """<W, J D> from the adjoint equals the central difference of the forward
    oracle along D, for random out-of-equilibrium states with every transport
    and exchange term active (Sec. 3.2 stages, Sec. 3.3 transport and solve)."""
    O = oracle_mod
    n = {1: (16,), 2: (8, 6), 3: (5, 4, 6)}[ndim]
    ci = CASES.index((ndim, bc, hll, clo, order))
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), c=1e3,
                          chat=1e3 if ci % 2 else 1e2, bc=bc, hll_mode=hll,
                          closure=clo, vc_order=order)
    U = I.random_state(prob, seed=100 + ci, tau_range=(1e-2, 1e2))
    dt = O.dt(prob)
    rng = np.random.default_rng(ci)
    U1 = U.copy()
    tape = O.step_tape(prob, U1, dt)
    live = np.array([np.abs(U[i]).max() > 0 for i in _slots(O)], dtype=float)
    mag = np.array([np.abs(U[i]).max() for i in _slots(O)]) + 1e-300
    W = rng.standard_normal(tape[2].shape) * (live / mag)[:, None, None, None]
    kbar = np.zeros_like(U[0])
    ybar = O.step_adjoint(prob, U[I.F_RHO], U[I.F_KAPPA], tape, W, kbar, dt)
    D = np.zeros_like(U)
    for k, i in enumerate(_slots(O)):
        D[i] = rng.standard_normal(U[0].shape) * np.abs(U[i]) * live[k]
    D[I.F_KAPPA] = rng.standard_normal(U[0].shape) * U[I.F_KAPPA]
    lin = sum((ybar[k] * D[i]).sum() for k, i in enumerate(_slots(O))) + (kbar * D[I.F_KAPPA]).sum()
    fd = _fd_directional(O, prob, U, D, W, 1e-6, dt)
    assert abs(lin - fd) <= 1e-6 * abs(fd), (lin, fd)


def test_taped_step_equals_plain_step(oracle_mod):
    O = oracle_mod
    prob = I.base_problem(2, (8, 6), (1 / 8, 1 / 6), c=1e3, chat=1e2)
    U = I.random_state(prob, seed=3)
    A = U.copy()
    B = U.copy()
    tape = O.step_tape(prob, A, 0.0)
    O.step(prob, B, 1, 0.0)
    assert np.array_equal(A, B)
    assert np.array_equal(tape[0], U[_slots(O)])
    assert np.array_equal(tape[2], B[_slots(O)])


@pytest.mark.parametrize("bc", ["periodic", "reflect"])
@pytest.mark.parametrize("chat_frac", [1.0, 0.1])
def test_conserved_energy_is_a_left_null_vector(oracle_mod, bc, chat_frac):
    """Sec. 3.3: the step conserves sum(Egas + (c/chat) E) exactly (the energy
    closure and the telescoping fluxes; a reflecting wall passes no energy),
    so the adjoint maps the constant cotangent (1, 0, 0, 0, c/chat, 0, 0, 0)
    to itself and gives no opacity gradient."""
    O = oracle_mod
    c = 1e3
    prob = I.base_problem(2, (8, 7), (1 / 8, 1 / 7), c=c, chat=chat_frac * c, bc=bc)
    U = I.random_state(prob, seed=11)
    tape = O.step_tape(prob, U.copy(), 0.0)
    W = np.zeros_like(tape[2])
    W[0] = 1.0
    W[4] = 1.0 / chat_frac
    kbar = np.zeros_like(U[0])
    ybar = O.step_adjoint(prob, U[I.F_RHO], U[I.F_KAPPA], tape, W, kbar, 0.0)
    assert np.max(np.abs(ybar - W)) <= 1e-11 * np.max(np.abs(W))
    # dL/dkappa is zero up to the rounding of the per-cell terms
    scale = np.abs(U[I.F_EGAS]).max() / np.abs(U[I.F_KAPPA]).min()
    assert np.max(np.abs(kbar)) <= 1e-10 * scale


@pytest.mark.parametrize("axis", [0, 1])
def test_conserved_momentum_is_a_left_null_vector(oracle_mod, axis):
    """Sec. 3.3: in a periodic box sum(m + F/(c chat)) is conserved (momentum
    update and telescoping fluxes), so its cotangent maps to itself."""
    O = oracle_mod
    c = 1e3
    prob = I.base_problem(2, (8, 7), (1 / 8, 1 / 7), c=c, chat=0.1 * c)
    U = I.random_state(prob, seed=12)
    tape = O.step_tape(prob, U.copy(), 0.0)
    W = np.zeros_like(tape[2])
    W[1 + axis] = 1.0
    W[5 + axis] = 1.0 / (c * prob["chat"])
    kbar = np.zeros_like(U[0])
    ybar = O.step_adjoint(prob, U[I.F_RHO], U[I.F_KAPPA], tape, W, kbar, 0.0)
    assert np.max(np.abs(ybar - W)) <= 1e-12
    scale = np.abs(U[I.F_FX]).max() / (c * prob["chat"]) / np.abs(U[I.F_KAPPA]).min()
    assert np.max(np.abs(kbar)) <= 1e-10 * scale


@pytest.mark.parametrize("k", [1e-3, 1.0, 1e3])
@pytest.mark.parametrize("ratio", [1e-3, 1.0, 1e3])
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_local_solve_adjoint_equals_quartic_derivatives(oracle_mod, k, ratio, theta):
    """v = 0, F = 0: the solve's T is the root of A T^4 + Cv T = C with
    A = (c/chat) k a/(1+k), C = Eg0 + (c/chat) k E0/(1+k), k = chat chi theta dt,
    and E = (E0 + k a T^4)/(1+k).  Differentiating the quartic gives
    dT/dq = (dC/dq - T^4 dA/dq)/(4 A T^3 + Cv) for q in (Eg0, E0, chi); the
    adjoint of the solve must reproduce these to the solve's tolerance."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    O = oracle_mod
    c, chat = 1.0, 0.5
    prob = I.base_problem(1, [1], [1.0], c=c, chat=chat)
    rho = 1.0
    Cv = rho / (prob["gamma"] - 1.0)
    Eg0 = 2.0 * Cv
    E0 = ratio * Eg0
    dt = 1.0
    chi = k / (chat * theta * dt)
    st, y, _, _ = O.local_solve(prob, theta, dt, rho, chi, [Eg0, 0, 0, 0, E0, 0, 0, 0])
    assert st == 0

    cr = mp.mpf(c) / chat
    kk = mp.mpf(k)
    dk_dchi = mp.mpf(chat) * theta * dt
    A = cr * kk / (1 + kk)
    C = mp.mpf(Eg0) + cr * kk * E0 / (1 + kk)
    roots = mp.polyroots([A, 0, 0, Cv, -C], maxsteps=200, extraprec=200)
    T = [r.real for r in roots if abs(r.imag) < mp.mpf(10) ** -30 and r.real > 0][0]
    den = 4 * A * T ** 3 + Cv
    dA_dk = cr / (1 + kk) ** 2
    dC_dk = cr * E0 / (1 + kk) ** 2
    dT = {"Eg0": 1 / den, "E0": cr * kk / (1 + kk) / den,
          "chi": (dC_dk - T ** 4 * dA_dk) / den * dk_dchi}
    # E = (E0 + k T^4)/(1 + k)
    dE = {"Eg0": kk * 4 * T ** 3 * dT["Eg0"] / (1 + kk),
          "E0": (1 + kk * 4 * T ** 3 * dT["E0"]) / (1 + kk),
          "chi": dk_dchi * ((T ** 4 * (1 + kk) - (E0 + kk * T ** 4)) / (1 + kk) ** 2)
          + kk * 4 * T ** 3 * dT["chi"] / (1 + kk)}
    for out_slot, exact in ((0, {q: Cv * dT[q] for q in dT}), (4, dE)):
        b = np.zeros(8)
        b[out_slot] = 1.0
        st, bin_, chibar = O.local_solve_adjoint(prob, theta, dt, rho, chi, y, b)
        assert st == 0
        got = {"Eg0": bin_[0], "E0": bin_[4], "chi": chibar}
        for q in ("Eg0", "E0"):
            assert abs(got[q] - float(exact[q])) <= 1e-10 * max(1.0, abs(float(exact[q])))
        # chi-derivative relative to its natural scale (dE/dk ~ E)
        sc = float(abs(exact["chi"])) + 1e-12 * (Eg0 + E0) * float(dk_dchi)
        assert abs(got["chi"] - float(exact["chi"])) <= 1e-9 * sc


def test_local_solve_adjoint_matches_central_differences(oracle_mod):
    """Random cells with v, F != 0 (every O(v/c) term of eq. (Rnew) and
    (numF2) active): <w, dy_out> from the adjoint equals the central
    difference of the oracle's solve along random input directions."""
    O = oracle_mod
    rng = np.random.default_rng(21)
    worst = 0.0
    for case in range(40):
        c = 1e3
        chat = [1e3, 1e2][case % 2]
        prob = I.base_problem(1, [1], [1.0], c=c, chat=chat,
                              closure=["m1", "eddington"][(case // 2) % 2],
                              vc_order=[2, 1][(case // 4) % 2])
        rho = 10 ** rng.uniform(-0.5, 0.5)
        T = 10 ** rng.uniform(0, 0.5)
        Tr = 10 ** rng.uniform(0, 0.5)
        v = rng.uniform(-1, 1, 3) * 1e-2 * c
        E0 = Tr ** 4
        F0 = rng.standard_normal(3)
        F0 *= rng.uniform(0.05, 0.6) * c * E0 / np.linalg.norm(F0)
        y0 = np.array([1.5 * rho * T + 0.5 * rho * v @ v, *(rho * v), E0, *F0])
        chi = 10 ** rng.uniform(-2, 3)
        theta, dt = [1.0, 0.5][case % 2], 1e-3
        st, y, _, _ = O.local_solve(prob, theta, dt, rho, chi, y0)
        assert st == 0
        w = rng.standard_normal(8) / (np.abs(y) + 1e-3 * np.abs(y).max())
        st, bin_, chibar = O.local_solve_adjoint(prob, theta, dt, rho, chi, y, w)
        assert st == 0
        dy = rng.standard_normal(8) * np.abs(y0)
        dchi = rng.standard_normal() * chi
        lin = bin_ @ dy + chibar * dchi
        h = 1e-6
        vals = []
        for s in (1, -1):
            st2, ys, _, _ = O.local_solve(prob, theta, dt, rho, chi + s * h * dchi, y0 + s * h * dy)
            assert st2 == 0
            vals.append(w @ ys)
        fd = (vals[0] - vals[1]) / (2 * h)
        worst = max(worst, abs(lin - fd) / (abs(fd) + 1e-300))
    assert worst <= 1e-6, worst


# Relative difference steps for trajectories.  Over many steps some limiter,
# maximum or clip sits within h of its switch somewhere, and a central
# difference straddling a switch is off by a term proportional to h; smaller
# steps reach the rounding floor of the converged solves (~1e-13 / h).  The
# check takes the best of a short ladder of steps.
FD_STEPS = (1e-6, 3e-7, 1e-7, 3e-8)


def test_trajectory_gradient_matches_central_differences(oracle_mod):
    """The differentiation workload (pulse through a log-normal opacity field,
    L = sum (E - E_tgt)^2) on a 32^2 grid over 20 steps: the gradient with
    respect to the initial temperature and log opacity agrees with central
    differences along random directions to 1e-6."""
    O = oracle_mod
    prob, T0, lk, Et, _ = I.pulse_inverse_problem_2d(32)
    nsteps = 20
    dt = O.dt(prob)
    cv = prob["kB_over_mu"] / (prob["gamma"] - 1.0)
    a = prob["a_rad"]

    def loss(T, lk_):
        U = I.rest_state(prob, T, lk_)
        O.step(prob, U, nsteps, dt)
        return float(((U[I.F_ERAD] - Et) ** 2).sum())

    def loss_grad(Uf):
        r = Uf[I.F_ERAD] - Et
        yb = np.zeros((8,) + Uf.shape[1:])
        yb[4] = 2.0 * r
        return float((r * r).sum()), yb

    U0 = I.rest_state(prob, T0, lk)
    L, ybar, kbar = O.trajectory_gradient(prob, U0, nsteps, loss_grad, dt)
    assert L == pytest.approx(loss(T0, lk), rel=1e-15)
    gT = ybar[0] * cv + ybar[4] * 4.0 * a * T0 ** 3
    glk = kbar * np.exp(lk)
    rng = np.random.default_rng(2)
    for _ in range(2):
        dT = rng.standard_normal(T0.shape) * T0
        dk = rng.standard_normal(lk.shape)
        for vec_T, vec_k in ((dT, 0 * dk), (0 * dT, dk)):
            lin = float((gT * vec_T).sum() + (glk * vec_k).sum())
            errs = []
            for h in FD_STEPS:
                fd = (loss(T0 + h * vec_T, lk + h * vec_k) -
                      loss(T0 - h * vec_T, lk - h * vec_k)) / (2 * h)
                errs.append(abs(lin - fd) / abs(fd))
            assert min(errs) <= 1e-6, errs



@pytest.mark.parametrize("tau_cell", [1e-4, 1e-3, 0.03, 0.049, 0.051, 0.3])
def test_opacity_gradient_across_the_tau_series_switch(oracle_mod, tau_cell):
    """TAU mode with optical depths on both sides of the switch between the
    Taylor series (below tau = 0.05, where the closed form cancels) and the
    closed form (e^-tau (1 + tau) - 1)/tau^2 of d eps/d tau: dL/dkappa of one step
    equals central differences in kappa, cell by cell."""
    O = oracle_mod
    n = 12
    prob = I.base_problem(1, (n,), (1.0 / n,), c=1e3, chat=1e3, hll_mode="tau")
    U = I.random_state(prob, seed=31, tau_range=(tau_cell, tau_cell * 1.0001))
    dt = O.dt(prob)
    tape = O.step_tape(prob, U.copy(), dt)
    rng = np.random.default_rng(5)
    W = np.zeros_like(tape[2])
    W[4] = rng.standard_normal(W[4].shape) / np.abs(U[I.F_ERAD]).max()
    kbar = np.zeros_like(U[0])
    O.step_adjoint(prob, U[I.F_RHO], U[I.F_KAPPA], tape, W, kbar, dt)
    for i in range(0, n, 3):
        h = 1e-4 * U[I.F_KAPPA].flat[i]  # smooth in kappa; larger step, less rounding
        vals = []
        for sgn in (1.0, -1.0):
            V = U.copy()
            V[I.F_KAPPA].flat[i] += sgn * h
            O.step(prob, V, 1, dt)
            vals.append((W[4] * V[I.F_ERAD]).sum())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(kbar.flat[i] - fd) <= 1e-6 * abs(fd) + 1e-12 * np.abs(kbar).max(), \
            (i, kbar.flat[i], fd)
