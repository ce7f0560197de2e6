"""GPU adjoint (rhd_step_record, rhd_adjoint and the IMEXTrajectory autograd
Function) against the oracle's adjoint and against central differences of the
GPU forward step.

Element-by-element cases differentiate both sides at the same states: the
oracle's tape is uploaded and the GPU adjoint runs on it, so every limiter,
maximum and clip takes the same branch on both sides.
"""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SLOTS = [I.F_EGAS, I.F_MX, I.F_MY, I.F_MZ, I.F_ERAD, I.F_FX, I.F_FY, I.F_FZ]


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).copy()).cuda()


def gpu_adjoint(R, prob, U, tape, W, dt, nsteps=1):
    """GPU adjoint of `nsteps` steps recorded in `tape` (host array)."""
    N = U[0].size
    with R.RHDContext(prob) as ctx:
        ctx.set_stream(torch.cuda.current_stream())
        ctx.set_state(U)
        ybar = dev(W)
        kbar = torch.zeros(N, dtype=torch.float64, device="cuda")
        ctx.adjoint(dev(tape), nsteps, dt, ybar, kbar)
        return ybar.cpu().numpy().reshape(W.shape), kbar.cpu().numpy().reshape(U[0].shape)


def rel_err(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a)))


CASES = [
    (1, (300,), "periodic", "tau", "m1", 2),
    (1, (257,), "reflect", "none", "eddington", 1),
    (2, (40, 24), "periodic", "tau", "m1", 2),
    (2, (33, 17), "reflect", "tau", "m1", 1),
    (2, (24, 20), "periodic", "none", "eddington", 2),
    (3, (12, 10, 8), "periodic", "tau", "m1", 2),
    (3, (9, 7, 11), "reflect", "none", "m1", 2),
    (3, (8, 6, 5), "reflect", "tau", "eddington", 1),
]


@pytest.mark.parametrize("ndim,n,bc,hll,clo,order", CASES)
def test_adjoint_matches_oracle_adjoint(R, oracle_mod, ndim, n, bc, hll, clo, order):
    """One step, random out-of-equilibrium states: dL/dy(n) (8 slots) and
    dL/dkappa of the GPU agree with the oracle's to 1e-10 of each slot's
    largest value."""
    O = oracle_mod
    ci = CASES.index((ndim, n, bc, hll, clo, order))
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), c=1e3,
                          chat=[1e3, 1e2][ci % 2], bc=bc, hll_mode=hll, closure=clo,
                          vc_order=order)
    U = I.random_state(prob, seed=200 + ci, tau_range=(1e-2, 1e2))
    dt = O.dt(prob)
    tape = O.step_tape(prob, U.copy(), dt)
    rng = np.random.default_rng(ci)
    W = rng.standard_normal(tape[2].shape)
    for k, f in enumerate(SLOTS):
        m = np.abs(U[f]).max()
        W[k] = W[k] / m if m > 0 else 0.0
    kb_o = np.zeros_like(U[0])
    yb_o = O.step_adjoint(prob, U[I.F_RHO], U[I.F_KAPPA], tape, W, kb_o, dt)
    yb_g, kb_g = gpu_adjoint(R, prob, U, tape, W, dt)
    errs = {I.FIELDS[f]: rel_err(yb_g[k], yb_o[k]) for k, f in enumerate(SLOTS)}
    errs["kappa"] = rel_err(kb_g, kb_o)
    assert max(errs.values()) <= 1e-10, errs


def test_record_equals_step_and_tape_layout(R):
    prob = I.base_problem(2, (40, 24), (1 / 40, 1 / 24), c=1e3, chat=1e2)
    U = I.random_state(prob, seed=5)
    N = U[0].size
    with R.RHDContext(prob) as a, R.RHDContext(prob) as b:
        a.set_stream(torch.cuda.current_stream())
        a.set_state(U)
        b.set_state(U)
        tape = torch.empty(7 * 8 * N, dtype=torch.float64, device="cuda")
        info = a.step_record(3, 0.0, tape)
        b.step(3)
        assert info["steps_done"] == 3
        Ua, Ub = a.get_state(), b.get_state()
        assert np.array_equal(Ua, Ub)
        t = tape.cpu().numpy().reshape(7, 8, *U.shape[1:])
        assert np.array_equal(t[0], U[SLOTS])
        assert np.array_equal(t[6], Ub[SLOTS])
        assert a.time() == pytest.approx(b.time())


def test_adjoint_argument_errors(R):
    prob = I.base_problem(1, (64,), (1 / 64,), c=1e3, chat=1e2)
    U = I.random_state(prob, seed=6)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        tape = torch.zeros(3 * 8 * 64, dtype=torch.float64, device="cuda")
        ybar = torch.zeros(8 * 64, dtype=torch.float64, device="cuda")
        kbar = torch.zeros(64, dtype=torch.float64, device="cuda")
        with pytest.raises(R.RHDError):
            ctx.adjoint(tape, 2, 0.0, ybar, kbar)  # count does not match nsteps
        with pytest.raises(ValueError):
            ctx.adjoint(tape, 1, 0.0, ybar.cpu(), kbar)
        with pytest.raises(R.RHDError):
            ctx.step_record(2, 0.0, tape)


@pytest.mark.parametrize("bc", ["periodic", "reflect"])
def test_energy_total_is_a_left_null_vector(R, bc):
    """Sec. 3.3 conservation of sum(Egas + (c/chat) E): its cotangent is a
    fixed point of the adjoint, with no opacity gradient."""
    c, chat = 1e3, 1e2
    prob = I.base_problem(2, (40, 24), (1 / 40, 1 / 24), c=c, chat=chat, bc=bc)
    U = I.random_state(prob, seed=7)
    N = U[0].size
    with R.RHDContext(prob) as ctx:
        ctx.set_stream(torch.cuda.current_stream())
        ctx.set_state(U)
        tape = torch.empty(5 * 8 * N, dtype=torch.float64, device="cuda")
        ctx.step_record(2, 0.0, tape)
        W = np.zeros((8, N))
        W[0] = 1.0
        W[4] = c / chat
        ybar = dev(W)
        kbar = torch.zeros(N, dtype=torch.float64, device="cuda")
        ctx.adjoint(tape, 2, 0.0, ybar, kbar)
        yb = ybar.cpu().numpy().reshape(8, N)
        assert np.max(np.abs(yb - W)) <= 1e-11 * (c / chat)
        scale = np.abs(U[I.F_EGAS]).max() / np.abs(U[I.F_KAPPA]).min()
        assert np.max(np.abs(kbar.cpu().numpy())) <= 1e-10 * scale


@pytest.mark.parametrize("ndim,n,bc,hll,clo,order", CASES[::2])
def test_adjoint_matches_gpu_central_differences(R, ndim, n, bc, hll, clo, order):
    """Three recorded GPU steps: <dL/dy(0), D> + <dL/dkappa, Dk> equals the
    central difference of sum(W y(3)) computed with the GPU forward step."""
    ci = CASES.index((ndim, n, bc, hll, clo, order))
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), c=1e3,
                          chat=[1e3, 1e2][ci % 2], bc=bc, hll_mode=hll, closure=clo,
                          vc_order=order)
    U = I.random_state(prob, seed=300 + ci, tau_range=(1e-2, 1e2))
    N = U[0].size
    rng = np.random.default_rng(ci)
    live = np.array([np.abs(U[f]).max() > 0 for f in SLOTS], dtype=float)
    mag = np.array([np.abs(U[f]).max() for f in SLOTS]) + 1e-300
    W = rng.standard_normal((8, N)) * (live / mag)[:, None]
    D = np.zeros_like(U)
    for k, f in enumerate(SLOTS):
        D[f] = rng.standard_normal(U[0].shape) * np.abs(U[f]) * live[k]
    D[I.F_KAPPA] = rng.standard_normal(U[0].shape) * U[I.F_KAPPA]
    nst = 3
    with R.RHDContext(prob) as ctx:
        ctx.set_stream(torch.cuda.current_stream())
        ctx.set_state(U)
        tape = torch.empty((2 * nst + 1) * 8 * N, dtype=torch.float64, device="cuda")
        ctx.step_record(nst, 0.0, tape)
        ybar = dev(W)
        kbar = torch.zeros(N, dtype=torch.float64, device="cuda")
        ctx.adjoint(tape, nst, 0.0, ybar, kbar)
        yb = ybar.cpu().numpy().reshape(8, N)
        kb = kbar.cpu().numpy()
        lin = sum((yb[k] * D[f].reshape(-1)).sum() for k, f in enumerate(SLOTS)) + \
            (kb * D[I.F_KAPPA].reshape(-1)).sum()
        h = 1e-7
        vals = []
        for s in (1.0, -1.0):
            ctx.set_state(U + s * h * D)
            ctx.step(nst)
            V = ctx.get_state()
            vals.append(sum((W[k] * V[f].reshape(-1)).sum() for k, f in enumerate(SLOTS)))
        fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(lin - fd) <= 1e-6 * abs(fd), (lin, fd)


# ------------------------------------------------ the differentiation workload

def _pulse_loss_and_grad(R, prob, T0, lk, Et, nsteps, every, want_grad=True):
    from paper_2404_08247_gb300 import adjoint as A
    N = T0.size
    cv = prob["kB_over_mu"] / (prob["gamma"] - 1.0)
    a = prob["a_rad"]
    ctx = R.RHDContext(prob)
    try:
        U0 = I.rest_state(prob, T0, lk)
        ctx.set_stream(torch.cuda.current_stream())
        ctx.set_state(U0)
        T = torch.from_numpy(T0.reshape(-1).copy()).cuda().requires_grad_(want_grad)
        logk = torch.from_numpy(lk.reshape(-1).copy()).cuda().requires_grad_(want_grad)
        zero = torch.zeros_like(T)
        y0 = torch.stack([cv * T, zero, zero, zero, a * T ** 4, zero, zero, zero])
        y = A.trajectory(ctx, y0, torch.exp(logk), nsteps, 0.0, every)
        L = ((y[4] - torch.from_numpy(Et.reshape(-1).copy()).cuda()) ** 2).sum()
        if not want_grad:
            return float(L.detach())
        L.backward()
        return float(L.detach()), T.grad.cpu().numpy(), logk.grad.cpu().numpy()
    finally:
        ctx.close()


def test_checkpoint_segments_do_not_change_the_gradient(R):
    """45 steps with checkpoints every 20 (segments 20, 20, 5) give the same
    gradient, bit for bit, as one 45-step segment: every segment is re-run
    from its checkpoint with the same kernels."""
    prob, T0, lk, Et, _ = I.pulse_inverse_problem_2d(48)
    L1, gT1, gk1 = _pulse_loss_and_grad(R, prob, T0, lk, Et, 45, 20)
    L2, gT2, gk2 = _pulse_loss_and_grad(R, prob, T0, lk, Et, 45, 1000)
    assert L1 == L2
    assert np.array_equal(gT1, gT2) and np.array_equal(gk1, gk2)


def test_pulse_gradient_matches_oracle_gradient_64(R, oracle_mod):
    """The differentiation workload on its 64^2 copy, 200 steps, checkpoints
    every 20: the GPU gradient with respect to the initial temperature and
    the log opacity agrees with the oracle's FP64 gradient."""
    O = oracle_mod
    prob, T0, lk, Et, nsteps = I.pulse_inverse_problem_2d(64)
    Lg, gT, gk = _pulse_loss_and_grad(R, prob, T0, lk, Et, nsteps, 20)
    cv = prob["kB_over_mu"] / (prob["gamma"] - 1.0)

    def loss_grad(Uf):
        r = Uf[I.F_ERAD] - Et
        yb = np.zeros((8,) + Uf.shape[1:])
        yb[4] = 2.0 * r
        return float((r * r).sum()), yb

    Lo, yb, kb = O.trajectory_gradient(prob, I.rest_state(prob, T0, lk), nsteps, loss_grad)
    gT_o = (yb[0] * cv + yb[4] * 4.0 * prob["a_rad"] * T0 ** 3).reshape(-1)
    gk_o = (kb * np.exp(lk)).reshape(-1)
    assert Lg == pytest.approx(Lo, rel=1e-11)
    eT, ek = rel_err(gT, gT_o), rel_err(gk, gk_o)
    assert eT <= 1e-8 and ek <= 1e-8, (eT, ek)


FD_STEPS = (1e-6, 3e-7, 1e-7, 3e-8)


def test_pulse_gradient_matches_central_differences_64(R):
    """Same workload: directional derivatives of the GPU gradient against
    central differences of the GPU loss to 1e-6, the best of a short ladder
    of relative steps (a difference that straddles a limiter switch is off by
    a term proportional to its step; small steps meet the solves' rounding)."""
    prob, T0, lk, Et, nsteps = I.pulse_inverse_problem_2d(64)
    L, gT, gk = _pulse_loss_and_grad(R, prob, T0, lk, Et, nsteps, 20)
    rng = np.random.default_rng(4)
    for _ in range(2):
        dT = rng.standard_normal(T0.shape) * T0
        dk = rng.standard_normal(lk.shape)
        for vT, vk in ((dT, 0 * dk), (0 * dT, dk)):
            lin = float((gT * vT.reshape(-1)).sum() + (gk * vk.reshape(-1)).sum())
            errs = []
            for h in FD_STEPS:
                Lp = _pulse_loss_and_grad(R, prob, T0 + h * vT, lk + h * vk, Et, nsteps, 20,
                                          False)
                Lm = _pulse_loss_and_grad(R, prob, T0 - h * vT, lk - h * vk, Et, nsteps, 20,
                                          False)
                fd = (Lp - Lm) / (2 * h)
                errs.append(abs(lin - fd) / abs(fd))
            assert min(errs) <= 1e-6, errs
