"""FP64 GPU path vs the CPU oracle, element by element (tolerance 1e-11).

Every case feeds the same seeded input bytes to both sides through the C ABI
(host buffers, or torch CUDA tensors where noted) and compares all ten fields.
"""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def run_gpu(R, prob, U, nsteps, dt=0.0, precision="fp64"):
    with R.RHDContext(prob, precision) as ctx:
        ctx.set_state(U)
        info = ctx.step(nsteps, dt)
        return ctx.get_state(), info


def run_oracle(O, prob, U, nsteps, dt=0.0):
    Uo = U.copy()
    infos = O.step(prob, Uo, nsteps=nsteps, dt=dt)
    return Uo, infos


def test_static_diffusion_1d_full_run(R, oracle_mod):
    """256 cells, reflecting walls, tau_cell = 10, chat = c, 1000 steps."""
    prob, U, nsteps = I.static_diffusion_1d()
    Ug, info = run_gpu(R, prob, U, nsteps)
    Uo, _ = run_oracle(oracle_mod, prob, U, nsteps)
    assert info["steps_done"] == nsteps
    assert_parity(Ug, Uo, TOL, "static diffusion")


def test_regime_sweep_1d_full_run(R, oracle_mod):
    """4096 cells, tau_cell = 1e-3 / 1 / 1e3 bands, v = 1e-3 c, chat = c/10,
    2000 steps."""
    prob, U, nsteps = I.regime_sweep_1d()
    Ug, info = run_gpu(R, prob, U, nsteps)
    Uo, _ = run_oracle(oracle_mod, prob, U, nsteps)
    assert_parity(Ug, Uo, TOL, "regime sweep")


@pytest.mark.parametrize("hll", ["tau", "none"])
def test_turbulent_box_ragged_shape(R, oracle_mod, hll):
    """3-D workload on a ragged 37 x 23 x 19 box (16169 cells: 127 blocks of
    128 threads plus a partial one), 4 steps."""
    prob, U, _ = I.turbulent_box_3d(shape=(37, 23, 19), hll_mode=hll)
    Ug, info = run_gpu(R, prob, U, 4)
    Uo, oinfo = run_oracle(oracle_mod, prob, U, 4)
    assert_parity(Ug, Uo, TOL, "turbulent box")
    assert info["n_solves"] == sum(i["n_solves"] for i in oinfo)


VARIANTS = [
    dict(closure="m1", vc_order=2, hll_mode="tau", bc="periodic"),
    dict(closure="m1", vc_order=1, hll_mode="none", bc="periodic"),
    dict(closure="eddington", vc_order=2, hll_mode="none", bc="periodic"),
    dict(closure="m1", vc_order=2, hll_mode="tau",
         bc=[["reflect", "reflect"], ["periodic", "periodic"], ["periodic", "periodic"]]),
    dict(closure="eddington", vc_order=1, hll_mode="tau",
         bc=[["periodic", "periodic"], ["reflect", "reflect"], ["periodic", "periodic"]]),
]


@pytest.mark.parametrize("var", range(len(VARIANTS)))
def test_2d_variants(R, oracle_mod, var):
    kw = VARIANTS[var]
    prob = I.base_problem(2, [33, 17], [1 / 33, 1 / 17], c=1e3, chat=2e2, **kw)
    U = I.random_state(prob, seed=100 + var, beta_max=1e-2)
    Ug, _ = run_gpu(R, prob, U, 6)
    Uo, _ = run_oracle(oracle_mod, prob, U, 6)
    assert_parity(Ug, Uo, TOL, str(kw))


@pytest.mark.parametrize("shape,ndim,bc", [
    ((3, 1, 1), 1, "periodic"),
    ((2, 1, 1), 1, "reflect"),
    ((1, 1, 1), 1, "periodic"),
    ((5, 1, 4), 3, "periodic"),
    ((1, 6, 1), 3, "periodic"),
    ((4, 3, 1), 2, "reflect"),
])
def test_small_and_degenerate_grids(R, oracle_mod, shape, ndim, bc):
    n = list(shape[:ndim])
    prob = I.base_problem(ndim, n, [0.1 * (d + 1) for d in range(ndim)], c=1e3,
                          chat=1e3, bc=bc)
    U = I.random_state(prob, seed=7, beta_max=1e-2)
    Ug, _ = run_gpu(R, prob, U, 3)
    Uo, _ = run_oracle(oracle_mod, prob, U, 3)
    assert_parity(Ug, Uo, TOL, str(shape))


def test_streaming_beam_and_zero_opacity(R, oracle_mod):
    """chi = 0 everywhere (no local solve) with a beam along y in 3-D, plus a
    mixed case where a third of the cells have kappa = 0."""
    n = [4, 48, 5]
    prob = I.base_problem(3, n, [1 / v for v in n], c=1.0, chat=1.0)
    sh = (n[2], n[1], n[0])
    U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh), np.zeros((3,) + sh),
                            np.zeros(sh))
    y = I.cell_centres(prob)[1]
    U[I.F_ERAD] = 1e-3 + np.exp(-((y - 0.3) / 0.05) ** 2) * np.ones(sh)
    U[I.F_FY] = U[I.F_ERAD]
    Ug, _ = run_gpu(R, prob, U, 20)
    Uo, _ = run_oracle(oracle_mod, prob, U, 20)
    assert_parity(Ug, Uo, TOL, "beam")
    prob = I.base_problem(3, [9, 8, 7], [1 / 9, 1 / 8, 1 / 7], c=1e3, chat=1e2)
    U = I.random_state(prob, seed=3, beta_max=1e-2)
    U[I.F_KAPPA].reshape(-1)[::3] = 0.0
    Ug, _ = run_gpu(R, prob, U, 4)
    Uo, _ = run_oracle(oracle_mod, prob, U, 4)
    assert_parity(Ug, Uo, TOL, "kappa = 0 mix")


def test_split_batches_and_async_match(R):
    """step(5) == step(2) + step(3) == step_async(5) + sync, bit for bit."""
    prob, U, _ = I.turbulent_box_3d(shape=(16, 12, 10))
    with R.RHDContext(prob) as a, R.RHDContext(prob) as b, R.RHDContext(prob) as c:
        for ctx in (a, b, c):
            ctx.set_state(U)
        a.step(5)
        b.step(2)
        b.step(3)
        c.step_async(5)
        info = c.sync()
        assert info["steps_done"] == 5
        Ua, Ub, Uc = a.get_state(), b.get_state(), c.get_state()
        assert np.array_equal(Ua, Ub) and np.array_equal(Ua, Uc)
        assert a.time() == pytest.approx(5 * a.default_dt(), rel=1e-15)


def test_device_tensors_and_torch_stream(R):
    """Device-pointer get/set on torch's current stream gives the same bits as
    the host path."""
    prob, U, _ = I.turbulent_box_3d(shape=(12, 10, 8))
    Ud = torch.from_numpy(U).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with R.RHDContext(prob, stream=torch.cuda.current_stream()) as ctx:
            ctx.set_state(Ud)
            ctx.step(3)
            out = torch.full_like(Ud, float("nan"))
            ctx.get_state(out)
    torch.cuda.synchronize()
    Uh, _ = run_gpu(R, prob, U, 3)
    assert np.array_equal(out.cpu().numpy(), Uh)


def test_totals_conserved_and_match_oracle(R, oracle_mod):
    prob, U, _ = I.turbulent_box_3d(shape=(24, 20, 16))
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        t0 = ctx.totals()
        ctx.step(6)
        t1 = ctx.totals()
        Ug = ctx.get_state()
    o0 = oracle_mod.totals(prob, U)
    o1 = oracle_mod.totals(prob, Ug)
    assert abs(t0[0] - o0[0]) <= 1e-13 * abs(o0[0])
    assert abs(t1[0] - o1[0]) <= 1e-13 * abs(o1[0])
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    V = np.prod(prob["dx"])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(Ug[I.F_MX + d]).sum() + np.abs(Ug[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= 1e-13 * scale
        assert abs(t1[1 + d] - o1[1 + d]) <= 1e-13 * scale


def test_rejects_nonfinite_input(R):
    prob, U, _ = I.turbulent_box_3d(shape=(8, 8, 8))
    with R.RHDContext(prob) as ctx:
        with pytest.raises(R.RHDError) as e:
            ctx.step(1)
        assert e.value.status == R.RHD_ERR_STATE
        bad = U.copy()
        bad[I.F_ERAD, 3, 2, 1] = np.nan
        with pytest.raises(R.RHDError) as e:
            ctx.set_state(bad)
        assert e.value.status == R.RHD_ERR_ARG
        with pytest.raises(R.RHDError) as e:
            ctx.step(1)
        assert e.value.status == R.RHD_ERR_STATE
        neg = U[I.F_RHO].copy()
        neg[0, 0, 0] = -1.0
        ctx.set_state(U)
        with pytest.raises(R.RHDError):
            ctx.set_field(R.RHD_F_RHO, np.ascontiguousarray(neg))
        ctx.set_field(R.RHD_F_RHO, np.ascontiguousarray(U[I.F_RHO]))
        ctx.step(1)


def test_newton_failure_reports_first_cell_and_keeps_state(R, oracle_mod):
    """With one Newton update allowed the first stage fails; both sides must
    name the same smallest cell, and the context must stay at y(n)."""
    prob, U, _ = I.turbulent_box_3d(shape=(12, 10, 8), newton_max_iter=1)
    Uo = U.copy()
    infos = oracle_mod.step(prob, Uo, nsteps=1, raise_on_error=False)
    assert infos[-1]["status"] == R.RHD_ERR_NEWTON
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        info = ctx.step(3, raise_on_error=False)
        assert info["status"] == R.RHD_ERR_NEWTON
        assert info["steps_done"] == 0 and info["fail_step"] == 0
        assert info["fail_stage"] == 1
        assert info["fail_cell"] == infos[-1]["fail_cell"]
        assert np.array_equal(ctx.get_state(), U)
        assert ctx.time() == 0.0


TRANSPORT_CASES = {
    "1d": dict(ndim=1, n=[300], bc="periodic"),
    "1d_reflect": dict(ndim=1, n=[77], bc="reflect"),
    "2d": dict(ndim=2, n=[33, 17], bc="periodic"),
    "2d_reflect_x": dict(ndim=2, n=[33, 17],
                         bc=[["reflect", "reflect"], ["periodic", "periodic"],
                             ["periodic", "periodic"]]),
    "3d": dict(ndim=3, n=[37, 23, 19], bc="periodic"),
    "3d_small": dict(ndim=3, n=[9, 8, 7], bc="periodic"),
    # cell fluxes up to 1.5 c E: reconstructed faces beyond the free-streaming
    # limit are scaled back and the closure clips f to 1
    "3d_overflux": dict(ndim=3, n=[20, 12, 10], bc="periodic", flux_frac=1.5),
}


@pytest.mark.parametrize("case", sorted(TRANSPORT_CASES))
@pytest.mark.parametrize("closure", ["m1", "eddington"])
@pytest.mark.parametrize("hll", ["tau", "none"])
def test_transport_rates_match_oracle(R, oracle_mod, case, closure, hll):
    """s(y) of eq. (yrsla) alone: the rates of E and F from the GPU's shared
    face fluxes equal the oracle's per-cell faces (max-norm relative, 1e-11)."""
    cfg = TRANSPORT_CASES[case]
    n = cfg["n"]
    prob = I.base_problem(cfg["ndim"], n, [1.0 / v for v in n], c=1e3, chat=2e2,
                          bc=cfg["bc"], closure=closure, hll_mode=hll)
    U = I.random_state(prob, seed=31, beta_max=1e-2, flux_frac=cfg.get("flux_frac", 0.1))
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        rg = ctx.transport()
    ro = oracle_mod.transport(prob, U)
    for q in range(4):
        s = np.abs(ro[q]).max()
        err = np.abs(rg[q] - ro[q]).max() / s if s > 0 else np.abs(rg[q]).max()
        assert err <= TOL, (q, err)
