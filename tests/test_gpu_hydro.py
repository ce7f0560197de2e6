"""GPU parity of the hydrodynamic subsystem and the operator split (Sec. 3.1)
against the CPU oracle: the RK2-SSP/HLLC step over 1-, 2- and 3-D grids,
PLM and PPM, periodic and reflecting walls, to 1e-11 per field; the CFL step
and the subcycle count bit for bit; the split of a coupled gas to 1e-11;
Sod's tube; the stationary contact kept exactly; failures that leave the
state as it was."""
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


def random_gas(prob, seed, mach=0.5, kappa=0.0):
    rng = np.random.default_rng(seed)
    sh = I.shape_of(prob)[1:]
    rho = 1.0 + 0.3 * rng.uniform(-1, 1, sh)
    p = 1.0 + 0.3 * rng.uniform(-1, 1, sh)
    v = mach * rng.uniform(-1, 1, (3,) + sh)
    for d in range(prob["ndim"], 3):
        v[d] = 0.0
    return I.gas_state(prob, rho, v, p, kappa=kappa)


CASES = [
    # ndim, n, reconstruction, bc
    (1, (300,), "plm", "periodic"),
    (1, (257,), "ppm", "reflect"),
    (2, (33, 17), "plm", "reflect"),
    (2, (40, 21), "ppm", "periodic"),
    (3, (12, 10, 9), "plm", "periodic"),
    (3, (17, 9, 11), "ppm", "reflect"),
    (3, (3, 3, 3), "ppm", "reflect"),
    (2, (2, 16), "plm", "periodic"),
    (1, (300,), "ppm_cs", "periodic"),
    (2, (33, 17), "ppm_cs", "reflect"),
    (3, (17, 9, 11), "ppm_cs", "periodic"),
]


@pytest.mark.parametrize("ci", range(len(CASES)), ids=[str(c) for c in CASES])
def test_hydro_step_matches_oracle(R, oracle_mod, ci):
    ndim, n, rec, bc = CASES[ci]
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), gamma=1.4, reconstruction=rec,
                          bc=bc)
    U = random_gas(prob, 40 + ci)
    dt = oracle_mod.hydro_dt(prob, U)
    Uo = U.copy()
    oracle_mod.hydro_step(prob, Uo, 5, dt)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        info = ctx.hydro_step(5, dt)
        Ug = ctx.get_state()
        assert info["steps_done"] == 5 and ctx.time() == pytest.approx(5 * dt, rel=1e-15)
    assert_parity(Ug, Uo, TOL, str(CASES[ci]))
    for f in (I.F_ERAD, I.F_FX, I.F_FY, I.F_FZ, I.F_KAPPA):
        assert np.array_equal(Ug[f], U[f])


def test_hydro_dt_and_subcycles_equal_the_oracle(R, oracle_mod):
    """The CFL bound is evaluated in the oracle's operation order without
    contraction: the same double, hence the same number of subcycles."""
    for ci, (ndim, n, rec, bc) in enumerate(CASES):
        prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), gamma=1.4, bc=bc,
                              cfl_hydro=0.35)
        U = random_gas(prob, 70 + ci)
        with R.RHDContext(prob) as ctx:
            ctx.set_state(U)
            assert ctx.hydro_dt() == oracle_mod.hydro_dt(prob, U), CASES[ci]


@pytest.mark.parametrize("rec", ["plm", "ppm"])
def test_sod_matches_oracle(R, oracle_mod, rec):
    """Sod's tube, 100 cells to t = 0.2 (134 fixed steps).  PPM: 1e-9, the
    oracle's own rounding floor (half-ulp noise per step moves it by up to
    7e-10: tests/test_oracle_hydro.py), where PPM's constraint switches at the
    shock feed rounding back; measured 1.0e-10.  PLM: 1e-10 (measured 4e-11;
    its rounding floor is below 1e-13, so the rest is the kernel's own
    rounding of the HLLC star state and its contractions at the shock)."""
    prob, U = I.riemann_problem_1d(100, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1),
                                   reconstruction=rec)
    Uo = U.copy()
    oracle_mod.hydro_step(prob, Uo, 134, 0.2 / 134)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        ctx.hydro_step(134, 0.2 / 134)
        Ug = ctx.get_state()
    assert_parity(Ug, Uo, 1e-9 if rec == "ppm" else 1e-10, rec)


def test_stationary_contact_is_exact(R):
    n = 64
    prob, U = I.riemann_problem_1d(n, (1.0, 0.0, 1.0), (0.1, 0.0, 1.0), bc="periodic")
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        ctx.hydro_step(50, 0.3 / n / np.sqrt(14.0))
        Ug = ctx.get_state()
    for f in (I.F_RHO, I.F_MX, I.F_EGAS):
        assert np.max(np.abs(Ug[f] - U[f])) <= 1e-14 * np.max(np.abs(U[I.F_EGAS])), f


@pytest.mark.parametrize("ndim,rec,hll", [(1, "plm", "tau"), (2, "plm", "none"),
                                          (2, "ppm", "tau"), (3, "plm", "tau")])
def test_split_matches_oracle(R, oracle_mod, ndim, rec, hll):
    """Two operator-split steps of a coupled gas (tau_cell ~ 0.1-1, c = 3 chat):
    hydrodynamics, then the radiation step subcycled; the TAU factors follow
    the evolving density."""
    n = {1: (96,), 2: (24, 20), 3: (12, 10, 8)}[ndim]
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), gamma=5 / 3, c=30.0, chat=10.0,
                          reconstruction=rec, hll_mode=hll)
    U = random_gas(prob, 90 + ndim, mach=0.3, kappa=2.0)
    Uo = U.copy()
    subs = oracle_mod.split_step(prob, Uo, 2)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        info = ctx.step_split(2)
        Ug = ctx.get_state()
    assert info["steps_done"] == 2 and min(subs) > 3
    assert info["n_solves"] == 2 * sum(subs) * int(np.prod(n))
    assert_parity(Ug, Uo, TOL, "split %dD %s" % (ndim, rec))


def test_failed_step_leaves_the_state_unchanged(R):
    """A step far beyond the CFL bound drives a density negative: reported as
    nonphysical with the hydrodynamic stage, the state as before the step."""
    prob = I.base_problem(1, [64], [1 / 64], gamma=1.4, bc="periodic")
    U = random_gas(prob, 5, mach=0.9)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        dt = ctx.hydro_dt()
        ctx.hydro_step(1, dt)
        U1 = ctx.get_state()
        info = ctx.hydro_step(3, 40.0 * dt, raise_on_error=False)
        assert info["status"] == R.RHD_ERR_NONPHYSICAL and info["steps_done"] == 0
        assert info["fail_stage"] in (3, 4)
        assert np.array_equal(ctx.get_state(), U1)


def test_inflow_axis_is_refused(R):
    prob, U = I.marshak_wave_1d(16)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        with pytest.raises(R.RHDError, match="periodic and reflecting"):
            ctx.hydro_step(1)


def test_split_in_mixed_precision(R, oracle_mod):
    """A mixed-precision context runs its radiation update in the mixed form
    and the hydrodynamic step in FP64: two split steps of a coupled 3-D gas
    within 1e-5 of the FP64 oracle, total energy and momentum conserved to
    1e-13."""
    n = (16, 12, 10)
    prob = I.base_problem(3, n, tuple(1.0 / v for v in n), gamma=5 / 3, c=30.0, chat=10.0,
                          reconstruction="ppm", hll_mode="tau")
    U = random_gas(prob, 97, mach=0.3, kappa=2.0)
    Uo = U.copy()
    oracle_mod.split_step(prob, Uo, 2)
    with R.RHDContext(prob, "mixed") as ctx:
        ctx.set_state(U)
        t0 = ctx.totals()
        ctx.step_split(2)
        t1 = ctx.totals()
        Ug = ctx.get_state()
    assert_parity(Ug, Uo, 1e-5, "mixed split")
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    V = np.prod(prob["dx"])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(Ug[I.F_MX + d]).sum() + np.abs(Ug[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= 1e-13 * scale


def test_edge_cases(R):
    """Zero steps change nothing; a one-cell periodic grid (every ghost is the
    cell itself) keeps its state exactly; a state with negative pressure has
    no hydrodynamic step (nonphysical, state untouched)."""
    prob = I.base_problem(2, [12, 10], [1 / 12, 1 / 10], gamma=1.4)
    U = random_gas(prob, 3)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        info = ctx.hydro_step(0)
        assert info["steps_done"] == 0 and np.array_equal(ctx.get_state(), U)
        info = ctx.step_split(0)
        assert info["steps_done"] == 0 and np.array_equal(ctx.get_state(), U)
    for ndim in (1, 3):
        n = [1] * ndim
        p1 = I.base_problem(ndim, n, [1.0] * ndim, gamma=1.4)
        U1 = random_gas(p1, 4)
        with R.RHDContext(p1) as ctx:
            ctx.set_state(U1)
            ctx.hydro_step(3, 0.1)
            assert np.array_equal(ctx.get_state(), U1)
    Ub = U.copy()
    Ub[I.F_EGAS, 0, 3, 4] = 0.25 * Ub[I.F_RHO, 0, 3, 4] * (
        (Ub[I.F_MX, 0, 3, 4] / Ub[I.F_RHO, 0, 3, 4]) ** 2)  # below the kinetic energy
    with R.RHDContext(prob) as ctx:
        ctx.set_state(Ub)
        with pytest.raises(R.RHDError, match="rho <= 0 or p <= 0"):
            ctx.hydro_dt()
        info = ctx.hydro_step(1, raise_on_error=False)
        assert info["status"] == R.RHD_ERR_NONPHYSICAL and info["steps_done"] == 0
        assert np.array_equal(ctx.get_state(), Ub)
