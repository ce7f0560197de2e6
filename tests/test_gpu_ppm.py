"""GPU parity of the PPM faces (Sec. 3.3; Colella & Woodward 1984 edge
values with their monotonicity constraint) against the CPU oracle: FP64 to
1e-11 per field, the mixed form to 1e-5 with conservation to 1e-13, every
boundary kind, both schemes, the general physics, tiles with ragged tails,
the smallest reflecting axis (n = 3), and the Marshak wave of Sec. 5.2."""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from parity import assert_parity, field_errors
from parity import MARSHAK_CFL10_TOL, marshak_errors
from test_gpu_schemes import inflow_bc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11
TOL_MIXED = 1e-5
TOL_CONS = 1e-13


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
        t0 = ctx.totals()
        info = ctx.step(nsteps, dt)
        return ctx.get_state(), info, t0, ctx.totals()


def run_oracle(O, prob, U, nsteps, dt=0.0):
    Uo = U.copy()
    O.step(prob, Uo, nsteps=nsteps, dt=dt)
    return Uo


CASES = [
    # ndim, n, scheme, hll, kappa_T_exp, bc, (chi_0P, chi_0F) / chi_0E
    (1, (300,), "imex", "tau", 0.0, "periodic", None),
    (1, (257,), "imex", "none", 0.0, "reflect", None),
    (2, (33, 17), "imex", "tau", 0.0, "reflect", None),
    (2, (40, 21), "rk2ssp", "none", 0.0, "periodic", None),
    (3, (12, 10, 9), "imex", "tau", 0.0, "periodic", None),
    (3, (35, 9, 17), "imex", "none", 0.0, "reflect", None),
    (3, (9, 8, 7), "imex", "none", -3.0, "inflow", None),
    (2, (24, 20), "imex", "tau", 0.0, "periodic", (0.5, 0.3)),
    (3, (3, 3, 3), "imex", "tau", 0.0, "reflect", None),
    (2, (2, 16), "imex", "none", 0.0, "periodic", None),
]


def case_problem(ci):
    ndim, n, scheme, hll, pexp, bc, ratios = CASES[ci]
    c = 1e3
    kw = dict(c=c, chat=[1e3, 2e2][ci % 2], scheme=scheme, hll_mode=hll, kappa_T_exp=pexp,
              kappa_T_ref=1.5, reconstruction="ppm", cfl=0.3, newton_max_iter=400,
              outer_max_iter=200)
    if bc == "inflow":
        kw["bc"], kw["bc_state"] = inflow_bc(ndim, np.random.default_rng(ci), c)
    else:
        kw["bc"] = bc
    if ratios:
        kw["kappa_P_ratio"], kw["kappa_F_ratio"] = ratios
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), **kw)
    U = I.random_state(prob, seed=900 + ci, tau_range=(1e-2, 1e2), beta_max=1e-2)
    return prob, U


@pytest.mark.parametrize("ci", range(len(CASES)), ids=[str(c[:2]) for c in CASES])
def test_ppm_matches_oracle(R, oracle_mod, ci):
    prob, U = case_problem(ci)
    Ug, info, _, _ = run_gpu(R, prob, U, 5)
    Uo = run_oracle(oracle_mod, prob, U, 5)
    assert info["steps_done"] == 5
    assert_parity(Ug, Uo, TOL, str(CASES[ci]))


def test_ppm_transport_rate_matches_oracle(R, oracle_mod):
    """The transport-only launch (s(y) of eq. yrsla) with PPM faces."""
    prob, U = case_problem(5)
    with R.RHDContext(prob, "fp64") as ctx:
        ctx.set_state(U)
        rg = ctx.transport()
    ro = oracle_mod.transport(prob, U)
    for q in range(4):
        s = np.max(np.abs(ro[q]))
        assert np.max(np.abs(rg[q] - ro[q])) <= 1e-12 * s, q


@pytest.mark.parametrize("hll", ["tau", "none"])
def test_ppm_turbulent_box(R, oracle_mod, hll):
    """The 3-D turbulent box (lognormal density, tau_cell 1e-3 .. 1e3) with
    PPM faces at CFL 0.4: FP64 to 1e-11, mixed to 1e-5 with the totals
    conserved to 1e-13."""
    prob, U, _ = I.turbulent_box_3d(shape=(37, 23, 19), hll_mode=hll, reconstruction="ppm")
    Uo = run_oracle(oracle_mod, prob, U, 10)
    Ug, info, _, _ = run_gpu(R, prob, U, 10)
    assert_parity(Ug, Uo, TOL, "fp64")
    Um, info, t0, t1 = run_gpu(R, prob, U, 10, precision="mixed")
    errs = field_errors(Um, Uo)
    assert max(errs.values()) <= TOL_MIXED, errs
    assert abs(t1[0] - t0[0]) <= TOL_CONS * abs(t0[0]), (t0[0], t1[0])
    V = np.prod(prob["dx"])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(Um[I.F_MX + d]).sum() + np.abs(Um[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= TOL_CONS * scale


def test_ppm_refuses_a_negative_stage_state(R):
    """A free-streaming step at CFL 0.4 undershoots in the first stage (PPM
    keeps E > 0 for CFL <= 1/3): reported as nonphysical, as by the oracle."""
    n = 96
    prob = I.base_problem(1, [n], [1.0 / n], c=1.0, chat=1.0, reconstruction="ppm", cfl=0.4)
    sh = (1, 1, n)
    U = I.equilibrium_state(prob, np.ones(sh), np.ones(sh), np.zeros((3,) + sh), np.zeros(sh))
    x = I.cell_centres(prob)[0].reshape(-1)
    E = 1e-3 + (np.abs(x - 0.4) < 0.1)
    U[I.F_ERAD] = E.reshape(sh)
    U[I.F_FX] = E.reshape(sh)
    with pytest.raises(R.RHDError, match="nonphysical"):
        run_gpu(R, prob, U, 10)


@pytest.mark.parametrize("cfl", [0.9, 10.0])
def test_ppm_marshak_wave_matches_oracle(R, oracle_mod, cfl):
    """The asymptotic Marshak wave of Sec. 5.2 with the paper's PPM faces
    (60 cells, to 3e-9 s), with the metric of the PLM Marshak parity test:
    E against the local E_tot to 1e-11, E_gas, m and F to 1e-11 at CFL 0.9
    and to ten times the oracle's own rounding floor at CFL 10."""
    prob, U = I.marshak_wave_1d(60, scheme="imex", cfl=cfl, reconstruction="ppm")
    dt = oracle_mod.dt(prob)
    nsteps = int(round(3e-9 / dt))
    tol = TOL if cfl < 1.0 else MARSHAK_CFL10_TOL["ppm"]
    for n in sorted({min(500, nsteps), nsteps}):
        Ug, _, _, _ = run_gpu(R, prob, U, n, dt)
        Uo = run_oracle(oracle_mod, prob, U, n, dt)
        e = marshak_errors(Ug, Uo)
        print("ppm", cfl, n, e)
        assert e["erad_vs_etot"] <= TOL, (n, e)
        assert max(e["egas"], e["mx"], e["fx"]) <= tol, (n, e)


def test_batch_with_ppm_problems_equals_single_grids(R):
    """The batched form runs PPM and PLM problems side by side (a batch with a
    PPM problem runs the default 2-D tile shape), each bit for bit as alone,
    in both precisions; the autotuner's tile choice is ignored."""
    for precision in ("fp64", "mixed"):
        probs = []
        for i, (rec, n, extra) in enumerate((("ppm", (200,), {}), ("plm", (24, 20), {}),
                                             ("ppm", (33, 17), {"scheme": "rk2ssp"}),
                                             ("ppm", (3, 40), {"bc": "reflect"}),
                                             ("plm", (96,), {"kappa_T_exp": -3.0}))):
            kw = dict(c=1e3, chat=2e2, hll_mode="none", reconstruction=rec, cfl=0.3,
                      newton_max_iter=400)
            kw.update(extra)
            prob = I.base_problem(len(n), n, tuple(1.0 / v for v in n), **kw)
            probs.append((prob, I.random_state(prob, seed=800 + i, tau_range=(1e-2, 1e2))))
        with R.RHDBatch([p for p, _ in probs], precision) as b:
            b.configure(1, 2)
            for i, (_, U) in enumerate(probs):
                b.set_state(i, U)
            b.step(3)
            got = [b.get_state(i) for i in range(len(probs))]
        for (p, U), G in zip(probs, got):
            A, _, _, _ = run_gpu(R, p, U, 3, precision=precision)
            assert np.array_equal(A, G), (precision, p["reconstruction"], p["n"])


CS_CASES = [
    # ndim, n, scheme, hll, bc: the Colella-Sekora limiter (reconstruction ppm_cs)
    (1, (300,), "imex", "tau", "periodic"),
    (2, (33, 17), "imex", "none", "reflect"),
    (3, (12, 10, 9), "rk2ssp", "tau", "periodic"),
    (3, (35, 9, 17), "imex", "none", "reflect"),
    (3, (3, 3, 3), "imex", "tau", "reflect"),
]


@pytest.mark.parametrize("ci", range(len(CS_CASES)), ids=[str(c[:2]) for c in CS_CASES])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", TOL_MIXED)])
def test_ppm_cs_matches_oracle(R, oracle_mod, ci, precision, tol):
    """The Colella-Sekora limiter on the radiation faces, FP64 to 1e-11 and
    mixed to 1e-5, on random states with a temperature contrast of 1.3 (the
    limiter does not keep edges within the neighbours' range, so rougher data
    can turn a face state nonphysical)."""
    ndim, n, scheme, hll, bc = CS_CASES[ci]
    prob = I.base_problem(ndim, n, tuple(1.0 / v for v in n), c=1e3, chat=[1e3, 2e2][ci % 2],
                          scheme=scheme, hll_mode=hll, bc=bc, reconstruction="ppm_cs",
                          cfl=0.3)
    U = I.random_state(prob, seed=950 + ci, tau_range=(1e-2, 1e2), beta_max=1e-2,
                       T_range=(1.0, 1.3))
    Ug, info, _, _ = run_gpu(R, prob, U, 5, precision=precision)
    Uo = run_oracle(oracle_mod, prob, U, 5)
    assert info["steps_done"] == 5
    assert_parity(Ug, Uo, tol, str(CS_CASES[ci]))


def test_batch_with_cs_problems_equals_single_grids(R):
    probs = []
    for i, (rec, n) in enumerate((("ppm_cs", (200,)), ("plm", (24, 20)),
                                  ("ppm_cs", (33, 17)), ("ppm", (40,)))):
        prob = I.base_problem(len(n), n, tuple(1.0 / v for v in n), c=1e3, chat=2e2,
                              hll_mode="none", reconstruction=rec, cfl=0.3)
        probs.append((prob, I.random_state(prob, seed=860 + i, tau_range=(1e-2, 1e2),
                                           T_range=(1.0, 1.3))))
    with R.RHDBatch([p for p, _ in probs], "fp64") as b:
        for i, (_, U) in enumerate(probs):
            b.set_state(i, U)
        b.step(3)
        got = [b.get_state(i) for i in range(len(probs))]
    for (p, U), G in zip(probs, got):
        A, _, _, _ = run_gpu(R, p, U, 3)
        assert np.array_equal(A, G), (p["reconstruction"], p["n"])
