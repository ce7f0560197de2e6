"""Mixed-precision form (RHD_PREC_MIXED) against the FP64 CPU oracle.

Reconstruction, closure and HLL fluxes run in single precision; the state,
flux differences, updates and the local solve stay double.  Bounds: every
field within 1e-5 of the oracle (pointwise relative for the positive fields,
max-norm relative for the signed ones), and the conserved totals within 1e-13
(the face fluxes telescope exactly because their differences are taken in
double).
"""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from parity import field_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def run(R, prob, U, nsteps, precision):
    with R.RHDContext(prob, precision) as ctx:
        ctx.set_state(U)
        t0 = ctx.totals()
        info = ctx.step(nsteps)
        t1 = ctx.totals()
        return ctx.get_state(), info, t0, t1


def check_conservation(prob, Ug, t0, t1):
    assert abs(t1[0] - t0[0]) <= TOL_CONS * abs(t0[0]), (t0[0], t1[0])
    V = np.prod(prob["dx"])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(Ug[I.F_MX + d]).sum() + np.abs(Ug[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= TOL_CONS * scale


@pytest.mark.parametrize("hll", ["tau", "none"])
def test_mixed_turbulent_box(R, oracle_mod, hll):
    prob, U, _ = I.turbulent_box_3d(shape=(37, 23, 19), hll_mode=hll)
    Ug, info, t0, t1 = run(R, prob, U, 10, "mixed")
    Uo = U.copy()
    oracle_mod.step(prob, Uo, nsteps=10)
    errs = field_errors(Ug, Uo)
    assert max(errs.values()) <= TOL_MIXED, errs
    check_conservation(prob, Ug, t0, t1)


def test_mixed_static_diffusion_1d(R, oracle_mod):
    prob, U, nsteps = I.static_diffusion_1d()
    Ug, info, t0, t1 = run(R, prob, U, nsteps, "mixed")
    Uo = U.copy()
    oracle_mod.step(prob, Uo, nsteps=nsteps)
    errs = field_errors(Ug, Uo)
    assert max(errs.values()) <= TOL_MIXED, errs
    assert abs(t1[0] - t0[0]) <= TOL_CONS * abs(t0[0])


def test_mixed_regime_sweep_1d(R, oracle_mod):
    """4096 cells, three optical-depth bands, chat = c/10, the full 2000
    steps (and 1000): every field pointwise within 1e-5 of the FP64 oracle.
    Near isotropy (|F| ~ 1e-3 cE) the flux of F is dominated by P ~ E/3; the
    mixed kernel carries that isotropic part in double (hll_states_mixed),
    so single-precision rounding of P_dd at every face does not drive F."""
    prob, U, nsteps = I.regime_sweep_1d()
    for n in (nsteps // 2, nsteps):
        Ug, info, t0, t1 = run(R, prob, U, n, "mixed")
        Uo = U.copy()
        oracle_mod.step(prob, Uo, nsteps=n)
        errs = field_errors(Ug, Uo)
        print("regime sweep, %d steps:" % n, {k: "%.2e" % v for k, v in errs.items()})
        assert max(errs.values()) <= TOL_MIXED, (n, errs)
        check_conservation(prob, Ug, t0, t1)


@pytest.mark.parametrize("var", range(3))
def test_mixed_2d_variants(R, oracle_mod, var):
    kw = [dict(closure="m1", vc_order=2, hll_mode="tau", bc="periodic"),
          dict(closure="eddington", vc_order=1, hll_mode="none", bc="periodic"),
          dict(closure="m1", vc_order=2, hll_mode="none",
               bc=[["reflect", "reflect"], ["reflect", "reflect"],
                   ["periodic", "periodic"]])][var]
    prob = I.base_problem(2, [33, 17], [1 / 33, 1 / 17], c=1e3, chat=2e2, **kw)
    U = I.random_state(prob, seed=200 + var, beta_max=1e-2)
    Ug, info, t0, t1 = run(R, prob, U, 6, "mixed")
    Uo = U.copy()
    oracle_mod.step(prob, Uo, nsteps=6)
    errs = field_errors(Ug, Uo)
    assert max(errs.values()) <= TOL_MIXED, errs
    assert abs(t1[0] - t0[0]) <= TOL_CONS * abs(t0[0])


def test_mixed_transport_rates(R, oracle_mod):
    """s(y) in single precision: within 1e-6 of the FP64 rates (max norm)."""
    prob, U, _ = I.turbulent_box_3d(shape=(40, 24, 16))
    with R.RHDContext(prob, "mixed") as ctx:
        ctx.set_state(U)
        rg = ctx.transport()
    ro = oracle_mod.transport(prob, U)
    for q in range(4):
        err = np.abs(rg[q] - ro[q]).max() / np.abs(ro[q]).max()
        assert err <= 1e-6, (q, err)
