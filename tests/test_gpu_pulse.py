"""The advecting radiation pulse in the static diffusion limit (Sec. 5.3),
the paper's test of the full operator-split system, run on the GPU through
rhd_step_split: a pulse in pressure balance carried at v0 = 1e6 cm/s (the
lab-frame run) and the same pulse at rest (the comoving run), 512 cells,
PPM faces (Sec. 3.3), chat = c, to t = 4.8e-5 s (about 2,800 hydrodynamic
steps and 1.8 million radiation steps).

The paper reports that the two runs, the lab-frame one shifted back by
v0 t, differ by less than 0.03 % in density and temperature anywhere, and
that gas and radiation temperatures stay within 3e-9 of each other.  v0 t =
48 cm is exactly 24 cells, so the comparison needs no interpolation.  One
split step of the lab-frame run is also checked against the oracle."""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_END = 4.8e-5
MU = 3.9e-24


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def gas_T(prob, U):
    rho = U[I.F_RHO]
    v = U[I.F_MX] / rho
    cv = prob["kB_over_mu"] / (prob["gamma"] - 1.0)
    return (U[I.F_EGAS] - 0.5 * rho * v * v) / (rho * cv)


def rad_T(prob, U):
    """Radiation temperature from the comoving energy density E - 2 v.F/c^2."""
    v = U[I.F_MX] / U[I.F_RHO]
    E0 = U[I.F_ERAD] - 2.0 * v * U[I.F_FX] / prob["c"] ** 2
    return (E0 / prob["a_rad"]) ** 0.25


def test_split_step_of_the_pulse_matches_oracle(R, oracle_mod):
    prob, U = I.advecting_pulse_1d(1e6)
    Uo = U.copy()
    subs = oracle_mod.split_step(prob, Uo, 1)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        info = ctx.step_split(1)
        Ug = ctx.get_state()
    assert info["n_solves"] == 2 * subs[0] * 512
    assert_parity(Ug, Uo, 1e-11, "pulse split step")


@pytest.fixture(scope="module")
def runs(R):
    """Both frames with the paper's PPM faces, at once: each context runs on
    its own stream from its own host thread (the library releases the
    interpreter during a call), so the two 512-cell runs share the GPU."""
    from concurrent.futures import ThreadPoolExecutor
    prob, U = I.advecting_pulse_1d(1e6, reconstruction="ppm")
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        dth = ctx.hydro_dt()
    nh = int(np.ceil(T_END / (0.9 * dth)))

    def run(v0):
        prob, U = I.advecting_pulse_1d(v0, reconstruction="ppm")
        with R.RHDContext(prob) as ctx:
            ctx.set_state(U)
            info = ctx.step_split(nh, T_END / nh)
            return prob, ctx.get_state(), info, ctx.time()

    with ThreadPoolExecutor(2) as ex:
        res = dict(zip((1e6, 0.0), ex.map(run, (1e6, 0.0))))
    for v0, (prob, U, info, t) in res.items():
        assert info["steps_done"] == nh
        assert t == pytest.approx(T_END, rel=1e-12)
    return {v0: r[:3] for v0, r in res.items()}


def test_advected_pulse_equals_the_comoving_pulse(runs):
    prob, lab, _ = runs[1e6]
    _, com, _ = runs[0.0]
    shift = int(round(1e6 * T_END / prob["dx"][0]))
    assert shift == 24
    lab_s = np.roll(lab, -shift, axis=-1)
    d_rho = np.max(np.abs(lab_s[I.F_RHO] - com[I.F_RHO]) / com[I.F_RHO])
    Tl, Tc = gas_T(prob, lab_s), gas_T(prob, com)
    d_T = np.max(np.abs(Tl - Tc) / Tc)
    print("advected vs comoving: rho %.3e, T %.3e" % (d_rho, d_T))
    assert d_rho < 3e-4 and d_T < 3e-4, (d_rho, d_T)
    # the pulse has diffused: the comparison is not between two unchanged states
    _, U0 = I.advecting_pulse_1d(0.0)
    assert np.max(np.abs(Tc - gas_T(prob, U0)) / Tc) > 1e-2


def test_gas_and_radiation_stay_in_equilibrium(runs):
    prob, lab, _ = runs[1e6]
    Tg, Tr = gas_T(prob, lab), rad_T(prob, lab)
    print("T_gas vs T_rad: %.3e" % np.max(np.abs(Tg - Tr) / Tg))
    assert np.max(np.abs(Tg - Tr) / Tg) < 3e-9
