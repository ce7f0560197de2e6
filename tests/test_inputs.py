"""The seeded synthetic workloads (paper_2404_08247_gb300/inputs.py) against
their stated recipes: the values a generator must produce are checked from
the state it returns, not from its own code, so a changed seed, slope,
clip, band or scale shows up here before it silently changes what the
benchmark and the parity tests measure."""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I


def temperature(prob, U):
    rho = U[I.F_RHO]
    ke = 0.5 * (U[I.F_MX] ** 2 + U[I.F_MY] ** 2 + U[I.F_MZ] ** 2) / rho
    cv = prob["kB_over_mu"] / (prob["gamma"] - 1.0)
    return (U[I.F_EGAS] - ke) / (rho * cv)


def velocity(U):
    return U[I.F_MX:I.F_MZ + 1] / U[I.F_RHO]


def test_comoving_equilibrium():
    """Radiation in comoving equilibrium with the gas (Sec. 5.5): E = aT^4
    (1 + 4 beta^2/3) at v/c order 2, aT^4 at order 1, F = (4/3) v aT^4."""
    for order in (1, 2):
        prob = I.base_problem(1, [5], [0.2], c=10.0, chat=10.0, a_rad=2.0, vc_order=order)
        rho = np.full((1, 1, 5), 1.5)
        T = np.linspace(1.0, 2.0, 5).reshape(1, 1, 5)
        v = np.zeros((3, 1, 1, 5))
        v[0], v[1] = 0.3, -0.4
        U = I.equilibrium_state(prob, rho, T, v, kappa=7.0)
        aT4 = 2.0 * T ** 4
        beta2 = 0.25 / 100.0
        np.testing.assert_allclose(U[I.F_ERAD], aT4 * (1 + 4 * beta2 / 3 if order == 2 else 1),
                                   rtol=1e-15)
        np.testing.assert_allclose(U[I.F_FX], 4.0 / 3.0 * 0.3 * aT4, rtol=1e-15)
        np.testing.assert_allclose(U[I.F_FY], -4.0 / 3.0 * 0.4 * aT4, rtol=1e-15)
        np.testing.assert_allclose(temperature(prob, U), T, rtol=1e-14)
        assert np.all(U[I.F_KAPPA] == 7.0)


def test_gaussian_random_field_spectrum():
    """Zero mean, unit variance, and a power spectrum falling as k^-4: a
    least-squares fit of log P against log |k| over the modes 2 <= |k| <= 24
    of a 64^3 field (white noise only scatters log P about a constant)."""
    n = 64
    f = I.gaussian_random_field((n, n, n), -4.0, np.random.default_rng(1))
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12
    P = np.abs(np.fft.fftn(f)) ** 2
    k = np.fft.fftfreq(n) * n
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    m = (kk >= 2) & (kk <= 24)
    slope = np.polyfit(np.log(kk[m]), np.log(P[m]), 1)[0]
    assert abs(slope + 4.0) < 0.05, slope


def test_turbulent_box_recipe():
    """ln rho a unit-variance field with <rho> = 1; kappa rho dx = clip(rho^2,
    1e-3, 1e3); T in [1, 10]; rms Mach 1 with c_s = sqrt(gamma T); chat =
    30 max|v|, c = 10 chat; periodic, dx = 1/n; radiation in comoving
    equilibrium."""
    prob, U, nsteps = I.turbulent_box_3d(n=32)
    assert nsteps == 100 and U.shape == (10, 32, 32, 32)
    assert prob["bc"] == "periodic" and prob["dx"] == [1 / 32] * 3 and prob["ndim"] == 3
    rho = U[I.F_RHO]
    assert abs(rho.mean() - 1.0) < 1e-12
    assert abs(np.log(rho).std() - 1.0) < 1e-12
    tau = U[I.F_KAPPA] * rho * prob["dx"][0]
    np.testing.assert_allclose(tau, np.clip(rho * rho, 1e-3, 1e3), rtol=1e-14)
    T = temperature(prob, U)
    assert T.min() >= 1.0 - 1e-12 and T.max() <= 10.0 + 1e-12
    assert np.log10(T).std() == pytest.approx(1 / np.sqrt(12), rel=0.02)  # log-uniform
    v = velocity(U)
    speed = np.sqrt((v * v).sum(axis=0))
    mach = speed / np.sqrt(prob["gamma"] * T)
    assert np.sqrt((mach * mach).mean()) == pytest.approx(1.0, rel=1e-12)
    assert prob["chat"] == pytest.approx(30.0 * speed.max(), rel=1e-14)
    assert prob["c"] == pytest.approx(10.0 * prob["chat"], rel=1e-15)
    aT4 = T ** 4
    np.testing.assert_allclose(U[I.F_FX], 4.0 / 3.0 * v[0] * aT4, rtol=1e-12, atol=0)


def test_static_diffusion_and_regime_sweep_recipes():
    prob, U, nsteps = I.static_diffusion_1d()
    assert (nsteps, prob["n"][0], prob["bc"]) == (1000, 256, "reflect")
    assert prob["c"] == prob["chat"] == 1e5
    np.testing.assert_allclose(U[I.F_KAPPA] * U[I.F_RHO] * prob["dx"][0], 10.0, rtol=1e-14)
    T = temperature(prob, U).reshape(-1)
    # the peak 1 + 10 lies between the two central cell centres, 1/512 away
    assert 10.9 < T.max() < 11.0 and T.min() == pytest.approx(1.0, abs=1e-12)
    assert np.argmax(T) in (127, 128)
    assert np.all(U[I.F_FX] == 0.0)

    prob, U, nsteps = I.regime_sweep_1d()
    assert (nsteps, prob["n"][0], prob["bc"]) == (2000, 4096, "periodic")
    assert prob["chat"] == pytest.approx(prob["c"] / 10.0)
    tau = (U[I.F_KAPPA] * U[I.F_RHO] * prob["dx"][0]).reshape(-1)
    x = (np.arange(4096) + 0.5) / 4096  # cell centres
    bands = (x < 1 / 3, (x >= 1 / 3) & (x < 2 / 3), x >= 2 / 3)
    for band, want in zip(bands, (1e-3, 1.0, 1e3)):
        np.testing.assert_allclose(tau[band], want, rtol=1e-14)
    v = velocity(U).reshape(3, -1)
    np.testing.assert_allclose(v[0], 1e-3 * prob["c"], rtol=1e-14)
    T = temperature(prob, U).reshape(-1)
    for xb in (1 / 6, 1 / 2, 5 / 6):  # one pulse of height 1 per band
        assert T[np.argmin(abs(x - xb))] == pytest.approx(2.0, abs=1e-3)


def test_batched_workload_recipe():
    """512 problems: 1-D with N in [64, 4096] or 2-D with side in [32, 256],
    about half each; log10 tau_cell iid uniform on [-3, 3]; |v|/c <= 1e-3;
    c = 1e3, chat = 100; 6,586,398 cells in all (the benchmarked pool)."""
    probs = I.batched_problems()
    assert len(probs) == 512
    one = [p for p, _ in probs if p["ndim"] == 1]
    two = [p for p, _ in probs if p["ndim"] == 2]
    assert 200 < len(one) < 312 and len(one) + len(two) == 512
    assert all(64 <= p["n"][0] <= 4096 for p in one)
    assert all(32 <= p["n"][0] == p["n"][1] <= 256 for p in two)
    cells = sum(int(np.prod(p["n"])) for p, _ in probs)
    assert cells == 6_586_398
    lt = np.concatenate([np.log10(U[I.F_KAPPA] * U[I.F_RHO] * p["dx"][0]).reshape(-1)
                         for p, U in probs])
    assert lt.min() >= -3.0 and lt.max() <= 3.0
    assert abs(lt.mean()) < 0.01 and lt.std() == pytest.approx(6 / np.sqrt(12), rel=0.01)
    for p, U in probs:
        assert p["c"] == 1e3 and p["chat"] == 100.0 and p["bc"] == "periodic"
        v = velocity(U).reshape(3, -1)
        beta = np.sqrt((v * v).sum(axis=0)) / p["c"]
        assert beta.max() <= 1e-3 and np.ptp(beta) < 1e-15  # uniform velocity
        if p["ndim"] == 1:
            assert np.all(v[1:] == 0.0)


def test_pulse_inverse_problem_recipe():
    """The differentiation workload at 64^2: rest state, median tau_cell = 1,
    c = chat = 1e3, F = 0, T peaked at the centre."""
    prob, T0, log_kappa, E_tgt, nsteps = I.pulse_inverse_problem_2d(n=64)
    assert prob["n"][:2] == [64, 64] and prob["c"] == prob["chat"] == 1e3 and nsteps == 200
    tau = np.exp(log_kappa) * prob["dx"][0]  # rho = 1
    assert np.median(tau) == pytest.approx(1.0, rel=1e-12)
    assert abs(np.log(tau).std() - 1.0) < 1e-12  # sigma of ln chi
    U = I.rest_state(prob, T0, log_kappa)
    assert np.all(U[I.F_FX] == 0.0) and np.all(U[I.F_MX] == 0.0)
    np.testing.assert_allclose(temperature(prob, U), T0, rtol=1e-14)
    T = T0[0]
    c = np.unravel_index(np.argmax(T), T.shape)
    assert abs(c[0] - 31.5) <= 3 and abs(c[1] - 31.5) <= 3 and T.max() > 8.0
    # the target a (1 + 9 g)^4 with 0 < g <= 1 lies within [a, 10^4 a]
    assert E_tgt.min() >= prob.get("a_rad", 1.0) and E_tgt.max() <= 1e4 * (1 + 1e-12)
