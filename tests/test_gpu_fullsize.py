"""Parity at the benchmark's full size (256^3 turbulent box, FP64) on sampled
cells, plus properties that hold at any size: the IMEX radiation step, and
the hydrodynamic step of the operator split.

One IMEX step at cell i depends only on y(n) within 4 cells of i (2 per
stage), so the oracle reproduces a sampled cell exactly from the 9^3 block of
y(n) around it, evolved as its own periodic box with the full problem's dt:
wrap-around only corrupts cells within 4 of the block's faces.
"""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11
RAD = 4


@pytest.fixture(scope="module")
def box():
    """The 256^3 turbulent box (generated once for the module)."""
    from paper_2404_08247_gb300 import build as B
    B.build()
    prob, U, _ = I.turbulent_box_3d(n=256)
    return prob, U


def one_step(prob, U, precision="fp64"):
    from paper_2404_08247_gb300 import rhd
    Ud = torch.from_numpy(U).cuda()
    with rhd.RHDContext(prob, precision, stream=torch.cuda.current_stream()) as ctx:
        ctx.set_state(Ud)
        info = ctx.step(1)
        out = torch.full_like(Ud, float("nan"))
        ctx.get_state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), info["dt"]


def sampled_worst(oracle_mod, prob, U, Ug, dt, rad, seed):
    """Largest per-field error at 48 sampled cells (two corners) against the
    oracle stepping the (2 rad + 1)^3 periodic block around each cell."""
    n = prob["n"][0]
    rng = np.random.default_rng(seed)
    cells = rng.integers(0, n, size=(48, 3))
    cells[0] = (0, 0, 0)
    cells[1] = (n - 1, n - 1, n - 1)
    w = 2 * rad + 1
    sub = I.base_problem(3, [w, w, w], prob["dx"], **{k: prob[k] for k in (
        "c", "chat", "gamma", "a_rad", "kB_over_mu", "cfl", "closure", "vc_order",
        "hll_mode", "newton_rtol", "outer_rtol", "newton_max_iter", "outer_max_iter")},
        reconstruction=prob.get("reconstruction", "plm"))
    worst = 0.0
    for (i, j, k) in cells:
        zi = (np.arange(k - rad, k + rad + 1) % n)
        yi = (np.arange(j - rad, j + rad + 1) % n)
        xi = (np.arange(i - rad, i + rad + 1) % n)
        blk = np.ascontiguousarray(U[:, zi][:, :, yi][:, :, :, xi])
        oracle_mod.step(sub, blk, nsteps=1, dt=dt)
        for f in range(I.NFIELD):
            b = blk[f, rad, rad, rad]
            a = Ug[f, k, j, i]
            scale = abs(b) if f in (I.F_RHO, I.F_EGAS, I.F_ERAD, I.F_KAPPA) else \
                np.abs(blk[f]).max()
            e = abs(a - b) / scale if scale > 0 else abs(a)
            worst = max(worst, e)
    return worst


def test_fullsize_ppm_sampled_cells_match_oracle(box, oracle_mod):
    """The PPM form as bench.py times it: a step depends on the state within
    6 cells (3 per stage), so 13^3 blocks reproduce sampled cells."""
    prob, U = box
    prob = dict(prob, reconstruction="ppm")
    Ug, dt = one_step(prob, U)
    assert sampled_worst(oracle_mod, prob, U, Ug, dt, 6, 2026) <= TOL


def test_fullsize_mixed_sampled_cells_match_oracle(box, oracle_mod):
    """The mixed form as bench.py times it, against the FP64 oracle: 1e-5."""
    prob, U = box
    Ug, dt = one_step(prob, U, "mixed")
    assert sampled_worst(oracle_mod, prob, U, Ug, dt, RAD, 2027) <= 1e-5


@pytest.fixture(scope="module")
def big(box):
    from paper_2404_08247_gb300 import rhd
    prob, U = box
    Ud = torch.from_numpy(U).cuda()
    with rhd.RHDContext(prob, stream=torch.cuda.current_stream()) as ctx:
        ctx.set_state(Ud)
        t0 = ctx.totals()
        info = ctx.step(1)
        t1 = ctx.totals()
        out = torch.full_like(Ud, float("nan"))
        ctx.get_state(out)
        dt = info["dt"]
    torch.cuda.synchronize()
    return prob, U, out.cpu().numpy(), dt, t0, t1, info


def test_fullsize_sampled_cells_match_oracle(big, oracle_mod):
    prob, U, Ug, dt, _, _, _ = big
    n = prob["n"][0]
    rng = np.random.default_rng(2024)
    cells = rng.integers(0, n, size=(48, 3))
    cells[0] = (0, 0, 0)            # corner: every ghost wraps
    cells[1] = (n - 1, n - 1, n - 1)
    w = 2 * RAD + 1
    sub = I.base_problem(3, [w, w, w], prob["dx"], **{k: prob[k] for k in (
        "c", "chat", "gamma", "a_rad", "kB_over_mu", "cfl", "closure", "vc_order",
        "hll_mode", "newton_rtol", "outer_rtol", "newton_max_iter", "outer_max_iter")})
    worst = 0.0
    for (i, j, k) in cells:
        zi = (np.arange(k - RAD, k + RAD + 1) % n)
        yi = (np.arange(j - RAD, j + RAD + 1) % n)
        xi = (np.arange(i - RAD, i + RAD + 1) % n)
        box = np.ascontiguousarray(U[:, zi][:, :, yi][:, :, :, xi])
        oracle_mod.step(sub, box, nsteps=1, dt=dt)
        for f in range(I.NFIELD):
            b = box[f, RAD, RAD, RAD]
            a = Ug[f, k, j, i]
            scale = abs(b) if f in (I.F_RHO, I.F_EGAS, I.F_ERAD, I.F_KAPPA) else \
                np.abs(box[f]).max()
            e = abs(a - b) / scale if scale > 0 else abs(a)
            worst = max(worst, e)
    assert worst <= TOL, worst


def test_fullsize_conservation_and_sanity(big):
    prob, U, Ug, dt, t0, t1, info = big
    assert info["status"] == 0 and info["steps_done"] == 1
    assert np.all(np.isfinite(Ug))
    assert np.all(Ug[I.F_ERAD] > 0)
    assert np.array_equal(Ug[I.F_RHO], U[I.F_RHO])
    assert np.array_equal(Ug[I.F_KAPPA], U[I.F_KAPPA])
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    V = np.prod(prob["dx"])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(Ug[I.F_MX + d]).sum() + np.abs(Ug[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= 1e-13 * scale
    assert info["n_solves"] == 2 * U[0].size


@pytest.fixture(scope="module")
def big_hydro(box):
    """One hydrodynamic step (RK2-SSP, HLLC, PLM) of the same 256^3 box at its
    CFL step, as bench.py's hydro_split leg times it."""
    from paper_2404_08247_gb300 import rhd
    prob, U = box
    Ud = torch.from_numpy(U).cuda()
    with rhd.RHDContext(prob, stream=torch.cuda.current_stream()) as ctx:
        ctx.set_state(Ud)
        dt = ctx.hydro_dt()
        t0 = ctx.totals()
        info = ctx.hydro_step(1, dt)
        t1 = ctx.totals()
        out = torch.full_like(Ud, float("nan"))
        ctx.get_state(out)
    torch.cuda.synchronize()
    return prob, U, out.cpu().numpy(), dt, t0, t1, info


def test_fullsize_hydro_dt_equals_the_oracle(big_hydro, oracle_mod):
    prob, U, _, dt, _, _, _ = big_hydro
    assert dt == oracle_mod.hydro_dt(prob, U)


def test_fullsize_hydro_sampled_cells_match_oracle(big_hydro, oracle_mod):
    """A hydrodynamic step at a cell depends on the state within 4 cells (2
    per stage with PLM): the oracle reproduces sampled cells from the 9^3
    block around each, evolved as its own periodic box with the same dt."""
    prob, U, Ug, dt, _, _, _ = big_hydro
    n = prob["n"][0]
    rng = np.random.default_rng(2025)
    cells = rng.integers(0, n, size=(48, 3))
    cells[0] = (0, 0, 0)
    cells[1] = (n - 1, n - 1, n - 1)
    w = 2 * RAD + 1
    sub = I.base_problem(3, [w, w, w], prob["dx"], gamma=prob["gamma"],
                         kB_over_mu=prob["kB_over_mu"], c=prob["c"], chat=prob["chat"])
    worst = 0.0
    for (i, j, k) in cells:
        zi = (np.arange(k - RAD, k + RAD + 1) % n)
        yi = (np.arange(j - RAD, j + RAD + 1) % n)
        xi = (np.arange(i - RAD, i + RAD + 1) % n)
        box = np.ascontiguousarray(U[:, zi][:, :, yi][:, :, :, xi])
        oracle_mod.hydro_step(sub, box, 1, dt)
        for f in (I.F_RHO, I.F_MX, I.F_MY, I.F_MZ, I.F_EGAS):
            b = box[f, RAD, RAD, RAD]
            a = Ug[f, k, j, i]
            scale = abs(b) if f in (I.F_RHO, I.F_EGAS) else np.abs(box[f]).max()
            worst = max(worst, abs(a - b) / scale)
    assert worst <= TOL, worst


def test_fullsize_hydro_conserves_and_leaves_radiation(big_hydro):
    prob, U, Ug, dt, t0, t1, info = big_hydro
    assert info["status"] == 0 and info["steps_done"] == 1
    for f in (I.F_ERAD, I.F_FX, I.F_FY, I.F_FZ, I.F_KAPPA):
        assert np.array_equal(Ug[f], U[f])
    V = np.prod(prob["dx"])
    assert abs(Ug[I.F_RHO].sum() - U[I.F_RHO].sum()) <= 1e-13 * U[I.F_RHO].sum()
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    cc = prob["c"] * prob["chat"]
    for d in range(3):
        scale = (np.abs(Ug[I.F_MX + d]).sum() + np.abs(Ug[I.F_FX + d]).sum() / cc) * V
        assert abs(t1[1 + d] - t0[1 + d]) <= 1e-13 * scale
