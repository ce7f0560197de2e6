"""Parity at the benchmark's full size (256^3 turbulent box, FP64) on sampled
cells, plus properties that hold at any size.

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
def big():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    prob, U, _ = I.turbulent_box_3d(n=256)
    Ud = torch.from_numpy(U).cuda()
    with rhd.RHDContext(prob, stream=torch.cuda.current_stream()) as ctx:
        ctx.set_state(Ud)
        t0 = ctx.totals()
        info = ctx.step(1)
        t1 = ctx.totals()
        out = torch.empty_like(Ud)
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
