"""rhd_step_host (a host-held state stepped with the copies overlapping the
stage kernels) against the unpipelined calls rhd_state_set_all + rhd_step +
rhd_state_get_all on the same context type: the same bits, the same step
info, for every kind of grid the chunking has to handle (1-D, 2-D and 3-D,
ragged tile rows, a single chunk, PPM's three ghost planes, periodic,
reflecting and inflow faces, both precisions), in place and out of place,
from pinned and pageable buffers, and over several steps.  The unpipelined
calls are themselves checked against the oracle by the parity tests.
"""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def problem(ndim, n, seed, **kw):
    prob = I.base_problem(ndim, n, [1.0 / v for v in n], c=30.0, chat=10.0, **kw)
    return prob, I.random_state(prob, seed, tau_range=(1e-2, 30.0), T_range=(1.0, 1.5))


INFO_KEYS = ("status", "steps_done", "fail_cell", "fail_step", "fail_stage", "max_newton",
             "max_outer", "sum_newton", "n_solves", "sum_outer", "t", "dt")


def reference(R, prob, U, nsteps, precision, dt=0.0):
    with R.RHDContext(prob, precision) as ctx:
        ctx.set_state(U)
        info = ctx.step(nsteps, dt, raise_on_error=False)
        return ctx.get_state(), info


def check_same(R, prob, U, nsteps=1, precision="fp64", pinned=True, inplace=False):
    Ur, ir = reference(R, prob, U, nsteps, precision)
    src = torch.from_numpy(U.copy())
    if pinned:
        src = src.pin_memory()
    with R.RHDContext(prob, precision) as ctx:
        dst = src if inplace else (torch.full_like(src, float("nan")).pin_memory() if pinned
                                   else np.full(U.shape, np.nan))
        ih = ctx.step_host(src, dst, nsteps, raise_on_error=False)
        out = dst.numpy() if hasattr(dst, "numpy") else dst
        assert np.array_equal(out, Ur), "step_host differs from set/step/get"
        for k in INFO_KEYS:
            assert ih[k] == ir[k], k
        # the device state is the stepped one: a further step continues from it
        assert np.array_equal(ctx.get_state(), Ur)
    return Ur, ir


CASES = {
    # 3-D: 70 planes = 9 tile rows (the last one 6 planes), 4 chunks
    "3d_periodic_tau": (dict(ndim=3, n=(40, 24, 70)), 1, {}),
    "3d_reflect_mixed": (dict(ndim=3, n=(33, 9, 37), bc="reflect"), 2, {"precision": "mixed"}),
    "3d_ppm": (dict(ndim=3, n=(21, 13, 48), reconstruction="ppm", cfl=0.3), 3, {}),
    "3d_ppm_mixed_reflect": (dict(ndim=3, n=(17, 11, 33), reconstruction="ppm", cfl=0.3,
                                  bc="reflect"), 4, {"precision": "mixed"}),
    # one tile row of planes: a single chunk
    "3d_one_chunk": (dict(ndim=3, n=(9, 7, 5)), 5, {}),
    # 2-D: rows of 8 along y, 70 rows = 9 tile rows
    "2d_periodic_none": (dict(ndim=2, n=(45, 70), hll_mode="none"), 6, {}),
    "2d_inflow_general": (dict(ndim=2, n=(36, 41), hll_mode="none",
                               bc=[["inflow", "reflect"], ["reflect", "reflect"],
                                   ["periodic"] * 2],
                               bc_state={(0, 0): (2.0, 10.0, 3.0, 0.0)}), 7, {}),
    # 1-D: tiles of 256 cells along x, 2,000 cells = 8 tile rows
    "1d_periodic": (dict(ndim=1, n=(2000,)), 8, {}),
    "1d_ppm_reflect": (dict(ndim=1, n=(1100,), reconstruction="ppm", cfl=0.3,
                            bc="reflect"), 9, {}),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_step_equals_set_step_get(R, name):
    kw, seed, opt = CASES[name]
    kw = dict(kw)
    ndim, n = kw.pop("ndim"), kw.pop("n")
    prob, U = problem(ndim, n, 900 + seed, **kw)
    check_same(R, prob, U, 1, opt.get("precision", "fp64"))


@pytest.mark.parametrize("nsteps", [2, 3])
def test_host_step_several_steps(R, nsteps):
    prob, U = problem(3, (40, 24, 70), 920)
    check_same(R, prob, U, nsteps)


def test_host_step_in_place_and_pageable(R):
    prob, U = problem(3, (32, 16, 64), 921, reconstruction="ppm", cfl=0.3)
    check_same(R, prob, U, 1, inplace=True)
    check_same(R, prob, U, 2, pinned=False)
    check_same(R, prob, U, 1, pinned=False, inplace=True)


def test_host_step_then_device_steps(R):
    """The context holds the stepped state: host step, then a device step,
    equals two device steps; a second host step reloads rho and kappa."""
    prob, U = problem(3, (24, 16, 40), 922)
    U2, _ = reference(R, prob, U, 2, "fp64")
    with R.RHDContext(prob) as ctx:
        ctx.step_host(U.copy(), None, 1)
        ctx.step(1)
        assert np.array_equal(ctx.get_state(), U2)
        # a new host state with other opacities: the TAU factors follow it
        V = U.copy()
        V[I.F_KAPPA] *= 3.0
        out = ctx.step_host(V, None, 1)["out"]
    Vr, _ = reference(R, prob, V, 1, "fp64")
    assert np.array_equal(out, Vr)


def test_host_step_rejects_bad_input_and_arguments(R):
    prob, U = problem(3, (16, 8, 24), 923)
    bad = U.copy()
    bad[I.F_ERAD, 20, 3, 5] = np.nan
    with R.RHDContext(prob) as ctx:
        info = ctx.step_host(bad, None, 1, raise_on_error=False)
        assert info["status"] == R.RHD_ERR_ARG and info["steps_done"] == 0
        assert ctx.time() == 0.0
        with pytest.raises(R.RHDError):
            ctx.step(1)  # no state after a rejected input
        st = ctx.step_host(U.copy(), None, 0, raise_on_error=False)["status"]
        assert st == R.RHD_ERR_ARG
        with pytest.raises(R.RHDError):
            ctx.step_host(U.copy(), None, 1, dt=float("inf"))
        with pytest.raises(ValueError):
            ctx.step_host(torch.from_numpy(U.copy()).cuda(), None, 1)
        # a destination that overlaps the source without being it
        buf = np.zeros(U.size + 8)
        buf[: U.size] = U.ravel()
        st = ctx.step_host(buf[: U.size], buf[8:], 1, raise_on_error=False)["status"]
        assert st == R.RHD_ERR_ARG
        # a good call afterwards works
        out = ctx.step_host(U.copy(), None, 1)["out"]
    Ur, _ = reference(R, prob, U, 1, "fp64")
    assert np.array_equal(out, Ur)


def test_host_step_failure_keeps_state(R, oracle_mod):
    """One Newton update allowed: stage 1 fails; the step info names the same
    smallest cell as the oracle and the context stays at y(n)."""
    prob, U, _ = I.turbulent_box_3d(shape=(12, 10, 40), newton_max_iter=1)
    Uo = U.copy()
    infos = oracle_mod.step(prob, Uo, nsteps=1, raise_on_error=False)
    assert infos[-1]["status"] == R.RHD_ERR_NEWTON
    with R.RHDContext(prob) as ctx:
        info = ctx.step_host(U.copy(), None, 2, raise_on_error=False)
        assert info["status"] == R.RHD_ERR_NEWTON
        assert info["steps_done"] == 0 and info["fail_stage"] == 1
        assert info["fail_cell"] == infos[-1]["fail_cell"]
        assert np.array_equal(ctx.get_state(), U)
        assert ctx.time() == 0.0
