"""rhd_step_noalloc, the entry point that allocates no device memory.

Some callers cannot allocate device memory: their memory belongs wholly to
another allocator (a framework's caching pool), or they must not call
cudaMalloc/cudaFree because those calls can synchronise the whole device.
rhd_step_noalloc serves them: the caller passes device input and output
buffers, and the stage buffer lives in a file-scope device array of at most
RHD_NOALLOC_MAX_CELLS cells.  These tests check it against rhd_step, the
context-based entry point, through the C ABI.  The file sorts last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

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


def noalloc_step(R, p, x_in, x_out, stream_handle, dt=0.0):
    info = R.rhd_step_info()
    st = R.load().rhd_step_noalloc(ctypes.byref(p), ctypes.c_void_p(x_in.data_ptr()),
                                   ctypes.c_void_p(x_out.data_ptr()), float(dt),
                                   ctypes.c_void_p(stream_handle), ctypes.byref(info))
    return st, info


@pytest.mark.parametrize("recon", ["plm", "ppm"])
def test_two_calls_in_a_row_match_rhd_step(R, recon):
    """Two successive no-allocation steps (the second reads the first's output)
    equal two rhd_step calls of a context on the same input (PLM and PPM
    faces)."""
    prob, U, _ = I.turbulent_box_3d(shape=(24, 20, 18), reconstruction=recon)
    p = R.params_from_problem(prob)
    stream = torch.cuda.current_stream()
    want = []
    with R.RHDContext(prob, stream=stream) as ctx:
        ctx.set_state(U)
        for _ in range(2):
            ctx.step(1)
            want.append(ctx.get_state())
    x0 = torch.from_numpy(U).cuda()
    x1 = torch.full_like(x0, float("nan"))
    x2 = torch.full_like(x0, float("nan"))
    st, info = noalloc_step(R, p, x0, x1, stream.cuda_stream)
    assert st == R.RHD_OK and info.steps_done == 1
    st, info = noalloc_step(R, p, x1, x2, stream.cuda_stream)
    assert st == R.RHD_OK and info.steps_done == 1
    assert info.n_solves == 2 * U[0].size
    torch.cuda.synchronize()
    assert_parity(x1.cpu().numpy(), want[0], TOL, "first no-alloc call")
    assert_parity(x2.cpu().numpy(), want[1], TOL, "second no-alloc call")


def test_rejects_grids_beyond_the_limit_and_overlap(R):
    n = [64, 64, 65]  # 266240 cells > RHD_NOALLOC_MAX_CELLS
    assert np.prod(n) > R.RHD_NOALLOC_MAX_CELLS
    p = R.params_from_problem(I.base_problem(3, n, [1.0 / v for v in n]))
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, _ = noalloc_step(R, p, x, y, 0)
    assert st == R.RHD_ERR_ARG
    assert b"limit" in R.load().rhd_last_error(None)
    prob, U, _ = I.turbulent_box_3d(shape=(8, 8, 8))
    p = R.params_from_problem(prob)
    x0 = torch.from_numpy(U).cuda()
    st, _ = noalloc_step(R, p, x0, x0, 0)
    assert st == R.RHD_ERR_ARG
    assert b"overlap" in R.load().rhd_last_error(None)


def wall_problem():
    """A 3-D box with an inflow face (low x), reflecting walls (high x, both
    y faces) and periodic z, TAU factors on: this entry point computes them
    from kappa and rho on the fly, rhd_step from its precomputed table."""
    bc = [["inflow", "reflect"], ["reflect", "reflect"], ["periodic", "periodic"]]
    n = (20, 14, 12)
    prob = I.base_problem(3, n, [1.0 / v for v in n], c=30.0, chat=10.0, bc=bc,
                          hll_mode="tau", bc_state={(0, 0): (3.0, 6.0, 1.5, 0.0)},
                          newton_max_iter=400, outer_max_iter=200)
    return prob, I.random_state(prob, 23, tau_range=(1e-2, 10.0), T_range=(1.0, 1.3))


@pytest.mark.parametrize("case,precision,tol", [("walls", "fp64", TOL),
                                                 ("walls", "mixed", 1e-5),
                                                 ("box", "mixed", 1e-5)])
def test_walls_and_mixed_precision_match_rhd_step(R, case, precision, tol):
    """Reflecting and inflow walls with the optical-depth factors, and the
    mixed-precision stage kernels: two calls in a row against rhd_step."""
    if case == "walls":
        prob, U = wall_problem()
    else:
        prob, U, _ = I.turbulent_box_3d(shape=(24, 20, 18))
    p = R.params_from_problem(prob, precision)
    stream = torch.cuda.current_stream()
    want = []
    with R.RHDContext(prob, precision, stream=stream) as ctx:
        ctx.set_state(U)
        for _ in range(2):
            ctx.step(1)
            want.append(ctx.get_state())
    x0 = torch.from_numpy(U).cuda()
    x1 = torch.full_like(x0, float("nan"))
    x2 = torch.full_like(x0, float("nan"))
    for xa, xb, w in ((x0, x1, want[0]), (x1, x2, want[1])):
        st, info = noalloc_step(R, p, xa, xb, stream.cuda_stream)
        assert st == R.RHD_OK and info.steps_done == 1
        torch.cuda.synchronize()
        errs = assert_parity(xb.cpu().numpy(), w, tol, "%s %s" % (case, precision))
        print(case, precision, "max field error %.2e" % max(errs.values()))


def test_rejects_an_infinite_dt(R):
    """dt = +inf is refused as by rhd_step (dt <= 0, or NaN, selects the
    default step in both)."""
    prob, U, _ = I.turbulent_box_3d(shape=(8, 8, 8))
    p = R.params_from_problem(prob)
    x0 = torch.from_numpy(U).cuda()
    x1 = torch.full_like(x0, float("nan"))
    st, _ = noalloc_step(R, p, x0, x1, 0, dt=float("inf"))
    assert st == R.RHD_ERR_ARG
    assert b"finite" in R.load().rhd_last_error(None)
