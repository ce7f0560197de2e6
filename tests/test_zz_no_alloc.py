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
    x1 = torch.empty_like(x0)
    x2 = torch.empty_like(x0)
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
