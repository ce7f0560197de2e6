"""The bounds-checked build of the library on small and degenerate grids.

librhd_bounds.so is the library compiled with -DRHD_BOUNDS_CHECK: the stage
kernels check every global index (state, rates, opacity tables, ghost
planes of neighbouring slabs) and every shared-memory ring index before
using it, and an index outside its array is reported as RHD_ERR_BOUNDS
instead of being accessed.  A child process steps the cases of
bounds_cases.py (one-cell grids, ragged tiles, a one-plane z-chunk tail,
the smallest reflecting PPM axis, inflow faces, both precisions, the batched
kernel, slabs) through it; every case must finish with RHD_OK and agree with
the default build (1e-11, 1e-5 for mixed precision).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import bounds_cases as BC
from parity import field_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def test_bounds_checked_build_on_degenerate_grids(R, tmp_path):
    from paper_2404_08247_gb300 import build as B
    lib = B.build(bounds_check=True)
    out = str(tmp_path / "bounds.npz")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), lib, out],
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    checked = np.load(out)
    want = BC.run_all(R)
    precision = {name: prec for name, _, _, _, prec in BC.grid_cases()}
    for name, (Uw, st) in want.items():
        assert st == R.RHD_OK, (name, st)
        st_c = int(checked["status_" + name])
        assert st_c == R.RHD_OK, (name, "bounds-checked build returned status %d" % st_c)
        Uc = checked[name]
        tol = 1e-5 if precision.get(name) == "mixed" or name.endswith("rates") else 1e-11
        if Uw.ndim == 4:
            errs = field_errors(Uc, Uw)
            assert max(errs.values()) <= tol, (name, errs)
        else:  # transport rates (4 fields)
            for q in range(Uw.shape[0]):
                s = np.abs(Uw[q]).max()
                assert np.abs(Uc[q] - Uw[q]).max() <= tol * max(s, 1e-300), (name, q)
