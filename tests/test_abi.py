"""The C ABI library: loads, exports every declared symbol, and its host-side
logic (parameter validation, default step) behaves as the header states.
No GPU work: nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

from paper_2404_08247_gb300 import build as B
from paper_2404_08247_gb300 import inputs as I

HEADER = os.path.join(B.INCLUDE, "rhd.h")


@pytest.fixture(scope="module")
def rhd():
    B.build()
    from paper_2404_08247_gb300 import rhd as R
    R.load()
    return R


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rhd_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rhd_init", "rhd_step", "rhd_state_get", "rhd_state_set",
                     "rhd_totals", "rhd_destroy", "rhd_set_stream"):
        assert required in names


def test_library_exports_every_declared_symbol(rhd):
    lib = ctypes.CDLL(B.LIB)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared functions
    assert sorted(rhd.SIGNATURES) == declared_functions()


def test_binding_constants_match_header_enums():
    """Every enumerator of the header (status codes, boundary kinds, plane
    kinds, fields, options) has the same value in the Python binding, and
    every status code has a name for the binding's errors."""
    from paper_2404_08247_gb300 import rhd as R
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    seen = 0
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        value = -1
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, expr = item.partition("=")
            name = name.strip()
            value = int(expr.strip(), 0) if expr.strip() else value + 1
            if hasattr(R, name):
                assert getattr(R, name) == value, name
                seen += 1
    assert seen >= 40
    for code in range(R.RHD_ERR_BOUNDS + 1):
        assert code in R.STATUS_NAMES


def test_struct_layouts_match_header(rhd, tmp_path):
    """sizeof/offsetof of the ABI structs, as the C compiler lays them out,
    equal the ctypes mirrors of the binding."""
    fields = {"rhd_params": [f for f, _ in rhd.rhd_params._fields_],
              "rhd_step_info": [f for f, _ in rhd.rhd_step_info._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rhd.h"',
             "int main(void) {"]
    for st, fl in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st, st))
        for f in fl:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st, f, st, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True,
                                                 text=True, check=True).stdout.splitlines())
    for st, fl in fields.items():
        cls = getattr(rhd, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fl:
            assert int(out["%s.%s" % (st, f)]) == getattr(cls, f).offset, (st, f)


def test_defaults_and_validation(rhd):
    p = rhd.rhd_params_default()
    assert p.c == 1.0 and p.chat == 1.0 and abs(p.gamma - 5 / 3) < 1e-15
    assert p.newton_rtol == 1e-13 and p.outer_rtol == 1e-13
    assert p.hll_mode == rhd.RHD_HLL_TAU and p.vc_order == 2
    st, msg = rhd.rhd_params_validate(p)
    assert st == rhd.RHD_OK, msg

    def bad(**kw):
        q = rhd.rhd_params_default()
        for k, v in kw.items():
            setattr(q, k, v)
        st, msg = rhd.rhd_params_validate(q)
        assert st == rhd.RHD_ERR_ARG and msg, kw
        return msg

    bad(ndim=0)
    bad(ndim=4)
    bad(gamma=1.0)
    bad(chat=2.0)          # chat > c
    bad(chat=0.0)
    bad(cfl=-1.0)
    bad(vc_order=3)
    bad(closure=7)
    bad(precision=5)
    bad(newton_max_iter=0)
    q = rhd.rhd_params_default()
    q.n[0] = 1
    q.bc[0][0] = q.bc[0][1] = rhd.RHD_BC_REFLECT
    assert rhd.rhd_params_validate(q)[0] == rhd.RHD_ERR_ARG
    q = rhd.rhd_params_default()
    q.n[1] = 4  # axis beyond ndim must be 1
    assert rhd.rhd_params_validate(q)[0] == rhd.RHD_ERR_ARG
    q = rhd.rhd_params_default()
    q.dx[0] = float("nan")
    assert rhd.rhd_params_validate(q)[0] == rhd.RHD_ERR_ARG
    q = rhd.rhd_params_default()
    q.n[0] = 1 << 31
    assert rhd.rhd_params_validate(q)[0] == rhd.RHD_ERR_ARG


def test_init_rejects_bad_params_before_touching_the_device(rhd):
    q = rhd.rhd_params_default()
    q.gamma = 0.5
    h = ctypes.c_void_p()
    st = rhd.load().rhd_init(ctypes.byref(q), ctypes.byref(h))
    assert st == rhd.RHD_ERR_ARG and not h.value
    assert b"gamma" in rhd.load().rhd_last_error(None)


def test_default_dt_matches_oracle(rhd, oracle_mod):
    for prob in (I.static_diffusion_1d(n=64)[0],
                 I.base_problem(3, [8, 6, 4], [0.1, 0.2, 0.3], c=5.0, chat=2.0)):
        p = rhd.params_from_problem(prob)
        assert rhd.rhd_default_dt(p) == pytest.approx(oracle_mod.dt(prob), rel=1e-15)


def test_problem_mapping(rhd):
    prob = I.regime_sweep_1d(n=64)[0]
    p = rhd.params_from_problem(prob, "mixed")
    assert p.precision == rhd.RHD_PREC_MIXED
    assert p.n[0] == 64 and p.n[1] == 1 and p.ndim == 1
    assert p.chat == prob["chat"] and p.c == prob["c"]


def test_reconstruction_option_is_validated(rhd):
    """PPM reads three cells on each side of a face: a reflecting or inflow
    axis needs n >= 3 (a periodic one wraps); an unknown value is refused."""
    def params(n, bc, recon):
        q = rhd.rhd_params_default()
        q.n[0] = n
        q.bc[0][0] = q.bc[0][1] = bc
        q.reconstruction = recon
        return q

    assert rhd.rhd_params_default().reconstruction == rhd.RHD_RECON_PLM
    assert rhd.rhd_params_validate(params(2, rhd.RHD_BC_REFLECT, rhd.RHD_RECON_PLM))[0] == rhd.RHD_OK
    st, msg = rhd.rhd_params_validate(params(2, rhd.RHD_BC_REFLECT, rhd.RHD_RECON_PPM))
    assert st == rhd.RHD_ERR_ARG and "n >= 3" in msg
    assert rhd.rhd_params_validate(params(3, rhd.RHD_BC_REFLECT, rhd.RHD_RECON_PPM))[0] == rhd.RHD_OK
    assert rhd.rhd_params_validate(params(1, rhd.RHD_BC_PERIODIC, rhd.RHD_RECON_PPM))[0] == rhd.RHD_OK
    assert rhd.rhd_params_validate(params(8, rhd.RHD_BC_PERIODIC, 3))[0] == rhd.RHD_ERR_ARG
    st, msg = rhd.rhd_params_validate(params(2, rhd.RHD_BC_REFLECT, rhd.RHD_RECON_PPM_CS))
    assert st == rhd.RHD_ERR_ARG and "n >= 3" in msg
    p = rhd.params_from_problem(I.base_problem(1, [16], [1 / 16], reconstruction="ppm_cs"))
    assert p.reconstruction == rhd.RHD_RECON_PPM_CS
    p = rhd.params_from_problem(I.base_problem(1, [16], [1 / 16], reconstruction="ppm"))
    assert p.reconstruction == rhd.RHD_RECON_PPM


def test_hydro_cfl_is_validated(rhd):
    assert rhd.rhd_params_default().cfl_hydro == 0.3
    q = rhd.rhd_params_default()
    q.cfl_hydro = 0.0
    st, msg = rhd.rhd_params_validate(q)
    assert st == rhd.RHD_ERR_ARG and "cfl_hydro" in msg
    p = rhd.params_from_problem(I.base_problem(1, [16], [1 / 16], cfl_hydro=0.2))
    assert p.cfl_hydro == 0.2


def test_halo_faces_are_validated(rhd):
    """HALO faces join z-slabs of one 3-D grid: z faces only, n[2] >= 3, never
    paired with a periodic face; the no-allocation step refuses them."""
    def params(ndim, n, bc):
        q = rhd.rhd_params_default()
        q.ndim = ndim
        for d in range(3):
            q.n[d] = n[d] if d < ndim else 1
            q.dx[d] = 0.1
        for d, s, kind in bc:
            q.bc[d][s] = kind
        return q

    H, R, P = rhd.RHD_BC_HALO, rhd.RHD_BC_REFLECT, rhd.RHD_BC_PERIODIC
    assert rhd.rhd_params_validate(params(3, [4, 4, 3], [(2, 0, H), (2, 1, H)]))[0] == rhd.RHD_OK
    assert rhd.rhd_params_validate(params(3, [4, 4, 3], [(2, 0, R), (2, 1, H)]))[0] == rhd.RHD_OK
    st, msg = rhd.rhd_params_validate(params(3, [4, 4, 2], [(2, 0, H), (2, 1, H)]))
    assert st == rhd.RHD_ERR_ARG and "n[2] >= 3" in msg
    st, msg = rhd.rhd_params_validate(params(3, [4, 4, 4], [(0, 0, H), (0, 1, H)]))
    assert st == rhd.RHD_ERR_ARG and "z faces" in msg
    st, msg = rhd.rhd_params_validate(params(2, [4, 4], [(1, 0, H), (1, 1, H)]))
    assert st == rhd.RHD_ERR_ARG and "z faces" in msg
    st, msg = rhd.rhd_params_validate(params(3, [4, 4, 4], [(2, 0, P), (2, 1, H)]))
    assert st == rhd.RHD_ERR_ARG and "periodic" in msg
    assert rhd.rhd_params_validate(params(3, [4, 4, 4], [(2, 0, 4)]))[0] == rhd.RHD_ERR_ARG
    q = params(3, [4, 4, 4], [(2, 0, H), (2, 1, H)])
    info = rhd.rhd_step_info()
    st = rhd.load().rhd_step_noalloc(ctypes.byref(q), None, None, 0.0, None,
                                     ctypes.byref(info))
    assert st == rhd.RHD_ERR_ARG and b"rhd_step_slabs" in rhd.load().rhd_last_error(None)
    st = rhd.load().rhd_step_slabs(None, 0, 1, 0.0, ctypes.byref(info))
    assert st == rhd.RHD_ERR_ARG and info.fail_cell == -1


def test_slab_problems_split_the_z_axis(rhd):
    prob = I.base_problem(3, [8, 6, 12], [1 / 8, 1 / 6, 1 / 12], bc="reflect")
    qs = rhd.slab_problems(prob, [0, 4, 9, 12])
    assert [q["n"][2] for q in qs] == [4, 5, 3]
    assert [q["bc"][2] for q in qs] == [["reflect", "halo"], ["halo", "halo"],
                                        ["halo", "reflect"]]
    assert all(q["bc"][0] == ["reflect", "reflect"] for q in qs)
    qs = rhd.slab_problems(I.base_problem(3, [8, 6, 12], [1 / 8, 1 / 6, 1 / 12]), [0, 6, 12])
    assert [q["bc"][2] for q in qs] == [["halo", "halo"], ["halo", "halo"]]
    for q in qs:
        p = rhd.params_from_problem(q)
        assert p.bc[2][0] == p.bc[2][1] == rhd.RHD_BC_HALO
        assert rhd.rhd_params_validate(p)[0] == rhd.RHD_OK
    with pytest.raises(ValueError):
        rhd.slab_problems(prob, [0, 5])
    with pytest.raises(ValueError):
        rhd.slab_problems(I.base_problem(2, [8, 6], [1 / 8, 1 / 6]), [0, 6])


# grids for the host-step plan: every dimension, tile rows that are ragged,
# a single tile row, fewer rows than two chunks need, and the benchmark box
PLAN_SHAPES = [(1,), (255,), (256,), (257,), (600,), (4000,), (100000,),
               (7, 1), (33, 8), (45, 70), (64, 9), (512, 512),
               (9, 7, 5), (40, 24, 70), (33, 9, 37), (16, 16, 8), (16, 16, 9), (8, 8, 17),
               (12, 10, 40), (32, 32, 129), (256, 256, 256), (64, 64, 1000)]


@pytest.mark.parametrize("n", PLAN_SHAPES, ids=lambda n: "x".join(map(str, n)))
def test_host_step_plan_partitions_the_grid(rhd, n):
    """The chunks of rhd_step_host cover the cells once, in order, each a run
    of whole tile rows along the slowest axis; every chunk spans at least
    three cells along that axis (the deepest face stencil, PPM's, reaches
    only its neighbour chunks) unless there is one chunk; the stage-1 and
    stage-2 launch groups each partition the chunks into contiguous runs,
    within the compute streams (3 and 6), no stage-2 group above a quarter
    of the chunks (rounded up) when there are five or more, and chunk 0
    first in stage 1 and last in stage 2."""
    ndim = len(n)
    prob = I.base_problem(ndim, n, [1.0 / v for v in n])
    plan = rhd.host_step_plan(prob)
    cells, rows = plan["cells"], plan["rows"]
    K = len(cells) - 1
    ncell = 1
    for v in n:
        ncell *= v
    plane = ncell // n[-1]  # cells per index of the slowest axis
    tile = {1: 256, 2: 8, 3: 8}[ndim]  # cells of a tile row along that axis
    assert 1 <= K <= 16
    assert cells[0] == 0 and cells[-1] == ncell
    assert all(b > a for a, b in zip(cells, cells[1:]))
    assert rows[0] == 0 and rows[-1] == -(-n[-1] // tile)
    for k in range(K):
        lo, hi = cells[k] // plane, cells[k + 1] // plane
        assert cells[k] % plane == 0
        assert lo == rows[k] * tile and hi == min(n[-1], rows[k + 1] * tile)
        assert K == 1 or hi - lo >= 3
    for groups, most in ((plan["stage1"], 3), (plan["stage2"], 6)):
        assert 1 <= len(groups) <= most
        cover = sorted(c for a, b in groups for c in range(a, b))
        assert cover == list(range(K))
        assert all(b > a for a, b in groups)
    if K >= 2:
        assert plan["stage2"][-1] == (0, 1) and plan["stage1"][0] == (0, 1)
    if K >= 5:
        assert max(b - a for a, b in plan["stage2"]) <= -(-K // 4)


def test_host_step_plan_rejects_bad_arguments(rhd):
    p = rhd.params_from_problem(I.base_problem(3, (64, 64, 64), [1 / 64] * 3))
    K = ctypes.c_int()
    cells = (ctypes.c_int64 * 4)()
    rows = (ctypes.c_int * 4)()
    groups = (ctypes.c_int * 8)()
    ng = (ctypes.c_int * 2)()
    lib = rhd.load()
    # 64 planes: 8 tile rows, 4 chunks: 5 entries needed
    assert lib.rhd_host_step_plan(ctypes.byref(p), ctypes.byref(K), cells, rows, groups, ng,
                                  4) == rhd.RHD_ERR_ARG
    assert lib.rhd_host_step_plan(None, ctypes.byref(K), cells, rows, groups, ng,
                                  4) == rhd.RHD_ERR_ARG


def test_binding_refuses_buffers_smaller_than_the_call_needs():
    """The binding passes the library a count derived from the grid, so it
    checks the caller's buffer against it first: a smaller array or tensor
    is refused before any library call could overrun it."""
    import numpy as np
    import torch
    from paper_2404_08247_gb300 import rhd as R
    a = np.zeros(12)
    assert R._ptr(a, 12) == (a.ctypes.data, 0)
    assert R._ptr(a, 10)[1] == 0
    with pytest.raises(ValueError, match="holds 12 doubles, the call needs 13"):
        R._ptr(a, 13)
    t = torch.zeros(7, dtype=torch.float64)
    assert R._ptr(t, 7) == (t.data_ptr(), 0)
    with pytest.raises(ValueError):
        R._ptr(t, 8)
    with pytest.raises(ValueError):
        R._ptr(np.zeros(12, dtype=np.float32), 12)
    with pytest.raises(ValueError):
        R._ptr(np.zeros((4, 6))[:, ::2], 12)
