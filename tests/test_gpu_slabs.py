"""z-slab decomposition on one GPU (rhd_step_slabs): the radiation step needs
only ghost layers of (E, F) from face neighbours (Sec. 3.2), so slabs that
exchange their boundary planes before every stage step exactly like the
undecomposed grid.  Every case compares all ten fields bit for bit with the
single-context run (itself pinned to the oracle by the parity tests), and the
iteration statistics with its own."""
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


def whole(R, prob, U, nsteps, dt, precision):
    with R.RHDContext(prob, precision) as ctx:
        ctx.set_state(U)
        info = ctx.step(nsteps, dt, raise_on_error=False)
        return ctx.get_state(), info


def slabs(R, prob, U, cuts, nsteps, dt, precision, calls=1):
    """The slabs of cuts, stepped in `calls` calls of nsteps / calls steps."""
    stream = torch.cuda.current_stream()
    ctxs = [R.RHDContext(q, precision, stream=stream) for q in R.slab_problems(prob, cuts)]
    try:
        for c, z0, z1 in zip(ctxs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        infos = [R.step_slabs(ctxs, nsteps // calls, dt, raise_on_error=False)
                 for _ in range(calls)]
        Us = np.concatenate([c.get_state() for c in ctxs], axis=1)
        times = [c.time() for c in ctxs]
    finally:
        for c in ctxs:
            c.close()
    return Us, infos, times


CASES = [
    # shape, cuts, options, precision, steps
    ((37, 23, 19), [0, 9, 19], dict(hll_mode="tau"), "fp64", 4),
    ((37, 23, 19), [0, 3, 11, 19], dict(hll_mode="none"), "fp64", 4),
    ((24, 20, 18), [0, 5, 11, 18], dict(hll_mode="tau", walls=True), "mixed", 4),
    ((24, 20, 18), [0, 18], dict(hll_mode="tau"), "fp64", 3),
    ((20, 17, 16), [0, 3, 9, 16], dict(hll_mode="tau", reconstruction="ppm"), "fp64", 3),
    ((20, 17, 16), [0, 8, 16], dict(hll_mode="none", reconstruction="ppm"), "mixed", 3),
    ((20, 17, 16), [0, 6, 16],
     dict(hll_mode="tau", scheme="rk2ssp", kappa_P_ratio=2.0, kappa_F_ratio=0.5), "fp64", 3),
]


def case_problem(shape, opts):
    """The turbulent box of shape with opts; walls: reflecting y and z axes."""
    opts = dict(opts)
    walls = opts.pop("walls", False)
    prob, U, _ = I.turbulent_box_3d(shape=shape, **opts)
    if walls:
        prob = dict(prob, bc=[["periodic"] * 2, ["reflect"] * 2, ["reflect"] * 2])
    return prob, U


@pytest.mark.parametrize("ci", range(len(CASES)), ids=[str(c[:2]) for c in CASES])
def test_slabs_step_like_the_whole_grid(R, ci):
    shape, cuts, opts, precision, nsteps = CASES[ci]
    prob, U = case_problem(shape, opts)
    dt = R.rhd_default_dt(R.params_from_problem(prob))
    Uw, iw = whole(R, prob, U, nsteps, dt, precision)
    assert iw["status"] == R.RHD_OK
    Us, infos, times = slabs(R, prob, U, cuts, nsteps, dt, precision)
    info = infos[0]
    assert info["status"] == R.RHD_OK and info["steps_done"] == nsteps
    assert all(t == pytest.approx(nsteps * dt, rel=1e-15) for t in times)
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), (CASES[ci], f)
    for k in ("n_solves", "sum_newton", "sum_outer", "max_newton", "max_outer"):
        assert info[k] == iw[k], k


def test_colella_sekora_faces_on_slabs(R):
    """PPM with the Colella-Sekora limiter (its second differences reach two
    cells beyond the face) on three slabs, FP64 and mixed, on a state whose
    temperatures vary smoothly enough for the limiter (iid within 30 %)."""
    shape = (14, 12, 15)
    prob = I.base_problem(3, list(shape), [1 / 14] * 3, c=30.0, chat=10.0,
                          reconstruction="ppm_cs", hll_mode="tau")
    U = I.random_state(prob, 31, tau_range=(1e-2, 10.0), T_range=(1.0, 1.3))
    dt = R.rhd_default_dt(R.params_from_problem(prob))
    for precision in ("fp64", "mixed"):
        Uw, iw = whole(R, prob, U, 3, dt, precision)
        assert iw["status"] == R.RHD_OK
        Us, infos, _ = slabs(R, prob, U, [0, 3, 9, 15], 3, dt, precision)
        assert infos[0]["status"] == R.RHD_OK
        for f in range(I.NFIELD):
            assert np.array_equal(Us[f], Uw[f]), (precision, f)


def test_inflow_and_reflecting_end_faces(R):
    """The outer z faces keep their own kind (an inflow source below, a wall
    above); the interior faces are HALO."""
    shape = (16, 12, 15)
    bc = [["periodic"] * 2, ["periodic"] * 2, ["inflow", "reflect"]]
    prob = I.base_problem(3, list(shape), [1 / 16] * 3, c=30.0, chat=10.0, bc=bc,
                          hll_mode="none", bc_state={(2, 0): (5.0, 2.0, 0.0, 1.0)})
    U = I.random_state(prob, 23, tau_range=(1e-2, 10.0))
    dt = R.rhd_default_dt(R.params_from_problem(prob))
    Uw, iw = whole(R, prob, U, 4, dt, "fp64")
    Us, infos, _ = slabs(R, prob, U, [0, 4, 8, 15], 4, dt, "fp64", calls=2)
    assert all(i["status"] == R.RHD_OK for i in infos)
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), f


def test_a_failure_stops_every_slab(R):
    """A step far beyond the transport's CFL bound drives E negative: the
    slabs report the whole grid's failing step and stage and a cell of the
    whole grid, and every slab keeps the state of the last step all of them
    completed."""
    prob, U, _ = I.turbulent_box_3d(shape=(24, 20, 18), hll_mode="none")
    dt = 60.0 * R.rhd_default_dt(R.params_from_problem(prob))
    Uw, iw = whole(R, prob, U, 2, dt, "fp64")
    assert iw["status"] != R.RHD_OK
    Us, infos, times = slabs(R, prob, U, [0, 6, 12, 18], 2, dt, "fp64")
    info = infos[0]
    for k in ("status", "steps_done", "fail_step", "fail_stage"):
        assert info[k] == iw[k], k
    # blocks that start after the first failure skip their cells, so the
    # smallest failing cell reported is one of the failing cells, not
    # necessarily the same one in both runs
    assert 0 <= info["fail_cell"] < U[0].size
    assert np.array_equal(Us, Uw)
    assert all(t == iw["steps_done"] * dt for t in times)


def test_slab_arguments_are_checked(R):
    prob, U, _ = I.turbulent_box_3d(shape=(16, 12, 12))
    stream = torch.cuda.current_stream()
    qs = R.slab_problems(prob, [0, 6, 12])
    a = R.RHDContext(qs[0], stream=stream)
    b = R.RHDContext(qs[1], stream=stream)
    other = dict(qs[1], n=[16, 12, 6], dx=[1 / 16, 1 / 12, 0.5])
    c = R.RHDContext(other, stream=stream)
    try:
        for ctx, z0 in ((a, 0), (b, 6), (c, 6)):
            ctx.set_state(np.ascontiguousarray(U[:, z0:z0 + 6]))
        with pytest.raises(R.RHDError, match="rhd_step_slabs"):
            a.step(1)
        with pytest.raises(R.RHDError, match="rhd_step_slabs"):
            a.transport()
        with pytest.raises(R.RHDError, match="params differ"):
            R.step_slabs([a, c])
        with pytest.raises(R.RHDError, match="one context"):
            R.step_slabs([a, a])
        b.set_stream(None)
        with pytest.raises(R.RHDError, match="one stream"):
            R.step_slabs([a, b])
        b.set_stream(stream)
        info = R.step_slabs([a, b], 0)
        assert info["status"] == R.RHD_OK and info["steps_done"] == 0
    finally:
        for ctx in (a, b, c):
            ctx.close()


def random_gas(prob, seed, mach=0.5, kappa=0.0):
    rng = np.random.default_rng(seed)
    sh = I.shape_of(prob)[1:]
    rho = 1.0 + 0.3 * rng.uniform(-1, 1, sh)
    p = 1.0 + 0.3 * rng.uniform(-1, 1, sh)
    v = mach * rng.uniform(-1, 1, (3,) + sh)
    return I.gas_state(prob, rho, v, p, kappa=kappa)


def run_slabs(R, prob, U, cuts, call):
    """call(contexts) on the slabs of cuts; returns (state, info, times)."""
    stream = torch.cuda.current_stream()
    ctxs = [R.RHDContext(q, stream=stream) for q in R.slab_problems(prob, cuts)]
    try:
        for c, z0, z1 in zip(ctxs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        info = call(ctxs)
        return (np.concatenate([c.get_state() for c in ctxs], axis=1), info,
                [c.time() for c in ctxs])
    finally:
        for c in ctxs:
            c.close()


HYDRO_CASES = [
    # n, cuts, reconstruction, bc
    ((12, 10, 15), [0, 5, 10, 15], "plm", "periodic"),
    ((12, 10, 15), [0, 3, 15], "ppm", "reflect"),
    ((9, 11, 12), [0, 4, 8, 12], "ppm_cs", "periodic"),
]


@pytest.mark.parametrize("ci", range(len(HYDRO_CASES)), ids=[str(c) for c in HYDRO_CASES])
def test_hydro_on_slabs_steps_like_the_whole_grid(R, ci):
    """Five fixed steps, then two at the CFL step of the whole grid: every
    field bit-identical, the same CFL step."""
    n, cuts, rec, bc = HYDRO_CASES[ci]
    prob = I.base_problem(3, list(n), [1.0 / v for v in n], gamma=1.4, reconstruction=rec,
                          bc=bc)
    U = random_gas(prob, 60 + ci)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        dt = ctx.hydro_dt()
        ctx.hydro_step(5, dt)
        iw = ctx.hydro_step(2)
        Uw = ctx.get_state()
        tw = ctx.time()

    def call(ctxs):
        R.hydro_step_slabs(ctxs, 5, dt)
        return R.hydro_step_slabs(ctxs, 2)
    Us, info, times = run_slabs(R, prob, U, cuts, call)
    assert info["steps_done"] == 2 and info["dt"] == iw["dt"]
    assert all(t == tw for t in times)
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), (HYDRO_CASES[ci], f)


@pytest.mark.parametrize("rec,hll", [("plm", "tau"), ("ppm", "none")])
def test_split_on_slabs_steps_like_the_whole_grid(R, rec, hll):
    """Two operator-split steps of a coupled gas (c = 3 chat, tau_cell ~ 0.1-1):
    the hydrodynamic step with its CFL step, then the radiation subcycles,
    on three slabs and on the whole grid."""
    n = (12, 10, 12)
    prob = I.base_problem(3, list(n), [1.0 / v for v in n], gamma=5 / 3, c=30.0, chat=10.0,
                          reconstruction=rec, hll_mode=hll)
    U = random_gas(prob, 95, mach=0.3, kappa=2.0)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        iw = ctx.step_split(2)
        Uw = ctx.get_state()
    Us, info, _ = run_slabs(R, prob, U, [0, 4, 7, 12], lambda c: R.step_split_slabs(c, 2))
    for k in ("steps_done", "n_solves", "sum_newton", "sum_outer", "dt"):
        assert info[k] == iw[k], k
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), f


def test_split_on_slabs_in_mixed_precision(R):
    """A mixed-precision split on slabs: the radiation update in the mixed
    form, the hydrodynamic step in FP64, as on the whole grid."""
    n = (10, 12, 12)
    prob = I.base_problem(3, list(n), [1.0 / v for v in n], gamma=5 / 3, c=30.0, chat=10.0,
                          reconstruction="ppm", hll_mode="tau",
                          bc=[["periodic"] * 2, ["periodic"] * 2, ["reflect"] * 2])
    U = random_gas(prob, 97, mach=0.3, kappa=2.0)
    with R.RHDContext(prob, "mixed") as ctx:
        ctx.set_state(U)
        ctx.step_split(2)
        Uw = ctx.get_state()
    stream = torch.cuda.current_stream()
    cuts = [0, 5, 12]
    ctxs = [R.RHDContext(q, "mixed", stream=stream) for q in R.slab_problems(prob, cuts)]
    try:
        for c, z0, z1 in zip(ctxs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        R.step_split_slabs(ctxs, 2)
        Us = np.concatenate([c.get_state() for c in ctxs], axis=1)
    finally:
        for c in ctxs:
            c.close()
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), f


def test_hydro_failure_on_slabs_leaves_every_slab(R):
    """A step far beyond the CFL bound: nonphysical, no slab committed."""
    n = (12, 10, 12)
    prob = I.base_problem(3, list(n), [1.0 / v for v in n], gamma=1.4)
    U = random_gas(prob, 7, mach=0.9)
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        dt = 40.0 * ctx.hydro_dt()
        iw = ctx.hydro_step(3, dt, raise_on_error=False)
    assert iw["status"] == R.RHD_ERR_NONPHYSICAL
    Us, info, times = run_slabs(
        R, prob, U, [0, 6, 12], lambda c: R.hydro_step_slabs(c, 3, dt, raise_on_error=False))
    for k in ("status", "steps_done", "fail_step"):
        assert info[k] == iw[k], k
    assert info["fail_stage"] in (3, 4) and np.array_equal(Us, U)
    assert all(t == 0.0 for t in times)


# ---- slabs stepped stage by stage (rhd_slab_*: the per-process form)

def stage_by_stage(R, prob, U, cuts, nsteps, dt, precision):
    """The slabs of cuts advanced through the per-slab calls that a process
    holding one slab makes, with the planes carried between the contexts
    here (what decomp.py does between ranks): material and face factors once,
    then per stage every slab's boundary planes into its neighbours' ghost
    planes, the stage on every slab, the statuses combined, the commit."""
    stream = torch.cuda.current_stream()
    probs = R.slab_problems(prob, cuts)
    ctxs = [R.RHDContext(q, precision, stream=stream) for q in probs]
    n = len(ctxs)
    halo = [(q["bc"][2][0] == "halo", q["bc"][2][1] == "halo") for q in probs]

    def get(c, what, stage=1):
        buf = torch.empty(c.slab_plane_doubles(what), dtype=torch.float64, device="cuda")
        return c.slab_planes_get(what, stage, buf)

    try:
        for c, z0, z1 in zip(ctxs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        if prob.get("hll_mode", "tau") == "tau":
            for s in range(n):
                if halo[s][1]:
                    ctxs[s].slab_planes_set(R.RHD_SLAB_MATERIAL_ABOVE,
                                            get(ctxs[(s + 1) % n], R.RHD_SLAB_MATERIAL_LOW))
            for s in range(n):
                if halo[s][0]:
                    ctxs[s].slab_planes_set(R.RHD_SLAB_EPS_BELOW,
                                            get(ctxs[(s - 1) % n], R.RHD_SLAB_EPS_HIGH))
        done, status = 0, R.RHD_OK
        for _ in range(nsteps):
            for stage in (1, 2):
                low = [get(c, R.RHD_SLAB_BOUNDARY_LOW, stage) if h[0] or h[1] else None
                       for c, h in zip(ctxs, halo)]
                high = [get(c, R.RHD_SLAB_BOUNDARY_HIGH, stage) if h[0] or h[1] else None
                        for c, h in zip(ctxs, halo)]
                for s in range(n):
                    if halo[s][0]:
                        ctxs[s].slab_planes_set(R.RHD_SLAB_GHOSTS_LOW, high[(s - 1) % n])
                    if halo[s][1]:
                        ctxs[s].slab_planes_set(R.RHD_SLAB_GHOSTS_HIGH, low[(s + 1) % n])
                for c in ctxs:
                    c.slab_stage(stage, dt)
            status = max(c.slab_status()["status"] for c in ctxs)
            for c in ctxs:
                c.slab_commit(status == R.RHD_OK)
            if status != R.RHD_OK:
                break
            done += 1
        Us = np.concatenate([c.get_state() for c in ctxs], axis=1)
    finally:
        for c in ctxs:
            c.close()
    return Us, done, status


STAGE_CASES = [
    ((37, 23, 19), [0, 9, 19], dict(hll_mode="tau"), "fp64", 4),
    ((24, 20, 18), [0, 5, 11, 18], dict(hll_mode="tau", walls=True), "mixed", 3),
    ((20, 17, 16), [0, 3, 9, 16], dict(hll_mode="none", reconstruction="ppm"), "fp64", 3),
    ((20, 17, 16), [0, 16], dict(hll_mode="tau"), "fp64", 2),
]


@pytest.mark.parametrize("ci", range(len(STAGE_CASES)), ids=[str(c[1]) for c in STAGE_CASES])
def test_stage_by_stage_slabs_step_like_the_whole_grid(R, ci):
    shape, cuts, opts, precision, nsteps = STAGE_CASES[ci]
    prob, U = case_problem(shape, opts)
    dt = R.rhd_default_dt(R.params_from_problem(prob))
    Uw, iw = whole(R, prob, U, nsteps, dt, precision)
    assert iw["status"] == R.RHD_OK
    Us, done, status = stage_by_stage(R, prob, U, cuts, nsteps, dt, precision)
    assert status == R.RHD_OK and done == nsteps
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), (STAGE_CASES[ci], f)


def test_stage_by_stage_failure_is_applied_on_no_slab(R):
    """A step far beyond the transport's CFL bound fails on some slab: no
    slab commits it, every slab keeps its state."""
    prob, U, _ = I.turbulent_box_3d(shape=(24, 20, 18), hll_mode="none")
    dt = 60.0 * R.rhd_default_dt(R.params_from_problem(prob))
    Us, done, status = stage_by_stage(R, prob, U, [0, 6, 12, 18], 2, dt, "fp64")
    assert status != R.RHD_OK and done == 0
    assert np.array_equal(Us, U)


def test_stage_calls_out_of_order_are_refused(R):
    prob, U, _ = I.turbulent_box_3d(shape=(12, 10, 9))
    q = R.slab_problems(prob, [0, 9])[0]
    with R.RHDContext(q) as c:
        c.set_state(U)
        with pytest.raises(R.RHDError):
            c.slab_stage(2)  # stage 2 before stage 1
        with pytest.raises(R.RHDError):
            c.slab_stage(1)  # TAU factors: the neighbours' planes are not set
        with R.RHDContext(prob) as plain:
            plain.set_state(U)
            with pytest.raises(R.RHDError):
                plain.slab_stage(1)  # not a slab


def test_decomp_step_on_one_rank(R):
    """decomp.step through a one-rank process group: the whole periodic box as
    one slab, its ghost planes its own opposite boundary planes."""
    import os
    import socket
    import torch.distributed as dist
    from paper_2404_08247_gb300 import decomp
    prob, U, _ = I.turbulent_box_3d(shape=(20, 16, 14))
    Uw, _ = whole(R, prob, U, 3, 0.0, "fp64")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        q = R.slab_problems(prob, [0, prob["n"][2]])[0]
        with R.RHDContext(q, stream=torch.cuda.current_stream()) as c:
            c.set_state(U)
            slab = decomp.CtxSlab(c, "cuda")
            decomp.exchange_material(slab, dist)
            res = decomp.step(slab, dist, 3)
            assert res == {"steps_done": 3, "status": R.RHD_OK}
            Us = c.get_state()
    finally:
        dist.destroy_process_group()
    assert np.array_equal(Us, Uw)


def hydro_stage_by_stage(R, prob, U, cuts, nsteps, precision="fp64"):
    """The hydrodynamic step of the slabs through the per-slab calls: the
    CFL step from the largest bound of any slab, then per phase pair the
    primitives' boundary planes into the neighbours' ghost planes."""
    stream = torch.cuda.current_stream()
    probs = R.slab_problems(prob, cuts)
    ctxs = [R.RHDContext(q, precision, stream=stream) for q in probs]
    n = len(ctxs)
    halo = [(q["bc"][2][0] == "halo", q["bc"][2][1] == "halo") for q in probs]

    def get(c, what):
        buf = torch.empty(c.slab_plane_doubles(what), dtype=torch.float64, device="cuda")
        return c.slab_planes_get(what, 1, buf)

    def swap():
        low = [get(c, R.RHD_SLAB_PRIM_BOUNDARY_LOW) for c in ctxs]
        high = [get(c, R.RHD_SLAB_PRIM_BOUNDARY_HIGH) for c in ctxs]
        for s in range(n):
            if halo[s][0]:
                ctxs[s].slab_planes_set(R.RHD_SLAB_PRIM_GHOSTS_LOW, high[(s - 1) % n])
            if halo[s][1]:
                ctxs[s].slab_planes_set(R.RHD_SLAB_PRIM_GHOSTS_HIGH, low[(s + 1) % n])

    try:
        for c, z0, z1 in zip(ctxs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        for _ in range(nsteps):
            smax = max(c.slab_hydro_speed() for c in ctxs)
            h = prob.get("cfl_hydro", 0.3) / smax
            for c in ctxs:
                c.slab_hydro_phase(0, h)
            swap()
            for c in ctxs:
                c.slab_hydro_phase(1, h)
            for c in ctxs:
                c.slab_hydro_phase(2, h)
            swap()
            for c in ctxs:
                c.slab_hydro_phase(3, h)
            status = max(c.slab_status()["status"] for c in ctxs)
            for c in ctxs:
                c.slab_commit(status == R.RHD_OK)
            assert status == R.RHD_OK
        Us = np.concatenate([c.get_state() for c in ctxs], axis=1)
    finally:
        for c in ctxs:
            c.close()
    return Us


@pytest.mark.parametrize("recon", ["plm", "ppm"])
def test_stage_by_stage_hydro_slabs_step_like_the_whole_grid(R, recon):
    prob, U = case_problem((20, 17, 16), dict(hll_mode="tau", reconstruction=recon))
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        for _ in range(3):
            ctx.hydro_step(1)
        Uw = ctx.get_state()
    Us = hydro_stage_by_stage(R, prob, U, [0, 5, 11, 16], 3)
    for f in range(I.NFIELD):
        assert np.array_equal(Us[f], Uw[f]), (recon, f)


def test_decomp_split_step_on_one_rank(R):
    """decomp.split_step through a one-rank process group (the whole periodic
    box as one slab): the hydrodynamic step, the material planes again, the
    subcycled radiation steps, bit for bit like rhd_step_split."""
    import os
    import socket
    import torch.distributed as dist
    from paper_2404_08247_gb300 import decomp
    prob, U, _ = I.turbulent_box_3d(shape=(20, 16, 14))
    with R.RHDContext(prob) as ctx:
        ctx.set_state(U)
        info = ctx.step_split(2)
        Uw = ctx.get_state()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        q = R.slab_problems(prob, [0, prob["n"][2]])[0]
        with R.RHDContext(q, stream=torch.cuda.current_stream()) as c:
            c.set_state(U)
            slab = decomp.CtxSlab(c, "cuda")
            decomp.exchange_material(slab, dist)
            res = decomp.split_step(slab, dist, 2)
            assert res["status"] == R.RHD_OK and res["steps_done"] == 2
            Us = c.get_state()
    finally:
        dist.destroy_process_group()
    assert np.array_equal(Us, Uw), info
