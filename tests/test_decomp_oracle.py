"""The z-slab decomposition across processes (paper_2404_08247_gb300/decomp.py)
with the method itself on every slab: gloo ranks on CPU, each advancing its
z-slab of a 3-D turbulent box by the oracle's transport operator s(y) and its
per-cell implicit solves, the ghost and material planes moved between ranks
by decomp's exchange schedule.

Sec. 3.2: beyond a cell's own data, the explicit part of a stage reads only
the radiation state of the cells its face stencil reaches (2 planes with PLM,
3 with PPM), and the implicit part is local to the cell.  So a step of the
decomposed box has to reproduce the whole-grid oracle step bit for bit:
stage 1 from the ghost planes of y(n), stage 2 from those of y(n+1/2), and
the optical-depth factor of each face between two slabs from the opacity of
the plane across it.  These slabs carry kappa and rho of their boundary
plane in the two material messages (the library's slabs carry the face
factors computed from them); the schedule, the plane kinds, the directions
and the ghost planes of each stage are decomp's.

The hydrodynamic step (Sec. 3.1; RK2-SSP with HLLC faces) and the operator
split run the same way: ghost planes of the gas state before each stage's
face fluxes, the CFL step from the largest signal-speed bound of any slab,
the material planes again after the hydrodynamic step has moved rho, then
the subcycled radiation steps.  Those slabs carry the conserved gas fields
(rho, m, E_gas) in the five-field primitive messages."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2404_08247_gb300 import decomp  # noqa: E402
from paper_2404_08247_gb300 import inputs as I  # noqa: E402
from paper_2404_08247_gb300 import rhd as R  # noqa: E402

RAD = [I.F_ERAD, I.F_FX, I.F_FY, I.F_FZ]  # rows of the transport rates
EVOLVED = [I.F_EGAS, I.F_MX, I.F_MY, I.F_MZ, I.F_ERAD, I.F_FX, I.F_FY, I.F_FZ]
HYD = [I.F_RHO, I.F_MX, I.F_MY, I.F_MZ, I.F_EGAS]  # rows of the hydrodynamic rates
SHAPE = (6, 5, 12)  # nx, ny, nz
NSTEPS = 2


def box(reconstruction="plm", hll_mode="tau", periodic=True):
    prob, U, _ = I.turbulent_box_3d(shape=SHAPE, reconstruction=reconstruction,
                                    hll_mode=hll_mode)
    if not periodic:
        prob = dict(prob, bc=[["periodic", "periodic"], ["periodic", "periodic"],
                              ["reflect", "reflect"]])
    return prob, np.ascontiguousarray(U)


def z_faces(prob):
    bc = prob.get("bc", "periodic")
    return [bc, bc] if isinstance(bc, str) else list(bc[2])


class OracleSlab:
    """Planes z0 .. z1 of the box, stepped stage by stage by the oracle.  A
    stage runs the oracle's transport on the slab extended by its ghost planes
    (rates of the ghost planes are discarded, so the extended grid's own z
    faces there do not matter), then the oracle's local solve of every cell,
    combined as the oracle's whole step combines them (eq. imex1, imex2)."""

    def __init__(self, prob, U, z0, z1, low, high):
        from oracle import oracle as O
        self.O = O
        self.prob = prob
        self.params = O.make_params(prob)
        self.depth = 2 if prob.get("reconstruction", "plm") == "plm" else 3
        self.y = np.ascontiguousarray(U[:, z0:z1]).copy()
        self.low, self.high = low, high
        self.tau = prob.get("hll_mode", "tau") == "tau"
        self.device = "cpu"
        self.nx, self.ny = prob["n"][0], prob["n"][1]
        self.nz = z1 - z0
        self.ghost = [None, None]  # E, F of the planes below / above
        self.mat = [None, None]    # kappa, rho of the plane below / above
        self.pghost = [None, None]  # rho, m, E_gas of the planes below / above
        self.code = R.RHD_OK
        self.hydro = False         # the step to commit is a hydrodynamic one
        self.nlo = self.depth if low else 0
        zf = z_faces(prob)
        bc = [["periodic", "periodic"], ["periodic", "periodic"],
              ["reflect" if low else zf[0], "reflect" if high else zf[1]]]
        if not isinstance(prob.get("bc", "periodic"), str):
            bc[0], bc[1] = list(prob["bc"][0]), list(prob["bc"][1])
        n_ext = self.nz + self.nlo + (self.depth if high else 0)
        self.ext = dict(prob, n=[self.nx, self.ny, n_ext], bc=bc)

    # ---- the CtxSlab interface decomp drives
    def buffer(self, what):
        P = self.nx * self.ny
        planes = 4 * self.depth * P
        size = {R.RHD_SLAB_BOUNDARY_LOW: planes, R.RHD_SLAB_BOUNDARY_HIGH: planes,
                R.RHD_SLAB_GHOSTS_LOW: planes, R.RHD_SLAB_GHOSTS_HIGH: planes,
                R.RHD_SLAB_MATERIAL_LOW: 2 * P, R.RHD_SLAB_MATERIAL_ABOVE: 2 * P,
                R.RHD_SLAB_EPS_HIGH: 2 * P, R.RHD_SLAB_EPS_BELOW: 2 * P,
                R.RHD_SLAB_PRIM_BOUNDARY_LOW: 5 * self.depth * P,
                R.RHD_SLAB_PRIM_BOUNDARY_HIGH: 5 * self.depth * P,
                R.RHD_SLAB_PRIM_GHOSTS_LOW: 5 * self.depth * P,
                R.RHD_SLAB_PRIM_GHOSTS_HIGH: 5 * self.depth * P}[what]
        return torch.empty(size, dtype=torch.float64)

    def planes_get(self, what, stage):
        u = self.y if stage == 1 else self.yh
        d = self.depth
        a = {R.RHD_SLAB_BOUNDARY_LOW: lambda: u[RAD, :d],
             R.RHD_SLAB_BOUNDARY_HIGH: lambda: u[RAD, -d:],
             R.RHD_SLAB_MATERIAL_LOW: lambda: u[[I.F_KAPPA, I.F_RHO], 0],
             R.RHD_SLAB_EPS_HIGH: lambda: u[[I.F_KAPPA, I.F_RHO], -1],
             R.RHD_SLAB_PRIM_BOUNDARY_LOW: lambda: self.hsrc[HYD, :d],
             R.RHD_SLAB_PRIM_BOUNDARY_HIGH: lambda: self.hsrc[HYD, -d:]}[what]()
        return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).copy())

    def planes_set(self, what, buf):
        a = buf.numpy().copy()
        if what == R.RHD_SLAB_GHOSTS_LOW:
            self.ghost[0] = a.reshape(4, self.depth, self.ny, self.nx)
        elif what == R.RHD_SLAB_GHOSTS_HIGH:
            self.ghost[1] = a.reshape(4, self.depth, self.ny, self.nx)
        elif what == R.RHD_SLAB_MATERIAL_ABOVE:
            self.mat[1] = a.reshape(2, self.ny, self.nx)
        elif what == R.RHD_SLAB_EPS_BELOW:
            self.mat[0] = a.reshape(2, self.ny, self.nx)
        elif what == R.RHD_SLAB_PRIM_GHOSTS_LOW:
            self.pghost[0] = a.reshape(5, self.depth, self.ny, self.nx)
        elif what == R.RHD_SLAB_PRIM_GHOSTS_HIGH:
            self.pghost[1] = a.reshape(5, self.depth, self.ny, self.nx)
        else:
            raise AssertionError("plane kind %d is not set" % what)

    def stage(self, stage, dt):
        if stage == 1:
            self.code = R.RHD_OK
            self.hydro = False
        if self.code != R.RHD_OK:
            return
        u = self.y if stage == 1 else self.yh
        ext = self.extend(u)
        rates = self.O.transport(self.ext, ext)[:, self.nlo:self.nlo + self.nz]
        if stage == 1:
            self.s0 = rates
            ystar = self.y.copy()
            for r, f in enumerate(RAD):
                ystar[f] = self.y[f] + dt * rates[r]
            self.ystar = ystar
            self.yh = ystar.copy()
            self.solve(self.yh, 1.0, dt)
        else:
            U2 = self.ystar.copy()
            for f in EVOLVED:
                if f in RAD:
                    sn, sh = self.s0[RAD.index(f)], rates[RAD.index(f)]
                else:
                    sn = sh = 0.0
                dtf = self.yh[f] - self.ystar[f]
                U2[f] = self.y[f] + dt * (0.5 * sn + 0.5 * sh) + 0.5 * dtf
            U2[I.F_RHO] = self.y[I.F_RHO]
            U2[I.F_KAPPA] = self.y[I.F_KAPPA]
            self.solve(U2, 0.5, dt)
            self.yn = U2
        self.ghost = [None, None]  # every stage receives its own ghost planes

    def status(self):
        return self.code

    def commit(self, ok):
        if ok:
            self.y = self.yn
            if self.hydro:
                self.mat = [None, None]  # rho has moved: the TAU planes are resent

    # ---- the hydrodynamic step (decomp.hydro_step drives it)
    @property
    def cfl_hydro(self):
        return float(self.prob.get("cfl_hydro", 0.3))

    def radiation_dt(self):
        return self.O.dt(self.prob)

    def hydro_speed(self):
        """Largest sum_d (|v_d| + a)/dx_d over the slab's cells, evaluated as
        the oracle's hydrodynamic time step evaluates it."""
        y, gamma = self.y, self.prob["gamma"]
        rho = y[I.F_RHO]
        v = [y[I.F_MX + j] / rho for j in range(3)]
        ke = 0.0
        for j in range(3):
            ke = ke + 0.5 * rho * v[j] * v[j]
        p = (gamma - 1.0) * (y[I.F_EGAS] - ke)
        a = np.sqrt(gamma * p / rho)
        s = 0.0
        for d in range(3):
            s = s + (np.abs(v[d]) + a) / self.prob["dx"][d]
        return float(np.max(s))

    def hydro_phase(self, phase, dt):
        if phase == 0:
            self.code = R.RHD_OK
            self.hydro = True
            self.hdt = dt
            self.hsrc = self.y
            return
        if phase == 2:
            self.hsrc = self.u1
            return
        if self.code != R.RHD_OK:
            return
        ext = self.extend(self.hsrc, self.pghost, HYD)
        L = self.O.hydro_rate(self.ext, ext)[:, self.nlo:self.nlo + self.nz]
        self.pghost = [None, None]
        if phase == 1:
            u1 = self.y.copy()
            for q, f in enumerate(HYD):
                u1[f] = u1[f] + dt * L[q]
            self.u1 = u1
        else:
            u2 = self.u1.copy()
            for q, f in enumerate(HYD):
                u2[f] = 0.5 * (self.y[f] + (self.u1[f] + dt * L[q]))
            self.yn = u2
        u = self.u1 if phase == 1 else self.yn
        rho = u[I.F_RHO]
        ke = sum(0.5 * u[I.F_MX + j] * u[I.F_MX + j] / rho for j in range(3))
        p = (self.prob["gamma"] - 1.0) * (u[I.F_EGAS] - ke)
        if not (np.all(rho > 0.0) and np.all(p > 0.0) and np.all(np.isfinite(p))):
            self.code = R.RHD_ERR_NONPHYSICAL

    # ---- the oracle on the slab
    def extend(self, u, ghosts=None, rows=RAD):
        ghosts = self.ghost if ghosts is None else ghosts
        blocks = []
        if self.low:
            blocks.append(self.ghost_block(u, 0, ghosts, rows))
        blocks.append(u)
        if self.high:
            blocks.append(self.ghost_block(u, 1, ghosts, rows))
        return np.ascontiguousarray(np.concatenate(blocks, axis=1))

    def ghost_block(self, u, side, ghosts, rows):
        """The ghost planes of one side: the received fields (E, F for the
        radiation transport; rho, m, E_gas for the hydrodynamic rates); for the
        transport, kappa and rho of the plane across the face (TAU) received,
        else the slab's own boundary plane's; the fields the operator does
        not read copied from the slab's boundary plane."""
        assert ghosts[side] is not None, "ghost planes not received"
        edge = u[:, :1] if side == 0 else u[:, -1:]
        g = np.repeat(edge, self.depth, axis=1)
        g[rows] = ghosts[side]
        if rows is RAD:
            if self.mat[side] is not None:
                g[[I.F_KAPPA, I.F_RHO]] = self.mat[side][:, None]
            elif self.tau:
                raise AssertionError("material plane not received")
        return g

    def solve(self, U, theta, dt):
        import ctypes
        L = self.O.lib()
        yy = np.zeros(8)
        nn, no = ctypes.c_int(0), ctypes.c_int(0)
        for idx in np.ndindex(U.shape[1:]):
            rho = U[(I.F_RHO,) + idx]
            chi = U[(I.F_KAPPA,) + idx] * rho
            for q, f in enumerate(EVOLVED):
                yy[q] = U[(f,) + idx]
            st = L.orc_local_solve(ctypes.byref(self.params), float(theta), float(dt),
                                   float(rho), float(chi),
                                   yy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(nn), ctypes.byref(no))
            if st != 0:
                self.code = st
                return
            for q, f in enumerate(EVOLVED):
                U[(f,) + idx] = yy[q]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, case, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, U = box(**case)
    periodic = case.get("periodic", True)
    cuts = np.linspace(0, SHAPE[2], world + 1).astype(int)
    slab = OracleSlab(prob, U, cuts[rank], cuts[rank + 1],
                      periodic or rank > 0, periodic or rank < world - 1)
    from oracle import oracle as O
    decomp.exchange_material(slab, dist)
    res = decomp.step(slab, dist, NSTEPS, O.dt(prob))
    out[rank] = (slab.y, res)
    dist.barrier()
    dist.destroy_process_group()


def whole_grid(case):
    from oracle import oracle as O
    prob, U = box(**case)
    O.step(prob, U, NSTEPS, O.dt(prob))
    return U


@pytest.mark.parametrize("world,case", [
    (2, {}),
    (3, {"periodic": False}),
    (2, {"reconstruction": "ppm"}),
    (3, {"hll_mode": "none"}),
])
def test_decomposed_oracle_step_equals_whole_grid(world, case):
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, case, out), nprocs=world, join=True)
    res = [out[r] for r in range(world)]
    assert all(r[1] == {"steps_done": NSTEPS, "status": R.RHD_OK} for r in res)
    y = np.concatenate([r[0] for r in res], axis=1)
    np.testing.assert_array_equal(y, whole_grid(case))


def _gas_worker(rank, world, port, case, mode, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, U = box(**case)
    periodic = case.get("periodic", True)
    cuts = np.linspace(0, SHAPE[2], world + 1).astype(int)
    slab = OracleSlab(prob, U, cuts[rank], cuts[rank + 1],
                      periodic or rank > 0, periodic or rank < world - 1)
    if mode == "hydro":
        res = decomp.hydro_step(slab, dist, 2)
    else:
        decomp.exchange_material(slab, dist)
        res = decomp.split_step(slab, dist, 1)
    out[rank] = (slab.y, res)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,case,mode", [
    (2, {}, "hydro"),
    (3, {"periodic": False, "reconstruction": "ppm"}, "hydro"),
    (2, {}, "split"),
    (3, {"periodic": False}, "split"),
])
def test_decomposed_oracle_hydro_and_split_equal_whole_grid(world, case, mode):
    """Two hydrodynamic steps at the CFL step, or one operator-split step
    (15 radiation substeps here), of the decomposed box equal the whole-grid
    oracle's bit for bit."""
    from oracle import oracle as O
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_gas_worker, args=(world, port, case, mode, out), nprocs=world, join=True)
    res = [out[r] for r in range(world)]
    prob, U = box(**case)
    if mode == "hydro":
        O.hydro_step(prob, U, 2)
        assert all(r[1]["steps_done"] == 2 and r[1]["status"] == R.RHD_OK for r in res)
    else:
        subs = O.split_step(prob, U, 1)
        assert all(r[1] == {"steps_done": 1, "status": R.RHD_OK, "substeps": subs}
                   for r in res)
    y = np.concatenate([r[0] for r in res], axis=1)
    np.testing.assert_array_equal(y, U)


def test_one_slab_without_a_process_group():
    """The whole periodic box as one slab (dist = None): its ghost planes are
    its own opposite boundary planes."""
    prob, U = box()
    from oracle import oracle as O
    slab = OracleSlab(prob, U, 0, SHAPE[2], True, True)
    decomp.exchange_material(slab, None)
    res = decomp.step(slab, None, NSTEPS, O.dt(prob))
    assert res == {"steps_done": NSTEPS, "status": R.RHD_OK}
    np.testing.assert_array_equal(slab.y, whole_grid({}))
