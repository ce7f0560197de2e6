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
and the ghost planes of each stage are decomp's."""
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
        self.code = R.RHD_OK
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
                R.RHD_SLAB_EPS_HIGH: 2 * P, R.RHD_SLAB_EPS_BELOW: 2 * P}[what]
        return torch.empty(size, dtype=torch.float64)

    def planes_get(self, what, stage):
        u = self.y if stage == 1 else self.yh
        d = self.depth
        a = {R.RHD_SLAB_BOUNDARY_LOW: lambda: u[RAD, :d],
             R.RHD_SLAB_BOUNDARY_HIGH: lambda: u[RAD, -d:],
             R.RHD_SLAB_MATERIAL_LOW: lambda: u[[I.F_KAPPA, I.F_RHO], 0],
             R.RHD_SLAB_EPS_HIGH: lambda: u[[I.F_KAPPA, I.F_RHO], -1]}[what]()
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
        else:
            raise AssertionError("plane kind %d is not set" % what)

    def stage(self, stage, dt):
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

    # ---- the oracle on the slab
    def extend(self, u):
        blocks = []
        if self.low:
            blocks.append(self.ghost_block(u, 0))
        blocks.append(u)
        if self.high:
            blocks.append(self.ghost_block(u, 1))
        return np.ascontiguousarray(np.concatenate(blocks, axis=1))

    def ghost_block(self, u, side):
        """The ghost planes of one side: E, F received; kappa, rho of the
        plane across the face (TAU) received, else the slab's own boundary
        plane's; the fields the transport does not read copied from it."""
        assert self.ghost[side] is not None, "ghost planes not received"
        edge = u[:, :1] if side == 0 else u[:, -1:]
        g = np.repeat(edge, self.depth, axis=1)
        g[RAD] = self.ghost[side]
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
