"""The exchange schedule of the z-slab decomposition across ranks
(paper_2404_08247_gb300/decomp.py) on CPU, with gloo ranks (world sizes 2
and 3) and a stand-in slab whose stages apply a z-stencil of the library's
ghost depth to numpy data: the decomposed run must equal the same stencil
on the whole grid, which it can only do if every rank received exactly the
neighbours' boundary planes that the single-process slab step copies
(E and F of 2 planes, [field][plane][n0 n1], periodic wrap or mirrored ends),
in both stages; the TAU material planes must arrive from the slab above and
the face factors from the slab below; and a step that fails on one rank
must be applied on none."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2404_08247_gb300 import decomp  # noqa: E402
from paper_2404_08247_gb300 import rhd as R  # noqa: E402

DEPTH = 2
W = np.array([0.05, -0.3, 0.5, 0.2, -0.1])  # z-stencil weights, offsets -2..2
SHAPE = (4, 12, 3, 5)  # fields, nz, n1, n0
DT = 0.1


def global_state():
    return np.random.default_rng(3).standard_normal(SHAPE)


def global_material():
    rng = np.random.default_rng(4)
    return rng.uniform(0.5, 2.0, SHAPE[1:]), rng.uniform(0.5, 2.0, SHAPE[1:])


def stencil(ext):
    """L(u) on the planes of ext that have DEPTH neighbours on both sides."""
    nz = ext.shape[1] - 2 * DEPTH
    return sum(W[o] * ext[:, o:o + nz] for o in range(5))


def extend(u, lo, hi):
    lo = u[:, [1, 0]] if lo is None else lo    # mirrored end
    hi = u[:, [-1, -2]] if hi is None else hi
    return np.concatenate([lo, u, hi], axis=1)


def whole_grid(nsteps, periodic):
    y = global_state()
    for _ in range(nsteps):
        ext = lambda u: extend(u, u[:, -DEPTH:] if periodic else None,  # noqa: E731
                               u[:, :DEPTH] if periodic else None)
        yh = y + DT * stencil(ext(y))
        y = 0.5 * (y + yh + DT * stencil(ext(yh)))
    return y


class FakeSlab:
    """Planes z0..z1 of the global state, stepped by the z-stencil."""

    def __init__(self, z0, z1, low, high, fail=None):
        self.y = global_state()[:, z0:z1].copy()
        k, r = global_material()
        self.k, self.r = k[z0:z1], r[z0:z1]
        self.low, self.high, self.tau = low, high, True
        self.device = "cpu"
        self.glo = self.ghi = None
        self.fail, self.steps = fail, 0
        self.log = []

    def buffer(self, what):
        n = SHAPE[2] * SHAPE[3]
        sizes = {R.RHD_SLAB_BOUNDARY_LOW: 4 * DEPTH * n, R.RHD_SLAB_BOUNDARY_HIGH: 4 * DEPTH * n,
                 R.RHD_SLAB_GHOSTS_LOW: 4 * DEPTH * n, R.RHD_SLAB_GHOSTS_HIGH: 4 * DEPTH * n,
                 R.RHD_SLAB_MATERIAL_LOW: 2 * n, R.RHD_SLAB_MATERIAL_ABOVE: 2 * n,
                 R.RHD_SLAB_EPS_HIGH: n, R.RHD_SLAB_EPS_BELOW: n}
        return torch.empty(sizes[what], dtype=torch.float64)

    def planes_get(self, what, stage):
        u = self.y if stage == 1 else self.yh
        if what == R.RHD_SLAB_BOUNDARY_LOW:
            out = u[:, :DEPTH]
        elif what == R.RHD_SLAB_BOUNDARY_HIGH:
            out = u[:, -DEPTH:]
        elif what == R.RHD_SLAB_MATERIAL_LOW:
            out = np.stack([self.k[0], self.r[0]])
        elif what == R.RHD_SLAB_EPS_HIGH:
            ka, ra = self.above
            out = 0.5 * (self.k[-1] * self.r[-1] + ka * ra)
        return torch.from_numpy(np.ascontiguousarray(out).reshape(-1).copy())

    def planes_set(self, what, buf):
        a = buf.numpy().copy()
        if what == R.RHD_SLAB_GHOSTS_LOW:
            self.glo = a.reshape(4, DEPTH, SHAPE[2], SHAPE[3])
        elif what == R.RHD_SLAB_GHOSTS_HIGH:
            self.ghi = a.reshape(4, DEPTH, SHAPE[2], SHAPE[3])
        elif what == R.RHD_SLAB_MATERIAL_ABOVE:
            self.above = a.reshape(2, SHAPE[2], SHAPE[3])
        elif what == R.RHD_SLAB_EPS_BELOW:
            self.eps_below = a.reshape(SHAPE[2], SHAPE[3])
        self.log.append(what)

    def stage(self, stage, dt):
        u = self.y if stage == 1 else self.yh
        L = stencil(extend(u, self.glo if self.low else None, self.ghi if self.high else None))
        if stage == 1:
            self.yh = self.y + dt * L
        else:
            self.yn = 0.5 * (self.y + self.yh + dt * L)
        self.glo = self.ghi = None  # each stage must receive its own planes

    def status(self):
        self.steps += 1
        return R.RHD_ERR_NEWTON if self.fail == self.steps - 1 else R.RHD_OK

    def commit(self, ok):
        if ok:
            self.y = self.yn


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, periodic, nsteps, fail, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cuts = np.linspace(0, SHAPE[1], world + 1).astype(int)
    low = periodic or rank > 0
    high = periodic or rank < world - 1
    slab = FakeSlab(cuts[rank], cuts[rank + 1], low, high,
                    fail=fail[1] if fail and fail[0] == rank else None)
    if periodic or world > 1:
        decomp.exchange_material(slab, dist)
    res = decomp.step(slab, dist, nsteps, DT)
    eps = getattr(slab, "eps_below", None)
    above = getattr(slab, "above", None)
    out[rank] = (slab.y, res, eps, above)
    dist.barrier()
    dist.destroy_process_group()


def run(world, periodic, nsteps, fail=None):
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, periodic, nsteps, fail, out), nprocs=world, join=True)
    return [out[r] for r in range(world)]


@pytest.mark.parametrize("world,periodic", [(2, True), (3, True), (2, False), (3, False)])
def test_decomposed_stencil_equals_whole_grid(world, periodic):
    nsteps = 3
    res = run(world, periodic, nsteps)
    y = np.concatenate([r[0] for r in res], axis=1)
    np.testing.assert_array_equal(y, whole_grid(nsteps, periodic))
    assert all(r[1] == {"steps_done": nsteps, "status": R.RHD_OK} for r in res)
    # TAU planes: material from the slab above, face factors from the slab below
    k, rho = global_material()
    cuts = np.linspace(0, SHAPE[1], world + 1).astype(int)
    for rank, r in enumerate(res):
        if periodic or rank < world - 1:
            za = cuts[(rank + 1) % world]
            np.testing.assert_array_equal(r[3], np.stack([k[za], rho[za]]))
        if periodic or rank > 0:
            zt = cuts[rank] - 1  # top plane of the slab below (wraps)
            zb = cuts[rank] % SHAPE[1]
            np.testing.assert_array_equal(r[2], 0.5 * (k[zt] * rho[zt] + k[zb] * rho[zb]))


def test_a_failure_on_one_rank_is_applied_on_none():
    """Rank 1 fails in its second step: both ranks report the status, keep
    the state of the first step and stop."""
    res = run(2, True, 4, fail=(1, 1))
    want = whole_grid(1, True)
    y = np.concatenate([r[0] for r in res], axis=1)
    np.testing.assert_array_equal(y, want)
    assert all(r[1] == {"steps_done": 1, "status": R.RHD_ERR_NEWTON} for r in res)


def test_one_periodic_slab_exchanges_with_itself():
    """One rank holding the whole periodic grid: its low ghosts are its own
    top planes and its high ghosts its bottom planes (a copy, no transfer)."""
    res = run(1, True, 2)
    np.testing.assert_array_equal(res[0][0], whole_grid(2, True))


# ---- the hydrodynamic step's schedule (five primitive fields, the CFL step)

CFL_H = 0.3


class FakeHydro(FakeSlab):
    """The five primitive fields (here the state itself) of planes z0..z1,
    stepped by the z-stencil in the RK2-SSP phases of the hydrodynamic
    step; the signal-speed bound is the largest |u| of the slab."""

    def __init__(self, z0, z1, low, high):
        super().__init__(z0, z1, low, high)
        self.u = hydro_state()[:, z0:z1].copy()

    def buffer(self, what):
        n = SHAPE[2] * SHAPE[3]
        return torch.empty(5 * DEPTH * n, dtype=torch.float64)

    def planes_get(self, what, stage):
        out = self.w[:, :DEPTH] if what == R.RHD_SLAB_PRIM_BOUNDARY_LOW else self.w[:, -DEPTH:]
        return torch.from_numpy(np.ascontiguousarray(out).reshape(-1).copy())

    def planes_set(self, what, buf):
        a = buf.numpy().copy().reshape(5, DEPTH, SHAPE[2], SHAPE[3])
        if what == R.RHD_SLAB_PRIM_GHOSTS_LOW:
            self.glo = a
        else:
            self.ghi = a

    def hydro_speed(self):
        return float(np.abs(self.u).max())

    cfl_hydro = CFL_H

    def hydro_phase(self, phase, dt):
        if phase in (0, 2):
            self.w = self.u if phase == 0 else self.u1
            self.glo = self.ghi = None
            return
        L = stencil(extend(self.w, self.glo if self.low else None,
                           self.ghi if self.high else None))
        if phase == 1:
            self.u1 = self.u + dt * L
        else:
            self.staged = 0.5 * (self.u + self.u1 + dt * L)

    def status(self):
        return R.RHD_OK

    def commit(self, ok):
        if ok:
            self.u = self.staged


def hydro_state():
    return np.random.default_rng(5).standard_normal((5,) + SHAPE[1:])


def whole_hydro(nsteps, periodic):
    u = hydro_state()
    for _ in range(nsteps):
        h = CFL_H / np.abs(u).max()
        ext = lambda v: extend(v, v[:, -DEPTH:] if periodic else None,  # noqa: E731
                               v[:, :DEPTH] if periodic else None)
        u1 = u + h * stencil(ext(u))
        u = 0.5 * (u + u1 + h * stencil(ext(u1)))
    return u


def _hydro_worker(rank, world, port, periodic, nsteps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cuts = np.linspace(0, SHAPE[1], world + 1).astype(int)
    slab = FakeHydro(cuts[rank], cuts[rank + 1], periodic or rank > 0,
                     periodic or rank < world - 1)
    res = decomp.hydro_step(slab, dist, nsteps)
    out[rank] = (slab.u, res)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (3, False)])
def test_decomposed_hydro_step_equals_whole_grid(world, periodic):
    """The primitives' ghost planes before both face phases, and the CFL step
    of the whole grid (the largest bound of any rank) on every rank."""
    nsteps = 3
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_hydro_worker, args=(world, port, periodic, nsteps, out), nprocs=world,
             join=True)
    u = np.concatenate([out[r][0] for r in range(world)], axis=1)
    np.testing.assert_array_equal(u, whole_hydro(nsteps, periodic))
    assert all(out[r][1]["steps_done"] == nsteps for r in range(world))
