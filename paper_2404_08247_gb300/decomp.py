"""One grid decomposed into z-slabs across processes (one slab per rank).

Sec. 3.2: a stage of the IMEX scheme needs, beyond a cell's own data, only
the ghost planes of its face neighbours, so a z-slab decomposition exchanges
E and F of `depth` boundary planes (2 with PLM faces, 3 with PPM) with the
slabs below and above before each stage, and nothing else; the local solves
need no communication.  The slabs are advanced stage by stage through the
C ABI (rhd_slab_planes_get/_set, rhd_slab_stage, rhd_slab_status,
rhd_slab_commit); this module moves the planes between ranks with
torch.distributed point-to-point transfers (NCCL between GPUs, gloo on CPU)
and combines the slabs' statuses, so that a step is applied on every rank
or on none.

The schedule works on any object with the methods of CtxSlab (plane kinds
of rhd.h), which lets the host-side logic run without a GPU.  dist = None
is a single process holding the whole grid as one slab (its ghost planes
are its own opposite boundary planes).
"""
from __future__ import annotations

from . import rhd as R

UP, DOWN = 0, 1  # tags: planes moving to the slab above / below


class CtxSlab:
    """The slab of an RHDContext (a 3-D grid with HALO z faces) on `device`
    ("cuda": device buffers for NCCL; "cpu": host buffers for gloo)."""

    def __init__(self, ctx: "R.RHDContext", device: str = "cuda"):
        import torch
        self.ctx = ctx
        self.device = device
        bc = ctx.prob.get("bc", "periodic")
        zb = ["halo", "halo"] if isinstance(bc, str) else list(bc[2])
        self.low = zb[0] == "halo"
        self.high = zb[1] == "halo"
        self.tau = ctx.prob.get("hll_mode", "tau") == "tau"
        self._torch = torch

    def buffer(self, what: int):
        n = self.ctx.slab_plane_doubles(what)
        return self._torch.empty(n, dtype=self._torch.float64, device=self.device)

    def planes_get(self, what: int, stage: int):
        return self.ctx.slab_planes_get(what, stage, self.buffer(what))

    def planes_set(self, what: int, buf):
        self.ctx.slab_planes_set(what, buf)

    def stage(self, stage: int, dt: float):
        self.ctx.slab_stage(stage, dt)

    def status(self) -> int:
        return self.ctx.slab_status()["status"]

    def commit(self, ok: bool):
        self.ctx.slab_commit(ok)

    # the hydrodynamic step and the split (Sec. 3.1)
    def hydro_speed(self) -> float:
        return self.ctx.slab_hydro_speed()

    def hydro_phase(self, phase: int, dt: float):
        self.ctx.slab_hydro_phase(phase, dt)

    @property
    def cfl_hydro(self) -> float:
        return float(self.ctx.prob.get("cfl_hydro", 0.3))

    def radiation_dt(self) -> float:
        return R.rhd_default_dt(R.params_from_problem(self.ctx.prob))


def neighbours(rank: int, world: int, low: bool, high: bool):
    """Ranks of the slabs below and above (None where the face is not HALO);
    slab r sits above slab r - 1, the last above the first when z is
    periodic (both end faces HALO)."""
    return ((rank - 1) % world if low else None), ((rank + 1) % world if high else None)


def _transfer(dist, send, dst, recv_like, src, tag, group):
    """Send `send` to rank dst and receive a buffer like recv_like from rank
    src (either may be None); a transfer to this rank itself is a copy."""
    me = dist.get_rank(group) if dist is not None else 0
    if dst is not None and dst == me:
        return send.clone() if recv_like is not None else None
    ops = []
    recv = None
    if recv_like is not None and src is not None:
        recv = recv_like
        ops.append(dist.P2POp(dist.irecv, recv, src, group, tag))
    if send is not None and dst is not None:
        ops.append(dist.P2POp(dist.isend, send, dst, group, tag))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return recv


def exchange(slab, dist, what_up, what_down, set_up, set_down, stage=1, group=None):
    """One exchange round: every slab sends what_up (got with `stage`) to the
    slab above, which stores it as set_up, and what_down to the slab below,
    which stores it as set_down (None: no transfer in that direction).
    Upward transfers all finish before the downward ones start, so that each
    pair of ranks has one transfer in flight in each round."""
    world = dist.get_world_size(group) if dist is not None else 1
    rank = dist.get_rank(group) if dist is not None else 0
    below, above = neighbours(rank, world, slab.low, slab.high)
    if what_up is not None:
        send = slab.planes_get(what_up, stage) if above is not None else None
        like = slab.buffer(set_up) if below is not None else None
        got = _transfer(dist, send, above, like, below, UP, group)
        if got is not None:
            slab.planes_set(set_up, got)
    if what_down is not None:
        send = slab.planes_get(what_down, stage) if below is not None else None
        like = slab.buffer(set_down) if above is not None else None
        got = _transfer(dist, send, below, like, above, DOWN, group)
        if got is not None:
            slab.planes_set(set_down, got)


def exchange_material(slab, dist, group=None):
    """The planes the TAU factors of the slab faces need, after rho or kappa
    of any slab has changed: plane 0's kappa and rho go down, then the top
    face's factors go up."""
    if not slab.tau:
        return
    exchange(slab, dist, None, R.RHD_SLAB_MATERIAL_LOW, None, R.RHD_SLAB_MATERIAL_ABOVE,
             group=group)
    exchange(slab, dist, R.RHD_SLAB_EPS_HIGH, None, R.RHD_SLAB_EPS_BELOW, None, group=group)


def step(slab, dist, nsteps: int = 1, dt: float = 0.0, group=None) -> dict:
    """nsteps IMEX steps of the decomposed grid.  Returns {"steps_done",
    "status"}: the largest status code of any slab; a step that failed on
    any slab is applied on none, and the stepping stops there."""
    import torch
    # the status reduction: NCCL reduces device tensors, gloo host tensors
    dev = "cpu"
    if dist is not None and dist.get_backend(group) == "nccl":
        dev = getattr(slab, "device", "cpu")
    for k in range(nsteps):
        for stage in (1, 2):
            exchange(slab, dist, R.RHD_SLAB_BOUNDARY_HIGH, R.RHD_SLAB_BOUNDARY_LOW,
                     R.RHD_SLAB_GHOSTS_LOW, R.RHD_SLAB_GHOSTS_HIGH, stage, group)
            slab.stage(stage, dt)
        worst = slab.status()
        if dist is not None:
            st = torch.tensor([worst], dtype=torch.int64, device=dev)
            dist.all_reduce(st, op=dist.ReduceOp.MAX, group=group)
            worst = int(st.item())
        slab.commit(worst == R.RHD_OK)
        if worst != R.RHD_OK:
            return {"steps_done": k, "status": worst}
    return {"steps_done": nsteps, "status": R.RHD_OK}


def _reduce(dist, x, op, dev, group):
    """x reduced over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op, group=group)
    return float(t.item())


def _status_device(slab, dist, group):
    if dist is not None and dist.get_backend(group) == "nccl":
        return getattr(slab, "device", "cpu")
    return "cpu"


def hydro_step(slab, dist, nsteps: int = 1, dt: float = 0.0, group=None) -> dict:
    """nsteps hydrodynamic steps (RK2-SSP, HLLC faces) of the decomposed grid:
    the primitives' ghost planes exchanged before each stage's face fluxes;
    dt <= 0: before each step the whole grid's CFL step, cfl_hydro over the
    largest signal-speed bound of any slab.  A step that failed on any slab
    is committed on none.  Returns {"steps_done", "status", "dt"}."""
    dev = _status_device(slab, dist, group)
    h = dt
    for k in range(nsteps):
        if not (dt > 0.0):
            smax = _reduce(dist, slab.hydro_speed(), dist.ReduceOp.MAX if dist else None,
                           dev, group)
            if not (smax > 0.0) or smax == float("inf") or smax != smax:
                return {"steps_done": k, "status": R.RHD_ERR_NONPHYSICAL, "dt": h}
            h = slab.cfl_hydro / smax
        slab.hydro_phase(0, h)
        exchange(slab, dist, R.RHD_SLAB_PRIM_BOUNDARY_HIGH, R.RHD_SLAB_PRIM_BOUNDARY_LOW,
                 R.RHD_SLAB_PRIM_GHOSTS_LOW, R.RHD_SLAB_PRIM_GHOSTS_HIGH, 1, group)
        slab.hydro_phase(1, h)
        slab.hydro_phase(2, h)
        exchange(slab, dist, R.RHD_SLAB_PRIM_BOUNDARY_HIGH, R.RHD_SLAB_PRIM_BOUNDARY_LOW,
                 R.RHD_SLAB_PRIM_GHOSTS_LOW, R.RHD_SLAB_PRIM_GHOSTS_HIGH, 1, group)
        slab.hydro_phase(3, h)
        worst = slab.status()
        if dist is not None:
            worst = int(_reduce(dist, worst, dist.ReduceOp.MAX, dev, group))
        slab.commit(worst == R.RHD_OK)
        if worst != R.RHD_OK:
            return {"steps_done": k, "status": worst, "dt": h}
    return {"steps_done": nsteps, "status": R.RHD_OK, "dt": h}


def split_step(slab, dist, nsteps: int = 1, dt_h: float = 0.0, group=None) -> dict:
    """nsteps operator-split steps (Sec. 3.1): one hydrodynamic step of dt_h
    (<= 0: the CFL step), then ceil(dt_h / dt_rad) radiation steps of
    dt_h / nsub (dt_rad the radiation step of rhd_default_dt), the material
    planes exchanged again after the hydrodynamic step has moved rho.
    Returns {"steps_done", "status", "substeps"}."""
    import math
    subs = []
    for k in range(nsteps):
        r = hydro_step(slab, dist, 1, dt_h, group)
        if r["status"] != R.RHD_OK:
            return {"steps_done": k, "status": r["status"], "substeps": subs}
        h = r["dt"]
        nsub = max(1, math.ceil(h / slab.radiation_dt() - 1e-12))
        exchange_material(slab, dist, group)
        r = step(slab, dist, nsub, h / nsub, group)
        subs.append(nsub)
        if r["status"] != R.RHD_OK:
            return {"steps_done": k, "status": r["status"], "substeps": subs}
    return {"steps_done": nsteps, "status": R.RHD_OK, "substeps": subs}
