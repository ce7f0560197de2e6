"""Python access to the serial FP64 CPU oracle in ``rhd_oracle.c``, its
adjoint in ``rhd_oracle_adj.c`` and the hydrodynamic subsystem with the
operator split in ``rhd_oracle_hydro.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The library never imports
this module and shares no code with it.

The oracle is compiled with ``-O2 -ffp-contract=off`` so that x86-64 and
aarch64 hosts evaluate the same expressions in the same way.

Problem descriptions are plain dicts (see ``paper_2404_08247_gb300.inputs``);
this module maps them onto the oracle's own ``orc_params`` struct.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rhd_oracle.c")
SRC_ADJ = os.path.join(HERE, "rhd_oracle_adj.c")
SRC_HYD = os.path.join(HERE, "rhd_oracle_hydro.c")
HDR = os.path.join(HERE, "rhd_oracle.h")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liborc.so")

NFIELD = 10
FIELDS = ("rho", "mx", "my", "mz", "egas", "erad", "fx", "fy", "fz", "kappa")
STATUS = {0: "ok", 1: "arg", 3: "newton", 4: "outer", 5: "nonphysical"}

_BC = {"periodic": 0, "reflect": 1, "inflow": 2}
_SCHEME = {"imex": 0, "rk2ssp": 1}
_CLOSURE = {"m1": 0, "eddington": 1}
_HLL = {"tau": 0, "none": 1}


def build(force: bool = False) -> str:
    """Compile the oracle into ``_build/liborc.so`` (if missing or stale)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    stale = force or not os.path.exists(LIB)
    if not stale:
        t = os.path.getmtime(LIB)
        stale = any(os.path.getmtime(f) > t for f in (SRC, SRC_ADJ, SRC_HYD, HDR))
    if stale:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, SRC, SRC_ADJ, SRC_HYD, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_longlong * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("gamma", ctypes.c_double),
        ("c", ctypes.c_double),
        ("chat", ctypes.c_double),
        ("a_rad", ctypes.c_double),
        ("kB_over_mu", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("closure", ctypes.c_int),
        ("vc_order", ctypes.c_int),
        ("hll_mode", ctypes.c_int),
        ("newton_rtol", ctypes.c_double),
        ("outer_rtol", ctypes.c_double),
        ("newton_max_iter", ctypes.c_int),
        ("outer_max_iter", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("kappa_T_exp", ctypes.c_double),
        ("kappa_T_ref", ctypes.c_double),
        ("bc_state", ((ctypes.c_double * 4) * 2) * 3),
        ("kappa_P_ratio", ctypes.c_double),
        ("kappa_F_ratio", ctypes.c_double),
        ("reconstruction", ctypes.c_int),
        ("cfl_hydro", ctypes.c_double),
    ]


class OrcInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("fail_cell", ctypes.c_longlong),
        ("max_newton", ctypes.c_int),
        ("max_outer", ctypes.c_int),
        ("sum_newton", ctypes.c_longlong),
        ("n_solves", ctypes.c_longlong),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(OrcParams)
        L.orc_dt.argtypes = [P]
        L.orc_dt.restype = ctypes.c_double
        L.orc_eddington_tensor.argtypes = [P, ctypes.c_double, dp, dp]
        L.orc_eddington_tensor.restype = None
        L.orc_transport.argtypes = [P, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.orc_transport.restype = ctypes.c_int
        L.orc_hydro_dt.argtypes = [P, dp]
        L.orc_hydro_dt.restype = ctypes.c_double
        L.orc_hydro_rate.argtypes = [P, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.orc_hydro_rate.restype = ctypes.c_int
        L.orc_hydro_step.argtypes = [P, dp, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_longlong)]
        L.orc_hydro_step.restype = ctypes.c_int
        L.orc_split_step.argtypes = [P, dp, ctypes.c_double, ctypes.POINTER(OrcInfo),
                                     ctypes.POINTER(ctypes.c_int)]
        L.orc_split_step.restype = ctypes.c_int
        L.orc_local_solve.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, dp,
                                      ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
        L.orc_local_solve.restype = ctypes.c_int
        L.orc_step.argtypes = [P, dp, ctypes.c_double, ctypes.POINTER(OrcInfo)]
        L.orc_step.restype = ctypes.c_int
        L.orc_totals.argtypes = [P, dp, dp]
        L.orc_totals.restype = None
        L.orc_step_tape.argtypes = [P, dp, ctypes.c_double, dp]
        L.orc_step_tape.restype = ctypes.c_int
        L.orc_step_adjoint.argtypes = [P, dp, dp, dp, ctypes.c_double, dp, dp, dp]
        L.orc_step_adjoint.restype = ctypes.c_int
        L.orc_local_solve_adjoint.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, dp, dp,
                                              dp, dp]
        L.orc_local_solve_adjoint.restype = ctypes.c_int
        _lib = L
    return _lib


def make_params(prob: dict) -> OrcParams:
    """Map a problem dict onto ``orc_params``."""
    p = OrcParams()
    p.ndim = int(prob["ndim"])
    n = list(prob["n"]) + [1] * (3 - len(prob["n"]))
    dx = list(prob["dx"]) + [1.0] * (3 - len(prob["dx"]))
    for d in range(3):
        p.n[d] = int(n[d])
        p.dx[d] = float(dx[d])
    bc = prob.get("bc", "periodic")
    for d in range(3):
        for s in range(2):
            kind = bc if isinstance(bc, str) else (
                bc[d][s] if d < len(bc) else "periodic")
            p.bc[d][s] = _BC[kind]
    p.gamma = float(prob["gamma"])
    p.c = float(prob["c"])
    p.chat = float(prob["chat"])
    p.a_rad = float(prob.get("a_rad", 1.0))
    p.kB_over_mu = float(prob.get("kB_over_mu", 1.0))
    p.cfl = float(prob.get("cfl", 0.4))
    p.closure = _CLOSURE[prob.get("closure", "m1")]
    p.vc_order = int(prob.get("vc_order", 2))
    p.hll_mode = _HLL[prob.get("hll_mode", "tau")]
    p.newton_rtol = float(prob.get("newton_rtol", 1e-13))
    p.outer_rtol = float(prob.get("outer_rtol", 1e-13))
    p.newton_max_iter = int(prob.get("newton_max_iter", 64))
    p.outer_max_iter = int(prob.get("outer_max_iter", 32))
    p.scheme = _SCHEME[prob.get("scheme", "imex")]
    p.kappa_T_exp = float(prob.get("kappa_T_exp", 0.0))
    p.kappa_T_ref = float(prob.get("kappa_T_ref", 1.0))
    p.kappa_P_ratio = float(prob.get("kappa_P_ratio", 1.0))
    p.kappa_F_ratio = float(prob.get("kappa_F_ratio", 1.0))
    p.reconstruction = {"plm": 0, "ppm": 1, "ppm_cs": 2}[prob.get("reconstruction", "plm")]
    p.cfl_hydro = float(prob.get("cfl_hydro", 0.3))
    # bc_state[d][side] = (E, Fx, Fy, Fz) of inflow faces; default E = 1, F = 0
    st = prob.get("bc_state", {})
    for d in range(3):
        for side in range(2):
            v = st.get((d, side), (1.0, 0.0, 0.0, 0.0)) if isinstance(st, dict) else st[d][side]
            for q in range(4):
                p.bc_state[d][side][q] = float(v[q])
    return p


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dt(prob: dict) -> float:
    p = make_params(prob)
    return lib().orc_dt(ctypes.byref(p))


def step(prob: dict, U: np.ndarray, nsteps: int = 1, dt: float = 0.0,
         raise_on_error: bool = True):
    """Advance U (shape (10, nz, ny, nx) float64, modified in place) by nsteps.

    Returns a list with one info dict per step taken."""
    p = make_params(prob)
    infos = []
    for _ in range(nsteps):
        info = OrcInfo()
        st = lib().orc_step(ctypes.byref(p), _dptr(U), float(dt), ctypes.byref(info))
        d = {k: getattr(info, k) for k, _ in OrcInfo._fields_}
        infos.append(d)
        if st != 0:
            if raise_on_error:
                raise RuntimeError("oracle step failed: %s at cell %d"
                                   % (STATUS.get(st, st), info.fail_cell))
            break
    return infos


def transport(prob: dict, U: np.ndarray) -> np.ndarray:
    """Rates (dE/dt, dFx/dt, dFy/dt, dFz/dt) of s(y), shape (4, nz, ny, nx)."""
    p = make_params(prob)
    rate = np.zeros((4,) + U.shape[1:], dtype=np.float64)
    fc = ctypes.c_longlong(-1)
    st = lib().orc_transport(ctypes.byref(p), _dptr(U), _dptr(rate), ctypes.byref(fc))
    if st != 0:
        raise RuntimeError("oracle transport failed at cell %d" % fc.value)
    return rate


def local_solve(prob: dict, theta: float, dt: float, rho: float, chi: float,
                y) -> tuple:
    """One cell's implicit solve.  y = (Egas, mx, my, mz, E, Fx, Fy, Fz).

    Returns (status, y_out, n_newton, n_outer)."""
    p = make_params(prob)
    yy = np.ascontiguousarray(np.asarray(y, dtype=np.float64).copy())
    nn = ctypes.c_int(0)
    no = ctypes.c_int(0)
    st = lib().orc_local_solve(ctypes.byref(p), float(theta), float(dt), float(rho),
                               float(chi), _dptr(yy), ctypes.byref(nn),
                               ctypes.byref(no))
    return st, yy, nn.value, no.value


def eddington_tensor(prob: dict, E: float, F) -> np.ndarray:
    p = make_params(prob)
    FF = np.ascontiguousarray(np.asarray(F, dtype=np.float64))
    D = np.zeros((3, 3), dtype=np.float64)
    lib().orc_eddington_tensor(ctypes.byref(p), float(E), _dptr(FF), _dptr(D))
    return D


def totals(prob: dict, U: np.ndarray) -> np.ndarray:
    p = make_params(prob)
    out = np.zeros(4, dtype=np.float64)
    lib().orc_totals(ctypes.byref(p), _dptr(U), _dptr(out))
    return out


# ------------------------------------------------------------------ adjoint

SLOT_FIELDS = ("egas", "mx", "my", "mz", "erad", "fx", "fy", "fz")
SLOT_INDEX = tuple(FIELDS.index(f) for f in SLOT_FIELDS)


def step_tape(prob: dict, U: np.ndarray, dt: float = 0.0) -> np.ndarray:
    """One step of U (modified in place); returns the tape, shape
    (3, 8) + grid: y(n), y(n+1/2), y(n+1) in the slot order SLOT_FIELDS."""
    p = make_params(prob)
    tape = np.zeros((3, 8) + U.shape[1:], dtype=np.float64)
    st = lib().orc_step_tape(ctypes.byref(p), _dptr(U), float(dt), _dptr(tape))
    if st != 0:
        raise RuntimeError("oracle taped step failed: %s" % STATUS.get(st, st))
    return tape


def step_adjoint(prob: dict, rho: np.ndarray, kappa: np.ndarray, tape: np.ndarray,
                 ybar1: np.ndarray, kbar: np.ndarray, dt: float = 0.0) -> np.ndarray:
    """Adjoint of one taped step: returns dL/dy(n) (8 slots) from
    ybar1 = dL/dy(n+1); adds dL/dkappa into kbar (modified in place)."""
    p = make_params(prob)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    ybar1 = np.ascontiguousarray(ybar1, dtype=np.float64)
    ybar0 = np.zeros_like(ybar1)
    assert kbar.dtype == np.float64 and kbar.flags["C_CONTIGUOUS"]
    st = lib().orc_step_adjoint(ctypes.byref(p), _dptr(rho), _dptr(kappa), _dptr(tape),
                                float(dt), _dptr(ybar1), _dptr(ybar0), _dptr(kbar))
    if st != 0:
        raise RuntimeError("oracle step adjoint failed: %s" % STATUS.get(st, st))
    return ybar0


def local_solve_adjoint(prob: dict, theta: float, dt: float, rho: float, chi: float,
                        yout, ybar_out) -> tuple:
    """Adjoint of one converged local solve with output yout.
    Returns (status, ybar_in, chibar)."""
    p = make_params(prob)
    y = np.ascontiguousarray(np.asarray(yout, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(ybar_out, dtype=np.float64))
    bin_ = np.zeros(8, dtype=np.float64)
    cb = np.zeros(1, dtype=np.float64)
    st = lib().orc_local_solve_adjoint(ctypes.byref(p), float(theta), float(dt),
                                       float(rho), float(chi), _dptr(y), _dptr(b),
                                       _dptr(bin_), _dptr(cb))
    return st, bin_, float(cb[0])


def trajectory_gradient(prob: dict, U0: np.ndarray, nsteps: int, loss_grad,
                        dt: float = 0.0):
    """Reverse-mode gradient of a loss of the final state after nsteps.

    loss_grad(U_final) -> (L, dL/dU_final as 8 slots).  Returns
    (L, ybar0 (8 slots, dL/dy(0)), kbar (dL/dkappa)).  Keeps every tape."""
    U = U0.copy()
    tapes = [step_tape(prob, U, dt) for _ in range(nsteps)]
    L, ybar = loss_grad(U)
    rho = U0[FIELDS.index("rho")]
    kappa = U0[FIELDS.index("kappa")]
    kbar = np.zeros_like(rho)
    for tape in reversed(tapes):
        ybar = step_adjoint(prob, rho, kappa, tape, ybar, kbar, dt)
    return L, ybar, kbar


# ------------------------------------------------ hydrodynamics (Sec. 3.1)

def hydro_dt(prob: dict, U: np.ndarray) -> float:
    """cfl_hydro / max_cells sum_d (|v_d| + a) / dx_d."""
    return lib().orc_hydro_dt(ctypes.byref(make_params(prob)), _dptr(U))


def hydro_rate(prob: dict, U: np.ndarray) -> np.ndarray:
    """d(rho, mx, my, mz, Egas)/dt of the Euler equations, shape (5, nz, ny, nx)."""
    rate = np.zeros((5,) + U.shape[1:], dtype=np.float64)
    fc = ctypes.c_longlong(-1)
    st = lib().orc_hydro_rate(ctypes.byref(make_params(prob)), _dptr(U), _dptr(rate),
                              ctypes.byref(fc))
    if st != 0:
        raise RuntimeError("oracle hydro rate failed: %s at cell %d"
                           % (STATUS.get(st, st), fc.value))
    return rate


def hydro_step(prob: dict, U: np.ndarray, nsteps: int = 1, dt: float = 0.0):
    """nsteps RK2-SSP steps of the hydrodynamic subsystem (U in place); dt <= 0
    takes hydro_dt of the state at each step."""
    p = make_params(prob)
    for _ in range(nsteps):
        h = dt if dt > 0.0 else lib().orc_hydro_dt(ctypes.byref(p), _dptr(U))
        fc = ctypes.c_longlong(-1)
        st = lib().orc_hydro_step(ctypes.byref(p), _dptr(U), float(h), ctypes.byref(fc))
        if st != 0:
            raise RuntimeError("oracle hydro step failed: %s at cell %d"
                               % (STATUS.get(st, st), fc.value))


def split_step(prob: dict, U: np.ndarray, nsteps: int = 1, dt_h: float = 0.0):
    """nsteps operator-split steps (hydrodynamics, then the subcycled
    radiation step); returns the list of subcycle counts."""
    p = make_params(prob)
    subs = []
    for _ in range(nsteps):
        info = OrcInfo()
        ns = ctypes.c_int(0)
        st = lib().orc_split_step(ctypes.byref(p), _dptr(U), float(dt_h), ctypes.byref(info),
                                  ctypes.byref(ns))
        if st != 0:
            raise RuntimeError("oracle split step failed: %s at cell %d"
                               % (STATUS.get(st, st), info.fail_cell))
        subs.append(ns.value)
    return subs

