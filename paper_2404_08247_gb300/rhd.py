"""ctypes binding of the C ABI in ``include/rhd.h`` (librhd.so).

Argument marshalling only: every step of the radiation update runs in the
CUDA kernels behind the ABI.  The functions keep the C names; ``RHDContext``
adds a small object wrapper that accepts numpy arrays (host) or torch CUDA
tensors (device) in the (10, nz, ny, nx) field-major layout of
``paper_2404_08247_gb300.inputs``.

There is no fallback: if librhd.so is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# plane kinds of rhd_slab_planes_get / rhd_slab_planes_set
(RHD_SLAB_BOUNDARY_LOW, RHD_SLAB_BOUNDARY_HIGH, RHD_SLAB_GHOSTS_LOW, RHD_SLAB_GHOSTS_HIGH,
 RHD_SLAB_MATERIAL_LOW, RHD_SLAB_MATERIAL_ABOVE, RHD_SLAB_EPS_HIGH,
 RHD_SLAB_EPS_BELOW, RHD_SLAB_PRIM_BOUNDARY_LOW, RHD_SLAB_PRIM_BOUNDARY_HIGH,
 RHD_SLAB_PRIM_GHOSTS_LOW, RHD_SLAB_PRIM_GHOSTS_HIGH) = range(12)
RHD_OK, RHD_ERR_ARG, RHD_ERR_CUDA, RHD_ERR_NEWTON, RHD_ERR_OUTER, \
    RHD_ERR_NONPHYSICAL, RHD_ERR_TIMEOUT, RHD_ERR_STATE, RHD_ERR_BOUNDS = range(9)
STATUS_NAMES = {0: "ok", 1: "arg", 2: "cuda", 3: "newton", 4: "outer",
                5: "nonphysical", 6: "timeout", 7: "state", 8: "bounds"}
RHD_BC_PERIODIC, RHD_BC_REFLECT, RHD_BC_INFLOW, RHD_BC_HALO = 0, 1, 2, 3
RHD_SCHEME_IMEX_PDARS, RHD_SCHEME_RK2_SSP = 0, 1
RHD_CLOSURE_M1, RHD_CLOSURE_EDDINGTON = 0, 1
RHD_HLL_TAU, RHD_HLL_NONE = 0, 1
RHD_PREC_FP64, RHD_PREC_MIXED = 0, 1
RHD_RECON_PLM, RHD_RECON_PPM, RHD_RECON_PPM_CS = 0, 1, 2
RHD_NFIELDS = 10
(RHD_F_RHO, RHD_F_MX, RHD_F_MY, RHD_F_MZ, RHD_F_EGAS, RHD_F_ERAD, RHD_F_FX,
 RHD_F_FY, RHD_F_FZ, RHD_F_KAPPA) = range(10)

_BC = {"periodic": RHD_BC_PERIODIC, "reflect": RHD_BC_REFLECT, "inflow": RHD_BC_INFLOW,
       "halo": RHD_BC_HALO}
_SCHEME = {"imex": RHD_SCHEME_IMEX_PDARS, "rk2ssp": RHD_SCHEME_RK2_SSP}
_CLOSURE = {"m1": RHD_CLOSURE_M1, "eddington": RHD_CLOSURE_EDDINGTON}
_HLL = {"tau": RHD_HLL_TAU, "none": RHD_HLL_NONE}
_PREC = {"fp64": RHD_PREC_FP64, "mixed": RHD_PREC_MIXED}
_RECON = {"plm": RHD_RECON_PLM, "ppm": RHD_RECON_PPM, "ppm_cs": RHD_RECON_PPM_CS}


class RHDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class rhd_params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
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
        ("precision", ctypes.c_int),
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


class rhd_step_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("steps_done", ctypes.c_int),
        ("fail_cell", ctypes.c_int64),
        ("fail_step", ctypes.c_int),
        ("fail_stage", ctypes.c_int),
        ("max_newton", ctypes.c_int),
        ("max_outer", ctypes.c_int),
        ("sum_newton", ctypes.c_int64),
        ("n_solves", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("sum_outer", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every function the header declares: name -> (restype, argtypes)
_P = ctypes.POINTER(rhd_params)
_V = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64
SIGNATURES = {
    "rhd_params_default": (None, [_P]),
    "rhd_params_validate": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_int]),
    "rhd_default_dt": (ctypes.c_double, [_P]),
    "rhd_init": (ctypes.c_int, [_P, ctypes.POINTER(_V)]),
    "rhd_set_stream": (ctypes.c_int, [_V, _V]),
    "rhd_use_private_stream": (ctypes.c_int, [_V]),
    "rhd_state_set": (ctypes.c_int, [_V, ctypes.c_int, _V, _I64, ctypes.c_int]),
    "rhd_state_set_all": (ctypes.c_int, [_V, _V, _I64, ctypes.c_int]),
    "rhd_state_get": (ctypes.c_int, [_V, ctypes.c_int, _V, _I64, ctypes.c_int]),
    "rhd_state_get_all": (ctypes.c_int, [_V, _V, _I64, ctypes.c_int]),
    "rhd_stage_get": (ctypes.c_int, [_V, ctypes.c_int, _V, _I64, ctypes.c_int]),
    "rhd_step": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double,
                                ctypes.POINTER(rhd_step_info)]),
    "rhd_step_async": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double]),
    "rhd_sync": (ctypes.c_int, [_V, ctypes.POINTER(rhd_step_info)]),
    "rhd_step_host": (ctypes.c_int, [_V, _V, _V, _I64, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(rhd_step_info)]),
    "rhd_host_step_plan": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "rhd_transport": (ctypes.c_int, [_V, _V, _I64, ctypes.c_int]),
    "rhd_totals": (ctypes.c_int, [_V, _D]),
    "rhd_profile": (ctypes.c_int, [_V, ctypes.c_int]),
    "rhd_profile_read": (ctypes.c_int, [_V, ctypes.POINTER(_I64), _D]),
    "rhd_launch_count": (_I64, [_V]),
    "rhd_slab_plane_doubles": (_I64, [_V, ctypes.c_int]),
    "rhd_slab_planes_get": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int, _V, _I64,
                                           ctypes.c_int]),
    "rhd_slab_planes_set": (ctypes.c_int, [_V, ctypes.c_int, _V, _I64, ctypes.c_int]),
    "rhd_slab_stage": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double]),
    "rhd_slab_status": (ctypes.c_int, [_V, ctypes.POINTER(rhd_step_info)]),
    "rhd_slab_commit": (ctypes.c_int, [_V, ctypes.c_int]),
    "rhd_slab_hydro_speed": (ctypes.c_int, [_V, _D]),
    "rhd_slab_hydro_phase": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double]),
    "rhd_time": (ctypes.c_double, [_V]),
    "rhd_last_error": (ctypes.c_char_p, [_V]),
    "rhd_destroy": (None, [_V]),
    "rhd_step_record": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double, _V, _I64,
                                       ctypes.POINTER(rhd_step_info)]),
    "rhd_adjoint": (ctypes.c_int, [_V, _V, _I64, ctypes.c_int, ctypes.c_double, _V, _V]),
    "rhd_eval_recip": (ctypes.c_int, [_V, _I64, _V, _V]),
    "rhd_fma_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _V, _D]),
    "rhd_hydro_dt": (ctypes.c_int, [_V, _D]),
    "rhd_hydro_step": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(rhd_step_info)]),
    "rhd_step_split": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(rhd_step_info)]),
    "rhd_step_slabs": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.POINTER(rhd_step_info)]),
    "rhd_hydro_step_slabs": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.POINTER(rhd_step_info)]),
    "rhd_step_split_slabs": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.POINTER(rhd_step_info)]),
    "rhd_step_noalloc": (ctypes.c_int, [_P, _V, _V, ctypes.c_double, _V,
                                        ctypes.POINTER(rhd_step_info)]),
    "rhd_batch_init": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_V)]),
    "rhd_batch_set_stream": (ctypes.c_int, [_V, _V]),
    "rhd_batch_configure": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int]),
    "rhd_batch_use_graphs": (ctypes.c_int, [_V, ctypes.c_int]),
    "rhd_batch_cells": (_I64, [_V, ctypes.c_int]),
    "rhd_batch_state_set": (ctypes.c_int, [_V, ctypes.c_int, _V, _I64, ctypes.c_int]),
    "rhd_batch_state_get": (ctypes.c_int, [_V, ctypes.c_int, _V, _I64, ctypes.c_int]),
    "rhd_batch_step": (ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(rhd_step_info)]),
    "rhd_batch_locate": (ctypes.c_int, [_V, _I64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(_I64)]),
    "rhd_batch_last_error": (ctypes.c_char_p, [_V]),
    "rhd_batch_destroy": (None, [_V]),
}
RHD_NOALLOC_MAX_CELLS = 262144

_lib = None


def load(path: str | None = None):
    """Load librhd.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            "librhd.so not found at %s: build it with __graft_entry__.build() "
            "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st, ctx=None):
    if st != RHD_OK:
        msg = load().rhd_last_error(ctx)
        raise RHDError(st, msg.decode() if msg else "")


# ------------------------------------------------------------ thin wrappers

def rhd_params_default() -> rhd_params:
    p = rhd_params()
    load().rhd_params_default(ctypes.byref(p))
    return p


def rhd_params_validate(p: rhd_params):
    buf = ctypes.create_string_buffer(256)
    st = load().rhd_params_validate(ctypes.byref(p), buf, 256)
    return st, buf.value.decode()


def rhd_default_dt(p: rhd_params) -> float:
    return load().rhd_default_dt(ctypes.byref(p))


def params_from_problem(prob: dict, precision: str | int = "fp64") -> rhd_params:
    """rhd_params for a problem dict of ``paper_2404_08247_gb300.inputs``."""
    p = rhd_params_default()
    p.ndim = int(prob["ndim"])
    n = list(prob["n"]) + [1] * (3 - len(prob["n"]))
    dx = list(prob["dx"]) + [1.0] * (3 - len(prob["dx"]))
    bc = prob.get("bc", "periodic")
    for d in range(3):
        p.n[d] = int(n[d])
        p.dx[d] = float(dx[d])
        for s in range(2):
            kind = bc if isinstance(bc, str) else (bc[d][s] if d < len(bc) else "periodic")
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
    p.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    p.newton_rtol = float(prob.get("newton_rtol", 1e-13))
    p.outer_rtol = float(prob.get("outer_rtol", 1e-13))
    p.newton_max_iter = int(prob.get("newton_max_iter", 64))
    p.outer_max_iter = int(prob.get("outer_max_iter", 32))
    p.scheme = _SCHEME[prob.get("scheme", "imex")]
    p.kappa_T_exp = float(prob.get("kappa_T_exp", 0.0))
    p.kappa_T_ref = float(prob.get("kappa_T_ref", 1.0))
    p.kappa_P_ratio = float(prob.get("kappa_P_ratio", 1.0))
    p.kappa_F_ratio = float(prob.get("kappa_F_ratio", 1.0))
    p.reconstruction = _RECON[prob.get("reconstruction", "plm")]
    p.cfl_hydro = float(prob.get("cfl_hydro", 0.3))
    st = prob.get("bc_state", {})
    for d in range(3):
        for side in range(2):
            v = st.get((d, side), (1.0, 0.0, 0.0, 0.0)) if isinstance(st, dict) else st[d][side]
            for q in range(4):
                p.bc_state[d][side][q] = float(v[q])
    return p


def _ptr(x, count=None):
    """(pointer, on_device) of a numpy array or torch tensor (float64,
    contiguous) that holds at least `count` doubles: the library reads or
    writes `count` of them, so a smaller buffer is refused here instead of
    being overrun on the host or the device."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 array")
        ptr, dev, size = x.ctypes.data, 0, x.size
    else:  # torch tensor
        if str(x.dtype) != "torch.float64" or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor")
        ptr, dev, size = x.data_ptr(), 1 if x.is_cuda else 0, x.numel()
    if count is not None and size < count:
        raise ValueError("buffer holds %d doubles, the call needs %d" % (size, count))
    return ptr, dev


def host_step_plan(prob: dict) -> dict:
    """rhd_host_step_plan for a problem dict: {"cells": K + 1 offsets,
    "rows": K + 1 tile-row offsets, "stage1": [(a, b)], "stage2": [(a, b)]}.
    Host only."""
    p = params_from_problem(prob)
    cap = 64
    K = ctypes.c_int()
    cells = (_I64 * cap)()
    rows = (ctypes.c_int * cap)()
    groups = (ctypes.c_int * (2 * cap))()
    ng = (ctypes.c_int * 2)()
    _check(load().rhd_host_step_plan(ctypes.byref(p), ctypes.byref(K), cells, rows, groups, ng,
                                     cap))
    n = K.value
    pairs = [(groups[2 * j], groups[2 * j + 1]) for j in range(ng[0] + ng[1])]
    return {"cells": list(cells[: n + 1]), "rows": list(rows[: n + 1]),
            "stage1": pairs[: ng[0]], "stage2": pairs[ng[0]:]}


def eval_recip(x):
    """rhd_eval_recip on a float64 CUDA tensor: (1/x, 1/sqrt(x)) as computed by
    the FP64 kernels."""
    import torch
    if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    r = torch.empty_like(x)
    q = torch.empty_like(x)
    torch.cuda.synchronize()
    _check(load().rhd_eval_recip(ctypes.c_void_p(x.data_ptr()), int(x.numel()),
                                 ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(q.data_ptr())))
    return r, q


def fma_probe(precision: str, nblocks: int, iters: int, stream=None) -> float:
    """rhd_fma_probe: launch the multiply-add throughput probe of the FP64
    ("fp64") or single-precision ("fp32") pipe on `stream` (a torch stream;
    None: the current one) without synchronising; returns its flop count."""
    import torch
    prec = {"fp64": RHD_PREC_FP64, "fp32": RHD_PREC_MIXED}[precision]
    st = stream if stream is not None else torch.cuda.current_stream()
    flops = ctypes.c_double(0.0)
    _check(load().rhd_fma_probe(prec, int(nblocks), int(iters), ctypes.c_void_p(st.cuda_stream),
                                ctypes.byref(flops)))
    return flops.value


class RHDContext:
    """One grid's device state behind the C ABI."""

    def __init__(self, prob: dict, precision="fp64", stream=None):
        self.lib = load()
        self.prob = prob
        self.params = params_from_problem(prob, precision)
        h = ctypes.c_void_p()
        _check(self.lib.rhd_init(ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h
        n = self.params.n
        self.ncell = int(n[0] * n[1] * n[2])
        self.shape = (RHD_NFIELDS, int(n[2]), int(n[1]), int(n[0]))
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.rhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream or an integer cudaStream_t handle (0 is
        CUDA's legacy default stream, torch's default); None switches back to
        the context's private stream."""
        if stream is None:
            _check(self.lib.rhd_use_private_stream(self.h), self.h)
            return
        handle = getattr(stream, "cuda_stream", stream)
        _check(self.lib.rhd_set_stream(self.h, ctypes.c_void_p(int(handle))), self.h)

    def set_state(self, U):
        ptr, dev = _ptr(U, RHD_NFIELDS * self.ncell)
        _check(self.lib.rhd_state_set_all(self.h, ctypes.c_void_p(ptr),
                                          RHD_NFIELDS * self.ncell, dev), self.h)

    def set_field(self, field: int, x):
        ptr, dev = _ptr(x, self.ncell)
        _check(self.lib.rhd_state_set(self.h, field, ctypes.c_void_p(ptr),
                                      self.ncell, dev), self.h)

    def get_state(self, out=None):
        """The state (10 fields) into `out`, or into a new array that starts as
        NaN, so that a cell the library failed to write cannot pass as data."""
        if out is None:
            out = np.full(self.shape, np.nan)
        ptr, dev = _ptr(out, RHD_NFIELDS * self.ncell)
        _check(self.lib.rhd_state_get_all(self.h, ctypes.c_void_p(ptr),
                                          RHD_NFIELDS * self.ncell, dev), self.h)
        return out

    def get_field(self, field: int, out=None):
        if out is None:
            out = np.full(self.shape[1:], np.nan)
        ptr, dev = _ptr(out, self.ncell)
        _check(self.lib.rhd_state_get(self.h, field, ctypes.c_void_p(ptr),
                                      self.ncell, dev), self.h)
        return out

    def get_stage_field(self, field: int, out=None):
        """One evolved field of y(n+1/2) of the last step."""
        if out is None:
            out = np.full(self.shape[1:], np.nan)
        ptr, dev = _ptr(out, self.ncell)
        _check(self.lib.rhd_stage_get(self.h, field, ctypes.c_void_p(ptr), self.ncell, dev),
               self.h)
        return out

    def step(self, nsteps: int = 1, dt: float = 0.0, raise_on_error=True) -> dict:
        info = rhd_step_info()
        st = self.lib.rhd_step(self.h, int(nsteps), float(dt), ctypes.byref(info))
        if raise_on_error:
            _check(st, self.h)
        d = info.as_dict()
        d["status"] = st
        return d

    def step_host(self, src, dst=None, nsteps: int = 1, dt: float = 0.0,
                  raise_on_error=True) -> dict:
        """rhd_step_host: step the host state `src` (10 fields, numpy array or
        CPU tensor; pinned memory lets the copies overlap the kernels) and write
        the result to `dst` (default: a new array that starts as NaN; may be
        src).  Returns the step info with "out" = dst."""
        if dst is None:
            dst = np.full(self.shape, np.nan)
        ps, ds = _ptr(src, RHD_NFIELDS * self.ncell)
        pd, dd = _ptr(dst, RHD_NFIELDS * self.ncell)
        if ds or dd:
            raise ValueError("step_host takes host buffers")
        info = rhd_step_info()
        st = self.lib.rhd_step_host(self.h, ctypes.c_void_p(ps), ctypes.c_void_p(pd),
                                    RHD_NFIELDS * self.ncell, int(nsteps), float(dt),
                                    ctypes.byref(info))
        if raise_on_error:
            _check(st, self.h)
        d = info.as_dict()
        d["status"] = st
        d["out"] = dst
        return d

    # ---- one z-slab stepped stage by stage by its own process
    def slab_plane_doubles(self, what: int) -> int:
        return int(self.lib.rhd_slab_plane_doubles(self.h, int(what)))

    def slab_planes_get(self, what: int, stage: int, out):
        """rhd_slab_planes_get into `out` (numpy array or torch tensor of
        slab_plane_doubles(what) doubles)."""
        ptr, dev = _ptr(out)
        _check(self.lib.rhd_slab_planes_get(self.h, int(what), int(stage), ctypes.c_void_p(ptr),
                                            int(out.size if isinstance(out, np.ndarray)
                                                else out.numel()), dev), self.h)
        return out

    def slab_planes_set(self, what: int, src):
        ptr, dev = _ptr(src)
        _check(self.lib.rhd_slab_planes_set(self.h, int(what), ctypes.c_void_p(ptr),
                                            int(src.size if isinstance(src, np.ndarray)
                                                else src.numel()), dev), self.h)

    def slab_stage(self, stage: int, dt: float = 0.0):
        _check(self.lib.rhd_slab_stage(self.h, int(stage), float(dt)), self.h)

    def slab_status(self) -> dict:
        """rhd_slab_status: the slab's own status (not raised) and counts."""
        info = rhd_step_info()
        st = self.lib.rhd_slab_status(self.h, ctypes.byref(info))
        d = info.as_dict()
        d["status"] = st
        return d

    def slab_commit(self, commit: bool):
        _check(self.lib.rhd_slab_commit(self.h, int(bool(commit))), self.h)

    def slab_hydro_speed(self) -> float:
        smax = ctypes.c_double(0.0)
        _check(self.lib.rhd_slab_hydro_speed(self.h, ctypes.byref(smax)), self.h)
        return smax.value

    def slab_hydro_phase(self, phase: int, dt: float = 0.0):
        _check(self.lib.rhd_slab_hydro_phase(self.h, int(phase), float(dt)), self.h)

    def step_async(self, nsteps: int = 1, dt: float = 0.0):
        _check(self.lib.rhd_step_async(self.h, int(nsteps), float(dt)), self.h)

    def sync(self, raise_on_error=True) -> dict:
        info = rhd_step_info()
        st = self.lib.rhd_sync(self.h, ctypes.byref(info))
        if raise_on_error:
            _check(st, self.h)
        return info.as_dict()

    def hydro_dt(self) -> float:
        """dt of the hydrodynamic step of the current state (Sec. 3.1)."""
        out = ctypes.c_double(0.0)
        _check(self.lib.rhd_hydro_dt(self.h, ctypes.byref(out)), self.h)
        return out.value

    def hydro_step(self, nsteps: int = 1, dt: float = 0.0, raise_on_error=True) -> dict:
        """nsteps RK2-SSP steps of the hydrodynamic subsystem alone."""
        info = rhd_step_info()
        st = self.lib.rhd_hydro_step(self.h, int(nsteps), float(dt), ctypes.byref(info))
        if raise_on_error:
            _check(st, self.h)
        return info.as_dict()

    def step_split(self, nsteps: int = 1, dt_h: float = 0.0, raise_on_error=True) -> dict:
        """nsteps operator-split steps: hydrodynamics, then the subcycled
        radiation update (Sec. 3.1)."""
        info = rhd_step_info()
        st = self.lib.rhd_step_split(self.h, int(nsteps), float(dt_h), ctypes.byref(info))
        if raise_on_error:
            _check(st, self.h)
        return info.as_dict()

    def transport(self, out=None):
        """Rates (dE/dt, dFx/dt, dFy/dt, dFz/dt) of s(y), shape (4, nz, ny, nx)."""
        if out is None:
            out = np.full((4,) + self.shape[1:], np.nan)
        ptr, dev = _ptr(out, 4 * self.ncell)
        _check(self.lib.rhd_transport(self.h, ctypes.c_void_p(ptr), 4 * self.ncell, dev),
               self.h)
        return out

    def totals(self) -> np.ndarray:
        out = np.zeros(4, dtype=np.float64)
        _check(self.lib.rhd_totals(self.h, out.ctypes.data_as(_D)), self.h)
        return out

    def profile(self, enable: bool):
        _check(self.lib.rhd_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self):
        launches = (_I64 * 3)()
        ms = (ctypes.c_double * 3)()
        _check(self.lib.rhd_profile_read(self.h, launches, ms), self.h)
        return list(launches), list(ms)

    def step_record(self, nsteps: int, dt: float, tape) -> dict:
        """rhd_step_record: nsteps steps that also write the tape (a device
        tensor of (2*nsteps+1)*8*ncell float64)."""
        ptr, dev = _ptr(tape)
        if not dev:
            raise ValueError("the tape must be a device tensor")
        info = rhd_step_info()
        _check(self.lib.rhd_step_record(self.h, int(nsteps), float(dt), ctypes.c_void_p(ptr),
                                        int(tape.numel()), ctypes.byref(info)), self.h)
        return info.as_dict()

    def adjoint(self, tape, nsteps: int, dt: float, ybar, kappa_bar):
        """rhd_adjoint: ybar (device, 8*ncell) from dL/dy(nsteps) to dL/dy(0) in
        place; dL/dkappa added to kappa_bar (device, ncell)."""
        tp, td = _ptr(tape)
        yp, yd = _ptr(ybar)
        kp, kd = _ptr(kappa_bar)
        if not (td and yd and kd):
            raise ValueError("tape, ybar and kappa_bar must be device tensors")
        if ybar.numel() != 8 * self.ncell or kappa_bar.numel() != self.ncell:
            raise ValueError("ybar must hold 8*ncell and kappa_bar ncell values")
        _check(self.lib.rhd_adjoint(self.h, ctypes.c_void_p(tp), int(tape.numel()),
                                    int(nsteps), float(dt), ctypes.c_void_p(yp),
                                    ctypes.c_void_p(kp)), self.h)

    def launch_count(self) -> int:
        return int(self.lib.rhd_launch_count(self.h))

    def time(self) -> float:
        return float(self.lib.rhd_time(self.h))

    def default_dt(self) -> float:
        return rhd_default_dt(self.params)


def slab_problems(prob: dict, cuts) -> list:
    """Problem dicts of the z-slabs [cuts[i], cuts[i+1]) of a 3-D problem for
    rhd_step_slabs (cuts from 0 to n[2], each slab >= 3 planes): the faces
    between slabs become "halo"; a periodic z axis makes the outer faces
    "halo" too (they face each other), otherwise they keep their kind."""
    if int(prob["ndim"]) != 3:
        raise ValueError("slabs are z ranges of a 3-D grid")
    cuts = [int(c) for c in cuts]
    if cuts[0] != 0 or cuts[-1] != int(prob["n"][2]) or len(cuts) < 2:
        raise ValueError("cuts must run from 0 to n[2]")
    bc = prob.get("bc", "periodic")
    axes = [[bc, bc] for _ in range(3)] if isinstance(bc, str) else \
        [list(bc[d]) if d < len(bc) else ["periodic", "periodic"] for d in range(3)]
    zper = axes[2][0] == "periodic"
    out = []
    for i in range(len(cuts) - 1):
        q = dict(prob)
        n = list(prob["n"])
        n[2] = cuts[i + 1] - cuts[i]
        q["n"] = n
        lo = "halo" if (i > 0 or zper) else axes[2][0]
        hi = "halo" if (i < len(cuts) - 2 or zper) else axes[2][1]
        q["bc"] = [axes[0], axes[1], [lo, hi]]
        out.append(q)
    return out


def _slab_call(fn, contexts, nsteps, dt, raise_on_error):
    arr = (_V * len(contexts))(*[c.h.value for c in contexts])
    info = rhd_step_info()
    st = fn(arr, len(contexts), int(nsteps), float(dt), ctypes.byref(info))
    if raise_on_error:
        _check(st, contexts[0].h)
    d = info.as_dict()
    d["status"] = st
    return d


def step_slabs(contexts, nsteps: int = 1, dt: float = 0.0, raise_on_error=True) -> dict:
    """rhd_step_slabs: nsteps radiation steps of the z-slabs (RHDContext,
    bottom to top) of one grid, the ghost planes exchanged before every stage."""
    return _slab_call(load().rhd_step_slabs, contexts, nsteps, dt, raise_on_error)


def hydro_step_slabs(contexts, nsteps: int = 1, dt: float = 0.0, raise_on_error=True) -> dict:
    """rhd_hydro_step_slabs: nsteps hydrodynamic steps of the z-slabs."""
    return _slab_call(load().rhd_hydro_step_slabs, contexts, nsteps, dt, raise_on_error)


def step_split_slabs(contexts, nsteps: int = 1, dt_h: float = 0.0,
                     raise_on_error=True) -> dict:
    """rhd_step_split_slabs: nsteps operator-split steps of the z-slabs."""
    return _slab_call(load().rhd_step_split_slabs, contexts, nsteps, dt_h, raise_on_error)


class RHDBatch:
    """Many independent 1-D/2-D problems behind the rhd_batch C ABI."""

    TILES = {0: (32, 8), 1: (64, 4), 2: (16, 16)}

    def __init__(self, probs, precision="fp64", stream=None):
        self.lib = load()
        self.probs = list(probs)
        arr = (rhd_params * len(self.probs))(
            *[params_from_problem(p, precision) for p in self.probs])
        h = ctypes.c_void_p()
        _check(self.lib.rhd_batch_init(arr, len(self.probs), ctypes.byref(h)))
        self.h = h
        self.shapes = [(RHD_NFIELDS, int(p["n"][2]), int(p["n"][1]), int(p["n"][0]))
                       for p in self.probs]
        if stream is not None:
            self.set_stream(stream)

    def _check(self, st):
        if st != RHD_OK:
            msg = self.lib.rhd_batch_last_error(self.h)
            raise RHDError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.rhd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.rhd_batch_set_stream(self.h, ctypes.c_void_p(int(handle or 0))))

    def configure(self, tile2d: int, blocks_per_sm: int):
        self._check(self.lib.rhd_batch_configure(self.h, int(tile2d), int(blocks_per_sm)))

    def use_graphs(self, enable: bool):
        """rhd_batch_use_graphs: replay captured CUDA graphs (default) or
        enqueue each step's launches directly."""
        self._check(self.lib.rhd_batch_use_graphs(self.h, int(bool(enable))))

    def cells(self, prob: int = -1) -> int:
        return int(self.lib.rhd_batch_cells(self.h, prob))

    def set_state(self, prob: int, U):
        ptr, dev = _ptr(U, RHD_NFIELDS * self.cells(prob))
        self._check(self.lib.rhd_batch_state_set(self.h, prob, ctypes.c_void_p(ptr),
                                                 RHD_NFIELDS * self.cells(prob), dev))

    def get_state(self, prob: int, out=None):
        if out is None:
            out = np.full(self.shapes[prob], np.nan)
        ptr, dev = _ptr(out, RHD_NFIELDS * self.cells(prob))
        self._check(self.lib.rhd_batch_state_get(self.h, prob, ctypes.c_void_p(ptr),
                                                 RHD_NFIELDS * self.cells(prob), dev))
        return out

    def step(self, nsteps: int = 1, raise_on_error=True) -> dict:
        info = rhd_step_info()
        st = self.lib.rhd_batch_step(self.h, int(nsteps), ctypes.byref(info))
        if raise_on_error:
            self._check(st)
        d = info.as_dict()
        d["status"] = st
        return d

    def locate(self, pooled_cell: int):
        p = ctypes.c_int()
        c = _I64()
        self._check(self.lib.rhd_batch_locate(self.h, int(pooled_cell), ctypes.byref(p),
                                              ctypes.byref(c)))
        return p.value, c.value
