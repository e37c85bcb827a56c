"""ctypes binding of libqg (include/qg.h), same entry-point names.

Argument marshalling only: every step of the evaluation and of the Adam update
runs in the library's CUDA kernels.  Device buffers are torch CUDA tensors
(contiguous; float64 in QG_FP64 mode, float32 in QG_MIXED mode; obj float64).
If the shared library is missing, importing this module raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .build import LIB

QG_OK = 0
QG_ERR_INVALID_ARG = -1
QG_ERR_ISLANDING = -2
QG_ERR_CUDA = -3
QG_ERR_NOT_CONVERGED = -4
QG_ERR_TIMEOUT = -5
QG_ERR_NONFINITE = -6
QG_ERR_NO_DEVICE = -7
QG_ERR_UNSUPPORTED = -8
QG_FP64, QG_MIXED = 0, 1
QG_LODF_F32, QG_LODF_BF16, QG_LODF_BF16X2 = 0, 1, 2
QG_DC_AUTO, QG_DC_DENSE, QG_DC_SPARSE = 0, 1, 2
QG_CTG_BOUND_AUTO, QG_CTG_BOUND_OFF, QG_CTG_BOUND_EAGER, QG_CTG_BOUND_LAZY = 0, 1, 2, 3

TERM_NAMES = ("cost", "zp", "zq", "zs", "zrz", "zhead", "zramp", "zctg")

_I32P = C.POINTER(C.c_int32)
_F64P = C.POINTER(C.c_double)


class qg_network(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("n_gen", C.c_int32), ("n_zone", C.c_int32),
                ("ref_bus", C.c_int32), ("br_from", _I32P), ("br_to", _I32P), ("br_r", _F64P), ("br_x", _F64P),
                ("br_b", _F64P), ("s_max", _F64P), ("s_max_ctg", _F64P), ("gen_bus", _I32P), ("gen_zone", _I32P),
                ("cost_a", _F64P), ("cost_b", _F64P), ("cost_r", _F64P), ("pmin", _F64P), ("pmax", _F64P),
                ("qmin", _F64P), ("qmax", _F64P), ("ramp", _F64P), ("vmin", _F64P), ("vmax", _F64P),
                ("n_xf", C.c_int32), ("xf_branch", _I32P), ("tau_min", _F64P), ("tau_max", _F64P),
                ("phi_min", _F64P), ("phi_max", _F64P), ("dev_cons", _I32P), ("n_blk", C.c_int32),
                ("blk_price", _F64P), ("blk_width", _F64P), ("commit", C.c_int32), ("c_on", _F64P),
                ("c_su", _F64P), ("c_sd", _F64P), ("u_init", _F64P)]


class qg_horizon(C.Structure):
    _fields_ = [("T", C.c_int32), ("dt", _F64P), ("load_p", _F64P), ("load_q", _F64P), ("reserve_req", _F64P)]


class qg_contingencies(C.Structure):
    _fields_ = [("K", C.c_int32), ("branch", _I32P)]


class qg_options(C.Structure):
    _fields_ = [("c_p", C.c_double), ("c_q", C.c_double), ("c_s", C.c_double), ("c_rz", C.c_double),
                ("rho", C.c_double), ("eps", C.c_double), ("beta", C.c_double), ("adam_eps", C.c_double),
                ("precision", C.c_int32), ("lodf_dtype", C.c_int32), ("adam_paper_eps", C.c_int32),
                ("dc_solver", C.c_int32), ("ctg_frac", C.c_double), ("ctg_bound", C.c_int32)]


def _load():
    # QG_LIBRARY: another build of the same library (the index-checked one of build(check_bounds=True))
    path = os.environ.get("QG_LIBRARY") or LIB
    if not os.path.exists(path):
        raise ImportError(f"libqg.so is not built ({path}); run paper_2310_06650_gb300.build.build()")
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "qg_default_options": (None, [C.POINTER(qg_options)]),
        "qg_create": (C.c_int, [C.POINTER(vp), C.POINTER(qg_network), C.POINTER(qg_horizon),
                                C.POINTER(qg_contingencies), C.POINTER(qg_options)]),
        "qg_create_batch": (C.c_int, [C.POINTER(vp), C.c_int32, C.POINTER(qg_network), C.POINTER(qg_horizon),
                                      C.POINTER(qg_contingencies), C.POINTER(qg_options)]),
        "qg_destroy": (None, [vp]),
        "qg_num_vars": (C.c_int64, [vp]),
        "qg_autotune": (C.c_int, [vp, vp, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
        "qg_tile_shape": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int32)]),
        "qg_round_batch": (C.c_int, [vp, vp, C.c_double, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "qg_round_reset": (C.c_int, [vp]),
        "qg_layout": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "qg_set_stream": (C.c_int, [vp, vp]),
        "qg_eval_grad": (C.c_int, [vp, vp, vp, vp]),
        "qg_eval_grad_host": (C.c_int, [vp, vp, vp, vp]),
        "qg_eval_grad_noalloc": (C.c_int, [vp, vp, vp, vp]),
        "qg_adam_step": (C.c_int, [vp, vp, vp, vp, C.c_double, C.c_double, C.c_double]),
        "qg_solve": (C.c_int, [vp, vp, C.c_int32, C.c_double, C.c_double, C.c_double, vp]),
        "qg_breakdown": (C.c_int, [vp, _F64P]),
        "qg_get_step": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "qg_set_step": (C.c_int, [vp, C.c_int64]),
        "qg_state_size": (C.c_int64, [vp]),
        "qg_get_state": (C.c_int, [vp, vp, C.c_int64]),
        "qg_set_state": (C.c_int, [vp, vp, C.c_int64]),
        "qg_set_profiling": (C.c_int, [vp, C.c_int]),
        "qg_phase_times": (C.c_int, [vp, C.POINTER(C.c_float), C.c_int32]),
        "qg_last_error": (C.c_char_p, [vp]),
        "qg_version": (C.c_int, []),
        "qg_launches_per_eval": (C.c_int32, [vp]),
        "qg_ctg_select": (C.c_int, [vp, C.c_int32, vp, C.c_int32]),
        "qg_ctg_scores": (C.c_int, [vp, vp]),
        "qg_solve_schedule": (C.c_int, [vp, vp, C.c_int32, vp, C.c_int32, C.c_int32, C.c_double, C.c_double, vp]),
        "qg_schedule": (C.c_int, [vp, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double]),
        "qg_mlp_create": (C.c_int, [C.POINTER(vp), C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64]),
        "qg_mlp_destroy": (None, [vp]),
        "qg_mlp_num_params": (C.c_int64, [vp]),
        "qg_mlp_set_stream": (C.c_int, [vp, vp]),
        "qg_mlp_forward": (C.c_int, [vp, vp, C.c_int32, vp]),
        "qg_mlp_train_step": (C.c_int, [vp, vp, vp, C.c_int32, C.c_double, C.c_double, C.c_double, vp]),
        "qg_mlp_get_params": (C.c_int, [vp, vp]),
        "qg_mlp_set_params": (C.c_int, [vp, vp]),
        "qg_mlp_get_grads": (C.c_int, [vp, vp]),
        "qg_mlp_last_error": (C.c_char_p, [vp]),
        "qg_mlp_check": (C.c_int, [vp]),
        "qg_bounds_report": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]),
        "qg_dc_flows": (C.c_int, [vp, vp]),
        "qg_ctg_path": (C.c_int32, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("qg_default_options", "qg_create", "qg_create_batch", "qg_destroy", "qg_num_vars", "qg_layout",
            "qg_set_stream", "qg_eval_grad", "qg_eval_grad_host", "qg_eval_grad_noalloc", "qg_adam_step", "qg_solve", "qg_breakdown",
            "qg_get_step", "qg_set_step", "qg_state_size", "qg_get_state", "qg_set_state", "qg_set_profiling", "qg_phase_times", "qg_launches_per_eval",
            "qg_solve_schedule", "qg_schedule", "qg_ctg_select", "qg_ctg_scores", "qg_autotune", "qg_tile_shape", "qg_round_batch", "qg_round_reset",
            "qg_last_error", "qg_version",
            "qg_mlp_create", "qg_mlp_destroy", "qg_mlp_num_params", "qg_mlp_set_stream", "qg_mlp_forward",
            "qg_mlp_train_step", "qg_mlp_get_params", "qg_mlp_set_params", "qg_mlp_get_grads", "qg_mlp_last_error",
            "qg_mlp_check", "qg_bounds_report", "qg_dc_flows", "qg_ctg_path")
PHASES = ("s1", "s2", "s3", "s4", "s5", "adam")


class QGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libqg error {code}: {msg}")
        self.code = code


def _check(rc: int, h=None):
    if rc != QG_OK:
        raise QGError(rc, _lib.qg_last_error(h).decode(errors="replace"))


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def qg_default_options(**overrides) -> qg_options:
    o = qg_options()
    _lib.qg_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class _Keep:
    """Holds the numpy arrays behind one set of C structs until qg_create returns."""

    def __init__(self):
        self.arrays = []

    def i32(self, a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.arrays.append(a)
        return a.ctypes.data_as(_I32P)

    def f64(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.arrays.append(a)
        return a.ctypes.data_as(_F64P)


def _structs(case, keep: _Keep):
    """C structs for one case (any object with the synthetic case's attribute names)."""
    net = qg_network(
        n_bus=case.n_bus, n_branch=case.n_branch, n_gen=case.n_gen, n_zone=case.n_zone, ref_bus=case.ref_bus,
        br_from=keep.i32(case.br_from), br_to=keep.i32(case.br_to), br_r=keep.f64(case.br_r),
        br_x=keep.f64(case.br_x), br_b=keep.f64(case.br_b), s_max=keep.f64(case.s_max),
        s_max_ctg=keep.f64(case.s_max_ctg), gen_bus=keep.i32(case.gen_bus), gen_zone=keep.i32(case.gen_zone),
        cost_a=keep.f64(case.cost_a), cost_b=keep.f64(case.cost_b), cost_r=keep.f64(case.cost_r),
        pmin=keep.f64(case.pmin), pmax=keep.f64(case.pmax), qmin=keep.f64(case.qmin), qmax=keep.f64(case.qmax),
        ramp=keep.f64(case.ramp), vmin=keep.f64(case.vmin), vmax=keep.f64(case.vmax))
    X = int(getattr(case, "n_xf", 0))
    if X:
        net.n_xf = X
        net.xf_branch = keep.i32(case.xf_branch)
        net.tau_min, net.tau_max = keep.f64(case.tau_min), keep.f64(case.tau_max)
        net.phi_min, net.phi_max = keep.f64(case.phi_min), keep.f64(case.phi_max)
    cons = getattr(case, "dev_cons", None)
    if cons is not None and len(cons) and np.any(cons):
        net.dev_cons = keep.i32(np.asarray(cons, bool).astype(np.int32))
    W = getattr(case, "blk_width", None)
    if W is not None and W.size:
        net.n_blk = W.shape[1]
        net.blk_price, net.blk_width = keep.f64(case.blk_price), keep.f64(W)
    if getattr(case, "commit", False):
        net.commit = 1
        net.c_on, net.c_su = keep.f64(case.c_on), keep.f64(case.c_su)
        net.c_sd, net.u_init = keep.f64(case.c_sd), keep.f64(case.u_init)
    hor = qg_horizon(T=case.T, dt=keep.f64(case.dt), load_p=keep.f64(case.load_p), load_q=keep.f64(case.load_q),
                     reserve_req=keep.f64(case.reserve_req))
    ctg = qg_contingencies(K=case.K, branch=keep.i32(case.ctg) if case.K > 0 else None)
    return net, hor, ctg


def case_options(case, precision=QG_FP64, lodf_dtype=QG_LODF_F32, **kw) -> qg_options:
    """Options carrying the case's penalty prices; keyword arguments override any field."""
    base = dict(c_p=case.c_p, c_q=case.c_q, c_s=case.c_s, c_rz=case.c_rz, rho=case.rho, eps=case.eps,
                beta=case.beta, precision=precision, lodf_dtype=lodf_dtype)
    base.update(kw)
    return qg_default_options(**base)


def qg_create_batch(cases: Sequence, opt: qg_options) -> int:
    """Returns the opaque handle (an int) for the given cases."""
    keep = _Keep()
    nets, hors, ctgs = zip(*[_structs(c, keep) for c in cases])
    NA = qg_network * len(cases)
    HA = qg_horizon * len(cases)
    CA = qg_contingencies * len(cases)
    h = C.c_void_p()
    rc = _lib.qg_create_batch(C.byref(h), len(cases), NA(*nets), HA(*hors), CA(*ctgs), C.byref(opt))
    _check(rc, None)
    return h.value


def qg_create(case, opt: qg_options) -> int:
    return qg_create_batch([case], opt)


def qg_destroy(h: int) -> None:
    _lib.qg_destroy(h)


def qg_num_vars(h: int) -> int:
    return int(_lib.qg_num_vars(h))


def qg_layout(h: int, inst: int = 0):
    first, n_x = C.c_int64(), C.c_int64()
    off = (C.c_int64 * 8)()
    _check(_lib.qg_layout(h, inst, C.byref(first), C.byref(n_x), off), h)
    return first.value, n_x.value, tuple(off)


def qg_set_stream(h: int, stream_ptr: int) -> None:
    _check(_lib.qg_set_stream(h, stream_ptr), h)


def qg_eval_grad(h: int, x, obj, g=None) -> None:
    _check(_lib.qg_eval_grad(h, _ptr(x), _ptr(obj), _ptr(g)), h)


def qg_eval_grad_noalloc(h: int, x, obj, g) -> None:
    """qg_eval_grad with every work buffer in the library's static device scratch (no allocation)."""
    _check(_lib.qg_eval_grad_noalloc(h, _ptr(x), _ptr(obj), _ptr(g)), h)


def _host_addr(a: np.ndarray) -> int:
    """Address of a contiguous float64 host array (the cheapest route; this call sits in the
    end-to-end loop)."""
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise ValueError("host buffers must be contiguous float64 arrays")
    return a.__array_interface__["data"][0]


def qg_eval_grad_host(h: int, x: np.ndarray, obj: np.ndarray, g: Optional[np.ndarray] = None) -> None:
    _check(_lib.qg_eval_grad_host(h, _host_addr(x), _host_addr(obj), _host_addr(g) if g is not None else None), h)


def qg_adam_step(h: int, x, m, v, lr: float, beta1: float = 0.9, beta2: float = 0.999) -> None:
    _check(_lib.qg_adam_step(h, _ptr(x), _ptr(m), _ptr(v), lr, beta1, beta2), h)


def qg_solve(h: int, x, iters: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, obj_trace=None) -> None:
    _check(_lib.qg_solve(h, _ptr(x), iters, lr, beta1, beta2, _ptr(obj_trace)), h)


def qg_solve_schedule(h: int, x, iters: int, sched, restart: bool = True, beta1: float = 0.9,
                      beta2: float = 0.999, obj_trace=None) -> None:
    """sched: device tensor of L x 3 doubles (lr, eps, beta per iteration of the run)."""
    _check(_lib.qg_solve_schedule(h, _ptr(x), iters, _ptr(sched), int(sched.shape[0]), 1 if restart else 0,
                                  beta1, beta2, _ptr(obj_trace)), h)


def qg_schedule(iters: int, lr0: float, lrf: float, eps0: float, epsf: float, beta0: float = 0.1,
                beta1: float = 1.0, lag: float = 0.25) -> np.ndarray:
    """The Sec. II-F schedule table (host, iters x 3: lr, eps, beta) computed by the library."""
    out = np.zeros((iters, 3))
    rc = _lib.qg_schedule(out.ctypes.data_as(C.c_void_p), iters, lr0, lrf, eps0, epsf, beta0, beta1, lag)
    if rc != QG_OK:
        raise QGError(rc, "qg_schedule: invalid arguments")
    return out


def qg_ctg_select(h: int, inst: int, ids) -> None:
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    _check(_lib.qg_ctg_select(h, inst, ids.ctypes.data_as(C.c_void_p), int(ids.shape[0])), h)


def qg_ctg_scores(h: int, count: int) -> np.ndarray:
    """Scores of the last evaluation's (period, selected outage) pairs: `count` doubles."""
    out = np.zeros(count)
    _check(_lib.qg_ctg_scores(h, out.ctypes.data_as(C.c_void_p)), h)
    return out


def qg_breakdown(h: int, n_inst: int = 1) -> np.ndarray:
    out = np.zeros(8 * n_inst)
    _check(_lib.qg_breakdown(h, out.ctypes.data_as(_F64P)), h)
    return out.reshape(n_inst, 8)


def qg_get_step(h: int) -> int:
    s = C.c_int64()
    _check(_lib.qg_get_step(h, C.byref(s)), h)
    return s.value


def qg_set_step(h: int, step: int) -> None:
    _check(_lib.qg_set_step(h, step), h)


def qg_state_size(h: int) -> int:
    n = int(_lib.qg_state_size(h))
    if n < 0:
        _check(n, h)
    return n


def qg_get_state(h: int) -> bytes:
    """The handle's solver state (Adam moments, step counters, screening selections, rounding state)
    as an opaque blob."""
    buf = C.create_string_buffer(qg_state_size(h))
    _check(_lib.qg_get_state(h, buf, len(buf)), h)
    return buf.raw


def qg_set_state(h: int, blob: bytes) -> None:
    buf = C.create_string_buffer(bytes(blob), len(blob))
    _check(_lib.qg_set_state(h, buf, len(blob)), h)


def qg_set_profiling(h: int, on: bool) -> None:
    _check(_lib.qg_set_profiling(h, 1 if on else 0), h)


def qg_phase_times(h: int) -> dict:
    buf = (C.c_float * len(PHASES))()
    n = _lib.qg_phase_times(h, buf, len(PHASES))
    if n < 0:
        _check(n, h)
    return {PHASES[k]: float(buf[k]) for k in range(n)}


def qg_last_error(h: Optional[int] = None) -> str:
    return _lib.qg_last_error(h).decode(errors="replace")


def qg_version() -> int:
    return int(_lib.qg_version())


def qg_autotune(h: int, x, reps: int = 10, cold: bool = False):
    """Times every candidate contingency-block shape at x and keeps the fastest (cold: each timed
    evaluation starts from a flushed L2); returns instance 0's (periods per block, 64-branch tiles
    per block)."""
    shape = (C.c_int32 * 2)()
    _check(_lib.qg_autotune(h, _ptr(x), reps, 1 if cold else 0, shape), h)
    return tuple(shape)


def qg_tile_shape(h: int, inst: int = 0):
    shape = (C.c_int32 * 2)()
    _check(_lib.qg_tile_shape(h, inst, shape), h)
    return tuple(shape)


def qg_round_batch(h: int, x, frac: float):
    """One round of batch rounding (Alg. 1); returns (fixed pairs, all pairs)."""
    nf, nb = C.c_int64(), C.c_int64()
    _check(_lib.qg_round_batch(h, _ptr(x), frac, C.byref(nf), C.byref(nb)), h)
    return nf.value, nb.value


def qg_round_reset(h: int) -> None:
    _check(_lib.qg_round_reset(h), h)


def qg_launches_per_eval(h: int) -> int:
    n = int(_lib.qg_launches_per_eval(h))
    if n < 0:
        _check(n, h)
    return n


class Solver:
    """Convenience owner of one handle (and its torch device buffers)."""

    def __init__(self, cases, precision=QG_FP64, lodf_dtype=QG_LODF_F32, device="cuda", **opt_kw):
        import torch
        self.torch = torch
        self.cases = list(cases) if isinstance(cases, (list, tuple)) else [cases]
        self.precision = precision
        self.dtype = torch.float64 if precision == QG_FP64 else torch.float32
        self.device = torch.device(device)
        opt = case_options(self.cases[0], precision=precision, lodf_dtype=lodf_dtype, **opt_kw)
        self.ctg_frac = opt.ctg_frac
        self.h = qg_create_batch(self.cases, opt)
        self.n_x = qg_num_vars(self.h)
        self.n_inst = len(self.cases)
        self.obj = torch.zeros(self.n_inst, dtype=torch.float64, device=self.device)
        self.g = torch.zeros(self.n_x, dtype=self.dtype, device=self.device)
        qg_set_stream(self.h, torch.cuda.current_stream(self.device).cuda_stream)

    def eval_grad(self, x):
        qg_eval_grad(self.h, x, self.obj, self.g)
        return self.obj, self.g

    def breakdown(self):
        return qg_breakdown(self.h, self.n_inst)

    def close(self):
        if self.h:
            qg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------------------
# learned warm start (MLP)
# ------------------------------------------------------------------------------------------------

def _mcheck(rc: int, m=None):
    if rc != QG_OK:
        raise QGError(rc, _lib.qg_mlp_last_error(m).decode(errors="replace"))


def qg_mlp_create(n_in: int, n_hidden: int, n_out: int, max_batch: int, seed: int = 0) -> int:
    m = C.c_void_p()
    _mcheck(_lib.qg_mlp_create(C.byref(m), n_in, n_hidden, n_out, max_batch, seed), None)
    return m.value


def qg_mlp_destroy(m: int) -> None:
    _lib.qg_mlp_destroy(m)


def qg_mlp_num_params(m: int) -> int:
    return int(_lib.qg_mlp_num_params(m))


def qg_mlp_set_stream(m: int, stream_ptr: int) -> None:
    _mcheck(_lib.qg_mlp_set_stream(m, stream_ptr), m)


def qg_mlp_forward(m: int, x, batch: int, y) -> None:
    _mcheck(_lib.qg_mlp_forward(m, _ptr(x), batch, _ptr(y)), m)


def qg_mlp_train_step(m: int, x, target, batch: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                      loss=None) -> None:
    _mcheck(_lib.qg_mlp_train_step(m, _ptr(x), _ptr(target), batch, lr, beta1, beta2, _ptr(loss)), m)


def qg_mlp_get_params(m: int, w) -> None:
    _mcheck(_lib.qg_mlp_get_params(m, _ptr(w)), m)


def qg_mlp_set_params(m: int, w) -> None:
    _mcheck(_lib.qg_mlp_set_params(m, _ptr(w)), m)


def qg_mlp_get_grads(m: int, g) -> None:
    _mcheck(_lib.qg_mlp_get_grads(m, _ptr(g)), m)


def qg_mlp_last_error(m: Optional[int] = None) -> str:
    return _lib.qg_mlp_last_error(m).decode(errors="replace")


def qg_dc_flows(h: int, n: int) -> np.ndarray:
    """The last evaluation's base DC flows as the contingency screen reads them (n = sum of T M)."""
    out = np.zeros(n, dtype=np.float32)
    _check(_lib.qg_dc_flows(h, out.ctypes.data_as(C.c_void_p)), h)
    return out


def qg_ctg_path(h: int) -> int:
    """The contingency stage's path: 0 no bound test, 1 eager bound test, 2 on-demand path."""
    r = _lib.qg_ctg_path(h)
    _check(min(r, 0), h)
    return r


def qg_bounds_report():
    """Index-checked builds: None if no checked access missed, else (source line, address) of the first;
    raises QGError (QG_ERR_UNSUPPORTED) on the normal build."""
    line, addr = C.c_int64(0), C.c_uint64(0)
    rc = _lib.qg_bounds_report(C.byref(line), C.byref(addr))
    if rc < 0:
        raise QGError(rc, "qg_bounds_report: not an index-checked build")
    return (line.value, addr.value) if rc == 1 else None


def qg_mlp_check(m: int) -> None:
    """Synchronizes; raises QGError if a tensor-core GEMM of this network gave up on a pipeline wait."""
    _mcheck(_lib.qg_mlp_check(m), m)
