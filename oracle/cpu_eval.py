"""ctypes wrapper of oracle/cpu_eval.cpp: the FP64 C++/OpenMP CPU evaluation of the objective and
its gradient (Sec. II: the AC terms, Example 1-4 penalties, Eq. nlp_updated, the contingency term of
Sec. II-E with the rank-1 correction of Eq. rank_correct and the adjoint of Eq. 2nd_lin_sys).

TEST INFRASTRUCTURE ONLY (see qg_oracle.py): the tests pin it to the numpy oracle; the benchmark
times it as the CPU baseline.  It covers plain producers without transformers; other cases raise.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_eval.cpp")
LIB = os.path.join(HERE, "_build", "libqgo.so")


def build(force: bool = False) -> str:
    """Compiles the shared library with g++ (C++17, -O2, OpenMP) next to this file."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


class _Case(C.Structure):
    _fields_ = [("n", C.c_int32), ("M", C.c_int32), ("G", C.c_int32), ("Z", C.c_int32), ("T", C.c_int32),
                ("K", C.c_int32), ("ref", C.c_int32),
                ("br_from", C.c_void_p), ("br_to", C.c_void_p), ("br_r", C.c_void_p), ("br_x", C.c_void_p),
                ("br_b", C.c_void_p), ("s_max", C.c_void_p), ("s_max_ctg", C.c_void_p),
                ("gen_bus", C.c_void_p), ("gen_zone", C.c_void_p), ("cost_a", C.c_void_p), ("cost_b", C.c_void_p),
                ("cost_r", C.c_void_p), ("pmax", C.c_void_p), ("ramp", C.c_void_p), ("dt", C.c_void_p),
                ("load_p", C.c_void_p), ("load_q", C.c_void_p), ("reserve_req", C.c_void_p), ("ctg", C.c_void_p),
                ("c_p", C.c_double), ("c_q", C.c_double), ("c_s", C.c_double), ("c_rz", C.c_double),
                ("rho", C.c_double), ("eps", C.c_double), ("beta", C.c_double)]


_libs = {}


def _load(path=None):
    """The library at `path` (default: the one built from cpu_eval.cpp), loaded once."""
    path = path or build()
    if path not in _libs:
        lib = C.CDLL(path)
        lib.qgo_prepare.restype = C.c_void_p
        lib.qgo_prepare.argtypes = [C.POINTER(_Case)]
        lib.qgo_free.argtypes = [C.c_void_p]
        lib.qgo_eval.restype = C.c_double
        lib.qgo_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        lib.qgo_max_threads.restype = C.c_int32
        _libs[path] = lib
    return _libs[path]


def in_scope(case) -> bool:
    """Plain producers: no bid blocks, consumers, on-status or transformers."""
    W = getattr(case, "blk_width", None)
    blocks = W is not None and np.size(W) > 0 and bool(np.any(np.asarray(W) > 0))
    cons = getattr(case, "dev_cons", None)
    consumers = cons is not None and bool(np.any(cons))
    return not (blocks or consumers or getattr(case, "commit", False) or int(getattr(case, "n_xf", 0)))


class CpuOracle:
    """The case's set-up (reduced-Laplacian inverse, outage columns) once; evaluations after."""

    def __init__(self, case, lib_path=None):
        if not in_scope(case):
            raise ValueError("cpu_eval covers plain producers without transformers; use oracle.evaluate")
        lib = self._lib = _load(lib_path)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)  # noqa: E731
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        self._keep = [i32(case.br_from), i32(case.br_to), f64(case.br_r), f64(case.br_x), f64(case.br_b),
                      f64(case.s_max), f64(case.s_max_ctg), i32(case.gen_bus), i32(case.gen_zone), f64(case.cost_a),
                      f64(case.cost_b), f64(case.cost_r), f64(case.pmax), f64(case.ramp), f64(case.dt),
                      f64(case.load_p), f64(case.load_q), f64(case.reserve_req), i32(case.ctg)]
        ptr = [a.ctypes.data for a in self._keep]
        c = _Case(case.n_bus, case.n_branch, case.n_gen, case.n_zone, case.T, case.K, case.ref_bus, *ptr,
                  case.c_p, case.c_q, case.c_s, case.c_rz, case.rho, case.eps, case.beta)
        self.h = lib.qgo_prepare(C.byref(c))
        if not self.h:
            raise ValueError("cpu_eval: the reduced Laplacian is not positive definite")
        self.case = case
        self.n_x = case.T * (2 * case.n_bus + 3 * case.n_gen)

    def evaluate(self, x, want_grad: bool = True, threads: int = 0):
        """(Phi, gradient or None, terms[8]) at x ([v | theta | p | q | r], period-major)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.n_x,)
        g = np.empty(self.n_x) if want_grad else None
        terms = np.empty(8)
        obj = self._lib.qgo_eval(self.h, x.ctypes.data, g.ctypes.data if want_grad else None, terms.ctypes.data,
                                 threads)
        return obj, g, terms

    def close(self):
        if getattr(self, "h", None):
            self._lib.qgo_free(self.h)
            self.h = None

    def __del__(self):
        self.close()


def max_threads() -> int:
    return int(_load().qgo_max_threads())
