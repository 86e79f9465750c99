"""Compiled oracle step (oracle/cstep.c) behind the interface of oracle/leapfrog.run.

Test infrastructure only: used to time the CPU baseline on one and on all host cores.  The
arithmetic is that of leapfrog.step (eqs. 3-6, 14-15) in C; tests/test_oracle_cstep.py pins it
to the numpy oracle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .leapfrog import Plasma, Source, State
from .operators import Operators

_lib = None


def lib():
    global _lib
    if _lib is None:
        from . import build_c
        _lib = C.CDLL(build_c.build())
        P = C.c_void_p
        _lib.ue_oracle_steps.restype = C.c_int
        _lib.ue_oracle_steps.argtypes = [C.c_int64, C.c_int64, P, P, P, P, P, P, P, P, P, P, C.c_double,
                                         C.c_int64, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_int64, C.c_int64, C.c_int]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Stepper:
    """Holds the CSR arrays of one operator set (int64 indices, float64 values)."""

    def __init__(self, ops: Operators):
        self.ops = ops
        lb, le = ops.L_B.tocsr(), ops.L_E.tocsr()
        lb.sort_indices()
        le.sort_indices()
        self.lb = [np.ascontiguousarray(lb.indptr, np.int64), np.ascontiguousarray(lb.indices, np.int64),
                   np.ascontiguousarray(lb.data, np.float64)]
        self.le = [np.ascontiguousarray(le.indptr, np.int64), np.ascontiguousarray(le.indices, np.int64),
                   np.ascontiguousarray(le.data, np.float64)]

    def run(self, st: State, dt: float, n_steps: int, plasma: Plasma | None = None,
            source: Source | None = None, threads: int = 1):
        """(state after n_steps, threads used); the input state is not modified."""
        E, B, j = st.E.copy(), st.B.copy(), st.j.copy()
        nbar = np.ascontiguousarray(plasma.nbar(self.ops)) if plasma is not None else None
        nu = plasma.nu if plasma is not None else 0.0
        if source is not None:
            cols = np.ascontiguousarray(self.ops.col_of_edge[source.edge_ids], np.int64)
            amp = np.ascontiguousarray(source.amp, np.float64)
            w0, t0, tau = source.omega0, source.t0, source.tau
        else:
            cols = amp = None
            w0 = t0 = tau = 0.0
        used = lib().ue_oracle_steps(self.ops.n_ei, self.ops.n_t, *(_p(a) for a in self.lb),
                                     *(_p(a) for a in self.le), _p(E), _p(B), _p(j), _p(nbar), nu,
                                     0 if cols is None else cols.size, _p(cols), _p(amp), w0, t0,
                                     tau if tau else 1.0, dt, st.n, n_steps, int(threads))
        return State(E, B, j, st.n + n_steps), used


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1
