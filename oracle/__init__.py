"""FP64 CPU oracle for the APO population update (ctypes binding).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU product path never imports it.

The C source (``apo_oracle.c``) restates the paper's method step by step; this
module only builds it with gcc and marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

(OBJ_SPHERE, OBJ_ELLIPTIC, OBJ_ROSENBROCK, OBJ_RASTRIGIN, OBJ_HYBRID, OBJ_COMPOSITION, OBJ_OTSU,
 OBJ_BENTCIGAR, OBJ_HGBAT, OBJ_GRIEWANK) = range(10)
MODE_DORMANCY, MODE_REPRODUCTION, MODE_AUTOTROPHIC, MODE_HETEROTROPHIC = range(4)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, no fast-math, no FP contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("D", C.c_int), ("kind", C.c_int),
        ("lb", C.POINTER(C.c_double)), ("ub", C.POINTER(C.c_double)),
        ("shift", C.POINTER(C.c_float)), ("rot", C.POINTER(C.c_float)),
        ("perm", C.POINTER(C.c_int32)), ("n_comp", C.c_int),
        ("comp_sigma", C.POINTER(C.c_double)), ("comp_bias", C.POINTER(C.c_double)),
        ("hist", C.POINTER(C.c_int64)),
    ]


class Params(C.Structure):
    _fields_ = [("ps", C.c_int), ("np", C.c_int), ("pf_max", C.c_double),
                ("max_iter", C.c_int), ("seed", C.c_uint32), ("run", C.c_uint32),
                ("pdr_form", C.c_int), ("pair_policy", C.c_int), ("max_fes", C.c_longlong)]


class StepInfo(C.Structure):
    _fields_ = [("order", C.POINTER(C.c_int32)), ("m", C.POINTER(C.c_int32)),
                ("in_dr", C.POINTER(C.c_int32)), ("mode", C.POINTER(C.c_int32)),
                ("mask_count", C.POINTER(C.c_int32)), ("mask", C.POINTER(C.c_uint8)),
                ("xnew_raw", C.POINTER(C.c_double)), ("xnew", C.POINTER(C.c_double)),
                ("fnew", C.POINTER(C.c_double)), ("accepted", C.POINTER(C.c_int32))]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_objective.argtypes = [P(Problem), P(C.c_double)]
        L.orc_objective.restype = C.c_double
        L.orc_objective_batch.argtypes = [P(Problem), C.c_int, P(C.c_double), P(C.c_double)]
        L.orc_init_population.argtypes = [P(Problem), P(Params), P(C.c_double), P(C.c_double)]
        L.orc_apo_step.argtypes = [P(Problem), P(Params), C.c_int, P(C.c_double),
                                   P(C.c_double), P(StepInfo)]
        L.orc_apo_step.restype = C.c_int
        L.orc_candidates.argtypes = [P(Problem), P(Params), C.c_int, C.c_int, P(C.c_double), P(C.c_double),
                                     P(C.c_double), P(C.c_int32)]
        L.orc_candidates.restype = C.c_int
        L.orc_apo_run.argtypes = [P(Problem), P(Params), P(C.c_double), P(C.c_double),
                                  P(C.c_double)]
        L.orc_apo_run.restype = C.c_int
        L.orc_iterations.argtypes = [P(Params)]
        L.orc_iterations.restype = C.c_int
        L.orc_apo_run_many.argtypes = [P(P(Problem)), P(Params), C.c_int, C.c_int, C.c_int,
                                       P(C.c_double), P(C.c_double)]
        L.orc_clamp_eval_select.argtypes = [P(Problem), C.c_int, P(C.c_double), P(C.c_double),
                                            P(C.c_double), P(C.c_double)]
        L.orc_histogram_u8.argtypes = [P(C.c_uint8), C.c_int64, P(C.c_int64)]
        L.orc_otsu_sigma_b2.argtypes = [P(C.c_int64), P(C.c_int), C.c_int]
        L.orc_otsu_sigma_b2.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


class OracleProblem:
    """Holds numpy buffers alive and exposes the C problem struct.

    kind: OBJ_*; lb, ub: [D] bounds; shift [D] / rot [D, D] float32 (composition:
    [n_comp, D] / [n_comp, D, D]); perm int32 [D] (composition [n_comp, D]);
    comp_sigma, comp_bias float64 [n_comp]; hist int64 [256] for Otsu.
    """

    def __init__(self, kind, D, lb, ub, shift=None, rot=None, perm=None,
                 comp_sigma=None, comp_bias=None, hist=None):
        self.kind, self.D = int(kind), int(D)
        self.lb = np.ascontiguousarray(np.broadcast_to(np.asarray(lb, np.float64), (D,)))
        self.ub = np.ascontiguousarray(np.broadcast_to(np.asarray(ub, np.float64), (D,)))
        f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
        self.shift, self.rot = f32(shift), f32(rot)
        self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        self.comp_sigma = None if comp_sigma is None else np.ascontiguousarray(comp_sigma, np.float64)
        self.comp_bias = None if comp_bias is None else np.ascontiguousarray(comp_bias, np.float64)
        self.hist = None if hist is None else np.ascontiguousarray(hist, dtype=np.int64)
        n_comp = 0 if self.comp_sigma is None else len(self.comp_sigma)
        self.c = Problem(self.D, self.kind, _ptr(self.lb, C.c_double), _ptr(self.ub, C.c_double),
                         _ptr(self.shift, C.c_float), _ptr(self.rot, C.c_float),
                         _ptr(self.perm, C.c_int32), n_comp,
                         _ptr(self.comp_sigma, C.c_double), _ptr(self.comp_bias, C.c_double),
                         _ptr(self.hist, C.c_int64))

    @classmethod
    def from_spec(cls, spec):
        """Build from a ProblemSpec of the seeded input generators."""
        return cls(spec.kind, spec.D, spec.lb, spec.ub, spec.shift, spec.rot, spec.perm,
                   spec.comp_sigma, spec.comp_bias,
                   None if spec.hist is None else np.asarray(spec.hist, np.int64))


def params(ps, np_=1, pf_max=0.1, max_iter=1000, seed=0, run=0, pdr_form=0, pair_policy=0, max_fes=0):
    return Params(int(ps), int(np_), float(pf_max), int(max_iter), int(seed) & 0xFFFFFFFF,
                  int(run) & 0xFFFFFFFF, int(pdr_form), int(pair_policy), int(max_fes))


def iterations(prm: Params) -> int:
    """Iterations a run takes (max_iter, or what the evaluation budget allows)."""
    return int(lib().orc_iterations(C.byref(prm)))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def objective(prob: OracleProblem, X):
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
    F = np.empty(X.shape[0], np.float64)
    lib().orc_objective_batch(C.byref(prob.c), X.shape[0], _ptr(X, C.c_double), _ptr(F, C.c_double))
    return F


def init_population(prob: OracleProblem, prm: Params):
    X = np.empty((prm.ps, prob.D), np.float64)
    F = np.empty(prm.ps, np.float64)
    lib().orc_init_population(C.byref(prob.c), C.byref(prm), _ptr(X, C.c_double), _ptr(F, C.c_double))
    return X, F


def apo_step(prob: OracleProblem, prm: Params, t, X, F, with_info=False):
    """One iteration; returns (X, F) in this iteration's rank order [+ info dict]."""
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    F = np.array(F, dtype=np.float64, copy=True)
    ps, D = prm.ps, prob.D
    info = None
    arrs = {}
    if with_info:
        arrs = dict(order=np.empty(ps, np.int32), m=np.empty(1, np.int32),
                    in_dr=np.empty(ps, np.int32), mode=np.empty(ps, np.int32),
                    mask_count=np.empty(ps, np.int32), mask=np.empty((ps, D), np.uint8),
                    xnew_raw=np.empty((ps, D)), xnew=np.empty((ps, D)), fnew=np.empty(ps),
                    accepted=np.empty(ps, np.int32))
        info = StepInfo(_ptr(arrs["order"], C.c_int32), _ptr(arrs["m"], C.c_int32),
                        _ptr(arrs["in_dr"], C.c_int32), _ptr(arrs["mode"], C.c_int32),
                        _ptr(arrs["mask_count"], C.c_int32), _ptr(arrs["mask"], C.c_uint8),
                        _ptr(arrs["xnew_raw"], C.c_double), _ptr(arrs["xnew"], C.c_double),
                        _ptr(arrs["fnew"], C.c_double), _ptr(arrs["accepted"], C.c_int32))
    rc = lib().orc_apo_step(C.byref(prob.c), C.byref(prm), int(t), _ptr(X, C.c_double),
                            _ptr(F, C.c_double), C.byref(info) if info is not None else None)
    if rc != 0:
        raise ValueError("orc_apo_step rejected its arguments")
    if with_info:
        arrs["m"] = int(arrs["m"][0])
        return X, F, arrs
    return X, F


def candidates(prob: OracleProblem, prm: Params, t, k, X, F):
    """Surrogate-assisted form: the k candidates of every protozoon at iteration
    t (candidate c draws from the plain slots | (c << 8)).  Returns
    (Xc[ps, k, D] in this iteration's rank order, order[ps])."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    ps, D = prm.ps, prob.D
    Xc = np.empty((ps, int(k), D), np.float64)
    order = np.empty(ps, np.int32)
    rc = lib().orc_candidates(C.byref(prob.c), C.byref(prm), int(t), int(k), _ptr(X, C.c_double),
                              _ptr(F, C.c_double), _ptr(Xc, C.c_double), _ptr(order, C.c_int32))
    if rc != 0:
        raise ValueError("orc_candidates rejected its arguments")
    return Xc, order


def apo_run(prob: OracleProblem, prm: Params, want_curve=True):
    best_x = np.empty(prob.D, np.float64)
    best_f = C.c_double()
    T = iterations(prm)
    if T < 1:
        raise ValueError("the evaluation budget allows no iteration")
    curve = np.empty(T + 1, np.float64) if want_curve else None
    rc = lib().orc_apo_run(C.byref(prob.c), C.byref(prm), _ptr(best_x, C.c_double), C.byref(best_f),
                           _ptr(curve, C.c_double))
    if rc != 0:
        raise ValueError("orc_apo_run rejected its arguments")
    return best_x, best_f.value, curve


def apo_run_many(probs, prms, n_threads):
    n = len(probs)
    dmax = max(p.D for p in probs)
    arr = (C.POINTER(Problem) * n)(*[C.pointer(p.c) for p in probs])
    prm_arr = (Params * n)(*prms)
    best_x = np.zeros((n, dmax))
    best_f = np.empty(n)
    lib().orc_apo_run_many(arr, prm_arr, n, dmax, int(n_threads), _ptr(best_x, C.c_double),
                           _ptr(best_f, C.c_double))
    return best_x, best_f


def clamp_eval_select(prob: OracleProblem, X, F, Xnew):
    X = np.array(X, dtype=np.float64, copy=True)
    F = np.array(F, dtype=np.float64, copy=True)
    Xnew = np.array(Xnew, dtype=np.float64, copy=True)
    Fnew = np.empty(X.shape[0])
    lib().orc_clamp_eval_select(C.byref(prob.c), X.shape[0], _ptr(X, C.c_double), _ptr(F, C.c_double),
                                _ptr(Xnew, C.c_double), _ptr(Fnew, C.c_double))
    return X, F, Xnew, Fnew


def histogram_u8(px):
    px = np.ascontiguousarray(px, dtype=np.uint8).reshape(-1)
    h = np.empty(256, np.int64)
    lib().orc_histogram_u8(_ptr(px, C.c_uint8), px.size, _ptr(h, C.c_int64))
    return h


def otsu_sigma_b2(hist, thresholds_sorted):
    h = np.ascontiguousarray(hist, dtype=np.int64)
    t = np.ascontiguousarray(thresholds_sorted, dtype=np.int32)
    return lib().orc_otsu_sigma_b2(_ptr(h, C.c_int64), t.ctypes.data_as(C.POINTER(C.c_int)), t.size)
