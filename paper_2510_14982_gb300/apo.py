"""Thin ctypes binding of libapo.so (declared in include/apo.h).

Every function keeps the C name and only marshals arguments: torch tensors
are passed as raw device pointers, streams as ``cudaStream_t`` handles.  All
of the optimiser's work runs in the library's CUDA kernels.  Importing this
module loads libapo.so and raises ImportError when it is missing; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapo.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libapo.so is not built (run paper_2510_14982_gb300/build.py or "
                      "__graft_entry__.build()); the APO path has no CPU fallback")
_lib = C.CDLL(LIB_PATH)

APO_OK, APO_ERR_INVALID_ARG, APO_ERR_CUDA, APO_ERR_OOM, APO_ERR_TIMEOUT, APO_ERR_UNSUPPORTED, APO_ERR_INTERNAL = range(7)
(APO_OBJ_SPHERE, APO_OBJ_ELLIPTIC, APO_OBJ_ROSENBROCK, APO_OBJ_RASTRIGIN, APO_OBJ_HYBRID,
 APO_OBJ_COMPOSITION, APO_OBJ_OTSU, APO_OBJ_BENTCIGAR, APO_OBJ_HGBAT, APO_OBJ_GRIEWANK) = range(10)

# every entry point declared in include/apo.h
EXPORTS = ("apo_problem_create", "apo_problem_destroy", "apo_problem_dim", "apo_run", "apo_run_device",
           "apo_run_device_noalloc",
           "apo_run_batch", "apo_batch_create", "apo_batch_launch", "apo_batch_autotune", "apo_batch_destroy",
           "apo_step", "apo_evaluate", "apo_clamp_eval_select", "apo_histogram_u8",
           "apo_effective_iterations", "apo_init_state", "apo_run_from_state",
           "apo_mlp_create", "apo_mlp_destroy", "apo_mlp_set_params", "apo_mlp_get_params", "apo_mlp_forward",
           "apo_mlp_gradients", "apo_mlp_train",
           "apo_run_surrogate", "apo_surrogate_candidates", "apo_barrier_selftest",
           "apo_philox4x32_10", "apo_set_timing_events", "apo_status_string", "apo_last_error",
           "apo_measure_peaks", "apo_large_stage_timing")


class apo_objective_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("shift", C.POINTER(C.c_float)), ("rotation", C.POINTER(C.c_float)),
                ("perm", C.POINTER(C.c_int32)), ("n_comp", C.c_int),
                ("comp_sigma", C.POINTER(C.c_double)), ("comp_bias", C.POINTER(C.c_double)),
                ("hist", C.POINTER(C.c_int32)), ("hist_on_device", C.c_int)]


class apo_params(C.Structure):
    _fields_ = [("ps", C.c_int), ("np", C.c_int), ("pf_max", C.c_double), ("max_iter", C.c_int),
                ("seed", C.c_uint32), ("run", C.c_uint32), ("pdr_form", C.c_int), ("pair_policy", C.c_int),
                ("max_fes", C.c_longlong)]


class apo_batch_options(C.Structure):
    _fields_ = [("smem_budget", C.c_size_t), ("ctas_per_sm", C.c_int), ("cluster_ps", C.c_int),
                ("cluster_size", C.c_int)]


class apo_surrogate_params(C.Structure):
    _fields_ = [("k", C.c_int), ("retrain_every", C.c_int), ("archive_cap", C.c_int), ("train_steps", C.c_int),
                ("batch", C.c_int), ("lr", C.c_float), ("min_rank_corr", C.c_float), ("net_seed", C.c_uint32),
                ("train_window", C.c_int)]


class apo_surrogate_stats(C.Structure):
    _fields_ = [("true_evals", C.c_longlong), ("screened", C.c_longlong), ("retrains", C.c_int),
                ("screening_iters", C.c_int), ("fallback_iters", C.c_int), ("last_rank_corr", C.c_double),
                ("train_ms", C.c_double), ("total_ms", C.c_double)]


_P = C.c_void_p
_lib.apo_problem_create.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(apo_objective_desc), C.POINTER(_P)]
_lib.apo_problem_create.restype = C.c_int
_lib.apo_problem_destroy.argtypes = [_P]
_lib.apo_problem_destroy.restype = None
_lib.apo_problem_dim.argtypes = [_P]
_lib.apo_problem_dim.restype = C.c_int
_lib.apo_run.argtypes = [_P, C.POINTER(apo_params), _P, C.POINTER(C.c_float), C.POINTER(C.c_double),
                         C.POINTER(C.c_float)]
_lib.apo_run_device.argtypes = [_P, C.POINTER(apo_params), _P, _P, _P, _P]
_lib.apo_run_device_noalloc.argtypes = [_P, C.POINTER(apo_params), _P, _P, _P, _P]
_lib.apo_run_batch.argtypes = [C.POINTER(_P), C.POINTER(apo_params), C.c_int, _P, _P, C.c_int, _P, _P, C.c_int]
_lib.apo_batch_create.argtypes = [C.POINTER(_P), C.POINTER(apo_params), C.c_int, _P, C.c_int, _P, _P, C.c_int,
                                  C.POINTER(apo_batch_options), C.POINTER(_P)]
_lib.apo_batch_launch.argtypes = [_P, _P]
_lib.apo_batch_autotune.argtypes = [_P, _P, C.c_int, C.POINTER(apo_batch_options)]
_lib.apo_batch_destroy.argtypes = [_P]
_lib.apo_batch_destroy.restype = None
_lib.apo_step.argtypes = [_P, C.POINTER(apo_params), C.c_int, _P, _P, _P]
_lib.apo_effective_iterations.argtypes = [C.POINTER(apo_params)]
_lib.apo_effective_iterations.restype = C.c_int
_lib.apo_init_state.argtypes = [_P, C.POINTER(apo_params), _P, _P, _P]
_lib.apo_init_state.restype = C.c_int
_lib.apo_run_from_state.argtypes = [_P, C.POINTER(apo_params), C.c_int, C.c_int, _P, _P, _P, _P, _P, _P]
_lib.apo_run_from_state.restype = C.c_int
_lib.apo_evaluate.argtypes = [_P, _P, _P, C.c_int, _P]
_lib.apo_clamp_eval_select.argtypes = [_P, _P, C.c_int, _P, _P, _P, _P]
_lib.apo_histogram_u8.argtypes = [_P, C.c_int64, C.c_int, _P, _P]
_lib.apo_philox4x32_10.argtypes = [_P, C.c_uint32, C.c_uint32, C.c_int, _P, _P]
_FP = C.POINTER(C.c_float)
_lib.apo_mlp_create.argtypes = [C.c_int, C.c_uint32, C.POINTER(_P)]
_lib.apo_mlp_destroy.argtypes = [_P]
_lib.apo_mlp_destroy.restype = None
_lib.apo_mlp_set_params.argtypes = [_P, _FP, _FP, _FP, _FP, _FP, C.c_float]
_lib.apo_mlp_get_params.argtypes = [_P, _FP, _FP, _FP, _FP, _FP, _FP]
_lib.apo_mlp_forward.argtypes = [_P, _P, C.c_int, _P, _P]
_lib.apo_mlp_gradients.argtypes = [_P, _P, _P, C.c_int, _FP, _FP, _FP, _FP, _FP, _FP, _FP]
_lib.apo_mlp_train.argtypes = [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_float, C.c_uint32, _P]
for _f in ("apo_mlp_create", "apo_mlp_set_params", "apo_mlp_get_params", "apo_mlp_forward", "apo_mlp_gradients",
           "apo_mlp_train"):
    getattr(_lib, _f).restype = C.c_int
_lib.apo_surrogate_candidates.argtypes = [_P, C.POINTER(apo_params), C.c_int, C.c_int, _P, _P, _P, _P]
_lib.apo_surrogate_candidates.restype = C.c_int
_lib.apo_barrier_selftest.argtypes = [C.c_int, C.c_int, C.c_int, _P]
_lib.apo_barrier_selftest.restype = C.c_int
_lib.apo_run_surrogate.argtypes = [_P, C.POINTER(apo_params), C.POINTER(apo_surrogate_params), _P, _FP,
                                   C.POINTER(C.c_double), _FP, C.POINTER(apo_surrogate_stats)]
_lib.apo_run_surrogate.restype = C.c_int
_lib.apo_set_timing_events.argtypes = [_P, _P]
_lib.apo_set_timing_events.restype = C.c_int
for _f in ("apo_batch_create", "apo_batch_launch", "apo_batch_autotune",
           "apo_run", "apo_run_device", "apo_run_device_noalloc", "apo_run_batch", "apo_step", "apo_evaluate", "apo_clamp_eval_select",
           "apo_histogram_u8", "apo_philox4x32_10"):
    getattr(_lib, _f).restype = C.c_int
_lib.apo_measure_peaks.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.apo_measure_peaks.restype = C.c_int
_lib.apo_large_stage_timing.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
_lib.apo_large_stage_timing.restype = C.c_int
_lib.apo_status_string.argtypes = [C.c_int]
_lib.apo_status_string.restype = C.c_char_p
_lib.apo_last_error.argtypes = []
_lib.apo_last_error.restype = C.c_char_p


class ApoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = "%s: %s (%s)" % (where, _lib.apo_status_string(status).decode(), _lib.apo_last_error().decode())
        super().__init__(msg)


def _check(rc: int, where: str):
    if rc != APO_OK:
        raise ApoError(rc, where)


def _dptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _np_ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def apo_status_string(status: int) -> str:
    return _lib.apo_status_string(status).decode()


def apo_last_error() -> str:
    return _lib.apo_last_error().decode()


def apo_params_make(ps, np_=1, pf_max=0.1, max_iter=1000, seed=0, run=0, pdr_form=0, pair_policy=0,
                    max_fes=0) -> apo_params:
    return apo_params(int(ps), int(np_), float(pf_max), int(max_iter), int(seed) & 0xFFFFFFFF,
                      int(run) & 0xFFFFFFFF, int(pdr_form), int(pair_policy), int(max_fes))


def apo_effective_iterations(params: apo_params) -> int:
    """Iterations a run with these params takes (max_iter, or what max_fes allows); -1 if invalid."""
    return int(_lib.apo_effective_iterations(C.byref(params)))


class Problem:
    """Owns an apo_problem handle (apo_problem_create / apo_problem_destroy)."""

    def __init__(self, handle, D, kind):
        self.handle, self.D, self.kind = handle, D, kind

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.apo_problem_destroy(h)
            self.handle = None

    @property
    def fit_dtype(self):
        import torch
        return torch.float64 if self.kind == APO_OBJ_OTSU else torch.float32


def apo_problem_create(D, lb, ub, kind, shift=None, rotation=None, perm=None, comp_sigma=None,
                       comp_bias=None, hist=None, hist_device=None) -> Problem:
    """apo_problem_create; array arguments are numpy arrays (hist_device: a torch int32 tensor)."""
    lb = np.ascontiguousarray(np.broadcast_to(np.asarray(lb, np.float64), (D,)))
    ub = np.ascontiguousarray(np.broadcast_to(np.asarray(ub, np.float64), (D,)))
    keep = []

    def f32(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(a)
        return _np_ptr(a, C.c_float)

    def arr(a, dt, ct):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return _np_ptr(a, ct)

    n_comp = 0 if comp_sigma is None else len(comp_sigma)
    desc = apo_objective_desc(int(kind), f32(shift), f32(rotation), arr(perm, np.int32, C.c_int32), n_comp,
                              arr(comp_sigma, np.float64, C.c_double), arr(comp_bias, np.float64, C.c_double),
                              None, 0)
    if hist_device is not None:
        desc.hist = C.cast(C.c_void_p(hist_device.data_ptr()), C.POINTER(C.c_int32))
        desc.hist_on_device = 1
    elif hist is not None:
        desc.hist = arr(hist, np.int32, C.c_int32)
    h = _P()
    _check(_lib.apo_problem_create(int(D), _np_ptr(lb, C.c_double), _np_ptr(ub, C.c_double), C.byref(desc),
                                   C.byref(h)), "apo_problem_create")
    return Problem(h, int(D), int(kind))


def problem_from_spec(spec) -> Problem:
    """apo_problem_create from a ProblemSpec of the seeded input generators."""
    return apo_problem_create(spec.D, spec.lb, spec.ub, spec.kind, spec.shift, spec.rot, spec.perm,
                              spec.comp_sigma, spec.comp_bias,
                              None if spec.hist is None else np.asarray(spec.hist, np.int32))


def apo_run(prob: Problem, params: apo_params, stream=None, want_curve=True):
    """apo_run (host outputs, synchronous): returns (best_x, best_f, curve)."""
    best_x = np.empty(prob.D, np.float32)
    best_f = C.c_double()
    T = apo_effective_iterations(params)
    curve = np.empty(max(T, 0) + 1, np.float32) if want_curve else None
    _check(_lib.apo_run(prob.handle, C.byref(params), _stream(stream), _np_ptr(best_x, C.c_float),
                        C.byref(best_f), _np_ptr(curve, C.c_float)), "apo_run")
    return best_x, best_f.value, curve


def apo_run_device(prob: Problem, params: apo_params, d_best_x, d_best_f, d_curve=None, stream=None):
    _check(_lib.apo_run_device(prob.handle, C.byref(params), _stream(stream), _dptr(d_best_x), _dptr(d_best_f),
                               _dptr(d_curve)), "apo_run_device")


def apo_run_device_noalloc(prob: Problem, params: apo_params, d_best_x, d_best_f, d_curve=None, stream=None):
    """apo_run_device without any device allocation (shared static scratch; synchronous)."""
    _check(_lib.apo_run_device_noalloc(prob.handle, C.byref(params), _stream(stream), _dptr(d_best_x),
                                       _dptr(d_best_f), _dptr(d_curve)), "apo_run_device_noalloc")


def apo_run_batch(probs, params, d_best_x, x_stride, d_best_f, d_curves=None, curve_stride=0, stream=None):
    n = len(probs)
    handles = (_P * n)(*[p.handle for p in probs])
    prm = (apo_params * n)(*params)
    _check(_lib.apo_run_batch(handles, prm, n, _stream(stream), _dptr(d_best_x), int(x_stride), _dptr(d_best_f),
                              _dptr(d_curves), int(curve_stride)), "apo_run_batch")


class Batch:
    """A prepared batch (apo_batch_create); keeps its problems and outputs alive."""

    def __init__(self, handle, probs, outs):
        self.handle, self._probs, self._outs = handle, probs, outs

    def launch(self, stream=None):
        _check(_lib.apo_batch_launch(self.handle, _stream(stream)), "apo_batch_launch")

    def autotune(self, probe_iters=50, stream=None):
        o = apo_batch_options()
        _check(_lib.apo_batch_autotune(self.handle, _stream(stream), int(probe_iters), C.byref(o)),
               "apo_batch_autotune")
        return {"smem_budget": int(o.smem_budget), "ctas_per_sm": int(o.ctas_per_sm),
                "cluster_ps": int(o.cluster_ps), "cluster_size": int(o.cluster_size)}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.apo_batch_destroy(h)
            self.handle = None


def apo_batch_create(probs, params, d_best_x, x_stride, d_best_f, d_curves=None, curve_stride=0,
                     smem_budget=0, ctas_per_sm=0, cluster_ps=0, cluster_size=0) -> Batch:
    n = len(probs)
    handles = (_P * n)(*[p.handle for p in probs])
    prm = (apo_params * n)(*params)
    opt = apo_batch_options(int(smem_budget), int(ctas_per_sm), int(cluster_ps), int(cluster_size))
    h = _P()
    _check(_lib.apo_batch_create(handles, prm, n, _dptr(d_best_x), int(x_stride), _dptr(d_best_f), _dptr(d_curves),
                                 int(curve_stride), C.byref(opt), C.byref(h)), "apo_batch_create")
    return Batch(h, list(probs), (d_best_x, d_best_f, d_curves))


def apo_step(prob: Problem, params: apo_params, it: int, d_X, d_F, stream=None):
    _check(_lib.apo_step(prob.handle, C.byref(params), int(it), _stream(stream), _dptr(d_X), _dptr(d_F)),
           "apo_step")


def apo_init_state(prob: Problem, params: apo_params, d_X, d_F, stream=None):
    """apo_init_state: the run's initial population into d_X [ps, D], d_F [ps] (protozoon order)."""
    _check(_lib.apo_init_state(prob.handle, C.byref(params), _stream(stream), _dptr(d_X), _dptr(d_F)),
           "apo_init_state")


def apo_run_from_state(prob: Problem, params: apo_params, t_begin: int, t_end: int, d_X, d_F, d_best_x=None,
                       d_best_f=None, d_curve=None, stream=None):
    """apo_run_from_state: iterations t_begin..t_end from the state (d_X, d_F), which is updated in place."""
    _check(_lib.apo_run_from_state(prob.handle, C.byref(params), int(t_begin), int(t_end), _stream(stream),
                                   _dptr(d_X), _dptr(d_F), _dptr(d_best_x), _dptr(d_best_f), _dptr(d_curve)),
           "apo_run_from_state")


def apo_evaluate(prob: Problem, d_X, d_F, stream=None):
    _check(_lib.apo_evaluate(prob.handle, _stream(stream), _dptr(d_X), int(d_X.shape[0]), _dptr(d_F)),
           "apo_evaluate")


def apo_clamp_eval_select(prob: Problem, d_X, d_F, d_Xnew, d_Fnew, stream=None):
    _check(_lib.apo_clamp_eval_select(prob.handle, _stream(stream), int(d_X.shape[0]), _dptr(d_X), _dptr(d_F),
                                      _dptr(d_Xnew), _dptr(d_Fnew)), "apo_clamp_eval_select")


def apo_histogram_u8(d_pixels, n_per_image, n_images, d_hist, stream=None):
    _check(_lib.apo_histogram_u8(_dptr(d_pixels), int(n_per_image), int(n_images), _dptr(d_hist),
                                 _stream(stream)), "apo_histogram_u8")


def apo_philox4x32_10(d_ctr, key0, key1, d_out, stream=None):
    _check(_lib.apo_philox4x32_10(_dptr(d_ctr), int(key0) & 0xFFFFFFFF, int(key1) & 0xFFFFFFFF,
                                  int(d_ctr.numel() // 4), _dptr(d_out), _stream(stream)), "apo_philox4x32_10")


def apo_set_timing_events(before, after):
    """before / after: torch.cuda.Event objects (or None, None to clear)."""
    if before is not None and (not before.cuda_event or not after.cuda_event):
        raise ValueError("record the events once before registering them (torch creates them lazily)")
    b = None if before is None else C.c_void_p(before.cuda_event)
    a = None if after is None else C.c_void_p(after.cuda_event)
    _check(_lib.apo_set_timing_events(b, a), "apo_set_timing_events")


class Mlp:
    """Surrogate network handle (apo_mlp_create / apo_mlp_destroy)."""

    H = 256

    def __init__(self, D, seed=0):
        self.D = int(D)
        h = _P()
        _check(_lib.apo_mlp_create(self.D, int(seed) & 0xFFFFFFFF, C.byref(h)), "apo_mlp_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.apo_mlp_destroy(h)
            self.handle = None

    def set_params(self, W1, b1, W2, b2, w3, b3):
        a = [np.ascontiguousarray(x, np.float32) for x in (W1, b1, W2, b2, w3)]
        _check(_lib.apo_mlp_set_params(self.handle, *[_np_ptr(x, C.c_float) for x in a], float(b3)),
               "apo_mlp_set_params")

    def get_params(self):
        H = self.H
        out = [np.empty((self.D, H), np.float32), np.empty(H, np.float32), np.empty((H, H), np.float32),
               np.empty(H, np.float32), np.empty(H, np.float32), np.empty(1, np.float32)]
        _check(_lib.apo_mlp_get_params(self.handle, *[_np_ptr(x, C.c_float) for x in out]), "apo_mlp_get_params")
        return dict(W1=out[0], b1=out[1], W2=out[2], b2=out[3], w3=out[4], b3=float(out[5][0]))

    def forward(self, d_X, d_y, stream=None):
        _check(_lib.apo_mlp_forward(self.handle, _dptr(d_X), int(d_X.shape[0]), _dptr(d_y), _stream(stream)),
               "apo_mlp_forward")

    def gradients(self, d_X, d_t):
        H = self.H
        g = [np.empty((self.D, H), np.float32), np.empty(H, np.float32), np.empty((H, H), np.float32),
             np.empty(H, np.float32), np.empty(H, np.float32), np.empty(1, np.float32), np.empty(1, np.float32)]
        _check(_lib.apo_mlp_gradients(self.handle, _dptr(d_X), _dptr(d_t), int(d_X.shape[0]),
                                      *[_np_ptr(x, C.c_float) for x in g]), "apo_mlp_gradients")
        return dict(W1=g[0], b1=g[1], W2=g[2], b2=g[3], w3=g[4], b3=float(g[5][0])), float(g[6][0])

    def train(self, d_X, d_t, steps, batch, lr=1e-3, seed=0, stream=None):
        _check(_lib.apo_mlp_train(self.handle, _dptr(d_X), _dptr(d_t), int(d_X.shape[0]), int(steps), int(batch),
                                  float(lr), int(seed) & 0xFFFFFFFF, _stream(stream)), "apo_mlp_train")


def surrogate_params(k=8, retrain_every=10, archive_cap=50000, train_steps=100, batch=1024, lr=1e-3,
                     min_rank_corr=0.3, net_seed=0, train_window=0):
    return apo_surrogate_params(int(k), int(retrain_every), int(archive_cap), int(train_steps), int(batch), float(lr),
                                float(min_rank_corr), int(net_seed) & 0xFFFFFFFF, int(train_window))


def apo_run_surrogate(prob: Problem, params: apo_params, sp: apo_surrogate_params, stream=None, want_curve=True):
    """apo_run_surrogate (host outputs, synchronous): (best_x, best_f, curve, stats dict)."""
    best_x = np.empty(prob.D, np.float32)
    best_f = C.c_double()
    curve = np.empty(max(apo_effective_iterations(params), 0) + 1, np.float32) if want_curve else None
    st = apo_surrogate_stats()
    _check(_lib.apo_run_surrogate(prob.handle, C.byref(params), C.byref(sp), _stream(stream),
                                  _np_ptr(best_x, C.c_float), C.byref(best_f), _np_ptr(curve, C.c_float),
                                  C.byref(st)), "apo_run_surrogate")
    stats = {f: getattr(st, f) for f, _ in apo_surrogate_stats._fields_}
    return best_x, best_f.value, curve, stats


def apo_surrogate_candidates(prob: Problem, params: apo_params, it: int, k: int, d_X, d_F, d_Xcand, stream=None):
    """apo_surrogate_candidates (test hook, synchronous): the k candidates of every
    protozoon into d_Xcand [ps, k, D], rank-major."""
    _check(_lib.apo_surrogate_candidates(prob.handle, C.byref(params), int(it), int(k), _stream(stream), _dptr(d_X),
                                         _dptr(d_F), _dptr(d_Xcand)), "apo_surrogate_candidates")


def apo_barrier_selftest(launched: int, expected: int, rounds: int = 1, stream=None) -> int:
    """apo_barrier_selftest (test hook): the raw status code (0 = APO_OK,
    4 = APO_ERR_TIMEOUT); does not raise."""
    return int(_lib.apo_barrier_selftest(int(launched), int(expected), int(rounds), _stream(stream)))


def raw_lib():
    """The loaded ctypes library (for callers that time the raw C entry points)."""
    return _lib


def apo_measure_peaks(stream=None):
    """apo_measure_peaks: measured FP32 FMA (TFLOP/s), IMAD and plain ALU (Tops/s) throughputs."""
    f, i, a = C.c_double(), C.c_double(), C.c_double()
    _check(_lib.apo_measure_peaks(_stream(stream), C.byref(f), C.byref(i), C.byref(a)), "apo_measure_peaks")
    return {"ffma_tflops": f.value, "imad_tops": i.value, "alu_tops": a.value}


LARGE_STAGES = ("rank", "generate", "gemm_eval", "greedy")


def apo_large_stage_timing(on: bool):
    """apo_large_stage_timing: the per-stage device ms and launch counts since the last call; sets the switch."""
    ms = (C.c_double * 4)()
    n = (C.c_longlong * 4)()
    _check(_lib.apo_large_stage_timing(int(bool(on)), ms, n), "apo_large_stage_timing")
    return {k: {"ms": ms[i], "launches": int(n[i])} for i, k in enumerate(LARGE_STAGES)}
