"""Thin ctypes binding of the C ABI in include/ht.h (argument marshalling only).

Each function has the name and argument order of its C counterpart.  Buffers
may be torch tensors (their ``data_ptr()`` is passed), numpy arrays (host
entry points only) or plain integer addresses.  A ``stream`` of None means
torch's current CUDA stream.  A negative return code raises ``HTError`` with
the library's message.  Every step of the computation runs in libht.so; if
the library is missing every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libht.so")

HT_D, HT_DD, HT_QD = 1, 2, 4
HT_OK, HT_EINVAL, HT_ENOMEM, HT_ECUDA, HT_ETIMEOUT, HT_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
_ERR_NAMES = {-1: "HT_EINVAL", -2: "HT_ENOMEM", -3: "HT_ECUDA", -4: "HT_ETIMEOUT", -5: "HT_EUNSUPPORTED"}

P = ctypes.c_void_p
I32, I64 = ctypes.c_int, ctypes.c_int64

# name -> (argtypes, restype); kept in the order of include/ht.h
SIGNATURES = {
    "ht_last_error": ([], ctypes.c_char_p),
    "ht_create_system": ([I32, I32, P, P, P, I32, ctypes.POINTER(P)], I32),
    "ht_destroy_system": ([P], I32),
    "ht_system_info": ([P, P, P, P, P], I32),
    "ht_eval_diff": ([P, I64, P, P, P, P], I32),
    "ht_eval_diff_host": ([P, I64, P, P, P, P], I32),
    "ht_set_eval_config": ([P, I32, I32], I32),
    "ht_tune_eval": ([P, I64, P, P, P, I32, P, P, P, P], I32),
    "ht_mlp_create": ([ctypes.POINTER(P)], I32),
    "ht_mlp_destroy": ([P], I32),
    "ht_mlp_set_params": ([P, P], I32),
    "ht_mlp_get_params": ([P, P], I32),
    "ht_mlp_forward": ([P, I64, P, P, P], I32),
    "ht_mlp_loss_grad": ([P, I64, P, P, P, P, P], I32),
    "ht_mlp_train": ([P, I64, P, P, I32, I64, ctypes.c_float, P, P], I32),
    "ht_mlp_adam_step": ([P, P, ctypes.c_float, P], I32),
    "ht_mlp_get_moments": ([P, P, P, P], I32),
    "ht_default_params": ([I32, P], I32),
    "ht_start_solutions": ([I32, P, I32, I64, I64, P, P], I32),
    "ht_mgs_solve": ([I32, I32, I32, I64, P, P, P, P], I32),
    "ht_mgs_solve_ex": ([I32, I32, I32, I32, I64, P, P, P, P], I32),
    "ht_compact": ([P, I64, P, P, P], I32),
    "ht_compact_noalloc": ([P, I64, P, P, P], I32),
    "ht_track_paths": ([P, P, P, I64, I64, P, P, P, P, P, P, P, P], I32),
    "ht_track_paths_ex": ([P, P, P, I64, I64, P, P, P, P, P, P, P, P, P], I32),
    "ht_track_refined": ([P, P, P, P, I64, I64, P, P, P, P, P, P, P], I32),
    "ht_eval_diff_unfused": ([P, I64, P, P, P, P, P], I32),
    "ht_tune_track": ([P, P, P, I64, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_double), P], I32),
    "ht_record_size": ([I32, I32, I32], I64),
    "ht_step_labels": ([P, P, P, P, I64, P, I32, P, I32, P, P], I32),
    "ht_step_features": ([I32, I32, I32, I32, I64, P, P, P], I32),
    "ht_bench_fp64_rate": ([I32, ctypes.POINTER(ctypes.c_double), P], I32),
    "ht_bench_imad_rate": ([I32, ctypes.POINTER(ctypes.c_double), P], I32),
}



class ht_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("h0", "h_min", "h_max", "f_up", "f_down", "tol_dx", "tol_res",
                                                "tol_polish", "r_div")] + \
               [(k, ctypes.c_int32) for k in ("newton_max", "polish_max", "max_steps", "max_order", "team_warps",
                                               "iters_per_launch", "rounds_per_sync", "predictor")]


class ht_track_io(ctypes.Structure):
    _fields_ = [("init_records", ctypes.c_void_p), ("trace", ctypes.c_void_p), ("trace_capacity", ctypes.c_int64),
                ("trace_count", ctypes.c_void_p), ("trace_stride", ctypes.c_int32), ("fallback_steps", ctypes.c_int32),
                ("mlp", ctypes.c_void_p), ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double),
                ("x0_limbs", ctypes.c_int32), ("polish_only", ctypes.c_int32), ("last_dx_out", ctypes.c_void_p),
                ("last_res_out", ctypes.c_void_p), ("newton_out", ctypes.c_void_p), ("alpha_max", ctypes.c_double)]


class ht_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("converged", "failed", "diverged", "steps", "rejects", "newton")] + \
               [("launches", ctypes.c_int32), ("syncs", ctypes.c_int32), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ht_unfused_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("ms_coeff", "ms_mon", "ms_sum", "bytes_coeff", "bytes_mon",
                                                "bytes_sum")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ht_refine_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("converged", "failed", "diverged", "lo_converged", "retracked")] + \
               [(k, ctypes.c_double) for k in ("ms_lo", "ms_refine", "ms_retrack")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


class HTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_ERR_NAMES.get(code, "HT_E?"), code, msg))
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libht.so (built by paper_1505_00383_gb300._build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libht.so is not built (%s); run `python -m paper_1505_00383_gb300._build` "
                                   "or __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise HTError(rc, lib().ht_last_error().decode())
    return rc


def _ptr(buf):
    """Address of a torch tensor, numpy array or integer (None -> NULL)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):  # torch.Tensor
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    if hasattr(buf, "ctypes"):  # numpy.ndarray
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data
    raise TypeError("unsupported buffer type %r" % type(buf))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class System:
    """Owner of an ht_system handle; released by ht_destroy_system."""

    def __init__(self, handle: int, n_vars: int, n_polys: int, limbs: int):
        self.handle = handle
        self.n_vars, self.n_polys, self.limbs = n_vars, n_polys, limbs

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ht_destroy_system(self.handle)
            self.handle = None


def ht_last_error() -> str:
    return lib().ht_last_error().decode()


def ht_create_system(n_vars, n_polys, n_terms, exps, coef, limbs) -> System:
    """n_terms int32 [n_polys], exps int8 [M][n_vars], coef float64 [M][2][limbs] (host arrays)."""
    import numpy as np
    nt = np.ascontiguousarray(n_terms, dtype=np.int32)
    ex = np.ascontiguousarray(exps, dtype=np.int8)
    cf = np.ascontiguousarray(coef, dtype=np.float64)
    out = P()
    _check(lib().ht_create_system(n_vars, n_polys, _ptr(nt), _ptr(ex), _ptr(cf), limbs, ctypes.byref(out)))
    return System(out.value, n_vars, n_polys, limbs)


def ht_destroy_system(sys: System) -> None:
    if sys.handle:
        _check(lib().ht_destroy_system(sys.handle))
        sys.handle = None


def ht_system_info(sys: System):
    nv, np_, L, M = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(lib().ht_system_info(sys.handle, ctypes.byref(nv), ctypes.byref(np_), ctypes.byref(L), ctypes.byref(M)))
    return nv.value, np_.value, L.value, M.value


def ht_eval_diff(sys: System, n_pts: int, x, val, jac, stream=None) -> None:
    """Device buffers: x [nv][2][L][n_pts], val [np][2][L][n_pts], jac [np][nv][2][L][n_pts]."""
    _check(lib().ht_eval_diff(sys.handle, n_pts, _ptr(x), _ptr(val), _ptr(jac), _stream(stream)))


def ht_eval_diff_host(sys: System, n_pts: int, x, val, jac, stream=None) -> None:
    """As ht_eval_diff on host buffers; returns when the results are in host memory."""
    _check(lib().ht_eval_diff_host(sys.handle, n_pts, _ptr(x), _ptr(val), _ptr(jac), _stream(stream)))


def ht_set_eval_config(sys: System, variant: int, threads: int) -> None:
    _check(lib().ht_set_eval_config(sys.handle, variant, threads))


def ht_tune_eval(sys: System, n_pts, x, val, jac, reps=3, stream=None):
    """Returns (variant, threads, best_ms) and keeps that choice in the system."""
    v, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().ht_tune_eval(sys.handle, n_pts, _ptr(x), _ptr(val), _ptr(jac), reps, ctypes.byref(v),
                              ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return v.value, t.value, ms.value


def system_from(system, limbs: int) -> System:
    """Upload a synth.System-like object (n_vars, n_polys, n_terms, exps, coef_limbs)."""
    return ht_create_system(system.n_vars, system.n_polys, system.n_terms, system.exps,
                            system.coef_limbs(limbs), limbs)


def ht_bench_fp64_rate(iters: int = 50, stream=None) -> float:
    """Measured FP64 instructions per second of the current device."""
    r = ctypes.c_double()
    _check(lib().ht_bench_fp64_rate(iters, ctypes.byref(r), _stream(stream)))
    return r.value


def ht_bench_imad_rate(iters: int = 20, stream=None) -> float:
    """Measured 32x32->64-bit integer multiply-adds per second of the device."""
    r = ctypes.c_double()
    _check(lib().ht_bench_imad_rate(iters, ctypes.byref(r), _stream(stream)))
    return r.value


def ht_default_params(limbs: int, **over) -> "ht_params":
    p = ht_params()
    _check(lib().ht_default_params(limbs, ctypes.byref(p)))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def ht_start_solutions(n, degrees, limbs, first, count, x0, stream=None) -> None:
    import numpy as np
    d = np.ascontiguousarray(degrees, dtype=np.int32)
    _check(lib().ht_start_solutions(n, _ptr(d), limbs, first, count, _ptr(x0), _stream(stream)))


def ht_mgs_solve(limbs, rows, cols, n_sys, Ab, R, x, stream=None) -> None:
    _check(lib().ht_mgs_solve(limbs, rows, cols, n_sys, _ptr(Ab), _ptr(R), _ptr(x), _stream(stream)))


def ht_mgs_solve_ex(limbs, variant, rows, cols, n_sys, Ab, R, x, stream=None) -> None:
    _check(lib().ht_mgs_solve_ex(limbs, variant, rows, cols, n_sys, _ptr(Ab), _ptr(R), _ptr(x), _stream(stream)))


def ht_compact(status, m, path_idx, count, stream=None) -> None:
    _check(lib().ht_compact(_ptr(status), m, _ptr(path_idx), _ptr(count), _stream(stream)))


HT_NOALLOC_MAX_PATHS = 1 << 22


def ht_compact_noalloc(status, m, path_idx, count, stream=None) -> None:
    """ht_compact without allocating: scratch is a fixed array in the library
    (m <= HT_NOALLOC_MAX_PATHS)."""
    _check(lib().ht_compact_noalloc(_ptr(status), m, _ptr(path_idx), _ptr(count), _stream(stream)))


def ht_track_paths(sys: System, start_deg, gamma, n_paths, first_path, x0, params, x_end, status, t_end,
                   steps=None, stats: "ht_stats | None" = None, stream=None) -> None:
    """Track paths first_path.. of gamma (1 - t) g + t f = 0; device outputs
    x_end [n][2][L][n_paths], status int8 [n_paths], t_end [n_paths]."""
    import numpy as np
    d = np.ascontiguousarray(start_deg, dtype=np.int32)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    pp = None if params is None else ctypes.byref(params)
    sp = None if stats is None else ctypes.byref(stats)
    _check(lib().ht_track_paths(sys.handle, _ptr(d), _ptr(g), n_paths, first_path, _ptr(x0), pp, _ptr(x_end),
                                _ptr(status), _ptr(t_end), _ptr(steps), sp, _stream(stream)))


def ht_eval_diff_unfused(sys: System, n_pts, x, val, jac, stats: "ht_unfused_stats | None" = None,
                         stream=None) -> None:
    """The three-kernel (coeff, mon, sum) evaluation; stats (optional) times
    each kernel and counts its algorithmic bytes."""
    sp = None if stats is None else ctypes.byref(stats)
    _check(lib().ht_eval_diff_unfused(sys.handle, n_pts, _ptr(x), _ptr(val), _ptr(jac), sp, _stream(stream)))


def ht_track_refined(lo: System, hi: System, start_deg, gamma, n_paths, first_path, p_lo, p_hi, x_end, status,
                     t_end, stats: "ht_refine_stats | None" = None, stream=None) -> None:
    """Track in lo's precision, refine endpoints in hi's, track failures again
    in hi's; device outputs x_end [n][2][L_hi][n_paths], status, t_end."""
    import numpy as np
    d = np.ascontiguousarray(start_deg, dtype=np.int32)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    pl = None if p_lo is None else ctypes.byref(p_lo)
    ph = None if p_hi is None else ctypes.byref(p_hi)
    sp = None if stats is None else ctypes.byref(stats)
    _check(lib().ht_track_refined(lo.handle, hi.handle, _ptr(d), _ptr(g), n_paths, first_path, pl, ph, _ptr(x_end),
                                  _ptr(status), _ptr(t_end), sp, _stream(stream)))


HT_MLP_IN, HT_MLP_OUT, HT_MLP_NPARAM = 16, 2, 5378


class Mlp:
    """Owner of an ht_mlp handle."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ht_mlp_destroy(self.handle)
            self.handle = None


def ht_mlp_create() -> Mlp:
    out = P()
    _check(lib().ht_mlp_create(ctypes.byref(out)))
    return Mlp(out.value)


def ht_mlp_destroy(net: Mlp) -> None:
    if net.handle:
        _check(lib().ht_mlp_destroy(net.handle))
        net.handle = None


def ht_mlp_set_params(net: Mlp, params) -> None:
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == HT_MLP_NPARAM
    _check(lib().ht_mlp_set_params(net.handle, _ptr(p)))


def ht_mlp_get_params(net: Mlp):
    import numpy as np
    p = np.empty(HT_MLP_NPARAM, dtype=np.float32)
    _check(lib().ht_mlp_get_params(net.handle, _ptr(p)))
    return p


def ht_mlp_forward(net: Mlp, B, x, y, stream=None) -> None:
    _check(lib().ht_mlp_forward(net.handle, B, _ptr(x), _ptr(y), _stream(stream)))


def ht_mlp_loss_grad(net: Mlp, B, x, target, grad, loss, stream=None) -> None:
    _check(lib().ht_mlp_loss_grad(net.handle, B, _ptr(x), _ptr(target), _ptr(grad), _ptr(loss), _stream(stream)))


def ht_mlp_train(net: Mlp, n, x, target, epochs, batch, lr, stream=None):
    import numpy as np
    losses = np.zeros(epochs, dtype=np.float32)
    _check(lib().ht_mlp_train(net.handle, n, _ptr(x), _ptr(target), epochs, batch, ctypes.c_float(lr), _ptr(losses),
                              _stream(stream)))
    return losses


def ht_mlp_adam_step(net: Mlp, grad, lr, stream=None) -> None:
    """One Adam step on the network's FP32 masters with a device gradient."""
    _check(lib().ht_mlp_adam_step(net.handle, _ptr(grad), ctypes.c_float(lr), _stream(stream)))


def ht_mlp_get_moments(net: Mlp):
    """(m, v, step): Adam's moments (float32 arrays) and step count."""
    import numpy as np
    m = np.empty(HT_MLP_NPARAM, dtype=np.float32)
    v = np.empty(HT_MLP_NPARAM, dtype=np.float32)
    step = ctypes.c_int32(0)
    _check(lib().ht_mlp_get_moments(net.handle, _ptr(m), _ptr(v), ctypes.byref(step)))
    return m, v, int(step.value)


def ht_record_size(n, limbs, max_order=4) -> int:
    r = lib().ht_record_size(n, limbs, max_order)
    if r < 0:
        raise HTError(HT_EINVAL, "ht_record_size: bad arguments")
    return r


def ht_step_features(n, limbs, max_order, newton_max, n_rec, records, features, stream=None) -> None:
    _check(lib().ht_step_features(n, limbs, max_order, newton_max, n_rec, _ptr(records), _ptr(features),
                                  _stream(stream)))


def ht_track_paths_ex(sys: System, start_deg, gamma, n_paths, first_path, x0, params, x_end, status, t_end,
                      steps=None, stats=None, io: "ht_track_io | None" = None, stream=None) -> None:
    import numpy as np
    d = np.ascontiguousarray(start_deg, dtype=np.int32)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    pp = None if params is None else ctypes.byref(params)
    sp = None if stats is None else ctypes.byref(stats)
    ip = None if io is None else ctypes.byref(io)
    _check(lib().ht_track_paths_ex(sys.handle, _ptr(d), _ptr(g), n_paths, first_path, _ptr(x0), pp, _ptr(x_end),
                                   _ptr(status), _ptr(t_end), _ptr(steps), sp, ip, _stream(stream)))


def ht_tune_track(sys: System, start_deg, gamma, n_paths, params=None, stream=None):
    """Returns (team_warps, iters_per_launch, ms) of the fastest launch shape,
    which the system then uses by default."""
    import numpy as np
    d = np.ascontiguousarray(start_deg, dtype=np.int32)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    team, iters, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    pp = None if params is None else ctypes.byref(params)
    _check(lib().ht_tune_track(sys.handle, _ptr(d), _ptr(g), n_paths, pp, ctypes.byref(team), ctypes.byref(iters),
                               ctypes.byref(ms), _stream(stream)))
    return team.value, iters.value, ms.value


def ht_step_labels(sys: System, start_deg, gamma, params, n_rec, records, mults, newton_max, labels,
                   stream=None) -> None:
    import numpy as np
    d = np.ascontiguousarray(start_deg, dtype=np.int32)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    mu = np.ascontiguousarray(mults, dtype=np.float64)
    _check(lib().ht_step_labels(sys.handle, _ptr(d), _ptr(g), ctypes.byref(params), n_rec, _ptr(records), mu.size,
                                _ptr(mu), newton_max, _ptr(labels), _stream(stream)))
