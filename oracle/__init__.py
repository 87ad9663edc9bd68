"""CPU oracle for many-path homotopy tracking (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and
the two share no code: this side is a plain C++ library (``ht_oracle.cpp``)
built with g++ and called through ctypes.

Every function follows a passage of Verschelde & Yu (2015):
  * ``eval_``            Table tabcpugpu host loop; method "naive" = product rule,
                         "speelpenning" = reverse mode of Table tabmoneval;
  * ``speelpenning_slots`` Table tabmoneval slot values for one product;
  * ``mgs_solve``        least squares by modified Gram-Schmidt (Section 1);
  * ``compact``          Table tabjobidx scan and path_idx;
  * ``start_solutions``  roots of x_i^d_i - 1 for the homotopy of Eq. eqlinhom;
  * ``track``            the predictor-corrector loop of Section 2;
  * ``real_op``          L-limb arithmetic (double, double double, quad double);
  * ``predict``, ``homotopy``  the tracker's extrapolation predictor and the
                         homotopy of Eq. eqlinhom with its Jacobian, alone;
  * ``tangent``, ``predict_tangent``  the path tangent from J v = -dh/dt and
                         the Euler and Hermite predictors built on it;
  * ``mlp_*``, ``adam_step``  the learned step-size network (not in the paper):
                         fp64 forward, loss gradient, Adam, and the error
                         bound of a reduced-precision evaluation.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.cpp")
_LIB = os.path.join(_HERE, "libhtoracle.so")
_lock = threading.Lock()
_lib = None

# Tracker parameters, in the order the C side reads them.
PARAM_NAMES = ("h0", "h_min", "h_max", "f_up", "f_down", "newton_max", "tol_dx", "tol_res",
               "polish_max", "tol_polish", "r_div", "max_steps", "max_order", "predictor")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no fp contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _open(_LIB)
    return _lib


@contextlib.contextmanager
def loaded_from(path: str):
    """Run the wrappers against another build of the oracle source for the
    duration of the block: the planted-mistake copies that check the pins
    catch mistakes."""
    global _lib
    other = _open(path)
    with _lock:
        saved, _lib = _lib, other
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def compile_variant(source: str, out: str) -> str:
    """Compile C++ source text with the oracle's own flags into the shared
    library `out` (used for the planted-mistake copies)."""
    src = out + ".cpp"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-pthread", "-o", out, src])
    return out


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _open(path: str):
    """Load a build of the oracle and declare its entry points."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int, ctypes.c_int64
    sig = {
        "hto_version": ([], i32),
        "hto_param_count": ([], i32),
        "hto_real_op": ([i32, i32, i64, P, P, P], i32),
        "hto_value_diff": ([i32, i64, P, P, P], i32),
        "hto_eval": ([i32, i32, i32, i32, P, P, P, i64, P, i64, P, P, P, i32], i32),
        "hto_eval_magnitude": ([i32, i32, i32, P, P, P, i64, P, i64, P, P, P], i32),
        "hto_speelpenning_slots": ([i32, i32, P, P], i32),
        "hto_mgs_solve": ([i32, i32, i32, i64, P, P, P], i32),
        "hto_start_solutions": ([i32, i32, P, i64, i64, P], i32),
        "hto_compact": ([P, i64, P, P], i64),
        "hto_track": ([i32, i32, P, P, P, P, P, i64, P, P, i32, P, P, P, P, P, P], i32),
        "hto_predict": ([i32, i32, i32, P, P, ctypes.c_double, P], i32),
        "hto_homotopy": ([i32, i32, P, P, P, P, P, ctypes.c_double, i64, P, P, P], i32),
        "hto_tangent": ([i32, i32, P, P, P, P, P, ctypes.c_double, i64, P, P], i32),
        "hto_predict_tangent": ([i32, i32, i32, ctypes.c_double, P, P, ctypes.c_double, P, P, ctypes.c_double, P],
                                i32),
        "hto_mlp_nparam": ([], i32),
        "hto_mlp_forward": ([i64, P, P, P], i32),
        "hto_mlp_loss_grad": ([i64, P, P, P, P], ctypes.c_double),
        "hto_mlp_error_bound": ([i64, P, P, P, ctypes.c_double, ctypes.c_double, P, P, P], i32),
        "hto_adam_step": ([i64, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, i32], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def real_op(op: str, a: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """Element-wise L-limb arithmetic; a, b: [n][L]."""
    code = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4}[op]
    a = _c(a, np.float64)
    n, L = a.shape
    bb = None if b is None else _c(b, np.float64)
    out = np.empty_like(a)
    rc = lib().hto_real_op(code, L, n, _p(a), _p(bb), _p(out))
    assert rc == 0
    return out


def value_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact (value(a) - value(b)) rounded to double; a, b: [..., L] limbs last."""
    a = _c(a, np.float64)
    b = _c(b, np.float64)
    L = a.shape[-1]
    out = np.empty(a.shape[:-1])
    rc = lib().hto_value_diff(L, out.size, _p(a), _p(b), _p(out))
    assert rc == 0
    return out


def _sys_args(system, limbs):
    nt = _c(system.n_terms, np.int32)
    ex = _c(system.exps, np.int8)
    cf = _c(system.coef_limbs(limbs), np.float64)
    return nt, ex, cf


def eval_(system, x: np.ndarray, pts=None, method: str = "speelpenning", n_threads: int = 0):
    """Values [np][2][L][n_sel] and Jacobian [np][nv][2][L][n_sel] at the points
    x[:, :, :, pts] (all points if pts is None); x: [nv][2][L][n_pts]."""
    x = _c(x, np.float64)
    nv, _, L, n_pts = x.shape
    nt, ex, cf = _sys_args(system, L)
    sel = None if pts is None else _c(pts, np.int64)
    n_sel = n_pts if sel is None else sel.size
    val = np.empty((system.n_polys, 2, L, n_sel))
    jac = np.empty((system.n_polys, nv, 2, L, n_sel))
    rc = lib().hto_eval({"naive": 0, "speelpenning": 1}[method], L, nv, system.n_polys, _p(nt), _p(ex), _p(cf),
                        n_pts, _p(sel), n_sel, _p(x), _p(val), _p(jac), n_threads)
    assert rc == 0
    return val, jac


def eval_magnitude(system, x: np.ndarray, pts=None):
    """Sum of term moduli per output: val [np][n_sel], jac [np][nv][n_sel]."""
    x = _c(x, np.float64)
    nv, _, L, n_pts = x.shape
    nt, ex, cf = _sys_args(system, L)
    sel = None if pts is None else _c(pts, np.int64)
    n_sel = n_pts if sel is None else sel.size
    val = np.empty((system.n_polys, n_sel))
    jac = np.empty((system.n_polys, nv, n_sel))
    rc = lib().hto_eval_magnitude(L, nv, system.n_polys, _p(nt), _p(ex), _p(cf), n_pts, _p(sel), n_sel, _p(x),
                                  _p(val), _p(jac))
    assert rc == 0
    return val, jac


def speelpenning_slots(x: np.ndarray):
    """x: [k][2][L] -> (slots [2k][2][L], number of multiplications)."""
    x = _c(x, np.float64)
    k, _, L = x.shape
    slots = np.zeros((2 * k, 2, L))
    nmul = lib().hto_speelpenning_slots(L, k, _p(x), _p(slots))
    return slots, nmul


def mgs_solve(A: np.ndarray, b: np.ndarray):
    """A: [n_sys][rows][cols][2][L], b: [n_sys][rows][2][L] -> x [n_sys][cols][2][L]."""
    A = _c(A, np.float64)
    b = _c(b, np.float64)
    n_sys, rows, cols, _, L = A.shape
    x = np.empty((n_sys, cols, 2, L))
    rc = lib().hto_mgs_solve(L, rows, cols, n_sys, _p(A), _p(b), _p(x))
    assert rc == 0
    return x


def start_solutions(degrees, first: int, count: int, limbs: int) -> np.ndarray:
    d = _c(degrees, np.int32)
    x = np.empty((d.size, 2, limbs, count))
    rc = lib().hto_start_solutions(limbs, d.size, _p(d), first, count, _p(x))
    assert rc == 0
    return x


def compact(status: np.ndarray):
    """Returns (inclusive scan of status == 0, path_idx of continuing paths)."""
    st = _c(status, np.int8)
    scan = np.empty(st.size, dtype=np.int64)
    idx = np.empty(st.size, dtype=np.int32)
    c = lib().hto_compact(_p(st), st.size, _p(scan), _p(idx))
    return scan, idx[:c].copy()


def default_params(limbs: int, **over) -> dict:
    """Tracker parameters (the paper leaves them open; these are the readings
    used by both the oracle and the CUDA library)."""
    p = dict(h0=0.05, h_min=1e-5, h_max=0.1, f_up=1.5, f_down=0.5, newton_max=3, tol_dx=1e-6, tol_res=1e-4,
             polish_max=4, tol_polish={1: 1e-12, 2: 1e-24, 4: 1e-48}[limbs], r_div=1e8, max_steps=2000,
             max_order=4, predictor=0)
    p.update(over)
    return p


def track(system, start_degrees, gamma, path_ids, limbs: int, params: dict | None = None, n_threads: int = 0):
    """Track the given paths; returns dict with x_end [n][2][L][m], status, t_end,
    steps, rejects, newton."""
    n = system.n_vars
    nt, ex, cf = _sys_args(system, limbs)
    d = _c(start_degrees, np.int32)
    g = _c(np.array(gamma, dtype=np.float64), np.float64)
    ids = _c(path_ids, np.int64)
    m = ids.size
    P = default_params(limbs) if params is None else params
    pv = _c(np.array([P[k] for k in PARAM_NAMES], dtype=np.float64), np.float64)
    assert pv.size == lib().hto_param_count()
    out = dict(x_end=np.empty((n, 2, limbs, m)), status=np.empty(m, np.int8), t_end=np.empty(m),
               steps=np.empty(m, np.int32), rejects=np.empty(m, np.int32), newton=np.empty(m, np.int32))
    rc = lib().hto_track(limbs, n, _p(nt), _p(ex), _p(cf), _p(d), _p(g), m, _p(ids), _p(pv), n_threads,
                         _p(out["x_end"]), _p(out["status"]), _p(out["t_end"]), _p(out["steps"]),
                         _p(out["rejects"]), _p(out["newton"]))
    assert rc == 0
    return out


def predict(ts: np.ndarray, xs: np.ndarray, t1: float) -> np.ndarray:
    """The tracker's extrapolation predictor (Section 2): through the points
    (ts[j], xs[j]), xs [m][n][2][L], to t1; returns [n][2][L]."""
    ts = _c(ts, np.float64)
    xs = _c(xs, np.float64)
    m, n, _, L = xs.shape
    out = np.empty((n, 2, L))
    assert lib().hto_predict(L, n, m, _p(ts), _p(xs), float(t1), _p(out)) == 0
    return out


def homotopy(system, start_degrees, gamma, t: float, x: np.ndarray):
    """gamma (1 - t) g(x) + t f(x) (Eq. eqlinhom, g_i = x_i^d_i - 1) and its
    Jacobian in x at x [n][2][L][n_pts]: h [n][2][L][n_pts], J [n][n][2][L][n_pts]."""
    x = _c(x, np.float64)
    n, _, L, n_pts = x.shape
    nt, ex, cf = _sys_args(system, L)
    d = _c(start_degrees, np.int32)
    g = _c(np.array(gamma, dtype=np.float64), np.float64)
    h = np.empty((n, 2, L, n_pts))
    J = np.empty((n, n, 2, L, n_pts))
    assert lib().hto_homotopy(L, n, _p(nt), _p(ex), _p(cf), _p(d), _p(g), float(t), n_pts, _p(x), _p(h), _p(J)) == 0
    return h, J


def tangent(system, start_degrees, gamma, t: float, x: np.ndarray) -> np.ndarray:
    """The path tangent dx/dt of Eq. eqlinhom at points x [n][2][L][n_pts] and
    time t, from J_x v = -dh/dt by the Newton step's least squares."""
    x = _c(x, np.float64)
    n, _, L, n_pts = x.shape
    nt, ex, cf = _sys_args(system, L)
    d = _c(start_degrees, np.int32)
    g = _c(np.array(gamma, dtype=np.float64), np.float64)
    v = np.empty_like(x)
    assert lib().hto_tangent(L, n, _p(nt), _p(ex), _p(cf), _p(d), _p(g), float(t), n_pts, _p(x), _p(v)) == 0
    return v


def predict_tangent(mode: int, s0, x0, v0, s1, x1, v1, t1) -> np.ndarray:
    """The tracker's tangent predictors (points [n][2][L]): mode 1 Euler from
    (s1, x1, v1), mode 2 the cubic Hermite through (s0, x0, v0), (s1, x1, v1)."""
    x1 = _c(x1, np.float64)
    n, _, L = x1.shape
    z = np.zeros_like(x1)
    x0 = z if x0 is None else _c(x0, np.float64)
    v0 = z if v0 is None else _c(v0, np.float64)
    v1 = _c(v1, np.float64)
    out = np.empty_like(x1)
    assert lib().hto_predict_tangent(L, n, mode, float(s0), _p(x0), _p(v0), float(s1), _p(x1), _p(v1), float(t1),
                                     _p(out)) == 0
    return out


# ------------------------------------------------------------------ learned step
MLP_IN, MLP_HID, MLP_OUT = 16, 64, 2


def mlp_nparam() -> int:
    return lib().hto_mlp_nparam()


def mlp_forward(x: np.ndarray, params: np.ndarray) -> np.ndarray:
    """x [B][16] -> y [B][2] with the fp64 MLP (16 -> 64 -> 64 -> 2, ReLU)."""
    x = _c(x, np.float64)
    p = _c(params, np.float64)
    y = np.empty((x.shape[0], MLP_OUT))
    lib().hto_mlp_forward(x.shape[0], _p(x), _p(p), _p(y))
    return y


def mlp_loss_grad(x, target, params):
    """(mean squared error, gradient over the flat parameters)."""
    x = _c(x, np.float64)
    t = _c(target, np.float64)
    p = _c(params, np.float64)
    g = np.empty(p.size)
    loss = lib().hto_mlp_loss_grad(x.shape[0], _p(x), _p(t), _p(p), _p(g))
    return float(loss), g


def mlp_error_bound(x, target, params, u_act=2.0 ** -8, u_grad=2.0 ** -8):
    """Rigorous bounds on the distance between the exact network output,
    loss and gradient (mlp_forward, mlp_loss_grad) and a computation that
    accumulates in FP32 and rounds the hidden activations (u_act) and the
    weight-gradient operands (u_grad) to a narrower format: (ybound [B][2],
    gbound [n_param], loss bound).  The model is stated in ht_oracle.cpp."""
    x = _c(x, np.float64)
    t = _c(target, np.float64)
    p = _c(params, np.float64)
    yb = np.empty((x.shape[0], MLP_OUT))
    gb = np.empty(p.size)
    lb = np.empty(1)
    assert lib().hto_mlp_error_bound(x.shape[0], _p(x), _p(t), _p(p), float(u_act), float(u_grad), _p(yb), _p(gb),
                                     _p(lb)) == 0
    return yb, gb, float(lb[0])


def adam_step(p, g, m, v, lr, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """In place on p, m, v (float64 arrays)."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    gg = _c(g, np.float64)
    lib().hto_adam_step(p.size, _p(p), _p(gg), _p(m), _p(v), lr, b1, b2, eps, step)
