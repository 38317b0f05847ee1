"""ctypes wrapper around the FP64 CPU oracle (``oracle/oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The CUDA library never
imports, links or calls anything here, and this module imports nothing from
the library.

Every function mirrors one step of the batched patch update of the paper
(Sec. II, Eq. 1-4); the C++ source documents the formulas.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FV, FD, FV2 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            L.or_num_threads.argtypes = [i]
            L.or_num_threads.restype = i
            L.or_stage.argtypes = [i, i, i, vp, i, i, i64, vp, vp, vp, vp, vp, d, d, d, d, d, d, vp, i, vp]
            L.or_stage.restype = i
            L.or_stage_subset.argtypes = [i, i, i, vp, i, i, i64, vp, vp, vp, vp, vp, d, d, d, d, d, d, vp, i, vp,
                                          i]
            L.or_stage_subset.restype = i
            L.or_max_wave_speed.argtypes = [i, i, vp, i, i64, vp, vp, vp, i]
            L.or_max_wave_speed.restype = d
            L.or_cfl_dt.argtypes = [d, d, i, d]
            L.or_cfl_dt.restype = d
            L.or_rk_steps.argtypes = [i, i, i, vp, i, i, i64, vp, vp, vp, vp, vp, i, i, d, d, d, vp, i, vp]
            L.or_rk_steps.restype = i
            L.or_prim2con.argtypes = [i, vp, vp, i64, i64, vp, i]
            L.or_prim2con.restype = i
            L.or_con2prim.argtypes = [vp, vp, i64, i64, vp, vp, d, i, vp, vp, d, i]
            L.or_con2prim.restype = i
            L.or_refine_seed.argtypes = [vp, i64, i64, vp, i, d, vp]
            L.or_refine_seed.restype = None
            L.or_srhd_invariants.argtypes = [vp, i64, i64, vp]
            L.or_srhd_invariants.restype = None
            L.or_mlp_loss_grad.argtypes = [vp, vp, vp, i, vp]
            L.or_mlp_loss_grad.restype = d
            L.or_mlp_forward.argtypes = [vp, vp, i64, vp]
            L.or_mlp_forward.restype = None
            L.or_adam.argtypes = [vp, vp, vp, vp, i, i, d, d, d, d]
            L.or_adam.restype = None
            L.or_count_flops.argtypes = [i, i, i, i, i, i, i, vp, vp, vp, i]
            L.or_count_flops.restype = ctypes.c_longlong
            L.or_count_con2prim.argtypes = [vp, i64, i64, vp, d, i, d, vp]
            L.or_count_con2prim.restype = ctypes.c_longlong
            L.or_count_max_speed.argtypes = [i, i, vp, vp, i64, i64, vp, i]
            L.or_count_max_speed.restype = ctypes.c_longlong
            _lib = L
    return _lib


def _p(a):
    """Pointer of a C-contiguous numpy array (or None)."""
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], "oracle wants C-contiguous numpy arrays"
    return a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def num_threads(n: int = 0) -> int:
    return lib().or_num_threads(int(n))


def stage(scheme, pde, dim, patches, halo, var_stride, qs, q0=None, out=None, acc=None, mat=None,
          dt=0.0, a=0.0, b=1.0, g=1.0, d=0.0, sigma=0.1, params=None, want_lam=False):
    """One stage  out = a q0 + b qs + g dt L(qs);  acc += d dt L(qs).

    ``out``/``acc`` are updated in place.  Returns lambda_max of the result
    when ``want_lam``."""
    prm = _f64(params)
    lam = np.zeros(1)
    lib().or_stage(scheme, pde, dim, _p(patches), len(patches), halo, var_stride, _p(qs), _p(q0),
                   _p(out), _p(acc), _p(mat), dt, a, b, g, d, sigma, _p(prm),
                   0 if prm is None else len(prm), _p(lam) if want_lam else None)
    return float(lam[0]) if want_lam else None


def stage_subset(scheme, pde, dim, patches, halo, var_stride, qs, only, q0=None, out=None, acc=None, mat=None,
                 dt=0.0, a=0.0, b=1.0, g=1.0, d=0.0, sigma=0.1, params=None):
    """One stage on the listed patches only (their halos still come from every patch)."""
    prm = _f64(params)
    only = np.ascontiguousarray(only, dtype=np.int32)
    lib().or_stage_subset(scheme, pde, dim, _p(patches), len(patches), halo, var_stride, _p(qs), _p(q0), _p(out),
                          _p(acc), _p(mat), dt, a, b, g, d, sigma, _p(prm), 0 if prm is None else len(prm), _p(only),
                          len(only))


def max_wave_speed(pde, dim, patches, var_stride, q, mat=None, params=None):
    prm = _f64(params)
    return lib().or_max_wave_speed(pde, dim, _p(patches), len(patches), var_stride, _p(q), _p(mat),
                                   _p(prm), 0 if prm is None else len(prm))


def cfl_dt(cfl, dx, dim, lam):
    return lib().or_cfl_dt(cfl, dx, dim, lam)


def rk_steps(scheme, pde, dim, patches, halo, var_stride, q, mat=None, rk=3, steps=1, dt_fixed=0.0,
             cfl=0.4, sigma=0.1, params=None):
    """Advance q in place by ``steps`` full Runge-Kutta steps; returns the dt of each step."""
    u1 = np.empty_like(q)
    u2 = np.empty_like(q)
    acc = np.empty_like(q) if rk == 4 else None
    prm = _f64(params)
    dts = np.zeros(max(steps, 1))
    rc = lib().or_rk_steps(scheme, pde, dim, _p(patches), len(patches), halo, var_stride, _p(q), _p(u1),
                           _p(u2), _p(acc), _p(mat), rk, steps, dt_fixed, cfl, sigma, _p(prm),
                           0 if prm is None else len(prm), _p(dts))
    if rc != 0:
        raise ValueError(f"or_rk_steps failed ({rc})")
    return dts[:steps]


def prim2con(pde, prim, var_stride, params=None):
    nq = prim.shape[0]
    cons = np.zeros_like(prim)
    prm = _f64(params)
    rc = lib().or_prim2con(pde, _p(prim), _p(cons), var_stride, var_stride, _p(prm),
                           0 if prm is None else len(prm))
    if rc != 0:
        raise ValueError("prim2con: unsupported pde")
    del nq
    return cons


def con2prim(cons, stride, n=None, p_prev=None, mlp=None, tol=1e-12, max_iter=50, Gamma=5.0 / 3.0, refine=0):
    """Returns (prim, status, iterations, n_fail); refine: FP32 Newton steps applied to the first seed."""
    n = stride if n is None else n
    prim = np.zeros((5, stride))
    status = np.zeros(stride, dtype=np.uint8)
    iters = np.zeros(stride, dtype=np.int32)
    mlpw = None if mlp is None else np.ascontiguousarray(mlp, dtype=np.float32)
    fails = lib().or_con2prim(_p(cons), _p(prim), n, stride, _p(_f64(p_prev)), _p(mlpw), tol, max_iter,
                              _p(status), _p(iters), Gamma, int(refine))
    return prim, status, iters, fails


def refine_seed(cons, seed, k, Gamma=5.0 / 3.0):
    """The FP32 Newton refinement of the first seed, alone: k steps on each of the voxels of a flat
    conserved array (stride = cons.shape[1]) from the given seeds."""
    cons = _f64(cons)
    seed = _f64(seed)
    out = np.zeros(len(seed))
    lib().or_refine_seed(_p(cons), len(seed), cons.shape[1], _p(seed), int(k), Gamma, _p(out))
    return out


def srhd_invariants(cons, stride, n=None):
    n = stride if n is None else n
    x = np.zeros((n, 3))
    lib().or_srhd_invariants(_p(cons), n, stride, _p(x))
    return x


def mlp_loss_grad(w, x, t):
    w = _f64(w)
    x = _f64(x)
    t = _f64(t)
    g = np.zeros(1217)
    loss = lib().or_mlp_loss_grad(_p(w), _p(x), _p(t), len(t), _p(g))
    return loss, g


def mlp_forward(w, x):
    w = _f64(w)
    x = _f64(x)
    y = np.zeros(len(x))
    lib().or_mlp_forward(_p(w), _p(x), len(x), _p(y))
    return y


def adam(w, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place FP64 Adam step on w, m, v."""
    lib().or_adam(_p(w), _p(m), _p(v), _p(_f64(g)), len(w), t, lr, b1, b2, eps)


def count_flops(scheme, pde, dim, p, halo, qs, mat=None, rk=0, with_lam=False, params=None):
    prm = _f64(params)
    return lib().or_count_flops(scheme, pde, dim, p, halo, rk, int(with_lam), _p(_f64(qs)), _p(_f64(mat)),
                                _p(prm), 0 if prm is None else len(prm))


def count_con2prim(cons, n, p_prev=None, tol=1e-12, max_iter=50, Gamma=5.0 / 3.0):
    """(FP64 operations, Newton iterations) of the plain-seeded recovery of the first n voxels of a
    flat conserved array (variable v of voxel i at v * stride + i, stride = cons.shape[1])."""
    cons = _f64(cons)
    it = ctypes.c_longlong(0)
    fl = lib().or_count_con2prim(_p(cons), int(n), cons.shape[1], _p(_f64(p_prev)), tol, max_iter, Gamma,
                                 ctypes.byref(it))
    return int(fl), int(it.value)


def count_max_speed(pde, dim, q, mat, n, params=None):
    """FP64 operations of the maximum characteristic speed (all directions) of n voxels of flat arrays."""
    q, mat, prm = _f64(q), _f64(mat), _f64(params)
    return int(lib().or_count_max_speed(pde, dim, _p(q), _p(mat), int(n), q.shape[1], _p(prm),
                                        0 if prm is None else len(prm)))
