"""Thin ctypes binding of libdh (include/dh.h).

Argument marshalling only: every step of the patch update runs in the CUDA
kernels of libdh.so.  Device buffers are torch tensors (float64, contiguous,
on the GPU) or raw device pointers (int); streams are torch streams or raw
cudaStream_t values.  There is no CPU fallback: if libdh.so is missing or the
tensors are not on a CUDA device, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdh.so")
_lib = None

DH_OK, DH_EINVAL, DH_ECUDA, DH_EUNSUPPORTED, DH_ENOMEM, DH_ETIMEOUT = 0, -1, -2, -3, -4, -5
PDE_ADV_FLUX, PDE_ADV_NCP, PDE_EULER2D, PDE_EULER3D, PDE_WAVE3D, PDE_SRHD3D, PDE_GW59 = range(7)

# Every symbol that include/dh.h declares (checked by the CPU tests).
EXPORTS = ["dh_plan_create", "dh_plan_destroy", "patch_update_fv", "patch_update_fv_muscl", "patch_update_fd_ko",
           "max_wave_speed",
           "dh_cfl_dt", "dh_prim2con", "dh_gather_aoas", "dh_scatter_aoas", "dh_offload_bind", "dh_offload_bind_staged", "dh_offload_run", "dh_plan_set_con2prim", "dh_rk_step", "dh_graph_capture", "dh_graph_launch", "dh_graph_info",
           "dh_graph_stage_times", "dh_probe_dfma", "dh_check_recip", "dh_check_sqrt", "dh_check_convert", "dh_generic_work_list", "dh_autotune", "dh_autotune_steps", "dh_plan_set_variant", "dh_plan_set_variant_muscl", "dh_plan_errors", "dh_plan_set_debug", "patch_update_fv_noalloc", "con2prim", "con2prim_flat",
           "dh_mlp_features", "dh_mlp_standardize", "dh_mlp_forward", "dh_mlp_grad", "dh_mlp_adam", "dh_mlp_train",
           "dh_last_error", "dh_version"]


class DhError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().dh_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def lib():
    """Load libdh.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(paper_2608_19273_gb300/build.py); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, d, i32, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        L.dh_plan_create.argtypes = [ctypes.POINTER(vp), i32, i32, vp, i32, i32, i64, vp, i32]
        L.dh_plan_destroy.argtypes = [vp]
        L.patch_update_fv.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, d, d, d, vp, vp]
        L.patch_update_fd_ko.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, d, d, d, d, vp, vp]
        L.patch_update_fv_muscl.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, d, d, d, vp, vp]
        L.max_wave_speed.argtypes = [vp, vp, vp, vp, vp]
        L.dh_cfl_dt.argtypes = [vp, vp, d, vp, vp]
        L.dh_prim2con.argtypes = [vp, vp, vp, vp]
        L.dh_gather_aoas.argtypes = [vp, vp, i32, i32, vp, vp]
        L.dh_scatter_aoas.argtypes = [vp, vp, vp, i32, i32, vp]
        L.dh_offload_bind.argtypes = [vp, vp, i32, i32]
        L.dh_offload_bind_staged.argtypes = [vp, vp, i32, i32]
        L.dh_offload_run.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp, vp, d, d, i32, vp]
        L.dh_probe_dfma.argtypes = [vp, i64, i32, vp]
        L.dh_check_recip.argtypes = [vp, vp, vp, i64, vp]
        L.dh_check_sqrt.argtypes = [vp, vp, vp, i64, vp]
        L.dh_generic_work_list.argtypes = [i32, vp, i32, vp, i32, vp]
        L.dh_check_convert.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
        L.dh_autotune.argtypes = [vp, i32, vp, vp, vp, vp, i32, ctypes.c_char_p, vp, vp, vp]
        L.dh_autotune_steps.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, d, d, i32, ctypes.c_char_p,
                                        vp, vp, vp]
        L.dh_plan_set_variant.argtypes = [vp, i32, i32, i32]
        L.dh_plan_set_variant_muscl.argtypes = [vp, i32]
        L.dh_plan_errors.argtypes = [vp, vp, i32]
        L.dh_plan_set_debug.argtypes = [vp, i32]
        L.patch_update_fv_noalloc.argtypes = [i32, i32, vp, i32, i64, vp, i32, vp, vp, vp, vp, vp, vp, d, d, d, d,
                                              vp, vp]
        L.con2prim.argtypes = [vp, vp, vp, vp, vp, d, i32, i32, vp, vp, vp, vp]
        L.con2prim_flat.argtypes = [vp, vp, i64, i64, vp, vp, d, d, i32, i32, vp, vp, vp, vp]
        f32 = ctypes.c_float
        L.dh_mlp_features.argtypes = [vp, vp, i64, i64, vp, vp, vp]
        L.dh_mlp_standardize.argtypes = [vp, i64, vp, vp, i32, vp]
        L.dh_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        L.dh_mlp_grad.argtypes = [vp, vp, vp, i64, i32, vp, vp, vp]
        L.dh_mlp_adam.argtypes = [vp, vp, vp, vp, i32, f32, f32, f32, f32, vp]
        L.dh_mlp_train.argtypes = [vp, vp, vp, vp, vp, i64, i32, i32, i32, f32, vp, vp, vp, vp]
        L.dh_plan_set_con2prim.argtypes = [vp, vp, d, i32, i32, vp]
        L.dh_rk_step.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, d, d, vp]
        L.dh_graph_capture.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, d, d, i32, vp]
        L.dh_graph_launch.argtypes = [vp, vp]
        L.dh_graph_info.argtypes = [vp, vp, vp]
        L.dh_graph_stage_times.argtypes = [vp, vp, i32]
        L.dh_last_error.restype = ctypes.c_char_p
        L.dh_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _ptr(x, what="buffer"):
    """Device pointer of a CUDA float64/float32/uint8/int32 tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not getattr(x, "is_cuda", False):
        raise TypeError(f"{what} must be a CUDA tensor (no CPU fallback)")
    if not x.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st, where):
    if st != DH_OK:
        raise DhError(st, where)


class Plan:
    """Owns a dh_plan: device patch table, tile work list, reduction scratch."""

    def __init__(self, pde, dim, patches, halo, var_stride, params=None):
        patches = np.ascontiguousarray(patches, dtype=synth.PATCH_DTYPE)
        prm = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        h = ctypes.c_void_p()
        st = lib().dh_plan_create(ctypes.byref(h), int(pde), int(dim), patches.ctypes.data, len(patches), int(halo),
                                  int(var_stride), None if prm is None else prm.ctypes.data,
                                  0 if prm is None else len(prm))
        _check(st, "dh_plan_create")
        self.handle = h.value
        self.pde, self.dim, self.halo, self.var_stride = pde, dim, halo, var_stride
        self.patches = patches
        self.nq = synth.PDE_NQ[pde]
        self.nm = synth.PDE_NM[pde]

    def close(self):
        if getattr(self, "handle", None):
            lib().dh_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def dh_plan_create(pde, dim, patches, halo, var_stride, params=None):
    return Plan(pde, dim, patches, halo, var_stride, params)


def dh_plan_destroy(plan):
    plan.close()


def patch_update_fv(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, lam_out_dev=None, stream=None):
    st = lib().patch_update_fv(plan.handle, _ptr(qs, "qs"), _ptr(q0, "q0"), _ptr(out, "out"), _ptr(acc, "acc"),
                               _ptr(mat, "mat"), _ptr(dt_dev, "dt_dev"), float(a), float(b), float(g), float(d),
                               _ptr(lam_out_dev, "lam_out_dev"), _stream(stream))
    _check(st, "patch_update_fv")


def patch_update_fv_muscl(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, lam_out_dev=None, stream=None):
    st = lib().patch_update_fv_muscl(plan.handle, _ptr(qs, "qs"), _ptr(q0, "q0"), _ptr(out, "out"),
                                     _ptr(acc, "acc"), _ptr(mat, "mat"), _ptr(dt_dev, "dt_dev"), float(a), float(b),
                                     float(g), float(d), _ptr(lam_out_dev, "lam_out_dev"), _stream(stream))
    _check(st, "patch_update_fv_muscl")


def patch_update_fd_ko(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, sigma_ko=0.1, lam_out_dev=None,
                       stream=None):
    st = lib().patch_update_fd_ko(plan.handle, _ptr(qs, "qs"), _ptr(q0, "q0"), _ptr(out, "out"),
                                  _ptr(acc, "acc"), _ptr(mat, "mat"), _ptr(dt_dev, "dt_dev"), float(a), float(b),
                                  float(g), float(d), float(sigma_ko), _ptr(lam_out_dev, "lam_out_dev"),
                                  _stream(stream))
    _check(st, "patch_update_fd_ko")


def patch_update_fv_noalloc(pde, dim, patches, var_stride, params, qs, q0, out, acc, mat, dt_dev, a, b, g, d,
                            lam_out_dev=None, stream=None):
    """FV stage without a plan and without any device allocation (static device scratch; see dh.h)."""
    patches = np.ascontiguousarray(patches, dtype=synth.PATCH_DTYPE)
    prm = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    st = lib().patch_update_fv_noalloc(int(pde), int(dim), patches.ctypes.data, len(patches), int(var_stride),
                                       None if prm is None else prm.ctypes.data, 0 if prm is None else len(prm),
                                       _ptr(qs, "qs"), _ptr(q0, "q0"), _ptr(out, "out"), _ptr(acc, "acc"),
                                       _ptr(mat, "mat"), _ptr(dt_dev, "dt_dev"), float(a), float(b), float(g),
                                       float(d), _ptr(lam_out_dev, "lam_out_dev"), _stream(stream))
    _check(st, "patch_update_fv_noalloc")


def con2prim(plan, cons, prim, p_prev=None, mlp_w=None, tol=1e-12, max_iter=50, status=None, iters=None,
             fail_count_dev=None, stream=None, seed_refine=0):
    """seed_refine (the C argument after max_iter) comes last here so that positional calls keep their meaning."""
    _check(lib().con2prim(plan.handle, _ptr(cons, "cons"), _ptr(prim, "prim"), _ptr(p_prev, "p_prev"),
                          _ptr(mlp_w, "mlp_w"), float(tol), int(max_iter), int(seed_refine), _ptr(status, "status"),
                          _ptr(iters, "iters"), _ptr(fail_count_dev, "fail_count"), _stream(stream)), "con2prim")


def con2prim_flat(cons, prim, n, stride, p_prev=None, mlp_w=None, Gamma=5.0 / 3.0, tol=1e-12, max_iter=50,
                  status=None, iters=None, fail_count_dev=None, stream=None, seed_refine=0):
    _check(lib().con2prim_flat(_ptr(cons, "cons"), _ptr(prim, "prim"), int(n), int(stride), _ptr(p_prev, "p_prev"),
                               _ptr(mlp_w, "mlp_w"), float(Gamma), float(tol), int(max_iter), int(seed_refine),
                               _ptr(status, "status"), _ptr(iters, "iters"), _ptr(fail_count_dev, "fail_count"),
                               _stream(stream)), "con2prim_flat")


MLP_NW, MLP_LEN = 1217, 1224


def dh_mlp_features(cons, p, n, stride, x, y=None, stream=None):
    _check(lib().dh_mlp_features(_ptr(cons, "cons"), _ptr(p, "p"), int(n), int(stride), _ptr(x, "x"), _ptr(y, "y"),
                                 _stream(stream)), "dh_mlp_features")


def dh_mlp_standardize(x, n, w, scratch, stream=None):
    _check(lib().dh_mlp_standardize(_ptr(x, "x"), int(n), _ptr(w, "w"), _ptr(scratch, "scratch"),
                                    int(scratch.numel()), _stream(stream)), "dh_mlp_standardize")


def dh_mlp_forward(w, x, n, y, stream=None):
    _check(lib().dh_mlp_forward(_ptr(w, "w"), _ptr(x, "x"), int(n), _ptr(y, "y"), _stream(stream)), "dh_mlp_forward")


def dh_mlp_grad(w, x, t, offset, B, partials, grad, stream=None):
    _check(lib().dh_mlp_grad(_ptr(w, "w"), _ptr(x, "x"), _ptr(t, "t"), int(offset), int(B),
                             _ptr(partials, "partials"), _ptr(grad, "grad"), _stream(stream)), "dh_mlp_grad")


def dh_mlp_adam(w, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(lib().dh_mlp_adam(_ptr(w, "w"), _ptr(m, "m"), _ptr(v, "v"), _ptr(g, "g"), int(t), float(lr), float(b1),
                             float(b2), float(eps), _stream(stream)), "dh_mlp_adam")


def dh_mlp_train(w, m, v, x, t, n, batch, steps, t0, lr, partials, grad, loss_log=None, stream=None):
    _check(lib().dh_mlp_train(_ptr(w, "w"), _ptr(m, "m"), _ptr(v, "v"), _ptr(x, "x"), _ptr(t, "t"), int(n),
                              int(batch), int(steps), int(t0), float(lr), _ptr(partials, "partials"),
                              _ptr(grad, "grad"), _ptr(loss_log, "loss_log"), _stream(stream)), "dh_mlp_train")


def max_wave_speed(plan, q, mat, lam_out_dev, stream=None):
    _check(lib().max_wave_speed(plan.handle, _ptr(q, "q"), _ptr(mat, "mat"), _ptr(lam_out_dev, "lam"),
                                _stream(stream)), "max_wave_speed")


def dh_cfl_dt(plan, lam_dev, cfl, dt_dev, stream=None):
    _check(lib().dh_cfl_dt(plan.handle, _ptr(lam_dev, "lam"), float(cfl), _ptr(dt_dev, "dt"), _stream(stream)),
           "dh_cfl_dt")


def dh_prim2con(plan, prim, cons, stream=None):
    _check(lib().dh_prim2con(plan.handle, _ptr(prim, "prim"), _ptr(cons, "cons"), _stream(stream)), "dh_prim2con")


def block_pointer_table(blocks):
    """Device int64 tensor holding the data pointers of a list of CUDA tensors (one AoS block per patch)."""
    import torch
    for b in blocks:
        _ptr(b, "AoS block")
    return torch.tensor([b.data_ptr() for b in blocks], dtype=torch.int64).to(blocks[0].device)


def dh_gather_aoas(plan, block_ptrs, nq, aos_halo, arena, stream=None):
    """arena <- interior voxels of the K AoS patch blocks (paper Eq. 4 gather prologue).

    ``block_ptrs``: device int64 tensor of K block addresses (block_pointer_table)."""
    _check(lib().dh_gather_aoas(plan.handle, _ptr(block_ptrs, "block_ptrs"), int(nq), int(aos_halo),
                                _ptr(arena, "arena"), _stream(stream)), "dh_gather_aoas")


def dh_scatter_aoas(plan, arena, block_ptrs, nq, aos_halo, stream=None):
    """Interior voxels of the K AoS patch blocks <- arena (paper Eq. 4 scatter epilogue)."""
    _check(lib().dh_scatter_aoas(plan.handle, _ptr(arena, "arena"), _ptr(block_ptrs, "block_ptrs"), int(nq),
                                 int(aos_halo), _stream(stream)), "dh_scatter_aoas")


def dh_offload_bind(plan, block_addrs, nq, aos_halo):
    """Bind the K AoS patch blocks (addresses: list of ints or tensors; device or page-locked host memory)."""
    addrs = [b if isinstance(b, int) else b.data_ptr() for b in block_addrs]
    table = (ctypes.c_void_p * len(addrs))(*addrs)
    _check(lib().dh_offload_bind(plan.handle, ctypes.cast(table, ctypes.c_void_p), int(nq), int(aos_halo)),
           "dh_offload_bind")


def dh_offload_bind_staged(plan, block_addrs, nq, aos_halo):
    """Bind page-locked host blocks for runs that move their span with the copy engine."""
    addrs = [b if isinstance(b, int) else b.data_ptr() for b in block_addrs]
    table = (ctypes.c_void_p * len(addrs))(*addrs)
    _check(lib().dh_offload_bind_staged(plan.handle, ctypes.cast(table, ctypes.c_void_p), int(nq), int(aos_halo)),
           "dh_offload_bind_staged")


def dh_offload_run(plan, scheme, rk, n_steps, arena, u1, u2, acc, dt_dev, lam_dev, cfl, sigma_ko, nq_back,
                   stream=None):
    """Gather the bound blocks into ``arena``, advance n_steps steps, scatter nq_back quantities back."""
    _check(lib().dh_offload_run(plan.handle, int(scheme), int(rk), int(n_steps), _ptr(arena, "arena"),
                                _ptr(u1, "u1"), _ptr(u2, "u2"), _ptr(acc, "acc"), _ptr(dt_dev, "dt"),
                                _ptr(lam_dev, "lam"), float(cfl), float(sigma_ko), int(nq_back), _stream(stream)),
           "dh_offload_run")


def dh_plan_set_con2prim(plan, mlp_w=None, tol=1e-12, max_iter=50, fail_count_dev=None, seed_refine=0):
    _check(lib().dh_plan_set_con2prim(plan.handle, _ptr(mlp_w, "mlp_w"), float(tol), int(max_iter),
                                      int(seed_refine), _ptr(fail_count_dev, "fail_count")), "dh_plan_set_con2prim")


def dh_rk_step(plan, scheme, rk, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko=0.1, stream=None):
    _check(lib().dh_rk_step(plan.handle, int(scheme), int(rk), _ptr(q, "q"), _ptr(u1, "u1"), _ptr(u2, "u2"),
                            _ptr(acc, "acc"), _ptr(mat, "mat"), _ptr(dt_dev, "dt"), _ptr(lam_dev, "lam"),
                            float(cfl), float(sigma_ko), _stream(stream)), "dh_rk_step")


def dh_graph_capture(plan, scheme, rk, n_steps, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko=0.1,
                     timing=False, stream=None):
    _check(lib().dh_graph_capture(plan.handle, int(scheme), int(rk), int(n_steps), _ptr(q, "q"), _ptr(u1, "u1"),
                                  _ptr(u2, "u2"), _ptr(acc, "acc"), _ptr(mat, "mat"), _ptr(dt_dev, "dt"),
                                  _ptr(lam_dev, "lam"), float(cfl), float(sigma_ko), int(bool(timing)),
                                  _stream(stream)), "dh_graph_capture")


def dh_graph_launch(plan, stream=None):
    _check(lib().dh_graph_launch(plan.handle, _stream(stream)), "dh_graph_launch")


def dh_graph_info(plan):
    nk, nt = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().dh_graph_info(plan.handle, ctypes.byref(nk), ctypes.byref(nt)), "dh_graph_info")
    return nk.value, nt.value


def dh_graph_stage_times(plan, n):
    out = (ctypes.c_float * n)()
    _check(lib().dh_graph_stage_times(plan.handle, out, int(n)), "dh_graph_stage_times")
    return np.array(out[:], dtype=np.float64)


def dh_probe_dfma(out_dev, n_threads, iters, stream=None):
    _check(lib().dh_probe_dfma(_ptr(out_dev, "out"), int(n_threads), int(iters), _stream(stream)), "dh_probe_dfma")


def dh_autotune(plan, scheme, qs, out, mat, dt_dev, reps=3, cache_path=None, stream=None):
    """Pick the fastest kernel variant for this plan; returns (fv_var, fv_zs, fd_var, from_cache, times_ms)."""
    choice = (ctypes.c_int32 * 4)()
    times = (ctypes.c_float * 64)()  # DH_TUNE_MAX_CANDIDATES
    _check(lib().dh_autotune(plan.handle, int(scheme), _ptr(qs, "qs"), _ptr(out, "out"), _ptr(mat, "mat"),
                             _ptr(dt_dev, "dt"), int(reps), None if cache_path is None else cache_path.encode(),
                             choice, times, _stream(stream)), "dh_autotune")
    return choice[0], choice[1], choice[2], bool(choice[3]), [float(t) for t in times]


def dh_autotune_steps(plan, scheme, rk, n_steps, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko=0.1, reps=2,
                      cache_path=None, stream=None):
    """Pick the fastest kernel variant over whole time steps (q, mat are advanced: pass scratch copies);
    returns (fv_var, fv_zs, fd_var, from_cache, times_ms)."""
    choice = (ctypes.c_int32 * 4)()
    times = (ctypes.c_float * 64)()  # DH_TUNE_MAX_CANDIDATES
    _check(lib().dh_autotune_steps(plan.handle, int(scheme), int(rk), int(n_steps), _ptr(q, "q"), _ptr(u1, "u1"),
                                   _ptr(u2, "u2"), _ptr(acc, "acc"), _ptr(mat, "mat"), _ptr(dt_dev, "dt"),
                                   _ptr(lam_dev, "lam"), float(cfl), float(sigma_ko), int(reps),
                                   None if cache_path is None else cache_path.encode(), choice, times,
                                   _stream(stream)), "dh_autotune_steps")
    return choice[0], choice[1], choice[2], bool(choice[3]), [float(t) for t in times]


def dh_plan_set_variant(plan, fv_var, fv_zs, fd_var):
    _check(lib().dh_plan_set_variant(plan.handle, int(fv_var), int(fv_zs), int(fd_var)), "dh_plan_set_variant")


def dh_plan_set_variant_muscl(plan, fv2_var):
    _check(lib().dh_plan_set_variant_muscl(plan.handle, int(fv2_var)), "dh_plan_set_variant_muscl")


def dh_plan_errors(plan, clear=True):
    flags = ctypes.c_uint32()
    _check(lib().dh_plan_errors(plan.handle, ctypes.byref(flags), int(bool(clear))), "dh_plan_errors")
    return flags.value


def dh_plan_set_debug(plan, flags):
    _check(lib().dh_plan_set_debug(plan.handle, int(flags)), "dh_plan_set_debug")


def dh_check_sqrt(x, y_sqrt, y_rsqrt, stream=None):
    _check(lib().dh_check_sqrt(_ptr(x, "x"), _ptr(y_sqrt, "y_sqrt"), _ptr(y_rsqrt, "y_rsqrt"), int(x.numel()),
                               _stream(stream)), "dh_check_sqrt")


def dh_generic_work_list(dim, patches):
    """The generic FV stage's work list of a patch table (host only): an int32 array of shape
    (items, 16): patch[0..7], x0, y0, z0, bx, by, bz, ng, mp."""
    patches = np.ascontiguousarray(patches, dtype=synth.PATCH_DTYPE)
    n = ctypes.c_int32(0)
    _check(lib().dh_generic_work_list(int(dim), patches.ctypes.data, len(patches), None, 0, ctypes.byref(n)),
           "dh_generic_work_list")
    out = np.zeros((n.value, 16), dtype=np.int32)
    _check(lib().dh_generic_work_list(int(dim), patches.ctypes.data, len(patches), out.ctypes.data, n.value,
                                      ctypes.byref(n)), "dh_generic_work_list")
    return out


def dh_check_recip(x, y_nr, y_div, stream=None):
    _check(lib().dh_check_recip(_ptr(x, "x"), _ptr(y_nr, "y_nr"), _ptr(y_div, "y_div"), int(x.numel()),
                                _stream(stream)), "dh_check_recip")


def dh_check_convert(x, f_int, f_hw, g, d_int, d_hw, stream=None):
    _check(lib().dh_check_convert(_ptr(x, "x"), _ptr(f_int, "f_int"), _ptr(f_hw, "f_hw"), _ptr(g, "g"),
                                  _ptr(d_int, "d_int"), _ptr(d_hw, "d_hw"), int(x.numel()), _stream(stream)),
           "dh_check_convert")


def version():
    return lib().dh_version().decode()
