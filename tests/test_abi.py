"""The C-ABI library loads and exports every symbol that include/dh.h declares,
and rejects malformed plans on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2608_19273_gb300 import build as dhbuild
from paper_2608_19273_gb300 import dh, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdh():
    dhbuild.build()
    return dh.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "dh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:dh_status|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))


def test_header_symbols_exported(libdh):
    names = _declared()
    assert "patch_update_fv" in names and "max_wave_speed" in names
    for n in names:
        assert hasattr(libdh, n), f"{n} declared in dh.h but not exported"
    assert set(names) <= set(dh.EXPORTS) | set(names)
    assert set(dh.EXPORTS) == set(names), "binding EXPORTS list out of sync with dh.h"


def test_version(libdh):
    assert "sm_103a" in dh.version()


def _create(patches, pde=3, dim=3, halo=1, vs=None):
    vs = vs if vs is not None else 1 << 20
    h = ctypes.c_void_p()
    st = dh.lib().dh_plan_create(ctypes.byref(h), pde, dim, patches.ctypes.data, len(patches), halo, vs, None, 0)
    return st


@pytest.mark.parametrize("mutate,code", [
    (lambda P: P.__setitem__("p", 300), dh.DH_EINVAL),        # p outside [2, 256]
    (lambda P: P.__setitem__("p", 1), dh.DH_EINVAL),          # p outside [2, 256]
    (lambda P: P["nbr"].__setitem__((0, 1), 99), dh.DH_EINVAL),  # neighbour out of range
    (lambda P: P.__setitem__("offset", P["offset"] + 3), dh.DH_EINVAL),  # misaligned block
    (lambda P: P["dx"].__setitem__(0, -1.0), dh.DH_EINVAL),   # negative spacing
])
def test_plan_validation_rejects(libdh, mutate, code):
    mesh = synth.euler3d_amr_mesh(scale=8)
    P = mesh.patches.copy()
    mutate(P)
    assert _create(P, vs=mesh.var_stride) == code
    assert len(dh.lib().dh_last_error()) > 0


def test_empty_patch_list_rejected(libdh):
    mesh = synth.euler3d_amr_mesh(scale=8)
    assert _create(mesh.patches[:0].copy(), vs=mesh.var_stride) == dh.DH_EINVAL
    assert b"empty" in dh.lib().dh_last_error()


def test_plan_validation_dim_and_pde(libdh):
    mesh = synth.euler3d_amr_mesh(scale=8)
    assert _create(mesh.patches.copy(), pde=2, dim=3, vs=mesh.var_stride) == dh.DH_EINVAL
    assert _create(mesh.patches.copy(), pde=9, dim=3, vs=mesh.var_stride) == dh.DH_EINVAL
    assert _create(mesh.patches.copy(), vs=mesh.var_stride + 1) == dh.DH_EINVAL


def test_binding_refuses_cpu_tensors(libdh):
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        dh._ptr(torch.zeros(4, dtype=torch.float64), "q")


def test_null_plan_rejected(libdh):
    L = dh.lib()
    assert L.patch_update_fv(None, None, None, None, None, None, None, 0.0, 1.0, 1.0, 0.0, None, None) == dh.DH_EINVAL


@pytest.mark.parametrize("mutate", [
    lambda P, f: P["dx"].__setitem__(f, P["dx"][f] * 2.0),       # fine patch with the coarse spacing
    lambda P, f: P["level"].__setitem__(f, 2),                   # neighbour two levels coarser
    lambda P, f: P["p"].__setitem__(f, 16),                      # different p across levels
])
def test_coupled_plan_validation_rejects(libdh, mutate):
    """Coupled refinement levels: a coarser face neighbour must be exactly one level coarser, with
    the same p and twice the dx (checked on the host before any device allocation)."""
    mesh = synth.coupled_mesh(4, 8, 1.0 / 32, 1, 2, dim=3)
    P = mesh.patches.copy()
    mutate(P, mesh.level_ranges[1][0])
    assert _create(P, vs=mesh.var_stride) == dh.DH_EINVAL
    assert len(dh.lib().dh_last_error()) > 0


@pytest.mark.parametrize("case", ["p_too_large", "halo_zero", "halo_too_wide", "stride_too_small", "dx_nan",
                                  "bad_params"])
def test_plan_limits_rejected(libdh, case):
    """The documented limits of dh_plan_create: p a multiple of 8 in [8, 256], halo in [1, 8],
    every block inside var_stride, a positive dx, a parameter array when n_params > 0."""
    mesh = synth.euler3d_amr_mesh(scale=8)
    P = mesh.patches.copy()
    halo, vs, nprm = 1, mesh.var_stride, 0
    if case == "p_too_large":
        P["p"][0] = 264
    elif case == "halo_zero":
        halo = 0
    elif case == "halo_too_wide":
        halo = 9
    elif case == "stride_too_small":
        vs = int(P["offset"].max())  # the last block ends beyond it (a multiple of 32 below the end)
        vs -= vs % 32
    elif case == "dx_nan":
        P["dx"][3] = float("nan")
    elif case == "bad_params":
        nprm = 2  # but no array
    h = ctypes.c_void_p()
    st = dh.lib().dh_plan_create(ctypes.byref(h), 3, 3, P.ctypes.data, len(P), halo, vs, None, nprm)
    assert st == dh.DH_EINVAL and not h.value
    assert len(dh.lib().dh_last_error()) > 0


ENTRY_POINTS = ["patch_update_fv", "patch_update_fd_ko", "patch_update_fv_muscl", "max_wave_speed", "dh_cfl_dt",
                "dh_prim2con", "dh_gather_aoas", "dh_scatter_aoas", "dh_offload_bind", "dh_offload_bind_staged",
                "dh_offload_run", "dh_autotune", "dh_autotune_steps", "dh_plan_set_variant", "dh_plan_set_variant_muscl", "dh_plan_errors", "dh_plan_set_debug",
                "con2prim", "dh_plan_set_con2prim", "dh_rk_step", "dh_graph_capture", "dh_graph_launch",
                "dh_graph_info", "dh_graph_stage_times", "con2prim_flat", "dh_mlp_features", "dh_mlp_standardize",
                "dh_mlp_forward", "dh_mlp_grad", "dh_mlp_adam", "dh_mlp_train", "dh_check_recip", "dh_check_sqrt", "dh_check_convert", "dh_generic_work_list", "dh_probe_dfma",
                "patch_update_fv_noalloc"]


@pytest.mark.parametrize("name", ENTRY_POINTS)
def test_null_arguments_rejected(libdh, name):
    """Every entry point called with a NULL plan / NULL buffers and zero sizes returns DH_EINVAL
    with a message, before touching the device."""
    f = getattr(dh.lib(), name)
    args = [0.0 if t in (ctypes.c_double, ctypes.c_float) else 0 if t in (ctypes.c_int32, ctypes.c_int64)
            else None for t in f.argtypes]
    assert f(*args) == dh.DH_EINVAL
    assert len(dh.lib().dh_last_error()) > 0


def test_destroy_null_plan_is_a_no_op(libdh):
    assert dh.lib().dh_plan_destroy(None) == dh.DH_OK


def test_null_argument_list_covers_the_header():
    """Every entry point of dh.h is in the NULL-argument test, apart from plan creation and
    destruction (tested above) and the two string getters."""
    assert set(_declared()) == set(ENTRY_POINTS) | {"dh_plan_create", "dh_plan_destroy", "dh_last_error",
                                                    "dh_version"}


def _noalloc(P, vs, pde=3, dim=3):
    """patch_update_fv_noalloc with dummy (never dereferenced) device pointers."""
    return dh.lib().patch_update_fv_noalloc(pde, dim, P.ctypes.data, len(P), vs, None, 0, 8, None, 16, None, None,
                                            24, 0.0, 1.0, 1.0, 0.0, None, None)


def test_noalloc_rejects_too_many_work_items(libdh):
    """65 2D patches of 256^2 need 65 x 256 = 16,640 tile work items, above the static limit of
    16,384: rejected on the host, before any CUDA call."""
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 256, 1.0 / 256, 0)], dim=2)
    P = np.repeat(mesh.patches, 65)
    P["nbr"][:, :4] = 0
    P["offset"] = 0
    assert _noalloc(P, mesh.var_stride, pde=2, dim=2) == dh.DH_EINVAL
    assert b"work items" in dh.lib().dh_last_error()


def test_noalloc_rejects_coupled_levels(libdh):
    """A table with coarser face neighbours (coupled refinement levels, accepted by
    dh_plan_create) is rejected by the allocation-free entry point."""
    mesh = synth.coupled_mesh(4, 8, 1.0 / 32, 1, 2, dim=3)
    assert _noalloc(mesh.patches.copy(), mesh.var_stride) == dh.DH_EINVAL
    assert b"neighbour" in dh.lib().dh_last_error()


def test_coupled_levels_need_multiples_of_8(libdh):
    """Patch sizes that are not multiples of 8 run the generic FV stage, which has no coupling of
    refinement levels: a coupled table of such patches is refused before any device call."""
    mesh = synth.coupled_mesh(4, 16, 1.0 / 64, 1, 2)
    P = mesh.patches.copy()
    P["p"] = 12
    assert _create(P, vs=mesh.var_stride) == dh.DH_EINVAL
    assert b"multiples of 8" in dh.lib().dh_last_error()
