"""ctypes declarations of libgadep's C ABI (include/gadep.h), argument marshalling only.

The library must have been built (``paper_2605_25963_gb300.build``); loading
fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

GADEP_OK, GADEP_E_INVAL, GADEP_E_MESH, GADEP_E_NOMEM, GADEP_E_CUDA, GADEP_E_TIMEOUT, GADEP_E_DEVICE = (
    0, -1, -2, -3, -4, -5, -6)
STATUS_NAMES = {0: "GADEP_OK", -1: "GADEP_E_INVAL", -2: "GADEP_E_MESH", -3: "GADEP_E_NOMEM",
                -4: "GADEP_E_CUDA", -5: "GADEP_E_TIMEOUT", -6: "GADEP_E_DEVICE"}
MAX_GROUPS = 8

# every symbol include/gadep.h declares
EXPORTS = (
    "gadep_last_error", "gadep_abi_version", "detmesh_build", "detmesh_from_arrays", "detmesh_get",
    "detmesh_solid_stats", "detmesh_locate", "detmesh_destroy", "gadep_xs_build", "gadep_erange_build", "gadep_bvh_build",
    "gadep_bvh_build_opts", "gadep_bvh_opts_default", "gadep_bvh_get_stats", "gadep_bvh_validate", "gadep_bvh_destroy", "gadep_nearest_hit",
    "gadep_opts_default", "gadep_run", "gadep_run_batch", "gadep_grad", "gadep_plan_create",
    "gadep_plan_launch", "gadep_plan_results", "gadep_plan_shape", "gadep_plan_destroy",
    "gadep_count_work", "gadep_philox_words", "gadep_run_noalloc", "gadep_plan_set_timing", "gadep_plan_queue_sizes",
    "gadep_plan_kernel_stats", "gadep_measure_peaks",
)
# kernel kinds of gadep_kernel_stats
KERNEL_KINDS = ("mega", "spawn", "trace", "physics", "gen", "ctrl", "init", "sort", "etrack")


class GadepError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class detmesh_params(C.Structure):
    _fields_ = [("kind", C.c_int32), ("d", C.c_double * 10), ("D", C.c_double * 7),
                ("n_theta", C.c_int32), ("n_phi", C.c_int32), ("z_slices", C.c_int32),
                ("cup_rim_drop", C.c_double), ("sep_delta", C.c_double),
                ("has_source_solid", C.c_int32), ("src_r", C.c_double), ("src_h", C.c_double),
                ("src_z0", C.c_double), ("src_n_sides", C.c_int32),
                ("groove_r", C.c_double), ("groove_w", C.c_double), ("groove_d", C.c_double),
                ("flange_r_in", C.c_double), ("flange_r_out", C.c_double), ("flange_h", C.c_double),
                ("flange_z_top", C.c_double), ("n_bolt_holes", C.c_int32), ("bolt_n_sides", C.c_int32),
                ("bolt_r", C.c_double), ("bolt_rc", C.c_double)]


class gadep_solid(C.Structure):
    _fields_ = [("material", C.c_int32), ("active", C.c_int32), ("group", C.c_int32),
                ("parent", C.c_int32)]


class gadep_bvh_opts(C.Structure):
    _fields_ = [("max_leaf", C.c_int32), ("c_trav", C.c_float), ("c_tri", C.c_float), ("split_alpha", C.c_float),
                ("max_dup", C.c_float), ("clip_ratio", C.c_float), ("clip_pieces", C.c_int32)]


class gadep_bvh_stats(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_leaves", C.c_int32), ("max_depth", C.c_int32),
                ("max_leaf_tris", C.c_int32), ("n_tri", C.c_int32), ("n_region", C.c_int32),
                ("sah_cost", C.c_double), ("node_bytes", C.c_int64), ("tri_bytes", C.c_int64),
                ("n_refs", C.c_int64), ("opts", gadep_bvh_opts)]


class gadep_materials(C.Structure):
    _fields_ = [("n_mat", C.c_int32), ("n_grid", C.c_int32), ("E_min", C.c_double),
                ("E_max", C.c_double), ("mu", C.POINTER(C.c_float)), ("e_n", C.c_int32),
                ("T_min", C.c_double), ("T_max", C.c_double), ("e_range", C.POINTER(C.c_float))]


class gadep_source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos", C.c_float * 3), ("dir", C.c_float * 3),
                ("radius", C.c_float), ("height", C.c_float), ("n_sides", C.c_int32),
                ("solid", C.c_int32)]


class gadep_opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("history_offset", C.c_uint64), ("e_cut_keV", C.c_float),
                ("fep_delta_keV", C.c_float), ("e_max_keV", C.c_float), ("n_bins", C.c_int32),
                ("step_cap", C.c_int32), ("variant", C.c_int32), ("block", C.c_int32),
                ("chunk", C.c_int32), ("blocks_per_sm", C.c_int32), ("n_group", C.c_int32),
                ("group_scale", C.c_float * MAX_GROUPS), ("wf_slots", C.c_int32), ("e_model", C.c_int32)]


class gadep_result(C.Structure):
    _fields_ = [("n_hist", C.c_uint64), ("n_fep", C.c_uint64), ("n_zero", C.c_uint64),
                ("n_over", C.c_uint64), ("n_err", C.c_uint64), ("n_segments", C.c_uint64),
                ("n_interactions", C.c_uint64), ("n_culled", C.c_uint64), ("fepe", C.c_double),
                ("sigma", C.c_double),
                ("sum_dep_active", C.c_double), ("sum_dep_all", C.c_double), ("sum_esc", C.c_double),
                ("dev_err", C.c_uint32)]


class gadep_kernel_stats(C.Structure):
    _fields_ = [("launches", C.c_uint64 * 16), ("ms", C.c_double * 16)]


class gadep_instance(C.Structure):
    _fields_ = [("energy_keV", C.c_float), ("src", gadep_source), ("n_hist", C.c_uint64),
                ("instance", C.c_uint32), ("group_scale", C.c_float * MAX_GROUPS)]


P = C.POINTER
vp = C.c_void_p
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgadep.so (building it first if needed); raise if it cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError("libgadep.so is not built (run paper_2605_25963_gb300.build)")
    L = C.CDLL(path)
    st = C.c_int
    sig = {
        "gadep_last_error": (C.c_char_p, []),
        "gadep_abi_version": (C.c_int32, []),
        "detmesh_build": (st, [P(detmesh_params), P(vp)]),
        "detmesh_from_arrays": (st, [P(C.c_float), C.c_int32, P(C.c_int32), P(C.c_int32), C.c_int32,
                                     P(C.c_int32), P(C.c_int32), P(C.c_int32), C.c_int32, P(vp)]),
        "detmesh_get": (st, [vp, P(P(C.c_float)), P(C.c_int32), P(P(C.c_int32)), P(P(C.c_int32)),
                             P(C.c_int32), P(P(gadep_solid)), P(C.c_int32)]),
        "detmesh_solid_stats": (st, [vp, C.c_int32, P(C.c_double), P(C.c_int32)]),
        "detmesh_locate": (st, [vp, P(C.c_double), P(C.c_int32)]),
        "detmesh_destroy": (None, [vp]),
        "gadep_xs_build": (st, [P(C.c_int32), C.c_int32, C.c_int32, C.c_double, C.c_double, P(C.c_float)]),
        "gadep_erange_build": (st, [P(C.c_int32), C.c_int32, C.c_int32, C.c_double, C.c_double, P(C.c_float)]),
        "gadep_bvh_build": (st, [vp, C.c_int32, P(vp)]),
        "gadep_bvh_build_opts": (st, [vp, P(gadep_bvh_opts), C.c_int32, P(vp)]),
        "gadep_bvh_opts_default": (None, [P(gadep_bvh_opts)]),
        "gadep_bvh_get_stats": (st, [vp, P(gadep_bvh_stats)]),
        "gadep_bvh_validate": (st, [vp]),
        "gadep_bvh_destroy": (None, [vp]),
        "gadep_nearest_hit": (st, [vp, vp, vp, C.c_int64, vp, vp, vp, vp]),
        "gadep_opts_default": (None, [P(gadep_opts)]),
        "gadep_run": (st, [vp, P(gadep_materials), P(gadep_source), C.c_float, C.c_uint64, C.c_uint32,
                           P(gadep_opts), vp, vp, C.c_uint64, P(gadep_result), vp]),
        "gadep_run_batch": (st, [vp, P(gadep_materials), C.c_int32, P(gadep_instance), P(gadep_opts), vp,
                                 P(gadep_result), vp]),
        "gadep_grad": (st, [vp, P(gadep_materials), C.c_int32, P(gadep_instance), P(gadep_opts), vp,
                            P(gadep_result), P(C.c_double), P(C.c_double), vp]),
        "gadep_plan_create": (st, [vp, P(gadep_materials), C.c_int32, P(gadep_instance), P(gadep_opts),
                                   C.c_int32, P(vp)]),
        "gadep_plan_launch": (st, [vp, vp, vp]),
        "gadep_plan_results": (st, [vp, vp, P(gadep_result), P(C.c_double), P(C.c_double), vp]),
        "gadep_plan_shape": (st, [vp, P(C.c_int32), P(C.c_int32), P(C.c_int32)]),
        "gadep_plan_destroy": (None, [vp]),
        "gadep_plan_set_timing": (st, [vp, C.c_int32]),
        "gadep_plan_queue_sizes": (st, [vp, P(C.c_uint32), C.c_int32, P(C.c_int32), vp]),
        "gadep_measure_peaks": (st, [C.c_int32, P(C.c_double), P(C.c_double)]),
        "gadep_plan_kernel_stats": (st, [vp, P(gadep_kernel_stats), C.c_int32]),
        "gadep_count_work": (st, [vp, P(gadep_materials), C.c_int32, P(gadep_instance), P(gadep_opts),
                                  P(gadep_result), P(C.c_uint64), P(C.c_uint64), P(C.c_uint64), P(C.c_uint64),
                                  vp]),
        "gadep_philox_words": (st, [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int32, vp, vp]),
        "gadep_run_noalloc": (st, [vp, P(gadep_materials), P(gadep_source), C.c_float, C.c_uint64, C.c_uint32,
                                   P(gadep_opts), vp, P(gadep_result), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int):
    if status != GADEP_OK:
        raise GadepError(status, load().gadep_last_error().decode())
    return status
