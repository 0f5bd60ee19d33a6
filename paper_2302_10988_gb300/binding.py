"""ctypes binding of the C ABI in include/alifmm.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The library
``_build/libalifmm.so`` must exist (``paper_2302_10988_gb300.build.build()``
makes it); loading fails with an error when it does not -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libalifmm.so")

ALF_OK = 0
STATUS_NAMES = {0: "ALF_OK", 1: "ALF_ERR_INVALID_ARG", 2: "ALF_ERR_NONPHYSICAL_MATERIAL", 3: "ALF_ERR_OUT_OF_GRID",
                4: "ALF_ERR_CUDA", 5: "ALF_ERR_OOM", 6: "ALF_ERR_NOT_CONVERGED", 7: "ALF_ERR_RAY_INCOMPLETE",
                8: "ALF_ERR_UNSUPPORTED", 9: "ALF_ERR_INCONSISTENT_RECORDS"}
ALF_FP64, ALF_FP32 = 0, 1
ALF_GROUP_PAPER, ALF_GROUP_EXACT = 0, 1
ALF_INIT_RADIUS, ALF_INIT_HIERARCHY = 0, 1

# every symbol include/alifmm.h declares
EXPORTS = ("alf_default_options", "alf_create", "alf_destroy", "alf_last_error", "alf_plan_create",
           "alf_plan_destroy", "alf_plan_field_offset", "alf_plan_nfields", "alf_plan_options", "alf_solve",
           "alf_check64", "alf_trace_rays", "alf_backward", "alf_sync_status", "alf_plan_stats", "alf_plan_autotune",
           "alf_eval_velocity", "alf_solve_field_noalloc", "alf_ray_gradient", "alf_check64_nodes",
           "alf_solve_check64",
           "alf_pack_rays")


class AlfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class alf_material(C.Structure):
    _fields_ = [("c", (C.c_double * 6) * 6), ("rho", C.c_double)]


class alf_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("group_model", C.c_int), ("init_mode", C.c_int), ("init_radius", C.c_int),
                ("n_levels", C.c_int), ("level_density", C.c_int * 4), ("level_radius", C.c_int * 4),
                ("plane_step", C.c_int), ("ray_halfwidth", C.c_int), ("stop_radius", C.c_double),
                ("max_ray_points", C.c_int), ("max_rounds", C.c_int), ("sweep", C.c_int),
                ("ray_family", C.c_int), ("keep_records", C.c_int), ("band_cells", C.c_double),
                ("use_graph", C.c_int), ("time_kernels", C.c_int), ("velocity_table", C.c_int),
                ("cta_threads", C.c_int), ("cta_cluster", C.c_int), ("subgrid", C.c_int),
                ("wave_mode", C.c_int)]


class alf_stats(C.Structure):
    _fields_ = [("node_evaluations", C.c_uint64), ("rounds", C.c_uint64), ("nodes", C.c_uint64),
                ("eval_launches", C.c_uint64), ("eval_ms", C.c_double), ("kernel_launches", C.c_uint64),
                ("dirty_entries", C.c_uint64)]


class alf_geometry(C.Structure):
    _fields_ = [("nsamples", C.c_int), ("nx", C.POINTER(C.c_int32)), ("ny", C.POINTER(C.c_int32)),
                ("h", C.POINTER(C.c_double)), ("region_map", C.POINTER(C.c_uint16)), ("nregions", C.c_int),
                ("region_material", C.POINTER(C.c_uint16)), ("nmaterials", C.c_int),
                ("materials", C.POINTER(alf_material)), ("nsources", C.c_int), ("src_ij", C.POINTER(C.c_int32)),
                ("nreceivers", C.c_int), ("rec_ij", C.POINTER(C.c_int32)),
                ("region_map32", C.POINTER(C.c_uint32)), ("region_material32", C.POINTER(C.c_uint32))]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libalifmm.so and declare its signatures; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libalifmm.so not found at {path}: build it with paper_2302_10988_gb300.build.build()"
                               " (the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(path)
        vp, P = C.c_void_p, C.POINTER
        L.alf_default_options.restype = None
        L.alf_default_options.argtypes = [P(alf_options)]
        L.alf_create.restype = C.c_int
        L.alf_create.argtypes = [P(vp), C.c_int]
        L.alf_destroy.restype = C.c_int
        L.alf_destroy.argtypes = [vp]
        L.alf_last_error.restype = C.c_char_p
        L.alf_last_error.argtypes = [vp]
        L.alf_plan_create.restype = C.c_int
        L.alf_plan_create.argtypes = [vp, P(alf_geometry), P(alf_options), P(vp)]
        L.alf_plan_destroy.restype = C.c_int
        L.alf_plan_destroy.argtypes = [vp]
        L.alf_plan_field_offset.restype = C.c_size_t
        L.alf_plan_field_offset.argtypes = [vp, C.c_int]
        L.alf_plan_nfields.restype = C.c_int
        L.alf_plan_nfields.argtypes = [vp]
        L.alf_plan_options.restype = C.c_int
        L.alf_plan_options.argtypes = [vp, P(alf_options)]
        L.alf_solve.restype = C.c_int
        L.alf_solve.argtypes = [vp, vp, vp, vp, vp, vp]
        L.alf_check64.restype = C.c_int
        L.alf_check64.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.alf_check64_nodes.restype = C.c_int
        L.alf_check64_nodes.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.alf_solve_check64.restype = C.c_int
        L.alf_solve_check64.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.alf_trace_rays.restype = C.c_int
        L.alf_trace_rays.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.alf_pack_rays.restype = C.c_int
        L.alf_pack_rays.argtypes = [vp, vp, vp, vp, vp, vp]
        L.alf_ray_gradient.restype = C.c_int
        L.alf_ray_gradient.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.alf_backward.restype = C.c_int
        L.alf_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.alf_sync_status.restype = C.c_int
        L.alf_sync_status.argtypes = [vp, vp, P(C.c_int32)]
        L.alf_plan_stats.restype = C.c_int
        L.alf_plan_stats.argtypes = [vp, vp, P(alf_stats)]
        L.alf_plan_autotune.restype = C.c_int
        L.alf_plan_autotune.argtypes = [vp, vp, vp, vp, vp]
        L.alf_solve_field_noalloc.restype = C.c_int
        L.alf_solve_field_noalloc.argtypes = [C.c_int, P(alf_material), C.c_int, vp, C.c_int, vp, vp, C.c_int,
                                              C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp,
                                              vp, C.c_char_p, C.c_size_t]
        L.alf_eval_velocity.restype = C.c_int
        L.alf_eval_velocity.argtypes = [vp, P(alf_material), C.c_int, C.c_int, C.c_int, vp, vp, C.c_int, vp]
        _lib = L
        return L


def _check(ctx, code):
    if code != ALF_OK:
        msg = load().alf_last_error(ctx)
        raise AlfError(code, msg.decode() if msg else "")


def alf_default_options() -> alf_options:
    o = alf_options()
    load().alf_default_options(C.byref(o))
    return o


def alf_create(device: int = 0):
    h = C.c_void_p()
    code = load().alf_create(C.byref(h), int(device))
    if code != ALF_OK:
        raise AlfError(code, f"alf_create(device={device}) failed")
    return h


def alf_destroy(ctx):
    return load().alf_destroy(ctx)


def alf_last_error(ctx) -> str:
    m = load().alf_last_error(ctx)
    return m.decode() if m else ""


def alf_plan_create(ctx, geom: alf_geometry, opt: alf_options):
    h = C.c_void_p()
    _check(ctx, load().alf_plan_create(ctx, C.byref(geom), C.byref(opt), C.byref(h)))
    return h


def alf_plan_destroy(plan):
    return load().alf_plan_destroy(plan)


def alf_plan_field_offset(plan, f: int) -> int:
    return int(load().alf_plan_field_offset(plan, int(f)))


def alf_plan_nfields(plan) -> int:
    return int(load().alf_plan_nfields(plan))


def alf_plan_options(plan) -> alf_options:
    o = alf_options()
    load().alf_plan_options(plan, C.byref(o))
    return o


def alf_solve(ctx, plan, theta_ptr, times_ptr, rec_ptr, records_ptr, stream):
    _check(ctx, load().alf_solve(plan, theta_ptr, times_ptr, rec_ptr, records_ptr, stream))


def alf_solve_check64(ctx, plan, theta_ptr, times_ptr, rec_ptr, records_ptr, max_rel_ptr, flips_ptr, stream):
    _check(ctx, load().alf_solve_check64(plan, theta_ptr, times_ptr, rec_ptr, records_ptr, max_rel_ptr, flips_ptr,
                                         stream))


def alf_check64(ctx, plan, theta_ptr, times_ptr, records_ptr, max_rel_ptr, flips_ptr, stream):
    _check(ctx, load().alf_check64(plan, theta_ptr, times_ptr, records_ptr, max_rel_ptr, flips_ptr, stream))


def alf_check64_nodes(ctx, plan, theta_ptr, times_ptr, records_ptr, ctimes_ptr, crec_ptr, max_rel_ptr, flips_ptr,
                      stream):
    _check(ctx, load().alf_check64_nodes(plan, theta_ptr, times_ptr, records_ptr, ctimes_ptr, crec_ptr, max_rel_ptr,
                                         flips_ptr, stream))


def alf_pack_rays(ctx, plan, pts_ptr, npts_ptr, packed_ptr, offsets_ptr, stream):
    _check(ctx, load().alf_pack_rays(plan, pts_ptr, npts_ptr, packed_ptr, offsets_ptr, stream))


def alf_trace_rays(ctx, plan, theta_ptr, times_ptr, pts_ptr, npts_ptr, time_ptr, status_ptr, stream):
    _check(ctx, load().alf_trace_rays(plan, theta_ptr, times_ptr, pts_ptr, npts_ptr, time_ptr, status_ptr, stream))


def alf_ray_gradient(ctx, plan, theta_ptr, pts_ptr, npts_ptr, dray_ptr, grad_ptr, stream):
    _check(ctx, load().alf_ray_gradient(plan, theta_ptr, pts_ptr, npts_ptr, dray_ptr, grad_ptr, stream))


def alf_backward(ctx, plan, theta_ptr, times_ptr, records_ptr, dl_ptr, grad_ptr, stream):
    _check(ctx, load().alf_backward(plan, theta_ptr, times_ptr, records_ptr, dl_ptr, grad_ptr, stream))


def alf_sync_status(plan, stream) -> int:
    w = C.c_int32(0)
    code = load().alf_sync_status(plan, stream, C.byref(w))
    return int(code if code != ALF_OK else w.value)


def alf_plan_stats(ctx, plan, stream):
    out = alf_stats()
    _check(ctx, load().alf_plan_stats(plan, stream, C.byref(out)))
    return {"evaluations": int(out.node_evaluations), "rounds": int(out.rounds), "nodes": int(out.nodes),
            "eval_launches": int(out.eval_launches), "eval_ms": float(out.eval_ms),
            "kernel_launches": int(out.kernel_launches), "dirty_entries": int(out.dirty_entries)}


def alf_plan_autotune(ctx, plan, theta_ptr, times_ptr, records_ptr, stream):
    _check(ctx, load().alf_plan_autotune(plan, theta_ptr, times_ptr, records_ptr, stream))


def alf_eval_velocity(ctx, mat: alf_material, kind, group_model, precision, angles_ptr, out_ptr, n, stream):
    _check(ctx, load().alf_eval_velocity(ctx, C.byref(mat), int(kind), int(group_model), int(precision),
                                         angles_ptr, out_ptr, int(n), stream))


def alf_solve_field_noalloc(device, materials, nmaterials, region_material_ptr, nregions, theta_ptr, region_map_ptr,
                            nx, ny, h, si, sj, init_radius, group_model, times_ptr, stream, max_rounds=0):
    """Allocation-free single-field solve; returns (status, message)."""
    buf = C.create_string_buffer(256)
    code = load().alf_solve_field_noalloc(int(device), materials, int(nmaterials), region_material_ptr,
                                          int(nregions), theta_ptr, region_map_ptr, int(nx), int(ny), float(h),
                                          int(si), int(sj), int(init_radius), int(group_model), int(max_rounds),
                                          times_ptr, stream, buf, 256)
    return int(code), buf.value.decode()
