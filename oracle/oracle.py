"""Python front end of the FP64 CPU oracle (``alifmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports
it, and it imports nothing from the CUDA package.

The C file is compiled with gcc on first use into ``oracle/_build/``.
All arrays are numpy; angles are radians; SI units.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alifmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Mat(C.Structure):
    _fields_ = [("c22", C.c_double), ("c23", C.c_double), ("c33", C.c_double), ("c44", C.c_double),
                ("rho", C.c_double), ("c55", C.c_double), ("c66", C.c_double)]


class Medium(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("h", C.c_double),
                ("mat_id", C.POINTER(C.c_int32)), ("theta", C.POINTER(C.c_double)),
                ("mats", C.POINTER(Mat)), ("nmats", C.c_int), ("group_model", C.c_int), ("vtable", C.c_int),
                ("wave_mode", C.c_int), ("env", C.POINTER(C.c_double))]


QP, QSV, SH = 0, 1, 2
ENV_N = 1441  # envelope table entries: 0, 1/8, ..., 180 degrees


class RayOpts(C.Structure):
    _fields_ = [("plane_step", C.c_int), ("halfwidth", C.c_int), ("stop_radius", C.c_double),
                ("max_pts", C.c_int), ("family", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.om_qp_lambda.restype = C.c_double
            L.om_qp_lambda.argtypes = [P(Mat), C.c_double]
            L.om_phase_velocity.restype = C.c_double
            L.om_phase_velocity.argtypes = [P(Mat), C.c_double]
            L.om_mode_lambda.restype = C.c_double
            L.om_mode_lambda.argtypes = [P(Mat), C.c_int, C.c_double]
            L.om_mode_velocity.restype = C.c_double
            L.om_mode_velocity.argtypes = [P(Mat), C.c_int, C.c_double]
            L.om_envelope_slowness.restype = C.c_double
            L.om_envelope_slowness.argtypes = [P(Mat), C.c_int, C.c_double]
            L.om_envelope_table.restype = None
            L.om_envelope_table.argtypes = [P(Mat), C.c_int, P(C.c_double)]
            L.om_envelope_speed.restype = C.c_double
            L.om_envelope_speed.argtypes = [P(C.c_double), C.c_double]
            L.om_group_paper.restype = None
            L.om_group_paper.argtypes = [P(Mat), C.c_double, P(C.c_double), P(C.c_double)]
            L.om_group_exact.restype = None
            L.om_group_exact.argtypes = [P(Mat), C.c_double, P(C.c_double), P(C.c_double)]
            L.om_group_speed.restype = C.c_double
            L.om_group_speed.argtypes = [P(Mat), C.c_int, C.c_double, C.c_double]
            L.om_counter.restype = C.c_int64
            L.om_counter.argtypes = [C.c_int]
            L.om_reset_counters.restype = None
            L.om_stencil_table.restype = P(C.c_int)
            L.om_diamond_table.restype = P(C.c_int)
            L.om_stencil_value.restype = C.c_double
            L.om_stencil_value.argtypes = [P(Medium), P(C.c_double), C.c_int, C.c_int, C.c_int]
            L.om_fmm.restype = C.c_int
            L.om_fmm.argtypes = [P(Medium), P(C.c_uint8), P(C.c_double), P(C.c_int16), P(C.c_int32),
                                 P(C.c_int64)]
            L.om_F_node.restype = C.c_double
            L.om_F_node.argtypes = [P(Medium), P(C.c_uint8), P(C.c_double), C.c_int, C.c_int, P(C.c_int)]
            L.om_F_all.restype = None
            L.om_F_all.argtypes = [P(Medium), P(C.c_uint8), P(C.c_double), P(C.c_double), P(C.c_int16)]
            L.om_F_check_all.restype = None
            L.om_F_check_all.argtypes = [P(Medium), P(C.c_uint8), P(C.c_double), P(C.c_double), P(C.c_int16)]
            L.om_jacobi.restype = C.c_int
            L.om_jacobi.argtypes = [P(Medium), P(C.c_uint8), P(C.c_double), P(C.c_int16), C.c_int]
            L.om_init_radius.restype = None
            L.om_init_radius.argtypes = [P(Medium), C.c_int, C.c_int, C.c_int, P(C.c_uint8), P(C.c_double)]
            L.om_init_hierarchy.restype = C.c_int
            L.om_init_hierarchy.argtypes = [P(Medium), C.c_int, C.c_int, C.c_int, P(C.c_int), P(C.c_int),
                                            P(C.c_uint8), P(C.c_double)]
            L.om_adjoint.restype = None
            L.om_adjoint.argtypes = [P(Medium), P(C.c_uint8), P(C.c_double), P(C.c_int16), P(C.c_int32),
                                     P(C.c_double), C.c_int, C.c_int, P(C.c_int32), C.c_int, P(C.c_double)]
            L.om_trace_ray.restype = C.c_int
            L.om_trace_ray.argtypes = [P(Medium), P(C.c_double), C.c_double, C.c_double, C.c_double,
                                       C.c_double, P(RayOpts), P(C.c_double), P(C.c_int)]
            L.om_path_time.restype = C.c_double
            L.om_path_time.argtypes = [P(Medium), P(C.c_double), C.c_int]
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# --------------------------------------------------------------------------- materials
def mat_from_voigt(c6, rho) -> Mat:
    """In-plane constants of the YZ plane (Sec. 3.2): c22, c23, c33, c44 of the 6x6 Voigt matrix."""
    c6 = np.asarray(c6, dtype=np.float64)
    return Mat(c6[1, 1], c6[1, 2], c6[2, 2], c6[3, 3], float(rho), c6[4, 4], c6[5, 5])


def qp_lambda(m: Mat, theta: float) -> float:
    return lib().om_qp_lambda(C.byref(m), float(theta))


def phase_velocity(m: Mat, theta: float) -> float:
    return lib().om_phase_velocity(C.byref(m), float(theta))


def mode_velocity(m: Mat, mode: int, theta: float) -> float:
    """Phase speed of wave mode 0 (qP), 1 (qSV) or 2 (SH) at phase angle theta (Sec. 3.2, Sec. 7)."""
    return lib().om_mode_velocity(C.byref(m), int(mode), float(theta))


def envelope_slowness(m: Mat, mode: int, psi: float) -> float:
    """First-arrival group slowness along psi: max over theta of cos(theta - psi) / v(theta)."""
    return lib().om_envelope_slowness(C.byref(m), int(mode), float(psi))


def envelope_table(m: Mat, mode: int) -> np.ndarray:
    tab = np.empty(ENV_N, np.float64)
    lib().om_envelope_table(C.byref(m), int(mode), _ptr(tab, C.c_double))
    return tab


def mode_group_speed(m: Mat, mode: int, psi: float) -> float:
    """Group speed of a shear mode along psi from the material axis: the envelope table, interpolated [R20]."""
    tab = envelope_table(m, mode)
    return lib().om_envelope_speed(_ptr(tab, C.c_double), float(psi))


def group_paper(m: Mat, phi: float):
    th, V = C.c_double(), C.c_double()
    lib().om_group_paper(C.byref(m), float(phi), C.byref(th), C.byref(V))
    return th.value, V.value


def group_exact(m: Mat, phi: float):
    th, V = C.c_double(), C.c_double()
    lib().om_group_exact(C.byref(m), float(phi), C.byref(th), C.byref(V))
    return th.value, V.value


GROUP_PAPER, GROUP_EXACT = 0, 1


def stencil_table() -> np.ndarray:
    p = lib().om_stencil_table()
    return np.array([p[k] for k in range(32 * 6)], dtype=np.int64).reshape(32, 3, 2)


def diamond_table() -> np.ndarray:
    p = lib().om_diamond_table()
    return np.array([p[k] for k in range(24)], dtype=np.int64).reshape(12, 2)


# --------------------------------------------------------------------------- media
class OMedium:
    """A medium on an nx x ny grid: per-node material index and orientation."""

    def __init__(self, nx, ny, h, mat_id, theta, mats, group_model=GROUP_PAPER, vtable=0, wave_mode=QP):
        self.nx, self.ny, self.h = int(nx), int(ny), float(h)
        self.mat_id = np.ascontiguousarray(mat_id, dtype=np.int32).reshape(ny * nx)
        self.theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(ny * nx)
        self._mats = (Mat * len(mats))(*mats)
        self.mats = list(mats)
        self.group_model = int(group_model)
        self.vtable = int(vtable)
        self.wave_mode = int(wave_mode)
        # shear modes: every material's envelope table (the group speeds of [R20])
        self.env = (np.concatenate([envelope_table(m, self.wave_mode) for m in mats]) if self.wave_mode
                    else np.zeros(1))
        self.c = Medium(self.nx, self.ny, self.h, _ptr(self.mat_id, C.c_int32), _ptr(self.theta, C.c_double),
                        self._mats, len(mats), self.group_model, self.vtable, self.wave_mode,
                        _ptr(self.env, C.c_double))

    @classmethod
    def from_regions(cls, nx, ny, h, region_map, region_theta, region_material, mats, group_model=GROUP_PAPER,
                     vtable=0, wave_mode=QP):
        rm = np.asarray(region_map).reshape(ny, nx).astype(np.int64)
        return cls(nx, ny, h, np.asarray(region_material)[rm], np.asarray(region_theta, np.float64)[rm], mats,
                   group_model, vtable, wave_mode)


def init_radius(M: OMedium, si: int, sj: int, r0: int):
    frozen = np.zeros(M.nx * M.ny, np.uint8)
    tau = np.empty(M.nx * M.ny, np.float64)
    lib().om_init_radius(C.byref(M.c), int(si), int(sj), int(r0), _ptr(frozen, C.c_uint8), _ptr(tau, C.c_double))
    return frozen, tau


def init_hierarchy(M: OMedium, si: int, sj: int, densities=(27, 9, 3), radii=(1, 6, 13)):
    """Sec. 4.4 near-source grid hierarchy; returns (frozen, tau) on the original grid."""
    d = np.ascontiguousarray(densities, np.int32)
    r = np.ascontiguousarray(radii, np.int32)
    frozen = np.zeros(M.nx * M.ny, np.uint8)
    tau = np.empty(M.nx * M.ny, np.float64)
    lib().om_init_hierarchy(C.byref(M.c), int(si), int(sj), int(d.size), _ptr(d, C.c_int), _ptr(r, C.c_int),
                            _ptr(frozen, C.c_uint8), _ptr(tau, C.c_double))
    return frozen, tau


def fmm(M: OMedium, frozen, tau0, with_order=False):
    """Heap-ordered ALI-FMM.  Returns (tau [ny, nx], rec [ny, nx], stats[, order])."""
    frozen = np.ascontiguousarray(frozen, np.uint8).reshape(-1)
    tau = np.ascontiguousarray(tau0, np.float64).reshape(-1).copy()
    rec = np.empty(tau.size, np.int16)
    order = np.empty(tau.size, np.int32)
    stats = np.zeros(3, np.int64)
    rc = lib().om_fmm(C.byref(M.c), _ptr(frozen, C.c_uint8), _ptr(tau, C.c_double), _ptr(rec, C.c_int16),
                      _ptr(order, C.c_int32), _ptr(stats, C.c_int64))
    out = (tau.reshape(M.ny, M.nx), rec.reshape(M.ny, M.nx),
           {"accepted": int(stats[0]), "fallback": int(stats[1]), "noncausal": int(stats[2]), "unreached": rc})
    if with_order:
        return out + (order.reshape(M.ny, M.nx),)
    return out


def F_all(M: OMedium, frozen, tau):
    frozen = np.ascontiguousarray(frozen, np.uint8).reshape(-1)
    tin = np.ascontiguousarray(tau, np.float64).reshape(-1)
    tout = np.empty_like(tin)
    rec = np.empty(tin.size, np.int16)
    lib().om_F_all(C.byref(M.c), _ptr(frozen, C.c_uint8), _ptr(tin, C.c_double), _ptr(tout, C.c_double),
                   _ptr(rec, C.c_int16))
    return tout.reshape(M.ny, M.nx), rec.reshape(M.ny, M.nx)


def F_check(M: OMedium, frozen, tau):
    """The update of every node of a solved field with its known set fixed by its own time (frozen neighbours
    and those whose key (tau, index) precedes the node's): the FP64 convergence check of a field solved in
    lower precision.  Equals tau, with the solve's records, at the causal fixed point."""
    frozen = np.ascontiguousarray(frozen, np.uint8).reshape(-1)
    tin = np.ascontiguousarray(tau, np.float64).reshape(-1)
    tout = np.empty_like(tin)
    rec = np.empty(tin.size, np.int16)
    lib().om_F_check_all(C.byref(M.c), _ptr(frozen, C.c_uint8), _ptr(tin, C.c_double), _ptr(tout, C.c_double),
                         _ptr(rec, C.c_int16))
    return tout.reshape(M.ny, M.nx), rec.reshape(M.ny, M.nx)


def ops_of_F_all(M: OMedium, frozen, tau):
    """Operations (the count defined in the C file) of one evaluation of F at every non-frozen node of a
    solved field, and the number of those nodes."""
    L = lib()
    L.om_reset_counters()
    F_all(M, frozen, tau)
    n = int(np.count_nonzero(np.asarray(frozen).reshape(-1) == 0))
    ops = int(L.om_counter(2))
    L.om_reset_counters()
    return ops, n


def jacobi(M: OMedium, frozen, tau0, max_iter=100000):
    frozen = np.ascontiguousarray(frozen, np.uint8).reshape(-1)
    tau = np.ascontiguousarray(tau0, np.float64).reshape(-1).copy()
    rec = np.empty(tau.size, np.int16)
    it = lib().om_jacobi(C.byref(M.c), _ptr(frozen, C.c_uint8), _ptr(tau, C.c_double), _ptr(rec, C.c_int16),
                         int(max_iter))
    return tau.reshape(M.ny, M.nx), rec.reshape(M.ny, M.nx), it


def stencil_value(M: OMedium, tau, i, j, row):
    t = np.ascontiguousarray(tau, np.float64).reshape(-1)
    return lib().om_stencil_value(C.byref(M.c), _ptr(t, C.c_double), int(i), int(j), int(row))


def solve_field(M: OMedium, si, sj, r0=2):
    """Convenience: simple-mode source initialisation followed by the heap FMM."""
    frozen, tau0 = init_radius(M, si, sj, r0)
    tau, rec, stats = fmm(M, frozen, tau0)
    return tau, rec, stats, frozen.reshape(M.ny, M.nx)


def trace_ray(M: OMedium, tau, start, target, plane_step=4, halfwidth=8, stop_radius=1.6, max_pts=None, family=-1):
    """Fermat plane-walk ray from `start` to `target` (the source of `tau`), grid units.  family -1: the
    plane set most perpendicular to the ray at every step; 0..3: one fixed set (x = c, y = c, x - y = c,
    x + y = c), Sec. 5.1."""
    if max_pts is None:
        max_pts = 4 * (M.nx + M.ny) + 2
    t = np.ascontiguousarray(tau, np.float64).reshape(-1)
    pts = np.zeros(2 * max_pts, np.float64)
    n = C.c_int(0)
    o = RayOpts(int(plane_step), int(halfwidth), float(stop_radius), int(max_pts), int(family))
    st = lib().om_trace_ray(C.byref(M.c), _ptr(t, C.c_double), float(start[0]), float(start[1]), float(target[0]),
                            float(target[1]), C.byref(o), _ptr(pts, C.c_double), C.byref(n))
    return pts[:2 * n.value].reshape(-1, 2).copy(), st


def path_time(M: OMedium, pts) -> float:
    p = np.ascontiguousarray(pts, np.float64).reshape(-1)
    return lib().om_path_time(C.byref(M.c), _ptr(p, C.c_double), int(p.size // 2))


def ray_gradient(M: OMedium, pts, region_of_node, nregions, eps=1e-6):
    """Gradient of the time along the fixed path `pts` with respect to the region orientations: for every
    region, the central difference of the path time (Sec. 5.1 integration) with that region's orientation
    moved by +-eps.  region_of_node: region index of every node (row-major)."""
    reg = np.asarray(region_of_node).reshape(-1)
    g = np.zeros(nregions)
    for r in np.unique(reg):
        tp, tm = M.theta.copy(), M.theta.copy()
        tp[reg == r] += eps
        tm[reg == r] -= eps
        Mp = OMedium(M.nx, M.ny, M.h, M.mat_id, tp, M.mats, M.group_model, M.vtable, M.wave_mode)
        Mm = OMedium(M.nx, M.ny, M.h, M.mat_id, tm, M.mats, M.group_model, M.vtable, M.wave_mode)
        g[r] = (path_time(Mp, pts) - path_time(Mm, pts)) / (2 * eps)
    return g


def trace_ray_best_family(M: OMedium, tau, start, target, **kw):
    """The fastest of the four fixed-family rays (ties to the lower family).  Returns (pts, status, family)."""
    best = None
    for fam in range(4):
        pts, st = trace_ray(M, tau, start, target, family=fam, **kw)
        if st != 0:
            continue
        t = path_time(M, pts)
        if best is None or t < best[0]:
            best = (t, pts, st, fam)
    if best is None:
        return None, 1, -1
    return best[1], best[2], best[3]


def adjoint(M: OMedium, frozen, tau, rec, order, seeds, src, region, nregions, grad=None):
    """Reverse-mode gradient: grad[r] += dL/dtheta_r given seeds[node] = dL/dtau."""
    fz = np.ascontiguousarray(frozen, np.uint8).reshape(-1)
    t = np.ascontiguousarray(tau, np.float64).reshape(-1)
    rc = np.ascontiguousarray(rec, np.int16).reshape(-1)
    od = np.ascontiguousarray(order, np.int32).reshape(-1)
    sd = np.ascontiguousarray(seeds, np.float64).reshape(-1)
    rg = np.ascontiguousarray(region, np.int32).reshape(-1)
    g = np.zeros(nregions, np.float64) if grad is None else grad
    lib().om_adjoint(C.byref(M.c), _ptr(fz, C.c_uint8), _ptr(t, C.c_double), _ptr(rc, C.c_int16),
                     _ptr(od, C.c_int32), _ptr(sd, C.c_double), int(src[0]), int(src[1]), _ptr(rg, C.c_int32),
                     int(nregions), _ptr(g, C.c_double))
    return g


def misfit_and_gradient(wl, sample, theta, t_obs, r0=2, group_model=0, wave_mode=QP):
    """L = sum over sources and receivers of (T - T_obs)^2 and dL/dtheta (oracle), for one sample."""
    s = wl.samples[sample]
    mats = [mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, theta, wl.region_material, mats, group_model,
                             wave_mode=wave_mode)
    region = np.asarray(s.region_map, np.int32).reshape(-1)
    L = 0.0
    grad = np.zeros(len(theta), np.float64)
    T = np.zeros((len(s.src), len(s.rec)))
    for k, (si, sj) in enumerate(s.src):
        fr, t0 = init_radius(M, si, sj, r0)
        tau, rec, st, order = fmm(M, fr, t0, with_order=True)
        tr = tau[s.rec[:, 1], s.rec[:, 0]]
        T[k] = tr
        res = tr - t_obs[k]
        L += float(np.sum(res ** 2))
        seeds = np.zeros(s.nx * s.ny)
        np.add.at(seeds, s.rec[:, 1] * s.nx + s.rec[:, 0], 2.0 * res)
        adjoint(M, fr, tau, rec, order, seeds, (si, sj), region, len(theta), grad)
    return L, grad, T
