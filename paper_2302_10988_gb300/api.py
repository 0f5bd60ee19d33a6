"""torch-facing wrapper of the C ABI: a plan over a workload, device buffers as tensors.

All computation happens in libalifmm.so; this module only converts a
``workloads.Workload`` into the C geometry, owns torch output tensors and
passes their device pointers and the current CUDA stream to the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import binding as B

_ctx_cache = {}


def context(device: int = 0):
    """One library context per CUDA device and process."""
    if device not in _ctx_cache:
        _ctx_cache[device] = B.alf_create(device)
    return _ctx_cache[device]


def _material(c6, rho) -> B.alf_material:
    m = B.alf_material()
    for a in range(6):
        for b in range(6):
            m.c[a][b] = float(c6[a][b])
    m.rho = float(rho)
    return m


PRECISIONS = {"fp64": B.ALF_FP64, "fp32": B.ALF_FP32}
GROUP = {"paper": B.ALF_GROUP_PAPER, "exact": B.ALF_GROUP_EXACT}


class Plan:
    """A batch of fields (samples x sources) of one workload, ready to solve.

    Keyword options map to ``alf_options`` fields (precision "fp32"/"fp64",
    group "paper"/"exact", init_mode, init_radius, n_levels, level_density, level_radius,
    plane_step, ray_halfwidth, ray_family, stop_radius, max_ray_points, max_rounds, sweep, keep_records,
    band_cells, use_graph, time_kernels, velocity_table, cta_threads, cta_cluster, subgrid); array fields take a
    sequence of 4 ints.  With subgrid s > 1 every field, record and ray lives on the grid refined s times
    (``shapes`` are the fine grids; the original nodes are every s-th fine node)."""

    def __init__(self, wl, precision="fp32", group="paper", device=0, **opts):
        self.wl = wl
        self.device = device
        self.ctx = context(device)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        o = B.alf_default_options()
        o.precision = PRECISIONS[precision]
        o.group_model = GROUP[group]
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            if k in ("level_density", "level_radius"):
                v = tuple(v) + (0,) * (4 - len(v))
            setattr(o, k, v)
        S = len(wl.samples[0].src)
        Rr = len(wl.samples[0].rec)
        for s in wl.samples:
            if len(s.src) != S or len(s.rec) != Rr:
                raise ValueError("every sample needs the same number of sources and receivers")
        self.nsamples, self.nsrc, self.nrec = len(wl.samples), S, Rr
        self.nregions = wl.nregions
        keep = []
        nx = np.array([s.nx for s in wl.samples], np.int32)
        ny = np.array([s.ny for s in wl.samples], np.int32)
        h = np.array([s.h for s in wl.samples], np.float64)
        # 16-bit region ids while they fit, else 32-bit ones (per-node orientation maps)
        wide = wl.nregions > 65536 or any(s.region_map.dtype.itemsize > 2 for s in wl.samples)
        rmap = np.ascontiguousarray(np.concatenate([s.region_map.astype(np.uint32 if wide else np.uint16).ravel()
                                                    for s in wl.samples]))
        wide_mat = len(wl.materials) > 65536
        rmat = np.ascontiguousarray(wl.region_material.astype(np.uint32 if wide_mat else np.uint16))
        mats = (B.alf_material * len(wl.materials))(*[_material(c6, rho) for c6, rho in wl.materials])
        src = np.ascontiguousarray(np.stack([s.src for s in wl.samples]).astype(np.int32))
        rec = np.ascontiguousarray(np.stack([s.rec for s in wl.samples]).astype(np.int32)) if Rr else \
            np.zeros((len(wl.samples), 0, 2), np.int32)
        keep += [nx, ny, h, rmap, rmat, mats, src, rec]

        def ptr(a, t):
            return a.ctypes.data_as(C.POINTER(t))
        g = B.alf_geometry(len(wl.samples), ptr(nx, C.c_int32), ptr(ny, C.c_int32), ptr(h, C.c_double),
                           None if wide else ptr(rmap, C.c_uint16), wl.nregions,
                           None if wide_mat else ptr(rmat, C.c_uint16), len(wl.materials), mats, S,
                           ptr(src, C.c_int32), Rr, ptr(rec, C.c_int32), ptr(rmap, C.c_uint32) if wide else None,
                           ptr(rmat, C.c_uint32) if wide_mat else None)
        self.plan = B.alf_plan_create(self.ctx, g, o)
        self.options = B.alf_plan_options(self.plan)
        self.nfields = B.alf_plan_nfields(self.plan)
        self.offsets = [B.alf_plan_field_offset(self.plan, f) for f in range(self.nfields + 1)]
        self.total_nodes = self.offsets[-1]
        sg = max(1, int(self.options.subgrid))
        self.subgrid = sg
        self.shapes = [((s.ny - 1) * sg + 1, (s.nx - 1) * sg + 1) for s in wl.samples for _ in range(S)]

    def __del__(self):
        try:
            if getattr(self, "plan", None):
                B.alf_plan_destroy(self.plan)
                self.plan = None
        except Exception:
            pass

    # ------------------------------------------------------------------ buffers
    def _dev(self):
        return torch.device("cuda", self.device)

    def new_times(self):
        return torch.empty(self.total_nodes, dtype=self.dtype, device=self._dev())

    def new_rec_times(self):
        return torch.empty((self.nsamples, self.nsrc, self.nrec), dtype=self.dtype, device=self._dev())

    def new_records(self):
        return torch.empty(self.total_nodes, dtype=torch.uint8, device=self._dev())

    def theta_tensor(self, theta=None):
        if theta is None:
            theta = np.stack([s.region_theta for s in self.wl.samples])
        t = torch.as_tensor(np.asarray(theta, np.float64)).reshape(self.nsamples, self.nregions)
        return t.to(self._dev()).contiguous()

    def field(self, times, f):
        ny, nx = self.shapes[f]
        return times[self.offsets[f]:self.offsets[f] + ny * nx].view(ny, nx)

    @staticmethod
    def _stream():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    # ------------------------------------------------------------------ calls
    def solve(self, theta, times=None, rec_times=None, records=None, with_receivers=True):
        times = self.new_times() if times is None else times
        if with_receivers and rec_times is None and self.nrec:
            rec_times = self.new_rec_times()
        assert theta.dtype == torch.float64 and theta.is_cuda and theta.is_contiguous()
        B.alf_solve(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                    C.c_void_p(rec_times.data_ptr()) if rec_times is not None else None,
                    C.c_void_p(records.data_ptr()) if records is not None else None, self._stream())
        return times, rec_times

    def solve_check64(self, theta, times=None, rec_times=None, records=None, with_receivers=True):
        """The solve and the FP64 check of its fields in one call: (times, rec_times, max_rel, flips)."""
        times = self.new_times() if times is None else times
        if with_receivers and rec_times is None and self.nrec:
            rec_times = self.new_rec_times()
        assert theta.dtype == torch.float64 and theta.is_cuda and theta.is_contiguous()
        max_rel = torch.empty(self.nfields, dtype=torch.float64, device=self._dev())
        flips = torch.empty(self.nfields, dtype=torch.int32, device=self._dev())
        B.alf_solve_check64(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                            C.c_void_p(rec_times.data_ptr()) if rec_times is not None else None,
                            C.c_void_p(records.data_ptr()) if records is not None else None,
                            C.c_void_p(max_rel.data_ptr()), C.c_void_p(flips.data_ptr()), self._stream())
        return times, rec_times, max_rel, flips

    def check64(self, theta, times, records=None):
        max_rel = torch.empty(self.nfields, dtype=torch.float64, device=self._dev())
        flips = torch.empty(self.nfields, dtype=torch.int32, device=self._dev())
        B.alf_check64(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                      C.c_void_p(records.data_ptr()) if records is not None else None,
                      C.c_void_p(max_rel.data_ptr()), C.c_void_p(flips.data_ptr()), self._stream())
        return max_rel, flips

    def check64_nodes(self, theta, times, records=None):
        """The FP64 check with every node's FP64 value and record: (check_times float64, check_records uint8,
        max_rel, flips)."""
        max_rel = torch.empty(self.nfields, dtype=torch.float64, device=self._dev())
        flips = torch.empty(self.nfields, dtype=torch.int32, device=self._dev())
        ct = torch.empty(self.total_nodes, dtype=torch.float64, device=self._dev())
        cr = torch.empty(self.total_nodes, dtype=torch.uint8, device=self._dev())
        B.alf_check64_nodes(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                            C.c_void_p(records.data_ptr()) if records is not None else None,
                            C.c_void_p(ct.data_ptr()), C.c_void_p(cr.data_ptr()), C.c_void_p(max_rel.data_ptr()),
                            C.c_void_p(flips.data_ptr()), self._stream())
        return ct, cr, max_rel, flips

    def trace_rays(self, theta, times):
        P = self.options.max_ray_points
        shape = (self.nsamples, self.nsrc, self.nrec)
        pts = torch.empty(shape + (P, 2), dtype=self.dtype, device=self._dev())
        npts = torch.empty(shape, dtype=torch.int32, device=self._dev())
        rt = torch.empty(shape, dtype=self.dtype, device=self._dev())
        st = torch.empty(shape, dtype=torch.int32, device=self._dev())
        B.alf_trace_rays(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                         C.c_void_p(pts.data_ptr()), C.c_void_p(npts.data_ptr()), C.c_void_p(rt.data_ptr()),
                         C.c_void_p(st.data_ptr()), self._stream())
        return pts, npts, rt, st

    def pack_rays(self, pts, npts, packed=None, offsets=None):
        """The traced paths back to back: (packed [capacity, 2] in the plan's dtype, offsets [nrays + 1] int64);
        ray r's points are packed[offsets[r]:offsets[r + 1]], offsets[-1] the total."""
        nrays = self.nsamples * self.nsrc * self.nrec
        if packed is None:
            packed = torch.empty((nrays * self.options.max_ray_points, 2), dtype=self.dtype, device=self._dev())
        if offsets is None:
            offsets = torch.empty(nrays + 1, dtype=torch.int64, device=self._dev())
        B.alf_pack_rays(self.ctx, self.plan, C.c_void_p(pts.data_ptr()), C.c_void_p(npts.data_ptr()),
                        C.c_void_p(packed.data_ptr()), C.c_void_p(offsets.data_ptr()), self._stream())
        return packed, offsets

    def ray_gradient(self, theta, pts, npts, dL_dray):
        """dL/dtheta [nsamples, nregions] (float64) from dL/dT of every ray, its path (from trace_rays) held
        fixed."""
        grad = torch.empty((self.nsamples, self.nregions), dtype=torch.float64, device=self._dev())
        g = dL_dray.to(self.dtype).contiguous()
        B.alf_ray_gradient(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(pts.data_ptr()),
                           C.c_void_p(npts.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(grad.data_ptr()),
                           self._stream())
        return grad

    def backward(self, theta, times, records, dL_drec):
        """dL/dtheta [nsamples, nregions] (float64) from dL/dT at the receivers (plan needs keep_records=1)."""
        grad = torch.empty((self.nsamples, self.nregions), dtype=torch.float64, device=self._dev())
        g = dL_drec.to(self.dtype).contiguous()
        B.alf_backward(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                       C.c_void_p(records.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(grad.data_ptr()),
                       self._stream())
        return grad

    def status(self) -> int:
        return B.alf_sync_status(self.plan, self._stream())

    def stats(self) -> dict:
        return B.alf_plan_stats(self.ctx, self.plan, self._stream())

    def autotune(self, theta, times=None, records=None):
        times = self.new_times() if times is None else times
        B.alf_plan_autotune(self.ctx, self.plan, C.c_void_p(theta.data_ptr()), C.c_void_p(times.data_ptr()),
                            C.c_void_p(records.data_ptr()) if records is not None else None, self._stream())
        self.options = B.alf_plan_options(self.plan)
        return self.options


MODES = {"qP": 0, "qSV": 1, "SH": 2}


def eval_velocity(c6, rho, angles, kind="phase", group="paper", precision="fp64", device=0, mode="qP"):
    """Device velocity model at angles (radians, relative to the material axis) -> numpy array; `mode` is the
    wave mode (qP, qSV, SH)."""
    ctx = context(device)
    a = torch.as_tensor(np.asarray(angles, np.float64), device=torch.device("cuda", device)).contiguous()
    out = torch.empty_like(a)
    k = 2 * MODES[mode] + (0 if kind == "phase" else 1)
    B.alf_eval_velocity(ctx, _material(c6, rho), k, GROUP[group], PRECISIONS[precision],
                        C.c_void_p(a.data_ptr()), C.c_void_p(out.data_ptr()), a.numel(),
                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return out.cpu().numpy()


class ReceiverTimes(torch.autograd.Function):
    """Receiver travel times T[b, s, r] as a differentiable function of the region orientations theta[b, R].

    forward: alf_solve (records kept); backward: alf_backward, the discrete adjoint of the solve.
    The plan must have been created with keep_records=1."""

    @staticmethod
    def forward(ctx, theta, plan):
        th = theta.detach().to(torch.float64).contiguous()
        times = plan.new_times()
        records = plan.new_records()
        _, rt = plan.solve(th, times=times, records=records)
        ctx.plan = plan
        ctx.save_for_backward(th, times, records)
        return rt

    @staticmethod
    def backward(ctx, grad_out):
        th, times, records = ctx.saved_tensors
        g = ctx.plan.backward(th, times, records, grad_out)
        return g.to(th.dtype), None
