"""The allocation-free single-field solve gives the same field as alf_solve and as the FP64 oracle.

alf_solve_field_noalloc is for callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or cudaMalloc's device-wide
synchronisation is not allowed where they run): it keeps its workspace in a
fixed device array inside the library.  Every call shares that array, so the
test also checks that a smaller call after larger ones is unaffected by what
they left there.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests.gpu_helpers import oracle_field, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(wl, dev):
    s = wl.samples[0]
    rmap = torch.from_numpy(np.ascontiguousarray(s.region_map.astype(np.uint16)).view(np.int16)).to(dev)
    rmat = torch.from_numpy(np.ascontiguousarray(wl.region_material.astype(np.uint16)).view(np.int16)).to(dev)
    theta = torch.from_numpy(np.ascontiguousarray(s.region_theta, np.float64)).to(dev)
    return rmap, rmat, theta


def _noalloc(B, api, wl, si, sj, r0, max_rounds=0, rmap=None):
    dev = torch.device("cuda", 0)
    s = wl.samples[0]
    m, rmat, theta = _inputs(wl, dev)
    rmap = m if rmap is None else rmap
    mats = (B.alf_material * len(wl.materials))(*[api._material(c6, rho) for c6, rho in wl.materials])
    out = torch.full((s.ny * s.nx,), float("nan"), dtype=torch.float32, device=dev)
    code, msg = B.alf_solve_field_noalloc(0, mats, len(wl.materials), C.c_void_p(rmat.data_ptr()), wl.nregions,
                                          C.c_void_p(theta.data_ptr()), C.c_void_p(rmap.data_ptr()), s.nx, s.ny, s.h,
                                          si, sj, r0, B.ALF_GROUP_PAPER, C.c_void_p(out.data_ptr()),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream), max_rounds)
    torch.cuda.synchronize()
    return code, msg, out.view(s.ny, s.nx).double().cpu().numpy()


def test_noalloc_matches_solve_and_oracle(oracle):
    from paper_2302_10988_gb300 import api, binding as B, build
    build.build()
    wl = W.weld_single(n=200, h=0.5e-3, rg=8, seed=21, nsrc=1, nrec=1)
    s = wl.samples[0]
    P = api.Plan(wl, precision="fp32")
    th = P.theta_tensor()
    t_ref, _ = P.solve(th)
    assert P.status() == 0
    ref = P.field(t_ref, 0).double().cpu().numpy()
    tau = oracle_field(oracle, wl, 0, 0)[0]
    si, sj = (int(v) for v in s.src[0])
    for call in range(2):
        code, msg, g = _noalloc(B, api, wl, si, sj, 2)
        assert code == 0, msg
        assert np.isfinite(g).all()
        assert rel_err(g, ref).max() < 1e-4, (call, rel_err(g, ref).max())
        assert rel_err(g, tau).max() < 1e-4, (call, rel_err(g, tau).max())
    # a smaller grid after the larger calls, a corner source and no frozen box: nothing the earlier calls
    # left in the shared array (bitmap tail, lists, counters, frozen box) may change the field
    small = W.weld_single(n=80, h=0.5e-3, rg=4, seed=22, nsrc=1, nrec=1)
    sm = small.samples[0]
    sm.nx, sm.ny = 64, 80
    sm.region_map = np.ascontiguousarray(sm.region_map[:, 8:72])
    sm.src[:] = [[63, 79]]
    for r0 in (0, 3):
        code, msg, g = _noalloc(B, api, small, 63, 79, r0)
        assert code == 0, msg
        Ps = api.Plan(small, precision="fp32", init_radius=r0)
        ts, _ = Ps.solve(Ps.theta_tensor())
        assert Ps.status() == 0
        assert rel_err(g, Ps.field(ts, 0).double().cpu().numpy()).max() < 1e-4
        tau_s = oracle_field(oracle, small, 0, 0, r0=r0)[0]
        assert rel_err(g, tau_s).max() < 1e-4, (r0, rel_err(g, tau_s).max())


def test_noalloc_rejects_oversize():
    from paper_2302_10988_gb300 import api, binding as B, build
    build.build()
    wl = W.homogeneous_ti()
    mats = (B.alf_material * 1)(api._material(*wl.materials[0]))
    code, msg = B.alf_solve_field_noalloc(0, mats, 1, C.c_void_p(1), 1, C.c_void_p(1), C.c_void_p(1), 1024, 1024,
                                          1e-3, 0, 0, 2, 0, C.c_void_p(1), None)
    assert code == 1 and "exceeds the limit" in msg
    code, msg = B.alf_solve_field_noalloc(0, mats, 1, None, 1, C.c_void_p(1), C.c_void_p(1), 64, 64, 1e-3, 0, 0, 2,
                                          0, C.c_void_p(1), None)
    assert code == 1 and "null" in msg


def test_noalloc_checks_ids_and_round_cap():
    """A region id outside the region table is refused before any kernel indexes with it, and a sweep stopped
    by its round cap reports ALF_ERR_NOT_CONVERGED instead of returning a partial field as a success."""
    from paper_2302_10988_gb300 import api, binding as B, build
    build.build()
    wl = W.weld_single(n=64, h=0.5e-3, rg=4, seed=3, nsrc=1, nrec=1)
    dev = torch.device("cuda", 0)
    bad = wl.samples[0].region_map.astype(np.uint16).copy()
    bad[40, 7] = wl.nregions
    rbad = torch.from_numpy(bad.view(np.int16)).to(dev)
    code, msg, _ = _noalloc(B, api, wl, 32, 0, 2, rmap=rbad)
    assert code == 1 and "region id" in msg
    code, msg, _ = _noalloc(B, api, wl, 32, 0, 2, max_rounds=1)
    assert code == 6, msg
    code, msg, g = _noalloc(B, api, wl, 32, 0, 2)
    assert code == 0 and np.isfinite(g).all(), msg
