"""The allocation-free single-field solve gives the same field as alf_solve.

alf_solve_field_noalloc is for callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or cudaMalloc's device-wide
synchronisation is not allowed where they run): it keeps its workspace in a
fixed device array inside the library.  This file is collected last on
purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_solve_twice():
    from paper_2302_10988_gb300 import api, binding as B, build
    build.build()
    wl = W.weld_single(n=200, h=0.5e-3, rg=8, seed=21, nsrc=1, nrec=1)
    s = wl.samples[0]
    P = api.Plan(wl, precision="fp32")
    th = P.theta_tensor()
    t_ref, _ = P.solve(th)
    assert P.status() == 0
    ref = P.field(t_ref, 0).double().cpu().numpy()

    dev = torch.device("cuda", 0)
    rmap = torch.from_numpy(np.ascontiguousarray(s.region_map.astype(np.uint16)).view(np.int16)).to(dev)
    rmat = torch.from_numpy(np.ascontiguousarray(wl.region_material.astype(np.uint16)).view(np.int16)).to(dev)
    theta = torch.from_numpy(np.ascontiguousarray(s.region_theta, np.float64)).to(dev)
    mats = (B.alf_material * len(wl.materials))(*[api._material(c6, rho) for c6, rho in wl.materials])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    si, sj = (int(v) for v in s.src[0])
    for call in range(2):
        out = torch.full((s.ny * s.nx,), float("nan"), dtype=torch.float32, device=dev)
        code, msg = B.alf_solve_field_noalloc(0, mats, len(wl.materials), C.c_void_p(rmat.data_ptr()),
                                              wl.nregions, C.c_void_p(theta.data_ptr()), C.c_void_p(rmap.data_ptr()),
                                              s.nx, s.ny, s.h, si, sj, 2, B.ALF_GROUP_PAPER,
                                              C.c_void_p(out.data_ptr()), stream)
        assert code == 0, msg
        torch.cuda.synchronize()
        g = out.view(s.ny, s.nx).double().cpu().numpy()
        m = ref > 0
        rel = np.abs(g - ref)[m] / ref[m]
        assert np.isfinite(g).all()
        assert rel.max() < 1e-4, (call, rel.max())


def test_noalloc_rejects_oversize():
    from paper_2302_10988_gb300 import api, binding as B, build
    build.build()
    wl = W.homogeneous_ti()
    mats = (B.alf_material * 1)(api._material(*wl.materials[0]))
    code, msg = B.alf_solve_field_noalloc(0, mats, 1, C.c_void_p(1), 1, C.c_void_p(1), C.c_void_p(1), 1024, 1024,
                                          1e-3, 0, 0, 2, 0, C.c_void_p(1), None)
    assert code == 1 and "exceeds the limit" in msg
