"""The global sub-grid option (alf_options.subgrid, Sec. 4.5 and Table 2; rays on the refined grid, Sec. 5.1).

With sub-grid size s the plan refines every sample s times in each direction, each fine node taking the
region of the nearest original node.  The oracle side builds that refined medium here, by hand, from the
original one, and runs its own solve and ray tracer on it with the lengths scaled to fine cells; the GPU
plan receives the ORIGINAL geometry and the option.  Table 2's ALI-FMM (Christoffel) row is then reproduced
through the option for s = 1, 3 and 5.
"""
import os

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests.gpu_helpers import record_mismatch, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


def refine(wl, s):
    """The sub-grid medium of Sec. 4.5 built directly: fine node (i, j) takes the region of the original node
    nearest to (i / s, j / s); sources and receivers move to (i s, j s)."""
    out = []
    for smp in wl.samples:
        nxf, nyf = (smp.nx - 1) * s + 1, (smp.ny - 1) * s + 1
        oi = np.floor(np.arange(nxf) / s + 0.5).astype(int)
        oj = np.floor(np.arange(nyf) / s + 0.5).astype(int)
        rm = smp.region_map[np.ix_(oj, oi)].astype(np.uint16)
        out.append(W.Sample(nxf, nyf, smp.h / s, rm, smp.region_theta, smp.src * s, smp.rec * s))
    return W.Workload(wl.name + f" refined {s}", wl.materials, wl.region_material, out)


def _oracle(oracle, wl, b, k, r0):
    smp = wl.samples[b]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = oracle.OMedium.from_regions(smp.nx, smp.ny, smp.h, smp.region_map, smp.region_theta, wl.region_material,
                                    mats)
    fr, t0 = oracle.init_radius(M, *smp.src[k], r0)
    tau, rec, st = oracle.fmm(M, fr, t0)
    return M, tau, rec, fr.reshape(tau.shape)


@pytest.mark.parametrize("s", [3, 5])
def test_subgrid_fields_and_rays_match_oracle(api, oracle, s):
    wl = W.weld_single(n=24, h=0.5e-3, rg=3, seed=9, nsrc=2, nrec=3)
    P = api.Plan(wl, precision="fp64", subgrid=s, init_radius=1)
    assert P.options.subgrid == s and P.options.init_radius == 1 and P.options.plane_step == 4
    th = P.theta_tensor()
    rec = P.new_records()
    times, rt = P.solve(th, records=rec)
    pts, npts, rtime, rst = P.trace_rays(th, times)
    assert P.status() == 0
    fine = refine(wl, s)
    assert P.shapes[0] == (fine.samples[0].ny, fine.samples[0].nx)
    for k in range(2):
        M, tau, orec, fr = _oracle(oracle, fine, 0, k, r0=1 * s)
        g = P.field(times, k).cpu().numpy()
        assert rel_err(g, tau).max() < 1e-6
        assert record_mismatch(P.field(rec, k).cpu().numpy(), orec, fr) == 0
        r = fine.samples[0].rec
        assert np.allclose(rt[0, k].cpu().numpy(), tau[r[:, 1], r[:, 0]], rtol=1e-12, atol=0)
        for q in range(3):
            o_pts, o_st = oracle.trace_ray(M, tau, r[q], fine.samples[0].src[k], plane_step=4 * s,
                                           halfwidth=8 * s, stop_radius=1.6 * s)
            n = int(npts[0, k, q])
            assert o_st == 0 and int(rst[0, k, q]) == 0
            assert n == len(o_pts)
            assert np.abs(pts[0, k, q, :n].cpu().numpy() - o_pts).max() < 1e-7
            assert float(rtime[0, k, q]) == pytest.approx(oracle.path_time(M, o_pts), rel=1e-10)


def _table2(api, oracle, s):
    """Mean absolute relative error (%) at the original nodes of the 21 x 21 cubic-steel grid, source at the
    centre, orientation 0, against distance / exact group speed."""
    c6, rho = W.PAPER_CUBIC
    n = 21
    dens, rad = ((27, 9, 3), (1, 6, 13)) if s == 1 else ((9, 3), (2, 5))
    smp = W.Sample(n, n, 1e-3, np.zeros((n, n), np.uint16), np.array([0.0]), np.array([[10, 10]], np.int32),
                   np.array([[n - 1, n - 1]], np.int32))
    wl = W.Workload("table 2", [W.PAPER_CUBIC], np.array([0], np.uint16), [smp])
    P = api.Plan(wl, precision="fp64", init_mode=1, n_levels=len(dens), level_density=dens, level_radius=rad,
                 subgrid=s)
    times, _ = P.solve(P.theta_tensor())
    assert P.status() == 0
    sub = P.field(times, 0).cpu().numpy()[::s, ::s]
    assert sub.shape == (n, n)
    m = oracle.mat_from_voigt(c6, rho)
    jj, ii = np.mgrid[0:n, 0:n]
    d = np.hypot(ii - 10, jj - 10) * 1e-3
    V = np.array([oracle.group_exact(m, a)[1] for a in np.arctan2(jj - 10, ii - 10).ravel()]).reshape(n, n)
    T = d / np.where(d > 0, V, 1.0)
    return 100.0 * (np.abs(sub - T)[d > 0] / T[d > 0]).mean()


def test_table2_through_the_subgrid_option(api, oracle):
    """Sec. 4.5, Table 2 (ALI-FMM solving Christoffel): sub-grid sizes 1, 3 and 5 through the option, within
    +-10 % of the printed mean errors, and the error falls as s grows."""
    ref = {int(a): float(b) for a, b in (l.split() for l in open(os.path.join(GOLDEN, "table2_subgrid_errors.txt"))
                                         if l.strip() and not l.startswith("#"))}
    errs = {}
    for s in (1, 3, 5):
        errs[s] = _table2(api, oracle, s)
        print(f"Table 2 sub-grid {s} through the option: GPU {errs[s]:.3f} %, paper {ref[s]:.3f} %")
        assert abs(errs[s] / ref[s] - 1.0) < 0.10, (s, errs[s], ref[s])
    assert errs[5] < errs[3] < errs[1] * 1.1


def test_subgrid_option_validation(api):
    from paper_2302_10988_gb300 import binding as B
    wl = W.weld_single(n=24, h=0.5e-3, rg=3, seed=9, nsrc=1, nrec=1)
    for bad in (2, 23, -1):
        with pytest.raises(B.AlfError) as e:
            api.Plan(wl, precision="fp32", subgrid=bad)
        assert e.value.code == 1
