"""Failure paths of the C ABI, each made to fire on purpose with a host-visible, bounded cause.

Nothing here faults or hangs the GPU: the round caps and point caps are plain counters checked by the
kernels, and the bad inputs are refused on the host before anything is launched.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOT_CONVERGED, RAY_INCOMPLETE, INVALID_ARG, NONPHYSICAL = 6, 7, 1, 2


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


@pytest.mark.parametrize("sweep", [1, 2, 3])
def test_round_cap_reports_not_converged(api, sweep):
    """A front band far narrower than a cell makes the sweep take about one round per node, far beyond a cap
    of (nx + ny) rounds: every schedule must report it, also when the cap falls on a chunk boundary."""
    wl = W.weld_single(n=64, h=0.5e-3, rg=4, seed=5, nsrc=2, nrec=2)
    P = api.Plan(wl, precision="fp32", sweep=sweep, band_cells=1e-6, max_rounds=1)
    th = P.theta_tensor()
    P.solve(th)
    assert P.status() == NOT_CONVERGED
    assert P.status() == 0  # the status word is cleared once read
    Pok = api.Plan(wl, precision="fp32", sweep=sweep)
    Pok.solve(th)
    assert Pok.status() == 0


def test_round_cap_in_the_hierarchy(api):
    wl = W.weld_single(n=64, h=0.5e-3, rg=4, seed=5, nsrc=1, nrec=2)
    P = api.Plan(wl, precision="fp32", init_mode=1, band_cells=1e-6, max_rounds=1)
    P.solve(P.theta_tensor())
    assert P.status() == NOT_CONVERGED


def test_ray_point_cap(api):
    wl = W.weld_single(n=64, h=0.5e-3, rg=4, seed=5, nsrc=2, nrec=3)
    P = api.Plan(wl, precision="fp32", max_ray_points=3)
    th = P.theta_tensor()
    times, _ = P.solve(th)
    assert P.status() == 0
    pts, npts, rt, st = P.trace_rays(th, times)
    assert P.status() == RAY_INCOMPLETE
    st = st.cpu().numpy()
    assert (st == 1).all() and (npts.cpu().numpy() <= 3).all()


def _plan_error(api, wl, **opts):
    from paper_2302_10988_gb300 import binding as B
    with pytest.raises(B.AlfError) as e:
        api.Plan(wl, precision="fp32", **opts)
    return e.value.code


def test_nonphysical_materials_refused(api):
    GPA = W.GPA
    cases = {
        "nan c22": W.ti_voigt(np.nan, 216 * GPA, 145 * GPA, 129 * GPA),
        "c22 < 0 (qP lambda < 0 along the axis)": W.ti_voigt(-234 * GPA, 216 * GPA, 145 * GPA, 129 * GPA),
        "c44 = 0": W.ti_voigt(234 * GPA, 216 * GPA, 145 * GPA, 0.0),
        "c22 c33 < c23^2 (not positive definite)": W.ti_voigt(234 * GPA, 216 * GPA, 300 * GPA, 129 * GPA),
    }
    for name, c6 in cases.items():
        wl = W.homogeneous_ti()
        wl.materials[0] = (c6, 8100.0)
        assert _plan_error(api, wl) == NONPHYSICAL, name
    wl = W.homogeneous_ti()
    wl.materials[0] = (wl.materials[0][0], np.inf)
    assert _plan_error(api, wl) == NONPHYSICAL


def test_bad_ids_and_sizes_refused(api):
    wl = W.weld_single(n=32, h=0.5e-3, rg=2, seed=1, nsrc=1, nrec=1)
    wl.samples[0].region_map[3, 4] = wl.nregions
    assert _plan_error(api, wl) == INVALID_ARG
    wl = W.weld_single(n=32, h=0.5e-3, rg=2, seed=1, nsrc=1, nrec=1)
    wl.region_material[1] = 7
    assert _plan_error(api, wl) == INVALID_ARG
    wl = W.weld_single(n=32, h=0.5e-3, rg=2, seed=1, nsrc=1, nrec=1)
    assert _plan_error(api, wl, max_rounds=0) == INVALID_ARG
    assert _plan_error(api, wl, max_ray_points=1) == INVALID_ARG
    assert _plan_error(api, wl, init_radius=9) == INVALID_ARG


def test_null_pointers_refused(api):
    from paper_2302_10988_gb300 import binding as B
    wl = W.weld_single(n=32, h=0.5e-3, rg=2, seed=1, nsrc=1, nrec=2)
    P = api.Plan(wl, precision="fp32", keep_records=1)
    th = P.theta_tensor()
    times = P.new_times()
    rec = P.new_records()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = B.load()
    vp = C.c_void_p
    assert L.alf_solve(P.plan, None, vp(times.data_ptr()), None, None, st) == INVALID_ARG
    assert L.alf_solve(P.plan, vp(th.data_ptr()), None, None, None, st) == INVALID_ARG
    assert L.alf_solve(None, vp(th.data_ptr()), vp(times.data_ptr()), None, None, st) == INVALID_ARG
    assert L.alf_check64(P.plan, vp(th.data_ptr()), vp(times.data_ptr()), None, None, None, st) == INVALID_ARG
    assert L.alf_trace_rays(P.plan, vp(th.data_ptr()), vp(times.data_ptr()), None, None, None, None,
                            st) == INVALID_ARG
    assert L.alf_backward(P.plan, vp(th.data_ptr()), vp(times.data_ptr()), None, None, None, st) == INVALID_ARG
    assert L.alf_plan_create(P.ctx, None, None, None) == INVALID_ARG
    # nothing was enqueued by the refused calls: a normal solve still succeeds
    P.solve(th, times=times, records=rec)
    assert P.status() == 0
