"""Shear-wave modes on the GPU (alf_options.wave_mode: qSV and SH, Sec. 7 with the eigenvalues of Sec. 3.2)
against the oracle: the velocity model, fields and records, the FP64 check node by node, rays and the adjoint.

The media are the weld layout with grains of the weld steel (its qSV ray surface has cusps) or of a general
orthotropic material (its SH curve is an ellipse), in isotropic parent steel."""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests.gpu_helpers import record_mismatch, rel_err
from tests.test_oracle_shear import ORTHO

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
MODE = {"qSV": 1, "SH": 2}


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


def _weld(grain, n=80, rg=4, seed=3, nsrc=3, nrec=4):
    wl = W.weld_single(n=n, h=0.5e-3, rg=rg, seed=seed, nsrc=nsrc, nrec=nrec)
    wl.materials[0] = grain
    return wl


def _oracle(oracle, wl, k, mode, r0=2):
    s = wl.samples[0]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, s.region_theta, wl.region_material, mats,
                                    group_model=1, wave_mode=mode)
    fr, t0 = oracle.init_radius(M, *(int(v) for v in s.src[k]), r0)
    tau, rec, st = oracle.fmm(M, fr, t0)
    assert st["noncausal"] == 0
    return M, tau, rec, fr.reshape(tau.shape)


@pytest.mark.parametrize("mode", ["qSV", "SH"])
def test_shear_velocity_model_on_device(api, oracle, mode):
    ang = np.radians(np.linspace(-180, 180, 361))
    for c6, rho in (W.WELD_TI, ORTHO, W.PARENT_ISO):
        m = oracle.mat_from_voigt(c6, rho)
        v_o = np.array([oracle.mode_velocity(m, MODE[mode], a) for a in ang])
        tab = oracle.envelope_table(m, MODE[mode])
        g_o = np.array([oracle.lib().om_envelope_speed(tab.ctypes.data_as(oracle.C.POINTER(oracle.C.c_double)), a)
                        for a in ang])
        for prec, tv, tg in (("fp64", 1e-13, 1e-11), ("fp32", 2e-6, 2e-7)):
            v = api.eval_velocity(c6, rho, ang, "phase", precision=prec, mode=mode)
            g = api.eval_velocity(c6, rho, ang, "group", precision=prec, mode=mode)
            assert np.max(np.abs(v / v_o - 1)) < tv, (mode, prec)
            assert np.max(np.abs(g / g_o - 1)) < tg, (mode, prec)


@pytest.mark.parametrize("mode,grain", [("qSV", "weld"), ("qSV", "ortho"), ("SH", "ortho")])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_shear_fields_rays_and_check(api, oracle, mode, grain, precision, tol):
    wl = _weld(W.WELD_TI if grain == "weld" else ORTHO)
    P = api.Plan(wl, precision=precision, wave_mode=MODE[mode], group="exact", keep_records=1)
    th = P.theta_tensor()
    rec = P.new_records()
    times, rt = P.solve(th, records=rec)
    ct, cr, mr, fl = P.check64_nodes(th, times, rec)
    pts, npts, rtime, rst = P.trace_rays(th, times)
    assert P.status() == 0
    flips = 0
    for k in range(3):
        M, tau, orec, fr = _oracle(oracle, wl, k, MODE[mode])
        g = P.field(times, k).cpu().numpy()
        e = rel_err(g, tau).max()
        flips += record_mismatch(P.field(rec, k).cpu().numpy(), orec, fr)
        assert e < tol, (k, e)
        # the FP64 check of this field, node by node against the oracle's evaluation of it
        F_o, rc_o = oracle.F_check(M, fr.astype(np.uint8), g.astype(np.float64))
        F_g = P.field(ct, k).cpu().numpy()
        m = np.isfinite(F_o) & (F_o > 0)
        assert (np.abs(F_g - F_o)[m] / F_o[m]).max() < 1e-12
        if precision == "fp64":
            s = wl.samples[0]
            for q in range(4):
                o_pts, o_st = oracle.trace_ray(M, tau, s.rec[q], s.src[k])
                n = int(npts[0, k, q])
                assert o_st == 0 and int(rst[0, k, q]) == 0 and n == len(o_pts)
                assert np.abs(pts[0, k, q, :n].cpu().numpy() - o_pts).max() < 1e-7
                assert float(rtime[0, k, q]) == pytest.approx(oracle.path_time(M, o_pts), rel=1e-10)
    print(f"{mode} {grain} {precision}: record flips {flips}, FP64 check residual {mr.max().item():.2e}")
    if precision == "fp64":
        assert flips == 0
        assert mr.max().item() < 1e-12


@pytest.mark.parametrize("mode", ["qSV", "SH"])
def test_shear_adjoint(api, oracle, mode):
    """The adjoint gradient of the shear modes: the stencil partials of the mode's root, the envelope table's
    derivative at the fallback and frozen nodes."""
    wl, truth = W.weld_adjoint(nsamples=2, n=48, rg=3, nsrc=3, nrec=5)
    for w in (wl, truth):
        w.materials[0] = ORTHO
    _, _, t_true = oracle.misfit_and_gradient(truth, 0, truth.samples[0].region_theta, np.zeros((3, 5)),
                                              group_model=1, wave_mode=MODE[mode])
    t_obs = t_true + W.observation_noise(t_true.shape)
    P = api.Plan(wl, precision="fp64", keep_records=1, wave_mode=MODE[mode], group="exact")
    th = P.theta_tensor()
    rec = P.new_records()
    times, rt = P.solve(th, records=rec)
    g = P.backward(th, times, rec, 2.0 * (rt - torch.as_tensor(t_obs, device=rt.device)[None])).cpu().numpy()
    assert P.status() == 0
    for b in range(2):
        _, g_o, _ = oracle.misfit_and_gradient(wl, b, wl.samples[b].region_theta, t_obs, group_model=1,
                                               wave_mode=MODE[mode])
        err = np.abs(g[b] - g_o).max() / np.abs(g_o).max()
        print(f"{mode} adjoint sample {b}: {err:.2e}")
        assert err < 1e-5
