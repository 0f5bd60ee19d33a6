"""Pin of the oracle's discrete adjoint: central finite differences of the whole oracle solve.

Three geometries, so that every branch of the adjoint carries weight:
 * sources on the bottom edge, in the isotropic parent steel: the stencil branch alone (the parent
   region has no orientation dependence, so its gradient is exactly zero);
 * sources inside weld grains: the frozen nodes around each source take straight-ray times that depend on
   the orientation of the source's grain, so that grain's gradient has a large frozen-node share;
 * the same without a frozen box (init radius 0 and 1): nodes next to the source have no usable stencil
   and are finalised by the straight-ray fallback, whose orientation derivative then enters the gradient.
"""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W


def _records(oracle, wl, theta, r0):
    s = wl.samples[0]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, theta, wl.region_material, mats)
    out, fallback = [], 0
    for si, sj in s.src:
        fr, t0 = oracle.init_radius(M, si, sj, r0)
        tau, rec, st = oracle.fmm(M, fr, t0)
        out.append(rec.copy())
        fallback += st["fallback"]
    return np.array(out), fallback


def _fd_check(oracle, wl, r0, seed=1):
    s = wl.samples[0]
    rng = np.random.default_rng(seed)
    _, _, t_true = oracle.misfit_and_gradient(wl, 0, s.region_theta, np.zeros((len(s.src), len(s.rec))), r0=r0)
    t_obs = t_true + rng.normal(0.0, 10e-9, t_true.shape)
    theta = s.region_theta + np.r_[0.0, rng.normal(0.0, 0.2, len(s.region_theta) - 1)]
    L, g, _ = oracle.misfit_and_gradient(wl, 0, theta, t_obs, r0=r0)
    checked = []
    for r in range(1, len(theta)):
        e = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp[r] += e
        tm[r] -= e
        if (_records(oracle, wl, tp, r0)[0] != _records(oracle, wl, tm, r0)[0]).any():
            continue  # a stencil choice flips inside the step: the misfit is not differentiable there
        fd = (oracle.misfit_and_gradient(wl, 0, tp, t_obs, r0=r0)[0]
              - oracle.misfit_and_gradient(wl, 0, tm, t_obs, r0=r0)[0]) / (2 * e)
        assert abs(g[r] - fd) <= 1e-4 * abs(fd) + 1e-20, (r, g[r], fd)
        checked.append(r)
    return g, theta, checked


def test_adjoint_matches_finite_differences(oracle):
    wl = W.weld_single(n=40, h=0.5e-3, rg=3, seed=5, nsrc=3, nrec=6)
    g, _, checked = _fd_check(oracle, wl, 2)
    assert len(checked) >= 4
    assert g[0] == 0.0  # the isotropic parent region has no orientation dependence


def _inside_sources(seed):
    """Weld of 3 x 3 grains (nodes 8..31 of 40), sources inside grains 5 (centre) and 7, receivers on top."""
    wl = W.weld_single(n=40, h=0.5e-3, rg=3, seed=seed, nsrc=2, nrec=6)
    wl.samples[0].src[:] = [[20, 20], [12, 28]]
    return wl


def test_adjoint_source_orientation_branch(oracle):
    """Sources inside grains: the grains holding them carry the frozen nodes' orientation derivative."""
    wl = _inside_sources(seed=5)
    rm = wl.samples[0].region_map
    src_regions = {int(rm[sj, si]) for si, sj in wl.samples[0].src}
    assert 0 not in src_regions
    g, theta, checked = _fd_check(oracle, wl, 2)
    assert src_regions <= set(checked), (src_regions, checked)
    assert all(g[r] != 0.0 for r in src_regions)


@pytest.mark.parametrize("r0", [0, 1])
def test_adjoint_fallback_branch(oracle, r0):
    """Without a frozen box the nodes around each source are finalised by the straight-ray fallback."""
    wl = _inside_sources(seed=5)
    _, fallback = _records(oracle, wl, wl.samples[0].region_theta, r0)
    assert fallback > 0
    rm = wl.samples[0].region_map
    src_regions = {int(rm[sj, si]) for si, sj in wl.samples[0].src}
    g, theta, checked = _fd_check(oracle, wl, r0, seed=2)
    assert src_regions <= set(checked), (src_regions, checked)
    assert len(checked) >= 4
