"""Pin of the oracle's discrete adjoint: central finite differences of the whole oracle solve."""
import numpy as np

from paper_2302_10988_gb300 import workloads as W


def _records(oracle, wl, theta):
    s = wl.samples[0]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, theta, wl.region_material, mats)
    out = []
    for si, sj in s.src:
        fr, t0 = oracle.init_radius(M, si, sj, 2)
        out.append(oracle.fmm(M, fr, t0)[1].copy())
    return np.array(out)


def test_adjoint_matches_finite_differences(oracle):
    wl = W.weld_single(n=40, h=0.5e-3, rg=3, seed=5, nsrc=3, nrec=6)
    s = wl.samples[0]
    rng = np.random.default_rng(1)
    _, _, t_true = oracle.misfit_and_gradient(wl, 0, s.region_theta, np.zeros((3, 6)))
    t_obs = t_true + rng.normal(0.0, 10e-9, t_true.shape)
    theta = s.region_theta + np.r_[0.0, rng.normal(0.0, 0.2, len(s.region_theta) - 1)]
    L, g, _ = oracle.misfit_and_gradient(wl, 0, theta, t_obs)
    checked = 0
    for r in range(1, len(theta)):
        e = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp[r] += e
        tm[r] -= e
        if (_records(oracle, wl, tp) != _records(oracle, wl, tm)).any():
            continue  # a stencil choice flips inside the step: the misfit is not differentiable there
        fd = (oracle.misfit_and_gradient(wl, 0, tp, t_obs)[0] - oracle.misfit_and_gradient(wl, 0, tm, t_obs)[0]) / (2 * e)
        assert abs(g[r] - fd) <= 1e-4 * abs(fd) + 1e-20, (r, g[r], fd)
        checked += 1
    assert checked >= 4
    assert g[0] == 0.0  # the isotropic parent region has no orientation dependence
