"""Pin of the oracle's straight-ray source initialisation (Sec. 4.4, radius mode).

Every node within Chebyshev distance r0 of the source is frozen with the straight-ray time
|x - x_s| / V_group(direction - theta_source), where the orientation is the SOURCE node's (the medium
around the source is taken as homogeneous) and V_group comes from the group model.  The medium here has
a different random orientation at every node, so taking any other node's orientation, another distance
scale or another direction convention fails.  The expected group speeds come from the eigen-solver
(tests/pins.py), not from the oracle.
"""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests import pins


def _medium(oracle, nx, ny, h, group_model, seed):
    rng = np.random.default_rng(seed)
    theta = rng.uniform(-np.pi / 2, np.pi / 2, nx * ny)
    mats = [oracle.mat_from_voigt(*W.WELD_TI)]
    return oracle.OMedium(nx, ny, h, np.zeros(nx * ny, np.int32), theta, mats, group_model), theta


@pytest.mark.parametrize("group_model", [0, 1])
@pytest.mark.parametrize("src,r0", [((10, 12), 2), ((0, 0), 3), ((23, 5), 1), ((7, 19), 0), ((12, 10), 4)])
def test_init_radius_straight_rays(oracle, group_model, src, r0):
    nx, ny, h = 24, 20, 0.7e-3
    M, theta = _medium(oracle, nx, ny, h, group_model, seed=17 + r0)
    si, sj = src
    fr, tau = oracle.init_radius(M, si, sj, r0)
    fr, tau = fr.reshape(ny, nx), tau.reshape(ny, nx)
    c6, rho = W.WELD_TI
    th_s = theta[sj * nx + si]
    jj, ii = np.mgrid[0:ny, 0:nx]
    box = (np.abs(ii - si) <= r0) & (np.abs(jj - sj) <= r0)
    assert np.array_equal(fr == 1, box)
    assert np.isinf(tau[~box]).all()
    assert tau[sj, si] == 0.0
    m = oracle.mat_from_voigt(c6, rho)
    for j, i in zip(*np.nonzero(box)):
        if (i, j) == (si, sj):
            continue
        di, dj = i - si, j - sj
        psi = np.arctan2(dj, di) - th_s
        dist = np.hypot(di, dj) * h
        V = pins.exact_group_speed(c6, rho, psi) if group_model else pins.paper_group_speed(c6, rho, psi)
        assert tau[j, i] == pytest.approx(dist / V, rel=1e-10), (i, j)
        # the geometry exactly: the same group model evaluated by the oracle's own (separately pinned) routine
        Vo = oracle.group_exact(m, psi)[1] if group_model else oracle.group_paper(m, psi)[1]
        assert tau[j, i] == pytest.approx(dist / Vo, rel=1e-14, abs=0), (i, j)
