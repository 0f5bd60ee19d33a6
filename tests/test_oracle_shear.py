"""Pins of the oracle's shear-wave modes (Sec. 7: the other eigenvalues of Sec. 3.2 give S-wave times).

qSV is the smaller in-plane eigenvalue of the Christoffel matrix, SH the out-of-plane one; their group
speeds for the source initialisation, the fallback and the rays are the envelope
1/V(psi) = max over theta of cos(theta - psi) / v(theta) (the Wulff construction: the eikonal's solution for a
point source in a homogeneous medium), which stays single valued where the qSV ray surface has cusps (it does
for both steels here), tabulated at 1/8 degree [R20].  Every expected value below comes
from the eigen-solver, a brute-force maximisation or a closed form, not from the oracle."""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests import pins

GPA = W.GPA
# a general orthotropic material whose SH curve is an ellipse (c55 != c66)
ORTHO = (lambda: (lambda C: (C, 8000.0))(np.array([[250, 110, 100, 0, 0, 0], [110, 230, 120, 0, 0, 0],
                                                   [100, 120, 200, 0, 0, 0], [0, 0, 0, 100, 0, 0],
                                                   [0, 0, 0, 0, 70, 0], [0, 0, 0, 0, 0, 90]], float) * GPA))()
MATS = {"weld_ti": W.WELD_TI, "paper_cubic": W.PAPER_CUBIC, "ortho": ORTHO}


def _modes(c6, rho, th):
    """(qSV, qP, SH) phase speeds from the eigen-solver: in-plane eigenvectors have no x component."""
    n = np.array([0.0, np.cos(th), np.sin(th)])
    w, V = np.linalg.eigh(pins.christoffel(c6, n))
    inplane = sorted(w[k] for k in range(3) if abs(V[0, k]) < 1e-9)
    sh = [w[k] for k in range(3) if abs(V[0, k]) > 1 - 1e-9]
    return np.sqrt(inplane[0] / rho), np.sqrt(inplane[1] / rho), np.sqrt(sh[0] / rho)


@pytest.mark.parametrize("name", list(MATS))
def test_mode_speeds_are_the_christoffel_eigenvalues(oracle, name):
    c6, rho = MATS[name]
    m = oracle.mat_from_voigt(c6, rho)
    for th in np.linspace(-np.pi, np.pi, 37):
        qsv, qp, sh = _modes(c6, rho, th)
        assert oracle.mode_velocity(m, 1, th) == pytest.approx(qsv, rel=1e-12)
        assert oracle.mode_velocity(m, 0, th) == pytest.approx(qp, rel=1e-12)
        assert oracle.mode_velocity(m, 2, th) == pytest.approx(sh, rel=1e-12)


@pytest.mark.parametrize("name", list(MATS))
def test_envelope_slowness(oracle, name):
    c6, rho = MATS[name]
    m = oracle.mat_from_voigt(c6, rho)
    a66, a55 = c6[5, 5] / rho, c6[4, 4] / rho
    for psi in np.radians([0.0, 7.0, 23.0, 41.0, 45.0, 66.0, 90.0, 118.0, 151.0, 179.0]):
        # qP: the envelope is the exact ray velocity (its slowness curve is convex)
        assert oracle.envelope_slowness(m, 0, psi) == pytest.approx(1.0 / oracle.group_exact(m, psi)[1], rel=1e-10)
        # SH: an elliptical phase curve has the elliptical ray surface x^2 / a66 + y^2 / a55 = t^2
        assert oracle.envelope_slowness(m, 2, psi) == pytest.approx(
            np.sqrt(np.cos(psi) ** 2 / a66 + np.sin(psi) ** 2 / a55), rel=1e-12)
        # qSV: brute force over the eigen-solver's qSV speeds
        bf = 1.0 / pins.hopf_lax_group_speed(lambda t: np.array([_modes(c6, rho, x)[0] for x in np.atleast_1d(t)]),
                                             psi, n=801)
        assert oracle.envelope_slowness(m, 1, psi) == pytest.approx(bf, rel=1e-9)


def test_qsv_envelope_is_the_wulff_shape(oracle):
    """The weld steel's qSV ray surface folds back (cusps: the ray angle psi(theta) = theta + atan(v'/v) runs
    backwards).  The envelope slowness is then the boundary of the Wulff shape, the set of points x with
    n.x <= v(n) for every unit normal n (the region a front moving with normal speed v(n) covers in unit time,
    which is what the eikonal's viscosity solution and hence the fast marching field converge to): every
    point V_env(psi) (cos psi, sin psi) lies in every half-plane and touches one."""
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    th = np.linspace(0, np.pi, 2001)
    v = np.array([_modes(c6, rho, t)[0] for t in th])
    dv = np.gradient(v, th)
    psi = th + np.arctan2(dv, v)
    assert (np.diff(psi[5:-5]) < 0).any()  # a cusp
    nth = np.linspace(-np.pi, np.pi, 20001)
    vn = np.array([_modes(c6, rho, t)[0] for t in nth])
    for p in np.radians(np.arange(0.0, 180.0, 7.5)):
        x = np.array([np.cos(p), np.sin(p)]) / oracle.envelope_slowness(m, 1, p)
        slack = vn - (np.cos(nth) * x[0] + np.sin(nth) * x[1])
        assert slack.min() > -1e-6 * vn.max()   # inside every half-plane
        assert slack.min() < 1e-4 * vn.max()    # on the boundary of one


def test_envelope_table_interpolation(oracle):
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    tab = oracle.envelope_table(m, 1)
    assert len(tab) == oracle.ENV_N
    k = np.arange(0, oracle.ENV_N, 37)
    assert np.allclose(tab[k], [oracle.envelope_slowness(m, 1, np.radians(x / 8.0)) for x in k], rtol=1e-15, atol=0)
    assert tab[0] == pytest.approx(tab[-1], rel=1e-13)  # 180-degree symmetry


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("ang_deg,th_deg", [(80.0, 30.0), (60.0, -20.0), (100.0, 65.0)])
def test_shear_linear_field_reproduced_exactly(oracle, mode, ang_deg, th_deg):
    """A plane shear wave frozen on the first two rows is continued exactly: the local update takes the mode's
    phase speed at the wavefront normal (Sec. 4.2)."""
    n = 24
    c6, rho = ORTHO
    m = oracle.mat_from_voigt(c6, rho)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, np.radians(th_deg)), [m], group_model=1,
                       wave_mode=mode)
    a = np.radians(ang_deg)
    v = _modes(c6, rho, a - np.radians(th_deg))[0 if mode == 1 else 2]
    jj, ii = np.mgrid[0:n, 0:n]
    exact = (ii * np.cos(a) + jj * np.sin(a)) * M.h / v
    exact -= exact.min()
    frozen = (jj < 2).astype(np.uint8).ravel()
    tau, rec, st = oracle.fmm(M, frozen, np.where(frozen, exact.ravel(), np.inf))
    ok = (rec < 32) & (rec >= 0)
    assert ok.sum() > 0.8 * (n - 2) * n
    err = np.abs(tau - exact)[ok] / exact.max()
    assert err.max() < 1e-12


@pytest.mark.parametrize("mode,name,th_deg,mean_gate,max_gate", [
    (2, "ortho", 30.0, 0.025, 0.06),    # SH: an elliptical (convex) slowness curve
    (2, "ortho", 0.0, 0.025, 0.06),
    (1, "ortho", 30.0, 0.015, 0.08),    # qSV of the orthotropic material
    (1, "weld_ti", 30.0, 0.010, 0.10),  # qSV of the weld steel, cusps off the grid axes
])
def test_shear_point_source_against_envelope(oracle, mode, name, th_deg, mean_gate, max_gate):
    """Homogeneous medium, 64 x 64, source (20, 32), straight-ray start of radius 4: the field approaches
    |x| / V_envelope (the eikonal's solution) within the method's discretisation error.  (With the weld
    steel's qSV cusps along the grid axes, orientation 0, the stencils miss the rays that leave the cusps and
    the mean error is about 10 %: the ALI update assumes the ray lies inside the stencil, which fails where
    the qSV ray and wavefront normal part by tens of degrees.)"""
    c6, rho = MATS[name]
    m = oracle.mat_from_voigt(c6, rho)
    n, th = 64, np.radians(th_deg)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m], group_model=1, wave_mode=mode)
    fr, t0 = oracle.init_radius(M, 20, 32, 4)
    tau, rec, st = oracle.fmm(M, fr, t0)
    assert st["noncausal"] == 0 and st["unreached"] == 0
    jj, ii = np.mgrid[0:n, 0:n]
    d = np.hypot(ii - 20, jj - 32) * 1e-3
    ang = np.arctan2(jj - 32, ii - 20) - th
    T = d * np.array([oracle.envelope_slowness(m, mode, a) for a in ang.ravel()]).reshape(n, n)
    msk = d > 4e-3
    rel = np.abs(tau - T)[msk] / T[msk]
    print(f"mode {mode} {name} {th_deg}: mean {rel.mean():.4f} max {rel.max():.4f}")
    assert rel.mean() < mean_gate
    assert rel.max() < max_gate


def test_shear_straight_ray_start(oracle):
    """The frozen times around a qSV source are distance x the tabulated envelope slowness of the source's
    orientation, which is the brute-force envelope to the table's interpolation error (< 1e-6)."""
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    n = 20
    theta = np.random.default_rng(3).uniform(-1.5, 1.5, n * n)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), theta, [m], group_model=1, wave_mode=1)
    si, sj, r0 = 9, 11, 3
    fr, tau = oracle.init_radius(M, si, sj, r0)
    th_s = theta[sj * n + si]
    for j in range(sj - r0, sj + r0 + 1):
        for i in range(si - r0, si + r0 + 1):
            if (i, j) == (si, sj):
                continue
            psi = np.arctan2(j - sj, i - si) - th_s
            bf = 1.0 / pins.hopf_lax_group_speed(
                lambda t: np.array([_modes(c6, rho, x)[0] for x in np.atleast_1d(t)]), psi, n=801)
            assert tau[j * n + i] == pytest.approx(np.hypot(i - si, j - sj) * 1e-3 * bf, rel=1e-6)
