"""Pins of the oracle's ray tracer and path-time integrator (Sec. 5)."""
import os

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    out = {}
    for l in open(os.path.join(GOLDEN, "velocity_gradient_ray.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            out[k] = float(v)
    return out


def _gradient_medium(oracle):
    wl = W.velocity_gradient()
    s = wl.samples[0]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    return oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, s.region_theta, wl.region_material, mats)


def _circle():
    """Circle through source and receiver for v = v0 + g x (Sec. 5.2, Eq. circle_vel_grad), with the
    relation between the launch angle and the receiver written without the print's dropped factor 2:
    g^2 y'^2 + (g x' + v0)^2 - v0^2 = 2 g y' v0 cot(theta0)."""
    g, v0 = 21.0, 3021.0
    xp, yp = 198.0, 150.0
    cot = ((g * yp) ** 2 + (g * xp + v0) ** 2 - v0 ** 2) / (2 * g * yp * v0)
    return 1.0 - v0 / g, 30.0 + v0 * cot / g, v0 * np.sqrt(1.0 + cot * cot) / g


def test_circle_matches_printed_geometry():
    G = _golden()
    cx, cy, R = _circle()
    assert cx == pytest.approx(G["circle_centre_x"], abs=1e-3)
    assert cy == pytest.approx(G["circle_centre_y"], abs=1e-3)
    assert R == pytest.approx(G["circle_radius"], abs=1e-3)


def test_path_time_of_true_arc(oracle):
    """Integrating the exact arc through the nearest-node cells gives the paper's time of the true
    path on the discretised grid; the continuum time (1/g) arccosh(1 + g^2 d^2 / (2 v_a v_b)) is
    close to it."""
    G = _golden()
    M = _gradient_medium(oracle)
    cx, cy, R = _circle()
    a0, a1 = np.arctan2(30 - cy, 1 - cx), np.arctan2(180 - cy, 199 - cx)
    aa = np.linspace(a0, a1, 20001)
    arc = np.stack([cx + R * np.cos(aa), cy + R * np.sin(aa)], 1)
    t = oracle.path_time(M, arc)
    assert t == pytest.approx(G["true_time_discretised"], rel=2e-6)
    g = 21.0
    cont = np.arccosh(1 + g * g * (198.0 ** 2 + 150.0 ** 2) / (2 * 3021.0 * 7179.0)) / g * 1e-3
    assert t == pytest.approx(cont, rel=1e-5)


def test_velocity_gradient_ray(oracle):
    """Sec. 5.2: the traced ray follows the circular arc (paper: within about 0.3 cells) and its
    integrated time is within a few 1e-5 of the true path's (paper: 7e-6)."""
    G = _golden()
    M = _gradient_medium(oracle)
    fr, t0 = oracle.init_hierarchy(M, 1, 30)
    tau, rec, st = oracle.fmm(M, fr, t0)
    pts, status = oracle.trace_ray(M, tau, (199, 180), (1, 30))
    assert status == 0
    assert tuple(pts[0]) == (199.0, 180.0) and tuple(pts[-1]) == (1.0, 30.0)
    cx, cy, R = _circle()
    dev = np.abs(np.hypot(pts[:, 0] - cx, pts[:, 1] - cy) - R)
    assert dev.max() < 0.5
    t = oracle.path_time(M, pts)
    assert t >= G["true_time_discretised"] * (1 - 1e-6)
    assert t == pytest.approx(G["ray_time"], rel=1e-4)


def test_homogeneous_ray_is_straight(oracle):
    """Sec. 5.3: in a homogeneous medium the fastest path is the straight segment."""
    n = 80
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    for th in (0.0, 0.6, -1.1):
        M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m])
        fr, t0 = oracle.init_hierarchy(M, 10, 0)
        tau = oracle.fmm(M, fr, t0)[0]
        for rec in ((70, 79), (10, 79), (79, 40)):
            pts, st = oracle.trace_ray(M, tau, rec, (10, 0))
            assert st == 0
            a = np.array([10.0, 0.0])
            b = np.array(rec, float)
            u = (b - a) / np.linalg.norm(b - a)
            off = np.abs((pts - a) @ np.array([-u[1], u[0]]))
            assert off.max() < 1.5  # the field's angle-dependent error bends the ray by about a cell
            straight = np.linalg.norm(b - a) * 1e-3 / oracle.group_exact(m, np.arctan2(*(b - a)[::-1]) - th)[1]
            t = oracle.path_time(M, pts)
            assert straight * (1 - 0.006) <= t <= straight * 1.01


def _homogeneous(oracle, th=0.6, n=80):
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m])
    fr, t0 = oracle.init_hierarchy(M, 10, 0)
    return M, oracle.fmm(M, fr, t0)[0], m


def test_fixed_family_points_lie_on_its_planes(oracle):
    """Sec. 5.1: with one fixed set of planes every interior ray point lies on a plane of that set
    (x = c, y = c, x - y = c, x + y = c with integer c), and successive points cross successive planes."""
    M, tau, m = _homogeneous(oracle)
    for fam, coord in ((0, lambda p: p[:, 0]), (1, lambda p: p[:, 1]), (2, lambda p: p[:, 0] - p[:, 1]),
                       (3, lambda p: p[:, 0] + p[:, 1])):
        pts, st = oracle.trace_ray(M, tau, (70, 79), (10, 0), family=fam)
        assert st == 0
        q = coord(pts[1:-1])
        assert np.allclose(q, np.round(q), atol=1e-9), fam
        steps = np.diff(coord(pts[:-1]))
        assert np.all(steps != 0) and (np.all(steps > 0) or np.all(steps < 0)), fam


def test_fixed_family_without_planes_between_gives_two_points(oracle):
    """Sec. 5.3: when source and receiver share the x coordinate no vertical plane lies between them, and
    the ray of the vertical planes is just the receiver and the source."""
    M, tau, m = _homogeneous(oracle)
    pts, st = oracle.trace_ray(M, tau, (10, 79), (10, 0), family=0)
    assert st == 0
    assert pts.shape == (2, 2) and tuple(pts[0]) == (10.0, 79.0) and tuple(pts[1]) == (10.0, 0.0)


def test_fixed_families_in_a_homogeneous_medium(oracle):
    """Sec. 5.3: in a homogeneous medium each set of planes that separates the ends gives a near-straight
    ray, and the best of the four is no slower than any of them."""
    M, tau, m = _homogeneous(oracle)
    a, b = np.array([10.0, 0.0]), np.array([70.0, 79.0])
    u = (b - a) / np.linalg.norm(b - a)
    times = []
    for fam in range(4):
        pts, st = oracle.trace_ray(M, tau, tuple(b), tuple(a), family=fam)
        assert st == 0
        off = np.abs((pts - a) @ np.array([-u[1], u[0]]))
        assert off.max() < 3.0, (fam, off.max())  # within one plane spacing (4 cells) of the segment
        times.append(oracle.path_time(M, pts))
    straight = np.linalg.norm(b - a) * 1e-3 / oracle.group_exact(m, np.arctan2(*(b - a)[::-1]) - 0.6)[1]
    assert min(times) >= straight * (1 - 0.006) and max(times) <= straight * 1.02
    pts, st, fam = oracle.trace_ray_best_family(M, tau, tuple(b), tuple(a))
    assert st == 0 and oracle.path_time(M, pts) == min(times) and fam == int(np.argmin(times))


def test_ray_gradient_closed_form(oracle):
    """Along a fixed straight path in a homogeneous medium the time is L h / V(phi - theta), so its
    derivative by the orientation is that closed form's, from the (pinned) exact ray velocity."""
    n = 60
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    th = 0.4
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m], group_model=oracle.GROUP_EXACT)
    a, b = np.array([5.0, 3.0]), np.array([52.0, 40.0])
    pts = np.stack([b, 0.5 * (a + b), a])
    L = np.linalg.norm(b - a) * 1e-3
    phi = np.arctan2(*(a - b)[::-1])
    e = 1e-5
    closed = (L / oracle.group_exact(m, phi - th - e)[1] - L / oracle.group_exact(m, phi - th + e)[1]) / (2 * e)
    g = oracle.ray_gradient(M, pts, np.zeros(n * n, np.int64), 1)
    assert g[0] == pytest.approx(closed, rel=1e-6)
    assert oracle.path_time(M, pts) == pytest.approx(L / oracle.group_exact(m, phi - th)[1], rel=1e-12)


def test_ray_gradient_sums_regions(oracle):
    """Moving every region by the same angle moves the whole medium: the region derivatives of a path
    through several regions add up to the derivative for one orientation shared by all of them."""
    wl = W.weld_single(n=40, h=0.5e-3, rg=4, seed=5, nsrc=1, nrec=1)
    s = wl.samples[0]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, s.region_theta, wl.region_material, mats)
    pts = np.array([[3.0, 39.0], [15.0, 25.0], [22.0, 12.0], [30.0, 0.0]])
    g = oracle.ray_gradient(M, pts, s.region_map.reshape(-1), wl.nregions)
    e = 1e-6
    Mp = oracle.OMedium(M.nx, M.ny, M.h, M.mat_id, M.theta + e, M.mats, M.group_model)
    Mm = oracle.OMedium(M.nx, M.ny, M.h, M.mat_id, M.theta - e, M.mats, M.group_model)
    total = (oracle.path_time(Mp, pts) - oracle.path_time(Mm, pts)) / (2 * e)
    assert np.sum(g) == pytest.approx(total, rel=1e-5)
    assert np.count_nonzero(g) >= 3
