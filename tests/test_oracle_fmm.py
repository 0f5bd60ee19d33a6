"""Pins of the oracle's ALI-FMM driver and whole-field results (Secs. 2, 4)."""
import os

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _medium(oracle, wl, k=0, group_model=0):
    s = wl.samples[k]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    return oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, s.region_theta, wl.region_material, mats,
                                       group_model)


def test_heap_equals_fixed_point_and_jacobi_tiny(oracle):
    """The heap FMM result is the unique fixed point of the local operator F: Jacobi iteration of F
    from +inf reproduces it bit for bit, records included, on random heterogeneous grids."""
    mats = [oracle.mat_from_voigt(*W.WELD_TI), oracle.mat_from_voigt(*W.PARENT_ISO),
            oracle.mat_from_voigt(*W.PAPER_CUBIC)]
    rng = np.random.default_rng(11)
    for trial in range(80):
        nx, ny = int(rng.integers(2, 10)), int(rng.integers(2, 10))
        mid = rng.integers(0, 3, nx * ny)
        th = rng.uniform(-np.pi / 2, np.pi / 2, nx * ny)
        M = oracle.OMedium(nx, ny, 1e-3, mid, th, mats, int(rng.integers(0, 2)))
        si, sj = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        frozen, t0 = oracle.init_radius(M, si, sj, int(rng.integers(0, 3)))
        tau, rec, st = oracle.fmm(M, frozen, t0)
        assert st["unreached"] == 0 and st["noncausal"] == 0
        tj, rj, it = oracle.jacobi(M, frozen, t0)
        assert it > 0
        assert np.array_equal(tau, tj) and np.array_equal(rec, rj)
        F, rF = oracle.F_all(M, frozen, tau)
        assert np.array_equal(F, tau) and np.array_equal(rF, rec)
        # the check's evaluation (known set fixed by each node's own key) is the identity there too
        Fc, rc = oracle.F_check(M, frozen, tau)
        assert np.array_equal(Fc, tau) and np.array_equal(rc, rec)


def test_heap_is_causal_on_weld(oracle):
    wl = W.weld_single(n=96, h=0.5e-3, rg=6, seed=7, nsrc=1, nrec=1)
    M = _medium(oracle, wl)
    s = wl.samples[0]
    for init in ("radius", "hierarchy"):
        fr, t0 = (oracle.init_radius(M, *s.src[0], 2) if init == "radius" else oracle.init_hierarchy(M, *s.src[0]))
        tau, rec, st, order = oracle.fmm(M, fr, t0, with_order=True)
        assert st["noncausal"] == 0 and st["unreached"] == 0
        # acceptance order is key order
        keys = [(tau.flat[n], n) for n in np.argsort(order.ravel()) if order.flat[n] >= 0]
        assert all(keys[a] < keys[a + 1] for a in range(len(keys) - 1))
        F, _ = oracle.F_all(M, fr, tau)
        assert np.array_equal(F, tau)
        Fc, rc = oracle.F_check(M, fr, tau)
        assert np.array_equal(Fc, tau) and np.array_equal(rc, rec)


@pytest.mark.parametrize("ang_deg,th_deg", [(80.0, 30.0), (60.0, -20.0), (100.0, 65.0), (90.0, 0.0)])
def test_linear_field_reproduced_exactly(oracle, ang_deg, th_deg):
    """A plane wave frozen on the first two rows of a homogeneous TI grid is continued exactly: every
    stencil the driver can use is exact on a linear field (Sec. 4.2)."""
    n = 24
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, np.radians(th_deg)), [m])
    a = np.radians(ang_deg)
    slow = M.h / oracle.phase_velocity(m, a - np.radians(th_deg))
    jj, ii = np.mgrid[0:n, 0:n]
    exact = (ii * np.cos(a) + jj * np.sin(a)) * slow
    exact -= exact.min()
    frozen = (jj < 2).astype(np.uint8).ravel()
    tau, rec, st = oracle.fmm(M, frozen, np.where(frozen, exact.ravel(), np.inf))
    ok = (rec < 32) & (rec >= 0)
    assert ok.sum() > 0.9 * (n - 2) * n
    err = np.abs(tau - exact)[ok] / exact.max()
    assert err.max() < 1e-12


def test_point_source_against_closed_form(oracle):
    """Homogeneous TI, 64 x 64, orientation 30 deg, source (0, 32): the field approaches the exact
    straight-ray time |x| / V_exact(direction) (Hopf-Lax) within the method's discretisation error."""
    wl = W.homogeneous_ti()
    for group_model in (0, 1):
        M = _medium(oracle, wl, group_model=group_model)
        fr, t0 = oracle.init_hierarchy(M, 0, 32)
        tau, rec, st = oracle.fmm(M, fr, t0)
        assert st["noncausal"] == 0
        jj, ii = np.mgrid[0:64, 0:64]
        d = np.hypot(ii, jj - 32) * 1e-3
        ang = np.arctan2(jj - 32, ii)
        m = M.mats[0]
        V = np.array([oracle.group_exact(m, a - np.radians(30.0))[1] for a in ang.ravel()]).reshape(64, 64)
        T = d / np.where(d > 0, V, 1.0)
        msk = d > 0
        rel = np.abs(tau - T)[msk] / T[msk]
        assert rel.mean() < 0.015
        assert rel.max() < 0.08


def test_isotropic_point_source(oracle):
    n = 48
    c6, rho = W.PARENT_ISO
    m = oracle.mat_from_voigt(c6, rho)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.zeros(n * n), [m])
    fr, t0 = oracle.init_hierarchy(M, 20, 3)
    tau, rec, st = oracle.fmm(M, fr, t0)
    jj, ii = np.mgrid[0:n, 0:n]
    T = np.hypot(ii - 20, jj - 3) * 1e-3 / np.sqrt(273e9 / 7850)
    rel = np.abs(tau - T)[T > 0] / T[T > 0]
    assert rel.mean() < 0.015 and rel.max() < 0.03


def _table2_error(oracle, s):
    c6, rho = W.PAPER_CUBIC
    m = oracle.mat_from_voigt(c6, rho)
    n = 20 * s + 1
    M = oracle.OMedium(n, n, 1e-3 / s, np.zeros(n * n), np.zeros(n * n), [m])
    dens, rad = ((27, 9, 3), (1, 6, 13)) if s == 1 else ((9, 3), (2 * s, 5 * s))
    fr, t0 = oracle.init_hierarchy(M, 10 * s, 10 * s, dens, rad)
    tau, rec, st = oracle.fmm(M, fr, t0)
    sub = tau[::s, ::s]
    jj, ii = np.mgrid[0:21, 0:21]
    d = np.hypot(ii - 10, jj - 10) * 1e-3
    V = np.array([oracle.group_exact(m, a)[1] for a in np.arctan2(jj - 10, ii - 10).ravel()]).reshape(21, 21)
    T = d / np.where(d > 0, V, 1.0)
    return 100.0 * (np.abs(sub - T)[d > 0] / T[d > 0]).mean()


def test_table2_subgrid_band(oracle):
    """Sec. 4.5, Table 2: mean abs relative error on the 21 x 21 cubic-steel grid for subgrid sizes
    1, 3, 5, 7.  The figure-only details of the paper's runs are unknown, so this is a band (+-10 %)."""
    ref = {int(a): float(b) for a, b in (l.split() for l in open(os.path.join(GOLDEN, "table2_subgrid_errors.txt"))
                                         if l.strip() and not l.startswith("#"))}
    for s in (1, 3, 5, 7):
        e = _table2_error(oracle, s)
        assert abs(e / ref[s] - 1.0) < 0.10, (s, e, ref[s])


def test_mirror_symmetry(oracle):
    """Mirroring the grid about the source row with orientations negated mirrors the field."""
    wl = W.weld_single(n=40, h=0.5e-3, rg=4, seed=3, nsrc=1, nrec=1)
    s = wl.samples[0]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    mid = wl.region_material[s.region_map.astype(int)]
    th = s.region_theta[s.region_map.astype(int)]
    M1 = oracle.OMedium(40, 40, s.h, mid, th, mats)
    M2 = oracle.OMedium(40, 40, s.h, mid[::-1], -th[::-1], mats)
    f1, t1 = oracle.init_radius(M1, 12, 20, 2)
    f2, t2 = oracle.init_radius(M2, 12, 19, 2)
    a = oracle.fmm(M1, f1, t1)[0]
    b = oracle.fmm(M2, f2, t2)[0]
    # rows j and 39 - j are mirror images about y = 19.5; compare where the mirrored source rows agree
    M3 = oracle.OMedium(40, 39, s.h, mid[:39], th[:39], mats)
    M4 = oracle.OMedium(40, 39, s.h, mid[:39][::-1], -th[:39][::-1], mats)
    f3, t3 = oracle.init_radius(M3, 12, 19, 2)
    f4, t4 = oracle.init_radius(M4, 12, 19, 2)
    c = oracle.fmm(M3, f3, t3)[0]
    d = oracle.fmm(M4, f4, t4)[0]
    assert np.allclose(c, d[::-1], rtol=1e-9, atol=0)
    assert a.shape == b.shape


def test_reciprocity(oracle):
    """tau_s(r) is close to tau_r(s) (the discretisation breaks exact symmetry, Sec. 5.1)."""
    wl = W.weld_single(n=64, h=0.5e-3, rg=4, seed=9, nsrc=4, nrec=4)
    M = _medium(oracle, wl)
    pts = [(5, 0), (40, 0), (20, 63), (60, 63)]
    fields = {}
    for p in pts:
        fr, t0 = oracle.init_hierarchy(M, *p)
        fields[p] = oracle.fmm(M, fr, t0)[0]
    for a in pts:
        for b in pts:
            if a < b:
                ta, tb = fields[a][b[1], b[0]], fields[b][a[1], a[0]]
                assert abs(ta - tb) / ta < 0.02


def test_table2_velocity_table_band(oracle):
    """Sec. 4.5, Table 2, row "ALI-FMM" (phase speeds from a table at integer degrees, linearly
    interpolated): mean abs relative error for sub-grid sizes 1, 3, 5, 7 within +-10 % of the printed
    values.  (The paper finds the table slightly less accurate than the run-time solve; here the two differ
    by less than 1 %, in either direction.)"""
    ref = {1: 1.083, 3: 1.073, 5: 0.715, 7: 0.565}  # Table 2, velocity-table row
    c6, rho = W.PAPER_CUBIC
    m = oracle.mat_from_voigt(c6, rho)
    for s in (1, 3, 5, 7):
        n = 20 * s + 1
        M = oracle.OMedium(n, n, 1e-3 / s, np.zeros(n * n), np.zeros(n * n), [m], vtable=1)
        dens, rad = ((27, 9, 3), (1, 6, 13)) if s == 1 else ((9, 3), (2 * s, 5 * s))
        fr, t0 = oracle.init_hierarchy(M, 10 * s, 10 * s, dens, rad)
        tau = oracle.fmm(M, fr, t0)[0]
        sub = tau[::s, ::s]
        jj, ii = np.mgrid[0:21, 0:21]
        d = np.hypot(ii - 10, jj - 10) * 1e-3
        V = np.array([oracle.group_exact(m, a)[1] for a in np.arctan2(jj - 10, ii - 10).ravel()]).reshape(21, 21)
        T = d / np.where(d > 0, V, 1.0)
        e = 100.0 * (np.abs(sub - T)[d > 0] / T[d > 0]).mean()
        assert abs(e / ref[s] - 1.0) < 0.10, (s, e, ref[s])


def test_velocity_table_exact_at_integer_degrees(oracle):
    """At integer degrees the table holds the Christoffel speed itself: a plane wave whose normal is at
    0, 45 or 90 degrees from the axis of a homogeneous medium gets the same update with and without it."""
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    n = 9
    for th_deg in (0.0, 45.0, 90.0):
        th = np.radians(th_deg)
        M0 = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m])
        M1 = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m], vtable=1)
        jj, ii = np.mgrid[0:n, 0:n]
        tau = (ii * 1e-3 / 5000.0).astype(np.float64)  # plane wave along +x: normal at -th from the axis
        for row in (1, 3, 4, 6):  # rows whose A, B, C are not all on one wavefront of this plane wave
            a = oracle.stencil_value(M0, tau.reshape(-1), 4, 4, row)
            b = oracle.stencil_value(M1, tau.reshape(-1), 4, 4, row)
            assert a == pytest.approx(b, rel=1e-12), (th_deg, row)
    # between integer degrees the table interpolates: close to, but not equal to, the run-time solve
    th = np.radians(30.5)
    M0 = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m])
    M1 = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, th), [m], vtable=1)
    jj, ii = np.mgrid[0:n, 0:n]
    tau = (ii * 1e-3 / 5000.0).astype(np.float64)
    a = oracle.stencil_value(M0, tau.reshape(-1), 4, 4, 1)
    b = oracle.stencil_value(M1, tau.reshape(-1), 4, 4, 1)
    assert a != b and abs(b / a - 1) < 1e-4


def test_check_evaluation_with_exact_ties(oracle):
    """On a homogeneous isotropic grid with a central source, mirror-image nodes get bit-identical times, and
    many of them are diamond neighbours of one another: the key order (tau, index) decides which of two tied
    nodes is known to the other.  The check's evaluation with its known set fixed by each node's own key
    reproduces the field, records included, exactly at those ties."""
    n = 21
    m = oracle.mat_from_voigt(*W.PARENT_ISO)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n, np.int64), np.zeros(n * n), [m])
    fr, t0 = oracle.init_radius(M, n // 2, n // 2, 0)
    tau, rec, st = oracle.fmm(M, fr, t0)
    assert st["unreached"] == 0
    ties = 0
    for j in range(n):
        for i in range(n):
            for di, dj in ((1, 1), (1, -1), (2, 0), (0, 2), (1, 0), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n and tau[j, i] == tau[jj, ii]:
                    ties += 1
    assert ties > 20  # the field does exercise the tie order
    Fc, rc = oracle.F_check(M, fr, tau)
    assert np.array_equal(Fc, tau) and np.array_equal(rc, rec)
